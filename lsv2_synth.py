"""Seeded synthetic inputs for the sparse-coefficient splatting path.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic (no projection, blending, decoding or relevancy).  Both the
FP64 oracle (``oracle/``) and the CUDA path read the identical float32 arrays
it produces, so any disagreement between the two comes from the method, never
from the inputs.

The paper evaluates on captured scenes (LERF, 3D-OVS, Mip-NeRF360) with trained
Gaussians, CLIP features and a learned codebook, none of which are available
here.  The generators below stand in for them with the same shapes: N Gaussians
with mean, scale, rotation and opacity (Sec. 3.1, Eq. 1-2), K=4 (index, weight)
pairs per Gaussian and semantic level over an L=64 codebook of D=512-d unit
features (Sec. 3.3, Eq. 5; Sec. 4.1 sets L=64, K=4, three levels), and unit
512-d text embeddings for the relevancy query (Sec. 3.2).

The decoder-based comparison path (LangSplat*, Sec. 3.1) needs per-Gaussian latent features
(d = 3 per level, Eq. 4) and the weights of a decoder MLP; the trained ones are not available,
so both are drawn at random with the right shapes (``latent_features``, ``decoder_mlp``).

Seeds: 20250707 scene, +1 codebook, +2 text, +3 L1 target, +4 batched scene, +5 relevancy maps,
+6 latent features, +7 decoder weights.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED = 20250707
L_CODEBOOK = 64
K_PAIRS = 4
D_FEAT = 512
LATENT_D = 3
# decoder widths, latent in -> CLIP feature out: the paper fixes only the ends (3 and 512); the
# hidden widths are a widening stack of the kind a scene autoencoder's decoder uses
DECODER_WIDTHS = (LATENT_D, 16, 32, 64, 128, 256, 256, D_FEAT)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Camera:
    """Pinhole camera, world -> camera ``t = R @ m + t0`` (x right, y down, z forward).

    Pixel (i, j) is sampled at image-plane point (i, j); the principal point is
    the image centre ``((W-1)/2, (H-1)/2)``.
    """

    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray  # float32 [3, 3]
    t: np.ndarray  # float32 [3]
    tile_w: int = 16
    tile_h: int = 16
    near: float = 0.2

    @property
    def grid(self) -> tuple[int, int]:
        return ((self.width + self.tile_w - 1) // self.tile_w,
                (self.height + self.tile_h - 1) // self.tile_h)

    @property
    def num_tiles(self) -> int:
        gx, gy = self.grid
        return gx * gy

    @property
    def num_pixels(self) -> int:
        return self.width * self.height

    def with_tile(self, tw: int, th: int) -> "Camera":
        return Camera(self.width, self.height, self.fx, self.fy, self.cx, self.cy,
                      self.R.copy(), self.t.copy(), tw, th, self.near)


def orbit_camera(width: int, height: int, radius: float, azimuth_deg: float = 0.0,
                 hfov_deg: float = 60.0, tile: tuple[int, int] = (16, 16)) -> Camera:
    """Camera on a circle of ``radius`` in the x-z plane, looking at the origin.

    Azimuth 0 puts the centre at (0, 0, -radius) with the identity rotation.
    Focal length from the horizontal field of view; square pixels (fy = fx).
    """
    th = math.radians(azimuth_deg)
    centre = np.array([radius * math.sin(th), 0.0, -radius * math.cos(th)])
    fwd = -centre / np.linalg.norm(centre)
    right = np.array([math.cos(th), 0.0, math.sin(th)])
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd]).astype(np.float64)
    t = -R @ centre
    fx = (width / 2.0) / math.tan(math.radians(hfov_deg) / 2.0)
    return Camera(width, height, float(np.float32(fx)), float(np.float32(fx)),
                  (width - 1) / 2.0, (height - 1) / 2.0,
                  R.astype(np.float32), t.astype(np.float32), tile[0], tile[1])


@dataclass
class Scene:
    means: np.ndarray      # f32 [N, 3]
    scales: np.ndarray     # f32 [N, 3]   activated (exp of log-scale)
    quats: np.ndarray      # f32 [N, 4]   (w, x, y, z), unit up to float32 rounding
    opacity: np.ndarray    # f32 [N]      activated (sigmoid of logit)
    idx: np.ndarray        # u8  [N, levels, K]
    weights: np.ndarray    # f32 [N, levels, K]
    codebook: np.ndarray   # f32 [levels, L, D]
    log_scales: np.ndarray = field(default=None)   # f32 [N, 3]
    opacity_logits: np.ndarray = field(default=None)  # f32 [N]

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def levels(self) -> int:
        return int(self.idx.shape[1])

    @property
    def K(self) -> int:
        return int(self.idx.shape[2])

    @property
    def L(self) -> int:
        return int(self.codebook.shape[1])

    @property
    def D(self) -> int:
        return int(self.codebook.shape[2])

    def subset(self, n: int) -> "Scene":
        return Scene(self.means[:n].copy(), self.scales[:n].copy(), self.quats[:n].copy(),
                     self.opacity[:n].copy(), self.idx[:n].copy(), self.weights[:n].copy(),
                     self.codebook.copy(),
                     None if self.log_scales is None else self.log_scales[:n].copy(),
                     None if self.opacity_logits is None else self.opacity_logits[:n].copy())


def unit_rows(x: np.ndarray) -> np.ndarray:
    return x / np.linalg.norm(x, axis=-1, keepdims=True)


def sparse_coefficients(rng: np.random.Generator, n: int, levels: int, K: int, L: int):
    """K distinct indices per (Gaussian, level), uniform over L; weights softmax(N(0,1)^K)."""
    keys = rng.random((n, levels, L))
    idx = np.argsort(keys, axis=-1)[..., :K].astype(np.uint8)
    logits = rng.standard_normal((n, levels, K))
    e = np.exp(logits - logits.max(-1, keepdims=True))
    w = (e / e.sum(-1, keepdims=True)).astype(np.float32)
    return idx, w


def codebooks(seed: int, levels: int, L: int = L_CODEBOOK, D: int = D_FEAT) -> np.ndarray:
    rng = _rng(seed)
    return unit_rows(rng.standard_normal((levels, L, D))).astype(np.float32)


def gaussians(rng: np.random.Generator, n: int, mean_kind: str, mean_param: float,
              log_scale_mu: float, log_scale_sigma: float, levels: int,
              K: int = K_PAIRS, L: int = L_CODEBOOK):
    if mean_kind == "uniform":
        means = rng.uniform(-mean_param, mean_param, (n, 3))
    else:
        means = rng.normal(0.0, mean_param, (n, 3))
    log_s = rng.normal(log_scale_mu, log_scale_sigma, (n, 3)).astype(np.float32)
    q = unit_rows(rng.standard_normal((n, 4))).astype(np.float32)
    logit = rng.normal(0.0, 1.5, n).astype(np.float32)
    idx, w = sparse_coefficients(rng, n, levels, K, L)
    scales = np.exp(log_s.astype(np.float64)).astype(np.float32)
    opac = (1.0 / (1.0 + np.exp(-logit.astype(np.float64)))).astype(np.float32)
    return means.astype(np.float32), scales, q, opac, idx, w, log_s, logit


def make_scene(n: int, levels: int, seed: int = SEED, mean_kind: str = "normal",
               mean_param: float = 2.0, log_scale_mu: float = -4.5,
               log_scale_sigma: float = 0.5, K: int = K_PAIRS, L: int = L_CODEBOOK,
               D: int = D_FEAT) -> Scene:
    rng = _rng(seed)
    m, s, q, o, idx, w, log_s, logit = gaussians(rng, n, mean_kind, mean_param, log_scale_mu,
                                                 log_scale_sigma, levels, K, L)
    cb = codebooks(seed + 1, levels, L, D)
    return Scene(m, s, q, o, idx, w, cb, log_s, logit)


def text_queries(seed: int, Q: int, n_neg: int, D: int = D_FEAT) -> np.ndarray:
    """Q queries, each one positive then ``n_neg`` negatives: f32 [Q, 1+n_neg, D], unit rows."""
    rng = _rng(seed)
    return unit_rows(rng.standard_normal((Q, 1 + n_neg, D))).astype(np.float32)


# --------------------------------------------------------------------------------------
# Named workloads (sizes follow the paper's setting: L=64, K=4, D=512, three levels).

def tiny():
    """2,000 Gaussians, means U[-1,1]^3, log-scales N(-3,0.3), 128x96, one level."""
    sc = make_scene(2000, 1, mean_kind="uniform", mean_param=1.0, log_scale_mu=-3.0,
                    log_scale_sigma=0.3)
    cam = orbit_camera(128, 96, 4.0)
    return sc, cam


def at_scale():
    """300,000 Gaussians, means N(0, 2^2), log-scales N(-4.5, 0.5), three levels, 1440x1080."""
    sc = make_scene(300_000, 3)
    cam = orbit_camera(1440, 1080, 6.0)
    text = text_queries(SEED + 2, 1, 4)
    return sc, cam, text


def differentiation():
    """100,000 Gaussians, 720x540, one level, L1 target N(0, 0.05^2) of shape [P, 512]."""
    sc = make_scene(100_000, 1)
    cam = orbit_camera(720, 540, 6.0)
    return sc, cam


def l1_target(cam: Camera, levels: int = 1, D: int = D_FEAT, seed: int = SEED + 3) -> np.ndarray:
    rng = _rng(seed)
    return rng.normal(0.0, 0.05, (levels, cam.num_pixels, D)).astype(np.float32)


def fd_subset():
    """First 200 Gaussians of the differentiation scene, rendered at 64x48."""
    sc, _ = differentiation()
    return sc.subset(200), orbit_camera(64, 48, 6.0)


def precision():
    """The tiny scene rendered at 1440x1080, one level."""
    sc, _ = tiny()
    return sc, orbit_camera(1440, 1080, 4.0)


BATCH_RESOLUTIONS = [(1440, 1080)] * 4 + [(960, 720)] * 4 + [(640, 480)] * 4 + [(320, 240)] * 4


def batched(tile=(16, 16)):
    """500,000 Gaussians, three levels, 16 views of uneven resolution on a radius-6 orbit,
    64 queries with four negatives each."""
    sc = make_scene(500_000, 3, seed=SEED + 4)
    cams = [orbit_camera(w, h, 6.0, azimuth_deg=22.5 * k, tile=tile)
            for k, (w, h) in enumerate(BATCH_RESOLUTIONS)]
    text = text_queries(SEED + 2, 64, 4)
    return sc, cams, text


def relevancy_maps(seed: int, Q: int, levels: int, H: int, W: int, blobs: int = 6) -> np.ndarray:
    """Relevancy-like maps for the post-processing stage, float32 [Q, levels, H*W] in (0, 1): a
    few random Gaussian bumps of random height and width over a low noisy background per map
    (relevancy maps of a text query are mostly low with a few high regions).  Seed: +5."""
    rng = _rng(seed)
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    out = np.empty((Q, levels, H * W), np.float32)
    for q in range(Q):
        for l in range(levels):
            m = 0.15 + 0.05 * rng.random((H, W))
            for _ in range(blobs):
                cx, cy = rng.uniform(0, W), rng.uniform(0, H)
                s = rng.uniform(1.5, 0.25 * max(H, W) + 2.0)
                h = rng.uniform(0.1, 0.8)
                m += h * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * s * s))
            out[q, l] = (m / (1.0 + m)).reshape(-1)
    return out


def latent_features(n: int, levels: int, d: int = LATENT_D, seed: int = SEED + 6) -> np.ndarray:
    """Per-Gaussian latent features f_i of the decoder-based path (Eq. 4): f32 [n, levels, d],
    N(0, 1) entries (an autoencoder's latent codes, of unit scale)."""
    return _rng(seed).standard_normal((n, levels, d)).astype(np.float32)


def bf16_representable(x: np.ndarray) -> np.ndarray:
    """float32 values rounded (to nearest, ties to even) onto the BF16 grid: weights stored in
    BF16, held as float32 so every consumer reads the same numbers."""
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def decoder_mlp(widths=DECODER_WIDTHS, seed: int = SEED + 7):
    """Random weights of the decoder MLP: a list of (W [w_in, w_out], b [w_out]) float32 pairs.
    W ~ N(0, 2 / w_in) before a ReLU and N(0, 1 / w_in) for the last layer (so activations keep
    their scale through the stack), and b ~ N(0, 0.05^2), both stored on the BF16 grid."""
    rng = _rng(seed)
    layers = []
    for l in range(len(widths) - 1):
        gain = 1.0 if l == len(widths) - 2 else 2.0
        W = rng.normal(0.0, math.sqrt(gain / widths[l]), (widths[l], widths[l + 1]))
        b = rng.normal(0.0, 0.05, widths[l + 1])
        layers.append((bf16_representable(W.astype(np.float32)), bf16_representable(b.astype(np.float32))))
    return layers


def latent_at_scale():
    """The at-scale frame's Gaussians (300,000, three levels, 1440x1080) carrying latent features
    instead of sparse coefficients, and the decoder's weights."""
    sc, cam, text = at_scale()
    return sc, cam, latent_features(sc.n, sc.levels), decoder_mlp()
