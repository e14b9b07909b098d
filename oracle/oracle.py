"""Python face of the FP64 CPU oracle (``lsv2_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the package smoke check and by
the benchmark's CPU-baseline leg, never by the product path.  It shares no code
with the CUDA library; both read the same float32 inputs from ``lsv2_synth``.

Each function names the passage of the paper it follows (LangSplatV2, arXiv
2507.07136):
  project       Sec. 3.1 Eq. 1-2 + EWA projection; FP32 decision path for the
                integer outputs (radius, tile rectangle, depth key)
  bin           "ordered Gaussian points within a tile" (Eq. 3)
  blend         Eq. 3 / Eq. 7 weights, Algorithm 1 sparse accumulation
  decode        Eq. 7, F = W S
  relevancy     Sec. 3.2 relevancy score (cosine + pairwise softmax, min over negatives)
  mean_filter,  appendix "Evaluation Details": average pooling of the relevancy map,
  postprocess   level selection, localisation point, normalise + threshold mask
  l1_grads      gradient of the L1 feature loss (decode adjoint as matmuls,
                l1_decode_adjoint for a given coefficient map,
                blend adjoint as the literal derivative, projection Jacobian by
                complex step)
  sparsify,     Sec. 3.3 sparse coefficients: softmax over the L-dim parameter, top K
  sparsify_backward   kept and renormalised by their sum; its gradient (NumPy, FP64)
  mlp_decode    Sec. 3.1: the decoder g_d of the decoder-based path (LangSplat*) applied to a
                rendered latent feature (Eq. 4 is ``blend`` mode 2 with d-dim features)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lsv2_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liblsv2_oracle.so")

ALPHA_MIN = float(np.float32(1.0) / np.float32(255.0))
T_MIN = float(np.float32(1e-4))


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-shared", "-fPIC", "-o", _LIB, _SRC, "-lm"])
    return _LIB


class _Cam(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("tile_w", C.c_int32),
                ("tile_h", C.c_int32), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float), ("near_z", C.c_float), ("R", C.c_float * 9), ("t", C.c_float * 3)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        I64, I32, D = C.c_int64, C.c_int32, C.c_double
        _lib.orc_project.argtypes = [P, I64, P, P, P, P, P, P, P, P, P, P]
        _lib.orc_project_jacobian.argtypes = [P, I64, P, P, P, P]
        _lib.orc_project64.argtypes = [P, I64, P, P, P, P, P]
        _lib.orc_count_instances.argtypes = [P, I64, P, P]
        _lib.orc_count_instances.restype = I64
        _lib.orc_bin.argtypes = [P, I64, P, P, P, P, P]
        _lib.orc_bin.restype = I64
        _lib.orc_blend.argtypes = [P, I64, P, P, P, P, P, P, P, I32, I32, I32, I32, P, P, P, P, P,
                                   P, P, P, P]
        _lib.orc_decode.argtypes = [I32, I64, I32, I32, P, P, P]
        _lib.orc_relevancy.argtypes = [I32, I64, I32, P, I32, I32, P, D, P]
        _lib.orc_blend_backward.argtypes = [P, I64, P, P, P, P, P, I32, I32, I32, P, P, P, P, P, P,
                                            P]
        _lib.orc_l1_loss_tiles.argtypes = [P, I64, P, P, P, P, P, P, P, I32, I32, I32, I32, P, P,
                                           P, P, P, P]
        _lib.orc_l1_loss_tiles.restype = D
        _lib.orc_mean_filter.argtypes = [I32, I32, I32, P, P]
        _lib.orc_postprocess.argtypes = [I32, I32, I32, P, I32, I32, D, P, P, P, P, P]
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(C.c_void_p)


def cam_struct(cam) -> _Cam:
    c = _Cam()
    c.width, c.height, c.tile_w, c.tile_h = cam.width, cam.height, cam.tile_w, cam.tile_h
    c.fx, c.fy, c.cx, c.cy, c.near_z = cam.fx, cam.fy, cam.cx, cam.cy, cam.near
    R = np.ascontiguousarray(cam.R, dtype=np.float32).reshape(-1)
    t = np.ascontiguousarray(cam.t, dtype=np.float32).reshape(-1)
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.t[i] = float(t[i])
    return c


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


@dataclass
class Projection:
    flags: np.ndarray      # u8 [N] bit0 visible, bit1 near-degenerate (FP64 decisions)
    radius: np.ndarray     # i32 [N]
    rect: np.ndarray       # i32 [N, 4] x0, y0, x1, y1 (tiles, exclusive max)
    depth_key: np.ndarray  # f32 [N]
    mean2d: np.ndarray     # f64 [N, 2]
    conic: np.ndarray      # f64 [N, 3]
    cov2d: np.ndarray      # f64 [N, 3] dilated (c00, c01, c11)

    @property
    def visible(self):
        return (self.flags & 1).astype(bool)

    @property
    def tiles_touched(self):
        r = self.rect.astype(np.int64)
        return np.where(self.visible, (r[:, 2] - r[:, 0]) * (r[:, 3] - r[:, 1]), 0)


def project(cam, means, scales, quats) -> Projection:
    """Sec. 3.1 (Eq. 1-2) and EWA projection of every Gaussian."""
    means, scales, quats = _f32(means), _f32(scales), _f32(quats)
    n = means.shape[0]
    out = Projection(np.zeros(n, np.uint8), np.zeros(n, np.int32), np.zeros((n, 4), np.int32),
                     np.zeros(n, np.float32), np.zeros((n, 2)), np.zeros((n, 3)), np.zeros((n, 3)))
    c = cam_struct(cam)
    lib().orc_project(C.byref(c), n, _p(means), _p(scales), _p(quats), _p(out.flags),
                      _p(out.radius), _p(out.rect), _p(out.depth_key), _p(out.mean2d),
                      _p(out.conic), _p(out.cov2d))
    return out


def project_jacobian(cam, means, scales, quats) -> np.ndarray:
    """d(u, v, a, b, c)/d(mean, scale, quaternion) by complex step: f64 [N, 5, 10]."""
    m = np.ascontiguousarray(means, np.float64)
    s = np.ascontiguousarray(scales, np.float64)
    q = np.ascontiguousarray(quats, np.float64)
    jac = np.zeros((m.shape[0], 5, 10))
    c = cam_struct(cam)
    lib().orc_project_jacobian(C.byref(c), m.shape[0], _p(m), _p(s), _p(q), _p(jac))
    return jac


def project64(cam, means, scales, quats):
    """FP64 projection from double inputs: (mean2d [N,2], conic [N,3])."""
    m = np.ascontiguousarray(means, np.float64)
    s = np.ascontiguousarray(scales, np.float64)
    q = np.ascontiguousarray(quats, np.float64)
    uv = np.zeros((m.shape[0], 2))
    cn = np.zeros((m.shape[0], 3))
    c = cam_struct(cam)
    lib().orc_project64(C.byref(c), m.shape[0], _p(m), _p(s), _p(q), _p(uv), _p(cn))
    return uv, cn


def bin(cam, proj: Projection):
    """Instances ordered by (tile, depth key bits, Gaussian id); returns (gauss_ids, tile_ranges)."""
    c = cam_struct(cam)
    n = proj.flags.shape[0]
    total = lib().orc_count_instances(C.byref(c), n, _p(proj.flags), _p(proj.rect))
    ids = np.zeros(max(total, 1), np.uint32)
    ranges = np.zeros((cam.num_tiles, 2), np.uint32)
    got = lib().orc_bin(C.byref(c), n, _p(proj.flags), _p(proj.rect), _p(proj.depth_key),
                        _p(ids), _p(ranges))
    assert got == total
    return ids[:total], ranges


@dataclass
class Blend:
    out: np.ndarray        # f64 [levels, npix, C]
    final_T: np.ndarray    # f64 [npix]
    n_last: np.ndarray     # i32 [npix] list position + 1 of the last contributor
    n_contrib: np.ndarray  # i32 [npix]
    margin: np.ndarray     # f64 [npix]
    n_eval: np.ndarray = None   # i32 [npix] list entries examined (up to and including the stop)


def all_pixels(cam):
    yy, xx = np.meshgrid(np.arange(cam.height, dtype=np.int32), np.arange(cam.width, dtype=np.int32),
                         indexing="ij")
    return xx.reshape(-1).copy(), yy.reshape(-1).copy()


def blend(cam, proj: Projection, opacity, ids, ranges, idx=None, w=None, dense=None, mode=0,
          px=None, py=None, levels=None, K=None, C_out=None) -> Blend:
    """Eq. 3 front-to-back blending with Eq. 7 weights e_i.

    mode 0: Algorithm 1, sparse (idx [N,lev,K], w [N,lev,K]) -> coefficient map W [lev,npix,L=C_out]
    mode 1: dense L-vectors dense [N,lev,L] -> W (blending the zeros too)
    mode 2: dense D-dim features dense [N,lev,D] (Eq. 6) -> F directly
    """
    if px is None:
        px, py = all_pixels(cam)
    px = np.ascontiguousarray(px, np.int32)
    py = np.ascontiguousarray(py, np.int32)
    npix = px.shape[0]
    opacity = _f32(opacity)
    if mode == 0:
        idx = np.ascontiguousarray(idx, np.uint8)
        w = _f32(w)
        levels, K = idx.shape[1], idx.shape[2]
        C_out = 64 if C_out is None else C_out
        dense_p = None
    else:
        dense = np.ascontiguousarray(dense, np.float64)
        levels, C_out = dense.shape[1], dense.shape[2]
        K = 0
        idx = np.zeros(1, np.uint8)
        w = np.zeros(1, np.float32)
        dense_p = _p(dense)
    out = np.zeros((levels, npix, C_out))
    res = Blend(out, np.zeros(npix), np.zeros(npix, np.int32), np.zeros(npix, np.int32),
                np.zeros(npix), np.zeros(npix, np.int32))
    ids = np.ascontiguousarray(ids, np.uint32)
    if ids.size == 0:
        ids = np.zeros(1, np.uint32)
    ranges = np.ascontiguousarray(ranges, np.uint32)
    c = cam_struct(cam)
    lib().orc_blend(C.byref(c), npix, _p(px), _p(py), _p(proj.mean2d), _p(proj.conic), _p(opacity),
                    _p(ids), _p(ranges), mode, levels, K, C_out, _p(idx), _p(w), dense_p,
                    _p(out), _p(res.final_T), _p(res.n_last), _p(res.n_contrib), _p(res.margin),
                    _p(res.n_eval))
    return res


def decode(W, S) -> np.ndarray:
    """Eq. 7: F_lev = W_lev S_lev (plain triple loop in FP64). W [lev,npix,L], S [lev,L,D]."""
    W = np.ascontiguousarray(W, np.float64)
    S = _f32(S)
    lev, npix, L = W.shape
    D = S.shape[2]
    F = np.zeros((lev, npix, D))
    lib().orc_decode(lev, npix, L, D, _p(W), _p(S), _p(F))
    return F


def relevancy(F, text, tau: float = 10.0) -> np.ndarray:
    """Sec. 3.2 relevancy: min over negatives of softmax(tau [cos_p, cos_n])_0. -> [Q, lev, npix]."""
    F = np.ascontiguousarray(F, np.float64)
    text = _f32(text)
    lev, npix, D = F.shape
    Q, nt, _ = text.shape
    assert nt - 1 <= 63
    rel = np.zeros((Q, lev, npix))
    lib().orc_relevancy(lev, npix, D, _p(F), Q, nt - 1, _p(text), float(tau), _p(rel))
    return rel


def sparsify(logits, K: int):
    """Sec. 3.3: the L-dim parameter of a Gaussian (per level) is normalised by a softmax, the K
    largest values are kept as the nonzeros and renormalised by their sum.  logits f32 [..., L] ->
    (idx u8 [..., K], w f64 [..., K]).  The kept entries are those with the largest logits (the
    softmax is monotone; selecting on the FP32 logits keeps the integer decision exact), the lower
    index first among equal logits, listed in that order (descending value)."""
    z = np.ascontiguousarray(logits, np.float32)
    L = z.shape[-1]
    assert 1 <= K <= L <= 256
    zr = z.reshape(-1, L)
    zd = zr.astype(np.float64)
    p = np.exp(zd - zd.max(axis=1, keepdims=True))
    p = p / p.sum(axis=1, keepdims=True)                       # softmax over the L entries
    order = np.argsort(-zr, axis=1, kind="stable")[:, :K]      # top K, lower index first on ties
    pk = np.take_along_axis(p, order, axis=1)
    w = pk / pk.sum(axis=1, keepdims=True)                     # renormalised by their sum
    shape = z.shape[:-1] + (K,)
    return order.astype(np.uint8).reshape(shape), w.reshape(shape)


def sparsify_backward(idx, w, dw, L: int) -> np.ndarray:
    """Gradient of sparsify's weights with respect to the logits.  The kept weights are
    p_k / sum_m p_m with p = softmax(z), in which the softmax's denominator cancels: they equal a
    softmax over the K kept logits.  With the selection fixed (it is piecewise constant), dL/dz
    is zero for the dropped entries and w_k (dw_k - sum_m w_m dw_m) for kept entry k.
    idx [..., K], w [..., K], dw [..., K] -> dlogits f64 [..., L]."""
    w = np.asarray(w, np.float64)
    dw = np.asarray(dw, np.float64)
    g = w * (dw - (w * dw).sum(axis=-1, keepdims=True))
    out = np.zeros(np.shape(idx)[:-1] + (L,))
    np.put_along_axis(out, np.asarray(idx).astype(np.int64), g, axis=-1)
    return out


def mean_filter(M, k: int) -> np.ndarray:
    """Appendix "Evaluation Details", Avg(M): mean over the in-image part of the k x k window
    centred on each pixel (k odd). M [H, W] -> [H, W] (FP64)."""
    M = np.ascontiguousarray(M, np.float64)
    H, W = M.shape
    out = np.zeros((H, W))
    lib().orc_mean_filter(H, W, int(k), _p(M), _p(out))
    return out


@dataclass
class Post:
    smoothed: np.ndarray   # f64 [Q, levels, H*W]
    point: np.ndarray      # i32 [Q, 2] (x, y)
    level: np.ndarray      # i32 [Q]
    score: np.ndarray      # f64 [Q]
    mask: np.ndarray       # u8 [Q, H*W]


def postprocess(rel, H: int, W: int, k: int, mode: int = 0, thr: float = 0.5) -> Post:
    """Appendix "Evaluation Details" post-processing of relevancy maps rel [Q, levels, H*W]:
    mode 0 = LERF (Avg(M), level of the highest value), mode 1 = 3D-OVS / Mip-NeRF360
    (0.5 (M + Avg(M)), level of the highest mean inside its mask)."""
    rel = np.ascontiguousarray(rel, np.float64)
    Q, levels, P = rel.shape
    assert P == H * W
    out = Post(np.zeros((Q, levels, P)), np.zeros((Q, 2), np.int32), np.zeros(Q, np.int32),
               np.zeros(Q), np.zeros((Q, P), np.uint8))
    for q in range(Q):
        pt = np.zeros(2, np.int32)
        lv = np.zeros(1, np.int32)
        sc = np.zeros(1)
        sm = np.zeros((levels, P))
        mk = np.zeros(P, np.uint8)
        lib().orc_postprocess(levels, H, W, _p(np.ascontiguousarray(rel[q])), int(k), int(mode), float(thr),
                              _p(sm), _p(pt), _p(lv), _p(sc), _p(mk))
        out.smoothed[q], out.point[q], out.level[q], out.score[q], out.mask[q] = sm, pt, lv[0], sc[0], mk
    return out


@dataclass
class Render:
    proj: Projection
    ids: np.ndarray
    ranges: np.ndarray
    blend: Blend


def render(scene, cam, px=None, py=None) -> Render:
    """Project, bin and sparse-blend (Algorithm 1) the scene for the given pixels (default: all)."""
    pr = project(cam, scene.means, scene.scales, scene.quats)
    ids, ranges = bin(cam, pr)
    bl = blend(cam, pr, scene.opacity, ids, ranges, idx=scene.idx, w=scene.weights, px=px, py=py,
               C_out=scene.L)
    return Render(pr, ids, ranges, bl)


# --------------------------------------------------------------------------------------
# Gradients of the L1 feature loss  Loss = mean_{lev,p,d} |F - target|,  F = W S.

@dataclass
class Grads:
    loss: float
    dW: np.ndarray        # [lev, P, L]
    dS: np.ndarray        # [lev, L, D]
    dw: np.ndarray        # [N, lev, K]
    dopacity: np.ndarray  # [N]
    dmean2d: np.ndarray   # [N, 2]
    dconic: np.ndarray    # [N, 3]
    dmeans: np.ndarray    # [N, 3]
    dscales: np.ndarray   # [N, 3]
    dquats: np.ndarray    # [N, 4]
    near_tie: np.ndarray  # [lev, P, D] bool, |F - target| tiny: sign decided by rounding


def l1_grads(scene, cam, target, tie_eps: float = 1e-6) -> Grads:
    """Analytic FP64 gradients of Loss = mean |W S - target| (W from Algorithm 1).

    Decode adjoint (Eq. 7 is a matmul): G_F = sign(F - target)/(lev P D), dW = G_F S^T,
    dS = W^T G_F (library matmuls).  Blend adjoint: literal derivative per pixel
    (orc_blend_backward).  Projection: complex-step Jacobian, chained by a matvec.
    """
    r = render(scene, cam)
    W = r.blend.out                      # [lev, P, L]
    adj = l1_decode_adjoint(W, scene.codebook, target, tie_eps)
    loss, dW, dS = adj.loss, adj.dW, adj.dS
    lev = W.shape[0]
    n = scene.n
    K = scene.K
    dw = np.zeros((n, lev, K))
    dop = np.zeros(n)
    dm2 = np.zeros((n, 2))
    dcn = np.zeros((n, 3))
    c = cam_struct(cam)
    ids = r.ids if r.ids.size else np.zeros(1, np.uint32)
    Gc = np.ascontiguousarray(dW)
    lib().orc_blend_backward(C.byref(c), n, _p(r.proj.mean2d), _p(r.proj.conic),
                             _p(_f32(scene.opacity)), _p(np.ascontiguousarray(ids, np.uint32)),
                             _p(np.ascontiguousarray(r.ranges, np.uint32)), lev, K, scene.L,
                             _p(np.ascontiguousarray(scene.idx, np.uint8)), _p(_f32(scene.weights)),
                             _p(Gc), _p(dw), _p(dop), _p(dm2), _p(dcn))
    jac = project_jacobian(cam, scene.means, scene.scales, scene.quats)
    up = np.concatenate([dm2, dcn], axis=1)                # [N, 5]
    vis = r.proj.visible
    dparams = np.einsum("nk,nkp->np", up, jac)
    dparams[~vis] = 0.0
    return Grads(loss, dW, dS, dw, dop, dm2, dcn, dparams[:, 0:3], dparams[:, 3:6],
                 dparams[:, 6:10], adj.near_tie)


@dataclass
class DecodeAdjoint:
    loss: float
    dW: np.ndarray        # [lev, P, L]
    dS: np.ndarray        # [lev, L, D]
    near_tie: np.ndarray  # [lev, P, D] bool: |F - target| < tie_eps (sign decided by rounding)
    tie_px: np.ndarray    # [lev, P] bool: the pixel holds at least one near-tie
    dS_tie_slack: np.ndarray   # [lev, L, D]: sum_p |W| [near tie] / (lev P D), what a flipped
                               # sign can move dS by (a flip changes G by up to 2/(lev P D))


def l1_decode_adjoint(W, S, target, tie_eps: float = 1e-6, chunk: int = 65536) -> DecodeAdjoint:
    """Adjoint of the decode (Eq. 7, F = W S, a matmul) under Loss = mean |F - target| for a
    given coefficient map W [lev, P, L] and codebook S [lev, L, D]: G_F = sign(F - target) /
    (lev P D) (sign(0) = 0), dW = G_F S^T, dS = W^T G_F.  FP64 library matmuls, taken over
    blocks of `chunk` pixels so full-size maps fit in memory (the per-pixel quantities do not
    depend on the blocking; dS is the sum of the blocks' products)."""
    W = np.asarray(W, np.float64)
    S = np.asarray(S, np.float64)
    lev, P, L = W.shape
    D = S.shape[2]
    denom = float(lev * P * D)
    dW = np.zeros((lev, P, L))
    dS = np.zeros((lev, L, D))
    slack = np.zeros((lev, L, D))
    near = np.zeros((lev, P, D), bool)
    total = 0.0
    for l in range(lev):
        for p0 in range(0, P, chunk):
            p1 = min(P, p0 + chunk)
            Wb = W[l, p0:p1]
            res = Wb @ S[l] - np.asarray(target[l, p0:p1], np.float64)
            total += float(np.abs(res).sum())
            G = np.sign(res) / denom
            dW[l, p0:p1] = G @ S[l].T
            dS[l] += Wb.T @ G
            tie = np.abs(res) < tie_eps
            near[l, p0:p1] = tie
            slack[l] += np.abs(Wb).T @ tie.astype(np.float64) / denom
    return DecodeAdjoint(total / denom, dW, dS, near, near.any(-1), slack)


def l1_loss_fd_eval(scene_params, cam, ids, ranges, tile_mask, idx, S, target):
    """Sum over the masked tiles of |F - target| with FP64 parameters (fixed binning).

    scene_params = (means, scales, quats, opacity, weights) as float64 arrays.
    Returns (per-pixel sums [P] (zero outside the mask), signature of all discrete decisions).
    """
    m, s, q, o, w = [np.ascontiguousarray(a, np.float64) for a in scene_params]
    n = m.shape[0]
    lev, K = idx.shape[1], idx.shape[2]
    L, D = S.shape[1], S.shape[2]
    sig = C.c_uint64(0)
    c = cam_struct(cam)
    per_pixel = np.zeros(cam.num_pixels)
    ids = np.ascontiguousarray(ids if ids.size else np.zeros(1, np.uint32), np.uint32)
    lib().orc_l1_loss_tiles(C.byref(c), n, _p(m), _p(s), _p(q), _p(o), _p(ids),
                                  _p(np.ascontiguousarray(ranges, np.uint32)),
                                  _p(np.ascontiguousarray(tile_mask, np.uint8)), lev, K, L, D,
                                  _p(np.ascontiguousarray(idx, np.uint8)), _p(w), _p(_f32(S)),
                                  _p(_f32(target)), _p(per_pixel), C.byref(sig))
    return per_pixel, sig.value


# --------------------------------------------------------------------------------------
# The decoder-based comparison path (LangSplat*).

def mlp_decode(x, layers) -> np.ndarray:
    """Sec. 3.1: the decoder g_d maps a rendered latent feature (Eq. 4) back to the D-dim CLIP space.
    g_d is an MLP: every layer but the last is affine then ReLU, the last is affine.  FP64 NumPy,
    one layer at a time.  x [rows, d_in]; layers: list of (W [w_in, w_out], b [w_out]).
    -> [rows, w_out of the last layer]."""
    h = np.asarray(x, np.float64)
    for i, (W, b) in enumerate(layers):
        h = h @ np.asarray(W, np.float64) + np.asarray(b, np.float64)
        if i < len(layers) - 1:
            h = np.maximum(h, 0.0)
    return h
