"""GPU parity of the forward path against the FP64 oracle, through the C ABI.

Bit-exact: visibility, radius, tile rectangles, depth keys, per-tile lists.  FP32 maps
(coefficient map W, final T, decoded features F, relevancy): 1e-5 relative, on every pixel
whose decisions are not within rounding of a threshold (those are counted and bounded).
"""
import numpy as np
import pytest

import lsv2_synth as syn
from oracle import oracle as O

from gpu_helpers import KNIFE_EDGE, assert_map_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_07136_b300 import _lib as L  # noqa: E402
from paper_2507_07136_b300.pipeline import DeviceScene, Frame  # noqa: E402


def gpu_frame(sc, cam, capacity=None):
    ds = DeviceScene.from_numpy(sc)
    fr = Frame(ds, cam, capacity=capacity)
    fr.render()
    fr.check()
    return ds, fr


def check_projection(fr, ref):
    flags = fr.flags.cpu().numpy()
    assert np.array_equal(flags, ref.flags)
    vis = ref.visible
    assert np.array_equal(fr.radius.cpu().numpy()[vis], ref.radius[vis])
    assert np.array_equal(fr.rect.cpu().numpy()[vis], ref.rect[vis])
    assert np.array_equal(fr.tiles_touched.cpu().numpy(), ref.tiles_touched.astype(np.int32))
    assert np.array_equal(fr.depth.cpu().numpy()[vis].view(np.uint32), ref.depth_key[vis].view(np.uint32))
    xy = fr.xy.cpu().numpy().astype(np.float64)
    mean = np.stack([xy[:, 0] + xy[:, 2], xy[:, 1] + xy[:, 3]], 1)
    np.testing.assert_allclose(mean[vis], ref.mean2d[vis], rtol=0, atol=1e-7)
    conic = fr.conic_o.cpu().numpy()[:, :3].astype(np.float64)
    scale = np.abs(ref.conic[vis]).max(1, keepdims=True)
    assert np.all(np.abs(conic[vis] - ref.conic[vis]) <= 2e-7 * scale)


def check_bins(fr, ids, ranges):
    got_ranges = fr.tile_ranges.cpu().numpy().astype(np.uint32)
    assert np.array_equal(got_ranges, ranges)
    n = int(fr.num_instances.item())
    assert n == ids.size
    assert np.array_equal(fr.gauss_ids[:n].cpu().numpy().astype(np.uint32), ids)


def check_blend(fr, bl, px, py, cam):
    W = fr.coeff.cpu().numpy()
    pix = py.astype(np.int64) * cam.width + px
    ok = bl.margin > KNIFE_EDGE
    assert_map_close(W[:, pix][:, ok], bl.out[:, ok], what="coefficient map")
    assert_map_close(fr.final_T.cpu().numpy()[pix][ok], bl.final_T[ok], what="final T")
    assert np.array_equal(fr.n_last.cpu().numpy()[pix][ok], bl.n_last[ok])
    # knife-edge pixels: one decision may flip, which moves W by at most one contribution
    if (~ok).any():
        err = np.abs(W[:, pix][:, ~ok] - bl.out[:, ~ok]).max()
        assert err < 0.05
    return int((~ok).sum())


@pytest.fixture(scope="module")
def tiny():
    sc, cam = syn.tiny()
    ref = O.render(sc, cam)
    ds, fr = gpu_frame(sc, cam)
    return sc, cam, ref, ds, fr


def test_project_tiny(tiny):
    sc, cam, ref, ds, fr = tiny
    check_projection(fr, ref.proj)


def test_binsort_tiny(tiny):
    sc, cam, ref, ds, fr = tiny
    check_bins(fr, ref.ids, ref.ranges)


def test_splat_tiny(tiny):
    sc, cam, ref, ds, fr = tiny
    px, py = O.all_pixels(cam)
    check_blend(fr, ref.blend, px, py, cam)


def test_decode_f32_tiny(tiny):
    sc, cam, ref, ds, fr = tiny
    F = torch.empty((1, cam.num_pixels, 512), device="cuda")
    fr.decode(F)
    fr.check()
    Fg = F.cpu().numpy()
    # decode kernel alone: against the FP64 product of the GPU's own W
    Wg = fr.coeff.cpu().numpy().astype(np.float64)
    S = sc.codebook.astype(np.float64)
    exact = np.matmul(Wg, S)
    bound = 1e-5 * np.matmul(np.abs(Wg), np.abs(S)) + 1e-9
    assert np.all(np.abs(Fg - exact) <= bound)
    # end to end against the oracle's decode of its own W (non knife-edge pixels)
    Fo = O.decode(ref.blend.out, sc.codebook)
    ok = ref.blend.margin > KNIFE_EDGE
    bound = 1e-5 * np.matmul(np.abs(ref.blend.out[:, ok]), np.abs(S)) + 1e-9
    assert np.all(np.abs(Fg[:, ok] - Fo[:, ok]) <= bound)


def test_query_f32_tiny(tiny):
    sc, cam, ref, ds, fr = tiny
    text = syn.text_queries(syn.SEED + 2, 2, 4)
    tt = torch.as_tensor(text, device="cuda")
    rel = torch.empty((2, 1, cam.num_pixels), device="cuda")
    fr.query(tt, rel, tau=10.0)
    fr.check()
    Fo = O.decode(ref.blend.out, sc.codebook)
    ro = O.relevancy(Fo, text, 10.0)
    ok = ref.blend.margin > KNIFE_EDGE
    assert_map_close(rel.cpu().numpy()[:, :, ok], ro[:, :, ok], rel=1e-5, floor=1e-7, what="relevancy")


@pytest.mark.parametrize("tile", [(8, 8), (32, 8)])
def test_tile_shapes(tile):
    sc, cam = syn.tiny()
    cam = cam.with_tile(*tile)
    ref = O.render(sc, cam)
    ds, fr = gpu_frame(sc, cam)
    check_projection(fr, ref.proj)
    check_bins(fr, ref.ids, ref.ranges)
    px, py = O.all_pixels(cam)
    check_blend(fr, ref.blend, px, py, cam)


@pytest.mark.parametrize("K", [2, 6, 8])
def test_k_variants(K):
    sc = syn.make_scene(1500, 1, seed=7, mean_kind="uniform", mean_param=1.0, log_scale_mu=-3.0,
                        log_scale_sigma=0.3, K=K)
    cam = syn.orbit_camera(96, 80, 4.0)
    ref = O.render(sc, cam)
    ds, fr = gpu_frame(sc, cam)
    px, py = O.all_pixels(cam)
    check_blend(fr, ref.blend, px, py, cam)


def test_three_levels_ragged_image():
    """Three levels, image size not a multiple of the tile (ragged right/bottom tiles)."""
    sc = syn.make_scene(3000, 3, seed=11, mean_kind="uniform", mean_param=1.0, log_scale_mu=-3.2,
                        log_scale_sigma=0.4)
    cam = syn.orbit_camera(141, 99, 4.0)
    ref = O.render(sc, cam)
    ds, fr = gpu_frame(sc, cam)
    check_projection(fr, ref.proj)
    check_bins(fr, ref.ids, ref.ranges)
    px, py = O.all_pixels(cam)
    check_blend(fr, ref.blend, px, py, cam)


def test_duplicate_indices_and_stacked_closed_form():
    """Repeated indices within a Gaussian add up; 20 stacked alpha = 0.5 Gaussians give the
    Eq. 3 closed form (13 contributors, T = 2^-13) on the GPU as well."""
    n = 20
    means = np.stack([np.zeros(n), np.zeros(n), 0.1 * np.arange(n)], 1).astype(np.float32)
    idx = np.stack([np.arange(n), np.arange(n), 40 + np.arange(n), 60 + np.arange(n) % 4], 1)[:, None, :]
    w = np.tile([0.5, 0.25, 0.125, 0.125], (n, 1))[:, None, :].astype(np.float32)
    sc = syn.Scene(means, np.full((n, 3), 0.05, np.float32), np.tile([1, 0, 0, 0], (n, 1)).astype(np.float32),
                   np.full(n, 0.5, np.float32), idx.astype(np.uint8), w, syn.codebooks(1, 1))
    cam = syn.orbit_camera(33, 33, 4.0)
    ref = O.render(sc, cam)
    ds, fr = gpu_frame(sc, cam)
    p = 16 * 33 + 16
    assert int(fr.n_last[p].item()) == 13
    assert float(fr.final_T[p].item()) == 2.0 ** -13
    px, py = O.all_pixels(cam)
    check_blend(fr, ref.blend, px, py, cam)


@pytest.mark.parametrize("opacity", [0.05, 0.9])
def test_crowded_tiles_three_levels(opacity):
    """Three levels on 16 x 16 tiles (the kernel whose warps 4-7 accumulate in TMEM): 3,000
    Gaussians packed into a few tiles, so a tile's list runs to thousands of records (many
    32-record batches through the 2-stage ring, the barriers' phases wrapping many times).
    Translucent Gaussians (opacity 0.05) keep every pixel blending to the end of its list;
    opaque ones (0.9) end most pixels early (warps done before the producer is)."""
    rng = np.random.default_rng(21)
    n = 3000
    means = np.stack([rng.uniform(-0.12, 0.12, n), rng.uniform(-0.12, 0.12, n), rng.uniform(-0.5, 0.5, n)],
                     1).astype(np.float32)
    scales = np.exp(rng.normal(-3.4, 0.3, (n, 3))).astype(np.float32)
    q = rng.normal(size=(n, 4))
    q = (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(np.float32)
    idx, w = syn.sparse_coefficients(rng, n, 3, 4, 64)
    sc = syn.Scene(means, scales, q, np.full(n, opacity, np.float32), idx, w, syn.codebooks(5, 3))
    cam = syn.orbit_camera(64, 48, 4.0)
    ref = O.render(sc, cam)
    ds, fr = gpu_frame(sc, cam)
    ranges = ref.ranges.reshape(-1, 2)
    assert int((ranges[:, 1] - ranges[:, 0]).max()) > 1000, "the scene should crowd some tiles"
    check_projection(fr, ref.proj)
    check_bins(fr, ref.ids, ref.ranges)
    px, py = O.all_pixels(cam)
    check_blend(fr, ref.blend, px, py, cam)


def test_medium_tiles_three_levels():
    """Tiles of 513 to 2,048 instances (sorted by four warps in registers and merged by rank):
    bins bit-exact and the blend against the oracle."""
    rng = np.random.default_rng(22)
    n = 2000
    means = np.stack([rng.uniform(-0.35, 0.35, n), rng.uniform(-0.35, 0.35, n), rng.uniform(-0.5, 0.5, n)],
                     1).astype(np.float32)
    scales = np.exp(rng.normal(-3.4, 0.3, (n, 3))).astype(np.float32)
    q = rng.normal(size=(n, 4))
    q = (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(np.float32)
    idx, w = syn.sparse_coefficients(rng, n, 3, 4, 64)
    sc = syn.Scene(means, scales, q, np.full(n, 0.5, np.float32), idx, w, syn.codebooks(5, 3))
    cam = syn.orbit_camera(64, 48, 4.0)
    ref = O.render(sc, cam)
    counts = np.diff(ref.ranges.reshape(-1, 2), axis=1)[:, 0]
    assert int(((counts > 512) & (counts <= 2048)).sum()) >= 2, "the scene should give medium tiles"
    ds, fr = gpu_frame(sc, cam)
    check_bins(fr, ref.ids, ref.ranges)
    px, py = O.all_pixels(cam)
    check_blend(fr, ref.blend, px, py, cam)


def test_repeated_indices_three_levels():
    """Three levels (TMEM-accumulator kernel): repeated indices in every level are merged into one
    pair and the emptied repeats accumulate nothing, whichever accumulator store a pixel's warp
    uses; the stacked closed form (13 contributors, T = 2^-13) holds at every level."""
    n = 20
    means = np.stack([np.zeros(n), np.zeros(n), 0.1 * np.arange(n)], 1).astype(np.float32)
    lev = [np.stack([np.arange(n), np.arange(n), 40 + np.arange(n), 60 + np.arange(n) % 4], 1),
           np.stack([7 + np.zeros(n, int), 7 + np.zeros(n, int), 7 + np.zeros(n, int), 9 + np.arange(n)], 1),
           np.stack([63 - np.arange(n), 1 + np.arange(n), 63 - np.arange(n), 1 + np.arange(n)], 1)]
    idx = np.stack(lev, 1).astype(np.uint8)
    w = np.tile([0.5, 0.25, 0.125, 0.125], (n, 3, 1)).astype(np.float32)
    sc = syn.Scene(means, np.full((n, 3), 0.05, np.float32), np.tile([1, 0, 0, 0], (n, 1)).astype(np.float32),
                   np.full(n, 0.5, np.float32), idx, w, syn.codebooks(1, 3))
    cam = syn.orbit_camera(33, 33, 4.0)
    ref = O.render(sc, cam)
    ds, fr = gpu_frame(sc, cam)
    p = 16 * 33 + 16
    assert int(fr.n_last[p].item()) == 13
    assert float(fr.final_T[p].item()) == 2.0 ** -13
    # level 1 of the centre pixel: entry 7 carries 0.875 of every contribution
    total = 1.0 - 2.0 ** -13
    assert abs(float(fr.coeff[1, p, 7].item()) - 0.875 * total) <= 1e-5 * total
    px, py = O.all_pixels(cam)
    check_blend(fr, ref.blend, px, py, cam)


def test_empty_and_culled_scenes():
    cam = syn.orbit_camera(64, 48, 4.0)
    # every Gaussian behind the camera or with a zero quaternion
    n = 64
    means = np.zeros((n, 3), np.float32)
    means[: n // 2, 2] = -10.0
    q = np.tile([1, 0, 0, 0], (n, 1)).astype(np.float32)
    q[n // 2:] = 0.0
    idx, w = syn.sparse_coefficients(np.random.default_rng(0), n, 1, 4, 64)
    sc = syn.Scene(means, np.full((n, 3), 0.05, np.float32), q, np.full(n, 0.9, np.float32), idx, w,
                   syn.codebooks(1, 1))
    ds, fr = gpu_frame(sc, cam, capacity=1024)
    assert int(fr.num_instances.item()) == 0
    assert float(fr.coeff.abs().max().item()) == 0.0
    assert bool((fr.final_T == 1.0).all().item())
    assert int(fr.n_last.max().item()) == 0


def test_capacity_overflow_reports_status():
    sc, cam = syn.tiny()
    ds = DeviceScene.from_numpy(sc)
    fr = Frame(ds, cam, capacity=1000)
    fr.render()
    torch.cuda.synchronize()
    assert int(fr.status.item()) == 3
    assert int(fr.num_instances.item()) > 1000
    r = fr.tile_ranges.cpu().numpy()
    assert r.max() <= 1000


def test_invalid_index_reports_status():
    sc, cam = syn.tiny()
    sc.idx[5, 0, 2] = 200
    ds = DeviceScene.from_numpy(sc)
    fr = Frame(ds, cam)
    fr.render()
    torch.cuda.synchronize()
    assert int(fr.status.item()) == 1


def test_degenerate_needles_take_fp64_branch():
    cam = syn.orbit_camera(128, 96, 4.0)
    rng = np.random.default_rng(5)
    n = 200
    s = np.exp(rng.normal(-3, 0.3, (n, 3))).astype(np.float32)
    s[:, 0] = np.exp(-14.0)
    s[:100, 1] = np.exp(-14.0)      # needles (two tiny axes)
    q = syn.unit_rows(rng.standard_normal((n, 4))).astype(np.float32)
    q[:100] = [1, 0, 0, 0]          # edge-on needles along z
    means = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
    idx, w = syn.sparse_coefficients(rng, n, 1, 4, 64)
    sc = syn.Scene(means, s, q, np.full(n, 0.8, np.float32), idx, w, syn.codebooks(1, 1))
    ref = O.render(sc, cam)
    assert (ref.proj.flags & 2).sum() > 0
    ds, fr = gpu_frame(sc, cam)
    check_projection(fr, ref.proj)
    check_bins(fr, ref.ids, ref.ranges)
    px, py = O.all_pixels(cam)
    check_blend(fr, ref.blend, px, py, cam)


def test_at_scale_sampled():
    """300,000 Gaussians, three levels, 1440x1080: full bit-exact binning, and W / F / relevancy
    on sampled pixels (random + every pixel of the densest tile)."""
    sc, cam, text = syn.at_scale()
    pr = O.project(cam, sc.means, sc.scales, sc.quats)
    ids, ranges = O.bin(cam, pr)
    ds, fr = gpu_frame(sc, cam)
    check_projection(fr, pr)
    check_bins(fr, ids, ranges)
    rng = np.random.default_rng(3)
    k = 3000
    px = rng.integers(0, cam.width, k).astype(np.int32)
    py = rng.integers(0, cam.height, k).astype(np.int32)
    dense = int(np.argmax(ranges[:, 1] - ranges[:, 0]))
    GX = cam.grid[0]
    tx, ty = dense % GX, dense // GX
    yy, xx = np.meshgrid(np.arange(16) + 16 * ty, np.arange(16) + 16 * tx, indexing="ij")
    px = np.concatenate([px, xx.reshape(-1)]).astype(np.int32)
    py = np.concatenate([py, yy.reshape(-1)]).astype(np.int32)
    bl = O.blend(cam, pr, sc.opacity, ids, ranges, idx=sc.idx, w=sc.weights, px=px, py=py)
    check_blend(fr, bl, px, py, cam)
    tt = torch.as_tensor(text, device="cuda")
    rel = torch.empty((1, 3, cam.num_pixels), device="cuda")
    fr.query(tt, rel, tau=10.0)
    fr.check()
    Fo = O.decode(bl.out, sc.codebook)
    ro = O.relevancy(Fo, text, 10.0)
    pix = py.astype(np.int64) * cam.width + px
    ok = bl.margin > KNIFE_EDGE
    assert_map_close(rel.cpu().numpy()[:, :, pix][:, :, ok], ro[:, :, ok], rel=1e-5, floor=1e-7, what="relevancy")
