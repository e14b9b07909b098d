"""Parity at the sizes the benchmark runs, where the persistent kernels loop.

* The whole at-scale frame (300,000 Gaussians, three levels, 1440x1080): all 1,555,200 pixels'
  coefficient maps, final transmittances and last contributors against the oracle's FP64 blend,
  the pixels split over a pool of host processes.

* lsv2_l1_decode_backward on the differentiation workload (100,000 Gaussians, one level,
  720x540, D = 512): 388,800 pixels, so every persistent CTA walks many pixel tiles and adds
  its codebook-gradient partial once at the end.  Loss, dLoss/dW on sampled pixels and the
  whole dLoss/dS against the oracle's FP64 decode adjoint of the same coefficient map.
* lsv2_query_views over four views with 7,800 16x16 tiles (about 26 per persistent splat CTA)
  and 64 queries (two query groups of 32 in the relevancy): equal bit for bit to four
  sequential single-view pipelines, and within the BF16 relevancy bound (1e-2) of the oracle on
  sampled pixels.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import lsv2_synth as syn
from oracle import oracle as O

import oracle_workers
from gpu_helpers import KNIFE_EDGE

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_07136_b300 import _lib as L  # noqa: E402
from paper_2507_07136_b300.pipeline import DeviceScene, Frame, _ptr, _stream  # noqa: E402
from paper_2507_07136_b300.views import ViewsBatch  # noqa: E402


def test_at_scale_whole_frame_coefficient_map():
    sc, cam, _ = syn.at_scale()
    pr = O.project(cam, sc.means, sc.scales, sc.quats)
    ids, ranges = O.bin(cam, pr)
    fr = Frame(DeviceScene.from_numpy(sc), cam)
    fr.render()
    fr.check()
    W = fr.coeff.cpu().numpy()
    T = fr.final_T.cpu().numpy()
    nl = fr.n_last.cpu().numpy()
    px, py = O.all_pixels(cam)
    workers = max(1, min(16, os.cpu_count() or 1))
    chunks = np.array_split(np.arange(cam.num_pixels), workers * 8)
    tasks = [(px[c], py[c], np.ascontiguousarray(W[:, c]), T[c], nl[c]) for c in chunks]
    with mp.get_context("spawn").Pool(workers, initializer=oracle_workers.init_blend,
                                      initargs=(cam, pr, sc.opacity, ids, ranges, sc.idx, sc.weights,
                                                KNIFE_EDGE)) as pool:
        res = pool.map(oracle_workers.blend_check, tasks)
    assert sum(r["pixels"] for r in res) == cam.num_pixels
    checked = sum(r["checked"] for r in res)
    assert checked > 0.99 * cam.num_pixels
    assert sum(r["contributions"] for r in res) > 10 * cam.num_pixels
    assert max(r["w_worst"] for r in res) <= 1.0, f"W: worst x{max(r['w_worst'] for r in res):.2f} of bound"
    assert max(r["t_worst"] for r in res) <= 1.0
    assert sum(r["n_last_mismatch"] for r in res) == 0
    # knife-edge pixels: one decision may flip, which moves W by at most one contribution
    assert max(r["knife_err"] for r in res) < 0.05


def test_l1_decode_backward_full_size():
    sc, cam = syn.differentiation()
    D = sc.D
    target = syn.l1_target(cam)
    ds = DeviceScene.from_numpy(sc)
    fr = Frame(ds, cam)
    fr.render()
    P = fr.P
    ntiles = (P + 127) // 128         # 128-pixel tiles of the persistent kernel
    assert ntiles >= 10 * torch.cuda.get_device_properties(0).multi_processor_count
    loss = torch.zeros(1, device="cuda")
    dW = torch.empty_like(fr.coeff)
    dS = torch.zeros_like(ds.codebook)
    tg = torch.as_tensor(target, device="cuda")
    L.lsv2_l1_decode_backward(1, P, 64, D, _ptr(fr.coeff), _ptr(ds.codebook), _ptr(tg), _ptr(loss), _ptr(dW),
                              _ptr(dS), _ptr(fr.status), _stream(None))
    fr.check()
    Wg = fr.coeff.cpu().numpy().astype(np.float64)   # the adjoint is checked on the GPU's own W
    S = sc.codebook.astype(np.float64)
    adj = O.l1_decode_adjoint(Wg, S, target)
    assert float(loss.item()) == pytest.approx(adj.loss, rel=1e-5)
    n = float(1 * P * D)
    # dLoss/dW on 20,000 sampled pixels holding no near-tie: |err| <= 1e-5 sum_d |G| |S|
    rng = np.random.default_rng(5)
    pix = rng.choice(P, 20000, replace=False)
    pix = pix[~adj.tie_px[0, pix]]
    assert pix.size > 15000
    got = dW[0, torch.as_tensor(pix, device="cuda")].cpu().numpy().astype(np.float64)
    Gs = np.sign(Wg[0, pix] @ S[0] - target[0, pix].astype(np.float64)) / n
    bound = 1e-5 * (np.abs(Gs) @ np.abs(S[0]).T) + 1e-12
    err = np.abs(got - adj.dW[0, pix])
    assert np.all(err <= bound), f"dW: worst x{(err / bound).max():.2f} of bound"
    # the whole dLoss/dS: |err| <= 1e-5 sum_p |W| |G| + what near-tie sign flips can move
    absWG = np.zeros_like(S)
    for p0 in range(0, P, 65536):
        Wb = Wg[0, p0:p0 + 65536]
        G = np.sign(Wb @ S[0] - target[0, p0:p0 + 65536].astype(np.float64)) / n
        absWG[0] += np.abs(Wb).T @ np.abs(G)
    dbound = 1e-5 * absWG + 2.0 * adj.dS_tie_slack + 1e-12
    derr = np.abs(dS.cpu().numpy().astype(np.float64) - adj.dS)
    assert np.all(derr <= dbound), f"dS: worst x{(derr / dbound).max():.2f} of bound"


FULL_RES = [(960, 720), (640, 480), (960, 720), (640, 480)]


def waves_batch(tile=(16, 16)):
    sc = syn.make_scene(100_000, 3, seed=syn.SEED + 4)
    cams = [syn.orbit_camera(w, h, 6.0, azimuth_deg=37.0 * k, tile=tile) for k, (w, h) in enumerate(FULL_RES)]
    text = syn.text_queries(syn.SEED + 2, 64, 4)
    return sc, cams, text


def single_view_rel(ds, cam, text):
    fr = Frame(ds, cam)
    fr.render()
    rel = torch.empty((text.shape[0], ds.levels, cam.num_pixels), dtype=torch.bfloat16, device="cuda")
    fr.query(torch.as_tensor(text, device="cuda"), rel, compute=L.LSV2_BF16)
    fr.check()
    return rel


@pytest.mark.parametrize("tile", [(16, 16), (8, 8)])
def test_views_many_waves_64_queries_equal_sequential(tile):
    sc, cams, text = waves_batch(tile)
    ntiles = sum(c.num_tiles for c in cams)
    assert ntiles >= 3 * 2 * torch.cuda.get_device_properties(0).multi_processor_count
    ds = DeviceScene.from_numpy(sc)
    vb = ViewsBatch(ds, cams, text.shape[0], text.shape[1] - 1, tile=tile)
    vb.capture(torch.as_tensor(text, device="cuda"))
    vb.replay()
    vb.check()
    for v, cam in enumerate(vb.cams):
        ref = single_view_rel(ds, cam, text)
        assert torch.equal(vb.rel_view(v), ref), f"view {v}"


def test_views_many_waves_64_queries_against_oracle():
    sc, cams, text = waves_batch()
    ds = DeviceScene.from_numpy(sc)
    vb = ViewsBatch(ds, cams, text.shape[0], text.shape[1] - 1)
    vb.run(torch.as_tensor(text, device="cuda"))
    vb.check()
    rng = np.random.default_rng(17)
    for v, cam in enumerate(cams):
        px = rng.integers(0, cam.width, 1500).astype(np.int32)
        py = rng.integers(0, cam.height, 1500).astype(np.int32)
        r = O.render(sc, cam, px=px, py=py)
        ro = O.relevancy(O.decode(r.blend.out, sc.codebook), text, 10.0)
        ok = r.blend.margin > KNIFE_EDGE
        flat = torch.as_tensor((py.astype(np.int64) * cam.width + px)[ok], device="cuda")
        got = vb.rel_view(v)[:, :, flat].float().cpu().numpy()
        assert np.abs(got - ro[:, :, ok]).max() <= 1e-2, f"view {v}"
