"""Tensor-core relevancy (tcgen05, BF16 operands, FP32 accumulation) through the C ABI.

Against the FP64 oracle (unrounded path): |rel - oracle| <= 1e-2 (the BF16 variant's bound).
Against FP64 evaluated on the BF16-rounded operands (W and the columns of [S S^T | S t]):
|rel - ref| <= 1e-4 (checks the kernel itself: FP32 accumulation, epilogue arithmetic)."""
import numpy as np
import pytest

import lsv2_synth as syn
from oracle import oracle as O

from gpu_helpers import KNIFE_EDGE

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_07136_b300 import _lib as L  # noqa: E402
from paper_2507_07136_b300.pipeline import DeviceScene, Frame  # noqa: E402


def bf16(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def rounded_reference(W, S, text, tau):
    """FP64 relevancy from BF16-rounded W and BF16-rounded columns of [S S^T | S t]."""
    S = S.astype(np.float64)
    T = text.reshape(-1, text.shape[-1]).astype(np.float64)
    G = bf16(np.einsum("lid,ljd->lij", S, S))            # [lev, 64, 64]
    U = bf16(np.einsum("lid,td->lit", S, T))             # [lev, 64, nt]
    Wb = bf16(W)
    n2 = np.einsum("lpi,lij,lpj->lp", Wb, G, Wb)
    s = np.einsum("lpi,lit->lpt", Wb, U)
    nf = np.sqrt(np.maximum(n2, 0))
    tn = np.linalg.norm(T, axis=-1)
    cos = np.where(nf[..., None] < 1e-12, 0.0, s / (np.maximum(nf, 1e-300)[..., None] * tn))
    Q, per = text.shape[0], text.shape[1]
    cos = cos.reshape(cos.shape[0], cos.shape[1], Q, per)
    rel = 1.0 / (1.0 + np.exp(-tau * (cos[..., 0] - cos[..., 1:].max(-1))))
    return np.transpose(rel, (2, 0, 1))                  # [Q, lev, P]


def run_query(sc, cam, text, out_dtype=torch.float32, tau=10.0):
    ds = DeviceScene.from_numpy(sc)
    fr = Frame(ds, cam)
    fr.render()
    rel = torch.empty((text.shape[0], sc.levels, cam.num_pixels), dtype=out_dtype, device="cuda")
    fr.query(torch.as_tensor(text, device="cuda"), rel, tau=tau, compute=L.LSV2_BF16)
    fr.check()
    return fr, rel.float().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("out_dtype", [torch.float32, torch.bfloat16])
def test_query_tc_tiny(out_dtype):
    sc, cam = syn.tiny()
    text = syn.text_queries(syn.SEED + 2, 2, 4)
    fr, rel = run_query(sc, cam, text, out_dtype)
    ref = O.render(sc, cam)
    ro = O.relevancy(O.decode(ref.blend.out, sc.codebook), text, 10.0)
    ok = ref.blend.margin > KNIFE_EDGE
    assert np.abs(rel[:, :, ok] - ro[:, :, ok]).max() <= 1e-2
    rb = rounded_reference(fr.coeff.cpu().numpy(), sc.codebook, text, 10.0)
    tol = 1e-4 if out_dtype == torch.float32 else 1e-4 + 2.0 ** -8
    assert np.abs(rel - rb).max() <= tol


def test_query_tc_many_queries_three_levels():
    """64 queries x (1 + 4) texts = 320 text columns: two MMA widths (256 + 144)."""
    sc = syn.make_scene(3000, 3, seed=11, mean_kind="uniform", mean_param=1.0, log_scale_mu=-3.2, log_scale_sigma=0.4)
    cam = syn.orbit_camera(141, 99, 4.0)
    text = syn.text_queries(syn.SEED + 2, 64, 4)
    fr, rel = run_query(sc, cam, text)
    ref = O.render(sc, cam)
    ro = O.relevancy(O.decode(ref.blend.out, sc.codebook), text, 10.0)
    ok = ref.blend.margin > KNIFE_EDGE
    assert np.abs(rel[:, :, ok] - ro[:, :, ok]).max() <= 1e-2
    rb = rounded_reference(fr.coeff.cpu().numpy(), sc.codebook, text, 10.0)
    assert np.abs(rel - rb).max() <= 1e-4


def test_query_tc_at_scale_sampled():
    sc, cam, text = syn.at_scale()
    fr, rel = run_query(sc, cam, text)
    rng = np.random.default_rng(4)
    pix = rng.integers(0, cam.num_pixels, 4000)
    W = fr.coeff.cpu().numpy()[:, pix]
    rb = rounded_reference(W, sc.codebook, text, 10.0)
    assert np.abs(rel[:, :, pix] - rb).max() <= 1e-4
    px = (pix % cam.width).astype(np.int32)
    py = (pix // cam.width).astype(np.int32)
    pr = O.project(cam, sc.means, sc.scales, sc.quats)
    ids, ranges = O.bin(cam, pr)
    bl = O.blend(cam, pr, sc.opacity, ids, ranges, idx=sc.idx, w=sc.weights, px=px, py=py)
    ro = O.relevancy(O.decode(bl.out, sc.codebook), text, 10.0)
    ok = bl.margin > KNIFE_EDGE
    assert np.abs(rel[:, :, pix][:, :, ok] - ro[:, :, ok]).max() <= 1e-2


@pytest.mark.parametrize("Q,n_neg", [(3, 1), (13, 2), (88, 4)])
def test_query_tc_ragged_query_counts(Q, n_neg):
    """Query counts that are not multiples of the 8-query chunk (padding columns), up to the
    largest count that fits 512 TMEM columns at four negatives."""
    sc = syn.make_scene(2000, 2, seed=12, mean_kind="uniform", mean_param=1.0, log_scale_mu=-3.2, log_scale_sigma=0.4)
    cam = syn.orbit_camera(97, 71, 4.0)
    text = syn.text_queries(syn.SEED + 2 + Q, Q, n_neg)
    fr, rel = run_query(sc, cam, text)
    rb = rounded_reference(fr.coeff.cpu().numpy(), sc.codebook, text, 10.0)
    assert np.abs(rel - rb).max() <= 1e-4
