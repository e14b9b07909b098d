"""Tensor-core relevancy (tcgen05, BF16 operands, FP32 accumulation) through the C ABI.

Against the FP64 oracle (unrounded path): |rel - oracle| <= 1e-2 (the BF16 variant's bound).
Against FP64 evaluated on the BF16-rounded operands (W and the columns of [C | S t], where the
kernels form |F|^2 = |W C|^2 with S S^T = C C^T): |rel - ref| <= 1e-4 (checks the kernel itself:
FP32 accumulation, epilogue arithmetic).  The factor C is the one the call formed (read back from
its workspace, where the header documents it) and is itself checked against S S^T in FP64."""
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


def factor_of(fr, levels, nt):
    """C^T [levels, 64, 64] from the call's workspace (the first 64 rows of each level's B^T)."""
    bt = fr.query_ws[: levels * (64 + nt) * 64 * 4].view(torch.float32).cpu().numpy()
    return bt.reshape(levels, 64 + nt, 64)[:, :64].astype(np.float64)


def rounded_reference(W, S, text, tau, Ct):
    """FP64 relevancy from BF16-rounded W and BF16-rounded columns of [C | S t]."""
    S = S.astype(np.float64)
    T = text.reshape(-1, text.shape[-1]).astype(np.float64)
    C = bf16(np.transpose(Ct, (0, 2, 1)))               # [lev, 64 (k), 64 (j)]: column j of C
    U = bf16(np.einsum("lid,td->lit", S, T))             # [lev, 64, nt]
    Wb = bf16(W)
    n2 = (np.einsum("lpi,lij->lpj", Wb, C) ** 2).sum(-1)
    s = np.einsum("lpi,lit->lpt", Wb, U)
    nf = np.sqrt(np.maximum(n2, 0))
    tn = np.linalg.norm(T, axis=-1)
    cos = np.where(nf[..., None] < 1e-12, 0.0, s / (np.maximum(nf, 1e-300)[..., None] * tn))
    Q, per = text.shape[0], text.shape[1]
    cos = cos.reshape(cos.shape[0], cos.shape[1], Q, per)
    rel = 1.0 / (1.0 + np.exp(-tau * (cos[..., 0] - cos[..., 1:].max(-1))))
    return np.transpose(rel, (2, 0, 1))                  # [Q, lev, P]


def check_factor(Ct, S, slack=0.0):
    """C lower triangular with a nonnegative diagonal, and C C^T = S S^T up to FP32 Cholesky's
    backward error (65 roundings of 2^-24 of |C||C^T|, plus the FP32 rounding of S S^T) and
    `slack` sqrt(G_ii G_jj) (dropped pivots)."""
    S = S.astype(np.float64)
    G = np.einsum("lid,ljd->lij", S, S)
    C = np.transpose(Ct, (0, 2, 1))
    assert np.all(np.triu(C, 1) == 0.0)
    assert np.all(np.diagonal(C, axis1=1, axis2=2) >= 0.0)
    absC = np.abs(C)
    dg = np.sqrt(np.diagonal(G, axis1=1, axis2=2))
    bound = 65 * 2.0 ** -24 * np.einsum("lik,ljk->lij", absC, absC) + 2.0 ** -23 * np.abs(G) \
        + slack * dg[:, :, None] * dg[:, None, :] + 1e-12
    err = np.abs(np.einsum("lik,ljk->lij", C, C) - G)
    assert np.all(err <= bound), f"C C^T - S S^T: worst x{(err / bound).max():.2f} of bound"


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
    Ct = factor_of(fr, sc.levels, text.shape[0] * text.shape[1])
    check_factor(Ct, sc.codebook)
    rb = rounded_reference(fr.coeff.cpu().numpy(), sc.codebook, text, 10.0, Ct)
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
    Ct = factor_of(fr, sc.levels, text.shape[0] * text.shape[1])
    check_factor(Ct, sc.codebook)
    rb = rounded_reference(fr.coeff.cpu().numpy(), sc.codebook, text, 10.0, Ct)
    assert np.abs(rel - rb).max() <= 1e-4


def test_query_tc_at_scale_sampled():
    sc, cam, text = syn.at_scale()
    fr, rel = run_query(sc, cam, text)
    rng = np.random.default_rng(4)
    pix = rng.integers(0, cam.num_pixels, 4000)
    W = fr.coeff.cpu().numpy()[:, pix]
    rb = rounded_reference(W, sc.codebook, text, 10.0, factor_of(fr, sc.levels, text.shape[0] * text.shape[1]))
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
    rb = rounded_reference(fr.coeff.cpu().numpy(), sc.codebook, text, 10.0, factor_of(fr, 2, Q * (1 + n_neg)))
    assert np.abs(rel - rb).max() <= 1e-4


def test_factor_of_a_rank_deficient_codebook():
    """A codebook with a repeated row, a zero row and a row in the span of two others (a singular
    S S^T): the factor drops those pivots and still reproduces S S^T within 3e-3 of sqrt(G_ii G_jj),
    and the relevancy stays within the BF16 bound of the oracle's."""
    sc, cam = syn.tiny()
    cb = sc.codebook.copy()
    cb[0, 5] = cb[0, 3]
    cb[0, 7] = 0.0
    cb[0, 9] = syn.unit_rows(cb[0, 2] + cb[0, 4])
    sc.codebook = cb
    text = syn.text_queries(syn.SEED + 2, 2, 4)
    fr, rel = run_query(sc, cam, text)
    Ct = factor_of(fr, 1, text.shape[0] * text.shape[1])
    for j in (5, 7, 9):
        assert Ct[0, j, j] == 0.0
    check_factor(Ct, sc.codebook, slack=3e-3)
    ref = O.render(sc, cam)
    ro = O.relevancy(O.decode(ref.blend.out, sc.codebook), text, 10.0)
    ok = ref.blend.margin > KNIFE_EDGE
    assert np.abs(rel[:, :, ok] - ro[:, :, ok]).max() <= 1e-2


@pytest.mark.parametrize("compute", [L.LSV2_BF16, L.LSV2_F32])
def test_prepared_query_equals_query(compute):
    """lsv2_query_prepare on a second stream, then lsv2_query_prepared on the first after an event:
    bit-equal to lsv2_query (BF16 map for the tensor-core path, FP32 map for both)."""
    sc = syn.make_scene(3000, 3, seed=11, mean_kind="uniform", mean_param=1.0, log_scale_mu=-3.2, log_scale_sigma=0.4)
    cam = syn.orbit_camera(141, 99, 4.0)
    text = torch.as_tensor(syn.text_queries(syn.SEED + 2, 16, 4), device="cuda")
    fr = Frame(DeviceScene.from_numpy(sc), cam)
    fr.render()
    fr.splat_bf16()
    maps = [False, True] if compute == L.LSV2_BF16 else [False]
    for from_bf16 in maps:
        ref = torch.empty((16, 3, fr.P), device="cuda")
        got = torch.full_like(ref, -7.0)
        fr.query(text, ref, compute=compute, from_bf16=from_bf16)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        fr.query_prepare(text, compute=compute, stream=side)
        done = torch.cuda.Event()
        done.record(side)
        torch.cuda.current_stream().wait_event(done)
        fr.query(text, got, compute=compute, from_bf16=from_bf16, prepared=True)
        fr.check()
        assert torch.equal(got, ref)
