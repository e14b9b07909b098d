"""lsv2_render_fused: splat + decode + relevancy in one kernel.

The fused kernel runs the same splat and hands the same BF16 operands to the same MMA sequence
as lsv2_splat_coeffs -> lsv2_decode (BF16 out) -> lsv2_query (BF16 compute), so its F, relevancy,
final T and last-contributor index must equal that path's bit for bit; the relevancy is also
checked against the FP64 oracle at the BF16 bound (1e-2)."""
import numpy as np
import pytest

import lsv2_synth as syn
from oracle import oracle as O

from gpu_helpers import KNIFE_EDGE

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_07136_b300 import _lib as L  # noqa: E402
from paper_2507_07136_b300.pipeline import DeviceScene, Frame  # noqa: E402


def small():
    sc = syn.make_scene(4000, 3, seed=31, mean_kind="uniform", mean_param=1.0, log_scale_mu=-3.2, log_scale_sigma=0.4)
    return sc, syn.orbit_camera(157, 113, 4.0)


def split_and_fused(sc, cam, text, decode=True):
    ds = DeviceScene.from_numpy(sc)
    a = Frame(ds, cam)
    a.render()
    Fa = Fb = None
    if decode:
        Fa = torch.empty((ds.levels, cam.num_pixels, ds.D), dtype=torch.bfloat16, device="cuda")
        a.decode(Fa)
    ra = rb = None
    td = None
    if text is not None:
        td = torch.as_tensor(text, device="cuda")
        ra = torch.empty((text.shape[0], ds.levels, cam.num_pixels), dtype=torch.float32, device="cuda")
        a.query(td, ra, compute=L.LSV2_BF16)
    a.check()
    b = Frame(ds, cam, capacity=a.capacity)
    b.project()
    b.bin_sort()
    if decode:
        Fb = torch.full_like(Fa, float("nan"))
    if text is not None:
        rb = torch.full_like(ra, float("nan"))
    b.render_fused(Fb, td, rb)
    b.check()
    assert torch.equal(a.final_T, b.final_T) and torch.equal(a.n_last, b.n_last)
    return a, (Fa, Fb), (ra, rb)


def test_fused_equals_split_path_bitwise():
    sc, cam = small()
    text = syn.text_queries(syn.SEED + 2, 1, 4)
    _, (Fa, Fb), (ra, rb) = split_and_fused(sc, cam, text)
    assert torch.equal(Fa.view(torch.int16), Fb.view(torch.int16)), "F differs from splat -> decode"
    assert torch.equal(ra, rb), "relevancy differs from splat -> query"


@pytest.mark.parametrize("Q,n_neg", [(1, 4), (8, 4), (13, 2), (16, 3)])
def test_fused_query_counts(Q, n_neg):
    sc, cam = small()
    text = syn.text_queries(syn.SEED + 2 + Q, Q, n_neg)
    _, _, (ra, rb) = split_and_fused(sc, cam, text, decode=False)
    assert torch.equal(ra, rb)


def test_fused_bf16_relevancy_equals_split_path():
    """BF16 relevancy output (sigmoid through the hardware tanh on both paths), ragged frame."""
    sc, cam = small()
    text = syn.text_queries(syn.SEED + 7, 3, 4)
    ds = DeviceScene.from_numpy(sc)
    a = Frame(ds, cam)
    a.render()
    td = torch.as_tensor(text, device="cuda")
    ra = torch.empty((3, ds.levels, cam.num_pixels), dtype=torch.bfloat16, device="cuda")
    a.query(td, ra, compute=L.LSV2_BF16)
    b = Frame(ds, cam, capacity=a.capacity)
    b.project()
    b.bin_sort()
    rb = torch.full_like(ra, float("nan"))
    b.render_fused(None, td, rb)
    b.check()
    assert torch.equal(ra.view(torch.int16), rb.view(torch.int16))


def test_fused_decode_only_and_against_oracle():
    sc, cam = small()
    _, (Fa, Fb), _ = split_and_fused(sc, cam, None)
    assert torch.equal(Fa.view(torch.int16), Fb.view(torch.int16))
    text = syn.text_queries(syn.SEED + 2, 2, 4)
    a, _, (ra, rb) = split_and_fused(sc, cam, text, decode=False)
    ref = O.render(sc, cam)
    ro = O.relevancy(O.decode(ref.blend.out, sc.codebook), text, 10.0)
    ok = ref.blend.margin > KNIFE_EDGE
    assert np.abs(rb.cpu().numpy()[:, :, ok] - ro[:, :, ok]).max() <= 1e-2


def test_fused_at_scale_equals_split_path():
    """The 300k-Gaussian, 3-level, 1440x1080 frame: F (4.8 GB) and the relevancy, bit for bit."""
    sc, cam, text = syn.at_scale()
    _, (Fa, Fb), (ra, rb) = split_and_fused(sc, cam, text)
    assert torch.equal(Fa.view(torch.int16), Fb.view(torch.int16))
    assert torch.equal(ra, rb)


def test_fused_rejects_unsupported():
    sc, cam = small()
    ds = DeviceScene.from_numpy(sc)
    assert L.lsv2_render_fused_workspace_bytes(ds.n, 3, 4, 500, 1, 4) == 0     # D not a multiple of 128
    assert L.lsv2_render_fused_workspace_bytes(ds.n, 2, 4, 512, 1, 4) == 0     # two levels
    assert L.lsv2_render_fused_workspace_bytes(ds.n, 3, 4, 512, 64, 4) == 0    # 64 + 5 * 64 > 128
    assert L.lsv2_render_fused_workspace_bytes(ds.n, 3, 4, 512, 9, 4) == 0     # 64 + 5 * 16 > 128
    fr = Frame(ds, cam.with_tile(8, 8))
    fr.project()
    fr.bin_sort()
    F = torch.empty((3, cam.num_pixels, ds.D), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(L.LSV2Error):
        fr.render_fused(F)
