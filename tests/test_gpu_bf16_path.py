"""The BF16 coefficient map (lsv2_splat_coeffs_bf16) feeding the tensor-core decode and relevancy:
the map is the FP32 blend rounded to nearest even, and both consumers round W to BF16 before their
products, so their results from it equal their results from the FP32 map bit for bit."""
import numpy as np
import pytest

import lsv2_synth as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_07136_b300 import _lib as L  # noqa: E402
from paper_2507_07136_b300.pipeline import DeviceScene, Frame  # noqa: E402


def both(sc, cam, text):
    ds = DeviceScene.from_numpy(sc)
    fr = Frame(ds, cam)
    fr.render()
    T, n = fr.final_T.clone(), fr.n_last.clone()
    fr.splat_bf16()
    fr.check()
    assert torch.equal(fr.coeff.to(torch.bfloat16).view(torch.int16), fr.coeff16.view(torch.int16))
    assert torch.equal(T, fr.final_T) and torch.equal(n, fr.n_last)
    F32w = torch.empty((ds.levels, fr.P, ds.D), dtype=torch.bfloat16, device="cuda")
    F16w = torch.full_like(F32w, float("nan"))
    fr.decode(F32w)
    fr.decode(F16w, from_bf16=True)
    td = torch.as_tensor(text, device="cuda")
    out = []
    for dt in (torch.float32, torch.bfloat16):
        ra = torch.empty((text.shape[0], ds.levels, fr.P), dtype=dt, device="cuda")
        rb = torch.full_like(ra, float("nan"))
        fr.query(td, ra, compute=L.LSV2_BF16)
        fr.query(td, rb, compute=L.LSV2_BF16, from_bf16=True)
        out.append((ra, rb))
    fr.check()
    assert torch.equal(F32w.view(torch.int16), F16w.view(torch.int16)), "decode from the BF16 map differs"
    for ra, rb in out:
        assert torch.equal(ra, rb), "relevancy from the BF16 map differs"
    return fr


def test_bf16_map_small_three_levels():
    sc = syn.make_scene(3000, 3, seed=11, mean_kind="uniform", mean_param=1.0, log_scale_mu=-3.2, log_scale_sigma=0.4)
    both(sc, syn.orbit_camera(141, 99, 4.0), syn.text_queries(syn.SEED + 2, 3, 4))


def test_texts_of_any_norm():
    """Text vectors scaled by 0.3 .. 3 (the cosine does not depend on the norms): the relevancy from
    the FP32 map, from the BF16 map and from the fused kernel agree bit for bit (all three fold
    1/|t| into the text rows the same way), and match the FP64 oracle's within the BF16 path's
    1e-2."""
    from oracle import oracle as O

    sc = syn.make_scene(3000, 3, seed=11, mean_kind="uniform", mean_param=1.0, log_scale_mu=-3.2, log_scale_sigma=0.4)
    cam = syn.orbit_camera(141, 99, 4.0)
    rng = np.random.default_rng(4)
    text = (syn.text_queries(syn.SEED + 2, 3, 4) * rng.uniform(0.3, 3.0, (3, 5, 1))).astype(np.float32)
    fr = both(sc, cam, text)
    td = torch.as_tensor(text, device="cuda")
    ra = torch.empty((3, 3, fr.P), dtype=torch.bfloat16, device="cuda")
    fr.query(td, ra, compute=L.LSV2_BF16, from_bf16=True)
    fb = Frame(fr.scene, cam, capacity=fr.capacity)
    fb.project()
    fb.bin_sort()
    rb = torch.full_like(ra, float("nan"))
    fb.render_fused(None, td, rb)
    fb.check()
    assert torch.equal(ra.view(torch.int16), rb.view(torch.int16)), "fused relevancy differs"
    ref = O.render(sc, cam)
    ro = O.relevancy(O.decode(ref.blend.out, sc.codebook), text.astype(np.float64), 10.0)
    ok = ref.blend.margin > 1e-4
    assert np.abs(ra.float().cpu().numpy()[:, :, ok] - ro[:, :, ok]).max() <= 1e-2


def test_bf16_map_at_scale():
    sc, cam, text = syn.at_scale()
    both(sc, cam, text)


def test_f32_query_of_a_bf16_map_is_unsupported():
    sc = syn.make_scene(500, 1, seed=3, mean_kind="uniform", mean_param=1.0, log_scale_mu=-3.2, log_scale_sigma=0.4)
    fr = Frame(DeviceScene.from_numpy(sc), syn.orbit_camera(64, 48, 4.0))
    fr.render()
    fr.splat_bf16()
    text = torch.as_tensor(syn.text_queries(syn.SEED + 2, 1, 4), device="cuda")
    rel = torch.empty((1, 1, fr.P), dtype=torch.float32, device="cuda")
    with pytest.raises(L.LSV2Error) as e:
        fr.query(text, rel, compute=L.LSV2_F32, from_bf16=True)
    assert e.value.code == 2


@pytest.mark.parametrize("D", [128, 256, 384, 512])
@pytest.mark.parametrize("out_dtype", [torch.bfloat16, torch.float32])
@pytest.mark.parametrize("size", [(141, 99), (10, 7)])
def test_decode_from_bf16_map_widths(D, out_dtype, size):
    """Every supported width and both output types, on a ragged frame (141x99 = 13959 pixels) and on
    one smaller than a 128-pixel tile: the decode from the BF16 map equals the decode from the FP32
    map bit for bit, and both are the FP64 product of the BF16-rounded operands within 1e-5 of
    sum |W||S| (plus the output rounding for BF16 output)."""
    sc = syn.make_scene(3000, 3, seed=12, mean_kind="uniform", mean_param=1.0, log_scale_mu=-3.2,
                        log_scale_sigma=0.4, D=D)
    ds = DeviceScene.from_numpy(sc)
    fr = Frame(ds, syn.orbit_camera(size[0], size[1], 4.0))
    fr.render()
    fr.splat_bf16()
    cb = ds.codebook.to(torch.bfloat16)
    Fa = torch.full((ds.levels, fr.P, D), float("nan"), dtype=out_dtype, device="cuda")
    Fb = torch.full_like(Fa, float("nan"))
    fr.decode(Fa, codebook=cb)
    fr.decode(Fb, codebook=cb, from_bf16=True)
    fr.check()
    assert torch.equal(Fa.view(torch.int16 if out_dtype == torch.bfloat16 else torch.int32),
                       Fb.view(torch.int16 if out_dtype == torch.bfloat16 else torch.int32))
    Wb = fr.coeff16.double().cpu().numpy()
    Sb = cb.double().cpu().numpy()
    ref = np.matmul(Wb, Sb)
    bound = 1e-5 * np.matmul(np.abs(Wb), np.abs(Sb)) + 1e-9
    if out_dtype == torch.bfloat16:
        bound = bound + 2.0 ** -8 * np.abs(ref)
    assert np.all(np.abs(Fb.double().cpu().numpy() - ref) <= bound)


@pytest.mark.parametrize("Q,n_neg", [(1, 1), (1, 4), (5, 4), (8, 1), (9, 4), (17, 3), (32, 4), (40, 4), (64, 4)])
@pytest.mark.parametrize("out_dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("size", [(141, 99), (10, 7)])
def test_query_from_bf16_map_counts(Q, n_neg, out_dtype, size):
    """Relevancy from the BF16 map (TMA-fed pipelined kernel, 3 or 2 TMEM accumulators by column
    count; 40 and 64 queries run as groups of 32) equals the relevancy from the FP32 map (rounded to
    BF16 in the kernel) bit for bit:
    query counts ragged against the 8-query chunks, both output types, a ragged frame and one
    smaller than a 128-pixel tile (its rows past a level's end belong to the next level)."""
    sc = syn.make_scene(3000, 3, seed=13, mean_kind="uniform", mean_param=1.0, log_scale_mu=-3.2, log_scale_sigma=0.4)
    fr = Frame(DeviceScene.from_numpy(sc), syn.orbit_camera(size[0], size[1], 4.0))
    fr.render()
    fr.splat_bf16()
    text = torch.as_tensor(syn.text_queries(syn.SEED + 21, Q, n_neg), device="cuda")
    ra = torch.full((Q, 3, fr.P), float("nan"), dtype=out_dtype, device="cuda")
    rb = torch.full_like(ra, float("nan"))
    fr.query(text, ra, compute=L.LSV2_BF16)
    fr.query(text, rb, compute=L.LSV2_BF16, from_bf16=True)
    fr.check()
    assert not torch.isnan(rb).any()
    assert torch.equal(ra, rb)
