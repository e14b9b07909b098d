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
