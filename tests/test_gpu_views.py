"""lsv2_query_views: many views and queries in one call (project, bin, persistent splat, tensor-
core relevancy), eager and as a CUDA graph.

The batch must equal V separate single-view pipelines exactly (the same per-tile code, the same
ordered lists), and the FP64 oracle within the BF16 relevancy bound (1e-2)."""
import numpy as np
import pytest

import lsv2_synth as syn
from oracle import oracle as O

from gpu_helpers import KNIFE_EDGE

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_07136_b300 import _lib as L  # noqa: E402
from paper_2507_07136_b300.pipeline import DeviceScene, Frame  # noqa: E402
from paper_2507_07136_b300.views import ViewsBatch, autotune  # noqa: E402

RES = [(160, 120), (141, 99), (64, 48), (97, 131)]


def small_batch(tile=(16, 16)):
    sc = syn.make_scene(4000, 3, seed=31, mean_kind="uniform", mean_param=1.0, log_scale_mu=-3.2,
                        log_scale_sigma=0.4)
    cams = [syn.orbit_camera(w, h, 4.0, azimuth_deg=40.0 * k, tile=tile) for k, (w, h) in enumerate(RES)]
    text = syn.text_queries(syn.SEED + 2, 3, 4)
    return sc, cams, text


def single_view_rel(ds, cam, text):
    fr = Frame(ds, cam)
    fr.render()
    rel = torch.empty((text.shape[0], ds.levels, cam.num_pixels), dtype=torch.bfloat16, device="cuda")
    fr.query(torch.as_tensor(text, device="cuda"), rel, compute=L.LSV2_BF16)
    fr.check()
    return rel


@pytest.mark.parametrize("batch", [0, 16])
def test_views_equal_sequential_single_views(batch):
    sc, cams, text = small_batch()
    ds = DeviceScene.from_numpy(sc)
    vb = ViewsBatch(ds, cams, text.shape[0], text.shape[1] - 1, stage_batch=batch)
    vb.run(torch.as_tensor(text, device="cuda"))
    vb.check()
    for v, cam in enumerate(cams):
        ref = single_view_rel(ds, cam, text)
        assert torch.equal(vb.rel_view(v), ref), f"view {v}"


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 8)])
def test_views_against_oracle(tile):
    sc, cams, text = small_batch(tile)
    ds = DeviceScene.from_numpy(sc)
    vb = ViewsBatch(ds, cams, text.shape[0], text.shape[1] - 1, tile=tile)
    vb.run(torch.as_tensor(text, device="cuda"))
    vb.check()
    for v, cam in enumerate(cams):
        r = O.render(sc, cam)
        ro = O.relevancy(O.decode(r.blend.out, sc.codebook), text, 10.0)
        ok = r.blend.margin > KNIFE_EDGE
        got = vb.rel_view(v).float().cpu().numpy()
        assert np.abs(got[:, :, ok] - ro[:, :, ok]).max() <= 1e-2


def test_views_graph_replay_equals_eager():
    sc, cams, text = small_batch()
    ds = DeviceScene.from_numpy(sc)
    vb = ViewsBatch(ds, cams, text.shape[0], text.shape[1] - 1)
    t = torch.as_tensor(text, device="cuda")
    vb.run(t)
    vb.check()
    eager = vb.rel.clone()
    vb.rel.zero_()
    vb.capture(t)
    vb.rel.zero_()
    vb.replay()
    vb.check()
    assert torch.equal(vb.rel, eager)
    # a new set of queries through the same graph (inputs are read from the captured buffer)
    text2 = syn.text_queries(syn.SEED + 9, 3, 4)
    vb.text.copy_(torch.as_tensor(text2, device="cuda"))
    vb.replay()
    vb.check()
    ref = single_view_rel(ds, cams[1], text2)
    assert torch.equal(vb.rel_view(1), ref)


def test_views_capacity_overflow_reports_status():
    sc, cams, text = small_batch()
    ds = DeviceScene.from_numpy(sc)
    vb = ViewsBatch(ds, cams, text.shape[0], text.shape[1] - 1, capacity=500)
    vb.run(torch.as_tensor(text, device="cuda"))
    torch.cuda.synchronize()
    assert int(vb.status.item()) == 3


def test_autotuner_picks_a_valid_configuration(tmp_path):
    sc, cams, text = small_batch()
    ds = DeviceScene.from_numpy(sc)
    tile, batch = autotune(ds, cams, torch.as_tensor(text, device="cuda"), reps=2, cache=str(tmp_path / "t.json"))
    assert tuple(tile) in [(16, 16), (8, 8), (32, 8)] and batch in (16, 32)
    again = autotune(ds, cams, torch.as_tensor(text, device="cuda"), cache=str(tmp_path / "t.json"))
    assert tuple(again[0]) == tuple(tile) and again[1] == batch
