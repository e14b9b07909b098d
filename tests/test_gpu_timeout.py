"""Failure detection on the device: a bounded wait that runs out.

lsv2_set_wait_limit_ns(0) makes every wait of the pipelined kernels on another warp's progress
give up unless its phase is complete at the first (non-blocking) check, which drives the expiry
path on purpose: the kernel
records LSV2_ERR_TIMEOUT in the status word, lets the copies and MMAs it issued complete, frees
its tensor memory and returns (no hang, no trap, the context stays usable).  After the default
limit is restored, the next call on the same buffers gives the correct result.  No wait is left
waiting on something that never happens: the limit only shortens waits on work that is in
flight anyway.
"""
import numpy as np
import pytest

import lsv2_synth as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_07136_b300 import _lib as L  # noqa: E402
from paper_2507_07136_b300.pipeline import DeviceScene, Frame, _ptr, _stream  # noqa: E402
from paper_2507_07136_b300.views import ViewsBatch  # noqa: E402

DEFAULT = 1_000_000_000


@pytest.fixture(autouse=True)
def default_limit_after():
    L.lsv2_set_wait_limit_ns(DEFAULT)
    yield
    L.lsv2_set_wait_limit_ns(DEFAULT)


def expire_then_recover(fr, run, outputs, inexact=()):
    """run() once with the default limit (the reference), once with limit 0 (must report
    LSV2_ERR_TIMEOUT and return), once more with the default limit on the same buffers (must
    equal the reference bit for bit, except the outputs listed in `inexact`).

    Those are sums of FP32 atomic additions in no fixed order (the decode adjoint's loss: one per
    epilogue warp, eight per persistent CTA, one CTA per SM): each addition rounds to within 2^-24
    of its running sum, so two orders of n partial sums differ by at most n 2^-24 sum|partial|.  For a sum of positive partials (a loss) that is n 2^-24 of the value;
    where partials of either sign cancel, the bound is taken as 1e-4 of the largest entry, 30x the
    largest difference seen between runs and far below what a lost or stale partial would leave
    (about 1/n of the magnitude)."""
    fr.status.zero_()
    run()
    fr.check()
    ref = [o.clone() for o in outputs]
    for o in outputs:
        o.fill_(-7)
    L.lsv2_set_wait_limit_ns(0)
    fr.status.zero_()
    run()
    torch.cuda.synchronize()          # the kernels returned
    assert int(fr.status.item()) == L.LSV2_ERR_TIMEOUT
    L.lsv2_set_wait_limit_ns(DEFAULT)
    for o in outputs:
        o.fill_(-7)
    fr.status.zero_()
    run()
    fr.check()
    for n, (o, r) in enumerate(zip(outputs, ref)):
        if n in inexact:
            if bool((r >= 0).all()):
                n = 8 * torch.cuda.get_device_properties(0).multi_processor_count
                assert torch.allclose(o, r, rtol=n * 2.0 ** -24, atol=0.0)
            else:
                assert float((o - r).abs().max()) <= 1e-4 * float(r.abs().max())
        else:
            assert torch.equal(o, r)


def dense_scene():
    """20,000 Gaussians in the tiny scene's volume: hundreds of records per tile, so a splat's
    producer reaches a stage its consumers still hold (the wait that a limit of 0 makes expire)."""
    return syn.make_scene(20000, 3, mean_kind="uniform", mean_param=1.0, log_scale_mu=-3.0, log_scale_sigma=0.3)


def three_level_frame():
    sc = dense_scene()
    _, cam = syn.tiny()
    fr = Frame(DeviceScene.from_numpy(sc), cam)
    fr.project()
    fr.bin_sort()
    fr.check()
    return fr


@pytest.mark.parametrize("tile", [(16, 16), (8, 8)])
def test_splat_wait_expires_and_recovers(tile):
    sc = dense_scene()
    _, cam = syn.tiny()
    fr = Frame(DeviceScene.from_numpy(sc), cam.with_tile(*tile))
    fr.project()
    fr.bin_sort()
    fr.check()
    expire_then_recover(fr, fr.splat, [fr.coeff, fr.final_T, fr.n_last])


def test_splat_bf16_wait_expires_and_recovers():
    fr = three_level_frame()
    fr.splat_bf16()
    fr.check()
    expire_then_recover(fr, fr.splat_bf16, [fr.coeff16, fr.final_T, fr.n_last])


def test_fused_render_wait_expires_and_recovers():
    fr = three_level_frame()
    text = torch.as_tensor(syn.text_queries(syn.SEED + 2, 1, 4), device="cuda")
    F = torch.empty((3, fr.P, 512), dtype=torch.bfloat16, device="cuda")
    rel = torch.empty((1, 3, fr.P), dtype=torch.float32, device="cuda")
    expire_then_recover(fr, lambda: fr.render_fused(F, text, rel), [F, rel, fr.final_T, fr.n_last])


@pytest.mark.parametrize("from_bf16", [True, False])
def test_decode_tc_wait_expires_and_recovers(from_bf16):
    """BF16 map: W arrives by TMA tensor loads; FP32 map: through registers."""
    fr = three_level_frame()
    fr.splat()
    fr.splat_bf16()
    fr.check()
    cb16 = fr.scene.codebook.to(torch.bfloat16)
    F = torch.empty((3, fr.P, 512), dtype=torch.bfloat16, device="cuda")
    expire_then_recover(fr, lambda: fr.decode(F, codebook=cb16, from_bf16=from_bf16), [F])


@pytest.mark.parametrize("Q", [3, 16])
@pytest.mark.parametrize("from_bf16", [True, False])
def test_query_tc_wait_expires_and_recovers(from_bf16, Q):
    """BF16 map: the pipelined relevancy kernel (3 queries: three accumulators, one epilogue
    warpgroup each; 16 queries: two accumulators, two warpgroups each meeting at a named barrier
    per tile); FP32 map: the converting one."""
    fr = three_level_frame()
    fr.splat()
    fr.splat_bf16()
    fr.check()
    text = torch.as_tensor(syn.text_queries(syn.SEED + 2, Q, 4), device="cuda")
    rel = torch.empty((Q, 3, fr.P), dtype=torch.bfloat16, device="cuda")
    expire_then_recover(fr, lambda: fr.query(text, rel, compute=L.LSV2_BF16, from_bf16=from_bf16), [rel])


def test_views_wait_expires_and_recovers():
    sc = dense_scene()
    cams = [syn.orbit_camera(w, h, 4.0, azimuth_deg=40.0 * k) for k, (w, h) in enumerate([(160, 120), (97, 131)])]
    text = torch.as_tensor(syn.text_queries(syn.SEED + 2, 3, 4), device="cuda")
    ds = DeviceScene.from_numpy(sc)
    vb = ViewsBatch(ds, cams, 3, 4)
    expire_then_recover(vb, lambda: vb.run(text), [vb.rel])
    assert np.isfinite(vb.rel.float().cpu().numpy()).all()


def test_l1_decode_backward_wait_expires_and_recovers():
    """The tensor-core decode adjoint (TMA ring, MMA warp, epilogue warps)."""
    fr = three_level_frame()
    fr.splat()
    fr.check()
    target = torch.as_tensor(syn.l1_target(fr.cam, levels=3), device="cuda")
    loss = torch.zeros(1, device="cuda")
    dW = torch.empty_like(fr.coeff)
    dS = torch.zeros_like(fr.scene.codebook)

    def run():
        loss.zero_()
        dS.zero_()
        L.lsv2_l1_decode_backward(3, fr.P, 64, 512, _ptr(fr.coeff), _ptr(fr.scene.codebook), _ptr(target), _ptr(loss),
                                  _ptr(dW), _ptr(dS), _ptr(fr.status), _stream(None))

    expire_then_recover(fr, run, [loss, dW, dS], inexact=(0, 2))


def test_mlp_fused_wait_expires_and_recovers():
    """The fused tensor-core MLP decoder (weight ring, MMA warp, two slots of epilogue warps)."""
    from paper_2507_07136_b300.decoder_path import LATENT_CHANNELS, Decoder

    dec = Decoder(syn.decoder_mlp())
    rows = 148 * 128 * 2 + 77
    rng = np.random.default_rng(26)
    x = torch.zeros((rows, LATENT_CHANNELS), device="cuda")
    x[:, :3] = torch.as_tensor(rng.standard_normal((rows, 3)), dtype=torch.float32, device="cuda")
    y = torch.empty((rows, dec.out_width), dtype=torch.bfloat16, device="cuda")
    ws = torch.empty(dec.workspace_bytes(rows, L.LSV2_F32, L.LSV2_MLP_FUSED), dtype=torch.uint8, device="cuda")

    class Holder:
        status = torch.zeros(1, dtype=torch.int32, device="cuda")

        def check(self):
            torch.cuda.synchronize()
            assert int(self.status.item()) == 0

    h = Holder()
    expire_then_recover(h, lambda: dec(x, y, ws, L.LSV2_MLP_FUSED, None, h.status), [y])
