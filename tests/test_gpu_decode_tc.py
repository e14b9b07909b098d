"""Tensor-core (tcgen05, BF16 operands, FP32 accumulation) decode against FP64 references.

Two bars: against the FP64 product of the BF16-rounded operands (checks the kernel itself:
FP32 accumulation, 1e-5 of sum |W||S|, plus the output rounding when the output is BF16), and
against the FP64 oracle of the unrounded path (the BF16 variant's accuracy: 1e-2 absolute)."""
import numpy as np
import pytest

import lsv2_synth as syn
from oracle import oracle as O

from gpu_helpers import KNIFE_EDGE

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_07136_b300.pipeline import DeviceScene, Frame  # noqa: E402


def bf16_round(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def run(sc, cam, out_dtype, cb_dtype):
    ds = DeviceScene.from_numpy(sc)
    fr = Frame(ds, cam)
    fr.render()
    F = torch.empty((sc.levels, cam.num_pixels, sc.D), dtype=out_dtype, device="cuda")
    cb = ds.codebook.to(cb_dtype)
    fr.decode(F, codebook=cb, tensor_cores=True)
    fr.check()
    return fr, F.float().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("out_dtype", ["bf16", "f32"])
@pytest.mark.parametrize("cb_dtype", ["bf16", "f32"])
def test_decode_tc_kernel_exactness(out_dtype, cb_dtype):
    """Ragged pixel count (141x99 = 13959, not a multiple of the 128-row tile), three levels."""
    od = torch.bfloat16 if out_dtype == "bf16" else torch.float32
    cd = torch.bfloat16 if cb_dtype == "bf16" else torch.float32
    if od == torch.float32 and cd == torch.float32:
        pytest.skip("FP32 everywhere selects the CUDA-core path")
    sc = syn.make_scene(3000, 3, seed=11, mean_kind="uniform", mean_param=1.0, log_scale_mu=-3.2, log_scale_sigma=0.4)
    cam = syn.orbit_camera(141, 99, 4.0)
    fr, F = run(sc, cam, od, cd)
    Wb = bf16_round(fr.coeff.cpu().numpy())
    Sb = bf16_round(sc.codebook)
    ref = np.matmul(Wb, Sb)
    mag = np.matmul(np.abs(Wb), np.abs(Sb))
    bound = 1e-5 * mag + 1e-9
    if od == torch.bfloat16:
        bound = bound + 2.0 ** -8 * np.abs(ref)
    assert np.all(np.abs(F - ref) <= bound)


def test_decode_tc_bf16_accuracy_vs_fp64_oracle():
    """Precision variant: the tiny scene rendered at 1440x1080 (one level), BF16 decode against the
    FP64 oracle on sampled pixels: max abs error <= 1e-2."""
    sc, cam = syn.precision()
    fr, F = run(sc, cam, torch.bfloat16, torch.bfloat16)
    pr = O.project(cam, sc.means, sc.scales, sc.quats)
    ids, ranges = O.bin(cam, pr)
    rng = np.random.default_rng(1)
    k = 4000
    px = rng.integers(0, cam.width, k).astype(np.int32)
    py = rng.integers(0, cam.height, k).astype(np.int32)
    bl = O.blend(cam, pr, sc.opacity, ids, ranges, idx=sc.idx, w=sc.weights, px=px, py=py)
    Fo = O.decode(bl.out, sc.codebook)
    pix = py.astype(np.int64) * cam.width + px
    err = np.abs(F[:, pix] - Fo)
    assert err.max() <= 1e-2


def test_decode_tc_at_scale_sampled():
    sc, cam, _ = syn.at_scale()
    fr, F = run(sc, cam, torch.bfloat16, torch.bfloat16)
    rng = np.random.default_rng(2)
    pix = rng.integers(0, cam.num_pixels, 5000)
    Wb = bf16_round(fr.coeff.cpu().numpy()[:, pix])
    Sb = bf16_round(sc.codebook)
    ref = np.matmul(Wb, Sb)
    bound = 1e-5 * np.matmul(np.abs(Wb), np.abs(Sb)) + 2.0 ** -8 * np.abs(ref) + 1e-9
    assert np.all(np.abs(F[:, pix] - ref) <= bound)
