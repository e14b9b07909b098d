"""lsv2_sparsify / lsv2_sparsify_backward (Sec. 3.3: softmax over the L-dim parameter, top K kept
and renormalised) against the FP64 oracle: the kept indices bit for bit (both sides select on the
same FP32 logits, lower index first among equal ones), the weights within 1e-6 relative (an FP32
softmax over at most 8 kept logits), the gradient within (K + 1) 1e-6 max|dw| per row (the FP32
rounding of its sum, whose difference with dw_k can cancel)."""
import numpy as np
import pytest

import lsv2_synth as syn
from oracle import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_07136_b300 import _lib as L  # noqa: E402
from paper_2507_07136_b300.pipeline import _ptr  # noqa: E402


def gpu_sparsify(z, K):
    zt = torch.as_tensor(np.ascontiguousarray(z), device="cuda")
    rows, Lz = z.shape
    idx = torch.full((rows, K), 255, dtype=torch.uint8, device="cuda")
    w = torch.full((rows, K), float("nan"), device="cuda")
    L.lsv2_sparsify(rows, Lz, K, _ptr(zt), _ptr(idx), _ptr(w), None)
    torch.cuda.synchronize()
    return idx, w


def gpu_backward(idx, w, dw, Lz):
    rows, K = w.shape
    dz = torch.full((rows, Lz), float("nan"), device="cuda")
    dwt = torch.as_tensor(np.ascontiguousarray(dw, np.float32), device="cuda")
    L.lsv2_sparsify_backward(rows, Lz, K, _ptr(idx), _ptr(w), _ptr(dwt), _ptr(dz), None)
    torch.cuda.synchronize()
    return dz.cpu().numpy()


def logits(rng, rows, Lz):
    z = rng.normal(0, 2, (rows, Lz)).astype(np.float32)
    z[::7] = np.round(z[::7] * 4) / 4        # rows with many equal logits
    z[5] = 0.0                               # every logit equal
    z[11, : Lz // 2] = 1.5                   # a tie across the boundary of the top K
    return z


def check_rows(z, K, idx, w, dw, dz):
    oi, ow = O.sparsify(z, K)
    assert np.array_equal(idx, oi)
    np.testing.assert_allclose(w, ow, rtol=1e-6, atol=1e-7)
    # the gradient w_k (dw_k - sum_m w_m dw_m) in FP32: the sum carries an absolute error of about
    # K eps max|dw| (the weights sum to one) and the difference can cancel, so the bound is
    # absolute, (K + 1) 1e-6 max_k |dw_k| per row (on the kernel's own w, so only the arithmetic differs)
    ref = O.sparsify_backward(oi, w.astype(np.float64), dw, z.shape[1])
    bound = (K + 1) * 1e-6 * np.abs(dw).max(axis=1, keepdims=True) + 1e-12
    assert np.all(np.abs(dz - ref) <= bound)


@pytest.mark.parametrize("Lz", [16, 32, 64, 128, 256])
@pytest.mark.parametrize("K", [1, 2, 4, 8])
def test_sparsify_matches_oracle(Lz, K):
    """Ragged row counts (not multiples of the 128- or 32-row blocks), ties, every supported shape."""
    if K > Lz:
        pytest.skip("K > L")
    rng = np.random.default_rng(Lz * 10 + K)
    rows = 1000 + 37
    z = logits(rng, rows, Lz)
    idx, w = gpu_sparsify(z, K)
    dw = rng.normal(0, 1, (rows, K)).astype(np.float32)
    dz = gpu_backward(idx, w, dw, Lz)
    check_rows(z, K, idx.cpu().numpy(), w.cpu().numpy(), dw, dz)


def test_sparsify_at_scale_sampled():
    """300,000 Gaussians x 3 levels = 900,000 rows of 64 logits, K = 4: 20,000 sampled rows."""
    rng = np.random.default_rng(9)
    rows, Lz, K = 900_000, 64, 4
    z = rng.normal(0, 2, (rows, Lz)).astype(np.float32)
    idx, w = gpu_sparsify(z, K)
    dw = rng.normal(0, 1, (rows, K)).astype(np.float32)
    dz = gpu_backward(idx, w, dw, Lz)
    pick = np.sort(rng.choice(rows, 20_000, replace=False))
    check_rows(z[pick], K, idx.cpu().numpy()[pick], w.cpu().numpy()[pick], dw[pick], dz[pick])


@pytest.mark.parametrize("Lz", [16, 64, 256])
def test_sparsify_unaligned_logits(Lz):
    """Logits that start one float into their buffer (4-byte, not 16-byte aligned) take the
    kernel's scalar loads; a ragged row count leaves a partial warp at the end."""
    rng = np.random.default_rng(Lz + 3)
    rows, K = 517, 4
    z = logits(rng, rows, Lz)
    buf = torch.empty(rows * Lz + 4, device="cuda")
    buf[1:1 + rows * Lz] = torch.as_tensor(z.ravel(), device="cuda")
    zt = buf[1:1 + rows * Lz]
    assert zt.data_ptr() % 16 != 0
    idx = torch.full((rows, K), 255, dtype=torch.uint8, device="cuda")
    w = torch.full((rows, K), float("nan"), device="cuda")
    L.lsv2_sparsify(rows, Lz, K, _ptr(zt), _ptr(idx), _ptr(w), None)
    torch.cuda.synchronize()
    oi, ow = O.sparsify(z, K)
    assert np.array_equal(idx.cpu().numpy(), oi)
    np.testing.assert_allclose(w.cpu().numpy(), ow, rtol=1e-6, atol=1e-7)


def test_sparsify_edges():
    z = torch.zeros((1, 64), device="cuda")
    idx = torch.empty((1, 4), dtype=torch.uint8, device="cuda")
    w = torch.empty((1, 4), device="cuda")
    L.lsv2_sparsify(0, 64, 4, _ptr(z), _ptr(idx), _ptr(w), None)          # no rows: nothing to do
    for Lz, K in [(48, 4), (64, 3), (16, 32)]:
        with pytest.raises(L.LSV2Error) as e:
            L.lsv2_sparsify(1, Lz, K, _ptr(z), _ptr(idx), _ptr(w), None)
        assert e.value.code == 2


def test_sparsify_feeds_the_render_and_its_gradient_chains():
    """logits -> sparsify -> render_l1 on the tiny scene: the render consumes the kernel's (idx, w)
    directly, and autograd's dLoss/dlogits equals the oracle's sparsify gradient of the render's
    dLoss/dw."""
    from paper_2507_07136_b300.autograd import render_l1, sparsify
    sc, cam = syn.tiny()
    rng = np.random.default_rng(12)
    z = torch.as_tensor(rng.normal(0, 2, (sc.means.shape[0], 1, 64)).astype(np.float32), device="cuda").requires_grad_()
    f = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    target = f(syn.l1_target(cam, levels=1))
    w, idx = sparsify(z, 4)
    w.retain_grad()
    loss = render_l1(f(sc.means), f(np.log(sc.scales)), f(sc.quats),
                     f(np.log(sc.opacity / (1 - sc.opacity))), w, f(sc.codebook), idx, cam, target)
    loss.backward()
    oi, ow = O.sparsify(z.detach().cpu().numpy(), 4)
    assert np.array_equal(idx.cpu().numpy(), oi)
    gw = w.grad.cpu().numpy().astype(np.float64)
    ref = O.sparsify_backward(oi, w.detach().cpu().numpy().astype(np.float64), gw, 64)
    got = z.grad.cpu().numpy()
    assert np.all(np.abs(got - ref) <= 5e-6 * np.abs(gw).max(axis=-1, keepdims=True) + 1e-15)
    assert np.abs(got).max() > 0
