"""The paper's speed ablation inputs (Table 9 and the K ablation): the dense-coefficient blend
(every Gaussian updates all 64 coefficients of every level, "Sparse, not Efficient") must equal
the sparse splatting bit for bit (blending zeros does not alter the result, Sec. 3.4), and the
three-level splat at K = 2, 6, 8 must match the FP64 oracle."""
import numpy as np
import pytest

import lsv2_synth as syn
from oracle import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_07136_b300 import _lib as L  # noqa: E402
from paper_2507_07136_b300.pipeline import DeviceScene, Frame  # noqa: E402
from test_gpu_forward import check_blend, gpu_frame  # noqa: E402


def sparse_and_dense(sc, cam):
    ds = DeviceScene.from_numpy(sc)
    fr = Frame(ds, cam)
    fr.render()
    fr.check()
    W, T, n = fr.coeff.clone(), fr.final_T.clone(), fr.n_last.clone()
    fr.coeff.fill_(float("nan"))
    fr.splat_dense()
    fr.check()
    return (W, T, n), (fr.coeff, fr.final_T, fr.n_last)


@pytest.mark.parametrize("levels", [1, 3])
def test_dense_blend_equals_sparse_splat(levels):
    sc = syn.make_scene(3000, levels, seed=11 + levels, mean_kind="uniform", mean_param=1.0, log_scale_mu=-3.2,
                        log_scale_sigma=0.4)
    cam = syn.orbit_camera(141, 99, 4.0)
    (W, T, n), (Wd, Td, nd) = sparse_and_dense(sc, cam)
    assert torch.equal(W, Wd) and torch.equal(T, Td) and torch.equal(n, nd)


def test_dense_blend_with_duplicate_indices():
    """Repeated indices within a level: the dense vector sums them in pair order, as the sparse
    record merges them."""
    sc = syn.make_scene(2000, 3, seed=5, mean_kind="uniform", mean_param=1.0, log_scale_mu=-3.2, log_scale_sigma=0.4)
    sc.idx[::3, :, 1] = sc.idx[::3, :, 0]
    sc.idx[::5, :, 3] = sc.idx[::5, :, 2]
    (W, T, n), (Wd, Td, nd) = sparse_and_dense(sc, syn.orbit_camera(96, 80, 4.0))
    assert torch.equal(W, Wd) and torch.equal(T, Td) and torch.equal(n, nd)


def test_dense_blend_at_scale():
    sc, cam, _ = syn.at_scale()
    (W, T, n), (Wd, Td, nd) = sparse_and_dense(sc, cam)
    assert torch.equal(W, Wd) and torch.equal(T, Td) and torch.equal(n, nd)


@pytest.mark.parametrize("K", [2, 6, 8])
def test_three_level_k_sweep_vs_oracle(K):
    sc = syn.make_scene(2500, 3, seed=20 + K, mean_kind="uniform", mean_param=1.0, log_scale_mu=-3.1,
                        log_scale_sigma=0.4, K=K)
    cam = syn.orbit_camera(112, 88, 4.0)
    ref = O.render(sc, cam)
    _, fr = gpu_frame(sc, cam)
    px, py = O.all_pixels(cam)
    check_blend(fr, ref.blend, px, py, cam)


def test_dense_unsupported_configurations():
    sc = syn.make_scene(500, 2, seed=3, mean_kind="uniform", mean_param=1.0, log_scale_mu=-3.2, log_scale_sigma=0.4)
    assert L.lsv2_splat_dense_workspace_bytes(500, 2) == 0
    fr = Frame(DeviceScene.from_numpy(sc), syn.orbit_camera(64, 48, 4.0))
    fr.render()
    with pytest.raises(L.LSV2Error):
        fr.splat_dense()


@pytest.mark.parametrize("Lc", [32, 128])
def test_three_level_codebook_size_sweep_vs_oracle(Lc):
    """The splat with codebooks of 32 and 128 entries (three levels, K = 4), against the FP64 oracle
    (coefficient map [levels][P][L]), and the BF16 map equal to the FP32 map rounded."""
    sc = syn.make_scene(2500, 3, seed=40 + Lc, mean_kind="uniform", mean_param=1.0, log_scale_mu=-3.1,
                        log_scale_sigma=0.4, L=Lc)
    cam = syn.orbit_camera(112, 88, 4.0)
    ref = O.render(sc, cam)
    _, fr = gpu_frame(sc, cam)
    assert fr.coeff.shape[2] == Lc
    px, py = O.all_pixels(cam)
    check_blend(fr, ref.blend, px, py, cam)
    fr.splat_bf16()
    fr.check()
    assert torch.equal(fr.coeff.to(torch.bfloat16).view(torch.int16), fr.coeff16.view(torch.int16))


def test_codebook_size_sweep_at_scale_sampled():
    """The at-scale frame (300k Gaussians, three levels) with a 128-entry codebook: the map on
    sampled pixels against the oracle."""
    sc = syn.make_scene(300_000, 3, L=128)
    cam = syn.orbit_camera(1440, 1080, 6.0)
    _, fr = gpu_frame(sc, cam)
    rng = np.random.default_rng(3)
    px = rng.integers(0, cam.width, 3000).astype(np.int32)
    py = rng.integers(0, cam.height, 3000).astype(np.int32)
    ref = O.render(sc, cam, px=px, py=py)
    check_blend(fr, ref.blend, px, py, cam)
