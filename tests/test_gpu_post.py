"""lsv2_postprocess (appendix "Evaluation Details") against the FP64 oracle on the same seeded
relevancy maps: smoothed maps element by element (FP32 box sums: 1e-5 relative + 1e-6), the
selected level and point where the decision is not a near-tie (otherwise: the GPU's choice
must be optimal to within the tolerance), and the mask bit-exact except for knife-edge pixels
whose normalised value lies within 1e-4 of the threshold."""
import numpy as np
import pytest

import lsv2_synth as syn
from oracle import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_07136_b300 import _lib as L  # noqa: E402
from paper_2507_07136_b300.pipeline import postprocess  # noqa: E402

RTOL, ATOL, TIE, KNIFE = 1e-5, 1e-6, 2e-5, 1e-4


def _level_crit(sm, mode, thr):
    """Per-level criterion from the oracle's smoothed maps [levels, P] (for near-tie checks)."""
    out = []
    for s in sm:
        if mode == 0:
            out.append(s.max())
        else:
            mx, mn = s.max(), s.min()
            nrm = (s - mn) / (mx - mn) if mx > mn else np.zeros_like(s)
            m = nrm > thr
            out.append(s[m].mean() if m.any() else -np.inf)
    return np.array(out)


def run_and_compare(rel_np, H, W, k, mode, thr, dtype=torch.float32):
    Q, levels, P = rel_np.shape
    rel = torch.as_tensor(rel_np, device="cuda").to(dtype).contiguous()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    got = postprocess(rel, H, W, k=k, mode=mode, threshold=thr, dev_status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ref = O.postprocess(rel.float().cpu().numpy().astype(np.float64), H, W, k, mode, thr)
    sm = got.smoothed.cpu().numpy()
    np.testing.assert_allclose(sm, ref.smoothed, rtol=RTOL, atol=ATOL)
    point, level, score = got.point.cpu().numpy(), got.level.cpu().numpy(), got.score.cpu().numpy()
    mask = got.mask.cpu().numpy()
    for q in range(Q):
        crit = _level_crit(ref.smoothed[q], mode, thr)
        best = crit.max()
        lv = int(level[q])
        if lv != ref.level[q]:
            assert crit[lv] >= best - TIE, f"query {q}: level {lv} is not optimal ({crit})"
        s = ref.smoothed[q, lv]
        x, y = int(point[q, 0]), int(point[q, 1])
        assert 0 <= x < W and 0 <= y < H
        assert s[y * W + x] >= s.max() - TIE, f"query {q}: point ({x}, {y}) is not a maximum"
        if lv == ref.level[q] and (x, y) != tuple(ref.point[q]):
            assert abs(s[y * W + x] - s[ref.point[q][1] * W + ref.point[q][0]]) <= TIE
        assert score[q] == pytest.approx(s.max(), rel=RTOL, abs=ATOL)
        mx, mn = s.max(), s.min()
        nrm = (s - mn) / (mx - mn) if mx > mn else np.zeros_like(s)
        want = (nrm > thr).astype(np.uint8)
        sure = np.abs(nrm - thr) > KNIFE
        assert np.array_equal(mask[q][sure], want[sure]), f"query {q}: mask differs"
    return got, ref


@pytest.mark.parametrize("H,W,k", [(37, 53, 1), (37, 53, 3), (96, 128, 15), (131, 97, 29), (40, 70, 63),
                                   (5, 200, 31), (1, 1, 3)])
@pytest.mark.parametrize("mode", [0, 1])
def test_postprocess_matches_oracle(H, W, k, mode):
    rel = syn.relevancy_maps(syn.SEED + 5 + k, 2, 3, H, W)
    run_and_compare(rel, H, W, k, mode, 0.5)


def test_postprocess_bf16_input_and_thresholds():
    """BF16 relevancy (the tensor-core query's output): both sides read the same rounded values."""
    rel = syn.relevancy_maps(syn.SEED + 5, 3, 2, 64, 80)
    for thr in (0.0, 0.3, 0.75):
        run_and_compare(rel, 64, 80, 9, 0, thr, dtype=torch.bfloat16)


def test_postprocess_level_rules_on_constructed_maps():
    """The constructed case of the oracle pins: LERF takes the spike's level, the blended rule the
    broad blob's level."""
    H, W = 24, 32
    lev0 = np.full((H, W), 0.6, np.float32)
    lev0[:, :4] = 0.0
    lev0[5, 20] = 0.9
    y, x = np.mgrid[0:H, 0:W]
    lev1 = (0.1 + 0.7 * np.exp(-((x - 10.0) ** 2 + (y - 12.0) ** 2) / 32.0)).astype(np.float32)
    rel = np.stack([lev0.reshape(-1), lev1.reshape(-1)])[None]
    got, _ = run_and_compare(rel, H, W, 1, 0, 0.5)
    assert int(got.level[0]) == 0 and tuple(got.point[0].tolist()) == (20, 5)
    got, _ = run_and_compare(rel, H, W, 1, 1, 0.5)
    assert int(got.level[0]) == 1 and tuple(got.point[0].tolist()) == (10, 12)


def test_postprocess_full_frame_three_levels():
    """The 1440 x 1080 frame of the at-scale workload, three levels, one query, k = 29."""
    H, W = 1080, 1440
    rel = syn.relevancy_maps(syn.SEED + 5, 1, 3, H, W, blobs=12)
    run_and_compare(rel, H, W, 29, 0, 0.5)


def test_postprocess_rejects_bad_arguments():
    rel = torch.rand((1, 1, 64), device="cuda")
    for k in (0, 2, 65):
        with pytest.raises(L.LSV2Error):
            postprocess(rel, 8, 8, k=k)
    with pytest.raises(L.LSV2Error):
        postprocess(rel, 8, 8, k=3, mode=2)
    with pytest.raises(L.LSV2Error):
        postprocess(rel, 8, 8, k=3, threshold=1.5)
