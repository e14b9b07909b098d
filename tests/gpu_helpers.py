"""Shared helpers for the GPU parity tests: comparisons against the FP64 oracle."""
from __future__ import annotations

import numpy as np

# FP32 maps: the tolerance the method's statement fixes (1e-5 relative), with an absolute floor
# far below any blended contribution (the smallest nonzero coefficient is >= (1/255) * 1e-4 * w).
REL_TOL = 1e-5
ABS_FLOOR = 1e-9
# Pixels where some decision quantity sits this close (relative) to its threshold are decided
# by rounding; they are counted and checked against a looser bound instead.
KNIFE_EDGE = 1e-4


def max_rel_violation(got, ref, rel=REL_TOL, floor=ABS_FLOOR):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    err = np.abs(got - ref)
    bound = rel * np.abs(ref) + floor
    return float((err / bound).max()) if err.size else 0.0


def assert_map_close(got, ref, mask=None, rel=REL_TOL, floor=ABS_FLOOR, what="map"):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    if mask is not None:
        got, ref = got[..., mask, :] if got.ndim == 3 else got[mask], ref[..., mask, :] if ref.ndim == 3 else ref[mask]
    err = np.abs(got - ref)
    bound = rel * np.abs(ref) + floor
    bad = err > bound
    if bad.any():
        i = np.unravel_index(np.argmax(err / bound), err.shape)
        raise AssertionError(f"{what}: {int(bad.sum())} of {bad.size} entries outside rel {rel}; worst at {i}: "
                             f"got {got[i]!r} ref {ref[i]!r} (x{float(err[i] / bound[i]):.2f} of bound)")
