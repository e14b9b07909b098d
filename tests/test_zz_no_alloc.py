"""lsv2_splat_coeffs_noalloc: the splat for callers that cannot allocate device memory (a
fixed-budget render loop, a runtime that owns all device memory, a host without its own
allocator).  Its scratch is a fixed device array inside the library instead of a workspace.

Called through the C ABI twice in a row (different scenes, so the second call runs over the
first call's leftover scratch) and compared with lsv2_splat_coeffs on the same inputs.  This
file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import lsv2_synth as syn

from gpu_helpers import assert_map_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_07136_b300 import _lib as L  # noqa: E402
from paper_2507_07136_b300.pipeline import DeviceScene, Frame, _ptr, _stream  # noqa: E402


def noalloc_splat(fr):
    s = fr.scene
    coeff = torch.full_like(fr.coeff, -1.0)
    final_T = torch.full_like(fr.final_T, -1.0)
    n_last = torch.full_like(fr.n_last, -1)
    code = L.lib().lsv2_splat_coeffs_noalloc(C.byref(fr.ccam), s.n, C.byref(fr.proj), _ptr(fr.tile_ranges),
                                             _ptr(fr.gauss_ids), s.levels, s.K, 64, _ptr(s.idx), _ptr(s.weights),
                                             _ptr(coeff), _ptr(final_T), _ptr(n_last), _ptr(fr.status),
                                             _stream(None))
    assert code == 0, L.STATUS.get(code, code)
    return coeff, final_T, n_last


def check_against_workspace_version(sc, cam):
    fr = Frame(DeviceScene.from_numpy(sc), cam)
    fr.render()          # lsv2_project, lsv2_bin_sort, lsv2_splat_coeffs (workspace version)
    fr.check()
    coeff, final_T, n_last = noalloc_splat(fr)
    fr.check()
    assert_map_close(coeff.cpu().numpy(), fr.coeff.cpu().numpy(), what="no-alloc coefficient map")
    assert_map_close(final_T.cpu().numpy(), fr.final_T.cpu().numpy(), what="no-alloc final T")
    assert np.array_equal(n_last.cpu().numpy(), fr.n_last.cpu().numpy())


def test_noalloc_matches_workspace_splat_twice():
    sc1, cam1 = syn.tiny()
    check_against_workspace_version(sc1, cam1)
    sc2 = syn.make_scene(3000, 3, seed=11, mean_kind="uniform", mean_param=1.0, log_scale_mu=-3.2,
                         log_scale_sigma=0.4)
    check_against_workspace_version(sc2, syn.orbit_camera(141, 99, 4.0))


def test_noalloc_capacity_boundary():
    """8 MiB of 160-byte records (3 levels, K = 4): 52,428 Gaussians fit, 52,429 do not.  The
    accepted call runs on a scene of exactly 52,428 Gaussians and matches the workspace splat;
    the rejected one returns LSV2_ERR_CAPACITY on the host and launches nothing."""
    rec = 160
    limit = (8 << 20) // rec
    assert limit == 52428
    assert L.lsv2_splat_workspace_bytes(limit, 3, 4) <= 8 << 20 < L.lsv2_splat_workspace_bytes(limit + 1, 3, 4)
    sc = syn.make_scene(limit, 3, seed=12, mean_kind="uniform", mean_param=1.0, log_scale_mu=-3.5,
                        log_scale_sigma=0.4)
    check_against_workspace_version(sc, syn.orbit_camera(96, 80, 4.0))
    fr = Frame(DeviceScene.from_numpy(sc), syn.orbit_camera(96, 80, 4.0))
    code = L.lib().lsv2_splat_coeffs_noalloc(C.byref(fr.ccam), limit + 1, C.byref(fr.proj), _ptr(fr.tile_ranges),
                                             _ptr(fr.gauss_ids), 3, 4, 64, _ptr(fr.scene.idx),
                                             _ptr(fr.scene.weights), _ptr(fr.coeff), _ptr(fr.final_T),
                                             _ptr(fr.n_last), _ptr(fr.status), _stream(None))
    assert code == L.LSV2_ERR_CAPACITY
