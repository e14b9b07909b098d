"""The C-ABI library loads, exports every entry point include/lsv2.h declares, and rejects bad
arguments on the host (no GPU needed: these paths return before any CUDA call)."""
import ctypes as C
import os
import re

import pytest

from paper_2507_07136_b300 import _lib as L
from paper_2507_07136_b300.build import build as build_lib

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "lsv2.h")


def declared_in_header():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lsv2_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build_lib()
    return L.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_in_header()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(L.declared_symbols()) == names


def test_version_and_status_strings(lib):
    assert L.lsv2_abi_version() == 2
    assert lib.lsv2_status_string(0) == b"ok"
    assert lib.lsv2_status_string(3) == b"instance capacity exceeded"


def test_workspace_queries(lib):
    assert L.lsv2_splat_workspace_bytes(1000, 3, 4) >= 1000 * 112
    assert L.lsv2_bin_sort_workspace_bytes(10, 1 << 20, 6120) >= 2 * 8 * (1 << 20)
    assert L.lsv2_query_workspace_bytes(3, 64, 1, 4) >= 3 * 69 * 64 * 4
    assert L.lsv2_query_workspace_bytes(3, 32, 1, 4) == 0


def _cam(w=64, h=48, tile=16):
    import lsv2_synth as syn
    return L.camera(syn.orbit_camera(w, h, 4.0, tile=(tile, tile)))


def test_host_validation_rejects_bad_arguments(lib):
    cam = _cam()
    proj = L.lsv2_proj()
    # null camera, null projection buffers, bad tile shape: all rejected before any launch
    assert lib.lsv2_project(None, 10, 0, 0, 0, 0, C.byref(proj), 0, 0) == 1
    assert lib.lsv2_project(C.byref(cam), 10, 0, 0, 0, 0, C.byref(proj), 0, 0) == 1
    bad = _cam(tile=12)
    assert lib.lsv2_project(C.byref(bad), 0, 0, 0, 0, 0, C.byref(proj), 0, 0) == 1
    # unsupported decode shapes
    assert lib.lsv2_decode(1, 10, 32, 512, 16, 0, 16, 0, 16, 0, 0, 0) == 2
    assert lib.lsv2_decode(1, 10, 64, 500, 16, 0, 16, 0, 16, 0, 0, 0) == 2
    assert lib.lsv2_decode(1, 10, 64, 512, 16, 0, 16, 7, 16, 0, 0, 0) == 1
    # query: null text
    assert lib.lsv2_query(1, 10, 64, 512, 16, 0, 16, 1, 4, 0, 10.0, 16, 1 << 20, 16, 0, 0, 0, 0) == 1
    with pytest.raises(L.LSV2Error):
        L.call("lsv2_decode", 1, 10, 32, 512, 16, 0, 16, 0, 16, 0, 0, 0)


def test_wait_limit_setting_round_trips(lib):
    """The bound of the kernels' device-side waits is a host setting read at launch (no GPU
    needed to set it); default 1 s."""
    assert L.lsv2_wait_limit_ns() == 1_000_000_000
    try:
        L.lsv2_set_wait_limit_ns(0)
        assert L.lsv2_wait_limit_ns() == 0
        L.lsv2_set_wait_limit_ns(123456789)
        assert L.lsv2_wait_limit_ns() == 123456789
    finally:
        L.lsv2_set_wait_limit_ns(1_000_000_000)


def test_mlp_decode_host_checks(lib):
    """Workspace sizing, the choice between the fused kernel and the library GEMMs, and the host-side
    rejections of lsv2_mlp_decode (all before any CUDA call)."""
    w = (C.c_int32 * 8)(8, 16, 32, 64, 128, 256, 256, 512)
    lt = 32 << 20
    # LSV2_MLP_FUSED: only the packed weights, per part its ceil(K / 64) chunks of N x 128 bytes
    # (the last layer in two parts of 256), for any row count
    fused = L.LSV2_MLP_FUSED
    image = (16 + 32 + 64 + 128) * 128 + 2 * 256 * 128 + 3 * 4 * 256 * 128
    for rows in (1, 1000, 1 << 22):
        for dt in (0, 1):
            assert L.lsv2_mlp_decode_workspace_bytes(rows, 7, w, dt, fused) == image
    # widths the fused kernel does not take: a hidden width not a multiple of 16, one above 256,
    # an output not a multiple of 16, an input above 32
    for ws in [(8, 24, 512), (8, 272, 512), (8, 64, 520), (40, 64, 512)]:
        wb = (C.c_int32 * 3)(*ws)
        assert L.lsv2_mlp_decode_workspace_bytes(10, 2, wb, 1, fused) == 0, ws
        assert lib.lsv2_mlp_decode(10, 2, wb, 256, 1, 256, 256, 256, fused, 256, 1 << 30, 0, 0) == 2, ws
    # block_rows >= 0: two activation buffers of a block at width 256, plus the BF16 copy of an F32 input
    blk = 1 << 20
    for b in (0, blk):
        assert L.lsv2_mlp_decode_workspace_bytes(1 << 22, 7, w, 0, b) == 2 * blk * 256 * 2 + blk * 8 * 2 + lt
        assert L.lsv2_mlp_decode_workspace_bytes(1 << 22, 7, w, 1, b) == 2 * blk * 256 * 2 + lt
    assert L.lsv2_mlp_decode_workspace_bytes(1000, 7, w, 1, 0) == 2 * 512000 + lt
    assert L.lsv2_mlp_decode_workspace_bytes(1 << 22, 7, w, 1, 1024) == 2 * 1024 * 256 * 2 + lt
    assert L.lsv2_mlp_decode_workspace_bytes(1 << 22, 7, w, 1, -2) == 0
    assert L.lsv2_mlp_decode_workspace_bytes(-1, 7, w, 0, 0) == 0
    assert L.lsv2_mlp_decode_workspace_bytes(10, 0, w, 0, 0) == 0
    assert L.lsv2_mlp_decode_workspace_bytes(10, 7, w, 2, 0) == 0
    big = 1 << 30
    ok = [10, 7, w, 256, 0, 256, 256, 256, 0, 256, big, 0, 0]
    assert lib.lsv2_mlp_decode(0, 7, w, 256, 0, 256, 256, 256, 0, 256, big, 0, 0) == 0   # no rows: nothing to do
    assert lib.lsv2_mlp_decode(0, 7, w, 256, 0, 256, 256, 256, fused, 256, image, 0, 0) == 0
    assert lib.lsv2_mlp_decode(10, 7, w, 256, 0, 256, 256, 256, fused, 256, image - 1, 0, 0) == 1
    for i, bad in [(3, 0), (3, 260), (4, 5), (8, 100), (8, -128), (8, -2), (10, 1000)]:
        args = list(ok)
        args[i] = bad
        assert lib.lsv2_mlp_decode(*args) == 1, (i, bad)
    for widths in [(8, 12, 512), (4, 16, 512), (8, 16, 8192)]:
        wb = (C.c_int32 * 3)(*widths)
        assert lib.lsv2_mlp_decode(10, 2, wb, 256, 0, 256, 256, 256, 0, 256, big, 0, 0) == 2, widths


def test_query_prepare_host_checks(lib):
    """lsv2_query_prepare / lsv2_query_prepared reject bad arguments on the host, before any launch."""
    big = 1 << 24
    # prepare: null codebook or text, unsupported L, a BF16 query count beyond 512 columns,
    # unknown compute dtype, workspace too small
    assert lib.lsv2_query_prepare(3, 64, 512, 0, 1, 4, 256, 1, 256, big, 0) == 1
    assert lib.lsv2_query_prepare(3, 64, 512, 256, 1, 4, 0, 1, 256, big, 0) == 1
    assert lib.lsv2_query_prepare(3, 32, 512, 256, 1, 4, 256, 1, 256, big, 0) == 2
    assert lib.lsv2_query_prepare(3, 64, 512, 256, 96, 4, 256, 1, 256, big, 0) == 2
    assert lib.lsv2_query_prepare(3, 64, 512, 256, 1, 4, 256, 7, 256, big, 0) == 1
    assert lib.lsv2_query_prepare(3, 64, 512, 256, 1, 4, 256, 1, 256, 16, 0) == 1
    # prepared: null map or output, unsupported map dtype with FP32 compute, small workspace
    assert lib.lsv2_query_prepared(3, 100, 64, 0, 0, 1, 4, 10.0, 256, big, 256, 0, 1, 0, 0) == 1
    assert lib.lsv2_query_prepared(3, 100, 64, 256, 0, 1, 4, 10.0, 256, big, 0, 0, 1, 0, 0) == 1
    assert lib.lsv2_query_prepared(3, 100, 64, 256, 1, 1, 4, 10.0, 256, big, 256, 0, 0, 0, 0) == 2
    assert lib.lsv2_query_prepared(3, 100, 64, 256, 0, 1, 4, 10.0, 256, 16, 256, 0, 1, 0, 0) == 1
