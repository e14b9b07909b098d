"""ctypes binding of ``include/lsv2.h``: the same function names, argument marshalling only.

Every compute step runs inside ``_build/liblsv2.so``.  If the library is missing this
module raises; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB

P = C.c_void_p
I32, I64, F32, SZ = C.c_int32, C.c_int64, C.c_float, C.c_size_t

LSV2_F32 = 0
LSV2_BF16 = 1
LSV2_MLP_FUSED = -1   # block_rows of lsv2_mlp_decode selecting the fused tensor-core kernel
LSV2_POST_LERF = 0
LSV2_POST_BLENDED = 1

LSV2_OK = 0
LSV2_ERR_INVALID_ARGUMENT = 1
LSV2_ERR_UNSUPPORTED = 2
LSV2_ERR_CAPACITY = 3
LSV2_ERR_CUDA = 4
LSV2_ERR_TIMEOUT = 5
LSV2_ERR_NONFINITE = 6

STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported configuration", 3: "instance capacity exceeded",
          4: "CUDA error", 5: "device wait timed out", 6: "non-finite value"}


class LSV2Error(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} failed: {STATUS.get(code, code)} ({code})")
        self.code = code


class lsv2_camera(C.Structure):
    _fields_ = [("width", I32), ("height", I32), ("tile_w", I32), ("tile_h", I32), ("fx", F32), ("fy", F32),
                ("cx", F32), ("cy", F32), ("near_z", F32), ("R", F32 * 9), ("t", F32 * 3)]


class lsv2_proj(C.Structure):
    _fields_ = [("xy", P), ("conic_o", P), ("extent", P), ("depth", P), ("radius", P), ("rect", P),
                ("tiles_touched", P), ("flags", P), ("axes", P)]


_SIGS = {
    "lsv2_abi_version": ([], I32),
    "lsv2_status_string": ([I32], C.c_char_p),
    "lsv2_set_wait_limit_ns": ([C.c_uint64], None),
    "lsv2_rate_probe_ops": ([I32, I64, I32], C.c_double),
    "lsv2_rate_probe": ([I32, I64, I32, P, P], I32),
    "lsv2_wait_limit_ns": ([], C.c_uint64),
    "lsv2_project": ([P, I64, P, P, P, P, P, P, P], I32),
    "lsv2_bin_sort_workspace_bytes": ([I64, I64, I32], SZ),
    "lsv2_bin_sort": ([P, I64, P, P, SZ, P, I64, P, P, P, P], I32),
    "lsv2_splat_workspace_bytes": ([I64, I32, I32], SZ),
    "lsv2_splat_coeffs": ([P, I64, P, P, P, I32, I32, I32, P, P, P, SZ, P, P, P, P, P], I32),
    "lsv2_splat_coeffs_bf16": ([P, I64, P, P, P, I32, I32, I32, P, P, P, SZ, P, P, P, P, P], I32),
    "lsv2_splat_dense_workspace_bytes": ([I64, I32], SZ),
    "lsv2_splat_coeffs_dense": ([P, I64, P, P, P, I32, I32, I32, P, P, P, SZ, P, P, P, P, P], I32),
    "lsv2_splat_coeffs_noalloc": ([P, I64, P, P, P, I32, I32, I32, P, P, P, P, P, P, P], I32),
    "lsv2_decode": ([I32, I64, I32, I32, P, I32, P, I32, P, I32, P, P], I32),
    "lsv2_query_workspace_bytes": ([I32, I32, I32, I32], SZ),
    "lsv2_query": ([I32, I64, I32, I32, P, I32, P, I32, I32, P, F32, P, SZ, P, I32, I32, P, P], I32),
    "lsv2_query_prepare": ([I32, I32, I32, P, I32, I32, P, I32, P, SZ, P], I32),
    "lsv2_query_prepared": ([I32, I64, I32, P, I32, I32, I32, F32, P, SZ, P, I32, I32, P, P], I32),
    "lsv2_query_views_workspace_bytes": ([I32, P, I64, I32, I32, I64, I32, I32], SZ),
    "lsv2_query_views": ([I32, P, I64, P, P, P, P, I32, I32, I32, P, P, P, I32, I32, I32, P, F32, I64, I32, P, SZ, P,
                          I32, P, P, P], I32),
    "lsv2_render_fused_workspace_bytes": ([I64, I32, I32, I32, I32, I32], SZ),
    "lsv2_render_fused": ([P, I64, P, P, P, I32, I32, I32, P, P, P, I32, I32, I32, P, F32, P, SZ, P, P, I32, P, P, P, P],
                          I32),
    "lsv2_sparsify": ([I64, I32, I32, P, P, P, P], I32),
    "lsv2_sparsify_backward": ([I64, I32, I32, P, P, P, P, P], I32),
    "lsv2_postprocess_workspace_bytes": ([I32, I32], SZ),
    "lsv2_postprocess": ([I32, I32, I32, I32, P, I32, I32, I32, F32, P, SZ, P, P, P, P, P, P, P], I32),
    "lsv2_l1_decode_backward": ([I32, I64, I32, I32, P, P, P, P, P, P, P, P], I32),
    "lsv2_splat_backward_workspace_bytes": ([I64], SZ),
    "lsv2_mlp_decode_workspace_bytes": ([I64, I32, P, I32, I64], SZ),
    "lsv2_mlp_decode": ([I64, I32, P, P, I32, P, P, P, I64, P, SZ, P, P], I32),
    "lsv2_splat_backward": ([P, I64, P, P, P, P, P, P, I32, I32, I32, P, P, P, P, P, P, SZ, P, P, P, P, P, P, P],
                            I32),
}

_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"CUDA library {LIB} is not built: run `python -m paper_2507_07136_b300.build`")
        _lib = C.CDLL(LIB)
        for name, (args, res) in _SIGS.items():
            fn = getattr(_lib, name)
            fn.argtypes = args
            fn.restype = res
    return _lib


def lib_path() -> str:
    """Path of the shared library this binding loads."""
    return LIB


def declared_symbols() -> list[str]:
    return list(_SIGS)


def call(name: str, *args) -> None:
    """Call an lsv2_* entry point; raise LSV2Error on a nonzero status."""
    code = getattr(lib(), name)(*args)
    if code != 0:
        raise LSV2Error(name, code)


def camera(cam) -> lsv2_camera:
    """lsv2_camera from any object with width/height/tile_w/tile_h/fx/fy/cx/cy/near/R/t."""
    c = lsv2_camera()
    c.width, c.height, c.tile_w, c.tile_h = int(cam.width), int(cam.height), int(cam.tile_w), int(cam.tile_h)
    c.fx, c.fy, c.cx, c.cy, c.near_z = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy), float(cam.near)
    R = [float(v) for v in list(cam.R.reshape(-1))]
    t = [float(v) for v in list(cam.t.reshape(-1))]
    for i in range(9):
        c.R[i] = R[i]
    for i in range(3):
        c.t[i] = t[i]
    return c


# thin wrappers with the ABI's names (pointers as Python ints, streams as cudaStream_t ints)
def lsv2_abi_version() -> int:
    return lib().lsv2_abi_version()


def lsv2_set_wait_limit_ns(ns: int) -> None:
    lib().lsv2_set_wait_limit_ns(int(ns))


def lsv2_wait_limit_ns() -> int:
    return int(lib().lsv2_wait_limit_ns())


def lsv2_project(cam, n, means, scales, quats, opacity, out, dev_status, stream):
    call("lsv2_project", C.byref(cam), n, means, scales, quats, opacity, C.byref(out), dev_status, stream)


def lsv2_bin_sort_workspace_bytes(n, capacity, num_tiles) -> int:
    return lib().lsv2_bin_sort_workspace_bytes(n, capacity, num_tiles)


def lsv2_bin_sort(cam, n, proj, ws, ws_bytes, gauss_ids, capacity, tile_ranges, dev_num, dev_status, stream):
    call("lsv2_bin_sort", C.byref(cam), n, C.byref(proj), ws, ws_bytes, gauss_ids, capacity, tile_ranges,
         dev_num, dev_status, stream)


def lsv2_splat_workspace_bytes(n, levels, K) -> int:
    return lib().lsv2_splat_workspace_bytes(n, levels, K)


def lsv2_splat_coeffs(cam, n, proj, tile_ranges, gauss_ids, levels, K, L, idx, w, ws, ws_bytes, coeff, final_T,
                      n_last, dev_status, stream):
    call("lsv2_splat_coeffs", C.byref(cam), n, C.byref(proj), tile_ranges, gauss_ids, levels, K, L, idx, w, ws,
         ws_bytes, coeff, final_T, n_last, dev_status, stream)


def lsv2_decode(levels, P_, L, D, coeff, coeff_dtype, codebook, codebook_dtype, feat, out_dtype, dev_status, stream):
    call("lsv2_decode", levels, P_, L, D, coeff, coeff_dtype, codebook, codebook_dtype, feat, out_dtype, dev_status,
         stream)


def lsv2_query_workspace_bytes(levels, L, Q, n_neg) -> int:
    return lib().lsv2_query_workspace_bytes(levels, L, Q, n_neg)


def lsv2_query(levels, P_, L, D, coeff, coeff_dtype, codebook, Q, n_neg, text, tau, ws, ws_bytes, rel, rel_dtype,
               compute_dtype, dev_status, stream):
    call("lsv2_query", levels, P_, L, D, coeff, coeff_dtype, codebook, Q, n_neg, text, tau, ws, ws_bytes, rel,
         rel_dtype, compute_dtype, dev_status, stream)


def lsv2_query_prepare(levels, L, D, codebook, Q, n_neg, text, compute_dtype, ws, ws_bytes, stream):
    call("lsv2_query_prepare", levels, L, D, codebook, Q, n_neg, text, compute_dtype, ws, ws_bytes, stream)


def lsv2_query_prepared(levels, P_, L, coeff, coeff_dtype, Q, n_neg, tau, ws, ws_bytes, rel, rel_dtype, compute_dtype,
                        dev_status, stream):
    call("lsv2_query_prepared", levels, P_, L, coeff, coeff_dtype, Q, n_neg, tau, ws, ws_bytes, rel, rel_dtype,
         compute_dtype, dev_status, stream)


def cameras(cams) -> C.Array:
    """Contiguous host array of lsv2_camera for lsv2_query_views."""
    arr = (lsv2_camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i] = camera(c)
    return arr


def lsv2_query_views_workspace_bytes(V, cams, n, levels, K, capacity, Q, n_neg) -> int:
    return lib().lsv2_query_views_workspace_bytes(V, cams, n, levels, K, capacity, Q, n_neg)


def lsv2_query_views(V, cams, n, means, scales, quats, opacity, levels, K, L, idx, w, codebook, D, Q, n_neg, text,
                     tau, capacity, stage_batch, ws, ws_bytes, rel, rel_dtype, dev_num, dev_status, stream):
    call("lsv2_query_views", V, cams, n, means, scales, quats, opacity, levels, K, L, idx, w, codebook, D, Q, n_neg,
         text, tau, capacity, stage_batch, ws, ws_bytes, rel, rel_dtype, dev_num, dev_status, stream)


def lsv2_l1_decode_backward(levels, P_, L, D, coeff, codebook, target, loss, dcoeff, dcodebook, dev_status, stream):
    call("lsv2_l1_decode_backward", levels, P_, L, D, coeff, codebook, target, loss, dcoeff, dcodebook, dev_status,
         stream)


def lsv2_splat_backward_workspace_bytes(n) -> int:
    return lib().lsv2_splat_backward_workspace_bytes(n)


def lsv2_splat_backward(cam, n, means, scales, quats, proj, tile_ranges, gauss_ids, levels, K, L, idx, w, final_T,
                        n_last, dcoeff, ws, ws_bytes, dw, dopacity, dmeans, dscales, dquats, dev_status, stream):
    call("lsv2_splat_backward", C.byref(cam), n, means, scales, quats, C.byref(proj), tile_ranges, gauss_ids,
         levels, K, L, idx, w, final_T, n_last, dcoeff, ws, ws_bytes, dw, dopacity, dmeans, dscales, dquats,
         dev_status, stream)


def lsv2_sparsify(rows, L, K, logits, idx, w, stream):
    call("lsv2_sparsify", rows, L, K, logits, idx, w, stream)


def lsv2_sparsify_backward(rows, L, K, idx, w, dw, dlogits, stream):
    call("lsv2_sparsify_backward", rows, L, K, idx, w, dw, dlogits, stream)


def lsv2_postprocess_workspace_bytes(Q, levels) -> int:
    return lib().lsv2_postprocess_workspace_bytes(Q, levels)


def lsv2_postprocess(Q, levels, H, W, rel, rel_dtype, k, mode, threshold, ws, ws_bytes, smoothed, point, level, score,
                     mask, dev_status, stream):
    call("lsv2_postprocess", Q, levels, H, W, rel, rel_dtype, k, mode, threshold, ws, ws_bytes, smoothed, point, level,
         score, mask, dev_status, stream)


def lsv2_render_fused_workspace_bytes(n, levels, K, D, Q, n_neg) -> int:
    return lib().lsv2_render_fused_workspace_bytes(n, levels, K, D, Q, n_neg)


def lsv2_render_fused(cam, n, proj, tile_ranges, gauss_ids, levels, K, L, idx, w, codebook, D, Q, n_neg, text, tau, ws,
                      ws_bytes, feat, rel, rel_dtype, final_T, n_last, dev_status, stream):
    call("lsv2_render_fused", C.byref(cam), n, C.byref(proj), tile_ranges, gauss_ids, levels, K, L, idx, w, codebook, D,
         Q, n_neg, text, tau, ws, ws_bytes, feat, rel, rel_dtype, final_T, n_last, dev_status, stream)


def lsv2_splat_dense_workspace_bytes(n, levels) -> int:
    return lib().lsv2_splat_dense_workspace_bytes(n, levels)


def lsv2_splat_coeffs_dense(cam, n, proj, tile_ranges, gauss_ids, levels, K, L, idx, w, ws, ws_bytes, coeff, final_T,
                            n_last, dev_status, stream):
    call("lsv2_splat_coeffs_dense", C.byref(cam), n, C.byref(proj), tile_ranges, gauss_ids, levels, K, L, idx, w, ws,
         ws_bytes, coeff, final_T, n_last, dev_status, stream)


def lsv2_splat_coeffs_bf16(cam, n, proj, tile_ranges, gauss_ids, levels, K, L, idx, w, ws, ws_bytes, coeff_bf16,
                           final_T, n_last, dev_status, stream):
    call("lsv2_splat_coeffs_bf16", C.byref(cam), n, C.byref(proj), tile_ranges, gauss_ids, levels, K, L, idx, w, ws,
         ws_bytes, coeff_bf16, final_T, n_last, dev_status, stream)


def lsv2_mlp_decode_workspace_bytes(rows, n_layers, widths, x_dtype, block_rows=0) -> int:
    """widths: host int32 array (ctypes array or anything accepted as a pointer)."""
    return lib().lsv2_mlp_decode_workspace_bytes(rows, n_layers, widths, x_dtype, block_rows)


def lsv2_mlp_decode(rows, n_layers, widths, x, x_dtype, weights, biases, y, block_rows, ws, ws_bytes, dev_status,
                    stream):
    call("lsv2_mlp_decode", rows, n_layers, widths, x, x_dtype, weights, biases, y, block_rows, ws, ws_bytes,
         dev_status, stream)
