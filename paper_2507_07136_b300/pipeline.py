"""Torch-side pipeline around the C ABI: device buffers, streams, and the call sequence.

PyTorch only provides device memory and streams here; every step of the path runs in the
CUDA library through ``_lib``.  ``Frame`` owns the per-camera buffers, so the steady-state
call sequence allocates nothing and can be captured in a CUDA graph.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import _lib as L

L_CODEBOOK = 64


def _ptr(t: torch.Tensor | None) -> int:
    return 0 if t is None else t.data_ptr()


def _stream(stream: torch.cuda.Stream | None) -> int:
    return (stream or torch.cuda.current_stream()).cuda_stream


@dataclass
class DeviceScene:
    """Gaussians and their sparse coefficients, resident in HBM (activated values)."""
    means: torch.Tensor      # f32 [N, 3]
    scales: torch.Tensor     # f32 [N, 3]
    quats: torch.Tensor      # f32 [N, 4]
    opacity: torch.Tensor    # f32 [N]
    idx: torch.Tensor        # u8  [N, levels, K]
    weights: torch.Tensor    # f32 [N, levels, K]
    codebook: torch.Tensor   # f32 [levels, L, D]

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def levels(self) -> int:
        return int(self.idx.shape[1])

    @property
    def K(self) -> int:
        return int(self.idx.shape[2])

    @property
    def L(self) -> int:
        return int(self.codebook.shape[1])

    @property
    def D(self) -> int:
        return int(self.codebook.shape[2])

    @staticmethod
    def from_numpy(sc, device="cuda") -> "DeviceScene":
        def f(a, dt=torch.float32):
            return torch.as_tensor(a).to(device=device, dtype=dt).contiguous()
        return DeviceScene(f(sc.means), f(sc.scales), f(sc.quats), f(sc.opacity), f(sc.idx, torch.uint8),
                           f(sc.weights), f(sc.codebook))


class Frame:
    """Per-camera buffers and the project -> bin_sort -> splat -> decode / query sequence."""

    def __init__(self, scene: DeviceScene, cam, capacity: int | None = None, device="cuda"):
        self.scene, self.cam, self.device = scene, cam, device
        self.ccam = L.camera(cam)
        n = scene.n
        dev = torch.device(device)
        self.xy = torch.empty((n, 4), dtype=torch.float32, device=dev)
        self.conic_o = torch.empty((n, 4), dtype=torch.float32, device=dev)
        self.extent = torch.empty((n, 2), dtype=torch.float32, device=dev)
        self.depth = torch.empty(n, dtype=torch.float32, device=dev)
        self.radius = torch.empty(n, dtype=torch.int32, device=dev)
        self.rect = torch.empty((n, 4), dtype=torch.int32, device=dev)
        self.tiles_touched = torch.empty(n, dtype=torch.int32, device=dev)
        self.flags = torch.empty(n, dtype=torch.uint8, device=dev)
        self.axes = torch.empty((n, 8), dtype=torch.float32, device=dev)
        self.proj = L.lsv2_proj(_ptr(self.xy), _ptr(self.conic_o), _ptr(self.extent), _ptr(self.depth),
                                _ptr(self.radius), _ptr(self.rect), _ptr(self.tiles_touched), _ptr(self.flags),
                                _ptr(self.axes))
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.num_instances = torch.zeros(1, dtype=torch.int64, device=dev)
        self.T = cam.num_tiles
        self.P = cam.num_pixels
        self.tile_ranges = torch.empty((self.T, 2), dtype=torch.int32, device=dev)
        if capacity is None:
            self.project()
            capacity = max(1024, int(self.tiles_touched.sum().item() * 1.25) + 1024)
        self.capacity = int(capacity)
        self.gauss_ids = torch.empty(self.capacity, dtype=torch.int32, device=dev)
        self.bin_ws_bytes = L.lsv2_bin_sort_workspace_bytes(n, self.capacity, self.T)
        self.bin_ws = torch.empty(self.bin_ws_bytes, dtype=torch.uint8, device=dev)
        self.splat_ws_bytes = L.lsv2_splat_workspace_bytes(n, scene.levels, scene.K)
        self.splat_ws = torch.empty(max(self.splat_ws_bytes, 16), dtype=torch.uint8, device=dev)
        self.coeff = torch.empty((scene.levels, self.P, scene.L), dtype=torch.float32, device=dev)
        self.final_T = torch.empty(self.P, dtype=torch.float32, device=dev)
        self.n_last = torch.empty(self.P, dtype=torch.int32, device=dev)
        self.query_ws = None

    # ------------------------------------------------------------------ steps
    def project(self, stream=None):
        s = self.scene
        L.lsv2_project(self.ccam, s.n, _ptr(s.means), _ptr(s.scales), _ptr(s.quats), _ptr(s.opacity), self.proj,
                       _ptr(self.status), _stream(stream))

    def bin_sort(self, stream=None):
        L.lsv2_bin_sort(self.ccam, self.scene.n, self.proj, _ptr(self.bin_ws), self.bin_ws_bytes,
                        _ptr(self.gauss_ids), self.capacity, _ptr(self.tile_ranges), _ptr(self.num_instances),
                        _ptr(self.status), _stream(stream))

    def splat(self, stream=None):
        s = self.scene
        L.lsv2_splat_coeffs(self.ccam, s.n, self.proj, _ptr(self.tile_ranges), _ptr(self.gauss_ids), s.levels, s.K,
                            s.L, _ptr(s.idx), _ptr(s.weights), _ptr(self.splat_ws), self.splat_ws_bytes,
                            _ptr(self.coeff), _ptr(self.final_T), _ptr(self.n_last), _ptr(self.status),
                            _stream(stream))

    def splat_dense(self, stream=None):
        """The blend without the sparse splatting (dense 64-entry coefficients per level;
        lsv2_splat_coeffs_dense): same outputs as splat(), for timing the comparison."""
        s = self.scene
        need = L.lsv2_splat_dense_workspace_bytes(s.n, s.levels)
        if need == 0:
            raise L.LSV2Error("lsv2_splat_dense_workspace_bytes", 2)
        if getattr(self, "dense_ws", None) is None or self.dense_ws.numel() < need:
            self.dense_ws = torch.empty(need, dtype=torch.uint8, device=self.device)
        L.lsv2_splat_coeffs_dense(self.ccam, s.n, self.proj, _ptr(self.tile_ranges), _ptr(self.gauss_ids), s.levels,
                                  s.K, s.L, _ptr(s.idx), _ptr(s.weights), _ptr(self.dense_ws), need,
                                  _ptr(self.coeff), _ptr(self.final_T), _ptr(self.n_last), _ptr(self.status),
                                  _stream(stream))

    def render_fused(self, feat: torch.Tensor | None, text: torch.Tensor | None = None, rel: torch.Tensor | None = None,
                     tau: float = 10.0, stream=None):
        """Splat + decode (BF16 feat [levels, P, D], or None) + relevancy (rel [Q, levels, P]) in one kernel
        (lsv2_render_fused); W is not written (self.coeff is left untouched)."""
        s = self.scene
        Q, n_neg = (0, 1) if text is None else (text.shape[0], text.shape[1] - 1)
        need = L.lsv2_render_fused_workspace_bytes(s.n, s.levels, s.K, s.D, Q, n_neg)
        if need == 0:
            raise L.LSV2Error("lsv2_render_fused_workspace_bytes", 2)
        if getattr(self, "fused_ws", None) is None or self.fused_ws.numel() < need:
            self.fused_ws = torch.empty(need, dtype=torch.uint8, device=self.device)
        rel_dt = L.LSV2_BF16 if (rel is not None and rel.dtype == torch.bfloat16) else L.LSV2_F32
        L.lsv2_render_fused(self.ccam, s.n, self.proj, _ptr(self.tile_ranges), _ptr(self.gauss_ids), s.levels, s.K,
                            s.L, _ptr(s.idx), _ptr(s.weights), _ptr(s.codebook), s.D, Q, n_neg, _ptr(text),
                            float(tau), _ptr(self.fused_ws), need, _ptr(feat), _ptr(rel), rel_dt, _ptr(self.final_T),
                            _ptr(self.n_last), _ptr(self.status), _stream(stream))

    def splat_bf16(self, stream=None):
        """The splat with the coefficient map written as BF16 into self.coeff16 (what the tensor-core
        decode and relevancy consume)."""
        s = self.scene
        if getattr(self, "coeff16", None) is None:
            self.coeff16 = torch.empty((s.levels, self.P, s.L), dtype=torch.bfloat16, device=self.device)
        L.lsv2_splat_coeffs_bf16(self.ccam, s.n, self.proj, _ptr(self.tile_ranges), _ptr(self.gauss_ids), s.levels,
                                 s.K, s.L, _ptr(s.idx), _ptr(s.weights), _ptr(self.splat_ws),
                                 self.splat_ws_bytes, _ptr(self.coeff16), _ptr(self.final_T), _ptr(self.n_last),
                                 _ptr(self.status), _stream(stream))

    def render(self, stream=None):
        self.project(stream)
        self.bin_sort(stream)
        self.splat(stream)

    def decode(self, out: torch.Tensor, codebook: torch.Tensor | None = None, tensor_cores: bool | None = None,
               stream=None, from_bf16: bool = False):
        """F = W S.  FP32 out + FP32 codebook -> CUDA-core FP32 path unless tensor_cores=True;
        any BF16 operand or tensor_cores=True -> tcgen05 path (BF16 operands, FP32 accumulation)."""
        cb = self.scene.codebook if codebook is None else codebook
        cb_dt = L.LSV2_BF16 if cb.dtype == torch.bfloat16 else L.LSV2_F32
        out_dt = L.LSV2_BF16 if out.dtype == torch.bfloat16 else L.LSV2_F32
        if tensor_cores and cb_dt == L.LSV2_F32 and out_dt == L.LSV2_F32:
            raise ValueError("the tensor-core decode needs a BF16 codebook or BF16 output")
        W, w_dt = (self.coeff16, L.LSV2_BF16) if from_bf16 else (self.coeff, L.LSV2_F32)
        L.lsv2_decode(self.scene.levels, self.P, self.scene.L, self.scene.D, _ptr(W), w_dt, _ptr(cb),
                      cb_dt, _ptr(out), out_dt, _ptr(self.status), _stream(stream))

    def _query_ws(self, Q: int, n_neg: int) -> int:
        need = L.lsv2_query_workspace_bytes(self.scene.levels, self.scene.L, Q, n_neg)
        if self.query_ws is None or self.query_ws.numel() < need:
            self.query_ws = torch.empty(need, dtype=torch.uint8, device=self.device)
        return need

    def query(self, text: torch.Tensor, out: torch.Tensor, tau: float = 10.0, compute=L.LSV2_F32, stream=None,
              from_bf16: bool = False, prepared: bool = False):
        """Relevancy maps out [Q, levels, P] of the texts [Q, 1 + n_neg, D] (lsv2_query); with
        prepared=True the query operands come from an earlier query_prepare of the same texts and
        compute dtype (lsv2_query_prepared)."""
        Q, nt, D = text.shape
        need = self._query_ws(Q, nt - 1)
        out_dt = L.LSV2_BF16 if out.dtype == torch.bfloat16 else L.LSV2_F32
        W, w_dt = (self.coeff16, L.LSV2_BF16) if from_bf16 else (self.coeff, L.LSV2_F32)
        if prepared:
            L.lsv2_query_prepared(self.scene.levels, self.P, self.scene.L, _ptr(W), w_dt, Q, nt - 1, float(tau),
                                  _ptr(self.query_ws), need, _ptr(out), out_dt, compute, _ptr(self.status),
                                  _stream(stream))
            return
        L.lsv2_query(self.scene.levels, self.P, self.scene.L, D, _ptr(W), w_dt, _ptr(self.scene.codebook),
                     Q, nt - 1, _ptr(text), float(tau), _ptr(self.query_ws), need, _ptr(out), out_dt, compute,
                     _ptr(self.status), _stream(stream))

    def query_prepare(self, text: torch.Tensor, compute=L.LSV2_F32, stream=None):
        """The query operands of the texts (lsv2_query_prepare), for a later query(prepared=True); it
        reads only the codebook and the texts, so it can run on another stream beside the render."""
        Q, nt, D = text.shape
        need = self._query_ws(Q, nt - 1)
        L.lsv2_query_prepare(self.scene.levels, self.scene.L, D, _ptr(self.scene.codebook), Q, nt - 1, _ptr(text),
                             compute, _ptr(self.query_ws), need, _stream(stream))

    def postprocess(self, rel: torch.Tensor, k: int = 29, mode: int = L.LSV2_POST_LERF, threshold: float = 0.5,
                    out: "PostResult | None" = None, with_mask: bool = True, stream=None) -> "PostResult":
        """Mean filter, level selection, localisation point and mask of relevancy maps rel [Q, levels, P]
        (lsv2_postprocess)."""
        return postprocess(rel, self.cam.height, self.cam.width, k, mode, threshold, out, with_mask, self.status,
                           stream)

    def check(self):
        """Synchronise and raise if a kernel reported a device-side condition."""
        torch.cuda.synchronize()
        code = int(self.status.item())
        if code != 0:
            raise L.LSV2Error("device status", code)


class PostResult:
    """Buffers written by lsv2_postprocess for Q queries over `levels` maps of H x W pixels."""

    def __init__(self, Q: int, levels: int, H: int, W: int, device, with_mask: bool = True):
        self.Q, self.levels, self.H, self.W = Q, levels, H, W
        self.smoothed = torch.empty((Q, levels, H * W), dtype=torch.float32, device=device)
        self.point = torch.empty((Q, 2), dtype=torch.int32, device=device)
        self.level = torch.empty(Q, dtype=torch.int32, device=device)
        self.score = torch.empty(Q, dtype=torch.float32, device=device)
        self.mask = torch.empty((Q, H * W), dtype=torch.uint8, device=device) if with_mask else None
        self.ws_bytes = L.lsv2_postprocess_workspace_bytes(Q, levels)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=device)


def postprocess(rel: torch.Tensor, H: int, W: int, k: int = 29, mode: int = L.LSV2_POST_LERF, threshold: float = 0.5,
                out: PostResult | None = None, with_mask: bool = True, dev_status: torch.Tensor | None = None,
                stream=None) -> PostResult:
    """lsv2_postprocess over relevancy maps rel [Q, levels, H*W] (F32 or BF16, on the GPU)."""
    Q, levels, P = rel.shape
    assert P == H * W and rel.is_contiguous()
    if out is None:
        out = PostResult(Q, levels, H, W, rel.device, with_mask)
    rel_dt = L.LSV2_BF16 if rel.dtype == torch.bfloat16 else L.LSV2_F32
    L.lsv2_postprocess(Q, levels, H, W, _ptr(rel), rel_dt, int(k), int(mode), float(threshold), _ptr(out.ws),
                       out.ws_bytes, _ptr(out.smoothed), _ptr(out.point), _ptr(out.level), _ptr(out.score),
                       _ptr(out.mask) if out.mask is not None else None,
                       _ptr(dev_status) if dev_status is not None else None, _stream(stream))
    return out
