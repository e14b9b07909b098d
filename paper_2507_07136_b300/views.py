"""Many views and many text queries of one scene in one call (lsv2_query_views), captured once
in a CUDA graph and replayed, with the tile shape and the shared-memory staging batch chosen by
a small autotuner.

    vb = ViewsBatch(scene, cams, Q=64, n_neg=4)        # buffers, instance capacity
    vb.run(text)                                       # eager: one C-ABI call
    vb.capture(text); vb.replay()                      # one CUDA graph launch per batch
    tile, batch = autotune(scene, cams, text)          # fastest (tile shape, staging batch)
"""
from __future__ import annotations

import hashlib
import json
import os

import torch

from . import _lib as L
from .pipeline import DeviceScene, _ptr, _stream

TILES = [(16, 16), (8, 8), (32, 8)]
BATCHES = [32, 16]
CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def _with_tile(cam, tile):
    return cam if (cam.tile_w, cam.tile_h) == tuple(tile) else cam.with_tile(*tile)


class ViewsBatch:
    """Buffers and the lsv2_query_views call for V cameras and Q queries (1 + n_neg texts each)."""

    def __init__(self, scene: DeviceScene, cams, Q: int, n_neg: int, tile=(16, 16), stage_batch: int = 0,
                 rel_dtype=torch.bfloat16, capacity: int | None = None, tau: float = 10.0, device="cuda"):
        self.scene, self.Q, self.n_neg, self.tau = scene, Q, n_neg, float(tau)
        self.cams = [_with_tile(c, tile) for c in cams]
        self.V = len(self.cams)
        self.ccams = L.cameras(self.cams)
        self.stage_batch = int(stage_batch)
        self.device = torch.device(device)
        self.P = [c.width * c.height for c in self.cams]
        self.rel = torch.empty(sum(Q * scene.levels * p for p in self.P), dtype=rel_dtype, device=self.device)
        self.status = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.num_instances = torch.zeros(1, dtype=torch.int64, device=self.device)
        self.text = torch.empty((Q, 1 + n_neg, scene.D), dtype=torch.float32, device=self.device)
        self.graph = None
        if capacity is None:
            # probe with a generous capacity, then size to the measured instance count
            self._alloc(max(1 << 20, 8 * scene.n * self.V))
            self.text.normal_()
            self.run()
            torch.cuda.synchronize()
            need = int(self.num_instances.item())
            self.status.zero_()
            capacity = max(1 << 16, int(need * 1.2) + 4096)
        self._alloc(int(capacity))

    def _alloc(self, capacity: int):
        s = self.scene
        self.capacity = capacity
        self.ws_bytes = L.lsv2_query_views_workspace_bytes(self.V, self.ccams, s.n, s.levels, s.K, capacity, self.Q,
                                                           self.n_neg)
        if self.ws_bytes == 0:
            raise L.LSV2Error("lsv2_query_views_workspace_bytes", 1)
        self.ws = None
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)

    def run(self, text: torch.Tensor | None = None, stream=None):
        if text is not None:
            self.text.copy_(text, non_blocking=True)
        s = self.scene
        rel_dt = L.LSV2_BF16 if self.rel.dtype == torch.bfloat16 else L.LSV2_F32
        L.lsv2_query_views(self.V, self.ccams, s.n, _ptr(s.means), _ptr(s.scales), _ptr(s.quats), _ptr(s.opacity),
                           s.levels, s.K, 64, _ptr(s.idx), _ptr(s.weights), _ptr(s.codebook), s.D, self.Q,
                           self.n_neg, _ptr(self.text), self.tau, self.capacity, self.stage_batch, _ptr(self.ws),
                           self.ws_bytes, _ptr(self.rel), rel_dt, _ptr(self.num_instances), _ptr(self.status),
                           _stream(stream))

    def capture(self, text: torch.Tensor | None = None):
        """Record one batch (every kernel of lsv2_query_views) as a CUDA graph."""
        if text is not None:
            self.text.copy_(text)
        side = torch.cuda.Stream(device=self.device)
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.run(stream=side)          # warm-up outside the graph (module loading, attributes)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.run(stream=torch.cuda.current_stream())
        return self.graph

    def replay(self):
        self.graph.replay()

    def rel_view(self, v: int) -> torch.Tensor:
        """Relevancy of view v: [Q][levels][H_v * W_v]."""
        off = sum(self.Q * self.scene.levels * p for p in self.P[:v])
        n = self.Q * self.scene.levels * self.P[v]
        return self.rel[off:off + n].view(self.Q, self.scene.levels, self.P[v])

    def check(self):
        torch.cuda.synchronize()
        code = int(self.status.item())
        if code != 0:
            raise L.LSV2Error("device status", code)


_LIB_DIGEST = None


def _lib_digest() -> str:
    """Digest of the loaded library file, so a rebuilt kernel invalidates cached choices."""
    global _LIB_DIGEST
    if _LIB_DIGEST is None:
        h = hashlib.sha1()
        with open(L.lib_path(), "rb") as f:
            for block in iter(lambda: f.read(1 << 20), b""):
                h.update(block)
        _LIB_DIGEST = h.hexdigest()[:16]
    return _LIB_DIGEST


def _key(scene, cams, Q, n_neg):
    name = torch.cuda.get_device_name()
    res = ",".join(f"{c.width}x{c.height}" for c in cams)
    return (f"{name}|lib={_lib_digest()}|{res}|n={scene.n}|levels={scene.levels}|K={scene.K}|"
            f"Q={Q}x{1 + n_neg}")


def autotune(scene: DeviceScene, cams, text: torch.Tensor, reps: int = 5, cache: str | None = CACHE,
             candidates=None, verbose: bool = False):
    """Time every (tile shape, staging batch) candidate on this batch and return the fastest,
    caching the choice in a JSON file keyed by (GPU, library build, resolutions, N, levels, K,
    queries)."""
    Q, nt = text.shape[0], text.shape[1]
    key = _key(scene, cams, Q, nt - 1)
    table = {}
    if cache and os.path.exists(cache):
        try:
            with open(cache) as f:
                table = json.load(f)
        except Exception:
            table = {}
    if key in table:
        return tuple(table[key]["tile"]), table[key]["batch"]
    results = {}
    for tile in TILES:
        for batch in (candidates or BATCHES):
            try:
                vb = ViewsBatch(scene, cams, Q, nt - 1, tile=tile, stage_batch=batch)
            except L.LSV2Error:
                continue
            vb.run(text)
            torch.cuda.synchronize()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            for _ in range(reps):
                vb.run()
            e.record()
            torch.cuda.synchronize()
            vb.check()
            results[(tile, batch)] = s.elapsed_time(e) / reps
            if verbose:
                print(f"tile {tile} batch {batch}: {results[(tile, batch)]:.3f} ms")
            del vb
            torch.cuda.empty_cache()
    (tile, batch), ms = min(results.items(), key=lambda kv: kv[1])
    table[key] = {"tile": list(tile), "batch": batch, "ms": ms,
                  "all": {f"{t[0]}x{t[1]}/{b}": v for (t, b), v in results.items()}}
    if cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        with open(cache, "w") as f:
            json.dump(table, f, indent=1)
    return tuple(tile), batch
