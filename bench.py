"""Benchmark of the sparse-coefficient splatting hot path on one B300 (or N replicas).

Workload: 300,000 Gaussians (means N(0, 2^2), log-scales N(-4.5, 0.5)), three semantic levels,
K = 4 pairs over an L = 64 codebook of D = 512 features, one 1440x1080 camera at radius 6, one
text query with four negatives.  One step renders one frame through every stage of the path:
project -> bin_sort -> splat_coeffs -> decode (F materialised in HBM) -> query (relevancy).

Printed as one JSON line.  `value` is frames per second over all ranks, device-timed with CUDA
events per step, the step launched as one CUDA graph (L2 flushed between steps, flush not
timed); `stages_ms` times the same step launched eagerly with events between its stages.  `e2e`
runs the same steps (as graphs) through the C ABI with the per-step inputs (text embeddings)
copied from pinned host memory and the relevancy maps copied back (on a copy stream, while the
next step computes), host-timed.  `roofline` is for the stage that dominates the
step.  `cpu_baseline` times the FP64 oracle (single thread) on a bounded sample of the frame.
The query's operands (which depend only on the codebook and the texts) are prepared on a second
stream while the frame renders and joined before the relevancy kernel.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coeff-splat+decode FPS and query FPS @1440x1080, 300k Gaussians; % HBM/tensor roofline"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_PEAKS = {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}
# FP32 FMA pipe: 148 SMs x 128 lanes x 2 flop x 2.032 GHz (maximum SM clock)
FP32_ALU_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12


# relevancy post-processing in the timed step: mean-filter window and mask threshold (the paper
# gives neither)
POST_WINDOW = 29
POST_THRESHOLD = 0.5

SPLAT_KERNEL = "splat_tm_kernel<3,4> (one CTA per 16x16 tile, consumer warps 4-7 accumulate in TMEM)"
# DRAM bytes (read + write) per launch from ncu (dram__bytes_read.sum + dram__bytes_write.sum) on
# the same frame via `bench.py --profile STAGE`, with the kernels as they are now (an entry is
# removed when its kernel changes): the splat and the relevancy as launched here; the decode
# captured over one level (one third of the launch's pixels and bytes) and scaled by 3.
TRAFFIC = {
    SPLAT_KERNEL: 47180288 + 551101696,
    "decode_tc_kernel": 3 * (199180032 + 1531681536),
    "query_pipe_kernel<3,1>": 597308672 + 18798336,
}


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except Exception:
        return FALLBACK_PEAKS, "fallback"


class _CtypesNvml:
    """The few read-only NVML queries the clock sampler makes, through libnvidia-ml directly (for
    hosts without the pynvml module).  Names and constants follow NVML's C API."""

    NVML_CLOCK_SM = 1
    nvmlClocksEventReasonSwPowerCap = 0x4
    nvmlClocksEventReasonHwSlowdown = 0x8
    nvmlClocksEventReasonSwThermalSlowdown = 0x20
    nvmlClocksEventReasonHwThermalSlowdown = 0x40
    nvmlClocksEventReasonHwPowerBrakeSlowdown = 0x80

    def __init__(self):
        import ctypes
        self.C = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")

    def _ok(self, r):
        if r != 0:
            raise RuntimeError(f"NVML error {r}")

    def nvmlInit(self):
        self._ok(self.lib.nvmlInit_v2())

    def _handle(self, fn, arg):
        h = self.C.c_void_p()
        self._ok(fn(arg, self.C.byref(h)))
        return h

    def nvmlDeviceGetHandleByPciBusId(self, bus):
        return self._handle(self.lib.nvmlDeviceGetHandleByPciBusId_v2, self.C.c_char_p(bus.encode()))

    def nvmlDeviceGetHandleByIndex(self, i):
        return self._handle(self.lib.nvmlDeviceGetHandleByIndex_v2, self.C.c_uint(i))

    def _uint(self, fn, h, *args):
        v = self.C.c_uint()
        self._ok(fn(h, *args, self.C.byref(v)))
        return v.value

    def nvmlDeviceGetClockInfo(self, h, which):
        return self._uint(self.lib.nvmlDeviceGetClockInfo, h, self.C.c_int(which))

    def nvmlDeviceGetMaxClockInfo(self, h, which):
        return self._uint(self.lib.nvmlDeviceGetMaxClockInfo, h, self.C.c_int(which))

    def nvmlDeviceGetPowerUsage(self, h):
        return self._uint(self.lib.nvmlDeviceGetPowerUsage, h)

    def nvmlDeviceGetCurrentClocksEventReasons(self, h):
        v = self.C.c_ulonglong()
        self._ok(self.lib.nvmlDeviceGetCurrentClocksEventReasons(h, self.C.byref(v)))
        return v.value


class ClockSampler:
    """SM clock, power and clock-event (throttle) reasons sampled while the timed region runs.

    Polls NVML from a thread every `period_s` (read-only queries, a few microseconds each), so a
    timed region of a few tens of milliseconds still gets samples; falls back to `nvidia-smi -lms`
    when NVML is unavailable.  The device is found by its PCI bus id, so the NVML index need not
    equal the CUDA ordinal."""

    REASONS = [("hw_slowdown", "nvmlClocksEventReasonHwSlowdown"),
               ("hw_thermal_slowdown", "nvmlClocksEventReasonHwThermalSlowdown"),
               ("sw_thermal_slowdown", "nvmlClocksEventReasonSwThermalSlowdown"),
               ("sw_power_cap", "nvmlClocksEventReasonSwPowerCap"),
               ("hw_power_brake_slowdown", "nvmlClocksEventReasonHwPowerBrakeSlowdown")]
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, cuda_index: int, period_s: float = 0.005):
        self.index, self.period = cuda_index, period_s
        self.rows = []          # (sm_mhz, max_mhz, power_w, set of reason names)
        self.proc = self.thread = None
        self.stop = threading.Event()
        self.source = "none"
        self.nvml_error = None

    def _nvml_handle(self):
        try:
            import pynvml
        except ImportError:
            pynvml = _CtypesNvml()
        pynvml.nvmlInit()
        try:
            import torch
            pr = torch.cuda.get_device_properties(self.index)
            bus = f"{pr.pci_domain_id:08X}:{pr.pci_bus_id:02X}:{pr.pci_device_id:02X}.0"
            return pynvml, pynvml.nvmlDeviceGetHandleByPciBusId(bus)
        except Exception:
            return pynvml, pynvml.nvmlDeviceGetHandleByIndex(self.index)

    def _poll_nvml(self, nv, h):
        mx = nv.nvmlDeviceGetMaxClockInfo(h, nv.NVML_CLOCK_SM)
        bits = [(name, getattr(nv, const, 0)) for name, const in self.REASONS]
        while not self.stop.is_set():
            try:
                sm = nv.nvmlDeviceGetClockInfo(h, nv.NVML_CLOCK_SM)
                pw = nv.nvmlDeviceGetPowerUsage(h) / 1000.0
                rs = nv.nvmlDeviceGetCurrentClocksEventReasons(h)
                self.rows.append((float(sm), float(mx), pw, {n for n, b in bits if b and rs & b}))
            except Exception:
                pass
            self.stop.wait(self.period)

    def _read_smi(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.proc.stdout:
            p = [x.strip() for x in line.split(",")]
            if len(p) == 7:
                try:
                    self.rows.append((float(p[0]), float(p[1]), float(p[2]),
                                      {names[i] for i in range(4) if p[3 + i].lower() == "active"}))
                except ValueError:
                    pass

    def __enter__(self):
        try:
            nv, h = self._nvml_handle()
            self.thread = threading.Thread(target=self._poll_nvml, args=(nv, h), daemon=True)
            self.source = "nvml"
        except Exception as e:
            self.nvml_error = f"{type(e).__name__}: {e}"[:200]
            try:
                self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                              "--format=csv,noheader,nounits", "-lms", "100"],
                                             stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
                self.thread = threading.Thread(target=self._read_smi, daemon=True)
                self.source = "nvidia-smi"
            except Exception:
                self.thread = None
        if self.thread:
            self.thread.start()
            if self.source == "nvidia-smi":   # wait (bounded) for its first row
                t0 = time.time()
                while not self.rows and time.time() - t0 < 5.0:
                    time.sleep(0.05)
        return self

    def __exit__(self, *a):
        self.stop.set()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0,
                    "source": self.source}
        sm = [r[0] for r in self.rows]
        reasons = sorted(set().union(*[r[3] for r in self.rows]))
        out = {"sm_mhz": float(np.median(sm)), "sm_min_mhz": float(min(sm)),
               "sm_max_mhz": max(r[1] for r in self.rows), "power_w_max": max(r[2] for r in self.rows),
               "reasons": reasons, "samples": len(self.rows), "source": self.source}
        if self.nvml_error:
            out["nvml_error"] = self.nvml_error
        return out


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def spawn_ranks(gpus: int, argv) -> int | None:
    """`--gpus N` outside a launcher: run this script as N ranks of one node under
    torch.distributed.run (rendezvous on 127.0.0.1, a free port) and return their exit code.
    Returns None when no launch is needed (N = 1, or already running as a rank)."""
    if gpus <= 1 or "WORLD_SIZE" in os.environ:
        return None
    import socket
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={gpus}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + list(argv)
    return subprocess.call(cmd)


def max_over_ranks(values, world: int, device=None):
    """Element-wise maximum of a list of floats over all ranks (one all_reduce(MAX); the identity
    for one rank).  `device` is where the reduction tensor lives: a CUDA device for NCCL, None
    (CPU) for gloo."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def host_cpu():
    """CPU model and logical core count of this host (for the CPU-baseline record)."""
    model = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"cpu": model, "nproc": os.cpu_count()}


# ----------------------------------------------------------------------------- CPU baseline
def cpu_tiny_full_frame():
    """The FP64 oracle on one whole frame of the tiny scene (2,000 Gaussians, 128x96, one level,
    one query with four negatives): projection, binning, the blend of every pixel, decode and
    relevancy, timed as it runs (no sampling, no extrapolation)."""
    import lsv2_synth as syn
    from oracle import oracle as O
    sc, cam = syn.tiny()
    text = syn.text_queries(syn.SEED + 2, 1, 4)
    t0 = time.perf_counter()
    r = O.render(sc, cam)
    O.relevancy(O.decode(r.blend.out, sc.codebook), text, 10.0)
    s = time.perf_counter() - t0
    return {"frame_s": s, "frames_per_s": 1.0 / s, "workload": "2,000 Gaussians, 1 level, 128x96, 1 query + 4 "
            "negatives: project, bin, blend of all 12,288 pixels, decode, relevancy (whole frame, timed)"}


def cpu_baseline(npix: int = 2000, at_scale=None):
    """The FP64 oracle as it stands, single-threaded, on a bounded sample of one at-scale frame:
    projection + binning of all 300k Gaussians, then blend + decode + relevancy of `npix` random
    pixels.  `value` estimates the oracle's whole-frame rate (the per-pixel time scaled to the
    1,555,200-pixel frame); `sample_s` is the time this sample took."""
    import lsv2_synth as syn
    from oracle import oracle as O
    sc, cam, text = at_scale if at_scale is not None else syn.at_scale()
    t0 = time.perf_counter()
    pr = O.project(cam, sc.means, sc.scales, sc.quats)
    ids, ranges = O.bin(cam, pr)
    t_geom = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    px = rng.integers(0, cam.width, npix).astype(np.int32)
    py = rng.integers(0, cam.height, npix).astype(np.int32)
    t1 = time.perf_counter()
    bl = O.blend(cam, pr, sc.opacity, ids, ranges, idx=sc.idx, w=sc.weights, px=px, py=py)
    F = O.decode(bl.out, sc.codebook)
    O.relevancy(F, text, 10.0)
    t_pix = (time.perf_counter() - t1) / npix
    frame_s = t_geom + t_pix * cam.num_pixels
    return {"value": 1.0 / frame_s, "unit": "frames/s", "cores": 1, "kind": "oracle",
            "sample_s": t_geom + t_pix * npix, "frame_fraction": (t_geom + t_pix * npix) / frame_s,
            "sample": f"project+bin all 300k Gaussians ({t_geom:.2f} s) + blend/decode/relevancy of {npix} random "
                      f"pixels ({t_pix * 1e3:.3f} ms/px), the per-pixel time scaled to 1,555,200 px; single "
                      f"thread, FP64",
            "host": host_cpu()}


def reference_arm(args):
    """The oracle as the reference arm.  Each step is one bounded sample of the at-scale frame
    (cpu_baseline); `ms_per_step` is the measured time of a step, `value` the whole-frame rate the
    samples estimate, `frames_per_step` the fraction of a frame's work one step does."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import lsv2_synth as syn
    data = syn.at_scale()
    for _ in range(args.warmup):
        cpu_baseline(args.cpu_pixels, data)
    t0 = time.perf_counter()
    samples = [cpu_baseline(args.cpu_pixels, data) for _ in range(args.steps)]
    elapsed = time.perf_counter() - t0
    v = float(np.mean([c["value"] for c in samples]))
    ms = elapsed * 1e3 / max(1, args.steps)
    cb = dict(samples[-1])
    cb["value"] = v
    cb["tiny_full_frame"] = cpu_tiny_full_frame()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "frames/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "frames_per_step": v * ms / 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "300k Gaussians, 3 levels, K=4, L=64, D=512, 1440x1080, 1 query + 4 negatives"},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "note": f"FP64 CPU oracle (single thread) as the reference arm on rank 0; each step projects and bins the "
                    f"whole frame and blends, decodes and queries {args.cpu_pixels} sampled pixels; {args.steps} steps "
                    f"in {elapsed:.1f} s"}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- measured unit rates
def unit_rates(dev, target_ms: float = 20.0):
    """Throughput of the units the splat's blend uses, measured on this device with the library's
    rate probes (lsv2_rate_probe): FP32 FMA (per second; one FP32 pipe operation each), ex2 on the
    MUFU unit, and 4-byte shared-memory accesses (a load + store stream without bank conflicts).
    Each probe fills every SM (4 CTAs of 512 threads per SM) and is timed with CUDA events."""
    import torch
    from paper_2507_07136_b300 import _lib as Lb
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = 4 * sms
    sink = torch.zeros(blocks, device=dev)
    st = torch.cuda.current_stream().cuda_stream
    out = {}
    for kind, name in ((0, "fp32_fma_per_s"), (1, "ex2_per_s"), (2, "smem_access_per_s")):
        iters = 1000
        for _ in range(8):   # grow the launch until it takes about target_ms
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            Lb.call("lsv2_rate_probe", kind, iters, blocks, sink.data_ptr(), st)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            if ms >= target_ms:
                break
            iters = int(iters * max(2.0, target_ms / max(ms, 1e-3)))
        out[name] = Lb.lib().lsv2_rate_probe_ops(kind, iters, blocks) / (ms * 1e-3)
    out["probe"] = f"{blocks} CTAs x 512 threads, 8 independent chains per thread, about {target_ms:.0f} ms per probe"
    return out


def splat_work(sc, cam, npix: int = 20000, seed: int = 0):
    """The blend's algorithmic work on this frame (Algorithm 1, counted by the FP64 oracle on `npix`
    random pixels and scaled to the frame): list entries evaluated (up to and including the one
    that stops a pixel's walk) and contributions (entries that add their K pairs per level)."""
    from oracle import oracle as O
    pr = O.project(cam, sc.means, sc.scales, sc.quats)
    ids, ranges = O.bin(cam, pr)
    rng = np.random.default_rng(seed)
    px = rng.integers(0, cam.width, npix).astype(np.int32)
    py = rng.integers(0, cam.height, npix).astype(np.int32)
    bl = O.blend(cam, pr, sc.opacity, ids, ranges, idx=sc.idx, w=sc.weights, px=px, py=py)
    P = cam.num_pixels
    return {"evaluations": float(bl.n_eval.mean()) * P, "contributions": float(bl.n_contrib.mean()) * P,
            "sample_pixels": npix}


def splat_alu_roofline(work, levels: int, K: int, splat_ms: float, rates):
    """The splat against the units its arithmetic needs, per frame: per evaluation 13 FP32
    operations (offset, quadratic form, scale, clamp, compare) and one ex2; per contribution
    4 + levels K FP32 operations (1 - alpha, T update, compare, alpha T, the levels K weighted adds)
    and 2 levels K accumulator accesses (a read and a write per pair, counted as shared-memory
    accesses whatever memory holds the accumulator).  The fraction of each unit's measured rate
    the splat stage reaches; the largest names the bound."""
    t = splat_ms * 1e-3
    E, C = work["evaluations"], work["contributions"]
    fp32 = E * 13 + C * (4 + levels * K)
    need = {"fp32": (fp32, rates["fp32_fma_per_s"]), "ex2": (E, rates["ex2_per_s"]),
            "shared_memory": (C * 2 * levels * K, rates["smem_access_per_s"])}
    fr = {k: (n / t) / peak for k, (n, peak) in need.items()}
    bound = max(fr, key=fr.get)
    return {"bound": bound, "frac": fr[bound], "fracs": fr,
            "ops_per_frame": {k: n for k, (n, _) in need.items()},
            "achieved_per_s": {k: n / t for k, (n, _) in need.items()},
            "peak_per_s": {k: p for k, (_, p) in need.items()}, "peak_source": "measured (lsv2_rate_probe)",
            "work": work}


def precision_report(dev, chunk: int = 131072):
    """The precision workload (the tiny scene rendered at 1440x1080, one level): the BF16 path
    (coefficient map stored as BF16, tensor-core decode to BF16 F, tensor-core relevancy with one
    query and four negatives) against the FP64 oracle over every pixel: max and mean absolute error
    of the coefficient map W, the feature map F and the relevancy map; pixels whose blend decisions
    sit within 1e-4 relative of a threshold (knife edges, decided by rounding) counted and also
    left out in a second set of figures."""
    import torch
    import lsv2_synth as syn
    from oracle import oracle as O
    from paper_2507_07136_b300 import _lib as Lb
    from paper_2507_07136_b300.pipeline import DeviceScene, Frame
    sc, cam = syn.precision()
    text = syn.text_queries(syn.SEED + 2, 1, 4)
    fr = Frame(DeviceScene.from_numpy(sc, device=dev), cam, device=dev)
    fr.project()
    fr.bin_sort()
    fr.splat_bf16()
    F = torch.empty((1, fr.P, sc.D), dtype=torch.bfloat16, device=dev)
    fr.decode(F, codebook=fr.scene.codebook.to(torch.bfloat16), from_bf16=True)
    rel = torch.empty((1, 1, fr.P), dtype=torch.float32, device=dev)
    fr.query(torch.as_tensor(text, device=dev), rel, compute=Lb.LSV2_BF16, from_bf16=True)
    fr.check()
    r = O.render(sc, cam)
    Wo = r.blend.out[0]
    ok = r.blend.margin > 1e-4
    S = sc.codebook[0].astype(np.float64)
    stats = {k: {"max": 0.0, "sum": 0.0, "max_ok": 0.0, "sum_ok": 0.0, "n": 0, "n_ok": 0} for k in ("W", "F", "rel")}

    def acc(name, err, okm):
        d = stats[name]
        d["max"] = max(d["max"], float(err.max()))
        d["sum"] += float(err.sum())
        d["n"] += err.size
        e2 = err[okm]
        if e2.size:
            d["max_ok"] = max(d["max_ok"], float(e2.max()))
            d["sum_ok"] += float(e2.sum())
            d["n_ok"] += e2.size

    for p0 in range(0, fr.P, chunk):
        p1 = min(fr.P, p0 + chunk)
        okc = ok[p0:p1]
        Wg = fr.coeff16[0, p0:p1].float().cpu().numpy().astype(np.float64)
        acc("W", np.abs(Wg - Wo[p0:p1]), np.repeat(okc[:, None], Wg.shape[1], 1))
        Fo = Wo[p0:p1] @ S
        Fg = F[0, p0:p1].float().cpu().numpy().astype(np.float64)
        acc("F", np.abs(Fg - Fo), np.repeat(okc[:, None], Fg.shape[1], 1))
        ro = O.relevancy(Fo[None], text, 10.0)[0, 0]
        acc("rel", np.abs(rel[0, 0, p0:p1].cpu().numpy().astype(np.float64) - ro), okc)
    out = {"workload": "2,000 Gaussians, 1 level, K=4, L=64, D=512, 1440x1080 (the tiny scene at full size), "
                       "1 query + 4 negatives, tau = 10",
           "path": "FP32 blend stored as BF16; BF16 tensor-core decode (BF16 F) and relevancy (FP32 accumulation)",
           "knife_edge_pixels": int((~ok).sum()), "pixels": int(fr.P)}
    for k, d in stats.items():
        out[k] = {"max_abs": d["max"], "mean_abs": d["sum"] / max(1, d["n"]),
                  "max_abs_excl_knife_edge": d["max_ok"], "mean_abs_excl_knife_edge": d["sum_ok"] / max(1, d["n_ok"])}
    return out


# ----------------------------------------------------------------------------- speed ablation
def ablation_section(dev, reps: int = 10):
    """The paper's speed ablation on B300 (Table 9 and the K ablation): at 300k Gaussians, three
    levels, 1440x1080, the splat (record packing + blend) with K = 2, 4, 6, 8 nonzeros per level,
    the dense blend over all 64 coefficients per level ("Sparse, not Efficient") at K = 4, and the
    splat with codebooks of L = 32, 64, 128 entries at K = 4.  Same Gaussians for every K and L;
    L2 flushed between repetitions."""
    import torch
    import lsv2_synth as syn
    from paper_2507_07136_b300.pipeline import DeviceScene, Frame

    _, cam, _ = syn.at_scale()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(fn):
        for _ in range(3):
            fn()
            flush.fill_(1)
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(reps):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            fn()
            e.record()
            flush.fill_(1)
            torch.cuda.synchronize()
            tot += s.elapsed_time(e)
        return tot / reps

    out = {"workload": "300k Gaussians, 3 levels, L=64, 1440x1080 (the at-scale frame)", "splat_ms": {}}
    for K in (2, 4, 6, 8):
        sc = syn.make_scene(300_000, 3, K=K)
        fr = Frame(DeviceScene.from_numpy(sc, device=dev), cam, device=dev)
        fr.render()
        fr.check()
        out["splat_ms"][str(K)] = timed(fr.splat)
        if K == 4:
            out["dense_ms"] = timed(fr.splat_dense)
        fr.check()
        del fr
        torch.cuda.empty_cache()
    out["dense_over_sparse"] = out["dense_ms"] / out["splat_ms"]["4"]
    # the codebook size at K = 4: the blend's work is the same, the map it writes is L columns wide
    out["splat_ms_by_L"] = {"64": out["splat_ms"]["4"]}
    for Lc in (32, 128):
        sc = syn.make_scene(300_000, 3, L=Lc)
        fr = Frame(DeviceScene.from_numpy(sc, device=dev), cam, device=dev)
        fr.render()
        fr.check()
        out["splat_ms_by_L"][str(Lc)] = timed(fr.splat)
        fr.check()
        del fr
        torch.cuda.empty_cache()
    out["paper_a100_ms"] = {"dense (Sparse, not Efficient)": 5.3, "sparse (Efficient)": 2.0}
    return out


def backward_section(dev, reps: int = 10):
    """The differentiation workload (100,000 Gaussians, one level, K = 4, 720x540, L1 loss against a
    seeded N(0, 0.05^2) target of D = 512 features): the forward (project, bin, FP32 splat), the
    fused decode + L1 + adjoint kernel (lsv2_l1_decode_backward: F recomputed, dLoss/dW and
    dLoss/dS in one pass, F never stored) and the splat and projection adjoints
    (lsv2_splat_backward), each CUDA-event timed with L2 flushed and the gradient buffers zeroed
    before it; `step_ms` is one whole training step (forward, both adjoints, the zeroing)."""
    import torch
    import lsv2_synth as syn
    from paper_2507_07136_b300 import _lib as Lb
    from paper_2507_07136_b300.pipeline import DeviceScene, Frame, _ptr
    sc, cam = syn.differentiation()
    scene = DeviceScene.from_numpy(sc, device=dev)
    fr = Frame(scene, cam, device=dev)
    target = torch.as_tensor(syn.l1_target(cam), device=dev).contiguous()
    P, lev, D, n = fr.P, scene.levels, scene.D, scene.n
    loss = torch.zeros(1, device=dev)
    dcoeff = torch.empty_like(fr.coeff)
    dcb = torch.zeros_like(scene.codebook)
    grads = [torch.zeros_like(scene.weights), torch.zeros(n, device=dev), torch.zeros_like(scene.means),
             torch.zeros_like(scene.scales), torch.zeros_like(scene.quats)]
    ws_bytes = Lb.lsv2_splat_backward_workspace_bytes(n)
    ws = torch.empty(max(ws_bytes, 16), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream().cuda_stream

    def zero_l1():
        loss.zero_()
        dcb.zero_()

    def zero_bwd():
        for t in grads:
            t.zero_()

    def l1():
        Lb.lsv2_l1_decode_backward(lev, P, 64, D, _ptr(fr.coeff), _ptr(scene.codebook), _ptr(target), _ptr(loss),
                                   _ptr(dcoeff), _ptr(dcb), _ptr(fr.status), st)

    def bwd():
        Lb.lsv2_splat_backward(fr.ccam, n, _ptr(scene.means), _ptr(scene.scales), _ptr(scene.quats), fr.proj,
                               _ptr(fr.tile_ranges), _ptr(fr.gauss_ids), scene.levels, scene.K, 64, _ptr(scene.idx),
                               _ptr(scene.weights), _ptr(fr.final_T), _ptr(fr.n_last), _ptr(dcoeff), _ptr(ws),
                               ws_bytes, *[_ptr(t) for t in grads], _ptr(fr.status), st)

    def step():
        fr.render()
        zero_l1()
        l1()
        zero_bwd()
        bwd()

    def timed(fn, before=None):
        for _ in range(3):
            if before:
                before()
            fn()
        ts = []
        for _ in range(reps):
            flush.fill_(1)
            if before:
                before()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.mean(ts))

    fwd_ms = timed(fr.render)
    l1_ms = timed(l1, zero_l1)
    bwd_ms = timed(bwd, zero_bwd)
    step_ms = timed(step)
    fr.check()
    pk, pk_kind = peaks()
    l1_flop = P * lev * 3 * 2 * 64 * D        # F = W S, dW = G_F S^T, dS += W^T G_F per pixel
    l1_tf = l1_flop / (l1_ms * 1e-3) / 1e12
    # the adjoint's bound: the target it streams, W read and dLoss/dW written (F is recomputed)
    l1_bytes = P * lev * (D * 4 + 64 * 4 + 64 * 4)
    l1_gbs = l1_bytes / (l1_ms * 1e-3) / 1e9
    inst = int(fr.num_instances.item())
    bwd_bytes = P * lev * 64 * 4 + P * 8 + inst * 4 + n * (lev * scene.K * 5 + 44) + n * (lev * scene.K + 11) * 4
    bwd_gbs = bwd_bytes / (bwd_ms * 1e-3) / 1e9
    return {"workload": "100,000 Gaussians, 1 level, K = 4, L = 64, D = 512, 720x540, L1 loss against a seeded "
                        "target; gradients of weights, codebook, opacities, means, scales, quaternions",
            "forward_ms": fwd_ms, "l1_decode_backward_ms": l1_ms, "splat_backward_ms": bwd_ms, "step_ms": step_ms,
            "steps_per_s": 1e3 / step_ms, "instances": inst,
            "l1_decode_backward": {"bound": "hbm", "achieved": l1_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                                   "frac": l1_gbs / pk["hbm_gbs"], "algorithmic_bytes": l1_bytes,
                                   "peak_source": pk_kind,
                                   "tensor": {"achieved": l1_tf, "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                                              "frac": l1_tf / pk["bf16_tflops"], "algorithmic_flop": l1_flop,
                                              "note": "the three products counted once; the kernel issues them "
                                                      "as BF16 hi/lo splits (3 + 2 + 2 MMAs per product term)"}},
            "splat_backward": {"bound": "hbm", "achieved": bwd_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                               "frac": bwd_gbs / pk["hbm_gbs"], "algorithmic_bytes": bwd_bytes,
                               "peak_source": pk_kind,
                               "note": "bound by its atomics and per-pixel latency, not HBM"}}


def decoder_path_section(dev, v2_render_decode_ms: float | None = None, reps: int = 10,
                         block_sizes=(1048576, 4194304, -1)):
    """Table 1's contrast on B300: the decoder-based path (LangSplat*: a d = 3 latent per level
    rendered by Eq. 4, then the MLP decoder g_d to 512-d features for every pixel and level) against
    LangSplatV2's render + linear decode (Eq. 7), both at the at-scale frame (300,000 Gaussians,
    three levels, 1440x1080).  The latent render is the library's splat at L = 8; the decoder is
    lsv2_mlp_decode over 4.67 M rows of the widths 8-16-32-64-128-256-256-512: one cuBLASLt GEMM per
    layer over row blocks of the given size, and block_rows -1 (LSV2_MLP_FUSED) the fused
    tensor-core kernel (one persistent launch, activations on chip).  Each timed as one CUDA graph;
    L2 flushed between repetitions; the line reports the fastest."""
    import torch
    import lsv2_synth as syn
    from paper_2507_07136_b300.decoder_path import Decoder, DecoderFrame
    from paper_2507_07136_b300.pipeline import DeviceScene

    sc, cam, lat, layers = syn.latent_at_scale()
    ds = DeviceScene.from_numpy(sc, device=dev)
    dec = Decoder(layers, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    F = torch.empty((sc.levels, cam.num_pixels, dec.out_width), dtype=torch.bfloat16, device=dev)
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(3):
            fn()
            flush.fill_(1)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            flush.fill_(1)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.mean(ts))

    def graph_of(fn):
        fn()                       # the first call of each shape plans the library's GEMMs on the host
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        return g

    decode_ms, fr = {}, None
    for block_rows in block_sizes:
        fr = DecoderFrame(ds, torch.as_tensor(lat), dec, cam, block_rows=block_rows, device=dev)
        fr.render()
        fr.check()
        g = graph_of(lambda: fr.decode(F))
        decode_ms[str(block_rows)] = timed(g.replay)
        fr.check()
        del g
    best = min(decode_ms, key=decode_ms.get)
    render = {"project": timed(fr.project), "bin_sort": timed(fr.bin_sort), "latent_splat": timed(fr.splat)}
    fr.check()
    render_ms = sum(render.values())
    rows = sc.levels * cam.num_pixels
    flop = rows * dec.flops_per_row()
    pk, pk_kind = peaks()
    tf = flop / (decode_ms[best] * 1e-3) / 1e12
    byts = rows * (8 * 4 + dec.out_width * 2)    # the F32 latent map in, the BF16 features out
    kernel = ("mlp_fused_kernel (tcgen05, persistent, activations in shared memory) + mlp_pack_kernel"
              if best == "-1" else "cuBLASLt BF16 GEMMs (library) + to_bf16_kernel")
    out = {"workload": "300k Gaussians, 3 levels, 1440x1080; latent d = 3 per level (padded to 8 channels), "
                       "decoder 8-16-32-64-128-256-256-512 (ReLU), BF16 out",
           "render_ms": render, "decode_ms_by_block_rows": decode_ms,
           "block_rows_note": "-1 = the fused tensor-core kernel; > 0 = library GEMMs over row blocks of that size",
           "block_rows": int(best),
           "render_decode_ms": render_ms + decode_ms[best],
           "render_decode_fps": 1e3 / (render_ms + decode_ms[best]),
           "decode": {"bound": "tensor", "achieved": tf, "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                      "frac": tf / pk["bf16_tflops"], "algorithmic_flop": flop, "algorithmic_bytes": byts,
                      "hbm_floor_ms": byts / pk["hbm_gbs"] / 1e6, "peak_source": pk_kind + " (burst)",
                      "kernel": kernel},
           "paper_a100_ms": {"LangSplat* rendering": 2.0, "LangSplat* decoding": 83.1,
                             "LangSplatV2 rendering": 2.0, "LangSplatV2 decoding": 0.1}}
    if "-1" in decode_ms and len(decode_ms) > 1:
        lib_best = min((v for k, v in decode_ms.items() if k != "-1"))
        out["fused_kernel"] = {"ms": decode_ms["-1"], "library_ms": lib_best,
                               "tflops": flop / (decode_ms["-1"] * 1e-3) / 1e12,
                               "frac": flop / (decode_ms["-1"] * 1e-3) / 1e12 / pk["bf16_tflops"],
                               "workspace_bytes": dec.workspace_bytes(rows, 0, -1),
                               "library_workspace_bytes": dec.workspace_bytes(rows, 0, int(min(
                                   (k for k in decode_ms if k != "-1"), key=decode_ms.get)))}
    if v2_render_decode_ms is not None:
        out["langsplatv2_render_decode_ms"] = v2_render_decode_ms
        out["decoder_over_v2"] = out["render_decode_ms"] / v2_render_decode_ms
    del fr, F
    torch.cuda.empty_cache()
    return out


def mlp_profile(dev, steps: int, warmup: int, rows: int = 1 << 20):
    """The decoder MLP alone (the workload's widths 8-16-32-64-128-256-256-512) on `rows` synthetic
    latent rows (standard normal in the 3 latent channels): the fused kernel (block_rows -1,
    LSV2_MLP_FUSED), eager launches timed with CUDA events.  A small case for a capture of the fused
    kernel (1 GB of output)."""
    import torch
    import lsv2_synth as syn
    from paper_2507_07136_b300.decoder_path import LATENT_CHANNELS, Decoder
    dec = Decoder(syn.decoder_mlp(), device=dev)
    gen = torch.Generator(device=dev).manual_seed(7)
    x = torch.zeros((rows, LATENT_CHANNELS), device=dev)
    x[:, :3] = torch.randn((rows, 3), generator=gen, device=dev)
    y = torch.empty((rows, dec.out_width), dtype=torch.bfloat16, device=dev)
    ws = torch.empty(dec.workspace_bytes(rows, 0, -1), dtype=torch.uint8, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    ts = []
    for i in range(warmup + steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        dec(x, y, ws, -1, None, st)
        b.record(stream)
        torch.cuda.synchronize()
        if i >= warmup:
            ts.append(a.elapsed_time(b))
    if int(st.item()) != 0:
        raise RuntimeError(f"device status {int(st.item())}")
    ms = float(np.mean(ts))
    return {"rows": rows, "ms": ms, "tflops": rows * dec.flops_per_row() / (ms * 1e-3) / 1e12,
            "device_gb": round(torch.cuda.max_memory_allocated(dev) / 1e9, 2)}


# ----------------------------------------------------------------------------- batched views
def sparsify_section(dev, reps: int = 20):
    """Sec. 3.3 sparse coefficients on the at-scale shape (300,000 Gaussians x 3 levels of 64 logits,
    K = 4): forward (top K + renormalised softmax) and backward, each against the HBM roofline of
    its algorithmic bytes (the logits read, or their gradient written, dominate)."""
    import torch
    from paper_2507_07136_b300 import _lib as Lb
    from paper_2507_07136_b300.pipeline import _ptr
    rows, Lz, K = 900_000, 64, 4
    g = torch.Generator(device=dev).manual_seed(5)
    z = torch.randn((rows, Lz), generator=g, device=dev) * 2
    idx = torch.empty((rows, K), dtype=torch.uint8, device=dev)
    w = torch.empty((rows, K), device=dev)
    dw = torch.randn((rows, K), generator=g, device=dev)
    dz = torch.empty((rows, Lz), device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream().cuda_stream

    def timed(fn):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.mean(ts))

    f_ms = timed(lambda: Lb.lsv2_sparsify(rows, Lz, K, _ptr(z), _ptr(idx), _ptr(w), st))
    b_ms = timed(lambda: Lb.lsv2_sparsify_backward(rows, Lz, K, _ptr(idx), _ptr(w), _ptr(dw), _ptr(dz), st))
    pk, pk_kind = peaks()
    f_bytes = rows * (Lz * 4 + K * 5)
    b_bytes = rows * (K * 9 + Lz * 4)
    f_gbs, b_gbs = f_bytes / (f_ms * 1e-3) / 1e9, b_bytes / (b_ms * 1e-3) / 1e9
    return {"workload": "900,000 rows (300k Gaussians x 3 levels) of 64 logits, K = 4",
            "forward_ms": f_ms, "backward_ms": b_ms,
            "forward": {"bound": "hbm", "achieved": f_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                        "frac": f_gbs / pk["hbm_gbs"], "algorithmic_bytes": f_bytes, "peak_source": pk_kind},
            "backward": {"bound": "hbm", "achieved": b_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": b_gbs / pk["hbm_gbs"], "algorithmic_bytes": b_bytes, "peak_source": pk_kind}}


def batched_section(dev, reps: int = 5, rank: int = 0, world: int = 1):
    """500,000 Gaussians, three levels, 16 views (4 each at 1440x1080, 960x720, 640x480, 320x240),
    64 queries with four negatives each: one CUDA-graph launch of lsv2_query_views (tile shape and
    staging batch from the autotuner) against sequential single-view pipelines.  With several
    ranks the views are sharded by pixel count (no collective on the data path) and the batch time
    is the maximum over ranks."""
    import torch
    import torch.distributed as dist
    import lsv2_synth as syn
    from paper_2507_07136_b300 import _lib as Lb
    from paper_2507_07136_b300.pipeline import DeviceScene, Frame
    from paper_2507_07136_b300.shard import rank_views
    from paper_2507_07136_b300.views import ViewsBatch, autotune

    sc, all_cams, text = syn.batched()
    n_views = len(all_cams)
    mine = rank_views([c.width * c.height for c in all_cams], rank, world)
    cams = [all_cams[v] for v in mine]
    scene = DeviceScene.from_numpy(sc, device=dev)
    t = torch.as_tensor(text, device=dev)
    tile, batch = autotune(scene, cams, t, reps=3)
    vb = ViewsBatch(scene, cams, text.shape[0], text.shape[1] - 1, tile=tile, stage_batch=batch)
    vb.capture(t)
    for _ in range(2):
        vb.replay()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        vb.replay()
    e.record()
    torch.cuda.synchronize()
    vb.check()
    batched_ms = s.elapsed_time(e) / reps
    inst = int(vb.num_instances.item())
    pix = sum(vb.P)
    rel_elems = vb.rel.numel()
    del vb
    torch.cuda.empty_cache()
    # 16 sequential single-view pipelines (same cameras, same tile shape), eager launches
    frames = [Frame(scene, c.with_tile(*tile), device=dev) for c in cams]
    rels = [torch.empty((text.shape[0], scene.levels, f.P), dtype=torch.bfloat16, device=dev) for f in frames]

    def sequential():
        for f, r in zip(frames, rels):
            f.render()
            f.query(t, r, compute=Lb.LSV2_BF16)
    sequential()
    torch.cuda.synchronize()
    s.record()
    for _ in range(reps):
        sequential()
    e.record()
    torch.cuda.synchronize()
    for f in frames:
        f.check()
    seq_ms = s.elapsed_time(e) / reps
    del frames, rels
    torch.cuda.empty_cache()
    # the relevancy part alone at the batch's size: one lsv2_query (BF16) over a coefficient map of
    # all views' pixels and the batch's 64 queries (the same kernels and query groups the batched
    # call runs over its per-view maps)
    Q = text.shape[0]
    W16 = (torch.rand((scene.levels, pix, 64), device=dev) * 0.05).to(torch.bfloat16)
    rel16 = torch.empty((Q, scene.levels, pix), dtype=torch.bfloat16, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    qws_bytes = Lb.lsv2_query_workspace_bytes(scene.levels, 64, Q, text.shape[1] - 1)
    qws = torch.empty(qws_bytes, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream().cuda_stream

    def rel_call():
        Lb.lsv2_query(scene.levels, pix, 64, scene.D, W16.data_ptr(), Lb.LSV2_BF16, scene.codebook.data_ptr(), Q,
                      text.shape[1] - 1, t.data_ptr(), 10.0, qws.data_ptr(), qws_bytes, rel16.data_ptr(), Lb.LSV2_BF16,
                      Lb.LSV2_BF16, status.data_ptr(), st)
    rel_call()
    torch.cuda.synchronize()
    s.record()
    for _ in range(reps):
        rel_call()
    e.record()
    torch.cuda.synchronize()
    rel_ms = s.elapsed_time(e) / reps
    assert int(status.item()) == 0
    del W16, rel16, qws
    torch.cuda.empty_cache()
    pk, pk_kind = peaks()
    rel_flop = 2.0 * pix * scene.levels * 64 * (64 + (text.shape[1]) * Q)
    rel_bytes = scene.levels * pix * 64 * 2 + Q * scene.levels * pix * 2
    if world > 1:
        batched_ms, seq_ms, rel_ms = max_over_ranks([batched_ms, seq_ms, rel_ms], world, dev)
        cnt = torch.tensor([inst, pix, rel_elems], dtype=torch.int64, device=dev)
        dist.all_reduce(cnt)
        inst, pix, rel_elems = (int(v) for v in cnt.tolist())
    nq = n_views * text.shape[0]
    return {"workload": "500k Gaussians, 3 levels, 16 views (4 each 1440x1080, 960x720, 640x480, 320x240), "
                        "64 queries x (1 + 4 negatives)",
            "queries_per_s": nq * 1e3 / batched_ms, "ms_per_batch": batched_ms,
            "sequential_ms": seq_ms, "sequential_queries_per_s": nq * 1e3 / seq_ms,
            "speedup_vs_sequential": seq_ms / batched_ms, "tile": list(tile), "stage_batch": batch,
            "pixels": pix, "instances": inst, "relevancy_values": rel_elems, "launch": "one CUDA graph",
            "relevancy_ms": rel_ms, "relevancy_share": rel_ms / batched_ms,
            "relevancy_roofline": {
                "tensor": {"achieved": rel_flop / (rel_ms * 1e-3) / 1e12, "peak": pk["bf16_tflops_sustained"],
                           "unit": "TFLOP/s", "frac": rel_flop / (rel_ms * 1e-3) / 1e12 / pk["bf16_tflops_sustained"],
                           "algorithmic_flop": rel_flop, "peak_source": pk_kind + " (sustained BF16)"},
                "hbm": {"achieved": rel_bytes / (rel_ms * 1e-3) / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                        "frac": rel_bytes / (rel_ms * 1e-3) / 1e9 / pk["hbm_gbs"], "algorithmic_bytes": rel_bytes,
                        "peak_source": pk_kind},
                "note": "relevancy of all views' pixels for the 64 queries (2 P levels 64 (64 + 5 Q) flop with "
                        "the 64 factor columns counted once; BF16 W read + BF16 relevancy write), one lsv2_query call "
                        "timed alone"}}


# ----------------------------------------------------------------------------- GPU arm
def profile_stage(args, frame, scene, text, dev):
    """One stage of the at-scale frame, repeated, for a profiler: the device holds the scene, the
    frame's buffers and the stage's output only (the decode writes one level's 1.59 GB feature
    map: the same kernel over the level's 1,555,200 pixels, its grid spread over one level)."""
    import torch
    from paper_2507_07136_b300 import _lib as Lb
    from paper_2507_07136_b300.pipeline import _ptr, L_CODEBOOK
    frame.project()
    frame.bin_sort()
    frame.splat_bf16()
    P, D = frame.P, scene.D
    if args.profile == "project":
        fn = frame.project
    elif args.profile == "bin":
        fn = frame.bin_sort
    elif args.profile == "splat":
        fn = frame.splat_bf16
    elif args.profile == "decode":
        F = torch.empty((1, P, D), dtype=torch.bfloat16, device=dev)
        cb16 = scene.codebook[:1].to(torch.bfloat16).contiguous()
        stream = torch.cuda.current_stream().cuda_stream

        def fn():
            Lb.lsv2_decode(1, P, L_CODEBOOK, D, _ptr(frame.coeff16), Lb.LSV2_BF16, _ptr(cb16), Lb.LSV2_BF16, _ptr(F),
                           Lb.LSV2_BF16, _ptr(frame.status), stream)
    elif args.profile == "query32":
        # the batched path's query group: 32 queries x (1 + 4 negatives), BF16 relevancy out
        g = torch.Generator(device=dev).manual_seed(11)
        text_d = torch.randn((32, text.shape[1], D), generator=g, device=dev)
        rel = torch.empty((32, scene.levels, P), dtype=torch.bfloat16, device=dev)

        def fn():
            frame.query(text_d, rel, compute=Lb.LSV2_BF16, from_bf16=True)
    else:
        text_d = torch.as_tensor(text, device=dev)
        rel = torch.empty((text.shape[0], scene.levels, P), dtype=torch.float32, device=dev)

        def fn():
            frame.query(text_d, rel, compute=Lb.LSV2_BF16, from_bf16=True)
    for _ in range(args.warmup + args.steps):
        fn()
    frame.check()
    print(json.dumps({"profile": args.profile, "launches": args.warmup + args.steps,
                      "device_gb": round(torch.cuda.max_memory_allocated(dev) / 1e9, 2)}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32-path", action="store_true", help="skip the plain FP32 comparison measurement")
    ap.add_argument("--no-batched", action="store_true", help="skip the 16-view x 64-query batched measurement")
    ap.add_argument("--no-ablation", action="store_true", help="skip the sparse/dense and K speed ablation")
    ap.add_argument("--no-decoder-path", action="store_true",
                    help="skip the decoder-based (LangSplat*) comparison measurement")
    ap.add_argument("--profile", choices=["project", "bin", "splat", "decode", "query", "query32", "backward", "sparsify", "decoder", "mlp",
                             "batched"], default=None,
                    help="for a profiler capture: prepare the at-scale frame, then run only this stage "
                         "(--warmup + --steps launches) with only the buffers it needs; `backward` runs the "
                         "training-step measurement of the differentiation workload instead, `decoder` the decoder-based "
                         "comparison path (--steps repetitions), `batched` eager lsv2_query_views calls of the "
                         "16-view, 64-query workload (16x16 tiles, 32 records per stage); prints one status line")
    ap.add_argument("--precision", action="store_true",
                    help="print the precision workload's max/mean errors against the FP64 oracle (about a minute of CPU)")
    ap.add_argument("--cpu-pixels", type=int, default=2000,
                    help="pixels the FP64 oracle blends, decodes and queries per CPU-baseline sample")
    args = ap.parse_args()
    rc = spawn_ranks(args.gpus, sys.argv[1:])
    if rc is not None:
        sys.exit(rc)
    if args.impl == "reference":
        reference_arm(args)
        return

    import torch
    import torch.distributed as dist
    import lsv2_synth as syn
    from paper_2507_07136_b300.pipeline import DeviceScene, Frame
    from paper_2507_07136_b300 import build as _  # noqa: F401

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    assert args.warmup >= 3, "at least 3 warm-up steps"
    dev = torch.device("cuda", local)
    if args.profile == "backward":
        r = backward_section(dev, reps=args.steps)
        print(json.dumps({"profile": "backward", "forward_ms": r["forward_ms"],
                          "l1_decode_backward_ms": r["l1_decode_backward_ms"],
                          "splat_backward_ms": r["splat_backward_ms"], "step_ms": r["step_ms"]}), flush=True)
        return
    if args.precision:
        print(json.dumps({"precision": precision_report(dev)}), flush=True)
        return
    if args.profile == "decoder":
        r = decoder_path_section(dev, reps=args.steps)
        print(json.dumps({"profile": "decoder", **r}), flush=True)
        return
    if args.profile == "mlp":
        print(json.dumps({"profile": "mlp", **mlp_profile(dev, args.steps, args.warmup)}), flush=True)
        return
    if args.profile == "batched":
        from paper_2507_07136_b300.views import ViewsBatch
        sc, cams, text = syn.batched()
        vb = ViewsBatch(DeviceScene.from_numpy(sc, device=dev), cams, text.shape[0], text.shape[1] - 1, tile=(16, 16),
                        stage_batch=32, device=dev)
        t = torch.as_tensor(text, device=dev)
        for _ in range(args.warmup + args.steps):
            vb.run(t)
        vb.check()
        print(json.dumps({"profile": "batched", "launches": args.warmup + args.steps,
                          "instances": int(vb.num_instances.item()),
                          "device_gb": round(torch.cuda.max_memory_allocated(dev) / 1e9, 2)}), flush=True)
        return
    if args.profile == "sparsify":
        r = sparsify_section(dev, reps=args.steps)
        print(json.dumps({"profile": "sparsify", "forward_ms": r["forward_ms"], "backward_ms": r["backward_ms"],
                          "device_gb": round(torch.cuda.max_memory_allocated(dev) / 1e9, 2)}), flush=True)
        return

    from paper_2507_07136_b300 import _lib as Lb
    sc, cam, text = syn.at_scale()
    scene = DeviceScene.from_numpy(sc, device=dev)
    frame = Frame(scene, cam, device=dev)
    P = cam.num_pixels
    levels, D = scene.levels, scene.D
    if args.profile:
        profile_stage(args, frame, scene, text, dev)
        return
    F = torch.empty((levels, P, D), dtype=torch.bfloat16, device=dev)
    cb16 = scene.codebook.to(torch.bfloat16)
    text_d = torch.as_tensor(text, device=dev)
    rel = torch.empty((text.shape[0], levels, P), dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    from paper_2507_07136_b300.pipeline import PostResult
    post_out = PostResult(text.shape[0], levels, cam.height, cam.width, dev)
    stages = ["project", "bin_sort", "splat", "decode", "query", "post"]
    # the tensor-core path: the splat writes the coefficient map as BF16 (what the decode and the
    # relevancy round it to before their products), the decode and the relevancy read it
    # the relevancy buffer the step writes (the end-to-end run alternates two); whether the query's
    # operands are prepared on a side stream while the frame renders
    cur = {"rel": rel, "prep": True}
    side = torch.cuda.Stream(device=dev)
    fns = {"project": frame.project, "bin_sort": frame.bin_sort, "splat": frame.splat_bf16,
           "decode": lambda: frame.decode(F, codebook=cb16, from_bf16=True),
           "query": lambda: frame.query(text_d, cur["rel"], compute=Lb.LSV2_BF16, from_bf16=True, prepared=True),
           "post": lambda: frame.postprocess(cur["rel"], k=POST_WINDOW, mode=Lb.LSV2_POST_LERF,
                                             threshold=POST_THRESHOLD, out=post_out)}
    # kernels per stage: project; hist/column/scan/scatter + warp, block and large-tile sorts (bin);
    # pack + splat; decode; prepare + factor + query; init + box filter + select + mask (post)
    launches_per_step = {"project": 1, "bin_sort": 7, "splat": 2, "decode": 1, "query": 3, "post": 4}

    def step(ev=None):
        main = torch.cuda.current_stream()
        joined = None
        if cur["prep"]:
            # the query's operands ([S S^T | S t] and the factor of S S^T) depend only on the
            # codebook and the texts: formed on a side stream while the frame renders
            fork = torch.cuda.Event()
            fork.record(main)
            side.wait_event(fork)
            with torch.cuda.stream(side):
                frame.query_prepare(text_d, compute=Lb.LSV2_BF16)
            joined = torch.cuda.Event()
            joined.record(side)
        for i, s in enumerate(stages):
            if ev is not None:
                ev[i].record(stream)
            if s == "query" and joined is not None:
                main.wait_event(joined)
            fns[s]()
        if ev is not None:
            ev[len(stages)].record(stream)

    def timed(n_steps):
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(stages) + 1)] for _ in range(n_steps)]
        for k in range(n_steps):
            step(evs[k])
            flush.fill_(1)
        torch.cuda.synchronize()
        st = {s: float(np.mean([evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(n_steps)]))
              for i, s in enumerate(stages)}
        return st, float(np.mean([evs[k][0].elapsed_time(evs[k][len(stages)]) for k in range(n_steps)]))

    def capture(rel_buf, text_from=None):
        """The whole step as one CUDA graph writing rel_buf (every stage is stream-ordered library
        calls on preallocated buffers, so it captures as is); with text_from (pinned host memory)
        the graph starts with the copy of the step's text embeddings to the device."""
        cur["rel"] = rel_buf
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            if text_from is not None:
                text_d.copy_(text_from, non_blocking=True)
            step()
        return g

    def timed_graph(g, n_steps):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_steps)]
        for k in range(n_steps):
            evs[k][0].record(stream)
            g.replay()
            evs[k][1].record(stream)
            flush.fill_(1)
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in evs]))

    for _ in range(args.warmup):
        step()
        flush.fill_(1)
    frame.check()
    graph = capture(rel)
    for _ in range(args.warmup):
        graph.replay()
        flush.fill_(1)
    frame.check()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        step_ms = timed_graph(graph, args.steps)
        t_wall = time.perf_counter() - t_wall
    if world > 1:
        dist.barrier()
    frame.check()
    del graph   # it holds pointers to F, which the FP32 comparison below reallocates
    # the per-stage breakdown: the same step with eager launches and events between the stages
    stage_ms, eager_ms = timed(max(3, args.steps // 2))
    step_ms = max_over_ranks([step_ms], world, dev)[0]
    value = world * 1e3 / step_ms

    # ---- the plain FP32 GPU form (CUDA-core decode to an FP32 feature map), for comparison ----
    fp32 = None
    if not args.no_fp32_path:
        del F
        F32 = torch.empty((levels, P, D), dtype=torch.float32, device=dev)
        fns["splat"] = frame.splat
        fns["decode"] = lambda: frame.decode(F32)
        fns["query"] = lambda: frame.query(text_d, rel)
        cur["prep"] = False
        timed(2)
        st32, ms32 = timed(max(3, args.steps // 4))
        fp32 = {"ms_per_step": ms32, "fps": 1e3 / ms32, "stages_ms": st32}
        del F32
        F = torch.empty((levels, P, D), dtype=torch.bfloat16, device=dev)
        fns["splat"] = frame.splat_bf16
        fns["decode"] = lambda: frame.decode(F, codebook=cb16, from_bf16=True)
        fns["query"] = lambda: frame.query(text_d, rel, compute=Lb.LSV2_BF16, from_bf16=True, prepared=True)
        cur["prep"] = True

    # ---- splat + decode + query in one kernel (lsv2_render_fused): W never leaves the SM ----
    fused_ms = None
    if not args.no_fp32_path:
        for _ in range(3):
            frame.render_fused(F, text_d, rel)
            flush.fill_(1)
        torch.cuda.synchronize()
        tot = 0.0
        n_f = max(3, args.steps // 4)
        for _ in range(n_f):
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            frame.render_fused(F, text_d, rel)
            s1.record(stream)
            flush.fill_(1)
            torch.cuda.synchronize()
            tot += s0.elapsed_time(s1)
        frame.check()
        fused_ms = tot / n_f
        frame.splat()   # restore the coefficient map the timed step left

    # ---- end to end through the C ABI with host buffers ----
    # Every step copies its text in and its relevancy maps out (pinned host buffers).  The copy-out
    # of step i runs on a copy stream while step i + 1 computes: two device relevancy buffers
    # alternate, and a buffer is reused only after its previous copy-out has finished.
    text_h = torch.as_tensor(text).pin_memory()
    rels = [rel, torch.empty_like(rel)]
    rel_hs = [torch.empty(rel.shape, dtype=rel.dtype).pin_memory() for _ in range(2)]
    copy_stream = torch.cuda.Stream(device=dev)
    copied = [None, None]

    graphs = [capture(rels[0], text_h), capture(rels[1], text_h)]

    def e2e_step(i):
        b = i % 2
        if copied[b] is not None:
            stream.wait_event(copied[b])
        graphs[b].replay()   # host -> device copy of the text, then the step
        computed = torch.cuda.Event()
        computed.record(stream)
        copy_stream.wait_event(computed)
        with torch.cuda.stream(copy_stream):
            rel_hs[b].copy_(rels[b], non_blocking=True)
        copied[b] = torch.cuda.Event()
        copied[b].record(copy_stream)

    for i in range(2):
        e2e_step(i)
    torch.cuda.synchronize()
    e2e_steps = max(3, args.steps // 2)
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        e2e_step(i)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
    e2e_ms = max_over_ranks([e2e_ms], world, dev)[0]

    # ---- rooflines (algorithmic bytes per launch / CUDA-event duration) ----
    pk, pk_kind = peaks()
    inst = int(frame.num_instances.item())
    rec_bytes = Lb.lsv2_splat_workspace_bytes(scene.n, levels, scene.K)
    splat_bytes = levels * P * 64 * 2 + rec_bytes + inst * 4 + P * 8      # BF16 coefficient map
    decode_bytes = levels * P * (64 * 2 + D * 2)                          # BF16 W in, BF16 F out
    query_bytes = levels * P * 64 * 2 + text.shape[0] * levels * P * 4     # BF16 W in, FP32 relevancy out
    roofs = {
        "splat": {"bound": "hbm", "achieved": splat_bytes / (stage_ms["splat"] * 1e-3) / 1e9, "peak": pk["hbm_gbs"],
                  "unit": "GB/s", "traffic": TRAFFIC.get(SPLAT_KERNEL), "kernel": SPLAT_KERNEL,
                  "algorithmic_bytes": splat_bytes, "peak_source": pk_kind},
        "decode": {"bound": "hbm", "achieved": decode_bytes / (stage_ms["decode"] * 1e-3) / 1e9, "peak": pk["hbm_gbs"],
                   "unit": "GB/s", "traffic": TRAFFIC.get("decode_tc_kernel"), "kernel": "decode_tc_kernel",
                   "algorithmic_bytes": decode_bytes, "peak_source": pk_kind},
        # the stage's time is the relevancy kernel's: its operands ([S S^T | S t], then C with S S^T = C C^T)
        # are prepared on a side stream while the frame renders
        "query": {"bound": "hbm", "achieved": query_bytes / (stage_ms["query"] * 1e-3) / 1e9, "peak": pk["hbm_gbs"],
                  "unit": "GB/s", "traffic": TRAFFIC.get("query_pipe_kernel<3,1>"),
                  "kernel": "query_pipe_kernel<3,1>",
                  "algorithmic_bytes": query_bytes, "peak_source": pk_kind},
    }
    for k, r in roofs.items():
        r["frac"] = r["achieved"] / r["peak"]
    # the splat against the units its blend needs (FP32 pipe, MUFU ex2, accumulator accesses)
    rates = unit_rates(dev)
    roofs["splat_units"] = splat_alu_roofline(splat_work(sc, cam), levels, scene.K, stage_ms["splat"], rates)
    roofs["splat_units"]["kernel"] = SPLAT_KERNEL + " + record packing"
    dom = max(["splat", "decode"], key=lambda k: stage_ms[k])
    gpu_launches = sum(launches_per_step.values()) * args.steps

    line = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16", "data": "synthetic",
            "config": {"workload": "300k Gaussians, 3 levels, K=4, L=64, D=512, 1440x1080, 1 query + 4 negatives",
                       "path": "FP32 projection and splat (coefficient map stored as BF16); BF16 tensor-core decode "
                               "to a BF16 feature map and BF16 tensor-core relevancy (FP32 accumulation); "
                               "post-processing (LERF rule, "
                               f"{POST_WINDOW}x{POST_WINDOW} mean filter, level, point, mask at {POST_THRESHOLD})",
                       "parallelism": f"replicas x{world}",
                       "l2": "flushed between steps (256 MiB write, untimed)", "instances": inst,
                       "launch": "each step is one CUDA graph replay (stages_ms: the same step launched eagerly)"},
            "stages_ms": stage_ms,
            "eager_ms_per_step": eager_ms,
            "splat_decode_fps": 1e3 / (stage_ms["project"] + stage_ms["bin_sort"] + stage_ms["splat"] + stage_ms["decode"]),
            "query_fps": 1e3 / (stage_ms["project"] + stage_ms["bin_sort"] + stage_ms["splat"] + stage_ms["query"]
                                + stage_ms["post"]),
            "roofline": dict(roofs[dom]),
            "rooflines": roofs,
            "unit_rates": rates,
            "fp32_path": fp32,
            "fused_splat_decode_query_ms": fused_ms,
            "split_splat_decode_query_ms": stage_ms["splat"] + stage_ms["decode"] + stage_ms["query"],
            "e2e": {"value": world * 1e3 / e2e_ms, "unit": "frames/s", "h2d_bytes_per_step": text_h.numel() * 4,
                    "d2h_bytes_per_step": rel_hs[0].numel() * 4},
            "gpu_launches": gpu_launches,
            "clocks": clk.summary(),
            "wall_s_timed_region": t_wall}
    if not args.no_batched:
        del F
        torch.cuda.empty_cache()
        line["batched"] = batched_section(dev, rank=rank, world=world)
    if world == 1:
        line["sparsify"] = sparsify_section(dev)
        line["backward"] = backward_section(dev)
    if not args.no_ablation and world == 1:
        torch.cuda.empty_cache()
        line["ablation"] = ablation_section(dev)
    if not args.no_decoder_path and world == 1:
        torch.cuda.empty_cache()
        v2 = stage_ms["project"] + stage_ms["bin_sort"] + stage_ms["splat"] + stage_ms["decode"]
        line["decoder_path"] = decoder_path_section(dev, v2)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.cpu_pixels)
            line["cpu_baseline"]["tiny_full_frame"] = cpu_tiny_full_frame()
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
