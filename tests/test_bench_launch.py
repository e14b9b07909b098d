"""The benchmark's multi-rank launch path on the CPU (no GPU): `bench.py --gpus N` started
outside a launcher runs N ranks under torch.distributed.run and reports the real world size,
and the timing each rank measures is reduced to the maximum over ranks before the job's
throughput (units of all ranks / that time) is formed."""
import json
import os
import socket
import subprocess
import sys
import time

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_gpus_2_outside_a_launcher_runs_two_ranks():
    """The reference arm (the FP64 oracle on rank 0, a tiny pixel sample) through the launch
    path: two ranks start, rank 0 alone prints one line, and it reports n_gpus = 2."""
    env = dict(os.environ)
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT"):
        env.pop(k, None)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--steps", "1", "--warmup", "0", "--cpu-pixels", "16"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2
    assert rec["ms_per_step"] > 0 and rec["value"] > 0
    assert rec["cpu_baseline"]["host"]["nproc"] >= 1
    # ms_per_step is the measured time of the sampled step, consistent with the whole run
    assert 0 < rec["frames_per_step"] < 1


def _rank(rank, world, port, out_q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    # a stub step whose duration differs per rank, timed between barriers as the GPU arm does
    dist.barrier()
    t0 = time.perf_counter()
    for _ in range(3):
        time.sleep(0.01 * (rank + 1))
    ms = (time.perf_counter() - t0) * 1e3 / 3
    dist.barrier()
    (job_ms,) = bench.max_over_ranks([ms], world)
    every = [None] * world
    dist.all_gather_object(every, ms)
    out_q.put((rank, ms, job_ms, max(every)))
    dist.destroy_process_group()


def test_two_gloo_ranks_report_the_maximum_time():
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    assert got[0][2] == got[1][2] == got[0][3]          # both ranks hold the maximum
    assert got[0][2] == pytest.approx(max(g[1] for g in got))
    assert got[1][1] > got[0][1]                         # rank 1's stub step is the slower one
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([1.5, 2.0], 1) == [1.5, 2.0]
