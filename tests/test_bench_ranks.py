"""The N > 1 path of bench.py on CPU: replica timing reduced with a MAX over
two gloo ranks, the whole-job throughput, and the reference arm launched as
two ranks (only rank 0 works and prints)."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 250.0][rank]
        bench.barrier(world)
        tot = bench.max_over_ranks(local_ms, world, "cpu")
        out.put((rank, tot, bench.job_rate(1.0e9, world, tot * 1e-3)))
    finally:
        dist.destroy_process_group()


def test_max_over_two_gloo_ranks_and_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slowest rank's time; the job rate counts both ranks' work
    assert [r[1] for r in res] == [250.0, 250.0]
    assert res[0][2] == pytest.approx(2 * 1.0e9 / 0.25)


def _sum_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank holds the field of its own part of the sources
        part = torch.arange(6, dtype=torch.float64).reshape(2, 3) * (rank + 1) + 0.25 * rank
        bench.sum_over_ranks(part, world)
        out.put((rank, part.tolist()))
    finally:
        dist.destroy_process_group()


def test_source_parts_are_summed_over_two_gloo_ranks():
    """The one exchange of a source-partitioned solve: a sum all-reduce of
    the ranks' partial fields, every rank ending with the whole field."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_sum_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = (torch.arange(6, dtype=torch.float64).reshape(2, 3) * 3 + 0.25).tolist()
    assert res[0][1] == want and res[1][1] == want


def test_single_rank_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_rate(10.0, 1, 2.0) == 5.0
    t = torch.ones(3)
    assert bench.sum_over_ranks(t, 1) is t and t.tolist() == [1.0, 1.0, 1.0]


def test_reference_arm_as_two_ranks_prints_one_line():
    env = dict(os.environ)
    env.pop("WORLD_SIZE", None)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--side", "16", "--stations", "8", "--sample-obs", "64"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
