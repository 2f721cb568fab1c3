"""The N > 1 path on the CPU: bench.py runs one rank per GPU, each on its own seeded mesh, with no
collective on the data path; the only communication is the barrier and the max-over-ranks time.
These tests run that host logic as two gloo ranks (127.0.0.1), and the reference arm under
torchrun with two processes (rank 0 prints the one JSON line, the other rank exits without work)."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local_ms = [120.0, 180.0][rank]          # the second rank is the slow one
        tmax = bench.max_over_ranks(local_ms, world)
        rate = bench.aggregate_rate(world, 10, tmax)
        items = list(range(11))
        mine = bench.shard(items, rank, world)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.rank_seed(rank))
        dist.barrier()
        q.put((rank, tmax, rate, gathered, seeds))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_rate_and_shards():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, tmax, rate, gathered, seeds in res:
        assert tmax == 180.0                                   # the slowest rank sets the time
        assert rate == pytest.approx(2 * 10 / 0.18)            # units of all ranks / that time
        flat = sorted(x for part in gathered for x in part)
        assert flat == list(range(11))                         # every unit once, no overlap
        assert seeds == [0, 1]                                 # distinct meshes per rank


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.aggregate_rate(1, 200, 2000.0) == 100.0
    assert bench.shard([1, 2, 3], 0, 1) == [1, 2, 3]


def test_reference_arm_under_torchrun_two_ranks():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--workload", "ico3"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["unit"] == "solves/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0
