"""The bench's multi-GPU bookkeeping on CPU: two gloo ranks.  Ranks evaluate
disjoint batches of designs (weak scaling, no data-path collective), the job's
time is the slowest rank's (one max all-reduce), and the reported value is the
designs of all ranks over that time."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, batch, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seeds = bench.rank_seeds(rank, world, batch)
        every = [None] * world
        dist.all_gather_object(every, seeds)
        local = 1.0 + 0.5 * rank  # rank-dependent step time (seconds)
        job = bench.slowest(local, world, dist)
        rate = bench.job_rate(world, batch, 3, job)
        out.put((rank, every, job, rate))
    finally:
        dist.destroy_process_group()


def test_two_rank_seeds_time_and_rate():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world, batch = 2, 8
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, batch, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, every, job, rate in res:
        flat = [s for seeds in every for s in seeds]
        assert sorted(flat) == list(range(world * batch))  # disjoint and complete
        assert every[rank] == list(range(rank * batch, (rank + 1) * batch))
        assert job == 1.5  # the slowest rank's time, on every rank
        assert rate == world * batch * 3 / 1.5


STUB = r'''
import json, os, sys
sys.path.insert(0, %(root)r)
import torch.distributed as dist
import bench
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
assert int(os.environ["LOCAL_RANK"]) == rank and os.environ["MASTER_ADDR"] == "127.0.0.1"
dist.init_process_group("gloo", rank=rank, world_size=world)
seeds = bench.rank_seeds(rank, world, 4)
job = bench.slowest(0.5 + 0.25 * rank, world, dist)  # stub step time of this rank
if rank == 0:
    print(json.dumps({"n_gpus": world, "value": bench.job_rate(world, 4, 2, job),
                      "seeds0": seeds, "job_s": job}))
else:
    print("rank %%d must not reach the driver's stdout" %% rank)
dist.destroy_process_group()
'''


def test_replica_launcher_runs_ranks(tmp_path):
    """bench.py --gpus N without torchrun starts N replica ranks itself: every
    rank gets its RANK / LOCAL_RANK / WORLD_SIZE and a 127.0.0.1 rendezvous,
    only rank 0's line reaches stdout, and the rate uses the slowest rank."""
    pytest.importorskip("torch")
    import json
    sys.path.insert(0, ROOT)
    import bench
    stub = tmp_path / "stub_rank.py"
    stub.write_text(STUB % {"root": ROOT})
    out = tmp_path / "out.txt"
    with open(out, "w") as f:
        rc = bench.launch_replicas([sys.executable, str(stub)], 2, stdout=f)
    assert rc == 0
    lines = [ln for ln in out.read_text().splitlines() if ln.strip()]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["n_gpus"] == 2 and rec["job_s"] == 0.75
    assert rec["value"] == 2 * 4 * 2 / 0.75
    assert rec["seeds0"] == [0, 1, 2, 3]


def test_replica_launcher_reports_a_failed_rank(tmp_path):
    sys.path.insert(0, ROOT)
    import bench
    stub = tmp_path / "fail.py"
    stub.write_text("import os, sys\nsys.exit(3 if os.environ['RANK'] == '1' else 0)\n")
    assert bench.launch_replicas([sys.executable, str(stub)], 2) == 3
