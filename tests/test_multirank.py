"""Multi-process host logic of the N > 1 bench path, on CPU with two gloo ranks.

One factorization does not shard, so N GPUs run replicas: every rank factors its own disjoint
set of seeded matrices, with no collective on the data path.  The only collectives are the
barriers around the timed region and the max over ranks of the timed duration; the whole-job
rate counts the matrices of all ranks over the slowest rank's time.  The reference arm runs on
rank 0 only; the other ranks exit 0 without work."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist_env() == (ws, rank, rank)
        nb = 3
        seeds = bench.rank_seeds(rank, nb)
        every = [None] * ws
        dist.all_gather_object(every, seeds)
        dist.barrier()
        # rank-dependent "timed region": the slowest rank's time is the job's
        t = bench.max_over_ranks(1.5 + rank)
        rate = bench.whole_job_rate(ws, nb, 4, t)
        rc = None
        if rank != 0:
            class A:
                warmup, steps, gpus = 1, 1, ws
            rc = bench.reference_arm(A())     # must return at once, without oracle work
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(repr({"every": every, "t": t, "rate": rate, "rc": rc}))
    finally:
        dist.destroy_process_group()


def test_replicas_two_gloo_ranks(tmp_path):
    ws = 2
    mp.spawn(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    res = [eval(open(tmp_path / f"r{r}.txt").read()) for r in range(ws)]
    for r in res:
        flat = [s for lst in r["every"] for s in lst]
        assert sorted(flat) == list(range(ws * 3))           # disjoint, nothing dropped
        assert r["t"] == 2.5                                  # max over ranks
        assert r["rate"] == pytest.approx(ws * 3 * 4 / 2.5)   # whole-job rate
    assert res[1]["rc"] == 0


def test_single_process_helpers():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    assert bench.rank_seeds(0, 4) == [0, 1, 2, 3] and bench.rank_seeds(2, 4) == [8, 9, 10, 11]
    assert bench.max_over_ranks(3.25) == 3.25                 # no process group: itself
    assert bench.whole_job_rate(1, 64, 20, 10.0) == pytest.approx(128.0)
