"""bench.py's multi-GPU contract on CPU: two gloo ranks, each an independent
replica; the job value is the sum of the ranks' pairs over the slowest
rank's time.  The reference arm prints only on rank 0."""
import os
import socket
import sys

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    d = bench.dist_init("gloo")
    pairs, ms = 1000.0 * (rank + 1), 2.0 + rank      # rank 1 is the slow one
    tot, slow = bench.aggregate(d, pairs, ms)
    out[rank] = (tot, slow, bench.dist_env())
    dist.destroy_process_group()


def test_two_rank_aggregation():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    for r in range(2):
        tot, slow, env = out[r]
        assert tot == 3000.0 and slow == 3.0
        assert env == (2, r, r)


def test_reference_arm_other_ranks_exit_quietly(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--config", "t0", "--steps", "1",
                                      "--warmup", "0"])
    assert bench.run_reference(bench.parse()) is None


def test_cost_study_n_c_matches_golden(golden):
    """bench.n_c (the §2.4 count used by --study cost) equals the pinned N_c values."""
    import bench
    for x, n in golden["N_c"].items():
        assert bench.n_c(float(x)) == n
