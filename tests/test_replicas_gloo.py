"""The multi-GPU form is replicas only: every rank searches its own seeded
observation with no data-path collective, and the job's time is the slowest
rank's.  The host logic of that (per-rank scenarios, max over ranks, the
whole-job value) is checked here with two gloo ranks on the CPU."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    class A:
        n_samp = 1 << 12
        dms = 4
    sc = bench.scenario(rank, A())
    ms = 10.0 + 5.0 * rank                       # rank 1 is the slower one
    worst = bench.max_over_ranks(ms, dist, "cpu")
    out[rank] = (sc.seed, float(sc.voltages()[0, 0].real), worst,
                 bench.job_value(1000, world, worst * 1e-3))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_own_seeds():
    world = 2
    port = 29500 + (os.getpid() % 1000)
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    (s0, v0, w0, j0), (s1, v1, w1, j1) = res[0], res[1]
    assert s0 != s1 and v0 != v1                  # independent observations
    assert w0 == w1 == 15.0                       # max over ranks on every rank
    assert j0 == j1 == pytest.approx(2 * 1000 / 15e-3)
