"""The N > 1 benchmark path runs independent replicas (the lattice is not
decomposed across GPUs). Its host logic -- process group, barrier, max over
ranks of the timed region, whole-job aggregation -- is checked here on CPU
with two gloo ranks, each timing its own oracle replica."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from paper_2112_08264_gb300 import inputs
    n, steps = 6, 3
    rA, rB = inputs.spinodal(n, n, n, seed=1234 + rank)      # each rank its own replica
    f = oracle.init(rA, rB)
    bench.barrier(world)
    ms_local = 10.0 * (rank + 1)                              # a known, rank-dependent time
    f = oracle.run(f, steps, 1.0, 0.65)
    glups, step_s = bench.replica_throughput(ms_local, steps, n ** 3, world)
    bench.barrier(world)
    out[rank] = (glups, step_s, float(oracle.stats(f)[0]), float(oracle.stats(oracle.init(rA, rB))[0]))
    dist.destroy_process_group()


def test_two_gloo_replicas_aggregate_over_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    slowest_ms = 10.0 * world
    for rank in range(world):
        glups, step_s, mass_end, mass_start = res[rank]
        assert step_s == pytest.approx(slowest_ms / 1e3 / 3)
        assert glups == pytest.approx(world * 6 ** 3 / (slowest_ms / 1e3 / 3) / 1e9)
        assert mass_end == pytest.approx(mass_start, rel=1e-13)   # each replica conserves its own mass
