"""Z-slab decomposition of one lattice over CPU ranks (gloo), each rank
stepping its extended slab with the FP64 oracle and exchanging two ghost
planes per side every step (paper Sec. 4: equal sub-domains with a border
exchange each step).

The per-node arithmetic of the oracle does not depend on how large the grid
is, so the owned planes of every rank must equal the single-lattice run bit
for bit -- with a mask (bounce-back links crossing the slab borders), a body
force, slabs of unequal height and three ranks -- and the FP64 totals summed
over the ranks' owned planes must equal the single lattice's totals.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


CASES = {
    "periodic": dict(shape=(12, 10, 20), masked=False, g=None, tau=1.0, G=0.65, steps=20),
    "masked": dict(shape=(10, 12, 21), masked=True, g=(2e-5, -1e-5, 3e-5), tau=0.8, G=1.1, steps=20),
}


def _inputs(case):
    from paper_2112_08264_gb300 import inputs
    c = CASES[case]
    nx, ny, nz = c["shape"]
    rA, rB = inputs.spinodal(nx, ny, nz, seed=nz)
    u = np.random.default_rng(3).normal(scale=0.01, size=(3, nz, ny, nx))
    mask = inputs.random_mask(nx, ny, nz, seed=4, solid_fraction=0.15) if c["masked"] else None
    return c, rA, rB, u, mask


def _rank(rank, world, port, case, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2112_08264_gb300 import decomp
    c, rA, rB, u, mask = _inputs(case)
    nz = c["shape"][2]
    f = oracle.init(rA, rB, u, mask)                   # the global initial state, on every rank
    ext = decomp.extend(f, nz, world, rank, axis=2)    # (2, 19, L + 4, ny, nx)
    mext = None if mask is None else decomp.extend(mask, nz, world, rank, axis=0)
    for _ in range(c["steps"]):
        ext = oracle.step(ext, c["tau"], c["G"], c["g"], mext)
        decomp.exchange(torch.from_numpy(ext), 2, rank, world)
    own = np.array(decomp.interior(ext, 2))
    own_mask = None if mext is None else np.array(decomp.interior(mext, 0))
    totals = decomp.allreduce_sum(oracle.stats(own, own_mask)).numpy()
    out[rank] = (decomp.slab_bounds(nz, world, rank), own, totals)
    dist.destroy_process_group()


@pytest.mark.parametrize("case,world", [("periodic", 2), ("masked", 2), ("masked", 3)])
def test_slabs_match_single_lattice_bitwise(case, world):
    import oracle
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, case, out), nprocs=world, join=True)
        res = dict(out)
    c, rA, rB, u, mask = _inputs(case)
    want = oracle.run(oracle.init(rA, rB, u, mask), c["steps"], c["tau"], c["G"], c["g"], mask)
    got = np.empty_like(want)
    covered = np.zeros(c["shape"][2], int)
    for rank in range(world):
        (z0, z1), own, totals = res[rank]
        got[:, :, z0:z1] = own
        covered[z0:z1] += 1
        np.testing.assert_allclose(totals, oracle.stats(want, mask), rtol=1e-13, atol=1e-13)
    assert np.all(covered == 1)
    assert np.array_equal(got, want)


def test_slab_bounds_and_extension():
    from paper_2112_08264_gb300 import decomp
    assert [decomp.slab_bounds(21, 3, r) for r in range(3)] == [(0, 7), (7, 14), (14, 21)]
    assert [decomp.slab_bounds(10, 4, r) for r in range(4)] == [(0, 2), (2, 5), (5, 7), (7, 10)]
    assert decomp.extended_planes(10, 4, 0) == [8, 9, 0, 1, 2, 3]
    assert decomp.extended_planes(10, 4, 3) == [5, 6, 7, 8, 9, 0, 1]
    with pytest.raises(ValueError):
        decomp.slab_bounds(5, 4, 0)   # a slab shorter than the two ghost planes
    a = np.arange(10 * 3).reshape(10, 3)
    e = decomp.extend(a, 10, 4, 1, axis=0)
    assert np.array_equal(e[:, 0], a[[0, 1, 2, 3, 4, 5, 6], 0])
    assert np.array_equal(decomp.interior(e, 0), a[2:5])
    # one rank: the slab is the periodic lattice, its borders wrap onto its ghosts
    t = torch.from_numpy(decomp.extend(a, 10, 1, 0, axis=0).copy())
    t[:2] = -1
    t[-2:] = -1
    decomp.exchange(t, 0, 0, 1)
    assert np.array_equal(t.numpy(), decomp.extend(a, 10, 1, 0, axis=0))
