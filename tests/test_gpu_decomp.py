"""Z-slab decomposition through the C ABI on one GPU (paper Sec. 4: equal
sub-domains that exchange their border planes every step).

Each rank of a lattice cut into W z-slabs is a context over its planes plus
two ghost planes per side (``slab_halo = 2``). Per step every rank runs
``lb_step_fluid``, the ghost planes are refilled from the neighbours' border
planes (``lb_planes`` gives their memory), and ``lb_step_links`` runs the
bounce-back pass. Here the W ranks are W contexts on one device, stepped one
after another, and the exchange is a device copy between their workspaces:
no kernel waits on another. The owned planes of every slab must equal the
whole-lattice run bit for bit (FP32 and 16-bit storage, with and without a
mask whose links cross the slab borders), and the FP64 totals of the owned
planes must add up to the whole lattice's.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2112_08264_gb300 import Solver, build, decomp, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def dev(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def exchange(slabs):
    """What decomp.exchange does between ranks, as copies on one device:
    lower ghosts <- the last two owned planes of the slab below, upper ghosts
    <- the first two owned planes of the slab above (periodic)."""
    h = decomp.HALO
    views = [s.planes() for s in slabs]
    sends = [(v.narrow(0, h, h).clone(), v.narrow(0, v.shape[0] - 2 * h, h).clone()) for v in views]
    W = len(slabs)
    for r, v in enumerate(views):
        v.narrow(0, 0, h).copy_(sends[(r - 1) % W][1])
        v.narrow(0, v.shape[0] - h, h).copy_(sends[(r + 1) % W][0])


@pytest.mark.parametrize("prec,masked,world", [("fp32", False, 2), ("fp32", True, 2), ("fp16", True, 3),
                                               ("bf16", False, 2)])
def test_slabs_match_whole_lattice_bitwise(prec, masked, world):
    nx, ny, nz, tau, G, steps = 32, 16, 24, 0.9, 1.0, 12
    g = (1e-5, 0.0, -2e-5)
    rA, rB = inputs.spinodal(nx, ny, nz, seed=17)
    u = np.random.default_rng(18).normal(scale=0.01, size=(3, nz, ny, nx))
    mask = inputs.random_mask(nx, ny, nz, seed=19, solid_fraction=0.12) if masked else None
    fluid = np.ones((nz, ny, nx), bool) if mask is None else mask == 0
    # one deviation base for every rank (the whole lattice's fluid mean)
    rho0 = (float(np.float32(rA)[fluid].astype(np.float64).mean()), float(np.float32(rB)[fluid].astype(np.float64).mean()))
    kw = dict(prec=prec, rho0=rho0, body_force=g)
    full = Solver(nx, ny, nz, tau, G, mask=mask, **kw)
    full.init(dev(rA), dev(rB), dev(u))
    full.step(steps)
    want = full.get_state()
    slabs = []
    for r in range(world):
        idx = decomp.extended_planes(nz, world, r)
        s = Solver(nx, ny, len(idx), tau, G, mask=None if mask is None else np.ascontiguousarray(mask[idx]),
                   slab_halo=decomp.HALO, **kw)
        s.init(dev(rA[idx]), dev(rB[idx]), dev(u[:, idx]))
        slabs.append(s)
    exchange(slabs)
    for s in slabs:
        s.step_links()
    for _ in range(steps):
        for s in slabs:
            s.step_fluid()
        exchange(slabs)
        for s in slabs:
            s.step_links()
    totals = np.zeros(5)
    for r, s in enumerate(slabs):
        z0, z1 = decomp.slab_bounds(nz, world, r)
        got = s.get_state()[:, :, decomp.HALO:decomp.HALO + z1 - z0]
        assert torch.equal(got, want[:, :, z0:z1]), r
        totals += s.stats_planes(decomp.HALO, z1 - z0)
        assert s.steps_done == steps
    whole = full.stats()
    np.testing.assert_allclose(totals, whole, rtol=1e-12, atol=1e-12 * abs(whole[0]))
    for s in slabs + [full]:
        s.close()


def test_split_step_order_is_enforced():
    from paper_2112_08264_gb300 import _lib
    nx, ny, nz = 16, 8, 10
    mask = inputs.random_mask(nx, ny, nz, seed=2, solid_fraction=0.1)
    rA, rB = inputs.spinodal(nx, ny, nz, seed=3)
    s = Solver(nx, ny, nz, 1.0, 0.5, mask=mask, slab_halo=2, rho0=(0.5, 0.5))
    s.init(dev(rA), dev(rB))
    s.step_fluid()
    for call in (lambda: s.step(1), lambda: s.moments(), lambda: s.stats(), lambda: s.step_fluid(),
                 lambda: s.stats_planes(2, 6)):
        with pytest.raises(_lib.LbError) as e:
            call()
        assert e.value.status == _lib.LB_ESTATE
    s.step_links()
    s.step(1)
    assert s.steps_done == 2
    with pytest.raises((ValueError, _lib.LbError)):   # a slab carries no spheres
        Solver(16, 8, 10, 1.0, 0.5, slab_halo=2, max_particles=4)
    s.close()


def test_slabs_at_256_cubed_match_whole_lattice_bitwise():
    """The benchmark's grid cut into two slabs of 128 planes (each stepped by
    the box kernel in its own launch configuration): the owned planes equal
    the whole-lattice run bit for bit after 3 steps."""
    n, steps = 256, 3
    rA, rB = inputs.spinodal(n, n, n, seed=1234)
    rho0 = (float(np.float32(rA).astype(np.float64).mean()), float(np.float32(rB).astype(np.float64).mean()))
    full = Solver(n, n, n, 1.0, 0.65, rho0=rho0)
    full.init(dev(rA), dev(rB))
    full.step(steps)
    want = full.get_state()
    full.close()
    slabs = []
    for r in range(2):
        idx = decomp.extended_planes(n, 2, r)
        s = Solver(n, n, len(idx), 1.0, 0.65, rho0=rho0, slab_halo=decomp.HALO)
        s.init(dev(rA[idx]), dev(rB[idx]))
        slabs.append(s)
    exchange(slabs)
    for _ in range(steps):
        for s in slabs:
            s.step_fluid()
        exchange(slabs)
        for s in slabs:
            s.step_links()
    for r, s in enumerate(slabs):
        z0, z1 = decomp.slab_bounds(n, 2, r)
        got = s.get_state()[:, :, decomp.HALO:decomp.HALO + z1 - z0]
        assert torch.equal(got, want[:, :, z0:z1]), r
        s.close()
