"""Write-side halfway bounce-back (Eq. LADDFLBE) with the links split between
the fused step kernel (links whose target lies in the source's tile and
z-chunk, copied inside the kernel) and the separate pass (the rest), against
the FP64 oracle, on grids whose tiles, row bands and z-chunks cut through the
solids. Also the two fallbacks: a list plane longer than the block (copied
in one go at the store point) and a mask with more links than sites (the
pass scans every site)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2112_08264_gb300 import Solver, build, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")


def run(shape, steps, mask, prec="fp32", kernel="fused", seed=3, tau=0.9, G=0.9, g=(1e-5, 0.0, -2e-5)):
    nx, ny, nz = shape
    rA, rB = inputs.spinodal(nx, ny, nz, seed=seed)
    u = np.random.default_rng(seed + 1).normal(scale=0.01, size=(3, nz, ny, nx))
    s = Solver(nx, ny, nz, tau, G, mask=mask, body_force=g, prec=prec, kernel=kernel)
    s.init(dev(rA), dev(rB), dev(u))
    if steps:
        s.step(steps)
    return s, (rA, rB, u, tau, G, g)


def oracle_state(shape, steps, mask, args):
    rA, rB, u, tau, G, g = args
    f = oracle.init(f32(rA), f32(rB), f32(u), mask)
    return oracle.run(f, steps, tau, G, g, mask) if steps else f


def spheres(shape, n, r, seed):
    nx, ny, nz = shape
    mask, _ = inputs.colloid_mask(nx, ny, nz, n_spheres=n, radius=r, seed=seed)
    return mask


# several 32-column strips, row bands and z-chunks
SHAPES = [(64, 40, 36), (96, 33, 20)]


@pytest.mark.parametrize("shape", SHAPES)
def test_tile_links_single_step_elementwise(shape):
    mask = spheres(shape, 8, 3.0, 11)
    s, args = run(shape, 1, mask)
    info = s.link_info()
    assert info["in_kernel"] and info["in_tile"] > 0 and info["listed"] > 0, info
    got = s.get_state().cpu().numpy()
    want = oracle_state(shape, 1, mask, args)
    assert np.abs(got - want).max() <= 4e-7 * np.abs(want).max()


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
def test_tile_links_kernels_bitwise(prec):
    """The box kernel copies the in-tile links itself; the two-pass and
    register kernels leave them to a pass of their own: same states."""
    shape = SHAPES[0]
    mask = spheres(shape, 8, 3.0, 12)
    ref, _ = run(shape, 10, mask, prec=prec, kernel="two_pass")
    assert not ref.link_info()["in_kernel"]
    want = ref.get_state()
    for kernel in ("fused", "fused_reg"):
        s, _ = run(shape, 10, mask, prec=prec, kernel=kernel)
        assert torch.equal(s.get_state(), want), kernel


def test_tile_links_moments_30_steps():
    shape = SHAPES[1]
    mask = spheres(shape, 10, 3.5, 13)
    s, args = run(shape, 30, mask)
    rA, rB, u = (x.cpu().numpy() for x in s.moments())
    f = oracle_state(shape, 30, mask, args)
    oA, oB, ou = oracle.moments(f, args[4], args[5], mask)
    for a, b in ((rA, oA), (rB, oB)):
        assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max()
    assert np.all(rA[mask == 1] == 0)


def test_long_list_plane_overflow():
    """Two half-solid planes: a (tile, plane) list far longer than the block
    (thousands of links against 32 x 14 threads), while the lists in total
    stay below the capacity of one entry per site."""
    shape = (64, 28, 40)
    nx, ny, nz = shape
    mask = np.zeros((nz, ny, nx), np.uint8)
    rng = np.random.default_rng(21)
    mask[17:19] = (rng.uniform(size=(2, ny, nx)) < 0.5)
    s, args = run(shape, 1, mask)
    info = s.link_info()
    assert info["in_kernel"] and info["in_tile"] > 4 * 32 * 16, info
    got = s.get_state().cpu().numpy()
    want = oracle_state(shape, 1, mask, args)
    assert np.abs(got - want).max() <= 4e-7 * np.abs(want).max()


def test_dense_mask_scans_every_site():
    """More links than sites: no lists, the pass scans every site."""
    shape = (40, 24, 18)
    mask = inputs.random_mask(*shape, seed=22, solid_fraction=0.5)
    s, args = run(shape, 2, mask)
    info = s.link_info()
    assert info["listed"] == -1 and info["in_tile"] == 0 and not info["in_kernel"], info
    got = s.get_state().cpu().numpy()
    want = oracle_state(shape, 2, mask, args)
    assert np.abs(got - want).max() <= 4e-7 * np.abs(want).max()


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
def test_full_size_256_tiled_masked_state(prec):
    """256^3 in the benchmark's launch configuration with a solid pattern: a
    16^3 periodic state and mask (a sphere of radius 4 and scattered solid
    sites) tiled 16 times per axis evolve exactly as the oracle's 16^3 run,
    at every site -- the tiles, bands and z-chunks of the step kernel cut
    through the spheres, so both kinds of link are exercised."""
    n, p, steps, tau, G = 256, 16, 3, 1.0, 0.65
    rA, rB = inputs.spinodal(p, p, p, seed=99)
    u = np.random.default_rng(7).normal(scale=0.01, size=(3, p, p, p))
    z, y, x = np.meshgrid(np.arange(p), np.arange(p), np.arange(p), indexing="ij")
    small = ((x - 7.3) ** 2 + (y - 8.1) ** 2 + (z - 6.6) ** 2 <= 16.0)
    small |= np.random.default_rng(8).uniform(size=(p, p, p)) < 0.02
    small = small.astype(np.uint8)
    reps = (n // p,) * 3
    s = Solver(n, n, n, tau, G, mask=np.tile(small, reps), prec=prec)
    info = s.link_info()
    assert info["in_kernel"] and info["in_tile"] > 0 and info["listed"] > 0, info
    big = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda").repeat(*reps).contiguous()
    s.init(big(rA), big(rB), torch.stack([big(u[a]) for a in range(3)]).contiguous())
    s.step(steps)
    got = s.get_state()
    f = oracle.run(oracle.init(f32(rA), f32(rB), f32(u), small), steps, tau, G, None, small)
    want_t = torch.tensor(f.astype(np.float32), device="cuda").repeat(1, 1, *reps)
    # BF16: the FP16 bound times the ratio of the half-ulps (2^-8 / 2^-11 = 8)
    tol = {"fp32": 4e-7, "fp16": 5e-5, "bf16": 4e-4}[prec] * float(want_t.abs().max())
    assert float((got - want_t).abs().max()) <= tol
