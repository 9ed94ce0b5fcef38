"""Writes stay inside the buffers the library is given (compute-sanitizer is
not used here; see the design notes). The workspace and every output buffer
are carved out of larger device allocations whose margins -- 64 KiB before
and after each -- hold a known byte pattern; a run of the hot kernels
(masked step with in-tile and crossing bounce-back links, 16-bit storage,
moving spheres with re-meshing, a slab context's split step, moments, state
export, FP64 totals, the allocation-free moments) must leave every margin
unchanged."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2112_08264_gb300 import Solver, _lib, build, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

GUARD = 1 << 16
PATTERN = 0xA5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


class Guarded:
    """A byte buffer of n bytes with GUARD bytes of PATTERN on each side."""

    def __init__(self, n):
        self.n = int(n)
        self.raw = torch.full((self.n + 2 * GUARD,), PATTERN, dtype=torch.uint8, device="cuda")
        self.body = self.raw[GUARD:GUARD + self.n]   # 256-byte aligned (allocations are)

    def floats(self, shape):
        return self.body.view(torch.float32)[:int(np.prod(shape))].view(*shape)

    def intact(self):
        torch.cuda.synchronize()
        return bool((self.raw[:GUARD] == PATTERN).all()) and bool((self.raw[GUARD + self.n:] == PATTERN).all())


def dev(a):
    return torch.tensor(np.asarray(a, np.float32), device="cuda")


def guarded_solver(nx, ny, nz, **kw):
    opt = _lib.options(**{k: v for k, v in kw.items() if k in ("prec", "max_particles", "slab_halo", "rho0")})
    ws = Guarded(_lib.workspace_bytes(nx, ny, nz, opt))
    return Solver(nx, ny, nz, 0.9, 0.9, workspace=ws.body, **kw), ws


def outputs(shape):
    bufs = {k: Guarded(4 * int(np.prod(s))) for k, s in
            (("rA", shape), ("rB", shape), ("u", (3,) + shape), ("f", (2, 19) + shape))}
    return bufs


def exercise(s, shape, bufs):
    rA, rB, u = bufs["rA"].floats(shape), bufs["rB"].floats(shape), bufs["u"].floats((3,) + shape)
    _lib.check(_lib.lib().lb_moments(s._h, rA.data_ptr(), rB.data_ptr(), u.data_ptr()), "lb_moments")
    s.get_state(out=bufs["f"].floats((2, 19) + shape))
    s.stats()


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_masked_step_writes_stay_inside(prec):
    nx, ny, nz = 64, 40, 30
    mask, _ = inputs.colloid_mask(nx, ny, nz, n_spheres=6, radius=4.0, seed=3)
    rA, rB = inputs.spinodal(nx, ny, nz, seed=4)
    s, ws = guarded_solver(nx, ny, nz, mask=mask, prec=prec)
    s.init(dev(rA), dev(rB))
    s.step(7)
    bufs = outputs((nz, ny, nx))
    exercise(s, (nz, ny, nx), bufs)
    assert ws.intact()
    assert all(b.intact() for b in bufs.values())
    s.close()


def test_moving_spheres_and_slab_writes_stay_inside():
    nx, ny, nz = 32, 24, 20
    rA, rB = inputs.spinodal(nx, ny, nz, seed=5)
    s, ws = guarded_solver(nx, ny, nz, max_particles=2)
    s.set_particles([[9.3, 8.4, 7.7], [23.6, 17.2, 12.9]], v=[[0.2, -0.1, 0.07], [-0.15, 0.08, 0.18]],
                    radius=3.2, mass=60.0)
    s.init(dev(rA), dev(rB))
    s.step(6)
    bufs = outputs((nz, ny, nx))
    exercise(s, (nz, ny, nx), bufs)
    assert ws.intact() and all(b.intact() for b in bufs.values())
    s.close()
    mask = inputs.random_mask(nx, ny, nz, seed=6, solid_fraction=0.1)
    t, wt = guarded_solver(nx, ny, nz, mask=mask, slab_halo=2, rho0=(0.5, 0.5))
    t.init(dev(rA), dev(rB))
    for _ in range(3):
        t.step_fluid()
        t.step_links()
    t.stats_planes(2, nz - 4)
    assert wt.intact()
    t.close()


def test_noalloc_writes_stay_inside():
    nx, ny, nz = 24, 20, 16
    rA, rB = inputs.spinodal(nx, ny, nz, seed=7)
    s = Solver(nx, ny, nz, 1.0, 0.7)
    s.init(dev(rA), dev(rB))
    s.step(3)
    f = s.get_state()
    bufs = outputs((nz, ny, nx))
    shape = (nz, ny, nx)
    st = _lib.lib().lb_moments_noalloc(nx, ny, nz, 0.7, None, f.data_ptr(), None,
                                       bufs["rA"].floats(shape).data_ptr(), bufs["rB"].floats(shape).data_ptr(),
                                       bufs["u"].floats((3,) + shape).data_ptr(), None)
    assert st == _lib.LB_OK
    assert all(b.intact() for k, b in bufs.items() if k != "f")
    s.close()
