"""One-component BGK step on the GPU (``include/lb1.h``, the paper's
single-fluid case) against the one-component FP64 oracle
(``oracle.single_bgk``), through the C ABI.

Bars: element-wise states within a few FP32 ulps after one step; densities
within 1e-5 (FP32) and 2e-3 (FP16/BF16 storage) after 100 steps; a shear wave
(flow-dominated) within 1e-5 of the oracle's velocity; mass and momentum
conserved step by step; the shear wave's decay rate nu k^2 with
nu = (tau - 1/2)/3 (Eq. viscosity) within 1 %.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lb_numpy as ln  # noqa: E402
from oracle import single_bgk as sb  # noqa: E402
from paper_2112_08264_gb300 import SingleFluid, build  # noqa: E402

pytestmark = pytest.mark.gpu

ORDER = [sb.velocity_index(c) for c in ln.PUBLIC]   # public index -> oracle index


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def oracle_init(rho, u):
    c = sb.VELOCITIES.astype(float)
    cu = np.einsum("id,dabc->iabc", c, u)
    uu = (u * u).sum(axis=0)
    return sb.WEIGHTS[:, None, None, None] * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu)


def oracle_moments(f, g=(0.0, 0.0, 0.0)):
    c = sb.VELOCITIES.astype(float)
    rho = f.sum(axis=0)
    u = (np.einsum("id,iabc->dabc", c, f) + 0.5 * rho * np.asarray(g)[:, None, None, None]) / rho
    return rho, u


def fields(shape, seed, amp_u=0.02):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    rho = f32(1.0 + 0.05 * rng.uniform(-1, 1, (nz, ny, nx)))
    u = f32(amp_u * rng.uniform(-1, 1, (3, nz, ny, nx)))
    return rho, u


def run_gpu(shape, steps, tau, rho, u, g=(0.0, 0.0, 0.0), prec="fp32"):
    s = SingleFluid(*shape, tau, body_force=g, prec=prec)
    s.init(dev(rho), dev(u))
    if steps:
        s.step(steps)
    return s


@pytest.mark.parametrize("shape", [(24, 16, 12), (32, 20, 9)])
def test_single_step_state_elementwise(shape):
    rho, u = fields(shape, 3)
    g = (1e-4, -2e-4, 5e-5)
    s = run_gpu(shape, 1, 0.8, rho, u, g)
    got = s.get_state().cpu().numpy().astype(np.float64)
    s.close()
    want = sb.step(oracle_init(rho, u), 0.8, g)[ORDER]
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err < 8 * 2.0 ** -24 * 4, err


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp16", 2e-3), ("bf16", 2e-3)])
def test_moments_100_steps_and_conservation(prec, tol):
    shape = (32, 32, 16)
    rho, u = fields(shape, 5)
    s = run_gpu(shape, 0, 1.0, rho, u, prec=prec)
    t0 = np.array(s.stats())
    for _ in range(4):
        s.step(25)
        t = np.array(s.stats())
        ctol = 1e-6 if prec == "fp32" else 1e-3
        assert abs(t[0] - t0[0]) <= ctol * t0[0]
        assert np.abs(t[1:] - t0[1:]).max() <= ctol * t0[0]
    gr, gu = (x.cpu().numpy().astype(np.float64) for x in s.moments())
    s.close()
    f = oracle_init(rho, u)
    for _ in range(100):
        f = sb.step(f, 1.0)
    orho, ou = oracle_moments(f)
    assert np.abs(gr - orho).max() / orho.max() <= tol


def test_shear_wave_velocity_and_decay():
    """u_x = A sin(2 pi y / ny): the velocity follows the oracle within 1e-5
    and decays as exp(-nu k^2 t), nu = (tau - 1/2)/3."""
    nx, ny, nz = 8, 64, 4
    tau, A, steps = 0.9, 1e-3, 200
    y = np.arange(ny)
    rho = np.ones((nz, ny, nx))
    u = np.zeros((3, nz, ny, nx))
    u[0] = A * np.sin(2 * np.pi * y / ny)[None, :, None]
    s = run_gpu((nx, ny, nz), steps, tau, rho, u)
    _, gu = (x.cpu().numpy().astype(np.float64) for x in s.moments())
    s.close()
    f = oracle_init(rho, u)
    for _ in range(steps):
        f = sb.step(f, tau)
    _, ou = oracle_moments(f)
    assert np.abs(gu - ou).max() <= 1e-5 * np.abs(ou).max()
    k = 2 * np.pi / ny
    nu = (tau - 0.5) / 3.0
    amp = (gu[0, 0, :, 0] * np.sin(k * y)).sum() * 2 / ny
    assert abs(amp / (A * np.exp(-nu * k * k * steps)) - 1.0) < 0.01


def test_rejects_unaligned_rows():
    with pytest.raises(Exception):
        SingleFluid(18, 16, 16, 1.0)          # nx not a multiple of 4
    with pytest.raises(Exception):
        SingleFluid(20, 16, 16, 1.0, prec="fp16")   # 16-bit storage wants nx % 8 == 0


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_full_size_256_tiled_state(prec):
    """256^3 in the benchmark's launch configuration: a random 16^3 periodic
    state tiled 16 times per axis evolves exactly as the oracle's 16^3 run."""
    n, p, steps, tau = 256, 16, 3, 1.0
    rho, u = fields((p, p, p), 17)
    reps = (n // p,) * 3
    s = SingleFluid(n, n, n, tau, prec=prec)
    big = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda").repeat(*reps).contiguous()
    s.init(big(rho), torch.stack([big(u[a]) for a in range(3)]).contiguous())
    s.step(steps)
    got = s.get_state()
    f = oracle_init(rho, u)
    for _ in range(steps):
        f = sb.step(f, tau)
    want_t = torch.tensor(f[ORDER].astype(np.float32), device="cuda").repeat(1, 1, *reps)
    tol = {"fp32": 4e-7, "fp16": 5e-4}[prec] * float(want_t.abs().max())
    assert float((got - want_t).abs().max()) <= tol
    s.close()
