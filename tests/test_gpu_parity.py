"""GPU path against the FP64 oracle, through the C ABI.

Tolerances: FP32 storage 1e-5 in the max-relative metric max|a-b|/max|b|
per field (rho_A, rho_B, each u component) after 100 steps; element-wise
states within a few FP32 ulps of the largest population; FP16/BF16
deviation storage 2e-3 on the densities. The oracle always starts from the
same float32-rounded fields the GPU receives.

Velocity floor: a velocity is a difference of stored deviations
d_i = f_i - w_i rho0 of opposite populations, each rounded to the storage
type, so its absolute error cannot go below about one ulp of the largest
moving-population deviation over the density. Where the flow is weak (the
miscible spinodal case decays to |u| ~ 4e-6 after 100 steps while
|d| ~ 3e-3) that floor exceeds 1e-5 max|u|; velocity checks therefore take
max(1e-5 max|u|, 8 half-ulps of max|d_moving| / min rho). A velocity-dominated
flow (test_velocity_dominated_flow_parity) checks the plain 1e-5 bar.
The velocity is compared as a vector field: max over nodes and components of
|u_gpu - u_oracle| over max over nodes of |u_oracle|.
"""
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


def rel(a, b):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / max(np.abs(b).max(), 1e-300))


def gpu_run(shape, steps, tau, G, rA, rB, u=None, mask=None, g=(0, 0, 0), **kw):
    nx, ny, nz = shape
    s = Solver(nx, ny, nz, tau, G, mask=mask, body_force=g, **kw)
    s.init(dev(rA), dev(rB), dev(u) if u is not None else None)
    if steps:
        s.step(steps)
    return s


def oracle_run(shape, steps, tau, G, rA, rB, u=None, mask=None, g=None):
    f = oracle.init(f32(rA), f32(rB), None if u is None else f32(u), mask)
    return oracle.run(f, steps, tau, G, g, mask) if steps else f


def moments_np(s):
    rA, rB, u = s.moments()
    torch.cuda.synchronize()
    return rA.cpu().numpy(), rB.cpu().numpy(), u.cpu().numpy()


# half an ulp, relative, of the stored deviation for each storage type
HALF_ULP = {"fp32": 2.0 ** -24, "fp16": 2.0 ** -11, "bf16": 2.0 ** -8}


def u_floor(f, rA, rB, mask, prec="fp32"):
    """Absolute velocity error allowed by rounding of the stored deviations;
    f is the state whose deviations set the scale (the initial one, where
    they are largest for a relaxing mixture)."""
    c, w, _ = oracle.lattice()
    r0 = deviation_base(rA, rB, mask)
    dev = f - np.stack([w[:, None, None, None] * r0[0], w[:, None, None, None] * r0[1]])
    fluid = np.ones(f.shape[2:], bool) if mask is None else (mask == 0)
    dmax = np.abs(dev[:, 1:][:, :, fluid]).max()
    rmin = f.sum(axis=1).sum(axis=0)[fluid].min()
    return 8 * HALF_ULP[prec] * dmax / rmin


def u_rel(gu, ou):
    """Vector-field metric: max |u_gpu - u_oracle| / max |u_oracle|."""
    err = np.abs(np.asarray(gu, np.float64) - ou).max()
    return err, float(np.sqrt((ou * ou).sum(axis=0)).max())


def check_u(gu, ou, floor):
    err, scale = u_rel(gu, ou)
    assert err <= max(1e-5 * scale, floor), (err, scale, floor)


def deviation_base(rA, rB, mask):
    fl = np.ones(np.shape(rA), bool) if mask is None else (mask == 0)
    return f32(rA)[fl].mean(), f32(rB)[fl].mean()


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("masked", [False, True])
def test_initial_state_matches_oracle(prec, masked):
    """Element-wise: |f_gpu - f_oracle| <= half an ulp of the stored deviation
    d = f - w_i rho0 (rounding to the storage type) + a few FP32 ulps of f."""
    shape = (19, 11, 7)
    nx, ny, nz = shape
    rA, rB = inputs.spinodal(nx, ny, nz, seed=3)
    u = np.random.default_rng(4).normal(scale=0.02, size=(3, nz, ny, nx))
    mask = inputs.random_mask(nx, ny, nz, seed=5, solid_fraction=0.2) if masked else None
    s = gpu_run(shape, 0, 1.0, 0.65, rA, rB, u, mask, prec=prec)
    got = s.get_state().cpu().numpy()
    want = oracle_run(shape, 0, 1.0, 0.65, rA, rB, u, mask)
    c, w, _ = oracle.lattice()
    r0 = deviation_base(rA, rB, mask)
    base = np.stack([w[:, None, None, None] * r0[0], w[:, None, None, None] * r0[1]])
    dev_abs = np.abs(want - base)
    if masked:
        dev_abs[:, :, mask == 1] = 0.0
    bound = HALF_ULP[prec] * dev_abs * 1.01 + 6e-8 + 3 * 2.0 ** -24 * np.abs(want).max()
    assert np.all(np.abs(got - want) <= bound)
    if masked:
        assert np.all(got[:, :, mask == 1] == 0)


@pytest.mark.parametrize("kernel", ["fused", "two_pass", "fused_reg"])
@pytest.mark.parametrize("shape,masked,tau,G,g", [
    ((32, 32, 32), False, 1.0, 0.65, (0, 0, 0)),
    ((37, 21, 13), True, 0.8, 1.3, (1e-5, -2e-5, 3e-6)),
    ((3, 3, 3), False, 0.7, 0.9, (0, 0, 0)),
    ((5, 4, 3), True, 1.2, 0.5, (0, 1e-5, 0)),
    ((33, 9, 70), True, 0.9, 1.0, (0, 0, 0)),
])
def test_single_step_state_elementwise(kernel, shape, masked, tau, G, g):
    nx, ny, nz = shape
    rA, rB = inputs.spinodal(nx, ny, nz, seed=nx * ny + nz)
    u = np.random.default_rng(8).normal(scale=0.01, size=(3, nz, ny, nx))
    mask = inputs.random_mask(nx, ny, nz, seed=9, solid_fraction=0.15) if masked else None
    s = gpu_run(shape, 1, tau, G, rA, rB, u, mask, g, kernel=kernel)
    got = s.get_state().cpu().numpy()
    want = oracle_run(shape, 1, tau, G, rA, rB, u, mask, g)
    assert np.abs(got - want).max() <= 4e-7 * np.abs(want).max()


@pytest.mark.parametrize("kernel", ["fused", "two_pass"])
def test_config0_parity_100_steps(kernel):
    """32^3 periodic, tau = 1, G = 0.65, rho_A = 0.5 + 0.05 U(-1,1) (seed
    1234), rho_B = 1 - rho_A, u = 0; 100 steps; conservation every step."""
    n, tau, G, steps = 32, 1.0, 0.65, 100
    rA, rB = inputs.spinodal(n, n, n, seed=1234)
    s = gpu_run((n, n, n), 0, tau, G, rA, rB, kernel=kernel)
    s0 = s.stats()
    M = s0[0] + s0[1]
    for _ in range(steps):
        s.step(1)
        st = s.stats()
        assert abs(st[0] - s0[0]) <= 1e-8 * s0[0]
        assert abs(st[1] - s0[1]) <= 1e-8 * s0[1]
        assert np.abs(st[2:] - s0[2:]).max() <= 1e-8 * M
    gA, gB, gu = moments_np(s)
    f = oracle_run((n, n, n), steps, tau, G, rA, rB)
    oA, oB, ou = oracle.moments(f, G)
    assert rel(gA, oA) <= 1e-5
    assert rel(gB, oB) <= 1e-5
    check_u(gu, ou, u_floor(oracle_run((n, n, n), 0, tau, G, rA, rB), rA, rB, None))
    # the oracle's totals agree with the GPU's FP64 reduction
    np.testing.assert_allclose(s.stats()[:2], oracle.stats(f)[:2], rtol=1e-7)


@pytest.mark.parametrize("kernel", ["fused", "two_pass"])
def test_masked_ragged_parity_50_steps(kernel):
    nx, ny, nz, tau, G, steps = 45, 27, 19, 0.9, 0.8, 50
    mask, _ = inputs.colloid_mask(nx, ny, nz, n_spheres=6, radius=3.0, seed=5)
    rA, rB = inputs.spinodal(nx, ny, nz, seed=77)
    g = (2e-6, 0.0, -1e-6)
    s = gpu_run((nx, ny, nz), steps, tau, G, rA, rB, mask=mask, g=g, kernel=kernel)
    gA, gB, gu = moments_np(s)
    f = oracle_run((nx, ny, nz), steps, tau, G, rA, rB, mask=mask, g=g)
    oA, oB, ou = oracle.moments(f, G, g, mask)
    assert rel(gA, oA) <= 1e-5 and rel(gB, oB) <= 1e-5
    check_u(gu, ou, u_floor(oracle_run((nx, ny, nz), 0, tau, G, rA, rB, mask=mask), rA, rB, mask))
    assert np.all(gA[mask == 1] == 0) and np.all(gu[:, mask == 1] == 0)


@pytest.mark.parametrize("kernel", ["fused", "two_pass"])
def test_velocity_dominated_flow_parity(kernel):
    """A decaying shear wave u_x = 1e-3 sin(2 pi y / ny) through the
    spinodal mixture: velocity errors far above the storage floor, so the
    plain 1e-5 max-relative bar applies to every field."""
    nx, ny, nz, tau, G, steps = 40, 32, 24, 0.8, 0.65, 100
    rA, rB = inputs.spinodal(nx, ny, nz, seed=55)
    u = np.zeros((3, nz, ny, nx))
    u[0] = 1e-3 * np.sin(2 * np.pi * np.arange(ny) / ny)[None, :, None]
    s = gpu_run((nx, ny, nz), steps, tau, G, rA, rB, u, kernel=kernel)
    gA, gB, gu = moments_np(s)
    f = oracle_run((nx, ny, nz), steps, tau, G, rA, rB, u)
    oA, oB, ou = oracle.moments(f, G)
    assert rel(gA, oA) <= 1e-5 and rel(gB, oB) <= 1e-5
    err, scale = u_rel(gu, ou)
    assert err <= 1e-5 * scale


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("shape,masked", [((40, 24, 18), True), ((64, 48, 20), False), ((3, 3, 3), False)])
def test_all_kernels_are_bitwise_equal(prec, shape, masked):
    """The three step kernels do the same arithmetic in the same order."""
    nx, ny, nz = shape
    rA, rB = inputs.spinodal(nx, ny, nz, seed=31)
    mask = inputs.random_mask(nx, ny, nz, seed=32, solid_fraction=0.1) if masked else None
    ref = gpu_run(shape, 10, 0.8, 1.1, rA, rB, mask=mask, kernel="two_pass", prec=prec).get_state()
    for kernel in ("fused", "fused_reg"):
        got = gpu_run(shape, 10, 0.8, 1.1, rA, rB, mask=mask, kernel=kernel, prec=prec).get_state()
        assert torch.equal(got, ref), kernel


@pytest.mark.parametrize("prec,tol_rho", [("fp16", 2e-3), ("bf16", 2e-3)])
def test_reduced_precision_storage_config0(prec, tol_rho):
    n, tau, G, steps = 32, 1.0, 0.65, 100
    rA, rB = inputs.spinodal(n, n, n, seed=1234)
    s = gpu_run((n, n, n), steps, tau, G, rA, rB, prec=prec)
    gA, gB, gu = moments_np(s)
    f = oracle_run((n, n, n), steps, tau, G, rA, rB)
    oA, oB, ou = oracle.moments(f, G)
    assert rel(gA, oA) <= tol_rho and rel(gB, oB) <= tol_rho


def test_set_state_round_trip_and_continuation():
    nx, ny, nz = 20, 12, 9
    rA, rB = inputs.spinodal(nx, ny, nz, seed=41)
    mask = inputs.random_mask(nx, ny, nz, seed=42, solid_fraction=0.1)
    s = gpu_run((nx, ny, nz), 3, 1.0, 0.7, rA, rB, mask=mask)
    f = s.get_state().clone()
    s.set_state(f)
    assert torch.allclose(s.get_state(), f, rtol=0, atol=1e-7)
    # continuing from an imported oracle state matches the oracle
    fo = oracle_run((nx, ny, nz), 3, 1.0, 0.7, rA, rB, mask=mask)
    s.set_state(torch.tensor(fo.astype(np.float32), device="cuda"))
    s.step(5)
    gA, _, _ = moments_np(s)
    oA, _, _ = oracle.moments(oracle.run(f32(fo.astype(np.float32)), 5, 1.0, 0.7, None, mask), 0.7, None, mask)
    assert rel(gA, oA) <= 2e-5   # the imported state is FP32-rounded twice (export, deviation import)


def test_init_rejects_nonpositive_or_nonfinite_density():
    from paper_2112_08264_gb300 import _lib
    nx = ny = nz = 6
    rA, rB = inputs.spinodal(nx, ny, nz, seed=1)
    s = Solver(nx, ny, nz, 1.0, 0.5)
    bad = rA.copy()
    bad[2, 3, 4] = 0.0
    with pytest.raises(_lib.LbError) as e:
        s.init(dev(bad), dev(rB))
    assert e.value.status == _lib.LB_EINVAL
    bad[2, 3, 4] = np.nan
    with pytest.raises(_lib.LbError):
        s.init(dev(bad), dev(rB))
    # zero density on a solid node is fine
    mask = np.zeros((nz, ny, nx), np.uint8)
    mask[2, 3, 4] = 1
    bad[2, 3, 4] = 0.0
    sm = Solver(nx, ny, nz, 1.0, 0.5, mask=mask)
    sm.init(dev(bad), dev(rB))
    sm.step(2)


def test_stats_flags_non_finite_state():
    from paper_2112_08264_gb300 import _lib
    nx = ny = nz = 8
    rA, rB = inputs.spinodal(nx, ny, nz, seed=2)
    s = gpu_run((nx, ny, nz), 1, 1.0, 0.5, rA, rB)
    f = s.get_state()
    f[0, 3, 1, 2, 3] = float("nan")
    s.set_state(f)
    with pytest.raises(_lib.LbError) as e:
        s.stats()
    assert e.value.status == _lib.LB_ENONFINITE


def test_all_solid_mask_is_inert():
    n = 5
    mask = np.ones((n, n, n), np.uint8)
    rA, rB = inputs.spinodal(n, n, n, seed=3)
    s = gpu_run((n, n, n), 3, 1.0, 0.5, rA, rB, mask=mask)
    np.testing.assert_array_equal(s.stats(), np.zeros(5))
    assert float(s.get_state().abs().max()) == 0.0


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
def test_full_size_256_tiled_state(prec):
    """256^3 in the benchmark's launch configuration: a random 16^3 periodic
    state tiled 16 times per axis must evolve exactly as the oracle's 16^3
    run, at every one of the 16.8M sites."""
    n, p, steps, tau, G = 256, 16, 3, 1.0, 0.65
    rA, rB = inputs.spinodal(p, p, p, seed=1234)
    u = np.random.default_rng(5).normal(scale=0.01, size=(3, p, p, p))
    reps = (n // p,) * 3
    s = Solver(n, n, n, tau, G, prec=prec)
    assert s.launch_info()["launches_per_step"] == 1
    big = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda").repeat(*reps).contiguous()
    s.init(big(rA), big(rB), torch.stack([big(u[a]) for a in range(3)]).contiguous())
    s.step(steps)
    got = s.get_state()
    want = oracle_run((p, p, p), steps, tau, G, rA, rB, u)
    want_t = torch.tensor(want.astype(np.float32), device="cuda").repeat(1, 1, *reps)
    # 16-bit storage: the FP16 bound scaled by the ratio of the two types'
    # half-ulps (2^-8 / 2^-11 = 8) for BF16
    tol = {"fp32": 4e-7, "fp16": 5e-5, "bf16": 4e-4}[prec] * float(want_t.abs().max())
    assert float((got - want_t).abs().max()) <= tol
    st = s.stats()
    assert abs(st[0] - float(rA.astype(np.float32).astype(np.float64).sum()) * (n // p) ** 3) <= 1e-6 * st[0]
