"""Hand-written adjoint (lb_backward) against the oracle.

The reference gradient is the complex-step directional derivative of the
oracle's numpy formulation (exact to rounding; itself pinned against central
differences of the C oracle in test_oracle_adjoint_pins.py). Loss:
L = sum_x (rho_A(final) - target)^2 with a smoothed random target.
Tolerance: 1e-3 relative on directional derivatives and on sampled entries
(FP32 adjoint against an exact FP64 derivative).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lb_numpy as lnp  # noqa: E402
from paper_2112_08264_gb300 import Solver, build, inputs  # noqa: E402
from paper_2112_08264_gb300.autograd import simulate  # noqa: E402

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


def gpu_gradients(shape, steps, K, tau, G, rA, rB, target, mask=None, g=(0, 0, 0), kernel="fused", prec="fp32"):
    nx, ny, nz = shape
    s = Solver(nx, ny, nz, tau, G, mask=mask, body_force=g, ckpt_every=K, ckpt_steps_max=steps, kernel=kernel,
               prec=prec)
    s.init(dev(rA), dev(rB))
    s.step(steps)
    fA, _, _ = s.moments(velocity=False)
    dL = 2.0 * (fA - dev(target))
    if mask is not None:
        dL = dL * dev(mask == 0)
    gA, gB, gG = s.backward(dL.contiguous())
    torch.cuda.synchronize()
    out = gA.cpu().numpy().astype(np.float64), gB.cpu().numpy().astype(np.float64), gG
    s.close()
    return out


def check_case(shape, steps, K, tau, G, mask=None, g=None, kernel="fused", n_dirs=3, n_sites=6, seed=0):
    nx, ny, nz = shape
    rA, rB = inputs.spinodal(nx, ny, nz, seed=100 + seed)
    target = inputs.smoothed_target(nx, ny, nz, seed=200 + seed)
    gA, gB, gG = gpu_gradients(shape, steps, K, tau, G, rA, rB, target, mask, g or (0, 0, 0), kernel)
    a0, b0 = f32(rA), f32(rB)
    rng = np.random.default_rng(300 + seed)
    fluid = np.ones(rA.shape) if mask is None else (mask == 0).astype(float)
    # directional derivatives
    for _ in range(n_dirs):
        vA = rng.normal(size=rA.shape) * fluid
        vB = rng.normal(size=rB.shape) * fluid
        ref = lnp.jvp(a0, b0, G, target, steps, tau, vA, vB, 0.0, g, mask)
        got = float((gA * vA).sum() + (gB * vB).sum())
        assert abs(got - ref) <= 1e-3 * abs(ref), (got, ref)
    # dL/dG
    ref = lnp.jvp(a0, b0, G, target, steps, tau, None, None, 1.0, g, mask)
    assert abs(gG - ref) <= 1e-3 * abs(ref), (gG, ref)
    # sampled entries
    flat = np.flatnonzero(fluid.ravel())
    scale = max(np.abs(gA).max(), np.abs(gB).max())
    for s in rng.choice(flat, size=n_sites, replace=False):
        e = np.zeros(rA.size)
        e[s] = 1.0
        e = e.reshape(rA.shape)
        refA = lnp.jvp(a0, b0, G, target, steps, tau, e, None, 0.0, g, mask)
        refB = lnp.jvp(a0, b0, G, target, steps, tau, None, e, 0.0, g, mask)
        assert abs(gA.ravel()[s] - refA) <= 1e-3 * abs(refA) + 1e-5 * scale
        assert abs(gB.ravel()[s] - refB) <= 1e-3 * abs(refB) + 1e-5 * scale
    if mask is not None:
        assert np.all(gA[mask == 1] == 0) and np.all(gB[mask == 1] == 0)


@pytest.mark.parametrize("kernel", ["fused", "two_pass"])
def test_adjoint_16cubed_50_steps(kernel):
    """The differentiation form's verification case: 16^3, 50 steps,
    checkpoints every 10 (tau = 1, G = 0.65)."""
    check_case((16, 16, 16), 50, 10, 1.0, 0.65, kernel=kernel)


def test_adjoint_masked_body_force_partial_segment():
    nx, ny, nz = 12, 10, 9
    mask, _ = inputs.colloid_mask(nx, ny, nz, n_spheres=2, radius=2.5, seed=6)
    check_case((nx, ny, nz), 20, 6, 0.85, 0.9, mask=mask, g=(2e-5, 0.0, -1e-5), seed=1)


def test_adjoint_demixing_coupling():
    """Above the stability limit (G rho > 2 (tau - 1/2) / tau) the gradient
    grows with time; still FP32-accurate over 30 steps."""
    check_case((10, 9, 8), 30, 7, 1.0, 1.3, seed=2, n_sites=4)


def test_autograd_function_matches_solver_backward():
    nx = ny = nz = 8
    rA, rB = inputs.spinodal(nx, ny, nz, seed=5)
    target = dev(inputs.smoothed_target(nx, ny, nz, seed=6))
    a = dev(rA).requires_grad_(True)
    b = dev(rB).requires_grad_(True)
    G = torch.tensor(0.65, dtype=torch.float64, requires_grad=True)
    fA, fB = simulate(a, b, G, 12, ckpt_every=5, tau=1.0)
    loss = ((fA - target) ** 2).sum()
    loss.backward()
    gA, gB, gG = gpu_gradients((nx, ny, nz), 12, 5, 1.0, 0.65, rA, rB, target.cpu().numpy())
    np.testing.assert_allclose(a.grad.cpu().numpy(), gA, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(b.grad.cpu().numpy(), gB, rtol=1e-5, atol=1e-7)
    assert abs(G.grad.item() - gG) <= 1e-6 * abs(gG)


def test_backward_requires_recorded_run():
    from paper_2112_08264_gb300 import _lib
    s = Solver(6, 6, 6, 1.0, 0.5)
    rA, rB = inputs.spinodal(6, 6, 6)
    s.init(dev(rA), dev(rB))
    s.step(3)
    with pytest.raises(_lib.LbError) as e:
        s.backward(dev(np.ones((6, 6, 6))))
    assert e.value.status == _lib.LB_ESTATE
    r = Solver(6, 6, 6, 1.0, 0.5, ckpt_every=2, ckpt_steps_max=4)
    r.init(dev(rA), dev(rB))
    r.step(4)
    with pytest.raises(_lib.LbError) as e:
        r.step(1)          # beyond ckpt_steps_max
    assert e.value.status == _lib.LB_ESTATE
