"""Pins of the colour-gradient oracle (Appendix: Eq. 1coll, 2coll, 3coll and
the coefficient table), each against something other than the oracle itself:
exact conservation, the reduction to one-component BGK, closed-form moments
of the perturbation and recolouring operators, and the Laplace law."""
import numpy as np
import pytest

from oracle import colour_gradient as cg
from oracle import lb_numpy as ln
from oracle import single_bgk


def random_state(n=10, seed=3, amp_u=0.02):
    rng = np.random.default_rng(seed)
    rA = 0.5 + 0.4 * rng.uniform(-1, 1, (n, n, n))
    rB = 1.0 - rA + 0.05 * rng.uniform(-1, 1, (n, n, n))
    u = amp_u * rng.uniform(-1, 1, (3, n, n, n))
    return ln.init(rA, rB, u)


def test_coefficient_table_isotropy():
    """The B_i of the table satisfy the isotropy constraints under Eq. 2coll."""
    c = ln.VEL.astype(float)
    assert abs(cg.B.sum() - 1.0 / 3.0) < 1e-15
    assert np.abs(np.einsum("i,ia->a", cg.B, c)).max() < 1e-15
    assert np.abs(np.einsum("i,ia,ib->ab", cg.B, c, c) - np.eye(3) / 3.0).max() < 1e-15


def test_mass_per_component_and_momentum_conserved():
    f = random_state()
    m0 = f.sum(axis=(1, 2, 3, 4))
    p0 = np.einsum("kiabc,id->d", f, ln.VEL.astype(float))
    for _ in range(5):
        f = cg.step(f, 1.0 / 6.0, 1.0 / 10.0, 0.02, 0.7)
    m1 = f.sum(axis=(1, 2, 3, 4))
    p1 = np.einsum("kiabc,id->d", f, ln.VEL.astype(float))
    assert np.abs(m1 - m0).max() < 1e-11 * m0.max()
    assert np.abs(p1 - p0).max() < 1e-11 * m0.max()


@pytest.mark.parametrize("nu", [1.0 / 6.0, 0.05, 0.3])
def test_reduces_to_one_component_bgk(nu):
    """sigma = beta = 0 and equal viscosities: the total f = f^A + f^B evolves
    as one-component BGK with tau = 3 nu + 1/2 (this pins the reading
    omega = 2 / (6 nu + 1) of Eq. 1coll)."""
    f = random_state(n=8, seed=5)
    tau = 3.0 * nu + 0.5
    tot = f[0] + f[1]
    order = [single_bgk.velocity_index(c) for c in ln.VEL]
    g = np.empty_like(tot)
    g[order] = tot
    for _ in range(4):
        f = cg.step(f, nu, nu, 0.0, 0.0)
        g = single_bgk.step(g, tau)
    assert np.abs((f[0] + f[1]) - g[order]).max() < 1e-13


def test_perturbation_moments_closed_form():
    """sum_i P_i = 0, sum_i P_i c_i = 0 and sum_i P_i c_i c_i = (A/9)|g|(n n - I),
    from sum_i w_i c c c c = (I I + ...)/9 and sum_i B_i c c = I/3."""
    rng = np.random.default_rng(11)
    grad = rng.normal(size=(3, 4, 4, 4))
    A = 0.37
    P = cg.perturbation(A, grad)
    c = ln.VEL.astype(float)
    gn = np.sqrt((grad * grad).sum(axis=0))
    n = grad / gn
    assert np.abs(P.sum(axis=0)).max() < 1e-14
    assert np.abs(np.einsum("iabc,id->dabc", P, c)).max() < 1e-14
    M = np.einsum("iabc,id,ie->deabc", P, c, c)
    want = (A / 9.0) * gn * (np.einsum("dabc,eabc->deabc", n, n) - np.eye(3)[:, :, None, None, None])
    assert np.abs(M - want).max() < 1e-13


def test_recolouring_flux_closed_form():
    """The recolouring moves colour along grad Theta: sum_i c_i X_i =
    beta (rho^A rho^B / rho) (1 + sqrt 2)/9 n, with X_i the recolouring term,
    since sum_i w_i c_i (c_i . n)/|c_i| = (1 + sqrt 2)/9 n on D3Q19."""
    rng = np.random.default_rng(2)
    grad = rng.normal(size=(3, 3, 3, 3))
    cphi = cg.cos_phi(grad)
    n = grad / np.sqrt((grad * grad).sum(axis=0))
    flux = np.einsum("i,iabc,id->dabc", ln.W, cphi, ln.VEL.astype(float))
    assert np.abs(flux - (1.0 + np.sqrt(2.0)) / 9.0 * n).max() < 1e-14
    assert np.abs(np.einsum("i,iabc->abc", ln.W, cphi)).max() < 1e-15   # colour mass conserved


def test_flat_interface_at_rest_stays_symmetric():
    """A flat A|B slab stays at rest and mirror-symmetric (no spurious drift)."""
    n = 16
    x = np.arange(n)
    phi = np.where((x >= n // 4) & (x < 3 * n // 4), 0.9, -0.9)[None, None, :] * np.ones((4, 4, n))
    f = ln.init(0.5 * (1 + phi), 0.5 * (1 - phi))
    f = cg.run(f, 200, 1.0 / 6.0, 1.0 / 6.0, 0.01, 0.7)
    rA, rB, u = cg.moments(f)
    assert np.abs(u).max() < 1e-10
    prof = rA[0, 0]
    assert np.abs(prof - prof[::-1]).max() < 1e-12   # mirror about the slab centre (x = 7.5)
    assert prof.max() > 0.9 and prof.min() < 0.1                             # stays segregated


def test_laplace_law():
    """A droplet of radius R: the pressure jump c_s^2 (rho_in - rho_out)
    follows 2 sigma / R (Eq. sigmaA relates sigma to A)."""
    n, sigma = 24, 0.01
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    out = []
    for R in (5.0, 7.0):
        r = np.sqrt((x - n / 2 + 0.5) ** 2 + (y - n / 2 + 0.5) ** 2 + (z - n / 2 + 0.5) ** 2)
        phi = np.where(r < R, 0.95, -0.95)
        f = ln.init(0.5 * (1 + phi), 0.5 * (1 - phi))
        f = cg.run(f, 500, 1.0 / 6.0, 1.0 / 6.0, sigma, 0.7)
        rA, rB, _ = cg.moments(f)
        rho = rA + rB
        dp = ln.CS2 * (rho[r < R - 3].mean() - rho[r > R + 3].mean())
        out.append(dp * R / (2 * sigma))
    assert all(abs(v - 1.0) < 0.1 for v in out), out   # measured 1.04 and 1.00


@pytest.mark.parametrize("gmax,active", [(1.2e-5, True), (0.8e-5, False)])
def test_gradient_threshold_decides(gmax, active):
    """The perturbation and the recolouring act only where |grad Theta| >
    GRAD_MIN = 1e-5 (the reading for a vanishing gradient, whose direction is
    undefined). A near-pure phase rho^A = 1 - eps(y), rho^B = eps(y) with a
    sine eps scaled so that max |grad Theta| is 1.2e-5 (above) or 0.8e-5
    (below): above, the collision differs from plain BGK (sigma = beta = 0)
    exactly at the nodes whose gradient passes the threshold; below, it is
    plain BGK at every node. A threshold on |grad Theta|^2, or none at all,
    fails one of the two cases."""
    n = 12
    y = np.arange(n)
    shape = np.broadcast_to(np.sin(2 * np.pi * y / n)[None, :, None], (n, n, n))
    # Theta = 1 - 2 eps at rho = 1, so grad Theta is linear in the amplitude
    eps0 = 1e-3 + 1e-4 * shape
    _, g0 = cg.phase_gradient(1.0 - eps0, eps0)
    g0n = np.sqrt((g0 * g0).sum(axis=0))
    amp = 1e-4 * gmax / g0n.max()
    eps = 1e-3 + amp * shape
    rA, rB = 1.0 - eps, eps
    _, grad = cg.phase_gradient(rA, rB)
    gn = np.sqrt((grad * grad).sum(axis=0))
    assert abs(gn.max() - gmax) <= 1e-3 * gmax
    f = ln.init(rA, rB, np.zeros((3, n, n, n)))
    nu = 1.0 / 6.0
    full = cg.collide(f, nu, nu, 0.01, 0.7)
    plain = cg.collide(f, nu, nu, 0.0, 0.0)
    diff = np.abs(full - plain).max(axis=(0, 1))
    if active:
        over = gn > cg.GRAD_MIN
        assert over.any() and (~over).any()
        assert np.all(diff[over] > 1e-12)
        assert np.all(diff[~over] == 0.0)
    else:
        assert np.all(diff == 0.0)
