"""Pins of the oracle step against exact invariants and closed forms.

* Mass of each component is invariant (collision keeps sum_i f_i^k since
  sum_i f_i^eq = rho^k by the lattice sums; streaming and bounce-back only
  move populations).
* Periodic, no body force: the Shan-Chen forces of the two components sum to
  zero over the box (index swap x -> x - c_i, i -> opposite), and with the
  common velocity u' the collision adds exactly sum_k F^k at each node, so
  total momentum is invariant. With a body force g it grows by g * M per step.
* A uniform mixture (any u) is a fixed point.
* A single density bump gives the force of one link in closed form.
* At G = 0 the summed populations follow one-component BGK.
"""
import numpy as np
import pytest

import oracle
from oracle import single_bgk
from paper_2112_08264_gb300 import inputs

TAU, G = 1.0, 0.65


def _random_state(n, seed, mask=None):
    rng = np.random.default_rng(seed)
    f = rng.uniform(0.01, 0.06, size=(2, 19, n[2], n[1], n[0]))
    if mask is not None:
        f[:, :, mask == 1] = 0.0
    return f


@pytest.mark.parametrize("masked", [False, True])
def test_mass_per_component_invariant(masked):
    nx, ny, nz = 12, 10, 8
    mask = inputs.random_mask(nx, ny, nz, seed=11, solid_fraction=0.15) if masked else None
    rA, rB = inputs.spinodal(nx, ny, nz, seed=5)
    f = oracle.init(rA, rB, mask=mask)
    s0 = oracle.stats(f, mask)
    for _ in range(20):
        f = oracle.step(f, 0.8, 1.3, mask=mask)
        s = oracle.stats(f, mask)
        assert abs(s[0] - s0[0]) / s0[0] < 1e-13
        assert abs(s[1] - s0[1]) / s0[1] < 1e-13


def test_momentum_invariant_periodic():
    nx, ny, nz = 12, 10, 8
    rA, rB = inputs.spinodal(nx, ny, nz, seed=6, amp=0.2)
    u = np.random.default_rng(1).normal(scale=0.01, size=(3, nz, ny, nx))
    f = oracle.init(rA, rB, u)
    p0 = oracle.stats(f)
    M = p0[0] + p0[1]
    for _ in range(20):
        f = oracle.step(f, 0.9, 0.9)
        p = oracle.stats(f)
        assert np.abs(p[2:] - p0[2:]).max() <= 1e-13 * M


def test_forces_cancel_over_periodic_box():
    f = _random_state((9, 8, 7), seed=3)
    rho, F = oracle.density_force(f, 1.7)
    tot = F.sum(axis=(2, 3, 4)).sum(axis=0)
    scale = np.abs(F).sum()
    assert np.abs(tot).max() <= 1e-14 * scale
    # each component alone does not cancel (the check is not vacuous)
    assert np.abs(F[0].sum(axis=(1, 2, 3))).max() > 1e-6 * scale


def test_body_force_momentum_growth():
    nx, ny, nz = 8, 8, 8
    g = np.array([2e-5, -1e-5, 3e-6])
    rA, rB = inputs.spinodal(nx, ny, nz, seed=8)
    f = oracle.init(rA, rB)
    for _ in range(10):
        p0 = oracle.stats(f)
        f = oracle.step(f, TAU, G, g)
        p1 = oracle.stats(f)
        M = p0[0] + p0[1]
        np.testing.assert_allclose(p1[2:] - p0[2:], g * M, rtol=1e-9, atol=1e-14 * M)


@pytest.mark.parametrize("u0", [(0.0, 0.0, 0.0), (0.03, -0.02, 0.01)])
def test_uniform_mixture_is_fixed_point(u0):
    n = 6
    rA = np.full((n, n, n), 0.3)
    rB = np.full((n, n, n), 0.8)
    u = np.broadcast_to(np.asarray(u0)[:, None, None, None], (3, n, n, n)).copy()
    f0 = oracle.init(rA, rB, u)
    f = oracle.run(f0, 5, 0.7, 1.4)
    np.testing.assert_allclose(f, f0, rtol=0, atol=1e-15)
    if not any(u0):
        c, w, _ = oracle.lattice()
        np.testing.assert_allclose(f[0], np.broadcast_to(w[:, None, None, None] * 0.3, f[0].shape),
                                   rtol=0, atol=1e-15)


def test_single_bump_force_closed_form():
    """psi^B = b + d at one node x0 only, psi^A uniform a: the force on A at
    x0 - c_j is -G a w_j d c_j (only the link j reaches the bump), and zero
    two sites away."""
    n = 7
    a, b, d, Gv = 0.4, 0.6, 0.05, 1.2
    rA = np.full((n, n, n), a)
    rB = np.full((n, n, n), b)
    x0 = (3, 3, 3)
    rB[x0[2], x0[1], x0[0]] += d
    f = oracle.init(rA, rB)
    rho, F = oracle.density_force(f, Gv)
    c, w, _ = oracle.lattice()
    for j in range(1, 19):
        x, y, z = (x0[0] - c[j][0]) % n, (x0[1] - c[j][1]) % n, (x0[2] - c[j][2]) % n
        np.testing.assert_allclose(F[0, :, z, y, x], -Gv * a * w[j] * d * c[j], rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(F[0, :, 0, 0, 0], 0.0, atol=1e-16)
    # the bump itself feels the uniform A field only: no force on B at x0
    np.testing.assert_allclose(F[1, :, x0[2], x0[1], x0[0]], 0.0, atol=1e-16)


def test_component_swap_symmetry():
    f = _random_state((6, 5, 4), seed=21)
    g = (1e-4, 0.0, -2e-4)
    a = oracle.step(f, 0.85, 1.1, g)
    b = oracle.step(f[::-1].copy(), 0.85, 1.1, g)
    np.testing.assert_allclose(a, b[::-1], rtol=0, atol=1e-16)


def test_zero_coupling_reduces_to_one_component_bgk():
    nx, ny, nz = 7, 6, 5
    f = _random_state((nx, ny, nz), seed=4)
    g = (3e-5, -1e-5, 2e-5)
    c_lib, _, _ = oracle.lattice()
    order = [single_bgk.velocity_index(v) for v in c_lib]   # library order -> single_bgk order
    s = np.empty((19, nz, ny, nx))
    s[order] = f[0] + f[1]
    for _ in range(12):
        f = oracle.step(f, 0.75, 0.0, g)
        s = single_bgk.step(s, 0.75, g)
        np.testing.assert_allclose((f[0] + f[1]), s[order], rtol=0, atol=1e-13)
