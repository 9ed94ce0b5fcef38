"""Pins of the oracle's derivative machinery used to check the adjoint.

The complex-step directional derivative of the numpy formulation must equal
the central finite difference of the C oracle (an independent code path) to
the finite-difference error, for directions in the initial rho_A field, the
initial rho_B field and the coupling G."""
import numpy as np
import pytest

import oracle
from oracle import lb_numpy as lnp
from paper_2112_08264_gb300 import inputs


def _c_loss(rA, rB, G, target, steps, tau, mask=None):
    f = oracle.init(rA, rB, mask=mask)
    f = oracle.run(f, steps, tau, G, mask=mask)
    return oracle.loss(f, target, mask)


@pytest.mark.parametrize("masked", [False, True])
def test_complex_step_matches_central_differences(masked):
    nx, ny, nz, steps, tau, G = 6, 5, 4, 8, 0.9, 0.65
    rA, rB = inputs.spinodal(nx, ny, nz, seed=12)
    target = inputs.smoothed_target(nx, ny, nz, seed=13)
    mask = inputs.random_mask(nx, ny, nz, seed=14, solid_fraction=0.15) if masked else None
    rng = np.random.default_rng(15)
    vA = rng.normal(size=rA.shape)
    vB = rng.normal(size=rB.shape)
    for dA, dB, dG in [(vA, None, 0.0), (None, vB, 0.0), (None, None, 1.0), (vA, vB, 0.5)]:
        cs = lnp.jvp(rA, rB, G, target, steps, tau, dA, dB, dG, mask=mask)
        h = 1e-5
        pa = rA + (h * dA if dA is not None else 0)
        ma = rA - (h * dA if dA is not None else 0)
        pb = rB + (h * dB if dB is not None else 0)
        mb = rB - (h * dB if dB is not None else 0)
        fd = (_c_loss(pa, pb, G + h * dG, target, steps, tau, mask)
              - _c_loss(ma, mb, G - h * dG, target, steps, tau, mask)) / (2 * h)
        assert abs(cs - fd) <= 1e-7 * max(abs(cs), 1e-12) + 1e-12


def test_complex_step_loss_real_part_is_the_loss():
    nx, ny, nz = 5, 4, 3
    rA, rB = inputs.spinodal(nx, ny, nz, seed=2)
    target = inputs.smoothed_target(nx, ny, nz, seed=3)
    real = lnp.loss(rA, rB, 0.65, target, 5, 1.0)
    cplx = lnp.loss(rA.astype(complex) + 1e-30j, rB.astype(complex), 0.65, target, 5, 1.0)
    assert abs(cplx.real - real) <= 1e-15 * abs(real)
    assert abs(real - _c_loss(rA, rB, 0.65, target, 5, 1.0)) <= 1e-13 * abs(real)
