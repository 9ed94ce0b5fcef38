"""One-component D3Q19 BGK, written on its own (TEST INFRASTRUCTURE).

At G = 0 the two-component Shan-Chen step must act on the summed populations
f = f^A + f^B exactly as this one-component update does (the equilibrium is
linear in rho at a common velocity, Eq. LEQ), with the body force entering as
the velocity shift u_eq = u + tau g. Periodic, no solid nodes.
Populations are ``(19, nz, ny, nx)`` in the order of ``VELOCITIES`` below.
"""
import numpy as np

VELOCITIES = np.array([[0, 0, 0]]
                      + [[s * (a == d) for d in range(3)] for a in range(3) for s in (1, -1)]
                      + [[s * (d == a) + t * (d == b) for d in range(3)]
                         for a in range(3) for b in range(a + 1, 3) for s in (1, -1) for t in (1, -1)])
WEIGHTS = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def step(f, tau, g=(0.0, 0.0, 0.0)):
    c = VELOCITIES.astype(float)
    rho = f.sum(axis=0)
    u = np.einsum("id,iabc->dabc", c, f) / rho + tau * np.asarray(g, float)[:, None, None, None]
    cu = np.einsum("id,dabc->iabc", c, u)
    uu = (u * u).sum(axis=0)
    feq = WEIGHTS[:, None, None, None] * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu)
    post = f - (f - feq) / tau
    return np.stack([np.roll(post[i], shift=tuple(VELOCITIES[i][::-1]), axis=(0, 1, 2))
                     for i in range(19)])


def velocity_index(cvec):
    """Index in VELOCITIES of the velocity vector ``cvec``."""
    return int(np.where((VELOCITIES == np.asarray(cvec)).all(axis=1))[0][0])
