"""Whole-field numpy formulation of the two-component D3Q19 BGK Shan-Chen step.

TEST INFRASTRUCTURE (see the package docstring). It is written apart from the
C oracle -- its own enumeration of the velocity set, ``np.roll`` for every
neighbour access, field-at-a-time arithmetic -- so that agreement between the
two pins both. Every operation is complex-analytic in the populations and in
G (sums, products, quotients, permutations), so running it on complex inputs
gives complex-step derivatives: Im L(x + i h v) / h = dL/dx . v to rounding
for tiny h, with no cancellation.

Populations here are ``(2, 19, nz, ny, nx)`` in THIS module's velocity order
``VEL``; ``to_public`` / ``from_public`` map to and from the library's public
order (rest, +-x, +-y, +-z, then the diagonals in opposite pairs).

Definitions followed: D3Q19 set and weights (Sec. 2 Method; Appendix table),
moments (Appendix), Eq. LEQ equilibrium, Eq. bgk relaxation and streaming,
halfway bounce-back at rest (Eq. LADDFLBE with u_b = 0); Shan-Chen force
F^A = -G psi^A sum_i w_i psi^B(x + c_i) c_i with psi = rho (0 on solid nodes)
and the velocity-shift forcing u_eq^k = u' + tau F^k / rho^k.
"""
import itertools
import numpy as np

# all (cx, cy, cz) in {-1,0,1}^3 with |c|^2 <= 2: 1 + 6 + 12 = 19 velocities
VEL = np.array([c for c in itertools.product((-1, 0, 1), repeat=3)
                if c[0] * c[0] + c[1] * c[1] + c[2] * c[2] <= 2], dtype=np.int64)
_W_BY_C2 = {0: 1.0 / 3.0, 1: 1.0 / 18.0, 2: 1.0 / 36.0}
W = np.array([_W_BY_C2[int((c * c).sum())] for c in VEL])
OPP = np.array([int(np.where((VEL == -c).all(axis=1))[0][0]) for c in VEL])
CS2 = 1.0 / 3.0

# the library's public velocity order, written out as vectors
PUBLIC = np.array([
    (0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
    (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1),
    (1, 0, -1), (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)], dtype=np.int64)
# PERM[p] = index in VEL of public velocity p
PERM = np.array([int(np.where((VEL == c).all(axis=1))[0][0]) for c in PUBLIC])


def to_public(f):
    return f[:, PERM]


def from_public(f):
    out = np.empty_like(f)
    out[:, PERM] = f
    return out


def shift_from(a, c):
    """Field whose value at x is a(x + c) (periodic)."""
    return np.roll(a, shift=(-int(c[2]), -int(c[1]), -int(c[0])), axis=(0, 1, 2))


def shift_to(a, c):
    """Field whose value at x + c is a(x) (periodic)."""
    return np.roll(a, shift=(int(c[2]), int(c[1]), int(c[0])), axis=(0, 1, 2))


def equilibrium(rho, u):
    """Eq. LEQ for every velocity: shape (19, ...)."""
    uu = (u * u).sum(axis=0)
    out = []
    for i, c in enumerate(VEL):
        cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2]
        out.append(W[i] * rho * (1 + cu / CS2 + cu * cu / (2 * CS2 * CS2) - uu / (2 * CS2)))
    return np.stack(out)


def init(rhoA, rhoB, u=None, mask=None):
    """Equilibrium populations (this module's order); 0 on solid nodes."""
    dtype = np.result_type(rhoA, rhoB, np.float64)
    if u is None:
        u = np.zeros((3,) + np.shape(rhoA), dtype=dtype)
    fluid = np.ones(np.shape(rhoA)) if mask is None else (np.asarray(mask) == 0).astype(np.float64)
    return np.stack([equilibrium(rhoA, u) * fluid, equilibrium(rhoB, u) * fluid])


def density_force(f, G, g=None, mask=None):
    fluid = np.ones(f.shape[2:]) if mask is None else (np.asarray(mask) == 0).astype(np.float64)
    rho = f.sum(axis=1) * fluid                       # psi = rho, 0 on solid
    F = []
    for k in range(2):
        other = rho[1 - k]
        acc = [0.0, 0.0, 0.0]
        for i, c in enumerate(VEL):
            if not c.any():
                continue
            nb = shift_from(other, c)
            for a in range(3):
                if c[a]:
                    acc[a] = acc[a] + W[i] * c[a] * nb
        Fk = [-G * rho[k] * acc[a] for a in range(3)]
        if g is not None:
            Fk = [Fk[a] + rho[k] * g[a] for a in range(3)]
        F.append(np.stack([Fk[a] * fluid for a in range(3)]))
    return rho, np.stack(F)


def step(f, tau, G, g=None, mask=None):
    """One step (this module's velocity order)."""
    fluid = np.ones(f.shape[2:]) if mask is None else (np.asarray(mask) == 0).astype(np.float64)
    solid = 1.0 - fluid
    rho, F = density_force(f, G, g, mask)
    mom = np.einsum("kiabc,id->dabc", f, VEL.astype(np.float64))
    safe = lambda r: r + solid                        # avoid 0/0 on solid nodes
    up = (mom / tau) / safe(rho[0] / tau + rho[1] / tau)
    post = []
    for k in range(2):
        ueq = up + tau * F[k] / safe(rho[k])
        post.append((f[k] - (f[k] - equilibrium(rho[k], ueq)) / tau) * fluid)
    out = np.zeros_like(f)
    for k in range(2):
        for i, c in enumerate(VEL):
            arrived = shift_to(post[k][i], c) * fluid          # destination fluid
            back = post[k][i] * fluid * shift_from(solid, c)   # destination solid
            out[k, i] = out[k, i] + arrived
            out[k, OPP[i]] = out[k, OPP[i]] + back
    return out


def run(f, nsteps, tau, G, g=None, mask=None):
    for _ in range(nsteps):
        f = step(f, tau, G, g, mask)
    return f


def moments(f, G, g=None, mask=None):
    fluid = np.ones(f.shape[2:]) if mask is None else (np.asarray(mask) == 0).astype(np.float64)
    rho, F = density_force(f, G, g, mask)
    mom = np.einsum("kiabc,id->dabc", f, VEL.astype(np.float64)) + 0.5 * (F[0] + F[1])
    r = rho[0] + rho[1]
    u = mom / (r + (1.0 - fluid)) * fluid
    return rho[0], rho[1], u


def loss(rhoA0, rhoB0, G, target, nsteps, tau, g=None, mask=None):
    """Sum over sites of (rho_A after nsteps - target)^2, from equilibrium
    initial populations at zero velocity (complex inputs allowed)."""
    f = init(rhoA0, rhoB0, mask=mask)
    f = run(f, nsteps, tau, G, g, mask)
    rA = f[0].sum(axis=0)
    if mask is not None:
        rA = rA * (np.asarray(mask) == 0)
    return ((rA - target) ** 2).sum()


def jvp(rhoA0, rhoB0, G, target, nsteps, tau, vA=None, vB=None, vG=0.0,
        g=None, mask=None, h=1e-30):
    """Directional derivative of ``loss`` along (vA, vB, vG) by complex step."""
    zA = np.asarray(rhoA0, dtype=np.complex128)
    zB = np.asarray(rhoB0, dtype=np.complex128)
    if vA is not None:
        zA = zA + 1j * h * np.asarray(vA)
    if vB is not None:
        zB = zB + 1j * h * np.asarray(vB)
    zG = complex(G) + 1j * h * vG
    return float(np.imag(loss(zA, zB, zG, target, nsteps, tau, g, mask)) / h)
