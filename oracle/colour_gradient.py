"""Two-component D3Q19 colour-gradient (CG) step, plain numpy FP64.

TEST INFRASTRUCTURE (see the package docstring): only tests, the smoke check
and the benchmark's CPU legs use it; the CUDA path shares nothing with it.

The step follows the paper's Appendix (colour-gradient model), sub-step by
sub-step, on periodic grids without solid nodes:

  densities      rho^k = sum_i f_i^k, rho = rho^A + rho^B,
                 rho u = sum_k sum_i f_i^k c_i                 (Appendix, moments)
  relaxation     1/nu_bar = (rho^A/rho)/nu_A + (rho^B/rho)/nu_B,
                 omega = 2 / (6 nu_bar + 1)                     (Eq. 1coll; read
                   with "+1": omega = 1/tau and nu = (tau - 1/2)/3)
                 f^k,(1) = f^k + omega (f^k,eq(rho^k, u) - f^k)  (Eq. 1coll, Eq. LEQ)
  perturbation   Theta = (rho^A - rho^B)/rho, grad Theta = (1/c_s^2) sum_i w_i c_i Theta(x + c_i),
                 A = 9 omega sigma / 4                          (Eq. sigmaA, A_1 = A_2 = A)
                 f^k,(2) = f^k,(1) + (A/2) |grad Theta| [w_i (c_i . grad Theta)^2
                           / |grad Theta|^2 - B_i]              (Eq. 2coll, table B_i)
  recolouring    f*_i = sum_k f_i^k,(2), f^eq,0_i = w_i rho,
                 f^A_i = (rho^A/rho) f*_i + beta (rho^A rho^B / rho^2) cos(phi_i) f^eq,0_i
                 f^B_i = (rho^B/rho) f*_i - beta (rho^A rho^B / rho^2) cos(phi_i) f^eq,0_i
                 with rho^2 the square of the total density and cos(phi_i) =
                 c_i . grad Theta / (|c_i| |grad Theta|), 0 for the rest
                 velocity or a vanishing gradient               (Eq. 3coll)
  streaming      f_i^k(x + c_i, t + 1) = f^k_i(x)               (Eq. CGLBE)

The perturbation and recolouring act only where |grad Theta| > GRAD_MIN =
1e-5 (the paper does not say how a vanishing gradient is treated; cos(phi_i)
has no limit there, and a gradient at the rounding level of a float32 state
has no meaningful direction). Populations are ``(2, 19, nz, ny, nx)`` in the velocity order of
``lb_numpy`` (``to_public`` / ``from_public`` map to the library's order).
"""
import numpy as np

from .lb_numpy import CS2, VEL, W, equilibrium, shift_from, shift_to

# B_i of the Appendix coefficient table, by |c|^2 = 0, 1, 2
_B_BY_C2 = {0: -2.0 / 9.0, 1: 1.0 / 54.0, 2: 1.0 / 27.0}
GRAD_MIN = 1e-5
B = np.array([_B_BY_C2[int((c * c).sum())] for c in VEL])
CNORM = np.sqrt((VEL * VEL).sum(axis=1).astype(np.float64))


def omega_of(rhoA, rhoB, nuA, nuB):
    """Relaxation rate from the mean viscosity of the mixture (Eq. 1coll)."""
    rho = rhoA + rhoB
    inv_nu = (rhoA / rho) / nuA + (rhoB / rho) / nuB
    return 2.0 / (6.0 / inv_nu + 1.0)


def phase_gradient(rhoA, rhoB):
    """Theta and its isotropic gradient (1/c_s^2) sum_i w_i c_i Theta(x + c_i)."""
    theta = (rhoA - rhoB) / (rhoA + rhoB)
    grad = np.zeros((3,) + theta.shape)
    for i, c in enumerate(VEL):
        if not c.any():
            continue
        nb = shift_from(theta, c)
        for a in range(3):
            if c[a]:
                grad[a] = grad[a] + W[i] * c[a] * nb
    return theta, grad / CS2


def perturbation(A, grad):
    """(Omega_i^k)^(2) of Eq. 2coll for one component: shape (19, ...)."""
    g2 = (grad * grad).sum(axis=0)
    gn = np.sqrt(g2)
    nz = gn > GRAD_MIN
    out = []
    for i, c in enumerate(VEL):
        cg = c[0] * grad[0] + c[1] * grad[1] + c[2] * grad[2]
        term = np.where(nz, W[i] * cg * cg / np.where(nz, g2, 1.0) - B[i], 0.0)
        out.append(0.5 * A * gn * term)
    return np.stack(out)


def cos_phi(grad):
    """cos of the angle between c_i and grad Theta: shape (19, ...)."""
    gn = np.sqrt((grad * grad).sum(axis=0))
    nz = gn > GRAD_MIN
    out = []
    for i, c in enumerate(VEL):
        if not c.any():
            out.append(np.zeros_like(gn))
            continue
        cg = c[0] * grad[0] + c[1] * grad[1] + c[2] * grad[2]
        out.append(np.where(nz, cg / (CNORM[i] * np.where(nz, gn, 1.0)), 0.0))
    return np.stack(out)


def collide(f, nuA, nuB, sigma, beta):
    """Post-collision populations (before streaming), this module's order."""
    rhoA, rhoB = f[0].sum(axis=0), f[1].sum(axis=0)
    rho = rhoA + rhoB
    u = np.einsum("kiabc,id->dabc", f, VEL.astype(np.float64)) / rho
    omega = omega_of(rhoA, rhoB, nuA, nuB)
    _, grad = phase_gradient(rhoA, rhoB)
    A = 9.0 * omega * sigma / 4.0
    pert = perturbation(A, grad)
    fstar = 0.0
    for k, rk in enumerate((rhoA, rhoB)):
        f1 = f[k] + omega * (equilibrium(rk, u) - f[k])
        fstar = fstar + f1 + pert
    cphi = cos_phi(grad)
    feq0 = W[:, None, None, None] * rho
    colour = beta * (rhoA * rhoB / (rho * rho)) * cphi * feq0
    return np.stack([(rhoA / rho) * fstar + colour, (rhoB / rho) * fstar - colour])


def step(f, nuA, nuB, sigma, beta):
    """One colour-gradient step on post-streaming populations (periodic)."""
    post = collide(f, nuA, nuB, sigma, beta)
    out = np.empty_like(post)
    for k in range(2):
        for i, c in enumerate(VEL):
            out[k, i] = shift_to(post[k, i], c)
    return out


def run(f, nsteps, nuA, nuB, sigma, beta):
    for _ in range(nsteps):
        f = step(f, nuA, nuB, sigma, beta)
    return f


def moments(f):
    """rho^A, rho^B and the barycentric velocity u = sum_k sum_i f c / rho."""
    rhoA, rhoB = f[0].sum(axis=0), f[1].sum(axis=0)
    u = np.einsum("kiabc,id->dabc", f, VEL.astype(np.float64)) / (rhoA + rhoB)
    return rhoA, rhoB, u
