"""FP64 CPU oracle for the two-component D3Q19 BGK Shan-Chen step.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs may import this
package. The product path (``paper_2112_08264_gb300``) never imports it, and
the two share no code: the only common module is the seeded input
generator, which holds none of the method's arithmetic.

Three independent formulations live here:

* ``lb_oracle.c`` (wrapped below): plain triple loops in the step order of the
  method -- densities, Shan-Chen force, velocity shift, BGK collision with
  the second-order equilibrium (Eq. LEQ), push streaming with halfway
  bounce-back at rest (Eq. LADDFLBE with u_b = 0).
* ``lb_numpy``: the same definition written with ``np.roll`` over whole
  fields, with its own enumeration of the velocity set; it runs in complex
  arithmetic, so complex-step differentiation gives exact directional
  derivatives for the adjoint checks.
* ``single_bgk``: one-component D3Q19 BGK, which the two-component step must
  reduce to at G = 0.
* ``particles``: moving rigid spheres (moving-wall bounce-back, link forces
  and torques, leap-frog, re-meshing) on the write-side state the library
  holds.

Arrays: populations ``f`` have shape ``(2, 19, nz, ny, nx)`` (component,
velocity in the library's public order, z, y, x), fields ``(nz, ny, nx)``,
velocities ``(3, nz, ny, nx)``; the mask is ``uint8`` with 1 = solid.
"""
import ctypes
import numpy as np

from .build import build_oracle

Q = 19
_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_ip = ctypes.POINTER(ctypes.c_int)


def lib():
    """Load (building first if needed) the C oracle."""
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build_oracle())
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        L.oracle_max_threads.restype = ctypes.c_int
        L.oracle_lattice.argtypes = [_ip, _dp, _ip]
        L.oracle_init.argtypes = [ctypes.c_int] * 3 + [_u8p, _dp, _dp, _dp, _dp]
        L.oracle_density_force.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double, _dp, _u8p, _dp, _dp, _dp]
        L.oracle_step.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double, ctypes.c_double, _dp, _u8p, _dp, _dp]
        L.oracle_step.restype = ctypes.c_int
        L.oracle_run.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double, ctypes.c_double, _dp, _u8p, ctypes.c_int, _dp]
        L.oracle_run.restype = ctypes.c_int
        L.oracle_moments.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double, _dp, _u8p, _dp, _dp, _dp, _dp]
        L.oracle_stats.argtypes = [ctypes.c_int] * 3 + [_u8p, _dp, _dp]
        _lib = L
    return _lib


def _d(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _m(mask):
    return None if mask is None else mask.ctypes.data_as(_u8p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _mask(mask):
    return None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)


def _g(g):
    return None if g is None else _f64(np.asarray(g, dtype=np.float64).reshape(3))


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def lattice():
    """The C oracle's velocity set, weights and opposite-direction table."""
    c = np.zeros(3 * Q, dtype=np.int32)
    w = np.zeros(Q, dtype=np.float64)
    opp = np.zeros(Q, dtype=np.int32)
    lib().oracle_lattice(c.ctypes.data_as(_ip), _d(w), opp.ctypes.data_as(_ip))
    return c.reshape(Q, 3), w, opp


def init(rhoA, rhoB, u=None, mask=None):
    """Equilibrium populations f_i^k = f_i^eq(rho^k, u) (0 at solid nodes)."""
    rhoA, rhoB = _f64(rhoA), _f64(rhoB)
    nz, ny, nx = rhoA.shape
    u = None if u is None else _f64(u)
    mask = _mask(mask)
    f = np.zeros((2, Q, nz, ny, nx), dtype=np.float64)
    lib().oracle_init(nx, ny, nz, _m(mask), _d(rhoA), _d(rhoB), _d(u), _d(f))
    return f


def step(f, tau, G, g=None, mask=None):
    """One step; returns the new state (post-streaming populations)."""
    f = _f64(f)
    _, _, nz, ny, nx = f.shape
    mask, g = _mask(mask), _g(g)
    out = np.empty_like(f)
    rc = lib().oracle_step(nx, ny, nz, float(tau), float(G), _d(g), _m(mask), _d(f), _d(out))
    if rc:
        raise FloatingPointError("oracle_step: non-positive component density at a fluid node")
    return out


def run(f, nsteps, tau, G, g=None, mask=None):
    """n steps; returns a new array."""
    f = _f64(f).copy()
    _, _, nz, ny, nx = f.shape
    mask, g = _mask(mask), _g(g)
    rc = lib().oracle_run(nx, ny, nz, float(tau), float(G), _d(g), _m(mask), int(nsteps), _d(f))
    if rc:
        raise FloatingPointError("oracle_run: non-positive component density at a fluid node")
    return f


def density_force(f, G, g=None, mask=None):
    """Densities rho (2, nz, ny, nx) and force F (2, 3, nz, ny, nx)."""
    f = _f64(f)
    _, _, nz, ny, nx = f.shape
    mask, g = _mask(mask), _g(g)
    rho = np.empty((2, nz, ny, nx))
    F = np.empty((2, 3, nz, ny, nx))
    lib().oracle_density_force(nx, ny, nz, float(G), _d(g), _m(mask), _d(f), _d(rho), _d(F))
    return rho, F


def moments(f, G, g=None, mask=None):
    """(rho_A, rho_B, u) with u the half-force-corrected mixture velocity."""
    f = _f64(f)
    _, _, nz, ny, nx = f.shape
    mask, g = _mask(mask), _g(g)
    rA = np.empty((nz, ny, nx))
    rB = np.empty((nz, ny, nx))
    u = np.empty((3, nz, ny, nx))
    lib().oracle_moments(nx, ny, nz, float(G), _d(g), _m(mask), _d(f), _d(rA), _d(rB), _d(u))
    return rA, rB, u


def stats(f, mask=None):
    """[mass_A, mass_B, Px, Py, Pz] over fluid nodes."""
    f = _f64(f)
    _, _, nz, ny, nx = f.shape
    mask = _mask(mask)
    out = np.zeros(5)
    lib().oracle_stats(nx, ny, nz, _m(mask), _d(f), _d(out))
    return out


def loss(f_final, target, mask=None):
    """Sum over sites of (rho_A(final) - target)^2."""
    rA = f_final[0].sum(axis=0)
    if mask is not None:
        rA = rA * (np.asarray(mask) == 0)
    return float(((rA - target) ** 2).sum())
