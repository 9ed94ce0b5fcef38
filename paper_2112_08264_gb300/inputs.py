"""Seeded synthetic inputs: initial density fields, colloid masks, loss targets.

This module holds none of the lattice-Boltzmann arithmetic. It only draws the
fields that both the CUDA path and the CPU oracle start from, so the same
arrays go to both sides. Every generator is numpy's PCG64 ``default_rng(seed)``
in float64; arrays are indexed ``[z, y, x]`` (x fastest, matching the site
index s = x + nx*(y + ny*z)).

Workload recipes (the paper's synthetic set-ups, Sec. 5):
  * ``spinodal``: rho_A = mean + amp*U(-1,1) per site, rho_B = 1 - rho_A,
    zero velocity -- a randomly filled two-fluid box as in the paper's case 2,
    with small-amplitude noise (default 0.5 +- 0.05, seed 1234).
  * ``random_order_parameter``: the paper's case-2 fill, phi = (rho_r - rho_b)
    / (rho_r + rho_b) = +-phi0 at random per site; phi0 < 1 keeps both
    densities positive, which the Shan-Chen velocity shift needs.
  * ``colloid_mask``: static solid spheres of radius R at uniformly random,
    non-overlapping centres (periodic distance >= 2R + 1), the paper's random
    particle placement of case 3 (Sec. 5.3) without particle motion.
  * ``smoothed_target``: a smooth random target field for the adjoint loss.
"""
import numpy as np


def spinodal(nx, ny, nz, seed=1234, mean=0.5, amp=0.05):
    """Return (rho_A, rho_B), each float64 of shape (nz, ny, nx)."""
    rng = np.random.default_rng(seed)
    rho_a = mean + amp * rng.uniform(-1.0, 1.0, size=(nz, ny, nx))
    return rho_a, 1.0 - rho_a


def random_order_parameter(nx, ny, nz, seed=1234, phi0=0.9, total=1.0):
    """Sites drawn at random with order parameter +phi0 or -phi0."""
    rng = np.random.default_rng(seed)
    phi = np.where(rng.integers(0, 2, size=(nz, ny, nx)) == 1, phi0, -phi0)
    rho_a = 0.5 * total * (1.0 + phi)
    return rho_a, total - rho_a


def colloid_mask(nx, ny, nz, n_spheres=4000, radius=5.0, seed=4321, max_tries=2_000_000):
    """uint8 mask (1 = solid) of ``n_spheres`` spheres; also returns the centres.

    A site is solid when its periodic distance to a centre is <= radius.
    Centres are rejection-sampled until every pair is at periodic distance
    >= 2*radius + 1.
    """
    rng = np.random.default_rng(seed)
    box = np.array([nx, ny, nz], dtype=np.float64)
    dmin2 = (2.0 * radius + 1.0) ** 2
    centres = np.empty((n_spheres, 3))
    n = 0
    tries = 0
    while n < n_spheres:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("colloid_mask: could not place %d spheres" % n_spheres)
        c = rng.uniform(0.0, 1.0, size=3) * box
        if n:
            d = np.abs(centres[:n] - c)
            d = np.minimum(d, box - d)
            if (d * d).sum(axis=1).min() < dmin2:
                continue
        centres[n] = c
        n += 1
    mask = np.zeros((nz, ny, nx), dtype=np.uint8)
    r = int(np.ceil(radius)) + 1
    off = np.arange(-r, r + 1)
    ox, oy, oz = np.meshgrid(off, off, off, indexing="ij")
    ox, oy, oz = ox.ravel(), oy.ravel(), oz.ravel()
    for c in centres:
        bx, by, bz = np.floor(c).astype(np.int64)
        px, py, pz = bx + ox, by + oy, bz + oz
        dx, dy, dz = px - c[0], py - c[1], pz - c[2]
        inside = dx * dx + dy * dy + dz * dz <= radius * radius
        mask[pz[inside] % nz, py[inside] % ny, px[inside] % nx] = 1
    return mask, centres


def smoothed_target(nx, ny, nz, seed=99, mean=0.5, amp=0.05, passes=3):
    """Uniform noise smoothed by ``passes`` periodic 3x3x3 box filters, then
    rescaled to mean +- amp (max deviation = amp)."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1.0, 1.0, size=(nz, ny, nx))
    for _ in range(passes):
        acc = np.zeros_like(a)
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    acc += np.roll(a, shift=(dz, dy, dx), axis=(0, 1, 2))
        a = acc / 27.0
    a = a - a.mean()
    m = np.abs(a).max()
    return mean + amp * a / (m if m > 0 else 1.0)


def random_mask(nx, ny, nz, seed=7, solid_fraction=0.2):
    """Independent random solid sites (small brute-force cases)."""
    rng = np.random.default_rng(seed)
    return (rng.uniform(size=(nz, ny, nx)) < solid_fraction).astype(np.uint8)
