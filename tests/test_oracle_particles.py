"""Pins of the moving-particle oracle (``oracle.particles``) against what the
method and the mathematics fix, independently of its own code:

* fixed particles at rest are static solids: the state follows the C oracle's
  static-mask step (a separate formulation: push streaming with the bounce
  read-side);
* the total momentum of fluid and particles is conserved, through the
  moving-wall bounce (Eq. LADDFLBE), the link forces (Eq. FORCEPP,
  Eq. FORCEPARTEQ), the leap-frog update (Eq. PARDYN) and re-meshing;
* a uniform flow at the wall velocity is a fixed point with zero force and
  torque (the bias 2 rho w_i u_b . c_i / c_s^2 turns f^eq_i(U) into
  f^eq_opp(i)(U) exactly);
* a sphere centred on a node, rotating in fluid at rest, feels no force and
  a torque antiparallel to its rotation (the symmetry of the cubic link set
  fixes the direction, dissipation the sign);
* a translating particle that covers no new node conserves the fluid mass
  exactly (the bias sums to zero over the closed set of links).
"""
import numpy as np
import pytest

import oracle
from oracle import lb_numpy as ln
from oracle import particles as op


def fluid_fields(shape, seed, G):
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    rA = 0.5 + 0.05 * rng.uniform(-1, 1, shape)
    rB = 1.0 - rA
    u = 0.01 * rng.normal(size=(3,) + shape)
    return rA, rB, u


def test_fixed_particles_at_rest_are_static_solids():
    shape = (14, 16, 18)          # (nz, ny, nx)
    nz, ny, nx = shape
    parts = op.Particles([[4.3, 5.1, 6.6], [12.2, 11.4, 5.0]], radius=2.6, mass=0.0)
    owner = op.coverage(shape, parts.r, parts.radius)
    mask = (owner >= 0).astype(np.uint8)
    rA, rB, u = fluid_fields(shape, 1, 0.9)
    tau, G, steps = 0.8, 0.9, 6
    rho0 = (rA[mask == 0].mean(), rB[mask == 0].mean())
    g = op.init(rA, rB, u, None, owner)
    for _ in range(steps):
        g, owner = op.step(g, owner, None, parts, tau, G, rho0)
    got = ln.to_public(op.pulled(g, owner, None, parts, rho0))
    want = oracle.run(oracle.init(rA, rB, u, mask), steps, tau, G, None, mask)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    assert np.abs(parts.F).max() > 0          # the links were found


def test_total_momentum_is_conserved_through_remeshing():
    shape = (16, 16, 20)
    rA, rB, u = fluid_fields(shape, 2, 0.6)
    parts = op.Particles([[5.2, 6.1, 7.3], [14.6, 11.2, 8.4]], v=[[0.3, -0.2, 0.1], [-0.25, 0.1, 0.3]],
                         w=[[0.0, 0.01, -0.02], [0.02, 0.0, 0.01]], radius=2.4, mass=40.0)
    owner = op.coverage(shape, parts.r, parts.radius)
    rho0 = (0.5, 0.5)
    g = op.init(rA, rB, u, None, owner)
    owner0 = owner.copy()

    def total(g, owner):
        return op.fluid_momentum(g, owner, None) + parts.mass * parts.v.sum(axis=0)

    p0 = total(g, owner)
    scale = np.abs(g).sum() * 1e-2
    for _ in range(5):
        g, owner = op.step(g, owner, None, parts, 0.9, 0.6, rho0)
        assert np.abs(total(g, owner) - p0).max() <= 1e-13 * scale
    assert (owner != owner0).sum() > 10      # nodes were covered and uncovered


def test_uniform_flow_at_the_wall_velocity_is_a_fixed_point():
    shape = (14, 14, 16)
    nz, ny, nx = shape
    U = np.array([0.04, -0.03, 0.02])
    parts = op.Particles([[7.4, 6.7, 6.9]], v=[U], radius=3.1, mass=0.0)
    owner = op.coverage(shape, parts.r, parts.radius)
    rho0 = (0.7, 0.3)
    fluid = owner < 0
    uu = np.broadcast_to(U[:, None, None, None], (3,) + shape)
    g = np.stack([ln.equilibrium(np.full(shape, rho0[k]), uu) for k in range(2)]) * fluid
    g1, owner1 = op.step(g, owner, None, parts, 0.8, 0.0, rho0)
    assert np.array_equal(owner1, owner)
    assert np.abs(g1 - g).max() <= 1e-15
    assert np.abs(parts.F).max() <= 1e-13 and np.abs(parts.T).max() <= 1e-12


@pytest.mark.parametrize("axis", [0, 2])
def test_rotating_sphere_torque_opposes_rotation(axis):
    shape = (20, 20, 20)
    w = np.zeros(3)
    w[axis] = 2e-3
    parts = op.Particles([[10.0, 10.0, 10.0]], w=[w], radius=4.2, mass=0.0)
    owner = op.coverage(shape, parts.r, parts.radius)
    rho0 = (0.5, 0.5)
    fluid = owner < 0
    g = np.stack([ln.equilibrium(np.full(shape, rho0[k]), np.zeros((3,) + shape)) for k in range(2)]) * fluid
    op.step(g, owner, None, parts, 1.0, 0.0, rho0)
    T = parts.T[0]
    assert np.abs(parts.F).max() <= 1e-14
    assert T[axis] < 0
    others = [a for a in range(3) if a != axis]
    assert np.abs(T[others]).max() <= 1e-12 * abs(T[axis])


def test_translating_particle_conserves_fluid_mass():
    shape = (16, 16, 16)
    rA, rB, u = fluid_fields(shape, 3, 0.8)
    parts = op.Particles([[8.0, 8.0, 8.0]], v=[[1e-4, -2e-4, 1e-4]], w=[[1e-3, 0.0, -1e-3]], radius=3.5,
                         mass=500.0)
    owner = op.coverage(shape, parts.r, parts.radius)
    g = op.init(rA, rB, u, None, owner)
    m0 = op.fluid_mass(g, owner, None)
    owner0 = owner.copy()
    for _ in range(4):
        g, owner = op.step(g, owner, None, parts, 0.9, 0.8, (0.5, 0.5))
    assert np.array_equal(owner, owner0)
    assert abs(op.fluid_mass(g, owner, None) - m0) <= 1e-13 * m0


def test_overlapping_particles_are_rejected():
    with pytest.raises(ValueError):
        op.coverage((10, 10, 10), [[3.0, 3.0, 3.0], [5.0, 3.0, 3.0]], 1.5)


def test_sphere_carried_by_a_uniform_flow_moves_with_it():
    """Free flight through re-meshing: a heavy sphere moving with the
    surrounding uniform flow feels no force, so it advances U per step
    (leap-frog), and the nodes it uncovers are refilled with the same
    uniform equilibrium."""
    shape = (12, 12, 16)
    U = np.array([0.3, -0.1, 0.05])
    parts = op.Particles([[6.3, 5.8, 6.1]], v=[U], radius=2.7, mass=1e12)
    owner = op.coverage(shape, parts.r, parts.radius)
    owner0 = owner.copy()
    rho0 = (0.6, 0.4)
    uu = np.broadcast_to(U[:, None, None, None], (3,) + shape)
    feq = np.stack([ln.equilibrium(np.full(shape, rho0[k]), uu) for k in range(2)])
    g = feq * (owner < 0)
    r0 = parts.r[0].copy()
    steps = 6
    for _ in range(steps):
        g, owner = op.step(g, owner, None, parts, 0.8, 0.0, rho0)
    assert (owner != owner0).sum() > 10
    assert np.abs(parts.r[0] - np.mod(r0 + steps * U, (16, 12, 12))).max() <= 1e-9
    assert np.abs((g - feq) * (owner < 0)).max() <= 1e-10


def test_contact_force_conserves_momentum_and_parts_spheres():
    """Two spheres sent at each other head-on through fluid at rest: the
    contact force is a central pair force (momentum is conserved with it),
    it turns them back before they share a node, and the mirror symmetry of
    the set-up keeps their velocities opposite."""
    shape = (16, 16, 32)
    rho0 = (0.5, 0.5)
    parts = op.Particles([[11.3, 8.0, 8.0], [20.7, 8.0, 8.0]], v=[[0.06, 0, 0], [-0.06, 0, 0]], radius=3.5,
                         mass=1000.0, contact=(0.5, 1.5))
    owner = op.coverage(shape, parts.r, parts.radius)
    fluid = owner < 0
    g = np.stack([ln.equilibrium(np.full(shape, rho0[k]), np.zeros((3,) + shape)) for k in range(2)]) * fluid
    p0 = op.fluid_momentum(g, owner, None) + parts.mass * parts.v.sum(axis=0)
    M = op.fluid_mass(g, owner, None)
    turned = touched = False
    for _ in range(120):
        g, owner = op.step(g, owner, None, parts, 1.0, 0.0, rho0)
        p1 = op.fluid_momentum(g, owner, None) + parts.mass * parts.v.sum(axis=0)
        assert np.abs(p1 - p0).max() <= 1e-14 * M
        assert np.abs(parts.v[0] + parts.v[1]).max() <= 1e-12
        turned = turned or parts.v[0][0] < 0
        touched = touched or np.abs(parts.Fc).max() > 0
    assert turned and touched


def test_coverage_matches_the_input_generators_masks():
    """The sphere coverage rule (periodic distance <= R) is the one the seeded
    colloid masks use, so a mask made from the same centres marks the same
    nodes (the benchmark takes its fluid fraction from such a mask)."""
    from paper_2112_08264_gb300 import inputs
    nx, ny, nz, R = 40, 36, 28, 5.5
    mask, centres = inputs.colloid_mask(nx, ny, nz, n_spheres=12, radius=R, seed=3)
    owner = op.coverage((nz, ny, nx), centres, R)
    assert np.array_equal(owner >= 0, mask == 1)


def test_lubrication_damps_the_approach_and_conserves_momentum():
    """Two spheres closing at a gap inside the lubrication range: the normal
    lubrication force is a pair force (total momentum conserved), it opposes
    the relative normal velocity, so the approach is slower than without it."""
    shape = (16, 16, 32)
    rho0 = (0.5, 0.5)

    def run(hc):
        parts = op.Particles([[12.6, 8.0, 8.0], [19.4, 8.0, 8.0]], v=[[0.004, 0, 0], [-0.004, 0, 0]], radius=3.2,
                             mass=2000.0, lubrication=hc)
        owner = op.coverage(shape, parts.r, parts.radius)
        g = np.stack([ln.equilibrium(np.full(shape, rho0[k]), np.zeros((3,) + shape)) for k in range(2)])
        g = g * (owner < 0)
        p0 = op.fluid_momentum(g, owner, None) + parts.mass * parts.v.sum(axis=0)
        M = op.fluid_mass(g, owner, None)
        work = 0.0
        for _ in range(8):
            g, owner = op.step(g, owner, None, parts, 1.0, 0.0, rho0)
            p1 = op.fluid_momentum(g, owner, None) + parts.mass * parts.v.sum(axis=0)
            assert np.abs(p1 - p0).max() <= 1e-14 * M
            work += (parts.Fc[0] * (parts.v[0] - parts.v[1])).sum()
        return parts.v[0][0] - parts.v[1][0], work, np.abs(parts.Fc).max()

    rel_free, _, f_free = run(0.0)
    rel_lub, work, f_lub = run(2.0 / 3.0)
    assert f_free == 0.0 and f_lub > 0.0
    assert work < 0.0                        # the force opposes the relative motion
    assert 0.0 < rel_lub < rel_free          # still closing, more slowly


@pytest.mark.parametrize("walls", [False, True])
def test_write_side_and_post_streaming_formulations_agree(walls):
    """The two particle oracles -- the write-side one (bounced populations kept
    in slots of the solid nodes) and the post-streaming one (the C oracle's
    representation, nothing stored on solid nodes, the moving-wall bounce
    applied while streaming) -- give the same states, sphere places,
    velocities, forces and torques, bit for bit, over steps that re-mesh both
    spheres (and with static walls)."""
    shape = (16, 14, 12)
    nz, ny, nx = shape
    rng = np.random.default_rng(2)
    rA = 0.5 + 0.05 * rng.uniform(-1, 1, shape)
    rB = 1.0 - rA
    u = 0.01 * rng.normal(size=(3,) + shape)
    mask = None
    if walls:
        mask = np.zeros(shape, np.uint8)
        mask[:, 0, :] = 1
        mask[:, ny - 1, :] = 1
    centres = [[5.2, 6.1, 7.3], [12.6, 8.2, 4.4]]
    kw = dict(v=[[0.21, -0.12, 0.07], [-0.15, 0.08, 0.18]], w=[[0, 0.01, -0.02], [0.015, 0, 0.01]],
              radius=2.8, mass=60.0, contact=(0.5, 1.0))
    a, b = op.Particles(centres, **kw), op.Particles(centres, **kw)
    owner_a = op.coverage(shape, a.r, a.radius)
    owner_b = owner_a.copy()
    fluid = (owner_a < 0) if mask is None else (owner_a < 0) & (mask == 0)
    rho0 = (rA[fluid].mean(), rB[fluid].mean())
    g = op.init(rA, rB, u, mask, owner_a)
    f = op.init_pull(rA, rB, u, mask, owner_b, b, rho0)
    moved = 0
    for _ in range(12):
        g, new_a = op.step(g, owner_a, mask, a, 0.9, 0.6, rho0)
        f, owner_b = op.step_pull(f, owner_b, mask, b, 0.9, 0.6, rho0)
        moved += int((new_a != owner_a).sum())
        owner_a = new_a
        assert np.array_equal(owner_a, owner_b)
        assert np.array_equal(op.pulled(g, owner_a, mask, a, rho0), f)
        for q in ("r", "v", "w", "F", "T", "Fc"):
            assert np.array_equal(getattr(a, q), getattr(b, q)), q
    assert moved > 50
