"""Moving rigid spheres on the GPU (``lb_particles_set`` / ``lb_step``)
against the FP64 particle oracle (``oracle.particles``, its post-streaming
formulation ``init_pull`` / ``step_pull``: the C oracle's representation, no
populations stored on solid nodes), through the C ABI.

Bars: fixed spheres at rest give, bit for bit, the state of the static mask
they cover (their slots carry no bias); moving spheres follow the oracle
step by step -- pulled states within a few FP32 ulps of the largest
population, positions, velocities, forces and torques within 1e-5 of their
scale -- through re-meshing; the total momentum of fluid and spheres is
conserved; the benchmark's 256^3 launch configuration reproduces a tiled
32^3 oracle run at every site and every sphere. Physics beyond the oracle: a
fixed sphere's drag in a forced periodic flow follows Hasimoto's cubic-array
law within 3 %, and a moving sphere feels the drag of a fixed one in the
Galilean-equivalent flow."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lb_numpy as ln  # noqa: E402
from oracle import particles as op  # noqa: E402
from paper_2112_08264_gb300 import Solver, build, inputs  # noqa: E402
from paper_2112_08264_gb300 import _lib  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def fields(shape, seed):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    rA = 0.5 + 0.05 * rng.uniform(-1, 1, (nz, ny, nx))
    u = 0.01 * rng.normal(size=(3, nz, ny, nx))
    return f32(rA), f32(1.0 - rA), f32(u)


def gpu_run(shape, spheres, steps, tau, G, rA, rB, u, prec="fp32", mask=None):
    nx, ny, nz = shape
    s = Solver(nx, ny, nz, tau, G, mask=mask, prec=prec, max_particles=max(1, len(spheres["r"])))
    s.set_particles(spheres["r"], spheres.get("v"), spheres.get("w"), spheres["radius"], spheres["mass"])
    s.init(dev(rA), dev(rB), dev(u))
    return s


def oracle_init(shape, spheres, rA, rB, u, mask=None):
    nx, ny, nz = shape
    parts = op.Particles(spheres["r"], spheres.get("v"), spheres.get("w"), spheres["radius"], spheres["mass"])
    owner = op.coverage((nz, ny, nx), parts.r, parts.radius)
    fluid = (owner < 0) if mask is None else (owner < 0) & (mask == 0)
    rho0 = (rA[fluid].mean(), rB[fluid].mean())
    f = op.init_pull(rA, rB, u, mask, owner, parts, rho0)
    return f, owner, parts, rho0


TWO = dict(r=[[9.3, 8.4, 7.7], [23.6, 17.2, 12.9]], v=[[0.21, -0.12, 0.07], [-0.15, 0.08, 0.18]],
           w=[[0.0, 0.01, -0.02], [0.015, 0.0, 0.01]], radius=3.2, mass=60.0)


def test_fixed_spheres_at_rest_equal_the_static_mask_bitwise():
    shape = (32, 24, 20)
    nx, ny, nz = shape
    sph = dict(r=[[9.3, 8.4, 7.7], [23.6, 17.2, 12.9]], radius=3.2, mass=0.0)
    rA, rB, u = fields(shape, 1)
    s = gpu_run(shape, sph, 0, 0.9, 0.8, rA, rB, u)
    mask = (op.coverage((nz, ny, nx), np.array(sph["r"]), sph["radius"]) >= 0).astype(np.uint8)
    m = Solver(nx, ny, nz, 0.9, 0.8, mask=mask)
    m.init(dev(rA), dev(rB), dev(u))
    for _ in range(3):
        s.step(4)
        m.step(4)
        assert torch.equal(s.get_state(), m.get_state())
    p = s.particles()
    assert np.array_equal(p["r"], np.array(sph["r"])) and np.abs(p["F"]).max() > 0


# per-quantity bars: FP32 storage; FP16 storage (forces sum hundreds of
# rounded populations with cancellation, so only positions and velocities
# are held close)
BARS = {"fp32": dict(r=1e-5, v=4e-6, w=4e-6, F=4e-6, T=4e-6, state=8e-7),
        "fp16": dict(r=1e-4, v=5e-2, w=None, F=None, T=None, state=2e-3)}


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_moving_spheres_follow_the_oracle(prec):
    bars = BARS[prec]
    shape = (32, 24, 20)
    nx, ny, nz = shape
    tau, G, steps = 0.9, 0.6, 8
    rA, rB, u = fields(shape, 2)
    s = gpu_run(shape, TWO, 0, tau, G, rA, rB, u, prec=prec)
    f, owner, parts, rho0 = oracle_init(shape, TWO, rA, rB, u)
    owner0 = owner.copy()
    for t in range(steps):
        s.step(1)
        f, owner = op.step_pull(f, owner, None, parts, tau, G, rho0)
        p = s.particles()
        for k, ref in (("r", parts.r), ("v", parts.v), ("w", parts.w), ("F", parts.F), ("T", parts.T)):
            if bars[k] is None:
                continue
            bar = bars[k] if k == "r" else bars[k] * max(np.abs(ref).max(), 1e-30)
            assert np.abs(p[k] - ref).max() <= bar, (t, k, p[k], ref)
    assert (owner != owner0).sum() > 20            # re-meshing happened
    got = s.get_state().cpu().numpy().astype(np.float64)
    want = ln.to_public(f)
    assert np.abs(got - want).max() <= bars["state"] * np.abs(want).max()


def test_total_momentum_is_conserved():
    """stats() reads the pulled state, in which the next step's bounce has
    already taken the next step's force F from the fluid: fluid momentum +
    F + sum m v is the conserved total."""
    shape = (32, 24, 20)
    rA, rB, u = fields(shape, 3)
    s = gpu_run(shape, TWO, 0, 0.9, 0.6, rA, rB, u)
    totals = []
    for _ in range(8):
        st = np.array(s.stats())
        v = s.particles()["v"]
        s.step(1)
        F = s.particles()["F"]
        totals.append(st[2:5] + F.sum(axis=0) + TWO["mass"] * v.sum(axis=0))
        M = st[0] + st[1]
    totals = np.array(totals)
    assert np.abs(totals - totals[0]).max() <= 1e-6 * M


def test_rejections():
    shape = (32, 24, 20)
    nx, ny, nz = shape
    rA, rB, u = fields(shape, 4)
    s = Solver(nx, ny, nz, 1.0, 0.5, max_particles=2)
    with pytest.raises(_lib.LbError):                       # overlapping
        s.set_particles([[8.0, 8.0, 8.0], [12.0, 8.0, 8.0]], radius=3.0, mass=1.0)
    with pytest.raises(_lib.LbError):                       # too many
        s.set_particles([[5.0, 5.0, 5.0], [15.0, 15.0, 10.0], [25.0, 5.0, 15.0]], radius=2.0, mass=1.0)
    with pytest.raises(_lib.LbError):                       # cube wider than the grid
        s.set_particles([[8.0, 8.0, 8.0]], radius=7.5, mass=1.0)
    mask = np.zeros((nz, ny, nx), np.uint8)
    mask[10, 12, 16] = 1
    sm = Solver(nx, ny, nz, 1.0, 0.5, mask=mask, max_particles=1)
    with pytest.raises(_lib.LbError):                       # covers a solid node of the mask
        sm.set_particles([[16.2, 12.1, 10.3]], radius=2.5, mass=1.0)
    s.set_particles([[8.0, 8.0, 8.0]], radius=3.0, mass=1.0)
    s.init(dev(rA), dev(rB), dev(u))
    with pytest.raises(_lib.LbError) as e:                  # after init
        s.set_particles([[8.0, 8.0, 8.0]], radius=3.0, mass=1.0)
    assert e.value.status == _lib.LB_ESTATE
    for bad in (dict(kernel="two_pass"), dict(ckpt_every=5, ckpt_steps_max=10)):
        with pytest.raises(Exception):
            Solver(nx, ny, nz, 1.0, 0.5, max_particles=1, **bad)
    with pytest.raises(Exception):                           # the box kernel needs nx % 4 == 0
        Solver(30, ny, nz, 1.0, 0.5, max_particles=1)


def test_full_size_256_tiled_moving_spheres():
    """256^3 in the benchmark's launch configuration: a 32^3 periodic state
    with one moving sphere, tiled 8 times per axis (512 spheres), evolves as
    the oracle's 32^3 run at every site, and every sphere as the oracle's."""
    n, p, steps, tau, G = 256, 32, 4, 1.0, 0.65
    rA, rB, u = fields((p, p, p), 5)
    one = dict(r=[[13.4, 15.7, 16.2]], v=[[0.23, -0.17, 0.11]], w=[[0.01, -0.02, 0.015]], radius=5.5, mass=700.0)
    reps = n // p
    offs = np.array([[i, j, k] for k in range(reps) for j in range(reps) for i in range(reps)], np.float64) * p
    r = np.array(one["r"]) + offs
    s = Solver(n, n, n, tau, G, max_particles=len(r))
    s.set_particles(r, np.repeat(one["v"], len(r), 0), np.repeat(one["w"], len(r), 0), one["radius"], one["mass"])
    big = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda").repeat(reps, reps, reps).contiguous()
    s.init(big(rA), big(rB), torch.stack([big(u[a]) for a in range(3)]).contiguous())
    s.step(steps)
    f, owner, parts, rho0 = oracle_init((p, p, p), one, rA, rB, u)
    for _ in range(steps):
        f, owner = op.step_pull(f, owner, None, parts, tau, G, rho0)
    got = s.get_state()
    want = ln.to_public(f)
    want_t = torch.tensor(want.astype(np.float32), device="cuda").repeat(1, 1, reps, reps, reps)
    assert float((got - want_t).abs().max()) <= 8e-7 * float(want_t.abs().max())
    q = s.particles()
    assert np.abs(q["r"] - np.mod(parts.r[0] + offs, n)).max() <= 1e-5
    assert np.abs(q["F"] - parts.F[0]).max() <= 4e-6 * np.abs(parts.F).max()


def test_contact_force_turns_spheres_back_as_the_oracle():
    """Two spheres sent at each other through fluid at rest, turned back by
    the contact force: positions and velocities follow the oracle's."""
    shape = (32, 16, 16)
    nx, ny, nz = shape
    rho0 = (0.5, 0.5)
    sph = dict(r=[[11.3, 8.0, 8.0], [20.7, 8.0, 8.0]], v=[[0.06, 0, 0], [-0.06, 0, 0]], radius=3.5, mass=1000.0)
    rA = np.full((nz, ny, nx), 0.5)
    rB = np.full((nz, ny, nx), 0.5)
    u = np.zeros((3, nz, ny, nx))
    s = Solver(nx, ny, nz, 1.0, 0.0, max_particles=2, rho0=rho0)
    s.set_particles(sph["r"], sph["v"], None, sph["radius"], sph["mass"], contact=(0.5, 1.5))
    s.init(dev(rA), dev(rB), dev(u))
    parts = op.Particles(sph["r"], sph["v"], None, sph["radius"], sph["mass"], contact=(0.5, 1.5))
    owner = op.coverage((nz, ny, nx), parts.r, parts.radius)
    f = op.init_pull(rA, rB, u, None, owner, parts, rho0)
    turned = False
    for _ in range(70):
        s.step(1)
        f, owner = op.step_pull(f, owner, None, parts, 1.0, 0.0, rho0)
        p = s.particles()
        assert np.abs(p["r"] - parts.r).max() <= 1e-5
        assert np.abs(p["v"] - parts.v).max() <= 1e-5 * 0.06       # of the initial speed
        turned = turned or parts.v[0][0] < 0
    assert turned and p["v"][0][0] < 0


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_moving_spheres_between_static_walls(prec):
    """Spheres and a static mask together: two solid planes (a channel in y)
    bounce back at rest through the mask's link lists, the spheres through
    their own links; the state and the spheres follow the oracle."""
    shape = (32, 28, 24)
    nx, ny, nz = shape
    mask = np.zeros((nz, ny, nx), np.uint8)
    mask[:, 0, :] = 1
    mask[:, ny - 1, :] = 1
    sph = dict(r=[[9.3, 10.4, 7.7], [23.6, 17.2, 15.9]], v=[[0.21, 0.05, 0.07], [-0.15, -0.04, 0.18]],
               w=[[0.0, 0.01, -0.02], [0.015, 0.0, 0.01]], radius=3.2, mass=60.0)
    rA, rB, u = fields(shape, 6)
    s = gpu_run(shape, sph, 0, 0.9, 0.6, rA, rB, u, prec=prec, mask=mask)
    f, owner, parts, rho0 = oracle_init(shape, sph, rA, rB, u, mask)
    for _ in range(6):
        s.step(1)
        f, owner = op.step_pull(f, owner, mask, parts, 0.9, 0.6, rho0)
    p = s.particles()
    bars = BARS[prec]
    assert np.abs(p["r"] - parts.r).max() <= bars["r"]
    assert np.abs(p["v"] - parts.v).max() <= bars["v"] * np.abs(parts.v).max()
    got = s.get_state().cpu().numpy().astype(np.float64)
    want = ln.to_public(f)
    assert np.abs(got - want).max() <= bars["state"] * np.abs(want).max()


def test_fixed_sphere_drag_follows_hasimoto():
    """Physics of the coupling: a fixed sphere in a periodic box of fluid
    driven by a body force. At steady state the sphere's link force balances
    the body force on the fluid, and the mean velocity follows the drag of a
    simple cubic array of spheres (Hasimoto's expansion, F = 6 pi mu a U / K
    with K = 1 - 1.7601 phi^(1/3) + phi - 1.5593 phi^2, a = R)."""
    n, R, g = 40, 5.0, 1e-6
    s = Solver(n, n, n, 1.0, 0.0, max_particles=1, body_force=(g, 0, 0), rho0=(0.5, 0.5))
    s.set_particles([[n / 2 + 0.3, n / 2 - 0.2, n / 2 + 0.1]], radius=R, mass=0.0)
    s.init(dev(np.full((n, n, n), 0.5)), dev(np.full((n, n, n), 0.5)))
    s.step(16000)
    rA, rB, u = (x.cpu().numpy() for x in s.moments())
    fluid = (rA + rB) > 0
    F = s.particles()["F"][0][0]
    assert abs(F / (1.0 * g * fluid.sum()) - 1.0) < 0.01          # force balance
    phi = 4.0 / 3.0 * np.pi * R ** 3 / n ** 3
    K = 1 - 1.7601 * phi ** (1 / 3) + phi - 1.5593 * phi ** 2
    U_pred = F * K / (6 * np.pi * (1.0 / 6.0) * R)                  # mu = rho nu, nu = 1/6 at tau = 1
    assert abs(u[0][fluid].mean() / U_pred - 1.0) < 0.03


def test_moving_sphere_drag_equals_fixed_sphere_in_uniform_flow():
    """Galilean check of the moving-wall bounce-back and re-meshing: a heavy
    sphere moving at U through fluid at rest feels the drag of a fixed
    sphere in a uniform flow at -U (within lattice Galilean errors)."""
    nx, ny, nz, U0, R = 64, 40, 40, 0.02, 5.0
    late = {}
    for mode in ("fixed", "moving"):
        s = Solver(nx, ny, nz, 1.0, 0.0, max_particles=1, rho0=(0.5, 0.5))
        u = np.zeros((3, nz, ny, nx))
        if mode == "fixed":
            s.set_particles([[20.3, 20.1, 19.8]], radius=R, mass=0.0)
            u[0] = -U0
        else:
            s.set_particles([[20.3, 20.1, 19.8]], v=[[U0, 0, 0]], radius=R, mass=1e12)
        s.init(dev(np.full((nz, ny, nx), 0.5)), dev(np.full((nz, ny, nx), 0.5)), dev(u))
        F = []
        for t in range(600):
            s.step(1)
            if t >= 300:
                F.append(s.particles()["F"][0][0])
        late[mode] = np.mean(F)
    assert late["fixed"] < 0 and late["moving"] < 0
    assert abs(late["moving"] / late["fixed"] - 1.0) < 0.03


def test_collision_with_the_mask_and_overspeed_are_reported():
    """Failure detection on the host: a sphere driven into a solid wall of
    the mask, or one moving faster than a node per step, leaves the run
    invalid, which lb_particles_get reports as LB_ESTATE (the arrays are
    still filled); no device fault is involved."""
    shape = (32, 24, 20)
    nx, ny, nz = shape
    rA, rB, u = fields(shape, 7)
    mask = np.zeros((nz, ny, nx), np.uint8)
    mask[:, :, 25:] = 1                                          # a wall at x >= 25
    s = Solver(nx, ny, nz, 1.0, 0.5, mask=mask, max_particles=1)
    # slow enough that every population stays positive (bias 0.017 < w rho0 = 0.028)
    s.set_particles([[20.0, 12.0, 10.0]], v=[[0.1, 0.0, 0.0]], radius=3.0, mass=1e9)
    s.init(dev(rA), dev(rB), dev(u))
    s.step(35)                                                   # reaches the wall after ~20 steps
    with pytest.raises(_lib.LbError) as e:
        s.particles()
    assert e.value.status == _lib.LB_ESTATE
    f = Solver(nx, ny, nz, 1.0, 0.5, max_particles=1)
    f.set_particles([[10.0, 12.0, 10.0]], v=[[1.5, 0.0, 0.0]], radius=3.0, mass=1e9)
    f.init(dev(rA), dev(rB), dev(u))
    f.step(1)
    with pytest.raises(_lib.LbError) as e:
        f.particles()
    assert e.value.status == _lib.LB_ESTATE


def test_lubrication_as_the_oracle():
    """Two spheres closing inside the lubrication range: positions and
    velocities follow the oracle's (the normal lubrication force from the
    velocities before each update)."""
    shape = (32, 16, 16)
    nx, ny, nz = shape
    rho0 = (0.5, 0.5)
    sph = dict(r=[[12.6, 8.0, 8.0], [19.4, 8.0, 8.0]], v=[[0.004, 0, 0], [-0.004, 0, 0]], radius=3.2, mass=2000.0)
    rA = np.full((nz, ny, nx), 0.5)
    rB = np.full((nz, ny, nx), 0.5)
    u = np.zeros((3, nz, ny, nx))
    s = Solver(nx, ny, nz, 1.0, 0.0, max_particles=2, rho0=rho0)
    s.set_particles(sph["r"], sph["v"], None, sph["radius"], sph["mass"], lubrication=2.0 / 3.0)
    s.init(dev(rA), dev(rB), dev(u))
    parts = op.Particles(sph["r"], sph["v"], None, sph["radius"], sph["mass"], lubrication=2.0 / 3.0)
    owner = op.coverage((nz, ny, nx), parts.r, parts.radius)
    f = op.init_pull(rA, rB, u, None, owner, parts, rho0)
    for _ in range(8):
        s.step(1)
        f, owner = op.step_pull(f, owner, None, parts, 1.0, 0.0, rho0)
        p = s.particles()
        assert np.abs(p["r"] - parts.r).max() <= 1e-6
        assert np.abs(p["v"] - parts.v).max() <= 1e-4 * 0.004
    assert np.abs(parts.Fc).max() > 0


def test_moving_spheres_are_deterministic():
    """Two runs from the same input give the same bits: state, places,
    velocities, forces and torques (the sphere kernels work their nodes in a
    fixed order and reduce in fixed trees), with spheres large enough that a
    sphere's links are gathered over several screening rounds."""
    n, R, steps = 64, 5.5, 20
    vol = 4.0 / 3.0 * np.pi * R ** 3
    _, centres = inputs.colloid_mask(n, n, n, n_spheres=24, radius=R, seed=77)
    rng = np.random.default_rng(78)
    sph = dict(r=centres, v=rng.uniform(-0.01, 0.01, (len(centres), 3)),
               w=rng.uniform(-0.005, 0.005, (len(centres), 3)), radius=R, mass=2.2 * vol)
    rA, rB, u = fields((n, n, n), 79)
    runs = []
    for _ in range(2):
        s = gpu_run((n, n, n), sph, 0, 0.9, 0.6, rA, rB, u)
        s.step(steps)
        runs.append((s.get_state().cpu(), s.particles()))
        s.close()
    (sa, pa), (sb, pb) = runs
    assert torch.equal(sa, sb)
    for k in ("r", "v", "w", "F", "T"):
        assert np.array_equal(pa[k], pb[k]), k
