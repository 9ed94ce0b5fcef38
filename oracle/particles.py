"""Moving rigid spheres coupled to the two-component step, FP64 numpy.

TEST INFRASTRUCTURE (see the package docstring): only tests and the
benchmark's CPU legs use it; the library never imports it.

Model (Sec. 2): each particle p is a rigid sphere of radius R with centre
r_p, velocity v_p and angular velocity w_p; a node x is covered by p when its
periodic (minimum-image) distance to r_p is at most R. Only the exterior
holds fluid (the Jansen-Harting form the paper adopts): covered nodes carry
no populations. Per step, in this order:

1. Links and forces. For every fluid node x and direction i whose neighbour
   x + c_i is covered by p, the wall sits at the link midpoint
   r_b = x + c_i / 2 and moves with u_b = v_p + w_p x (r_b - r_p) (Eq. UPI);
   the population g_i(x) leaving x returns to x as population opp(i) reduced
   by 2 rho w_i (u_b . c_i) / c_s^2 (Eq. LADDFLBE), and the link passes the
   momentum it exchanges with the fluid to the particle (Eq. FORCEPP, summed
   over links in Eq. FORCEPARTEQ and Eq. TORQUEPARTEQ with the arm r_b - r_p).
2. The fluid step: streaming (pull) and the Shan-Chen BGK collision, with
   psi = 0 on every solid node.
3. Newton's equations (Eq. PARDYN) by leap-frog: v += (F + F_c) / m,
   r += v, w += T / I, with I = 2 m R^2 / 5 (a uniform sphere); m <= 0 marks
   a fixed particle (its force and torque are still computed). F_c is the
   repulsive contact force that keeps spheres apart (the paper names a
   Hertzian one): between two spheres whose centres are d < 2 R + delta
   apart, k (2 R + delta - d)^(3/2) along the line of centres, pushing them
   apart (k = 0: none). With a lubrication cutoff h_c > 0, two spheres whose
   gap h = d - 2R is below h_c also exchange the normal lubrication force
   -(3/2) pi mu R^2 (1/h - 1/h_c) ((v_i - v_j) . n) n (mu = (rho0^A + rho0^B)
   (tau - 1/2) / 3, n the unit vector from j to i, h clamped at 0.01 from
   below), from the velocities before the update.
4. Re-meshing: nodes the moved sphere no longer covers become fluid with the
   equilibrium populations of density rho0^k and the local wall velocity;
   nodes it newly covers lose their fluid. The particle takes up the
   momentum (and its moment) that the fluid gains or loses there, so the
   total momentum of fluid and particles is unchanged.

Readings where the paper is silent (listed with the design notes):
* rho in the bias of Eq. LADDFLBE is each component's base density rho0^k;
* Eq. FORCEPP subtracts the populations of fluid inside the particle (Ladd's
  form), but under the exterior-only form the paper adopts there is none:
  the link force here is the momentum the bounce exchanges with the
  exterior fluid, c_i sum_k (2 g_i^k(x) - 2 rho0^k w_i (u_b . c_i) / c_s^2);
* the re-meshing rule (item 4) is not given in the paper; it is chosen to
  conserve momentum exactly;
* the contact force's law and constants are not given; the Hertzian form
  above with stiffness k and range delta is the reading;
* the lubrication force is named with its range (2/3 of a lattice unit)
  but not given: the normal lubrication correction above is the reading.

Two formulations of the same step. ``step`` keeps the library's write-side
representation: g holds the post-collision populations at fluid nodes and,
at solid nodes, the slots the next pull reads (slot opp(i) of solid
y = x + c_i holds the bounced population of fluid x); ``pulled`` gives the
post-streaming populations it stands for. ``step_pull`` keeps the C oracle's
post-streaming representation (nothing stored on solid nodes) and applies the
moving-wall bounce-back while streaming. They are written apart and pinned
against each other; the GPU is checked against ``step_pull``. Arrays use
``lb_numpy``'s velocity order (``VEL``), shape (2, 19, nz, ny, nx).
"""
import numpy as np

from . import lb_numpy as ln

VEL = ln.VEL
W = ln.W
OPP = ln.OPP
CS2 = ln.CS2


def shift_from(a, c):
    """Field whose value at x is a(x + c) (periodic; the last three axes are
    z, y, x)."""
    return np.roll(a, shift=(-int(c[2]), -int(c[1]), -int(c[0])), axis=(-3, -2, -1))


def shift_to(a, c):
    """Field whose value at x + c is a(x)."""
    return np.roll(a, shift=(int(c[2]), int(c[1]), int(c[0])), axis=(-3, -2, -1))


def min_image(d, n):
    """Minimum-image displacement along one axis of period n."""
    return d - n * np.round(d / n)


def coverage(shape, r, radius):
    """Per-node owner: -1 = not covered, p = covered by particle p (distance
    to r_p at most radius, periodic). Overlapping particles are an error."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    owner = np.full(shape, -1, dtype=np.int64)
    for p, c in enumerate(np.asarray(r, dtype=np.float64).reshape(-1, 3)):
        dx = min_image(x - c[0], nx)
        dy = min_image(y - c[1], ny)
        dz = min_image(z - c[2], nz)
        inside = dx * dx + dy * dy + dz * dz <= radius * radius
        if np.any(owner[inside] >= 0):
            raise ValueError("particles overlap")
        owner[inside] = p
    return owner


class Particles:
    """Rigid spheres: positions r, velocities v, angular velocities w (all
    (P, 3) float64), a common radius and mass (mass <= 0: fixed)."""

    def __init__(self, r, v=None, w=None, radius=5.0, mass=1.0, contact=(0.0, 0.0), lubrication=0.0):
        self.r = np.array(r, dtype=np.float64).reshape(-1, 3)
        P = len(self.r)
        self.v = np.zeros((P, 3)) if v is None else np.array(v, dtype=np.float64).reshape(P, 3)
        self.w = np.zeros((P, 3)) if w is None else np.array(w, dtype=np.float64).reshape(P, 3)
        self.radius = float(radius)
        self.mass = float(mass)
        self.F = np.zeros((P, 3))
        self.T = np.zeros((P, 3))
        self.Fc = np.zeros((P, 3))
        self.contact = (float(contact[0]), float(contact[1]))
        self.lubrication = float(lubrication)

    @property
    def inertia(self):
        return 0.4 * self.mass * self.radius ** 2

    def copy(self):
        c = Particles(self.r, self.v, self.w, self.radius, self.mass, self.contact, self.lubrication)
        c.F, c.T, c.Fc = self.F.copy(), self.T.copy(), self.Fc.copy()
        return c


def _arm(shape, x, y, z, centre):
    nz, ny, nx = shape
    return np.stack([min_image(x - centre[0], nx), min_image(y - centre[1], ny), min_image(z - centre[2], nz)])


def init(rhoA, rhoB, u, mask, owner):
    """The state whose pull is the equilibrium f^eq(rho^k, u) at every fluid
    node (0 on solid nodes): g_i(y) = f_i(y + c_i) where y + c_i is fluid,
    g_i(y) = f_opp(i)(y) at a fluid y whose neighbour y + c_i is solid (the
    bounce at rest), 0 elsewhere."""
    solid = _solid(mask, owner)
    f = ln.init(rhoA, rhoB, u, solid.astype(np.uint8))
    fluid = ~solid
    g = np.zeros_like(f)
    for i, c in enumerate(VEL):
        dest_fluid = shift_from(fluid, c)          # y + c_i fluid
        g[:, i] = np.where(dest_fluid, shift_from(f[:, i], c), 0.0)
        g[:, i] += np.where(fluid & ~dest_fluid, f[:, OPP[i]], 0.0)
    return g


def _solid(mask, owner):
    s = owner >= 0
    if mask is not None:
        s = s | (np.asarray(mask) != 0)
    return s


def links_and_forces(g, owner, mask, parts, rho0):
    """Step 1: write every solid slot a fluid node pulls (moving-wall bounce
    at particle nodes, bounce at rest at static solid nodes) and return the
    force and torque of every particle (FP64 sums over its links)."""
    shape = g.shape[2:]
    nz, ny, nx = shape
    solid = _solid(mask, owner)
    fluid = ~solid
    static = np.zeros(shape, bool) if mask is None else (np.asarray(mask) != 0)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    P = len(parts.r)
    F = np.zeros((P, 3))
    T = np.zeros((P, 3))
    out = g.copy()
    for i, c in enumerate(VEL):
        if not c.any():
            continue
        o = OPP[i]
        nb_owner = shift_from(owner, c)             # owner of x + c_i
        nb_static = shift_from(static, c)
        # static solid neighbour: the slot takes g_i(x) unchanged
        at = fluid & nb_static
        for k in range(2):
            slot = np.where(at, g[k, i], 0.0)
            out[k, o] = np.where(shift_to(at, c), shift_to(slot, c), out[k, o])
        for p in range(P):
            at = fluid & (nb_owner == p)
            if not at.any():
                continue
            xs, ys, zs = x[at], y[at], z[at]
            arm = _arm(shape, xs + 0.5 * c[0], ys + 0.5 * c[1], zs + 0.5 * c[2], parts.r[p])
            ub = parts.v[p][:, None] + np.cross(parts.w[p], arm.T).T
            cu = (c[:, None] * ub).sum(axis=0) / CS2
            exch = np.zeros(len(xs))
            tz, ty, tx = (zs + c[2]) % nz, (ys + c[1]) % ny, (xs + c[0]) % nx
            for k in range(2):
                gi = g[k, i][at]
                bias = 2.0 * rho0[k] * W[i] * cu
                out[k, o, tz, ty, tx] = gi - bias
                exch += 2.0 * gi - bias
            dF = c[:, None] * exch[None, :]
            F[p] += dF.sum(axis=1)
            T[p] += np.cross(arm.T, dF.T).sum(axis=0)
    return out, F, T


def pulled(g, owner, mask, parts, rho0):
    """The post-streaming populations a state stands for: its solid slots
    written (item 1, forces discarded), then pulled; 0 on solid nodes."""
    f = post_streaming(links_and_forces(g, owner, mask, parts, rho0)[0])
    return f * ~_solid(mask, owner)


def post_streaming(g):
    """Pull every node: f_i(x) = g_i(x - c_i) (solid sources are slots)."""
    f = np.empty_like(g)
    for i, c in enumerate(VEL):
        f[:, i] = shift_to(g[:, i], c)
    return f


def collide(f, tau, G, gbody, solid):
    """Step 2's collision at fluid nodes (Shan-Chen velocity shift and BGK,
    psi = 0 on solid nodes); 0 on solid nodes."""
    m = solid.astype(np.uint8)
    f = f * (~solid)
    fluid = (~solid).astype(np.float64)
    rho, Fsc = ln.density_force(f, G, gbody, m)
    mom = np.einsum("kiabc,id->dabc", f, VEL.astype(np.float64))
    safe = lambda r: r + (1.0 - fluid)
    up = (mom / tau) / safe(rho[0] / tau + rho[1] / tau)
    out = np.empty_like(f)
    for k in range(2):
        ueq = up + tau * Fsc[k] / safe(rho[k])
        out[k] = (f[k] - (f[k] - ln.equilibrium(rho[k], ueq)) / tau) * fluid
    return out


def contact_forces(parts, box, mu=0.0):
    """Pair forces: the repulsion k (2 R + delta - d)^(3/2) along the line of
    centres for centre distances d < 2 R + delta, and the normal lubrication
    force for gaps below the cutoff (minimum image; mu the dynamic
    viscosity)."""
    k, delta = parts.contact
    hc = parts.lubrication
    P = len(parts.r)
    Fc = np.zeros((P, 3))
    if k == 0.0 and hc == 0.0:
        return Fc
    R = parts.radius
    reach = 2.0 * R + delta
    for i in range(P):
        for j in range(P):
            if i == j:
                continue
            d = np.array([min_image(parts.r[i][a] - parts.r[j][a], box[a]) for a in range(3)])
            dist = np.sqrt((d * d).sum())
            n = d / dist
            if k != 0.0 and dist < reach:
                Fc[i] += k * (reach - dist) ** 1.5 * n
            h = dist - 2.0 * R
            if hc > 0.0 and h < hc:
                h = max(h, 0.01)
                vn = ((parts.v[i] - parts.v[j]) * n).sum()
                Fc[i] -= 1.5 * np.pi * mu * R * R * (1.0 / h - 1.0 / hc) * vn * n
    return Fc


def advance(parts, box, mu=0.0):
    """Step 3: leap-frog with the force and torque of step 1 and the pair
    forces of the current places and velocities (box = (nx, ny, nz))."""
    parts.Fc = contact_forces(parts, box, mu)
    if parts.mass <= 0:
        return
    parts.v = parts.v + (parts.F + parts.Fc) / parts.mass
    parts.r = parts.r + parts.v
    parts.w = parts.w + parts.T / parts.inertia


def remesh(g, owner, mask, parts, rho0):
    """Step 4 for moved particles: uncovered nodes first (all particles),
    then newly covered ones; returns the new owner field. Each particle's
    velocity takes the momentum change of its own nodes after each pass."""
    shape = g.shape[2:]
    nz, ny, nx = shape
    for p in range(len(parts.r)):
        parts.r[p] = np.mod(parts.r[p], (nx, ny, nz))
    new = coverage(shape, parts.r, parts.radius)
    static = np.zeros(shape, bool) if mask is None else (np.asarray(mask) != 0)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    g = g.copy()
    fixed = parts.mass <= 0
    # uncovered: fluid at the wall velocity and rho0
    for p in range(len(parts.r)):
        at = (owner == p) & (new != p)
        if not at.any():
            continue
        arm = _arm(shape, x[at], y[at], z[at], parts.r[p])
        ub = parts.v[p][:, None] + np.cross(parts.w[p], arm.T).T
        dP = np.zeros(3)
        dL = np.zeros(3)
        for k in range(2):
            feq = ln.equilibrium(np.full(arm.shape[1], rho0[k]), ub)
            g[k][:, at] = feq
            dP -= rho0[k] * ub.sum(axis=1)
            dL -= rho0[k] * np.cross(arm.T, ub.T).sum(axis=0)
        if not fixed:
            parts.v[p] += dP / parts.mass
            parts.w[p] += dL / parts.inertia
    owner_mid = np.where(owner >= 0, np.where(new == owner, owner, -1), -1)
    # newly covered: the fluid there goes to the particle
    for p in range(len(parts.r)):
        at = (new == p) & (owner_mid != p)
        if not at.any():
            continue
        if np.any(static[at]) or np.any(owner_mid[at] >= 0):
            raise ValueError("a particle covers a solid node")
        arm = _arm(shape, x[at], y[at], z[at], parts.r[p])
        mom = np.einsum("kin,id->dn", g[:, :, at], VEL.astype(np.float64))
        g[:, :, at] = 0.0
        if not fixed:
            parts.v[p] += mom.sum(axis=1) / parts.mass
            parts.w[p] += np.cross(arm.T, mom.T).sum(axis=0) / parts.inertia
    return g, new


def step(g, owner, mask, parts, tau, G, rho0, gbody=None):
    """One step (items 1-4); returns (g, owner). parts is updated in place
    and holds the force and torque of this step."""
    g, parts.F, parts.T = links_and_forces(g, owner, mask, parts, rho0)
    solid = _solid(mask, owner)
    gnew = collide(post_streaming(g), tau, G, gbody, solid)
    nz, ny, nx = g.shape[2:]
    advance(parts, (nx, ny, nz), (rho0[0] + rho0[1]) * (tau - 0.5) / 3.0)
    gnew, owner = remesh(gnew, owner, mask, parts, rho0)
    return gnew, owner


# ---------------------------------------------------------------------------
# The same step in the post-streaming representation of the C oracle: the
# state is the pulled, pre-collision f at fluid nodes and nothing at solid
# nodes; the moving-wall bounce-back of Eq. LADDFLBE is applied while
# streaming (push form), where the exchanged momentum of Eq. FORCEPP is
# summed. Written apart from the write-side form above (which stores the
# bounced populations in slots of the solid nodes, as the library does) so
# that the two can pin each other.
#
# Order: a step's force comes from the streaming that made its state, with
# the sphere velocities of that moment; then collision, leap-frog with that
# force, re-meshing of the post-collision field, and the streaming that makes
# the next state and the next step's force. parts.F, parts.T after a step are
# the force and torque that step's leap-frog used.


def stream(g, owner, mask, parts, rho0):
    """Push the post-collision g of the fluid nodes along c_i: into the
    neighbour when it is fluid, back into population opp(i) of the same node
    when it is solid -- at rest for a static solid, reduced by
    2 rho0^k w_i (u_b . c_i) / c_s^2 for a node covered by a sphere moving with
    u_b = v + w x (r_b - r) at the link midpoint r_b. Returns (f, F, T), F and
    T the momentum and its moment each sphere takes from its links."""
    shape = g.shape[2:]
    nz, ny, nx = shape
    solid = _solid(mask, owner)
    fluid = ~solid
    static = np.zeros(shape, bool) if mask is None else (np.asarray(mask) != 0)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    P = len(parts.r)
    F = np.zeros((P, 3))
    T = np.zeros((P, 3))
    f = np.zeros_like(g)
    for i, c in enumerate(VEL):
        o = OPP[i]
        into_fluid = fluid & shift_from(fluid, c)          # x fluid, x + c_i fluid
        for k in range(2):
            f[k, i] += shift_to(np.where(into_fluid, g[k, i], 0.0), c)
        if not c.any():
            continue
        back = fluid & shift_from(static, c)               # x + c_i a static solid
        for k in range(2):
            f[k, o] += np.where(back, g[k, i], 0.0)
        nb_owner = shift_from(owner, c)
        for p in range(P):
            at = fluid & (nb_owner == p)
            if not at.any():
                continue
            arm = _arm(shape, x[at] + 0.5 * c[0], y[at] + 0.5 * c[1], z[at] + 0.5 * c[2], parts.r[p])
            ub = parts.v[p][:, None] + np.cross(parts.w[p], arm.T).T
            cu = (c[:, None] * ub).sum(axis=0) / CS2
            exch = np.zeros(arm.shape[1])
            for k in range(2):
                gi = g[k, i][at]
                bias = 2.0 * rho0[k] * W[i] * cu
                f[k, o][at] += gi - bias
                exch += 2.0 * gi - bias
            dF = c[:, None] * exch[None, :]
            F[p] += dF.sum(axis=1)
            T[p] += np.cross(arm.T, dF.T).sum(axis=0)
    return f, F, T


def unstream(f, solid):
    """The post-collision field whose streaming with bounce-back at rest gives
    f back: g_i(y) = f_i(y + c_i) where y + c_i is fluid, f_opp(i)(y) where it
    is solid; 0 on solid nodes."""
    fluid = ~solid
    g = np.zeros_like(f)
    for i, c in enumerate(VEL):
        ahead_fluid = shift_from(fluid, c)
        for k in range(2):
            g[k, i] = np.where(fluid & ahead_fluid, shift_from(f[k, i], c), 0.0)
            g[k, i] += np.where(fluid & ~ahead_fluid, f[k, OPP[i]], 0.0)
    return g


def init_pull(rhoA, rhoB, u, mask, owner, parts, rho0):
    """Initial post-streaming state: the equilibrium f^eq(rho^k, u) at fluid
    nodes, streamed once more from the field that reproduces it at rest, so
    that nodes next to a moving sphere see its wall (the first step's force
    is set in parts.F_next, parts.T_next)."""
    solid = _solid(mask, owner)
    feq = ln.init(rhoA, rhoB, u, solid.astype(np.uint8))
    f, parts.F_next, parts.T_next = stream(unstream(feq, solid), owner, mask, parts, rho0)
    return f


def step_pull(f, owner, mask, parts, tau, G, rho0, gbody=None):
    """One step in the post-streaming representation; returns (f, owner)."""
    parts.F, parts.T = parts.F_next, parts.T_next
    g = collide(f, tau, G, gbody, _solid(mask, owner))
    nz, ny, nx = f.shape[2:]
    advance(parts, (nx, ny, nz), (rho0[0] + rho0[1]) * (tau - 0.5) / 3.0)
    g, owner = remesh(g, owner, mask, parts, rho0)
    f, parts.F_next, parts.T_next = stream(g, owner, mask, parts, rho0)
    return f, owner


def fluid_momentum(g, owner, mask):
    """Momentum of the populations held at fluid nodes (post-collision)."""
    fluid = ~_solid(mask, owner)
    return np.einsum("kiabc,id->d", g * fluid, VEL.astype(np.float64))


def fluid_mass(g, owner, mask):
    fluid = ~_solid(mask, owner)
    return float((g * fluid).sum())
