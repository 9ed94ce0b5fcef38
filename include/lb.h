/*
 * lb.h -- C ABI of the GB300 two-component D3Q19 lattice-Boltzmann library.
 *
 * The library advances two immiscible fluid components A and B on an
 * nx*ny*nz D3Q19 lattice (Sec. 2 Method: 19 velocities, rest + 6 at distance
 * 1 + 12 at distance sqrt 2) with BGK relaxation (Eq. bgk), the second-order
 * equilibrium (Eq. LEQ), streaming along c_i (Eq. bgk, left-hand side),
 * periodic wrap and halfway bounce-back at solid links for walls at rest
 * (Eq. LADDFLBE with u_b = 0; interior solid nodes hold no fluid, Sec. 2).
 * Components interact through a Shan-Chen pseudopotential force with
 * psi = rho, which the paper does not give (its two-component model is the
 * colour-gradient one); the library uses the standard form of the LBM text
 * the paper cites (Krueger et al. 2017):
 *     F^A(x) = -G psi^A(x) sum_{i=1..18} w_i psi^B(x + c_i) c_i,
 * F^B likewise with A and B swapped, psi = 0 on solid nodes, the lattice
 * weights w_i = 1/18, 1/36 as force weights, plus an optional body force
 * rho^k g. The force enters through the original Shan-Chen velocity shift:
 * u' = sum_k sum_i c_i f_i^k / sum_k rho^k (one relaxation time), and
 * component k relaxes to f^eq(rho^k, u' + tau F^k / rho^k).
 *
 * Conventions shared by every entry point:
 *   - Site index s = x + nx*(y + ny*z): x fastest, as the paper's column-major
 *     layout with x contiguous (Sec. 3 Implementation, Sec. 4).
 *   - Velocity order (public): 0 rest; 1..6 = +x, -x, +y, -y, +z, -z;
 *     7..18 = (+1,+1,0), (-1,-1,0), (+1,-1,0), (-1,+1,0), (+1,0,+1),
 *     (-1,0,-1), (+1,0,-1), (-1,0,+1), (0,+1,+1), (0,-1,-1), (0,+1,-1),
 *     (0,-1,+1); the opposite of an odd i is i + 1.
 *   - Population arrays are [k][i][s], k = 0 (A), 1 (B): 2*19*N floats. The
 *     state exchanged through the ABI is the post-streaming, pre-collision f.
 *   - Field pointers whose name starts with d_ are DEVICE pointers on the
 *     current device, caller-owned, contiguous, N = nx*ny*nz elements in
 *     site order (velocities: SoA, 3*N, component a at a*N + s).
 *   - The library never allocates device memory: every buffer it needs is a
 *     slice of the caller's workspace (lb_workspace_bytes tells its size).
 *   - All device work runs on the stream given at lb_create (or lb_set_stream),
 *     in order. Calls documented as synchronous wait for that stream.
 *   - Errors are returned as lb_status values; nothing throws across the ABI.
 *     A CUDA error becomes LB_ECUDA and lb_last_error() gives its text.
 *   - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef LB_H
#define LB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_ctx lb_ctx;

typedef enum {
    LB_OK = 0,
    LB_EINVAL = 1,      /* invalid argument */
    LB_ENOMEM = 2,      /* caller workspace too small */
    LB_ECUDA = 3,       /* CUDA error (text: lb_last_error) */
    LB_ENONFINITE = 4,  /* a non-finite population was found */
    LB_ESTATE = 5,      /* call not valid in the context's state */
    LB_ETIMEOUT = 6     /* a bounded device wait gave up */
} lb_status;

/* Storage of the populations. All three compute in FP32. The stored value is
 * the deviation d_i^k = f_i^k - w_i rho0^k from the rest equilibrium at the
 * base densities rho0^k, rounded to nearest-even for the 16-bit forms. */
typedef enum { LB_FP32 = 0, LB_FP16_DEV = 1, LB_BF16_DEV = 2 } lb_precision;

/* Time-stepping kernel. FUSED: one pass per step (pull streaming, densities
 * of the tile and its halo on chip, force, collision, store) -- the paper's
 * fused approach (Sec. 5.1) -- fed by an asynchronous copy pipeline through
 * shared memory. TWO_PASS: a density pass then a stream + force + collide
 * pass -- the paper's plain approach. FUSED_REG: the fused step with a
 * register double buffer instead of the copy pipeline (same arithmetic, same
 * results bit for bit). */
typedef enum { LB_KERNEL_FUSED = 0, LB_KERNEL_TWO_PASS = 1, LB_KERNEL_FUSED_REG = 2 } lb_kernel;

/* Two-component model. SHAN_CHEN: BGK with the Shan-Chen pseudopotential
 * force and the velocity shift (tau and G of lb_create). COLOUR_GRADIENT:
 * the paper's colour-gradient model (Appendix, Eq. 1coll, 2coll, 3coll): BGK
 * at the mixture viscosity, the perturbation that builds the interfacial
 * tension sigma, and the recolouring with parameter beta; periodic grids only
 * (no mask, no body force, no recording for lb_backward); lb_create's tau
 * and G are not used (pass tau > 0.5). */
typedef enum { LB_MODEL_SHAN_CHEN = 0, LB_MODEL_COLOUR_GRADIENT = 1 } lb_model;

typedef struct {
    int prec;              /* lb_precision (default LB_FP32) */
    int kernel;            /* lb_kernel (default LB_KERNEL_FUSED) */
    double rho0_A, rho0_B; /* deviation base; <= 0 means: the fluid-site mean of
                              the densities given to lb_init */
    double body_force[3];  /* g, added as rho^k g to F^k (default 0) */
    int ckpt_every;        /* K > 0: lb_step records a checkpoint every K steps
                              for lb_backward; 0 = no recording (default) */
    int ckpt_steps_max;    /* longest recorded run, in steps (needed when K > 0) */
    int model;             /* lb_model (default LB_MODEL_SHAN_CHEN) */
    double cg_nu_A, cg_nu_B; /* colour gradient: kinematic viscosities of the pure
                              components, > 0 (omega = 2 / (6 nu_bar + 1) with
                              1/nu_bar = (rho^A/rho)/nu_A + (rho^B/rho)/nu_B) */
    double cg_sigma;       /* colour gradient: surface tension, >= 0 (A = 9 omega sigma / 4) */
    double cg_beta;        /* colour gradient: recolouring parameter, in [0, 1] */
    int max_particles;     /* > 0: room for that many moving spheres (lb_particles_set);
                              needs the Shan-Chen model, LB_KERNEL_FUSED, no recording */
    int slab_halo;         /* > 0: the grid is one rank's slab of a lattice cut into
                              z-slabs (Sec. 4, equal sub-domains exchanging their
                              borders each step), extended by slab_halo ghost planes
                              below and above that the caller fills from the
                              neighbouring ranks (2 are needed: see lb_step_fluid).
                              Every bounce-back link is then copied by lb_step_links,
                              none inside the step kernel. Shan-Chen model, no
                              spheres, no recording. 0 = a whole periodic lattice. */
} lb_options;

/* Fill *opt with the defaults above. */
void lb_default_options(lb_options* opt);

/* Bytes of device workspace lb_create needs for this grid and options
 * (two population buffers, density scratch, reduction scratch, the solid
 * flags and the bounce-back link lists (up to N links of each kind: crossing
 * a tile of the step kernel, and inside one) when a mask is used -- counted
 * always -- and, when opt->ckpt_every > 0, checkpoints plus the
 * adjoint's buffers). opt may be NULL (defaults). Returns 0 for invalid
 * sizes. Pure host function. */
size_t lb_workspace_bytes(int nx, int ny, int nz, const lb_options* opt);

/* Create a context over the caller's workspace.
 *   nx, ny, nz  >= 3 each, nx*ny*nz < 2^31.
 *   tau         > 0.5 (positive viscosity, Eq. viscosity), finite.
 *   G           finite Shan-Chen coupling (G > 0 repels A from B).
 *   mask        HOST pointer to N bytes, 1 = solid node, 0 = fluid; NULL =
 *               all fluid (periodic box). Copied; the caller keeps ownership.
 *   opt         NULL = defaults.
 *   d_workspace device pointer, 256-byte aligned, ws_bytes >= lb_workspace_bytes.
 *   stream      a cudaStream_t (NULL = the legacy default stream).
 * Errors: LB_EINVAL for bad sizes/parameters/alignment, LB_ENOMEM for a short
 * workspace, LB_ECUDA. Synchronous (the mask upload and the construction of
 * its link list -- the fluid sites next to a solid one, per velocity -- wait). */
lb_status lb_create(int nx, int ny, int nz, float tau, float G, const uint8_t* mask,
                    const lb_options* opt, void* d_workspace, size_t ws_bytes,
                    void* stream, lb_ctx** out);

/* Set the stream used by all later calls on this context. */
lb_status lb_set_stream(lb_ctx* ctx, void* stream);

/* Initial state f_i^k = f_i^eq(rho^k, u) (Eq. LEQ) at every fluid node, from
 * device fields d_rhoA, d_rhoB (N floats) and d_u (3N floats SoA, or NULL
 * for u = 0). Resets the step counter and any recording. LB_EINVAL if a
 * fluid node has rho^k <= 0 or a non-finite input (the force shift divides
 * by rho^k); with the colour-gradient model pure phases are allowed
 * (rho^k >= 0, rho^A + rho^B > 0). Synchronous. */
lb_status lb_init(lb_ctx* ctx, const float* d_rhoA, const float* d_rhoB, const float* d_u);

/* Advance n >= 1 time steps (Eq. bgk with the force shift, then streaming
 * with bounce-back). Asynchronous on the context stream. When recording
 * (ckpt_every > 0) LB_ESTATE if the run would exceed ckpt_steps_max. */
lb_status lb_step(lb_ctx* ctx, int n);

/* One time step split in two, for a lattice cut into z-slabs over ranks
 * (opt->slab_halo = 2; Sec. 4: equal sub-domains, border exchange every
 * step). A rank holds its planes plus two ghost planes on each side. With
 * the two border planes of each neighbour in its ghosts, the step computes
 * every owned plane exactly as the whole lattice would (the force at a plane
 * needs the densities of the planes next to it, which sum populations pulled
 * from one plane further); the ghost planes come out wrong and the exchange
 * replaces them. Per step:
 *   lb_step_fluid(ctx)     the step kernel, without the bounce-back pass;
 *   exchange               the caller copies planes [2, 4) of each rank into
 *                          the upper ghosts [nz - 2, nz) of the rank below and
 *                          planes [nz - 4, nz - 2) into the lower ghosts [0, 2)
 *                          of the rank above (lb_planes gives their memory);
 *   lb_step_links(ctx)     the write-side halfway bounce-back of every link
 *                          (Eq. LADDFLBE at rest): a link whose source is a
 *                          ghost node reads that node's exchanged value.
 * lb_step(ctx, 1) is the two calls without the exchange. Between the two
 * calls every other call on the context returns LB_ESTATE. After lb_init the
 * caller exchanges once and calls lb_step_links before the first step.
 * Every rank must give lb_init the same rho0_A, rho0_B (lb_options; e.g. the
 * mean over the whole lattice) so that all ranks store the same deviations.
 * Asynchronous on the context stream. */
lb_status lb_step_fluid(lb_ctx* ctx);
lb_status lb_step_links(lb_ctx* ctx);

/* Device memory of planes [z0, z0 + nplanes) of the current state, in the
 * library's internal storage (contiguous; valid until the next step): for
 * copying border planes between ranks whose contexts have the same nx, ny,
 * precision and rho0. *d_ptr is a DEVICE pointer into the workspace, *bytes
 * its length. LB_EINVAL unless nx*ny is a multiple of 64 (planes must start
 * on a storage block) and 0 <= z0, nplanes >= 1, z0 + nplanes <= nz. */
lb_status lb_planes(lb_ctx* ctx, int z0, int nplanes, void** d_ptr, size_t* bytes);

/* lb_stats over the fluid nodes of planes [z0, z0 + nplanes) only (a rank's
 * owned planes; the totals of a decomposed lattice are their sum over the
 * ranks). out5 is a HOST pointer. Synchronous. */
lb_status lb_stats_planes(lb_ctx* ctx, int z0, int nplanes, double out5[5]);

/* Moments of the current state into device fields: rho^A, rho^B (N floats
 * each, 0 at solid nodes) and, when d_u != NULL, the mixture velocity
 * u = (sum_k sum_i c_i f_i^k + (F^A + F^B)/2) / (rho^A + rho^B) (3N floats
 * SoA, 0 at solid nodes). Any output pointer may be NULL. Asynchronous. */
lb_status lb_moments(lb_ctx* ctx, float* d_rhoA, float* d_rhoB, float* d_u);

/* Conserved totals over fluid nodes, accumulated in FP64: out5 = {sum rho^A,
 * sum rho^B, sum_k sum_i c_i f_i^k (x, y, z)}. out5 is a HOST pointer.
 * LB_ENONFINITE if any population is not finite. Synchronous. */
lb_status lb_stats(lb_ctx* ctx, double out5[5]);

/* Copy the current state (post-streaming f, [k][i][s], 2*19*N floats, 0 at
 * solid nodes) to / from device memory. Asynchronous. lb_set_state does not
 * change the step counter or the recording. */
lb_status lb_get_state(lb_ctx* ctx, float* d_dst);
lb_status lb_set_state(lb_ctx* ctx, const float* d_src);

/* Steps taken since lb_init. */
long long lb_steps_done(const lb_ctx* ctx);

/* Reverse-mode gradient of a loss of the final densities of a recorded run
 * (lb_init, then lb_step calls with ckpt_every = K > 0).
 *   d_dL_drhoA, d_dL_drhoB  device fields (N floats) dL/drho^k(final); either
 *                           may be NULL (= 0).
 *   d_grad_rhoA0, d_grad_rhoB0  device outputs (N floats, may be NULL):
 *                           dL/drho^k of the fields given to lb_init (u = 0
 *                           treated as a constant).
 *   grad_G                  HOST pointer to one double (may be NULL): dL/dG.
 * Recomputes each K-step segment from its checkpoint, then runs the adjoint
 * step backwards through it. LB_ESTATE without a recorded run. Synchronous.
 * The context's state is restored to the final state afterwards. */
lb_status lb_backward(lb_ctx* ctx, const float* d_dL_drhoA, const float* d_dL_drhoB,
                      float* d_grad_rhoA0, float* d_grad_rhoB0, double* grad_G);

/* Launch geometry the fused step uses (for measurement): number of kernel
 * launches per lb_step(1), and the tile/grid shape chosen at lb_create. */
lb_status lb_launch_info(const lb_ctx* ctx, int* launches_per_step, int* grid_blocks,
                         int* block_threads, int* z_split);

/* Moving rigid spheres (Sec. 2; the particles of Eq. PARDYN), all with one
 * radius and mass. A node is covered by a sphere when its periodic distance
 * to the centre is at most the radius; covered nodes hold no fluid. Each
 * lb_step then runs, per step: the moving-wall halfway bounce-back at every
 * link from a fluid node x to a covered node x + c_i (Eq. LADDFLBE with the
 * wall velocity u_b = v + w x (r_b - r) at the link midpoint r_b, Eq. UPI,
 * and rho = rho0^k of lb_init), whose exchanged momentum sums in FP64 into
 * the sphere's force and torque (Eq. FORCEPP, FORCEPARTEQ, TORQUEPARTEQ);
 * the fluid step; the leap-frog update v += F/m, r += v, w += T/I with
 * I = 2 m R^2 / 5 (Eq. PARDYN); and re-meshing: nodes a sphere leaves become
 * fluid at rho0^k and the local wall velocity, nodes it reaches give their
 * fluid's momentum to it (total momentum is conserved).
 *   n            number of spheres, 0 <= n <= opt->max_particles.
 *   r, v, w      HOST arrays of 3n doubles (x, y, z per sphere): centres
 *                (any real coordinates, wrapped into the box), velocities
 *                and angular velocities (NULL = 0).
 *   radius       > 0; 2 (ceil(radius) + 3) + 1 <= min(nx, ny, nz).
 *   mass         > 0, or <= 0 for spheres held fixed (forces still computed).
 * Call after lb_create and before lb_init (LB_ESTATE otherwise). LB_EINVAL
 * for bad values, spheres closer than 2 radius (periodic; checked on the host
 * with a cell list) or covering a solid node of the mask. Synchronous. The
 * contact force (lb_particles_contact) visits every pair of spheres each
 * step: meant for up to about 10^4 spheres. */
lb_status lb_particles_set(lb_ctx* ctx, int n, const double* r, const double* v, const double* w, double radius,
                           double mass);

/* Contact force between spheres (the paper's spheres repel on contact with a
 * Hertzian force; its constants are not given): two spheres whose centres
 * are d < 2 radius + range apart (periodic) are pushed apart along the line
 * of centres by stiffness (2 radius + range - d)^(3/2) each, added to the
 * force of the leap-frog update. stiffness = 0 (the default) turns it off.
 * Any time after lb_create; LB_EINVAL for negative or non-finite values,
 * LB_ESTATE without room for spheres. Host function. */
lb_status lb_particles_contact(lb_ctx* ctx, double stiffness, double range);

/* Lubrication between spheres (the paper adds one for particles closer than
 * 2/3 of a lattice unit; its form is not given): two spheres whose gap
 * h = d - 2 radius is below cutoff exchange the normal lubrication force
 * -(3/2) pi mu radius^2 (1/h - 1/cutoff) ((v_i - v_j) . n) n, n the unit
 * vector between the centres, mu = (rho0^A + rho0^B) (tau - 1/2) / 3, h
 * clamped at 0.01, from the velocities before the leap-frog update; added to
 * the contact force. cutoff = 0 (the default) turns it off. Any time after
 * lb_create; LB_EINVAL for a negative or non-finite cutoff, LB_ESTATE without
 * room for spheres. Host function. */
lb_status lb_particles_lubrication(lb_ctx* ctx, double cutoff);

/* The spheres after the last step, into HOST arrays of 3n doubles (any may
 * be NULL): r, v, w as above, and F, T = the force and torque of the last
 * step's links. LB_ESTATE (arrays still filled) when a step met spheres that
 * touch each other or the mask, or a sphere faster than one node per step:
 * the run is no longer valid. Synchronous. */
lb_status lb_particles_get(lb_ctx* ctx, double* r, double* v, double* w, double* F, double* T);

/* Bounce-back links of the mask (pairs of a fluid node x and a direction i
 * with x + c_i solid, Eq. LADDFLBE), as lb_create arranged them: *listed =
 * links in the per-velocity list of the bounce-back pass (-1: too many, the
 * pass scans every site; 0 without a mask); *in_tile = links grouped by tile
 * of the fused step kernel (target in the same tile and z-chunk as the
 * source); *in_kernel = 1 when lb_step copies those inside the step kernel,
 * 0 when it runs them as a pass of their own. Any pointer may be NULL. */
lb_status lb_link_info(const lb_ctx* ctx, long long* listed, long long* in_tile, int* in_kernel);

/* Allocation-free moments of a caller's population field. The paper has no
 * counterpart; this entry point exists for callers that may not allocate
 * device memory at all (no cudaMalloc, no allocator of any library) and so
 * cannot provide lb_create's workspace: for example code whose device memory
 * belongs to another framework's pool, or a plugin that must not allocate
 * after start-up. It computes, like lb_moments, rho^A, rho^B and the mixture
 * velocity u = (sum_k sum_i c_i f_i^k + (F^A + F^B)/2) / (rho^A + rho^B)
 * (0 at solid nodes), from
 *   d_f     DEVICE post-streaming populations [k][i][s], 2*19*N floats (the
 *           layout lb_get_state writes);
 *   d_mask  DEVICE solid mask, N bytes, 1 = solid, or NULL (all fluid);
 *   G, body_force (HOST, 3 doubles, or NULL = 0) as in lb_create/lb_options;
 * into DEVICE outputs d_rhoA, d_rhoB (N floats) and d_u (3N floats SoA), any
 * of which may be NULL. The velocity always includes the Shan-Chen shift: for
 * a colour-gradient state (whose velocity is sum_k sum_i c_i f_i^k / rho)
 * pass G = 0 and body_force = NULL. d_mask must mark every node that holds no
 * fluid (static solids and nodes covered by moving spheres); a node treated as
 * fluid whose populations are all zero gets u = 0. The populations arrive as
 * absolute FP32 values (about w_i rho each), so the moments carry their
 * rounding: about 1e-8 absolute on rho^k and on u near rho = 1, where
 * lb_moments, which sums the stored deviations from w_i rho0, resolves
 * smaller differences. It allocates nothing and calls no allocator: the
 * neighbour-density scratch it needs is a static device array of 2^20 nodes
 * (8 MiB, held on every GPU that loads the library until the process exits).
 * N = nx*ny*nz above 2^20 is rejected with LB_EINVAL and a message in
 * lb_last_error(). The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress): make that first call before any stream
 * capture. All calls share the array, so calls that overlap on the GPU race;
 * serialise them. Asynchronous on `stream` (a cudaStream_t, NULL = legacy). */
lb_status lb_moments_noalloc(int nx, int ny, int nz, float G, const double* body_force, const float* d_f,
                             const uint8_t* d_mask, float* d_rhoA, float* d_rhoB, float* d_u, void* stream);

/* Destroy the context (does not free the caller's workspace). NULL is a no-op. */
void lb_destroy(lb_ctx* ctx);

/* Static text for a status; text of the last CUDA error seen by the calling
 * thread, or of the last rejection lb_moments_noalloc explained ("" if none). */
const char* lb_status_str(lb_status s);
const char* lb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LB_H */
