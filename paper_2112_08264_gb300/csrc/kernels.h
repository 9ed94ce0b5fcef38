// kernels.h -- host-side launchers of the device kernels (internal to the
// library; the public interface is include/lb.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"
#include "reduce.cuh"

namespace lbgb {

// Launch plan of the asynchronous-copy fused kernel (lb_fused_async.cu).
struct AsyncPlan {
    int ncols;      // tiles along x (32 columns each)
    int R;          // tiles along y; tile cy covers [cy*ny/R, (cy+1)*ny/R)
    int tymax;      // tallest tile (rows)
    int zsplit;     // z-chunks per tile column
    int zchunk;     // planes per z-chunk
    int nst;        // copy stages in shared memory
    int threads;    // 32 * tymax
    int ns;         // copy slots per stage (own nodes + halo nodes)
    size_t smem;    // dynamic shared memory per block
    int box;        // 1: box copies (nx a multiple of the 16-byte chunk), 0: per-node copies
};

// One time step: src (post-collision state) -> dst.
// Bounce-back links of a static mask: for each velocity i, the fluid sites x
// whose neighbour x + c_i is solid, in segment [off[i], off[i + 1]) of
// `sites` (grouped by blocks of 256 consecutive sites, ascending within a
// warp). sites == nullptr: no list (the copy pass scans every site).
//
// Links that stay inside one tile of the box kernel (same 32-column strip,
// same row band, target plane inside the same z-chunk) are instead grouped
// by (tile, source plane) for that kernel's tiling: list (b, z) is
// tent[tstart[b nz + z], tstart[b nz + z + 1]), one LinkTiles entry per link.
// The box kernel copies them itself while both ends are still in L2; any
// other step kernel runs them as a separate pass. `sites` then holds only the
// remaining links. tent == nullptr: no tile lists (`sites` holds every link).
struct LinkList {
    const uint32_t* sites = nullptr;
    long long off[Q + 1] = {};
    LinkTiles tiles;
    TileMap map;              // the tiling the lists were built for
    long long tmost = 0;      // longest (tile, plane) list
    long long tcount = 0;     // links in the tile lists
};

struct StepLaunch {
    int prec;                 // 0 fp32, 1 fp16 deviation, 2 bf16 deviation
    int kernel;               // 0 fused (async copies), 1 two-pass, 2 fused (register double buffer)
    const void* src;
    void* dst;
    const uint32_t* flags;    // nullptr = no solid nodes
    float* rho;               // density scratch (two-pass), 2N floats
    float* mom_out;           // optional: per-node moments of the source state (mom_elems(N), fluid nodes)
    Geom g;
    Phys p;
    int zsplit;               // register fused kernel: z-chunks per tile column
    AsyncPlan plan;           // async fused kernel
    LinkList links;           // masked grids: the write-side bounce-back links
};

cudaError_t launch_step(const StepLaunch& L, cudaStream_t st);
// The two parts of launch_step: the step kernel(s), and the write-side
// bounce-back pass of a masked grid (nothing without a mask).
cudaError_t launch_step_fluid(const StepLaunch& L, cudaStream_t st);
cudaError_t launch_step_links(const StepLaunch& L, cudaStream_t st);

// Register fused kernel: launch geometry for a grid on a device with sm_count SMs.
void fused_geometry(int nx, int ny, int nz, int sm_count, int* tiles, int* zsplit, int* threads);

// Async fused kernel: plan for a grid, and its launcher (called by launch_step).
// model: 0 Shan-Chen, 1 colour gradient (the 16-bit tiling depends on it).
AsyncPlan plan_fused_async(int nx, int ny, int nz, int sm_count, int prec, bool masked, int model,
                           size_t smem_limit);
cudaError_t launch_fused_async(const StepLaunch& L, cudaStream_t st);

// Solid flags from a device mask (1 = solid).
cudaError_t launch_flags(const uint8_t* mask, uint32_t* flags, const Geom& g, cudaStream_t st);

// Build the link lists of a mask (flags); the host waits for the counts.
// Tile lists (map.R > 0): entries into tent (tcap entries), offsets into
// tstart (map.ncols * map.R * nz + 1 words), per-list counters in tscratch
// (as many words); skipped (L.tiles.tent left nullptr) when the in-tile
// links exceed tcap. The remaining links go into `sites` (capacity entries)
// with `cursor` (2Q words of scratch); L.sites stays nullptr when they do not
// fit (the pass then scans every site, in-tile links included: a second copy
// of a link writes the same value).
cudaError_t build_links(const uint32_t* flags, uint32_t* sites, size_t capacity, uint32_t* cursor, TileMap map,
                        uint16_t* tent, size_t tcap, uint32_t* tstart, uint32_t* tscratch, const Geom& g,
                        LinkList& L, cudaStream_t st);

// True when a step launched with L runs the tile lists inside its kernel
// (the box kernel of the tiling the lists were built for).
bool tiles_in_kernel(const StepLaunch& L);

// Write-side halfway bounce-back on a freshly written state g: for every fluid
// node x and direction i with x + c_i solid, copy g_i(x) into slot opp(i) of
// x + c_i. The next pull of population opp(i) at x, from x - c_opp(i) = x + c_i,
// then reads the bounced value without a mask test. Run after every masked step.
// With tile lists, `with_tiles` says whether this pass also copies them
// (false when the step kernel already did).
cudaError_t launch_reflect(int prec, void* g_state, const uint32_t* flags, const LinkList& links, bool with_tiles,
                           const Geom& g, cudaStream_t st);

// Moving spheres (lb_particles.cu). Arrays of 3n doubles on the device;
// owner[s] = p + 1 when sphere p covers site s, 0 otherwise; err collects
// bit 1 (spheres touching each other or the mask) and bit 2 (a sphere faster
// than one node per step).
struct Spheres {
    double *r = nullptr, *v = nullptr, *w = nullptr, *F = nullptr, *T = nullptr;
    double* Fc = nullptr;   // contact forces
    int* owner = nullptr;
    int* err = nullptr;
    // per sphere: centre at the last full re-meshing pass (3 doubles) and the
    // distance from there of the node nearest to its surface; a sphere that
    // has moved less than that changes no node
    double* ref = nullptr;
    float* margin = nullptr;
    // per sphere: how far the last leap-frog update moved its centre (|v|,
    // rounded up); the re-meshing's owners are the coverage at the centre
    // before that move
    float* step = nullptr;
    // per sphere: the centre in FP32 (x, y, z, 0), for the pair distance
    // screen of the contact forces (written where the centre changes)
    float4* rf = nullptr;
    int n = 0;
    double radius = 0.0, mass = 0.0, inertia = 0.0;
    double contact_k = 0.0, contact_range = 0.0;   // k (2R + range - d)^(3/2) for d < 2R + range
    double lub_cut = 0.0;   // lubrication below this gap (0: none)
    double mu = 0.0;        // dynamic viscosity for the lubrication force
    int half = 0;   // box half-width around a centre: ceil(radius) + 2
};
// Moving-wall bounce-back into the solid slots of `state` and, when
// `forces`, the spheres' force and torque of those links.
cudaError_t launch_sphere_links(int prec, void* state, const uint32_t* flags, const Spheres& S, bool forces,
                                const Geom& g, const Phys& p, cudaStream_t st);
// Leap-frog update, then re-meshing of `state` and the flags around every
// sphere (static solids from `mask`, may be nullptr).
cudaError_t launch_sphere_move(int prec, void* state, uint32_t* flags, const uint8_t* mask, const Spheres& S,
                               const Geom& g, const Phys& p, cudaStream_t st);
// Coverage of freshly placed spheres (owner zeroed first) and the flags of
// the whole grid from `mask` and the coverage.
cudaError_t launch_sphere_place(uint32_t* flags, const uint8_t* mask, const Spheres& S, const Geom& g,
                                cudaStream_t st);

// Internal state from a post-streaming population field:// Internal state from a post-streaming population field: either the
// equilibrium of (rhoA, rhoB, u) (f == nullptr) or the given f (float,
// [k][i][s]). Inverse of the pull: g_j(y) = f_j(y + c_j) if y + c_j is fluid,
// else f_opp(j)(y); solid slots are filled as launch_reflect fills them.
cudaError_t launch_unstream(int prec, void* dst, const uint32_t* flags, const float* f,
                            const float* rhoA, const float* rhoB, const float* u, const Geom& g,
                            const Phys& p, cudaStream_t st);

// Post-streaming populations (float, [k][i][s]; 0 on solid nodes).
cudaError_t launch_get_state(int prec, const void* src, const uint32_t* flags, float* f, const Geom& g,
                             const Phys& p, cudaStream_t st);

// Density deviations psi - rho0 (into rho, 2N) and moments rhoA, rhoB, u.
cudaError_t launch_densities(int prec, const void* src, const uint32_t* flags, float* rho, const Geom& g,
                             const Phys& p, cudaStream_t st);
cudaError_t launch_moments(int prec, const void* src, const uint32_t* flags, const float* rho,
                           float* rhoA, float* rhoB, float* u, const Geom& g, const Phys& p,
                           cudaStream_t st);

// FP64 conserved totals over the sites [s0, s1) (s1 < 0: to the end):
// partials[kRedBlocks][kRedVals] then out[kRedVals] = {mass A, mass B, Px,
// Py, Pz, non-finite count}.
cudaError_t launch_stats(int prec, const void* src, const uint32_t* flags, double* partials, double* out,
                         const Geom& g, const Phys& p, cudaStream_t st, long long s0 = 0, long long s1 = -1);

// Checks of lb_init inputs over fluid nodes: out = {sum rhoA, sum rhoB,
// fluid count, bad count, 0, 0}. Bad: not finite, or rho^k <= 0 (Shan-Chen
// divides by each rho^k), or, with allow_zero (colour gradient, which
// divides only by rho^A + rho^B), rho^k < 0 or rho^A + rho^B <= 0.
cudaError_t launch_check_init(const float* rhoA, const float* rhoB, const float* u, const uint32_t* flags,
                              double* partials, double* out, const Geom& g, bool allow_zero, cudaStream_t st);

// Message returned by lb_last_error() (host code only).
void record_error_text(const char* msg);

}  // namespace lbgb
