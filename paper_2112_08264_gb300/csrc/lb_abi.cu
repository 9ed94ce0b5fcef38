// lb_abi.cu -- the C ABI declared in include/lb.h.
//
// The library allocates no device memory: lb_create carves the caller's
// workspace into the two population buffers of the one-step two-grid scheme
// (Sec. 3), the solid mask and flags, density scratch, reduction scratch and,
// when recording for the adjoint, the checkpoints and adjoint buffers.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "adjoint.h"
#include "kernels.h"
#include "lb.h"

using namespace lbgb;

namespace {

thread_local char g_last_error[256] = "";

void set_error(const char* what, cudaError_t e) {
    std::snprintf(g_last_error, sizeof g_last_error, "%s: %s", what, cudaGetErrorString(e));
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

namespace lbgb {
// Message for lb_last_error() from code outside this file.
void record_error_text(const char* msg) { std::snprintf(g_last_error, sizeof g_last_error, "%s", msg); }
}  // namespace lbgb

namespace {

size_t store_bytes(int prec) { return prec == LB_FP32 ? 4 : 2; }

struct Layout {
    size_t pop[2], mask, flags, links, tent, tstart, cursor, rho, red_part, red_out, owner, spheres, rf;
    size_t ckpt, ckpt_slots, seg, adj;
    size_t state_bytes;
    size_t total;
};

bool valid_dims(int nx, int ny, int nz) {
    if (nx < 3 || ny < 3 || nz < 3) return false;
    const long long N = (long long)nx * ny * nz;
    return N < (1LL << 31);
}

bool valid_options(const lb_options& o) {
    if (o.prec < LB_FP32 || o.prec > LB_BF16_DEV) return false;
    if (o.kernel < LB_KERNEL_FUSED || o.kernel > LB_KERNEL_FUSED_REG) return false;
    if (!std::isfinite(o.rho0_A) || !std::isfinite(o.rho0_B)) return false;
    for (double g : o.body_force)
        if (!std::isfinite(g)) return false;
    if (o.ckpt_every < 0 || o.ckpt_steps_max < 0) return false;
    if (o.max_particles < 0) return false;
    if (o.max_particles > 0 &&
        (o.model != LB_MODEL_SHAN_CHEN || o.kernel != LB_KERNEL_FUSED || o.ckpt_every != 0))
        return false;
    if (o.ckpt_every > 0 && o.ckpt_steps_max < 1) return false;
    if (o.slab_halo < 0) return false;
    if (o.slab_halo > 0 && (o.model != LB_MODEL_SHAN_CHEN || o.max_particles > 0 || o.ckpt_every != 0))
        return false;
    if (o.model != LB_MODEL_SHAN_CHEN && o.model != LB_MODEL_COLOUR_GRADIENT) return false;
    if (o.model == LB_MODEL_COLOUR_GRADIENT) {
        if (!(std::isfinite(o.cg_nu_A) && o.cg_nu_A > 0.0 && std::isfinite(o.cg_nu_B) && o.cg_nu_B > 0.0))
            return false;
        if (!(std::isfinite(o.cg_sigma) && o.cg_sigma >= 0.0)) return false;
        if (!(std::isfinite(o.cg_beta) && o.cg_beta >= 0.0 && o.cg_beta <= 1.0)) return false;
        for (double g : o.body_force)
            if (g != 0.0) return false;
        if (o.ckpt_every != 0 || o.kernel == LB_KERNEL_FUSED_REG) return false;
    }
    return true;
}

Layout make_layout(int nx, int ny, int nz, const lb_options& o) {
    Layout L{};
    const size_t N = (size_t)nx * ny * nz;
    L.state_bytes = align256(state_elems((long long)N) * store_bytes(o.prec));
    size_t off = 0;
    L.pop[0] = off; off += L.state_bytes;
    L.pop[1] = off; off += L.state_bytes;
    L.mask = off; off += align256(N);
    L.flags = off; off += align256(N * 4);
    L.links = off; off += align256(N * 4);   // bounce-back link list (masked grids), up to N links
    L.tent = off; off += align256(N * 2);    // in-tile links grouped by (tile, plane), up to N
    // list offsets: at most one tile per 32-column strip and row, per plane
    L.tstart = off; off += align256((((size_t)nx + 31) / 32 * ny * nz + 1) * 4);
    L.cursor = off; off += align256(2 * Q * 4);
    L.rho = off; off += align256(2 * N * 4);
    L.red_part = off; off += align256((size_t)kRedBlocks * kRedVals * 8);
    L.red_out = off; off += align256(kRedVals * 8);
    if (o.max_particles > 0) {
        L.owner = off; off += align256(N * 4);   // sphere covering each site
        // r, v, w, F, T, F_c, ref (3 doubles each per sphere), the error word, and per sphere a
        // margin and the last step's displacement; then the FP32 centres
        L.spheres = off; off += align256((size_t)o.max_particles * 21 * 8 + 8 + (size_t)o.max_particles * 8);
        L.rf = off; off += align256((size_t)o.max_particles * 16);
    }
    if (o.ckpt_every > 0) {
        L.ckpt_slots = (size_t)(o.ckpt_steps_max / o.ckpt_every) + 1;
        L.ckpt = off; off += L.ckpt_slots * L.state_bytes;
        L.seg = off; off += (size_t)o.ckpt_every * L.state_bytes;   // states of one segment
        L.adj = off; off += adjoint_workspace_bytes(nx, ny, nz, o.ckpt_every);
    }
    L.total = off;
    return L;
}

}  // namespace

struct lb_ctx {
    Geom g;
    Phys p;
    lb_options opt;
    float tau, G;
    cudaStream_t stream;
    char* ws;
    Layout L;
    void* pop[2];
    int cur;
    bool has_mask;
    uint8_t* mask_dev;
    uint32_t* flags;
    float* rho;
    double* red_part;
    double* red_out;
    bool initialized;
    long long steps;
    int sm_count, tiles, zsplit, threads;
    AsyncPlan plan;
    AsyncPlan adjplan;
    LinkList links;     // write-side bounce-back links of the mask
    bool particles;     // room for moving spheres (max_particles > 0)
    Spheres sph;        // the spheres (device arrays in the workspace)
    // recording for the adjoint
    bool recording;       // lb_init was called with ckpt_every > 0 and the run is intact
    double rho0_d[2];
    bool links_pending;   // lb_step_fluid ran; lb_step_links completes the step
};

namespace {

Phys make_phys(float tau, float G, const lb_options& o) {
    Phys p{};
    p.tau = tau;
    p.omega = 1.0f / tau;
    p.G = G;
    for (int a = 0; a < 3; ++a) p.g[a] = (float)o.body_force[a];
    p.rho0[0] = p.rho0[1] = 1.0f;
    p.model = o.model;
    if (o.model == LB_MODEL_COLOUR_GRADIENT) {
        p.cg_inu[0] = (float)(1.0 / o.cg_nu_A);
        p.cg_inu[1] = (float)(1.0 / o.cg_nu_B);
        p.cg_sigma = (float)o.cg_sigma;
        p.cg_beta = (float)o.cg_beta;
    }
    return p;
}

lb_status cuda_status(const char* what, cudaError_t e) {
    if (e == cudaSuccess) return LB_OK;
    set_error(what, e);
    return LB_ECUDA;
}

// solid flags, when any node can be solid (a mask or spheres)
const uint32_t* flags_of(const lb_ctx* c) { return c->has_mask || c->particles ? c->flags : nullptr; }

// With spheres, the state readers first write the spheres' slots (no
// forces) and then pull every slot as stored.
cudaError_t reader_phys(lb_ctx* c, Phys& p) {
    p = c->p;
    if (!c->particles) return cudaSuccess;
    p.slots = 1;
    return launch_sphere_links(c->opt.prec, c->pop[c->cur], c->flags, c->sph, false, c->g, c->p, c->stream);
}

lb_status run_reduction(lb_ctx* c, double out[kRedVals], bool stats, const float* rA = nullptr,
                        const float* rB = nullptr, const float* u = nullptr) {
    Phys rp;
    cudaError_t e = stats ? reader_phys(c, rp) : cudaSuccess;
    if (e == cudaSuccess)
        e = stats ? launch_stats(c->opt.prec, c->pop[c->cur], flags_of(c), c->red_part, c->red_out, c->g, rp,
                                 c->stream)
                  : launch_check_init(rA, rB, u, flags_of(c), c->red_part,
                                              c->red_out, c->g, c->opt.model == LB_MODEL_COLOUR_GRADIENT,
                                              c->stream);
    if (e != cudaSuccess) return cuda_status("reduction launch", e);
    e = cudaMemcpyAsync(out, c->red_out, kRedVals * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_status("reduction copy", e);
    return cuda_status("reduction sync", cudaStreamSynchronize(c->stream));
}

}  // namespace

// ---------------------------------------------------------------------------

extern "C" {

void lb_default_options(lb_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->prec = LB_FP32;
    o->kernel = LB_KERNEL_FUSED;
}

size_t lb_workspace_bytes(int nx, int ny, int nz, const lb_options* opt) {
    lb_options o;
    lb_default_options(&o);
    if (opt) o = *opt;
    if (!valid_dims(nx, ny, nz) || !valid_options(o)) return 0;
    return make_layout(nx, ny, nz, o).total;
}

lb_status lb_create(int nx, int ny, int nz, float tau, float G, const uint8_t* mask, const lb_options* opt,
                    void* d_workspace, size_t ws_bytes, void* stream, lb_ctx** out) {
    if (!out) return LB_EINVAL;
    *out = nullptr;
    lb_options o;
    lb_default_options(&o);
    if (opt) o = *opt;
    if (!valid_dims(nx, ny, nz) || !valid_options(o)) return LB_EINVAL;
    if (!std::isfinite(tau) || !(tau > 0.5f) || !std::isfinite(G)) return LB_EINVAL;
    if (o.model == LB_MODEL_COLOUR_GRADIENT && mask) return LB_EINVAL;   // periodic grids only
    if (!d_workspace || ((uintptr_t)d_workspace & 255u)) return LB_EINVAL;
    const Layout L = make_layout(nx, ny, nz, o);
    if (ws_bytes < L.total) return LB_ENOMEM;

    int dev = 0, sms = 0, smem_optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return cuda_status("device query", e);

    lb_ctx* c = new (std::nothrow) lb_ctx();
    if (!c) return LB_EINVAL;
    c->g.nx = nx; c->g.ny = ny; c->g.nz = nz;
    c->g.plane = nx * ny;
    c->g.N = (long long)nx * ny * nz;
    c->opt = o;
    c->tau = tau;
    c->G = G;
    c->p = make_phys(tau, G, o);
    c->stream = static_cast<cudaStream_t>(stream);
    c->ws = static_cast<char*>(d_workspace);
    c->L = L;
    c->pop[0] = c->ws + L.pop[0];
    c->pop[1] = c->ws + L.pop[1];
    c->cur = 0;
    c->mask_dev = reinterpret_cast<uint8_t*>(c->ws + L.mask);
    c->flags = reinterpret_cast<uint32_t*>(c->ws + L.flags);
    c->rho = reinterpret_cast<float*>(c->ws + L.rho);
    c->red_part = reinterpret_cast<double*>(c->ws + L.red_part);
    c->red_out = reinterpret_cast<double*>(c->ws + L.red_out);
    c->has_mask = mask != nullptr;
    c->particles = o.max_particles > 0;
    c->sm_count = sms;
    fused_geometry(nx, ny, nz, sms, &c->tiles, &c->zsplit, &c->threads);
    // spheres make solid nodes too: the masked kernel (flag boxes in shared memory) steps them
    c->plan = plan_fused_async(nx, ny, nz, sms, o.prec, mask != nullptr || o.max_particles > 0, o.model,
                               (size_t)smem_optin);
    if ((o.kernel == LB_KERNEL_FUSED && c->plan.nst < 2) || (c->particles && !c->plan.box)) {
        // no tile fits in shared memory, or spheres on a grid the box kernel cannot step
        delete c;
        return LB_EINVAL;
    }
    c->adjplan = AsyncPlan{};
    if (o.ckpt_every > 0)
        c->adjplan = plan_adjoint_box(nx, ny, nz, sms, mask != nullptr, (size_t)smem_optin);

    if (mask) {
        e = cudaMemcpyAsync(c->mask_dev, mask, (size_t)c->g.N, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = launch_flags(c->mask_dev, c->flags, c->g, c->stream);
        // tile lists for the box kernel's tiling (counters in the density scratch)
        TileMap map;   // a slab's links all go to the pass after the exchange (no tile lists)
        if (c->plan.box && c->plan.R > 0 && o.slab_halo == 0) {
            map.ncols = c->plan.ncols;
            map.R = c->plan.R;
            map.zchunk = c->plan.zchunk;
        }
        if (e == cudaSuccess)
            e = build_links(c->flags, reinterpret_cast<uint32_t*>(c->ws + L.links), (size_t)c->g.N,
                            reinterpret_cast<uint32_t*>(c->ws + L.cursor), map,
                            reinterpret_cast<uint16_t*>(c->ws + L.tent), (size_t)c->g.N,
                            reinterpret_cast<uint32_t*>(c->ws + L.tstart), reinterpret_cast<uint32_t*>(c->rho), c->g,
                            c->links, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            delete c;
            return cuda_status("mask upload", e);
        }
    }
    if (c->particles) {
        Spheres& S = c->sph;
        double* a = reinterpret_cast<double*>(c->ws + L.spheres);
        const size_t P3 = (size_t)o.max_particles * 3;
        S.r = a;
        S.v = a + P3;
        S.w = a + 2 * P3;
        S.F = a + 3 * P3;
        S.T = a + 4 * P3;
        S.Fc = a + 5 * P3;
        S.ref = a + 6 * P3;
        S.err = reinterpret_cast<int*>(a + 7 * P3);
        S.margin = reinterpret_cast<float*>(S.err + 2);   // after the 8-byte error slot
        S.step = S.margin + o.max_particles;
        S.rf = reinterpret_cast<float4*>(c->ws + L.rf);
        S.owner = reinterpret_cast<int*>(c->ws + L.owner);
        S.n = 0;
        if (!mask) c->links.sites = reinterpret_cast<const uint32_t*>(c->ws + L.links);   // no static links
        e = cudaMemsetAsync(S.err, 0, sizeof(int), c->stream);
        if (e == cudaSuccess) e = launch_sphere_place(c->flags, mask ? c->mask_dev : nullptr, S, c->g, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            delete c;
            return cuda_status("sphere setup", e);
        }
    }
    *out = c;
    return LB_OK;
}

lb_status lb_set_stream(lb_ctx* c, void* stream) {
    if (!c) return LB_EINVAL;
    c->stream = static_cast<cudaStream_t>(stream);
    return LB_OK;
}

lb_status lb_init(lb_ctx* c, const float* rA, const float* rB, const float* u) {
    if (!c || !rA || !rB) return LB_EINVAL;
    double red[kRedVals];
    lb_status s = run_reduction(c, red, false, rA, rB, u);
    if (s != LB_OK) return s;
    if (red[3] > 0.0) return LB_EINVAL;
    const double n = red[2] > 0.0 ? red[2] : 1.0;
    c->rho0_d[0] = c->opt.rho0_A > 0.0 ? c->opt.rho0_A : (red[2] > 0.0 ? red[0] / n : 1.0);
    c->rho0_d[1] = c->opt.rho0_B > 0.0 ? c->opt.rho0_B : (red[2] > 0.0 ? red[1] / n : 1.0);
    c->p.rho0[0] = (float)c->rho0_d[0];
    c->p.rho0[1] = (float)c->rho0_d[1];
    c->cur = 0;
    cudaError_t e = launch_unstream(c->opt.prec, c->pop[0], flags_of(c), nullptr, rA, rB,
                                    u, c->g, c->p, c->stream);
    if (e == cudaSuccess && c->opt.ckpt_every > 0)
        e = cudaMemcpyAsync(c->ws + c->L.ckpt, c->pop[0], c->L.state_bytes, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_status("init", e);
    c->initialized = true;
    c->links_pending = false;
    c->steps = 0;
    c->recording = c->opt.ckpt_every > 0 && u == nullptr;
    return LB_OK;
}

namespace {
StepLaunch step_launch(const lb_ctx* c) {
    StepLaunch S;
    S.prec = c->opt.prec;
    S.kernel = c->opt.kernel;
    S.flags = flags_of(c);
    S.rho = c->rho;
    S.mom_out = nullptr;
    S.g = c->g;
    S.p = c->p;
    S.zsplit = c->zsplit;
    S.plan = c->plan;
    S.links = c->links;
    return S;
}

// launches of the bounce-back passes after a masked step kernel
int reflect_launches(const lb_ctx* c) {
    if (!c->has_mask) return 0;
    const LinkList& L = c->links;
    if (!L.sites) return 1;   // the pass scans every site
    long long most = 0;
    for (int i = 1; i < Q; ++i) most = std::max(most, L.off[i + 1] - L.off[i]);
    const bool tile_pass = L.tiles.ent && L.tmost > 0 && !tiles_in_kernel(step_launch(c));
    return (most > 0 ? 1 : 0) + (tile_pass ? 1 : 0);
}
}  // namespace

lb_status lb_step(lb_ctx* c, int n) {
    if (!c || n < 1) return LB_EINVAL;
    if (!c->initialized) return LB_ESTATE;
    if (c->links_pending) return LB_ESTATE;
    const int K = c->opt.ckpt_every;
    if (K > 0 && c->recording && c->steps + n > c->opt.ckpt_steps_max) return LB_ESTATE;
    StepLaunch S = step_launch(c);
    for (int t = 0; t < n; ++t) {
        S.src = c->pop[c->cur];
        S.dst = c->pop[1 - c->cur];
        cudaError_t e = cudaSuccess;
        if (c->particles)   // the spheres' links: slots of src, forces and torques
            e = launch_sphere_links(c->opt.prec, c->pop[c->cur], c->flags, c->sph, true, c->g, c->p, c->stream);
        if (e == cudaSuccess) e = launch_step(S, c->stream);
        if (e == cudaSuccess && c->particles)   // leap-frog and re-meshing of dst
            e = launch_sphere_move(c->opt.prec, c->pop[1 - c->cur], c->flags, c->has_mask ? c->mask_dev : nullptr,
                                   c->sph, c->g, c->p, c->stream);
        if (e != cudaSuccess) return cuda_status("step", e);
        c->cur ^= 1;
        c->steps += 1;
        if (K > 0 && c->recording && c->steps % K == 0) {
            const size_t slot = (size_t)(c->steps / K);
            e = cudaMemcpyAsync(c->ws + c->L.ckpt + slot * c->L.state_bytes, c->pop[c->cur], c->L.state_bytes,
                                cudaMemcpyDeviceToDevice, c->stream);
            if (e != cudaSuccess) return cuda_status("checkpoint", e);
        }
    }
    return LB_OK;
}

lb_status lb_step_fluid(lb_ctx* c) {
    if (!c) return LB_EINVAL;
    if (!c->initialized || c->links_pending || c->particles || c->opt.ckpt_every > 0) return LB_ESTATE;
    StepLaunch S = step_launch(c);
    S.src = c->pop[c->cur];
    S.dst = c->pop[1 - c->cur];
    const cudaError_t e = launch_step_fluid(S, c->stream);
    if (e != cudaSuccess) return cuda_status("step", e);
    c->cur ^= 1;
    c->steps += 1;
    c->links_pending = c->has_mask;
    return LB_OK;
}

lb_status lb_step_links(lb_ctx* c) {
    if (!c) return LB_EINVAL;
    if (!c->initialized) return LB_ESTATE;
    c->links_pending = false;
    if (!c->has_mask) return LB_OK;
    StepLaunch S = step_launch(c);
    S.dst = c->pop[c->cur];
    return cuda_status("links", launch_step_links(S, c->stream));
}

lb_status lb_planes(lb_ctx* c, int z0, int nplanes, void** d_ptr, size_t* bytes) {
    if (!c || !d_ptr || !bytes) return LB_EINVAL;
    if (c->g.plane % kBlk != 0 || z0 < 0 || nplanes < 1 || (long long)z0 + nplanes > c->g.nz) return LB_EINVAL;
    const size_t plane_bytes = (size_t)(c->g.plane / kBlk) * (2 * Q * kBlk) * store_bytes(c->opt.prec);
    *d_ptr = static_cast<char*>(c->pop[c->cur]) + (size_t)z0 * plane_bytes;
    *bytes = (size_t)nplanes * plane_bytes;
    return LB_OK;
}

lb_status lb_stats_planes(lb_ctx* c, int z0, int nplanes, double out5[5]) {
    if (!c || !out5 || z0 < 0 || nplanes < 1 || (long long)z0 + nplanes > c->g.nz) return LB_EINVAL;
    if (!c->initialized || c->links_pending) return LB_ESTATE;
    Phys rp;
    cudaError_t e = reader_phys(c, rp);
    if (e == cudaSuccess)
        e = launch_stats(c->opt.prec, c->pop[c->cur], flags_of(c), c->red_part, c->red_out, c->g, rp, c->stream,
                         (long long)z0 * c->g.plane, ((long long)z0 + nplanes) * c->g.plane);
    if (e != cudaSuccess) return cuda_status("reduction launch", e);
    double red[kRedVals];
    e = cudaMemcpyAsync(red, c->red_out, kRedVals * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_status("reduction", e);
    for (int q = 0; q < 5; ++q) out5[q] = red[q];
    return red[5] > 0.0 ? LB_ENONFINITE : LB_OK;
}

lb_status lb_moments(lb_ctx* c, float* rA, float* rB, float* u) {
    if (!c) return LB_EINVAL;
    if (!c->initialized) return LB_ESTATE;
    if (c->links_pending) return LB_ESTATE;
    const uint32_t* fl = flags_of(c);
    Phys rp;
    cudaError_t e = reader_phys(c, rp);
    if (e == cudaSuccess && u) e = launch_densities(c->opt.prec, c->pop[c->cur], fl, c->rho, c->g, rp, c->stream);
    if (e == cudaSuccess)
        e = launch_moments(c->opt.prec, c->pop[c->cur], fl, c->rho, rA, rB, u, c->g, rp, c->stream);
    return cuda_status("moments", e);
}

lb_status lb_stats(lb_ctx* c, double out5[5]) {
    if (!c || !out5) return LB_EINVAL;
    if (!c->initialized) return LB_ESTATE;
    if (c->links_pending) return LB_ESTATE;
    double red[kRedVals];
    lb_status s = run_reduction(c, red, true);
    if (s != LB_OK) return s;
    for (int q = 0; q < 5; ++q) out5[q] = red[q];
    return red[5] > 0.0 ? LB_ENONFINITE : LB_OK;
}

lb_status lb_get_state(lb_ctx* c, float* dst) {
    if (!c || !dst) return LB_EINVAL;
    if (!c->initialized) return LB_ESTATE;
    if (c->links_pending) return LB_ESTATE;
    Phys rp;
    cudaError_t e = reader_phys(c, rp);
    if (e == cudaSuccess) e = launch_get_state(c->opt.prec, c->pop[c->cur], flags_of(c), dst, c->g, rp, c->stream);
    return cuda_status("get_state", e);
}

lb_status lb_set_state(lb_ctx* c, const float* src) {
    if (!c || !src) return LB_EINVAL;
    if (!c->initialized) return LB_ESTATE;
    if (c->links_pending) return LB_ESTATE;
    c->recording = false;   // the recorded trajectory no longer leads to this state
    return cuda_status("set_state", launch_unstream(c->opt.prec, c->pop[c->cur], flags_of(c),
                                                    src, nullptr, nullptr, nullptr, c->g, c->p, c->stream));
}

long long lb_steps_done(const lb_ctx* c) { return c ? c->steps : -1; }

lb_status lb_backward(lb_ctx* c, const float* dLA, const float* dLB, float* gA, float* gB, double* gG) {
    if (!c) return LB_EINVAL;
    if (!c->initialized || !c->recording || c->opt.ckpt_every <= 0 || c->steps < 1) return LB_ESTATE;
    AdjointRun R;
    R.prec = c->opt.prec;
    R.flags = c->has_mask ? c->flags : nullptr;
    R.g = c->g;
    R.p = c->p;
    R.K = c->opt.ckpt_every;
    R.steps = c->steps;
    R.state_bytes = c->L.state_bytes;
    R.ckpt = c->ws + c->L.ckpt;
    R.seg = c->ws + c->L.seg;
    R.adj = c->ws + c->L.adj;
    R.scratch = c->pop[1 - c->cur];
    R.rho = c->rho;
    R.red_part = c->red_part;
    R.red_out = c->red_out;
    R.zsplit = c->zsplit;
    R.plan = c->plan;
    R.adjplan = c->adjplan;
    R.links = c->links;
    R.kernel = c->opt.kernel;
    double gG_host = 0.0;
    cudaError_t e = run_adjoint(R, dLA, dLB, gA, gB, &gG_host, c->stream);
    if (e != cudaSuccess) return cuda_status("backward", e);
    if (gG) *gG = gG_host;
    return LB_OK;
}

lb_status lb_launch_info(const lb_ctx* c, int* launches, int* blocks, int* threads, int* zsplit) {
    if (!c) return LB_EINVAL;
    const int k = c->opt.kernel;
    // a masked step adds the write-side bounce-back passes (launch_reflect)
    // spheres: their links, and when they move the update, two re-meshing passes and the flags
    const int sph = !c->particles || c->sph.n == 0
                        ? 0
                        : (c->sph.mass > 0.0 ? 4 + (c->sph.contact_k != 0.0 || c->sph.lub_cut > 0.0 ? 1 : 0) : 1);
    if (launches) *launches = (k == LB_KERNEL_TWO_PASS ? 2 : 1) + reflect_launches(c) + sph;
    if (blocks)
        *blocks = k == LB_KERNEL_FUSED ? c->plan.ncols * c->plan.R * c->plan.zsplit
                : k == LB_KERNEL_FUSED_REG ? c->tiles * c->zsplit : (int)((c->g.N + 255) / 256);
    if (threads) *threads = k == LB_KERNEL_FUSED ? c->plan.threads : k == LB_KERNEL_FUSED_REG ? c->threads : 256;
    if (zsplit) *zsplit = k == LB_KERNEL_FUSED ? c->plan.zsplit : c->zsplit;
    return LB_OK;
}

lb_status lb_particles_set(lb_ctx* c, int n, const double* r, const double* v, const double* w, double radius,
                           double mass) {
    if (!c) return LB_EINVAL;
    if (!c->particles || n < 0 || n > c->opt.max_particles || (n > 0 && !r)) return LB_EINVAL;
    if (c->initialized) return LB_ESTATE;
    if (!std::isfinite(radius) || !(radius > 0.0) || !std::isfinite(mass)) return LB_EINVAL;
    const int half = (int)std::ceil(radius) + 2;
    if (2 * (half + 1) + 1 > std::min(c->g.nx, std::min(c->g.ny, c->g.nz))) return LB_EINVAL;
    const int dims[3] = {c->g.nx, c->g.ny, c->g.nz};
    std::vector<double> h(18 * (size_t)n, 0.0);   // r, v, w, F, T, F_c
    for (int q = 0; q < n; ++q)
        for (int a = 0; a < 3; ++a) {
            const double x = r[3 * q + a];
            const double vv = v ? v[3 * q + a] : 0.0, ww = w ? w[3 * q + a] : 0.0;
            if (!std::isfinite(x) || !std::isfinite(vv) || !std::isfinite(ww)) return LB_EINVAL;
            const double m = std::fmod(x, (double)dims[a]);
            h[3 * q + a] = m < 0.0 ? m + dims[a] : m;
            h[3 * (size_t)n + 3 * q + a] = vv;
            h[6 * (size_t)n + 3 * q + a] = ww;
        }
    // spheres closer than two radii (periodic) would share nodes: checked over
    // cells at least two radii wide (at most about 4n of them), each sphere
    // against the spheres of the up to 27 distinct cells around its own
    if (n > 1) {
        int nc[3];
        long long cells = 1;
        for (int a = 0; a < 3; ++a) {
            nc[a] = std::max(1, (int)std::floor(dims[a] / (2.0 * radius)));
            cells *= nc[a];
        }
        while (cells > 4LL * n + 64) {   // coarser cells: fewer of them, more pairs each
            const int a = nc[0] >= nc[1] && nc[0] >= nc[2] ? 0 : (nc[1] >= nc[2] ? 1 : 2);
            cells = cells / nc[a] * ((nc[a] + 1) / 2);
            nc[a] = (nc[a] + 1) / 2;
        }
        auto cell_of = [&](int q, int (&ci)[3]) {
            for (int a = 0; a < 3; ++a) ci[a] = std::min(nc[a] - 1, (int)(h[3 * q + a] * nc[a] / dims[a]));
        };
        std::vector<int> key(n), order(n);
        for (int q = 0; q < n; ++q) {
            int ci[3];
            cell_of(q, ci);
            key[q] = ci[0] + nc[0] * (ci[1] + nc[1] * ci[2]);
            order[q] = q;
        }
        std::sort(order.begin(), order.end(), [&](int a, int b) { return key[a] < key[b]; });
        std::vector<int> start((size_t)cells + 1, 0);
        for (int q = 0; q < n; ++q) ++start[(size_t)key[q] + 1];
        for (long long k = 0; k < cells; ++k) start[(size_t)k + 1] += start[(size_t)k];
        for (int p = 0; p < n; ++p) {
            int ci[3];
            cell_of(p, ci);
            int near[27], m = 0;
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int k = (ci[0] + dx + nc[0]) % nc[0] +
                                      nc[0] * ((ci[1] + dy + nc[1]) % nc[1] + nc[1] * ((ci[2] + dz + nc[2]) % nc[2]));
                        if (std::find(near, near + m, k) == near + m) near[m++] = k;
                    }
            for (int j = 0; j < m; ++j)
                for (int t = start[(size_t)near[j]]; t < start[(size_t)near[j] + 1]; ++t) {
                    const int q = order[t];
                    if (q <= p) continue;
                    double d2 = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        double d = h[3 * p + a] - h[3 * q + a];
                        d -= dims[a] * std::nearbyint(d / dims[a]);
                        d2 += d * d;
                    }
                    if (d2 <= 4.0 * radius * radius) return LB_EINVAL;
                }
        }
    }
    Spheres& S = c->sph;
    const size_t P3 = (size_t)c->opt.max_particles * 3;
    cudaError_t e = cudaSuccess;
    if (n > 0) {
        const double* src[6] = {h.data(), h.data() + 3 * (size_t)n, h.data() + 6 * (size_t)n,
                                h.data() + 9 * (size_t)n, h.data() + 12 * (size_t)n, h.data() + 15 * (size_t)n};
        double* dst[6] = {S.r, S.v, S.w, S.F, S.T, S.Fc};
        for (int k = 0; k < 6 && e == cudaSuccess; ++k)
            e = cudaMemcpyAsync(dst[k], src[k], 3 * (size_t)n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    }
    (void)P3;
    S.n = n;
    S.radius = radius;
    S.mass = mass;
    S.inertia = 0.4 * mass * (radius * radius);
    S.half = half;
    int err = 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(S.err, 0, sizeof(int), c->stream);
    if (e == cudaSuccess && n > 0) e = cudaMemsetAsync(S.step, 0, (size_t)n * sizeof(float), c->stream);
    if (e == cudaSuccess) e = launch_sphere_place(c->flags, c->has_mask ? c->mask_dev : nullptr, S, c->g, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, S.err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_status("particles_set", e);
    if (err) {   // a sphere covers a solid node of the mask: no spheres
        S.n = 0;
        e = launch_sphere_place(c->flags, c->has_mask ? c->mask_dev : nullptr, S, c->g, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        return e == cudaSuccess ? LB_EINVAL : cuda_status("particles_set", e);
    }
    return LB_OK;
}

lb_status lb_particles_contact(lb_ctx* c, double stiffness, double range) {
    if (!c) return LB_EINVAL;
    if (!c->particles) return LB_ESTATE;
    if (!std::isfinite(stiffness) || stiffness < 0.0 || !std::isfinite(range) || range < 0.0) return LB_EINVAL;
    c->sph.contact_k = stiffness;
    c->sph.contact_range = range;
    return LB_OK;
}

lb_status lb_particles_lubrication(lb_ctx* c, double cutoff) {
    if (!c) return LB_EINVAL;
    if (!c->particles) return LB_ESTATE;
    if (!std::isfinite(cutoff) || cutoff < 0.0) return LB_EINVAL;
    c->sph.lub_cut = cutoff;
    return LB_OK;
}

lb_status lb_particles_get(lb_ctx* c, double* r, double* v, double* w, double* F, double* T) {
    if (!c) return LB_EINVAL;
    if (!c->particles) return LB_ESTATE;
    const Spheres& S = c->sph;
    const size_t bytes = 3 * (size_t)S.n * sizeof(double);
    double* out[5] = {r, v, w, F, T};
    const double* src[5] = {S.r, S.v, S.w, S.F, S.T};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 5 && e == cudaSuccess; ++k)
        if (out[k] && bytes) e = cudaMemcpyAsync(out[k], src[k], bytes, cudaMemcpyDeviceToHost, c->stream);
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, S.err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_status("particles_get", e);
    return err ? LB_ESTATE : LB_OK;
}

lb_status lb_link_info(const lb_ctx* c, long long* listed, long long* in_tile, int* in_kernel) {
    if (!c) return LB_EINVAL;
    const LinkList& L = c->links;
    if (listed) *listed = !c->has_mask ? 0 : (L.sites ? L.off[Q] : -1);
    if (in_tile) *in_tile = L.tiles.ent ? L.tcount : 0;
    if (in_kernel) *in_kernel = c->has_mask && tiles_in_kernel(step_launch(c)) ? 1 : 0;
    return LB_OK;
}

void lb_destroy(lb_ctx* c) { delete c; }

const char* lb_status_str(lb_status s) {
    switch (s) {
        case LB_OK: return "ok";
        case LB_EINVAL: return "invalid argument";
        case LB_ENOMEM: return "workspace too small";
        case LB_ECUDA: return "CUDA error";
        case LB_ENONFINITE: return "non-finite population";
        case LB_ESTATE: return "invalid state for this call";
        case LB_ETIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

const char* lb_last_error(void) { return g_last_error; }

}  // extern "C"
