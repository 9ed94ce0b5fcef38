// lb_step.cu -- time-step kernels.
//
// FUSED, register double buffer (kernel 2; the default fused kernel is the
// asynchronous-copy variant in lb_fused_async.cu, same arithmetic): the
// paper's fused approach (Sec. 5.1), redesigned for the Shan-Chen force: one
// launch per step. The force at node x needs the post-streaming
// densities of its 18 neighbours, i.e. sums of populations pulled up to two
// sites away, so a block owns a TX x TY tile of x-y columns and marches along
// z. For each plane z+1 it pulls the 38 populations of its own columns (kept
// in registers for the next iteration) and of a one-node halo ring around the
// tile (density only, reads that mostly hit L2), and writes (rho^A, rho^B)
// into a 4-plane ring in shared memory (as deviations from rho0, see
// density_at). After one barrier it collides plane z
// from registers, reading the 18 neighbour densities from the ring, and
// stores it. HBM traffic is one read and one write of every population.
//
// TWO_PASS (the paper's plain approach): a density kernel writes rho^k to a
// scratch field, then a second kernel pulls the populations again, reads the
// neighbour densities from the scratch field and collides.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace lbgb {

namespace {

constexpr int kTX = 32;
constexpr int kTY = 8;
constexpr int kHalo = 2 * kTX + 2 * (kTY + 2);

__device__ __forceinline__ int wrap_any(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

template <typename S, bool MASK>
__global__ void __launch_bounds__(kTX * kTY, 2)
fused_step_kernel(const S* __restrict__ src, S* __restrict__ dst, const uint32_t* __restrict__ flags,
                  float* __restrict__ mom_out, Geom g, Phys p, int zchunk) {
    __shared__ float2 ring[4][kTY + 2][kTX + 2];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kTX + tx;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(z0 + zchunk, g.nz);
    if (z0 >= z1) return;   // uniform over the block

    // own column (wrapped, so ragged tiles still fill the ring correctly)
    const int gx = wrap_any(x0 + tx, g.nx), gy = wrap_any(y0 + ty, g.ny);
    const bool active = (x0 + tx < g.nx) && (y0 + ty < g.ny);

    // halo node handled by this thread (tid < kHalo)
    int hlx = 0, hly = 0;
    const bool has_halo = tid < kHalo;
    if (tid < kTX) { hlx = tid; hly = -1; }
    else if (tid < 2 * kTX) { hlx = tid - kTX; hly = kTY; }
    else if (tid < 2 * kTX + kTY + 2) { hlx = -1; hly = tid - 2 * kTX - 1; }
    else { hlx = kTX; hly = tid - (2 * kTX + kTY + 2) - 1; }
    const int hgx = wrap_any(x0 + hlx, g.nx), hgy = wrap_any(y0 + hly, g.ny);

    float cur[2][Q], nxt[2][Q];
    uint32_t fl_cur = 0;

    // plane z0 - 1: densities only
    {
        const int zz = wrap_any(z0 - 1, g.nz);
        ring[0][ty + 1][tx + 1] = density_at<S, MASK>(src, flags, g, p, gx, gy, zz);
        if (has_halo) ring[0][hly + 1][hlx + 1] = density_at<S, MASK>(src, flags, g, p, hgx, hgy, zz);
    }
    // plane z0: own populations kept
    {
        PullIdx P;
        pull_indices(g, gx, gy, z0, P);
        float2 r = make_float2(-p.rho0[0], -p.rho0[1]);
        if constexpr (MASK) fl_cur = __ldg(flags + P.own);
        if (!MASK || !(fl_cur & kSolid)) {
            pull<S, MASK>(src, g, P, fl_cur, cur);
            r = make_float2(dens_sum(cur[0]), dens_sum(cur[1]));
        }
        ring[1][ty + 1][tx + 1] = r;
        if (has_halo) ring[1][hly + 1][hlx + 1] = density_at<S, MASK>(src, flags, g, p, hgx, hgy, z0);
    }

    for (int z = z0; z < z1; ++z) {
        const int slot_m = (z - z0) & 3, slot_c = (z - z0 + 1) & 3, slot_p = (z - z0 + 2) & 3;
        const int zn = (z + 1 == g.nz) ? 0 : z + 1;
        // plane z + 1: own populations into nxt, densities of own column and halo
        uint32_t fl_nxt = 0;
        {
            PullIdx P;
            pull_indices(g, gx, gy, zn, P);
            float2 r = make_float2(-p.rho0[0], -p.rho0[1]);
            if constexpr (MASK) fl_nxt = __ldg(flags + P.own);
            if (!MASK || !(fl_nxt & kSolid)) {
                pull<S, MASK>(src, g, P, fl_nxt, nxt);
                r = make_float2(dens_sum(nxt[0]), dens_sum(nxt[1]));
            }
            ring[slot_p][ty + 1][tx + 1] = r;
            if (has_halo)
                ring[slot_p][hly + 1][hlx + 1] = density_at<S, MASK>(src, flags, g, p, hgx, hgy, zn);
        }
        __syncthreads();

        // collide plane z
        if (active && (!MASK || !(fl_cur & kSolid))) {
            float dA, dB, j[3];
            sums<S>(cur, dA, dB, j);
            float SA[3], SB[3];
            neighbour_sums<kFactoredSums<S>>(
                [&](int dx, int dy, int dz) {
                    const int s = dz < 0 ? slot_m : (dz > 0 ? slot_p : slot_c);
                    return ring[s][ty + 1 + dy][tx + 1 + dx];
                },
                SA, SB);
            const int own = gx + g.nx * (gy + g.ny * z);
            if (mom_out != nullptr) store_moments(mom_out, g, own, dA, dB, j, SA, SB);
            collide_store<S>(cur, p, dA, dB, j, SA, SB, dst, g, own);
        }
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int i = 0; i < Q; ++i) cur[k][i] = nxt[k][i];
        fl_cur = fl_nxt;
    }
}

// ---- two-pass ("plain") variant ----

template <typename S, bool MASK>
__global__ void __launch_bounds__(256)
density_kernel(const S* __restrict__ src, const uint32_t* __restrict__ flags, float* __restrict__ rho,
               Geom g, Phys p) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.N) return;
    const int x = (int)(s % g.nx);
    const int y = (int)((s / g.nx) % g.ny);
    const int z = (int)(s / g.plane);
    const float2 r = density_at<S, MASK>(src, flags, g, p, x, y, z);
    rho[s] = r.x;
    rho[g.N + s] = r.y;
}

template <typename S, bool MASK>
__global__ void __launch_bounds__(256)
collide_kernel(const S* __restrict__ src, S* __restrict__ dst, const uint32_t* __restrict__ flags,
               const float* __restrict__ rho, float* __restrict__ mom_out, Geom g, Phys p) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.N) return;
    const int x = (int)(s % g.nx);
    const int y = (int)((s / g.nx) % g.ny);
    const int z = (int)(s / g.plane);
    uint32_t fl = 0;
    if constexpr (MASK) {
        fl = __ldg(flags + s);
        if (fl & kSolid) return;
    }
    PullIdx P;
    pull_indices(g, x, y, z, P);
    float d[2][Q];
    pull<S, MASK>(src, g, P, fl, d);
    float dA, dB, j[3];
    sums<S>(d, dA, dB, j);
    float SA[3], SB[3];
    const bool cg = p.model == 1;   // colour gradient: the neighbour sums of Theta
    neighbour_sums<kFactoredSums<S>>(
        [&](int dx, int dy, int dz) {
            const int xx = dx > 0 ? wrap_inc(x, g.nx) : (dx < 0 ? wrap_dec(x, g.nx) : x);
            const int yy = dy > 0 ? wrap_inc(y, g.ny) : (dy < 0 ? wrap_dec(y, g.ny) : y);
            const int zz = dz > 0 ? wrap_inc(z, g.nz) : (dz < 0 ? wrap_dec(z, g.nz) : z);
            const long long t = xx + (long long)g.nx * (yy + (long long)g.ny * zz);
            const float2 r = make_float2(__ldg(rho + t), __ldg(rho + g.N + t));
            if (cg) {
                const float th = phase_field(p, r.x, r.y);
                return make_float2(th, th);
            }
            return r;
        },
        SA, SB);
    if (cg) {
        const float gt[3] = {3.0f * SA[0], 3.0f * SA[1], 3.0f * SA[2]};
        cg_collide_store_g<S>([&](int k, int i) { return d[k][i]; }, p, dA, dB, j, gt, dst, (int)s);
        return;
    }
    if (mom_out != nullptr) store_moments(mom_out, g, s, dA, dB, j, SA, SB);
    collide_store<S>(d, p, dA, dB, j, SA, SB, dst, g, (int)s);
}

template <typename S, bool MASK>
cudaError_t launch_step_t(const StepLaunch& L, cudaStream_t st) {
    const S* src = static_cast<const S*>(L.src);
    S* dst = static_cast<S*>(L.dst);
    if (L.kernel == 2) {
        dim3 block(kTX, kTY, 1);
        dim3 grid((L.g.nx + kTX - 1) / kTX, (L.g.ny + kTY - 1) / kTY, L.zsplit);
        const int zchunk = (L.g.nz + L.zsplit - 1) / L.zsplit;
        fused_step_kernel<S, MASK><<<grid, block, 0, st>>>(src, dst, L.flags, L.mom_out, L.g, L.p, zchunk);
    } else {
        const unsigned nb = (unsigned)((L.g.N + 255) / 256);
        density_kernel<S, MASK><<<nb, 256, 0, st>>>(src, L.flags, L.rho, L.g, L.p);
        collide_kernel<S, MASK><<<nb, 256, 0, st>>>(src, dst, L.flags, L.rho, L.mom_out, L.g, L.p);
    }
    return cudaGetLastError();
}

}  // namespace

namespace {
cudaError_t launch_step_kernels(const StepLaunch& L, cudaStream_t st) {
    // the colour-gradient model runs on the box kernel or the two-pass kernels
    if (L.kernel == 0 && (L.p.model == 0 || L.plan.box)) return launch_fused_async(L, st);
    const bool m = L.flags != nullptr;
    switch (L.prec) {
        case 0: return m ? launch_step_t<float, true>(L, st) : launch_step_t<float, false>(L, st);
        case 1: return m ? launch_step_t<__half, true>(L, st) : launch_step_t<__half, false>(L, st);
        case 2:
            return m ? launch_step_t<__nv_bfloat16, true>(L, st) : launch_step_t<__nv_bfloat16, false>(L, st);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace

bool tiles_in_kernel(const StepLaunch& L) {
    const LinkList& k = L.links;
    return L.flags != nullptr && k.sites != nullptr && k.tiles.ent != nullptr && L.kernel == 0 && L.p.model == 0 &&
           L.plan.box && k.map.ncols == L.plan.ncols && k.map.R == L.plan.R && k.map.zchunk == L.plan.zchunk;
}

cudaError_t launch_step_fluid(const StepLaunch& L, cudaStream_t st) { return launch_step_kernels(L, st); }

cudaError_t launch_step_links(const StepLaunch& L, cudaStream_t st) {
    if (L.flags == nullptr) return cudaSuccess;
    return launch_reflect(L.prec, L.dst, L.flags, L.links, !tiles_in_kernel(L), L.g, st);
}

cudaError_t launch_step(const StepLaunch& L, cudaStream_t st) {
    const cudaError_t e = launch_step_fluid(L, st);
    if (e != cudaSuccess) return e;
    return launch_step_links(L, st);
}

void fused_geometry(int nx, int ny, int nz, int sm_count, int* tiles, int* zsplit, int* threads) {
    const int t = ((nx + kTX - 1) / kTX) * ((ny + kTY - 1) / kTY);
    // aim for at least two resident blocks per SM; a z-chunk shorter than 8
    // planes pays more than 25% extra density work for its two halo planes
    const int want = 2 * sm_count;
    int zs = (want + t - 1) / t;
    if (t >= sm_count) zs = 1;
    zs = zs < 1 ? 1 : zs;
    const int maxzs = nz / 8 > 1 ? nz / 8 : 1;
    if (zs > maxzs) zs = maxzs;
    *tiles = t;
    *zsplit = zs;
    *threads = kTX * kTY;
}

}  // namespace lbgb
