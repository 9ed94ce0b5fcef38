// lb_aux.cu -- kernels around the time step: solid flags, initial state
// (equilibrium, Eq. LEQ) and state import/export, moments, and the FP64
// conservation reduction.
#include <algorithm>
#include <vector>
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"
#include "reduce.cuh"

namespace lbgb {

namespace {

__device__ __forceinline__ void site_xyz(long long s, const Geom& g, int& x, int& y, int& z) {
    x = (int)(s % g.nx);
    y = (int)((s / g.nx) % g.ny);
    z = (int)(s / g.plane);
}

// Is link (x, i) -- fluid node (x, y, z), solid target x + c_i -- inside one
// tile of M: the target in the same column strip and row band (periodic in x
// and y), its plane inside the source's z-chunk? Never when M.R == 0.
template <int i>
__device__ __forceinline__ bool in_tile(int x, int y, int z, const Geom& g, const TileMap& M) {
    if (M.R == 0) return false;
    const int za = (z / M.zchunk) * M.zchunk;
    const int tz = z + Vel<i>::z;
    if (tz < za || tz >= min(za + M.zchunk, g.nz)) return false;
    const int tx = Vel<i>::x > 0 ? wrap_inc(x, g.nx) : (Vel<i>::x < 0 ? wrap_dec(x, g.nx) : x);
    const int ty = Vel<i>::y > 0 ? wrap_inc(y, g.ny) : (Vel<i>::y < 0 ? wrap_dec(y, g.ny) : y);
    return tx / kTileX == x / kTileX && band_of(ty, g.ny, M.R) == band_of(y, g.ny, M.R);
}
__device__ __forceinline__ int tile_index(int x, int y, const Geom& g, const TileMap& M) {
    return x / kTileX + M.ncols * band_of(y, g.ny, M.R);
}

__global__ void flags_kernel(const uint8_t* __restrict__ mask, uint32_t* __restrict__ flags, Geom g) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.N) return;
    int x, y, z;
    site_xyz(s, g, x, y, z);
    PullIdx P;
    pull_indices(g, x, y, z, P);
    uint32_t f = mask[s] ? kSolid : 0u;
    static_for<1, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if (mask[P.src[i]]) f |= (1u << i);
    });
    flags[s] = f;
}

// One thread per node. The read slots (velocity i at fluid x) and the
// written slots (velocity opp(i) at solid x + c_i) are disjoint, so the read
// and write views are restrict-qualified and every load of a node is in
// flight before its first store. Both components move as one pair.
template <typename S>
__global__ void reflect_kernel(const S* __restrict__ in, S* __restrict__ out,
                               const uint32_t* __restrict__ flags, Geom g) {
    using P = typename Store<S>::Pair;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.N) return;
    const uint32_t fl = __ldg(flags + s);
    if ((fl & kSolid) || !(fl & kNbSolidMask)) return;
    int x, y, z;
    site_xyz(s, g, x, y, z);
    P v[Q];
    static_for<1, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if (fl & (1u << Vel<i>::opp))   // x - c_opp(i) = x + c_i is solid
            v[i] = __ldg(reinterpret_cast<const P*>(in + pidx(0, i, (uint32_t)s)));
    });
    static_for<1, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int o = Vel<i>::opp;
        if (fl & (1u << o)) {
            const long long t = nb_index<i>(g, x, y, z);
            *reinterpret_cast<P*>(out + pidx(0, o, (uint32_t)t)) = v[i];
        }
    });
}

// Link list, pass 1: per velocity, the number of fluid sites x with x + c_i
// solid (flag bit opp(i)); block totals in shared memory, one global atomic
// per velocity and block.
__global__ void link_count_kernel(const uint32_t* __restrict__ flags, uint32_t* __restrict__ counts, TileMap M,
                                  Geom g) {
    __shared__ uint32_t cnt[Q];
    if (threadIdx.x < Q) cnt[threadIdx.x] = 0u;
    __syncthreads();
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t fl = s < g.N ? __ldg(flags + s) : kSolid;
    const bool fluid = !(fl & kSolid);
    int x = 0, y = 0, z = 0;
    if (s < g.N) site_xyz(s, g, x, y, z);
    static_for<1, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const unsigned b = __ballot_sync(0xffffffffu, fluid && (fl & (1u << Vel<i>::opp)) &&
                                                          !in_tile<i>(x, y, z, g, M));
        if ((threadIdx.x & 31) == 0 && b) atomicAdd(&cnt[i], (uint32_t)__popc(b));
    });
    __syncthreads();
    if (threadIdx.x >= 1 && threadIdx.x < Q && cnt[threadIdx.x]) atomicAdd(&counts[threadIdx.x], cnt[threadIdx.x]);
}

// Link list, pass 2: each block reserves its share of every velocity's
// segment with one atomic, warps take consecutive parts of it, lanes their
// rank within the warp.
__global__ void link_fill_kernel(const uint32_t* __restrict__ flags, uint32_t* __restrict__ cursor,
                                 uint32_t* __restrict__ sites, LinkList L, TileMap M, Geom g) {
    __shared__ uint32_t cnt[Q], base[Q];
    if (threadIdx.x < Q) cnt[threadIdx.x] = 0u;
    __syncthreads();
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t fl = s < g.N ? __ldg(flags + s) : kSolid;
    const bool fluid = !(fl & kSolid);
    int x = 0, y = 0, z = 0;
    if (s < g.N) site_xyz(s, g, x, y, z);
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t wpos[Q];
    uint32_t mine = 0u;   // this node's links that go into `sites`
    static_for<1, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const bool own = fluid && (fl & (1u << Vel<i>::opp)) && !in_tile<i>(x, y, z, g, M);
        mine |= own ? (1u << i) : 0u;
        const unsigned b = __ballot_sync(0xffffffffu, own);
        uint32_t w = 0u;
        if (lane == 0 && b) w = atomicAdd(&cnt[i], (uint32_t)__popc(b));
        wpos[i] = __shfl_sync(0xffffffffu, w, 0) + (uint32_t)__popc(b & lt);
    });
    __syncthreads();
    if (threadIdx.x >= 1 && threadIdx.x < Q)
        base[threadIdx.x] = cnt[threadIdx.x] ? atomicAdd(&cursor[threadIdx.x], cnt[threadIdx.x]) : 0u;
    __syncthreads();
    static_for<1, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if (mine & (1u << i)) sites[L.off[i] + base[i] + wpos[i]] = (uint32_t)s;
    });
}

// Tile lists, pass 1: per (tile, plane) the number of in-tile links of the
// fluid nodes there (all links of a node share its tile).
__global__ void tile_count_kernel(const uint32_t* __restrict__ flags, uint32_t* __restrict__ counts, TileMap M,
                                  Geom g) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.N) return;
    const uint32_t fl = __ldg(flags + s);
    if ((fl & kSolid) || !(fl & kNbSolidMask)) return;
    int x, y, z;
    site_xyz(s, g, x, y, z);
    uint32_t n = 0u;
    static_for<1, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if ((fl & (1u << Vel<i>::opp)) && in_tile<i>(x, y, z, g, M)) ++n;
    });
    if (n) atomicAdd(&counts[(size_t)tile_index(x, y, g, M) * g.nz + z], n);
}

// Tile lists, pass 2: each node reserves its links' places in its list with
// one atomic (the order within a list is immaterial: links are independent).
__global__ void tile_fill_kernel(const uint32_t* __restrict__ flags, uint32_t* __restrict__ cursor,
                                 const uint32_t* __restrict__ start, uint16_t* __restrict__ ent, TileMap M,
                                 Geom g) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.N) return;
    const uint32_t fl = __ldg(flags + s);
    if ((fl & kSolid) || !(fl & kNbSolidMask)) return;
    int x, y, z;
    site_xyz(s, g, x, y, z);
    uint32_t n = 0u;
    static_for<1, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if ((fl & (1u << Vel<i>::opp)) && in_tile<i>(x, y, z, g, M)) ++n;
    });
    if (!n) return;
    const size_t list = (size_t)tile_index(x, y, g, M) * g.nz + z;
    uint32_t pos = start[list] + atomicAdd(&cursor[list], n);
    const int lx = x % kTileX, ly = y - band_start(band_of(y, g.ny, M.R), g.ny, M.R);
    static_for<1, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if ((fl & (1u << Vel<i>::opp)) && in_tile<i>(x, y, z, g, M)) ent[pos++] = link_entry(lx, ly, i);
    });
}

// The tile lists as a pass of their own (step kernels other than the box
// kernel): one block per (tile, plane) list.
template <typename S>
__global__ void reflect_tiles_kernel(const S* __restrict__ in, S* __restrict__ out, LinkTiles T, TileMap M,
                                     Geom g) {
    using P = typename Store<S>::Pair;
    const long long b = blockIdx.x;
    const uint32_t a = __ldg(T.start + b), e = __ldg(T.start + b + 1);
    const int tile = (int)(b / g.nz), z = (int)(b - (long long)tile * g.nz);
    const int x0 = (tile % M.ncols) * kTileX, y0 = band_start(tile / M.ncols, g.ny, M.R);
    for (uint32_t k = a + threadIdx.x; k < e; k += blockDim.x) {
        const LinkSlots ls = tile_link_slots(__ldg(T.ent + k), x0, y0, z, g);
        *reinterpret_cast<P*>(out + ls.dst) = __ldg(reinterpret_cast<const P*>(in + ls.src));
    }
}

// The copy pass over the links: block row blockIdx.y + 1 = velocity i; one
// pair copy per link, g_i(x) into slot opp(i) of x + c_i.
template <typename S>
__global__ void reflect_links_kernel(const S* __restrict__ in, S* __restrict__ out, LinkList L, Geom g) {
    using P = typename Store<S>::Pair;
    const int vel = (int)blockIdx.y + 1;
    static_for<1, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if (vel != i) return;
        const long long k = L.off[i] + (long long)blockIdx.x * blockDim.x + threadIdx.x;
        if (k >= L.off[i + 1]) return;
        const uint32_t x0 = __ldg(L.sites + k);
        int x, y, z;
        site_xyz(x0, g, x, y, z);
        const P v = __ldg(reinterpret_cast<const P*>(in + pidx(0, i, x0)));
        x = Vel<i>::x > 0 ? wrap_inc(x, g.nx) : (Vel<i>::x < 0 ? wrap_dec(x, g.nx) : x);
        y = Vel<i>::y > 0 ? wrap_inc(y, g.ny) : (Vel<i>::y < 0 ? wrap_dec(y, g.ny) : y);
        z = Vel<i>::z > 0 ? wrap_inc(z, g.nz) : (Vel<i>::z < 0 ? wrap_dec(z, g.nz) : z);
        const uint32_t t = (uint32_t)x + (uint32_t)g.nx * ((uint32_t)y + (uint32_t)g.ny * (uint32_t)z);
        *reinterpret_cast<P*>(out + pidx(0, Vel<i>::opp, t)) = v;
    });
}

// g_j(y) = f_j(y + c_j) if y + c_j is fluid, else f_opp(j)(y); f is either the
// given field or the equilibrium of (rho^k, u). Solid nodes y get the same
// streaming source g_j(y) = f_j(y + c_j) where y + c_j is fluid (0 elsewhere):
// the fluid node x = y + c_j, whose population j bounces back at y, may read
// it there instead of g_opp(j)(x), which holds the same value.
template <typename S, bool FROM_F>
__global__ void unstream_kernel(S* __restrict__ dst, const uint32_t* __restrict__ flags,
                                const float* __restrict__ f, const float* __restrict__ rhoA,
                                const float* __restrict__ rhoB, const float* __restrict__ u, Geom g,
                                Phys p) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.N) return;
    int x, y, z;
    site_xyz(s, g, x, y, z);
    const uint32_t fl = flags ? flags[s] : 0u;
    const bool solid = (fl & kSolid) != 0u;
    const int xm = wrap_dec(x, g.nx), xp = wrap_inc(x, g.nx);
    const int ym = wrap_dec(y, g.ny), yp = wrap_inc(y, g.ny);
    const int zm = wrap_dec(z, g.nz), zp = wrap_inc(z, g.nz);
    static_for<0, Q>([&](auto J) {
        constexpr int j = decltype(J)::value;
        // destination neighbour y + c_j is solid <=> flag bit opp(j) (y - c_opp(j))
        const bool nb_solid = (j != 0) && (fl & (1u << Vel<j>::opp));
        const bool back = nb_solid && !solid;
        S* out = dst + pidx(0, j, (uint32_t)s);
        if (solid && (j == 0 || nb_solid)) {   // not read by any fluid node
            Store<S>::st2(out, 0.f, 0.f);
            return;
        }
        const int tx = Vel<j>::x == 1 ? xp : (Vel<j>::x == -1 ? xm : x);
        const int ty = Vel<j>::y == 1 ? yp : (Vel<j>::y == -1 ? ym : y);
        const int tz = Vel<j>::z == 1 ? zp : (Vel<j>::z == -1 ? zm : z);
        const long long t = back ? s : (tx + (long long)g.nx * (ty + (long long)g.ny * tz));
        float dev[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if constexpr (FROM_F) {
                const int pop = back ? Vel<j>::opp : j;
                dev[k] = f[(size_t)(k * Q + pop) * g.N + t] - wgt<j>() * p.rho0[k];
            } else {
                const float r = (k == 0 ? rhoA : rhoB)[t];
                float uu = 0.f, cu = 0.f;
                if (u) {
                    const float u0 = u[t], u1 = u[g.N + t], u2 = u[2 * g.N + t];
                    uu = u0 * u0 + u1 * u1 + u2 * u2;
                    cu = Vel<j>::x * u0 + Vel<j>::y * u1 + Vel<j>::z * u2;
                    if (back) cu = -cu;   // velocity opp(j) at node y
                }
                dev[k] = wgt<j>() * ((r - p.rho0[k]) + r * (cu * (3.0f + 4.5f * cu) - 1.5f * uu));
            }
        }
        Store<S>::st2(out, dev[0], dev[1]);
    });
}

template <typename S, bool MASK>
__global__ void get_state_kernel(const S* __restrict__ src, const uint32_t* __restrict__ flags,
                                 float* __restrict__ f, Geom g, Phys p) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.N) return;
    int x, y, z;
    site_xyz(s, g, x, y, z);
    uint32_t fl = 0;
    if constexpr (MASK) {
        fl = flags[s];
        if (fl & kSolid) {
            for (int j = 0; j < 2 * Q; ++j) f[(size_t)j * g.N + s] = 0.f;
            return;
        }
    }
    PullIdx P;
    pull_indices(g, x, y, z, P);
    float d[2][Q];
    pull<S, MASK>(src, g, P, p.slots ? 0u : fl, d);
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
#pragma unroll
        for (int k = 0; k < 2; ++k) f[(size_t)(k * Q + i) * g.N + s] = wgt<i>() * p.rho0[k] + d[k][i];
    });
}

template <typename S, bool MASK>
__global__ void densities_kernel(const S* __restrict__ src, const uint32_t* __restrict__ flags,
                                 float* __restrict__ rho, Geom g, Phys p) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.N) return;
    int x, y, z;
    site_xyz(s, g, x, y, z);
    const float2 r = density_at<S, MASK>(src, flags, g, p, x, y, z);
    rho[s] = r.x;
    rho[g.N + s] = r.y;
}

// rho^k, and u = (j + (F^A + F^B) / 2) / rho with F^A = -G psi^A S^B + rho^A g.
template <typename S, bool MASK>
__global__ void moments_kernel(const S* __restrict__ src, const uint32_t* __restrict__ flags,
                               const float* __restrict__ rho, float* __restrict__ oA, float* __restrict__ oB,
                               float* __restrict__ ou, Geom g, Phys p) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.N) return;
    int x, y, z;
    site_xyz(s, g, x, y, z);
    uint32_t fl = 0;
    if constexpr (MASK) fl = flags[s];
    if (fl & kSolid) {
        if (oA) oA[s] = 0.f;
        if (oB) oB[s] = 0.f;
        if (ou) ou[s] = ou[g.N + s] = ou[2 * g.N + s] = 0.f;
        return;
    }
    PullIdx P;
    pull_indices(g, x, y, z, P);
    float d[2][Q];
    pull<S, MASK>(src, g, P, p.slots ? 0u : fl, d);
    float dA, dB, j[3];
    sums<S>(d, dA, dB, j);
    const float rA = p.rho0[0] + dA, rB = p.rho0[1] + dB;
    if (oA) oA[s] = rA;
    if (oB) oB[s] = rB;
    if (!ou) return;
    if (p.model == 1) {   // colour gradient: no body force, u = j / rho
        const float inv = 1.0f / (rA + rB);
#pragma unroll
        for (int a = 0; a < 3; ++a) ou[a * g.N + s] = j[a] * inv;
        return;
    }
    float SA[3], SB[3];
    neighbour_sums<kFactoredSums<S>>(
        [&](int dx, int dy, int dz) {
            const int xx = dx > 0 ? wrap_inc(x, g.nx) : (dx < 0 ? wrap_dec(x, g.nx) : x);
            const int yy = dy > 0 ? wrap_inc(y, g.ny) : (dy < 0 ? wrap_dec(y, g.ny) : y);
            const int zz = dz > 0 ? wrap_inc(z, g.nz) : (dz < 0 ? wrap_dec(z, g.nz) : z);
            const long long t = xx + (long long)g.nx * (yy + (long long)g.ny * zz);
            return make_float2(rho[t], rho[g.N + t]);
        },
        SA, SB);
    const float inv = 1.0f / (rA + rB);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float F = -p.G * (rA * SB[a] + rB * SA[a]) + (rA + rB) * p.g[a];
        ou[a * g.N + s] = (j[a] + 0.5f * F) * inv;
    }
}

// ---- FP64 reductions ----

template <typename S, bool MASK>
__global__ void __launch_bounds__(256)
stats_kernel(const S* __restrict__ src, const uint32_t* __restrict__ flags, double* __restrict__ partials,
             Geom g, Phys p, long long s0, long long s1) {
    double v[kRedVals] = {0, 0, 0, 0, 0, 0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = s0 + (long long)blockIdx.x * blockDim.x + threadIdx.x; s < s1; s += stride) {
        int x, y, z;
        site_xyz(s, g, x, y, z);
        uint32_t fl = 0;
        if constexpr (MASK) {
            fl = flags[s];
            if (fl & kSolid) continue;
        }
        PullIdx P;
        pull_indices(g, x, y, z, P);
        float d[2][Q];
        pull<S, MASK>(src, g, P, p.slots ? 0u : fl, d);
        // per-node sums in FP32 (19 terms), accumulated across nodes in FP64
        float dA, dB, j[3];
        sums<S>(d, dA, dB, j);
        v[0] += (double)p.rho0[0] + (double)dA;
        v[1] += (double)p.rho0[1] + (double)dB;
        v[2] += (double)j[0];
        v[3] += (double)j[1];
        v[4] += (double)j[2];
        v[5] += (isfinite(dA) && isfinite(dB) && isfinite(j[0]) && isfinite(j[1]) && isfinite(j[2])) ? 0.0 : 1.0;
    }
    block_sum_store(v, partials + (size_t)blockIdx.x * kRedVals);
}

__global__ void check_init_kernel(const float* __restrict__ rA, const float* __restrict__ rB,
                                  const float* __restrict__ u, const uint32_t* __restrict__ flags,
                                  double* __restrict__ partials, Geom g, bool allow_zero) {
    double v[kRedVals] = {0, 0, 0, 0, 0, 0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.N; s += stride) {
        if (flags && (flags[s] & kSolid)) continue;
        const float a = rA[s], b = rB[s];
        bool ok = isfinite(a) && isfinite(b) &&
                  (allow_zero ? (a >= 0.f && b >= 0.f && a + b > 0.f) : (a > 0.f && b > 0.f));
        if (u) ok = ok && isfinite(u[s]) && isfinite(u[g.N + s]) && isfinite(u[2 * g.N + s]);
        v[0] += a;
        v[1] += b;
        v[2] += 1.0;
        v[3] += ok ? 0.0 : 1.0;
    }
    block_sum_store(v, partials + (size_t)blockIdx.x * kRedVals);
}

// Sum nblk rows of partials in a fixed order (one block).
__global__ void __launch_bounds__(256) finish_kernel(const double* __restrict__ partials, int nblk,
                                                     double* __restrict__ out) {
    double v[kRedVals] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < kRedVals; ++q) v[q] += partials[(size_t)b * kRedVals + q];
    block_sum_store(v, out);
}

unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename F4, typename F3, typename F2>
cudaError_t by_prec(int prec, F4&& f32, F3&& f16, F2&& bf16) {
    switch (prec) {
        case 0: f32(); break;
        case 1: f16(); break;
        case 2: bf16(); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_flags(const uint8_t* mask, uint32_t* flags, const Geom& g, cudaStream_t st) {
    flags_kernel<<<blocks_for(g.N, 256), 256, 0, st>>>(mask, flags, g);
    return cudaGetLastError();
}

cudaError_t build_links(const uint32_t* flags, uint32_t* sites, size_t capacity, uint32_t* cursor, TileMap M,
                        uint16_t* tent, size_t tcap, uint32_t* tstart, uint32_t* tscratch, const Geom& g,
                        LinkList& L, cudaStream_t st) {
    L = LinkList{};
    const unsigned nb = blocks_for(g.N, 256);
    cudaError_t e = cudaSuccess;
    LinkList T;
    if (M.R > 0 && tent && tstart && tscratch) {
        const size_t lists = (size_t)M.ncols * M.R * g.nz;
        if ((e = cudaMemsetAsync(tscratch, 0, lists * sizeof(uint32_t), st)) != cudaSuccess) return e;
        tile_count_kernel<<<nb, 256, 0, st>>>(flags, tscratch, M, g);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        std::vector<uint32_t> off(lists + 1);
        if ((e = cudaMemcpyAsync(off.data(), tscratch, lists * sizeof(uint32_t), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
        unsigned long long run = 0;
        long long most = 0;
        for (size_t k = 0; k < lists; ++k) {
            const uint32_t n = off[k];
            off[k] = (uint32_t)run;
            run += n;
            most = std::max(most, (long long)n);
        }
        if (run <= tcap && run < (1ull << 32)) {
            off[lists] = (uint32_t)run;
            if ((e = cudaMemcpyAsync(tstart, off.data(), (lists + 1) * sizeof(uint32_t), cudaMemcpyHostToDevice,
                                     st)) != cudaSuccess)
                return e;
            if ((e = cudaMemsetAsync(tscratch, 0, lists * sizeof(uint32_t), st)) != cudaSuccess) return e;
            tile_fill_kernel<<<nb, 256, 0, st>>>(flags, tscratch, tstart, tent, M, g);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            // the host copy of the offsets must outlive the upload
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
            T.tiles.start = tstart;
            T.tiles.ent = tent;
            T.map = M;
            T.tmost = most;
            T.tcount = (long long)run;
        }
    }
    const TileMap R = T.tiles.ent ? T.map : TileMap{};
    if ((e = cudaMemsetAsync(cursor, 0, 2 * Q * sizeof(uint32_t), st)) != cudaSuccess) return e;
    link_count_kernel<<<nb, 256, 0, st>>>(flags, cursor, R, g);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    uint32_t counts[Q];
    if ((e = cudaMemcpyAsync(counts, cursor, Q * sizeof(uint32_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    T.off[0] = T.off[1] = 0;
    for (int i = 1; i < Q; ++i) T.off[i + 1] = T.off[i] + counts[i];
    if ((size_t)T.off[Q] > capacity) {   // too many links: the pass scans every site (tile lists unused)
        L = LinkList{};
        return cudaSuccess;
    }
    T.sites = sites;
    if ((e = cudaMemsetAsync(cursor + Q, 0, Q * sizeof(uint32_t), st)) != cudaSuccess) return e;
    link_fill_kernel<<<nb, 256, 0, st>>>(flags, cursor + Q, sites, T, R, g);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    L = T;
    return cudaStreamSynchronize(st);
}

cudaError_t launch_reflect(int prec, void* g_state, const uint32_t* flags, const LinkList& links, bool with_tiles,
                           const Geom& g, cudaStream_t st) {
    if (links.sites) {
        if (links.tiles.ent && with_tiles && links.tmost > 0) {
            const unsigned lists = (unsigned)((long long)links.map.ncols * links.map.R * g.nz);
#define LBGB_TILES(T)                                                                                            \
    [&] {                                                                                                        \
        reflect_tiles_kernel<T><<<lists, 128, 0, st>>>((const T*)g_state, (T*)g_state, links.tiles, links.map, g); \
    }
            const cudaError_t e = by_prec(prec, LBGB_TILES(float), LBGB_TILES(__half), LBGB_TILES(__nv_bfloat16));
#undef LBGB_TILES
            if (e != cudaSuccess) return e;
        }
        long long most = 0;
        for (int i = 1; i < Q; ++i) most = std::max(most, links.off[i + 1] - links.off[i]);
        if (most == 0) return cudaSuccess;
        const dim3 grid((unsigned)((most + 255) / 256), Q - 1, 1);
#define LBGB_REFLECT(T) [&] { reflect_links_kernel<T><<<grid, 256, 0, st>>>((const T*)g_state, (T*)g_state, links, g); }
        return by_prec(prec, LBGB_REFLECT(float), LBGB_REFLECT(__half), LBGB_REFLECT(__nv_bfloat16));
#undef LBGB_REFLECT
    }
    const unsigned nb = blocks_for(g.N, 256);
#define LBGB_REFLECT(T) [&] { reflect_kernel<T><<<nb, 256, 0, st>>>((const T*)g_state, (T*)g_state, flags, g); }
    return by_prec(prec, LBGB_REFLECT(float), LBGB_REFLECT(__half), LBGB_REFLECT(__nv_bfloat16));
#undef LBGB_REFLECT
}

cudaError_t launch_unstream(int prec, void* dst, const uint32_t* flags, const float* f, const float* rhoA,
                            const float* rhoB, const float* u, const Geom& g, const Phys& p,
                            cudaStream_t st) {
    const unsigned nb = blocks_for(g.N, 256);
#define LBGB_UNSTREAM(T)                                                                          \
    [&] {                                                                                         \
        if (f) unstream_kernel<T, true><<<nb, 256, 0, st>>>((T*)dst, flags, f, rhoA, rhoB, u, g, p); \
        else unstream_kernel<T, false><<<nb, 256, 0, st>>>((T*)dst, flags, f, rhoA, rhoB, u, g, p); \
    }
    return by_prec(prec, LBGB_UNSTREAM(float), LBGB_UNSTREAM(__half), LBGB_UNSTREAM(__nv_bfloat16));
#undef LBGB_UNSTREAM
}

cudaError_t launch_get_state(int prec, const void* src, const uint32_t* flags, float* f, const Geom& g,
                             const Phys& p, cudaStream_t st) {
    const unsigned nb = blocks_for(g.N, 256);
#define LBGB_GET(T)                                                                          \
    [&] {                                                                                    \
        if (flags) get_state_kernel<T, true><<<nb, 256, 0, st>>>((const T*)src, flags, f, g, p); \
        else get_state_kernel<T, false><<<nb, 256, 0, st>>>((const T*)src, flags, f, g, p);      \
    }
    return by_prec(prec, LBGB_GET(float), LBGB_GET(__half), LBGB_GET(__nv_bfloat16));
#undef LBGB_GET
}

cudaError_t launch_densities(int prec, const void* src, const uint32_t* flags, float* rho, const Geom& g,
                             const Phys& p, cudaStream_t st) {
    const unsigned nb = blocks_for(g.N, 256);
#define LBGB_DEN(T)                                                                           \
    [&] {                                                                                     \
        if (flags) densities_kernel<T, true><<<nb, 256, 0, st>>>((const T*)src, flags, rho, g, p); \
        else densities_kernel<T, false><<<nb, 256, 0, st>>>((const T*)src, flags, rho, g, p);      \
    }
    return by_prec(prec, LBGB_DEN(float), LBGB_DEN(__half), LBGB_DEN(__nv_bfloat16));
#undef LBGB_DEN
}

cudaError_t launch_moments(int prec, const void* src, const uint32_t* flags, const float* rho, float* rhoA,
                           float* rhoB, float* u, const Geom& g, const Phys& p, cudaStream_t st) {
    const unsigned nb = blocks_for(g.N, 256);
#define LBGB_MOM(T)                                                                                  \
    [&] {                                                                                            \
        if (flags) moments_kernel<T, true><<<nb, 256, 0, st>>>((const T*)src, flags, rho, rhoA, rhoB, u, g, p); \
        else moments_kernel<T, false><<<nb, 256, 0, st>>>((const T*)src, flags, rho, rhoA, rhoB, u, g, p);      \
    }
    return by_prec(prec, LBGB_MOM(float), LBGB_MOM(__half), LBGB_MOM(__nv_bfloat16));
#undef LBGB_MOM
}

cudaError_t launch_stats(int prec, const void* src, const uint32_t* flags, double* partials, double* out,
                         const Geom& g, const Phys& p, cudaStream_t st, long long s0, long long s1) {
    if (s1 < 0 || s1 > g.N) s1 = g.N;
    if (s0 < 0) s0 = 0;
#define LBGB_STATS(T)                                                                                       \
    [&] {                                                                                                   \
        if (flags)                                                                                          \
            stats_kernel<T, true><<<kRedBlocks, 256, 0, st>>>((const T*)src, flags, partials, g, p, s0, s1); \
        else                                                                                                \
            stats_kernel<T, false><<<kRedBlocks, 256, 0, st>>>((const T*)src, flags, partials, g, p, s0, s1); \
    }
    cudaError_t e = by_prec(prec, LBGB_STATS(float), LBGB_STATS(__half), LBGB_STATS(__nv_bfloat16));
#undef LBGB_STATS
    if (e != cudaSuccess) return e;
    finish_kernel<<<1, 256, 0, st>>>(partials, kRedBlocks, out);
    return cudaGetLastError();
}

cudaError_t launch_check_init(const float* rhoA, const float* rhoB, const float* u, const uint32_t* flags,
                              double* partials, double* out, const Geom& g, bool allow_zero, cudaStream_t st) {
    check_init_kernel<<<kRedBlocks, 256, 0, st>>>(rhoA, rhoB, u, flags, partials, g, allow_zero);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    finish_kernel<<<1, 256, 0, st>>>(partials, kRedBlocks, out);
    return cudaGetLastError();
}

}  // namespace lbgb
