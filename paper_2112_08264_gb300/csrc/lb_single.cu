// lb_single.cu -- one-component D3Q19 BGK step (the paper's single-fluid
// case: plain BGK, Eq. bgk with the Eq. LEQ equilibrium, fused streaming) and
// the lb1_* entry points of include/lb1.h.
//
// Same data movement as the two-component box step, without the density
// ring: a step has no neighbour-density dependence, so a block of one thread
// per x-y column marches along z, and per plane and velocity copies one box
// of the previous state (the tile shifted by -c_i, plus PAD columns each side
// for the x shift) into shared memory with 16-byte cp.async chunks; each
// thread reads its 19 pulled values, collides and stores. The copies of
// event e + nst - 1 go into the stage read at event e - 1 right after the
// one barrier of event e. Storage: deviations d_i = f_i - w_i rho0 in blocks
// of 64 sites, element (i, s) = (s / 64) * 19 * 64 + i * 64 + s mod 64.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>

#include <cuda_runtime.h>

#include "common.cuh"
#include "lb1.h"
#include "reduce.cuh"

namespace lbgb {

void record_error_text(const char* msg);

namespace single {

constexpr int kTX = 32;
constexpr int kMaxTY = 16;
constexpr int kB = 64;   // sites per storage block

__host__ __device__ __forceinline__ size_t sbase(uint32_t s) {
    return (size_t)(s / (uint32_t)kB) * (size_t)(Q * kB) + (size_t)(s % (uint32_t)kB);
}
inline size_t selems(long long N) { return (size_t)((N + kB - 1) / kB) * (size_t)(Q * kB); }

struct Par {
    float tau, omega;
    float g[3];
    float rho0;
};

struct Plan1 {
    int ncols, R, tymax, zsplit, zchunk, nst, threads;
    size_t smem;
};

template <typename S> struct Geo1 {
    static constexpr int CW = 16 / (int)sizeof(S);   // sites per 16-byte chunk
    static constexpr int PAD = CW;                   // box columns each side of the tile
    static constexpr int BW = kTX + 2 * PAD;         // box width (sites)
    static constexpr int CPR = BW / CW;              // chunks per box row
    // stage row: the 19 boxes of a row, padded to 16 bytes mod 128
    static constexpr int ROW0B = Q * BW * (int)sizeof(S);
    static constexpr int ROW = (ROW0B + ((16 - ROW0B % 128) + 128) % 128) / (int)sizeof(S);
};

__device__ __forceinline__ int wrap_any(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}
__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* gptr) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(gptr) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_wait_n(int n) {
    switch (n) {
        case 0: cp_wait<0>(); break;
        case 1: cp_wait<1>(); break;
        case 2: cp_wait<2>(); break;
        default: cp_wait<3>(); break;
    }
}

// BGK collision in deviation form and store: with drho = sum_i d_i, j = sum_i
// c_i d_i (opposite pairs), u = j / rho + tau g, the stored value is
// (1 - omega) d_i + omega w_i (drho + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u.u)).
template <typename S>
__device__ __forceinline__ void collide1(const float (&d)[Q], const Par& p, S* __restrict__ out) {
    float drho = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) drho += d[i];
    float j[3] = {0.f, 0.f, 0.f};
    static_for<0, 9>([&](auto M) {
        constexpr int i = 2 * decltype(M)::value + 1;
        const float diff = d[i] - d[i + 1];
        if constexpr (Vel<i>::x != 0) j[0] += Vel<i>::x * diff;
        if constexpr (Vel<i>::y != 0) j[1] += Vel<i>::y * diff;
        if constexpr (Vel<i>::z != 0) j[2] += Vel<i>::z * diff;
    });
    const float rho = p.rho0 + drho;
    const float inv = __fdividef(1.0f, rho);
    float u[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] = j[a] * inv + p.tau * p.g[a];
    const float uu15 = 1.5f * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const float om1 = 1.0f - p.omega;
    const float wr1 = p.omega * (1.0f / 18.0f) * rho, wd1 = p.omega * (1.0f / 18.0f) * drho;
    const float wr2 = p.omega * (1.0f / 36.0f) * rho, wd2 = p.omega * (1.0f / 36.0f) * drho;
    Store<S>::st(out, om1 * d[0] + p.omega * (1.0f / 3.0f) * (drho - rho * uu15));
    static_for<0, 9>([&](auto M) {
        constexpr int i = 2 * decltype(M)::value + 1;
        float cu = 0.f;
        if constexpr (Vel<i>::x != 0) cu += Vel<i>::x * u[0];
        if constexpr (Vel<i>::y != 0) cu += Vel<i>::y * u[1];
        if constexpr (Vel<i>::z != 0) cu += Vel<i>::z * u[2];
        constexpr bool axis = Vel<i>::c2 == 1;
        const float wr = axis ? wr1 : wr2, wd = axis ? wd1 : wd2;
        const float even = wr * (4.5f * cu * cu - uu15) + wd;
        const float odd = 3.0f * wr * cu;
        Store<S>::st(out + i * kB, om1 * d[i] + (even + odd));
        Store<S>::st(out + (i + 1) * kB, om1 * d[i + 1] + (even - odd));
    });
}

template <typename S>
__global__ void __launch_bounds__(kTX * kMaxTY, 1)
step1_kernel(const S* __restrict__ src, S* __restrict__ dst, Geom g, Par p, Plan1 P) {
    using B = Geo1<S>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const size_t stage_bytes = (size_t)P.tymax * B::ROW * sizeof(S);
    auto stage_base = [&](int st) -> S* { return reinterpret_cast<S*>(smem_raw + (size_t)st * stage_bytes); };

    const int t = threadIdx.x, tx = t & 31, ty = t >> 5;
    const int cx = blockIdx.x % P.ncols, cy = blockIdx.x / P.ncols;
    const int x0 = cx * kTX;
    const int y0 = (int)(((long long)cy * g.ny) / P.R);
    const int y1 = (int)(((long long)(cy + 1) * g.ny) / P.R);
    const int TYt = y1 - y0;
    const int z0 = blockIdx.y * P.zchunk;
    const int z1 = min(z0 + P.zchunk, g.nz);
    if (z0 >= z1) return;
    const int L = z1 - z0;
    const bool active = ty < TYt && (x0 + tx < g.nx);
    const int gx = wrap_any(x0 + tx, g.nx), gy = y0 + (ty < TYt ? ty : 0);

    // copier t (< tymax * CPR) owns chunk (row jr, column jc) of all 19 boxes;
    // the source row of velocity i is y0 + jr - c_iy (pull)
    const bool copier = t < P.tymax * B::CPR;
    const int jr = t / B::CPR, jc = t - (t / B::CPR) * B::CPR;
    const int xs = wrap_any(x0 - B::PAD + jc * B::CW, g.nx);
    const int yoff_m = wrap_any(y0 + jr + 1, g.ny) * g.nx + xs;   // c_iy = -1
    const int yoff_0 = wrap_any(y0 + jr, g.ny) * g.nx + xs;       // c_iy =  0
    const int yoff_p = wrap_any(y0 + jr - 1, g.ny) * g.nx + xs;   // c_iy = +1
    const int sdst = jr * B::ROW + jc * B::CW;

    auto issue = [&](int e, int z, int st) {
        if (e < L && copier) {
            const size_t pz_m = (size_t)wrap_inc(z, g.nz) * g.plane;   // c_iz = -1: plane z + 1
            const size_t pz_0 = (size_t)z * g.plane;
            const size_t pz_p = (size_t)wrap_dec(z, g.nz) * g.plane;   // c_iz = +1: plane z - 1
            const uint32_t sbase_s = (uint32_t)__cvta_generic_to_shared(stage_base(st) + sdst);
            static_for<0, Q>([&](auto II) {
                constexpr int i = decltype(II)::value;
                const size_t pz = Vel<i>::z < 0 ? pz_m : (Vel<i>::z > 0 ? pz_p : pz_0);
                const int yo = Vel<i>::y < 0 ? yoff_m : (Vel<i>::y > 0 ? yoff_p : yoff_0);
                // a chunk starts at a multiple of CW sites: inside one storage block
                cp_async16(sbase_s + i * B::BW * (int)sizeof(S), src + sbase((uint32_t)(pz + yo)) + i * kB);
            });
        }
        cp_commit();
    };

    const int ahead = P.nst - 1;   // events in flight
    int z_iss = z0;
    for (int e = 0; e < ahead; ++e) {
        issue(e, z_iss, e);
        z_iss = wrap_inc(z_iss, g.nz);
    }
    int st_cur = 0, z_cur = z0;
    for (int e = 0; e < L; ++e) {
        cp_wait_n(ahead - 1);
        __syncthreads();   // copies of event e visible; stage of event e - 1 fully read
        issue(e + ahead, z_iss, st_cur == 0 ? P.nst - 1 : st_cur - 1);
        if (active) {
            const S* nb = stage_base(st_cur) + ty * B::ROW + tx + B::PAD;
            float d[Q];
            static_for<0, Q>([&](auto II) {
                constexpr int i = decltype(II)::value;
                d[i] = Store<S>::to_f(nb[i * B::BW - Vel<i>::x]);
            });
            const uint32_t own = (uint32_t)gx + (uint32_t)g.nx * ((uint32_t)gy + (uint32_t)g.ny * (uint32_t)z_cur);
            collide1<S>(d, p, dst + sbase(own));
        }
        z_iss = wrap_inc(z_iss, g.nz);
        z_cur = wrap_inc(z_cur, g.nz);
        st_cur = st_cur + 1 == P.nst ? 0 : st_cur + 1;
    }
    cp_wait<0>();
}

__device__ __forceinline__ void xyz_of(long long s, const Geom& g, int& x, int& y, int& z) {
    x = (int)(s % g.nx);
    y = (int)((s / g.nx) % g.ny);
    z = (int)(s / g.plane);
}

// site x + sign * c_i
template <int i>
__device__ __forceinline__ uint32_t nb_site(const Geom& g, int x, int y, int z, int sign) {
    const int cx = sign * Vel<i>::x, cy = sign * Vel<i>::y, cz = sign * Vel<i>::z;
    const int xx = cx > 0 ? wrap_inc(x, g.nx) : (cx < 0 ? wrap_dec(x, g.nx) : x);
    const int yy = cy > 0 ? wrap_inc(y, g.ny) : (cy < 0 ? wrap_dec(y, g.ny) : y);
    const int zz = cz > 0 ? wrap_inc(z, g.nz) : (cz < 0 ? wrap_dec(z, g.nz) : z);
    return (uint32_t)xx + (uint32_t)g.nx * ((uint32_t)yy + (uint32_t)g.ny * (uint32_t)zz);
}

// pulled deviations f_i(x) - w_i rho0 = g_i(x - c_i) - w_i rho0
template <typename S>
__device__ __forceinline__ void pull1(const S* __restrict__ src, const Geom& g, long long s, float (&d)[Q]) {
    int x, y, z;
    xyz_of(s, g, x, y, z);
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        d[i] = Store<S>::ld(src + sbase(nb_site<i>(g, x, y, z, -1)) + i * kB);
    });
}

// g_j(y) = f_j^eq(rho, u)(y + c_j): the inverse of the pull
template <typename S>
__global__ void unstream1_kernel(S* __restrict__ dst, const float* __restrict__ rho, const float* __restrict__ u,
                                 Geom g, Par p) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.N) return;
    int x, y, z;
    xyz_of(s, g, x, y, z);
    static_for<0, Q>([&](auto J) {
        constexpr int j = decltype(J)::value;
        const uint32_t t = nb_site<j>(g, x, y, z, +1);
        const float r = rho[t];
        float uu = 0.f, cu = 0.f;
        if (u) {
            const float u0 = u[t], u1 = u[g.N + t], u2 = u[2 * g.N + t];
            uu = u0 * u0 + u1 * u1 + u2 * u2;
            cu = Vel<j>::x * u0 + Vel<j>::y * u1 + Vel<j>::z * u2;
        }
        Store<S>::st(dst + sbase((uint32_t)s) + j * kB,
                     wgt<j>() * ((r - p.rho0) + r * (cu * (3.0f + 4.5f * cu) - 1.5f * uu)));
    });
}

template <typename S>
__global__ void get_state1_kernel(const S* __restrict__ src, float* __restrict__ f, Geom g, Par p) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.N) return;
    float d[Q];
    pull1<S>(src, g, s, d);
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        f[(size_t)i * g.N + s] = wgt<i>() * p.rho0 + d[i];
    });
}

template <typename S>
__global__ void moments1_kernel(const S* __restrict__ src, float* __restrict__ orho, float* __restrict__ ou, Geom g,
                                Par p) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.N) return;
    float d[Q];
    pull1<S>(src, g, s, d);
    float drho = 0.f, j[3] = {0.f, 0.f, 0.f};
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        drho += d[i];
        if constexpr (Vel<i>::x != 0) j[0] += Vel<i>::x * d[i];
        if constexpr (Vel<i>::y != 0) j[1] += Vel<i>::y * d[i];
        if constexpr (Vel<i>::z != 0) j[2] += Vel<i>::z * d[i];
    });
    const float rho = p.rho0 + drho;
    if (orho) orho[s] = rho;
    if (ou) {
#pragma unroll
        for (int a = 0; a < 3; ++a) ou[(size_t)a * g.N + s] = (j[a] + 0.5f * rho * p.g[a]) / rho;
    }
}

// FP64 totals {mass, Px, Py, Pz, non-finite count, 0}: per node in FP32, across nodes in FP64
template <typename S>
__global__ void __launch_bounds__(256) stats1_kernel(const S* __restrict__ src, double* __restrict__ partials,
                                                     Geom g, Par p) {
    double v[kRedVals] = {0, 0, 0, 0, 0, 0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.N; s += stride) {
        float d[Q];
        pull1<S>(src, g, s, d);
        float drho = 0.f, j[3] = {0.f, 0.f, 0.f};
        bool ok = true;
        static_for<0, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            ok = ok && isfinite(d[i]);
            drho += d[i];
            if constexpr (Vel<i>::x != 0) j[0] += Vel<i>::x * d[i];
            if constexpr (Vel<i>::y != 0) j[1] += Vel<i>::y * d[i];
            if constexpr (Vel<i>::z != 0) j[2] += Vel<i>::z * d[i];
        });
        v[0] += (double)p.rho0 + (double)drho;
        v[1] += j[0];
        v[2] += j[1];
        v[3] += j[2];
        v[4] += ok ? 0.0 : 1.0;
    }
    block_sum_store(v, partials + (size_t)blockIdx.x * kRedVals);
}

// lb1_init input check: {sum rho, count, bad count, ...}
__global__ void check1_kernel(const float* __restrict__ rho, const float* __restrict__ u, double* __restrict__ partials,
                              Geom g) {
    double v[kRedVals] = {0, 0, 0, 0, 0, 0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.N; s += stride) {
        const float r = rho[s];
        bool ok = isfinite(r) && r > 0.f;
        if (u) ok = ok && isfinite(u[s]) && isfinite(u[g.N + s]) && isfinite(u[2 * g.N + s]);
        v[0] += r;
        v[1] += 1.0;
        v[2] += ok ? 0.0 : 1.0;
    }
    block_sum_store(v, partials + (size_t)blockIdx.x * kRedVals);
}

__global__ void __launch_bounds__(256) finish1_kernel(const double* __restrict__ partials, int nblk,
                                                      double* __restrict__ out) {
    double v[kRedVals] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < kRedVals; ++q) v[q] += partials[(size_t)b * kRedVals + q];
    block_sum_store(v, out);
}

Plan1 plan1(int nx, int ny, int nz, int sm_count, int esize, size_t smem_limit) {
    Plan1 best{};
    double best_cost = 1e300;
    const int ncols = (nx + kTX - 1) / kTX;
    const size_t row_bytes = esize == 4 ? (size_t)Geo1<float>::ROW * 4 : (size_t)Geo1<__half>::ROW * 2;
    const int cpr = esize == 4 ? Geo1<float>::CPR : Geo1<__half>::CPR;
    // 16-bit storage: two blocks per SM (measured +5 %; FP32 loses 7 %)
    const int occ = esize == 2 ? 2 : 1;
    const int rmin = (ny + kMaxTY - 1) / kMaxTY;
    for (int R = rmin; R <= ny; ++R) {
        const int tymax = (ny + R - 1) / R;
        const int threads = kTX * tymax;
        if (threads < tymax * cpr) continue;   // a thread per chunk position
        const size_t stage = (size_t)tymax * row_bytes;
        const size_t lim = occ == 2 ? (size_t)113 * 1024 : smem_limit;
        if (lim < 2 * stage) continue;
        int nst = (int)(lim / stage);
        nst = nst > 4 ? 4 : nst;
        const long long bxy = (long long)ncols * R;
        const int zs_max = nz / 4 > 1 ? nz / 4 : 1;
        for (int zs = 1; zs <= zs_max; ++zs) {
            const int zchunk = (nz + zs - 1) / zs;
            const long long blocks = bxy * zs;
            const long long waves = (blocks + occ * sm_count - 1) / (occ * sm_count);
            const double cost = waves * occ * (double)tymax * zchunk * (1.0 + 4.0 / (occ * tymax));
            if (cost < best_cost * (1 - 1e-9)) {
                best_cost = cost;
                best = Plan1{ncols, R, tymax, zs, zchunk, nst, threads, (size_t)nst * stage};
            }
            if (blocks >= occ * sm_count) break;
        }
    }
    return best;
}

template <typename F>
cudaError_t by_prec1(int prec, F&& f) {
    switch (prec) {
        case 0: return f(float{});
        case 1: return f(__half{});
        case 2: return f(__nv_bfloat16{});
        default: return cudaErrorInvalidValue;
    }
}

unsigned blocks_of(long long n) { return (unsigned)((n + 255) / 256); }

}  // namespace single
}  // namespace lbgb

using namespace lbgb;
using namespace lbgb::single;

struct lb1_ctx {
    Geom g;
    Par p;
    int prec;
    cudaStream_t stream;
    char* ws;
    size_t state_bytes;
    void* pop[2];
    int cur;
    double* part;
    double* out;
    Plan1 plan;
    bool initialized;
};

namespace {

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

bool dims_ok(int nx, int ny, int nz) {
    return nx >= 3 && ny >= 3 && nz >= 3 && (long long)nx * ny * nz < (1LL << 31);
}

lb_status status_of(const char* what, cudaError_t e) {
    if (e == cudaSuccess) return LB_OK;
    char msg[256];
    std::snprintf(msg, sizeof msg, "%s: %s", what, cudaGetErrorString(e));
    record_error_text(msg);
    return LB_ECUDA;
}

lb_status reduce_to_host(lb1_ctx* c, cudaError_t launched, double out[kRedVals]) {
    if (launched != cudaSuccess) return status_of("reduction launch", launched);
    finish1_kernel<<<1, 256, 0, c->stream>>>(c->part, kRedBlocks, c->out);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, c->out, kRedVals * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return status_of("reduction", e);
}

}  // namespace

extern "C" {

size_t lb1_workspace_bytes(int nx, int ny, int nz, int prec) {
    if (!dims_ok(nx, ny, nz) || prec < LB_FP32 || prec > LB_BF16_DEV) return 0;
    const size_t N = (size_t)nx * ny * nz;
    const size_t state = a256(selems((long long)N) * (prec == LB_FP32 ? 4 : 2));
    return 2 * state + a256((size_t)kRedBlocks * kRedVals * 8) + a256(kRedVals * 8);
}

lb_status lb1_create(int nx, int ny, int nz, float tau, const double* body_force, int prec, void* d_workspace,
                     size_t ws_bytes, void* stream, lb1_ctx** out) {
    if (!out) return LB_EINVAL;
    *out = nullptr;
    const size_t need = lb1_workspace_bytes(nx, ny, nz, prec);
    if (need == 0 || !std::isfinite(tau) || !(tau > 0.5f)) return LB_EINVAL;
    if (body_force)
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(body_force[a])) return LB_EINVAL;
    if (!d_workspace || ((uintptr_t)d_workspace & 255u)) return LB_EINVAL;
    if (ws_bytes < need) return LB_ENOMEM;
    int dev = 0, sms = 0, smem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return status_of("device query", e);
    lb1_ctx* c = new (std::nothrow) lb1_ctx();
    if (!c) return LB_EINVAL;
    c->g.nx = nx;
    c->g.ny = ny;
    c->g.nz = nz;
    c->g.plane = nx * ny;
    c->g.N = (long long)nx * ny * nz;
    c->p.tau = tau;
    c->p.omega = 1.0f / tau;
    for (int a = 0; a < 3; ++a) c->p.g[a] = body_force ? (float)body_force[a] : 0.f;
    c->p.rho0 = 1.0f;
    c->prec = prec;
    c->stream = static_cast<cudaStream_t>(stream);
    c->ws = static_cast<char*>(d_workspace);
    c->state_bytes = a256(selems(c->g.N) * (prec == LB_FP32 ? 4 : 2));
    c->pop[0] = c->ws;
    c->pop[1] = c->ws + c->state_bytes;
    c->part = reinterpret_cast<double*>(c->ws + 2 * c->state_bytes);
    c->out = reinterpret_cast<double*>(c->ws + 2 * c->state_bytes + a256((size_t)kRedBlocks * kRedVals * 8));
    c->cur = 0;
    c->plan = plan1(nx, ny, nz, sms, prec == LB_FP32 ? 4 : 2, (size_t)smem);
    // the box copies move 16-byte chunks of x rows: nx a multiple of 4 (FP32) or 8 sites
    if (c->plan.nst < 2 || nx % (prec == LB_FP32 ? 4 : 8) != 0) {
        delete c;
        return LB_EINVAL;
    }
    *out = c;
    return LB_OK;
}

lb_status lb1_init(lb1_ctx* c, const float* rho, const float* u) {
    if (!c || !rho) return LB_EINVAL;
    check1_kernel<<<kRedBlocks, 256, 0, c->stream>>>(rho, u, c->part, c->g);
    double red[kRedVals];
    lb_status s = reduce_to_host(c, cudaGetLastError(), red);
    if (s != LB_OK) return s;
    if (red[2] > 0.0) return LB_EINVAL;
    c->p.rho0 = (float)(red[0] / red[1]);
    c->cur = 0;
    cudaError_t e = by_prec1(c->prec, [&](auto tag) {
        using T = decltype(tag);
        unstream1_kernel<T><<<blocks_of(c->g.N), 256, 0, c->stream>>>(static_cast<T*>(c->pop[0]), rho, u, c->g, c->p);
        return cudaGetLastError();
    });
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return status_of("init", e);
    c->initialized = true;
    return LB_OK;
}

lb_status lb1_step(lb1_ctx* c, int n) {
    if (!c || n < 1) return LB_EINVAL;
    if (!c->initialized) return LB_ESTATE;
    const Plan1& P = c->plan;
    for (int t = 0; t < n; ++t) {
        cudaError_t e = by_prec1(c->prec, [&](auto tag) {
            using T = decltype(tag);
            auto kern = step1_kernel<T>;
            static size_t configured = 0;
            if (configured < P.smem) {
                cudaError_t a = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.smem);
                if (a != cudaSuccess) return a;
                // room for two resident blocks where the plan wants them
                a = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
                if (a != cudaSuccess) return a;
                configured = P.smem;
            }
            dim3 grid(P.ncols * P.R, P.zsplit, 1);
            kern<<<grid, P.threads, P.smem, c->stream>>>(static_cast<const T*>(c->pop[c->cur]),
                                                         static_cast<T*>(c->pop[1 - c->cur]), c->g, c->p, P);
            return cudaGetLastError();
        });
        if (e != cudaSuccess) return status_of("step", e);
        c->cur ^= 1;
    }
    return LB_OK;
}

lb_status lb1_moments(lb1_ctx* c, float* rho, float* u) {
    if (!c) return LB_EINVAL;
    if (!c->initialized) return LB_ESTATE;
    cudaError_t e = by_prec1(c->prec, [&](auto tag) {
        using T = decltype(tag);
        moments1_kernel<T><<<blocks_of(c->g.N), 256, 0, c->stream>>>(static_cast<const T*>(c->pop[c->cur]), rho, u,
                                                                     c->g, c->p);
        return cudaGetLastError();
    });
    return status_of("moments", e);
}

lb_status lb1_stats(lb1_ctx* c, double out4[4]) {
    if (!c || !out4) return LB_EINVAL;
    if (!c->initialized) return LB_ESTATE;
    cudaError_t e = by_prec1(c->prec, [&](auto tag) {
        using T = decltype(tag);
        stats1_kernel<T><<<kRedBlocks, 256, 0, c->stream>>>(static_cast<const T*>(c->pop[c->cur]), c->part, c->g,
                                                            c->p);
        return cudaGetLastError();
    });
    double red[kRedVals];
    lb_status s = reduce_to_host(c, e, red);
    if (s != LB_OK) return s;
    for (int q = 0; q < 4; ++q) out4[q] = red[q];
    return red[4] > 0.0 ? LB_ENONFINITE : LB_OK;
}

lb_status lb1_get_state(lb1_ctx* c, float* f) {
    if (!c || !f) return LB_EINVAL;
    if (!c->initialized) return LB_ESTATE;
    cudaError_t e = by_prec1(c->prec, [&](auto tag) {
        using T = decltype(tag);
        get_state1_kernel<T><<<blocks_of(c->g.N), 256, 0, c->stream>>>(static_cast<const T*>(c->pop[c->cur]), f, c->g,
                                                                       c->p);
        return cudaGetLastError();
    });
    return status_of("get_state", e);
}

lb_status lb1_launch_info(const lb1_ctx* c, int* blocks, int* threads) {
    if (!c) return LB_EINVAL;
    if (blocks) *blocks = c->plan.ncols * c->plan.R * c->plan.zsplit;
    if (threads) *threads = c->plan.threads;
    return LB_OK;
}

void lb1_destroy(lb1_ctx* c) { delete c; }

}  // extern "C"
