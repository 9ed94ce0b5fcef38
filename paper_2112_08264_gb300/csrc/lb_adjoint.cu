// lb_adjoint.cu -- reverse-mode step with checkpoint recompute (derivation in
// adjoint.h).
//
// Backward over a recorded run of T steps with checkpoints every K steps:
// for each segment, last to first, the forward step is re-run from its
// checkpoint (the same kernel, so the same bits), keeping every state of the
// segment and, per node, the moments the reverse step needs (drho^A, drho^B,
// j, S^A, S^B). The adjoint then runs backwards through the segment:
//   box kernel (nx a multiple of 4): one launch per reverse step; per plane
//     the block copies boxes of lambda_{t+1} (shifted by +c_i, the transpose
//     of the pull) and of the moments, computes sigma^k for its tile and
//     halo into a 4-plane ring and, after one barrier, writes lambda_t of the
//     previous plane with the neighbour gather of sigma;
//   two-pass fallback: pass A writes W, q_k, sigma^k per node, pass B gathers.
// dL/dG accumulates in FP64 per block and is summed in a fixed order.
#include <cstdint>

#include <cuda_runtime.h>

#include "adjoint.h"
#include "kernels.h"
#include "reduce.cuh"

namespace lbgb {

namespace {

constexpr int kAux = 11;   // W[3], q[2], sigma^A[3], sigma^B[3]
constexpr int kTX = 32;
// tile rows of the box kernel: two stages of its boxes fit in shared memory
// for about 11 rows, and 12 rows (384 threads) leave 168 registers a thread
constexpr int kAdjMaxTY = 12;

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct AdjBufs {
    float* lam[2];
    float* aux;
    float* segmom;
    double* gacc;
};

AdjBufs carve(char* adj, size_t N, int K) {
    AdjBufs b;
    size_t off = 0;
    b.lam[0] = reinterpret_cast<float*>(adj + off); off += a256(state_elems((long long)N) * 4);
    b.lam[1] = reinterpret_cast<float*>(adj + off); off += a256(state_elems((long long)N) * 4);
    b.aux = reinterpret_cast<float*>(adj + off); off += a256((size_t)kAux * N * 4);
    b.segmom = reinterpret_cast<float*>(adj + off); off += a256((size_t)K * mom_elems((long long)N) * 4);
    b.gacc = reinterpret_cast<double*>(adj + off);
    return b;
}

__device__ __forceinline__ int wrap_any(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

__device__ __forceinline__ void site_xyz(long long s, const Geom& g, int& x, int& y, int& z) {
    x = (int)(s % g.nx);
    y = (int)((s / g.nx) % g.ny);
    z = (int)(s / g.plane);
}

// mu_i(x) = lambda_i(x + c_i) if x + c_i is fluid, else lambda_opp(i)(x).
// lambda is stored like the populations (blocked, (A, B) pairs; pidx).
template <bool MASK>
__device__ __forceinline__ void gather_mu(const float* __restrict__ lam, const Geom& g, int x, int y, int z,
                                          long long own, uint32_t fl, float (&mu)[2][Q]) {
    const int xm = wrap_dec(x, g.nx), xp = wrap_inc(x, g.nx);
    const int ym = wrap_dec(y, g.ny), yp = wrap_inc(y, g.ny);
    const int zm = wrap_dec(z, g.nz), zp = wrap_inc(z, g.nz);
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const int tx = Vel<i>::x == 1 ? xp : (Vel<i>::x == -1 ? xm : x);
        const int ty = Vel<i>::y == 1 ? yp : (Vel<i>::y == -1 ? ym : y);
        const int tz = Vel<i>::z == 1 ? zp : (Vel<i>::z == -1 ? zm : z);
        long long t = tx + (long long)g.nx * (ty + (long long)g.ny * tz);
        int pop = i;
        if constexpr (MASK && i != 0) {
            if (fl & (1u << Vel<i>::opp)) { t = own; pop = Vel<i>::opp; }
        }
        Store<float>::ld2(lam + pidx(0, pop, (uint32_t)t), mu[0][i], mu[1][i]);
    });
}

// Per-node adjoint quantities of the collision (see adjoint.h) from the
// forward moments (dA, dB, j, S^A, S^B) and the adjoint mu.
__device__ __forceinline__ void adj_node(const float (&mo)[kMom], const float (&mu)[2][Q], const Phys& p,
                                         float (&W)[3], float (&q)[2], float (&sA)[3], float (&sB)[3], float& dG) {
    const float rA = p.rho0[0] + mo[0], rB = p.rho0[1] + mo[1];
    const float inv = __fdividef(1.0f, rA + rB);   // as in the forward collision
    const float up[3] = {mo[2] * inv, mo[3] * inv, mo[4] * inv};
    const float SA[3] = {mo[5], mo[6], mo[7]}, SB[3] = {mo[8], mo[9], mo[10]};
    float V[2][3], E[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float (&Sk)[3] = (k == 0) ? SB : SA;
        const float rk = (k == 0) ? rA : rB;
        float v[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) v[a] = up[a] + p.tau * (p.g[a] - p.G * Sk[a]);
        float m0 = 0.f, m1[3] = {0.f, 0.f, 0.f}, mxx = 0.f, myy = 0.f, mzz = 0.f, mxy = 0.f, mxz = 0.f, myz = 0.f;
        static_for<0, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            const float wm = wgt<i>() * mu[k][i];
            m0 += wm;
            if constexpr (Vel<i>::x != 0) { m1[0] += Vel<i>::x * wm; mxx += wm; }
            if constexpr (Vel<i>::y != 0) { m1[1] += Vel<i>::y * wm; myy += wm; }
            if constexpr (Vel<i>::z != 0) { m1[2] += Vel<i>::z * wm; mzz += wm; }
            if constexpr (Vel<i>::x * Vel<i>::y != 0) mxy += (Vel<i>::x * Vel<i>::y) * wm;
            if constexpr (Vel<i>::x * Vel<i>::z != 0) mxz += (Vel<i>::x * Vel<i>::z) * wm;
            if constexpr (Vel<i>::y * Vel<i>::z != 0) myz += (Vel<i>::y * Vel<i>::z) * wm;
        });
        const float M2v[3] = {mxx * v[0] + mxy * v[1] + mxz * v[2], mxy * v[0] + myy * v[1] + myz * v[2],
                              mxz * v[0] + myz * v[1] + mzz * v[2]};
        const float vM2v = v[0] * M2v[0] + v[1] * M2v[1] + v[2] * M2v[2];
        const float vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        const float m1v = m1[0] * v[0] + m1[1] * v[1] + m1[2] * v[2];
        E[k] = p.omega * (m0 + 3.0f * m1v + 4.5f * vM2v - 1.5f * vv * m0);
#pragma unroll
        for (int a = 0; a < 3; ++a) V[k][a] = p.omega * rk * (3.0f * m1[a] + 9.0f * M2v[a] - 3.0f * v[a] * m0);
    }
    float Wu = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        W[a] = (V[0][a] + V[1][a]) * inv;
        Wu += W[a] * up[a];
        sB[a] = -p.tau * p.G * V[0][a];
        sA[a] = -p.tau * p.G * V[1][a];
    }
    q[0] = E[0] - Wu;
    q[1] = E[1] - Wu;
    dG = -p.tau * (V[0][0] * SB[0] + V[0][1] * SB[1] + V[0][2] * SB[2] +
                   V[1][0] * SA[0] + V[1][1] * SA[1] + V[1][2] * SA[2]);
}

// local part of lambda_t: (1 - omega) mu_i + c_i . W + q_k, in place
__device__ __forceinline__ void local_part(float (&mu)[2][Q], const Phys& p, const float (&W)[3],
                                           const float (&q)[2]) {
    const float om1 = 1.0f - p.omega;
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        float cW = 0.f;
        if constexpr (Vel<i>::x != 0) cW += Vel<i>::x * W[0];
        if constexpr (Vel<i>::y != 0) cW += Vel<i>::y * W[1];
        if constexpr (Vel<i>::z != 0) cW += Vel<i>::z * W[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) mu[k][i] = om1 * mu[k][i] + cW + q[k];
    });
}

// ---- two-pass fallback ----

template <bool MASK>
__global__ void __launch_bounds__(256)
adj_pass_a(const float* __restrict__ mom, const float* __restrict__ lam, const uint32_t* __restrict__ flags,
           float* __restrict__ aux, double* __restrict__ partials, Geom g, Phys p) {
    double v[kRedVals] = {0, 0, 0, 0, 0, 0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.N; s += stride) {
        int x, y, z;
        site_xyz(s, g, x, y, z);
        uint32_t fl = 0;
        if constexpr (MASK) fl = flags[s];
        if (fl & kSolid) {
#pragma unroll
            for (int c = 0; c < kAux; ++c) aux[(size_t)c * g.N + s] = 0.f;
            continue;
        }
        float mu[2][Q];
        gather_mu<MASK>(lam, g, x, y, z, s, fl, mu);
        float mo[kMom];
#pragma unroll
        for (int c = 0; c < kMom; ++c) mo[c] = __ldg(mom + mom_base((uint32_t)s) + c * kBlk);
        float W[3], q[2], sA[3], sB[3], dG;
        adj_node(mo, mu, p, W, q, sA, sB, dG);
        const float out[kAux] = {W[0], W[1], W[2], q[0], q[1], sA[0], sA[1], sA[2], sB[0], sB[1], sB[2]};
#pragma unroll
        for (int c = 0; c < kAux; ++c) aux[(size_t)c * g.N + s] = out[c];
        v[0] += (double)dG;
    }
    block_sum_store(v, partials + (size_t)blockIdx.x * kRedVals);
}

template <bool MASK>
__global__ void __launch_bounds__(256)
adj_pass_b(const float* __restrict__ lam_in, const float* __restrict__ aux, const uint32_t* __restrict__ flags,
           float* __restrict__ lam_out, Geom g, Phys p) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.N) return;
    int x, y, z;
    site_xyz(s, g, x, y, z);
    uint32_t fl = 0;
    if constexpr (MASK) fl = flags[s];
    float* out = lam_out + blk_base((uint32_t)s);
    if (fl & kSolid) {
        for (int i = 0; i < Q; ++i) Store<float>::st2(out + i * (2 * kBlk), 0.f, 0.f);
        return;
    }
    float mu[2][Q];
    gather_mu<MASK>(lam_in, g, x, y, z, s, fl, mu);
    const float W[3] = {aux[s], aux[g.N + s], aux[2 * g.N + s]};
    const float q[2] = {aux[3 * g.N + s], aux[4 * g.N + s]};
    local_part(mu, p, W, q);
    // h^k(x) = sum_{i>=1} w_i c_i . sigma^k(x - c_i)
    PullIdx P;
    pull_indices(g, x, y, z, P);
    float h[2] = {0.f, 0.f};
    static_for<1, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const long long t = P.src[i];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const float* sk = aux + (size_t)(5 + 3 * k) * g.N;
            float acc = 0.f;
            if constexpr (Vel<i>::x != 0) acc += Vel<i>::x * __ldg(sk + t);
            if constexpr (Vel<i>::y != 0) acc += Vel<i>::y * __ldg(sk + g.N + t);
            if constexpr (Vel<i>::z != 0) acc += Vel<i>::z * __ldg(sk + 2 * g.N + t);
            h[k] += wgt<i>() * acc;
        }
    });
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        Store<float>::st2(out + i * (2 * kBlk), mu[0][i] + h[0], mu[1][i] + h[1]);
    });
}

// ---- fused box adjoint ----

// Stage row of the box kernel: 19 lambda boxes of (A, B) pairs (2 sites per
// 16-byte chunk, 2 sites of halo each side), then 11 moment boxes (4 sites
// per chunk, 4 sites of halo each side), padded to 16 bytes mod 128 so that
// the column-halo nodes of consecutive rows spread over the banks.
constexpr int kLPAD = 2;                  // lambda box sites left of the tile
constexpr int kLBW = kTX + 2 * kLPAD;     // lambda box width (sites)
constexpr int kLCPR = kLBW / 2;           // 16-byte chunks per lambda box row
constexpr int kLVS = 2 * kLBW;            // floats per lambda box row
constexpr int kMPAD = 4;                  // moment and flag box sites left of the tile
constexpr int kMBW = kTX + 2 * kMPAD;     // moment and flag box width (sites)
constexpr int kMCPR = kMBW / 4;           // 16-byte chunks per moment box row
constexpr int kROW0 = Q * kLVS + kMom * kMBW;
constexpr int kROW = kROW0 + (((16 - (kROW0 * 4) % 128) + 128) % 128) / 4;   // stage row stride (floats)
static_assert((kROW * 4) % 16 == 0, "stage rows must stay 16-byte aligned");

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

struct Sig {
    float a[3], b[3];
};

template <bool MASK>
__global__ void __launch_bounds__(kTX * kAdjMaxTY, 1)
adj_box_kernel(const float* __restrict__ lam_in, const float* __restrict__ mom, const uint32_t* __restrict__ flags,
               float* __restrict__ lam_out, double* __restrict__ partials, Geom g, Phys p, AsyncPlan P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int RH = P.tymax + 2, RW = kTX + 2;
    const size_t box_bytes = (size_t)RH * kROW * 4;
    const size_t stage_bytes = box_bytes + (MASK ? (size_t)RH * kMBW * 4 : 0);
    auto stage_base = [&](int st) -> float* { return reinterpret_cast<float*>(smem_raw + (size_t)st * stage_bytes); };
    auto stage_flags = [&](int st) -> uint32_t* {
        return reinterpret_cast<uint32_t*>(smem_raw + (size_t)st * stage_bytes + box_bytes);
    };
    Sig* ring = reinterpret_cast<Sig*>(smem_raw + (size_t)P.nst * stage_bytes);
    auto ring_at = [&](int slot, int ly, int lx) -> Sig& { return ring[(slot * RH + ly + 1) * RW + lx + 1]; };

    const int t = threadIdx.x, tx = t & 31, ty = t >> 5;
    const int cx = blockIdx.x % P.ncols, cy = blockIdx.x / P.ncols;
    const int x0 = cx * kTX;
    const int y0 = (int)(((long long)cy * g.ny) / P.R);
    const int y1 = (int)(((long long)(cy + 1) * g.ny) / P.R);
    const int TYt = y1 - y0;
    const int z0 = blockIdx.y * P.zchunk;
    const int z1 = min(z0 + P.zchunk, g.nz);
    double dG_acc[kRedVals] = {0, 0, 0, 0, 0, 0};
    if (z0 < z1) {
        const int L = (z1 - z0) + 2;
        const bool own_row = ty < TYt;
        const int gx = wrap_any(x0 + tx, g.nx);
        const int gy = own_row ? y0 + ty : y0;
        const bool active = own_row && (x0 + tx < g.nx);
        const int nh = 2 * RW + 2 * TYt;
        const bool has_halo = t < nh;
        int hlx = 0, hly = 0;
        if (t < RW) { hlx = t - 1; hly = -1; }
        else if (t < 2 * RW) { hlx = t - RW - 1; hly = TYt; }
        else if (t < 2 * RW + TYt) { hlx = -1; hly = t - 2 * RW; }
        else { hlx = kTX; hly = t - 2 * RW - TYt; }
        const int hgx = wrap_any(x0 + hlx, g.nx), hgy = wrap_any(y0 + hly, g.ny);
        auto plane_of = [&](int e) { return wrap_any(z0 - 1 + e, g.nz); };

        // copier t (< RH * kLCPR) owns chunk (jr, jc) of every lambda box and,
        // for jc < kMCPR, of every moment box and the flag box
        const bool copier = t < RH * kLCPR;
        const int jr = t / kLCPR, jc = t - (t / kLCPR) * kLCPR;
        const bool mcopier = copier && jc < kMCPR;
        const int xs_chunk = wrap_any(x0 - kLPAD + jc * 2, g.nx);
        // lambda box of velocity i: rows from y0 - 1 + c_iy (gather x + c_i)
        const int yoff_m = wrap_any(y0 - 2 + jr, g.ny) * g.nx + xs_chunk;   // c_iy = -1
        const int yoff_0 = wrap_any(y0 - 1 + jr, g.ny) * g.nx + xs_chunk;   // c_iy =  0
        const int yoff_p = wrap_any(y0 + jr, g.ny) * g.nx + xs_chunk;       // c_iy = +1
        const int moff = wrap_any(y0 - 1 + jr, g.ny) * g.nx + wrap_any(x0 - kMPAD + jc * 4, g.nx);
        const int sdst = jr * kROW + jc * 4;
        const int mdst = jr * kROW + Q * kLVS + jc * 4;
        const int fdst = jr * kMBW + jc * 4;

        auto issue = [&](int e) {
            if (e < L && copier) {
                const int z = plane_of(e), st = e % P.nst;
                const size_t pz_m = (size_t)wrap_dec(z, g.nz) * g.plane;   // c_iz = -1: plane z - 1
                const size_t pz_0 = (size_t)z * g.plane;
                const size_t pz_p = (size_t)wrap_inc(z, g.nz) * g.plane;   // c_iz = +1: plane z + 1
                const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(stage_base(st) + sdst);
                static_for<0, Q>([&](auto II) {
                    constexpr int i = decltype(II)::value;
                    const size_t pz = Vel<i>::z < 0 ? pz_m : (Vel<i>::z > 0 ? pz_p : pz_0);
                    const int yo = Vel<i>::y < 0 ? yoff_m : (Vel<i>::y > 0 ? yoff_p : yoff_0);
                    // a chunk of 2 sites never straddles a storage block
                    cp_async16(sbase + i * kLVS * 4, lam_in + blk_base((uint32_t)(pz + yo)) + i * (2 * kBlk));
                });
                if (mcopier) {
                    const uint32_t mbase = (uint32_t)__cvta_generic_to_shared(stage_base(st) + mdst);
                    const float* msrc = mom + mom_base((uint32_t)(pz_0 + moff));
                    static_for<0, kMom>([&](auto CC) {
                        constexpr int c = decltype(CC)::value;
                        cp_async16(mbase + c * kMBW * 4, msrc + c * kBlk);
                    });
                    if constexpr (MASK)
                        cp_async16((uint32_t)__cvta_generic_to_shared(stage_flags(st) + fdst), flags + pz_0 + moff);
                }
            }
            cp_commit();
        };

        // sigma of node (lx, ly); for own nodes also the local part of lambda_t
        // (in mu) and the dL/dG term
        auto node = [&](int st, int lx, int ly, int x, int y, int z, float (&mu)[2][Q], bool& solid,
                        float& dG) -> Sig {
            Sig sg = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
            dG = 0.f;
            uint32_t fl = 0;
            solid = false;
            if constexpr (MASK) {
                fl = stage_flags(st)[(ly + 1) * kMBW + lx + kMPAD];
                solid = (fl & kSolid) != 0u;
                if (solid) return sg;
            }
            const float* row = stage_base(st) + (ly + 1) * kROW;
            const float* nb = row + (lx + kLPAD) * 2;
            static_for<0, Q>([&](auto II) {
                constexpr int i = decltype(II)::value;
                if constexpr (MASK && i != 0) {
                    if (fl & (1u << Vel<i>::opp)) {   // x + c_i solid: lambda_opp(i) at x
                        const size_t own = (size_t)x + (size_t)g.nx * ((size_t)y + (size_t)g.ny * z);
                        Store<float>::ld2(lam_in + pidx(0, Vel<i>::opp, (uint32_t)own), mu[0][i], mu[1][i]);
                        return;
                    }
                }
                Store<float>::lds2(nb + i * kLVS + 2 * Vel<i>::x, mu[0][i], mu[1][i]);
            });
            const float* mb = row + Q * kLVS + lx + kMPAD;
            float mo[kMom];
#pragma unroll
            for (int c = 0; c < kMom; ++c) mo[c] = mb[c * kMBW];
            float W[3], q[2];
            adj_node(mo, mu, p, W, q, sg.a, sg.b, dG);
            local_part(mu, p, W, q);
            return sg;
        };

        for (int e = 0; e < P.nst; ++e) issue(e);
        float cur[2][Q], nxt[2][Q];
        bool solid_cur = true;
        for (int e = 0; e < L; ++e) {
            cp_wait_n(P.nst - 1);
            __syncthreads();
            const int st = e % P.nst, slot = e & 3;
            const int z = plane_of(e);
            bool solid_nxt = true;
            if (own_row) {
                float dG;
                ring_at(slot, ty, tx) = node(st, tx, ty, gx, gy, z, nxt, solid_nxt, dG);
                // dL/dG of the own nodes of the chunk's planes (not of the halo planes)
                if (active && e >= 1 && e <= L - 2) dG_acc[0] += (double)dG;
            }
            if (has_halo) {
                float dh[2][Q], dGh;
                bool sh;
                ring_at(slot, hly, hlx) = node(st, hlx, hly, hgx, hgy, z, dh, sh, dGh);
            }
            __syncthreads();
            issue(e + P.nst);
            if (e >= 2 && active) {
                const int zc = plane_of(e - 1);
                const size_t own = (size_t)gx + (size_t)g.nx * ((size_t)gy + (size_t)g.ny * zc);
                float* out = lam_out + blk_base((uint32_t)own);
                if (solid_cur) {
#pragma unroll
                    for (int i = 0; i < Q; ++i) Store<float>::st2(out + i * (2 * kBlk), 0.f, 0.f);
                } else {
                    // h^k = sum_{i>=1} w_i c_i . sigma^k(x - c_i); x - c_i lies in
                    // plane (e - 1) - c_iz, i.e. ring slot e - 1 - c_iz
                    float h[2] = {0.f, 0.f};
                    static_for<1, Q>([&](auto II) {
                        constexpr int i = decltype(II)::value;
                        const int s2 = (e - 1 - Vel<i>::z) & 3;
                        const Sig& sg = ring_at(s2, ty - Vel<i>::y, tx - Vel<i>::x);
                        float acA = 0.f, acB = 0.f;
                        if constexpr (Vel<i>::x != 0) { acA += Vel<i>::x * sg.a[0]; acB += Vel<i>::x * sg.b[0]; }
                        if constexpr (Vel<i>::y != 0) { acA += Vel<i>::y * sg.a[1]; acB += Vel<i>::y * sg.b[1]; }
                        if constexpr (Vel<i>::z != 0) { acA += Vel<i>::z * sg.a[2]; acB += Vel<i>::z * sg.b[2]; }
                        h[0] += wgt<i>() * acA;
                        h[1] += wgt<i>() * acB;
                    });
                    static_for<0, Q>([&](auto II) {
                        constexpr int i = decltype(II)::value;
                        Store<float>::st2(out + i * (2 * kBlk), cur[0][i] + h[0], cur[1][i] + h[1]);
                    });
                }
            }
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int i = 0; i < Q; ++i) cur[k][i] = nxt[k][i];
            solid_cur = solid_nxt;
        }
        cp_wait<0>();
    }
    block_sum_store(dG_acc, partials + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * kRedVals);
}

// lambda_T^k_i(x) = dL/drho^k(x) at fluid nodes.
__global__ void adj_seed(const float* __restrict__ dLA, const float* __restrict__ dLB,
                         const uint32_t* __restrict__ flags, float* __restrict__ lam, Geom g) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.N) return;
    const bool fluid = !(flags && (flags[s] & kSolid));
    const float a = (fluid && dLA) ? dLA[s] : 0.f;
    const float b = (fluid && dLB) ? dLB[s] : 0.f;
    float* out = lam + blk_base((uint32_t)s);
    for (int i = 0; i < Q; ++i) Store<float>::st2(out + i * (2 * kBlk), a, b);
}

// dL/drho^k_0(x) = sum_i w_i lambda_0^k_i(x) (f_0 = f^eq(rho^k_0, 0) = w_i rho^k_0).
__global__ void adj_final(const float* __restrict__ lam, const uint32_t* __restrict__ flags,
                          float* __restrict__ gA, float* __restrict__ gB, Geom g) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.N) return;
    const bool fluid = !(flags && (flags[s] & kSolid));
    float acc[2] = {0.f, 0.f};
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        float a, b;
        Store<float>::ld2(lam + pidx(0, i, (uint32_t)s), a, b);
        acc[0] += wgt<i>() * a;
        acc[1] += wgt<i>() * b;
    });
    if (gA) gA[s] = fluid ? acc[0] : 0.f;
    if (gB) gB[s] = fluid ? acc[1] : 0.f;
}

// acc += sum of the first value of nblk partial rows, in a fixed order.
__global__ void __launch_bounds__(256) adj_accumulate(const double* __restrict__ partials, int nblk,
                                                      double* __restrict__ acc) {
    double v[kRedVals] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) v[0] += partials[(size_t)b * kRedVals];
    __shared__ double out[kRedVals];
    block_sum_store(v, out);
    __syncthreads();
    if (threadIdx.x == 0) *acc += out[0];
}

}  // namespace

size_t adjoint_workspace_bytes(int nx, int ny, int nz, int K) {
    const size_t N = (size_t)nx * ny * nz;
    return 2 * a256(state_elems((long long)N) * 4) + a256((size_t)kAux * N * 4) +
           a256((size_t)K * mom_elems((long long)N) * 4) + 256;
}

AsyncPlan plan_adjoint_box(int nx, int ny, int nz, int sm_count, bool masked, size_t smem_limit) {
    AsyncPlan best{};
    best.box = 0;
    if (nx % 4 != 0) return best;   // 16-byte chunks of float rows
    smem_limit = smem_limit > 4096 ? smem_limit - 4096 : 0;   // room for static shared memory
    double best_cost = 1e300;
    const int ncols = (nx + kTX - 1) / kTX;
    for (int R = (ny + kAdjMaxTY - 1) / kAdjMaxTY; R <= ny; ++R) {
        const int tymax = (ny + R - 1) / R;
        const int RH = tymax + 2;
        const int threads = kTX * tymax;
        if (threads < 2 * (kTX + 2) + 2 * tymax) continue;   // a thread per halo node
        if (threads < RH * kLCPR) continue;                    // a thread per chunk position
        const size_t stage = (size_t)RH * kROW * 4 + (masked ? (size_t)RH * kMBW * 4 : 0);
        const size_t ring = (size_t)4 * RH * (kTX + 2) * sizeof(float) * 6;
        if (smem_limit < ring + 2 * stage) continue;
        int nst = (int)((smem_limit - ring) / stage);
        nst = nst > 4 ? 4 : nst;
        const long long bxy = (long long)ncols * R;
        const int zs_max = nz / 4 > 1 ? nz / 4 : 1;
        for (int zs = 1; zs <= zs_max; ++zs) {
            const int zchunk = (nz + zs - 1) / zs;
            const long long blocks = bxy * zs;
            if (blocks > kRedBlocks) break;   // one partial row per block
            const long long waves = (blocks + sm_count - 1) / sm_count;
            const double work = (tymax + 0.6 * (2.0 * (kTX + 2) + 2.0 * tymax) / kTX) * (zchunk + 2);
            const double cost = waves * work * (1.0 + 4.0 / tymax);
            if (cost < best_cost * (1 - 1e-9)) {
                best_cost = cost;
                best = AsyncPlan{ncols, R, tymax, zs, zchunk, nst, threads, 0, ring + (size_t)nst * stage, 1};
            }
            if (blocks >= sm_count) break;
        }
    }
    return best;
}

cudaError_t run_adjoint(const AdjointRun& R, const float* dLA, const float* dLB, float* gA, float* gB,
                        double* gG, cudaStream_t st) {
    const size_t N = (size_t)R.g.N;
    const unsigned nb = (unsigned)((N + 255) / 256);
    const bool mask = R.flags != nullptr;
    const bool box = R.adjplan.box != 0;
    AdjBufs B = carve(R.adj, N, R.K);
    cudaError_t e;
    if (box) {
        // dynamic shared memory of this plan (the kernel also holds a small
        // static FP64 reduction buffer, which the plan's limit leaves room for)
        static size_t configured[2] = {0, 0};
        if (configured[mask] < R.adjplan.smem) {
            e = mask ? cudaFuncSetAttribute(adj_box_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)R.adjplan.smem)
                     : cudaFuncSetAttribute(adj_box_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)R.adjplan.smem);
            if (e != cudaSuccess) return e;
            configured[mask] = R.adjplan.smem;
        }
    }
    adj_seed<<<nb, 256, 0, st>>>(dLA, dLB, R.flags, B.lam[0], R.g);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(B.gacc, 0, sizeof(double), st)) != cudaSuccess) return e;
    int cur = 0;
    const long long T = R.steps;
    const long long M = (T + R.K - 1) / R.K;
    StepLaunch S;
    S.prec = R.prec;
    S.kernel = R.kernel;
    S.flags = R.flags;
    S.rho = R.rho;
    S.g = R.g;
    S.p = R.p;
    S.zsplit = R.zsplit;
    S.plan = R.plan;
    S.links = R.links;
    const AsyncPlan& AP = R.adjplan;
    const int adj_blocks = AP.ncols * AP.R * AP.zsplit;
    for (long long m = M - 1; m >= 0; --m) {
        const int Lm = (int)((T - m * R.K) < R.K ? (T - m * R.K) : R.K);
        if ((e = cudaMemcpyAsync(R.seg, R.ckpt + (size_t)m * R.state_bytes, R.state_bytes,
                                 cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
            return e;
        // recompute the segment: states seg[0..Lm-1] and their per-node moments
        for (int s = 0; s < Lm; ++s) {
            S.src = R.seg + (size_t)s * R.state_bytes;
            S.dst = (s + 1 < Lm) ? (void*)(R.seg + (size_t)(s + 1) * R.state_bytes) : R.scratch;
            S.mom_out = B.segmom + (size_t)s * mom_elems((long long)N);
            if ((e = launch_step(S, st)) != cudaSuccess) return e;
        }
        // reverse through it
        for (int s = Lm - 1; s >= 0; --s) {
            const float* mom = B.segmom + (size_t)s * mom_elems((long long)N);
            if (box) {
                dim3 grid(AP.ncols * AP.R, AP.zsplit, 1);
                if (mask)
                    adj_box_kernel<true><<<grid, AP.threads, AP.smem, st>>>(B.lam[cur], mom, R.flags, B.lam[1 - cur],
                                                                           R.red_part, R.g, R.p, AP);
                else
                    adj_box_kernel<false><<<grid, AP.threads, AP.smem, st>>>(B.lam[cur], mom, R.flags,
                                                                            B.lam[1 - cur], R.red_part, R.g, R.p, AP);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
                adj_accumulate<<<1, 256, 0, st>>>(R.red_part, adj_blocks, B.gacc);
            } else {
                if (mask)
                    adj_pass_a<true><<<kRedBlocks, 256, 0, st>>>(mom, B.lam[cur], R.flags, B.aux, R.red_part, R.g, R.p);
                else
                    adj_pass_a<false><<<kRedBlocks, 256, 0, st>>>(mom, B.lam[cur], R.flags, B.aux, R.red_part, R.g,
                                                                  R.p);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
                adj_accumulate<<<1, 256, 0, st>>>(R.red_part, kRedBlocks, B.gacc);
                if (mask)
                    adj_pass_b<true><<<nb, 256, 0, st>>>(B.lam[cur], B.aux, R.flags, B.lam[1 - cur], R.g, R.p);
                else
                    adj_pass_b<false><<<nb, 256, 0, st>>>(B.lam[cur], B.aux, R.flags, B.lam[1 - cur], R.g, R.p);
            }
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            cur ^= 1;
        }
    }
    if (gA || gB) {
        adj_final<<<nb, 256, 0, st>>>(B.lam[cur], R.flags, gA, gB, R.g);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = cudaMemcpyAsync(gG, B.gacc, sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

}  // namespace lbgb
