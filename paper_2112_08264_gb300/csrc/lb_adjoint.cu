// lb_adjoint.cu -- reverse-mode step with checkpoint recompute (derivation in
// adjoint.h).
//
// Backward over a recorded run of T steps with checkpoints every K steps:
// for each segment, last to first, the forward step is re-run from its
// checkpoint (the same kernel, so the same bits), keeping every state of the
// segment and its density deviations; the adjoint then runs backwards through
// the segment, two passes per step:
//   pass A (per node): pull f_t, gather mu = P^T lambda_{t+1}, force sums from
//           the stored densities; write W, q_k, sigma^k and a per-block FP64
//           partial of dL/dG;
//   pass B (per node): gather mu again, add the neighbour gather of sigma,
//           write lambda_t.
#include <cuda_runtime.h>

#include "adjoint.h"
#include "kernels.h"
#include "reduce.cuh"

namespace lbgb {

namespace {

constexpr int kAux = 11;   // W[3], q[2], sigma^A[3], sigma^B[3]

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct AdjBufs {
    float* lam[2];
    float* aux;
    float* segrho;
    double* gacc;
};

AdjBufs carve(char* adj, size_t N, int K) {
    AdjBufs b;
    size_t off = 0;
    b.lam[0] = reinterpret_cast<float*>(adj + off); off += a256(2 * Q * N * 4);
    b.lam[1] = reinterpret_cast<float*>(adj + off); off += a256(2 * Q * N * 4);
    b.aux = reinterpret_cast<float*>(adj + off); off += a256((size_t)kAux * N * 4);
    b.segrho = reinterpret_cast<float*>(adj + off); off += a256((size_t)K * 2 * N * 4);
    b.gacc = reinterpret_cast<double*>(adj + off);
    return b;
}

__device__ __forceinline__ void site_xyz(long long s, const Geom& g, int& x, int& y, int& z) {
    x = (int)(s % g.nx);
    y = (int)((s / g.nx) % g.ny);
    z = (int)(s / g.plane);
}

// mu_i(x) = lambda_i(x + c_i) if x + c_i is fluid, else lambda_opp(i)(x)
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
#pragma unroll
        for (int k = 0; k < 2; ++k) mu[k][i] = __ldg(lam + (size_t)(k * Q + pop) * g.N + t);
    });
}

// Force sums S^k from stored density deviations (neighbours of node x).
__device__ __forceinline__ void force_sums(const float* __restrict__ dpsi, const Geom& g, int x, int y, int z,
                                           float (&SA)[3], float (&SB)[3]) {
    neighbour_sums(
        [&](int dx, int dy, int dz) {
            const int xx = dx > 0 ? wrap_inc(x, g.nx) : (dx < 0 ? wrap_dec(x, g.nx) : x);
            const int yy = dy > 0 ? wrap_inc(y, g.ny) : (dy < 0 ? wrap_dec(y, g.ny) : y);
            const int zz = dz > 0 ? wrap_inc(z, g.nz) : (dz < 0 ? wrap_dec(z, g.nz) : z);
            const long long t = xx + (long long)g.nx * (yy + (long long)g.ny * zz);
            return make_float2(__ldg(dpsi + t), __ldg(dpsi + g.N + t));
        },
        SA, SB);
}

// Per-node adjoint quantities of the collision (see adjoint.h).
__device__ __forceinline__ void adj_node(const float (&d)[2][Q], const float (&mu)[2][Q], const Phys& p,
                                         const float (&SA)[3], const float (&SB)[3], float (&W)[3],
                                         float (&q)[2], float (&sA)[3], float (&sB)[3], float& dG) {
    float dA, dB, j[3];
    sums(d, dA, dB, j);
    const float rA = p.rho0[0] + dA, rB = p.rho0[1] + dB;
    const float inv = 1.0f / (rA + rB);
    const float up[3] = {j[0] * inv, j[1] * inv, j[2] * inv};
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

template <typename S, bool MASK>
__global__ void __launch_bounds__(256)
adj_pass_a(const S* __restrict__ gt, const float* __restrict__ dpsi, const float* __restrict__ lam,
           const uint32_t* __restrict__ flags, float* __restrict__ aux, double* __restrict__ partials, Geom g,
           Phys p) {
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
        PullIdx P;
        pull_indices(g, x, y, z, P);
        float d[2][Q], mu[2][Q];
        pull<S, MASK>(gt, g, P, fl, d);
        gather_mu<MASK>(lam, g, x, y, z, s, fl, mu);
        float SA[3], SB[3];
        force_sums(dpsi, g, x, y, z, SA, SB);
        float W[3], q[2], sA[3], sB[3], dG;
        adj_node(d, mu, p, SA, SB, W, q, sA, sB, dG);
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
    if (fl & kSolid) {
        for (int j = 0; j < 2 * Q; ++j) lam_out[(size_t)j * g.N + s] = 0.f;
        return;
    }
    float mu[2][Q];
    gather_mu<MASK>(lam_in, g, x, y, z, s, fl, mu);
    const float W[3] = {aux[s], aux[g.N + s], aux[2 * g.N + s]};
    const float q[2] = {aux[3 * g.N + s], aux[4 * g.N + s]};
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
        float cW = 0.f;
        if constexpr (Vel<i>::x != 0) cW += Vel<i>::x * W[0];
        if constexpr (Vel<i>::y != 0) cW += Vel<i>::y * W[1];
        if constexpr (Vel<i>::z != 0) cW += Vel<i>::z * W[2];
#pragma unroll
        for (int k = 0; k < 2; ++k)
            lam_out[(size_t)(k * Q + i) * g.N + s] = (1.0f - p.omega) * mu[k][i] + cW + q[k] + h[k];
    });
}

// lambda_T^k_i(x) = dL/drho^k(x) at fluid nodes.
__global__ void adj_seed(const float* __restrict__ dLA, const float* __restrict__ dLB,
                         const uint32_t* __restrict__ flags, float* __restrict__ lam, Geom g) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.N) return;
    const bool fluid = !(flags && (flags[s] & kSolid));
    const float a = (fluid && dLA) ? dLA[s] : 0.f;
    const float b = (fluid && dLB) ? dLB[s] : 0.f;
    for (int i = 0; i < Q; ++i) {
        lam[(size_t)i * g.N + s] = a;
        lam[(size_t)(Q + i) * g.N + s] = b;
    }
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
#pragma unroll
        for (int k = 0; k < 2; ++k) acc[k] += wgt<i>() * lam[(size_t)(k * Q + i) * g.N + s];
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

template <typename S>
cudaError_t pass_a(bool mask, const void* gt, const float* dpsi, const float* lam, const uint32_t* flags,
                   float* aux, double* partials, const Geom& g, const Phys& p, cudaStream_t st) {
    if (mask)
        adj_pass_a<S, true><<<kRedBlocks, 256, 0, st>>>((const S*)gt, dpsi, lam, flags, aux, partials, g, p);
    else
        adj_pass_a<S, false><<<kRedBlocks, 256, 0, st>>>((const S*)gt, dpsi, lam, flags, aux, partials, g, p);
    return cudaGetLastError();
}

}  // namespace

size_t adjoint_workspace_bytes(int nx, int ny, int nz, int K) {
    const size_t N = (size_t)nx * ny * nz;
    return 2 * a256(2 * Q * N * 4) + a256((size_t)kAux * N * 4) + a256((size_t)K * 2 * N * 4) + 256;
}

cudaError_t run_adjoint(const AdjointRun& R, const float* dLA, const float* dLB, float* gA, float* gB,
                        double* gG, cudaStream_t st) {
    const size_t N = (size_t)R.g.N;
    const unsigned nb = (unsigned)((N + 255) / 256);
    const bool mask = R.flags != nullptr;
    AdjBufs B = carve(R.adj, N, R.K);
    cudaError_t e;
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
    for (long long m = M - 1; m >= 0; --m) {
        const int Lm = (int)((T - m * R.K) < R.K ? (T - m * R.K) : R.K);
        if ((e = cudaMemcpyAsync(R.seg, R.ckpt + (size_t)m * R.state_bytes, R.state_bytes,
                                 cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
            return e;
        // recompute the segment: states seg[0..Lm-1] and their density deviations
        for (int s = 0; s < Lm; ++s) {
            S.src = R.seg + (size_t)s * R.state_bytes;
            S.dst = (s + 1 < Lm) ? (void*)(R.seg + (size_t)(s + 1) * R.state_bytes) : R.scratch;
            S.rho_out = B.segrho + (size_t)s * 2 * N;
            if ((e = launch_step(S, st)) != cudaSuccess) return e;
        }
        // reverse through it
        for (int s = Lm - 1; s >= 0; --s) {
            const void* gt = R.seg + (size_t)s * R.state_bytes;
            const float* dpsi = B.segrho + (size_t)s * 2 * N;
            switch (R.prec) {
                case 0: e = pass_a<float>(mask, gt, dpsi, B.lam[cur], R.flags, B.aux, R.red_part, R.g, R.p, st); break;
                case 1: e = pass_a<__half>(mask, gt, dpsi, B.lam[cur], R.flags, B.aux, R.red_part, R.g, R.p, st); break;
                case 2:
                    e = pass_a<__nv_bfloat16>(mask, gt, dpsi, B.lam[cur], R.flags, B.aux, R.red_part, R.g, R.p, st);
                    break;
                default: return cudaErrorInvalidValue;
            }
            if (e != cudaSuccess) return e;
            adj_accumulate<<<1, 256, 0, st>>>(R.red_part, kRedBlocks, B.gacc);
            if (mask)
                adj_pass_b<true><<<nb, 256, 0, st>>>(B.lam[cur], B.aux, R.flags, B.lam[1 - cur], R.g, R.p);
            else
                adj_pass_b<false><<<nb, 256, 0, st>>>(B.lam[cur], B.aux, R.flags, B.lam[1 - cur], R.g, R.p);
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
