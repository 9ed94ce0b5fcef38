// lb_particles.cu -- moving rigid spheres (Sec. 2): moving-wall halfway
// bounce-back at the links into a sphere (Eq. UPI, Eq. LADDFLBE), the
// momentum those links exchange summed in FP64 into each sphere's force and
// torque (Eq. FORCEPP, Eq. FORCEPARTEQ, Eq. TORQUEPARTEQ), the leap-frog
// update of Eq. PARDYN, and re-meshing of the nodes a moved sphere leaves or
// reaches (the rule conserves the total momentum of fluid and spheres).
//
// One block per sphere walks the cube of sites around its centre (half-width
// ceil(R) + 2: every covered node, every fluid node linked to one, and every
// node covered one step earlier by a sphere moving at most one node per
// step). Each thread accumulates its sites in a fixed order and the block
// reduces in a fixed tree, so forces and torques are deterministic. The
// coverage test and the position update use separately rounded FP64
// operations, so they decide exactly as plain IEEE evaluation does.
#include <cmath>
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace lbgb {
namespace {

constexpr int kPT = 256;   // threads per sphere block

__device__ __forceinline__ int wrapn(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

// minimum-image displacement along one axis of period n
__device__ __forceinline__ double min_image(double d, int n) {
    return __dsub_rn(d, __dmul_rn((double)n, rint(__ddiv_rn(d, (double)n))));
}

__device__ __forceinline__ double norm2(double a, double b, double c) {
    return __dadd_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)), __dmul_rn(c, c));
}

// The cube of sites of one sphere: site b of side^3 at unwrapped coordinates
// lo + (bx, by, bz).
struct Cube {
    int lo[3];
    int side;
    __device__ Cube(const double* c, int half) {
        side = 2 * half + 1;
#pragma unroll
        for (int a = 0; a < 3; ++a) lo[a] = (int)floor(c[a]) - half;
    }
    __device__ int count() const { return side * side * side; }
    // site b as wrapped grid coordinates
    __device__ void at(int b, const Geom& g, int (&u)[3]) const {
        u[0] = wrapn(lo[0] + b % side, g.nx);
        u[1] = wrapn(lo[1] + (b / side) % side, g.ny);
        u[2] = wrapn(lo[2] + b / (side * side), g.nz);
    }
};

__device__ __forceinline__ uint32_t site_of(const int (&u)[3], const Geom& g) {
    return (uint32_t)wrapn(u[0], g.nx) + (uint32_t)g.nx * ((uint32_t)wrapn(u[1], g.ny) +
                                                          (uint32_t)g.ny * (uint32_t)wrapn(u[2], g.nz));
}

__device__ __forceinline__ void cross(const double (&a)[3], const double (&b)[3], double (&o)[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// Fixed-tree block sum of NV doubles per thread; thread 0 gets the totals.
template <int NV>
__device__ void block_sum(double (&v)[NV]) {
    __shared__ double red[NV][kPT];
#pragma unroll
    for (int k = 0; k < NV; ++k) red[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int h = kPT / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
#pragma unroll
            for (int k = 0; k < NV; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + h];
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = red[k][0];
}

__device__ __forceinline__ void load3(const double* a, int q, double (&o)[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) o[k] = a[3 * q + k];
}

// Links from fluid nodes into sphere q: slot opp(i) of the covered node
// x + c_i takes g_i(x) - 2 rho0^k w_i (u_b . c_i) / c_s^2, and the link adds
// c_i sum_k (2 g_i^k(x) - 2 rho0^k w_i (u_b . c_i) / c_s^2) to the force and
// (r_b - r) x that to the torque.
template <typename S>
__global__ void __launch_bounds__(kPT) sphere_links_kernel(S* __restrict__ st, const uint32_t* __restrict__ flags,
                                                          Spheres A, int forces, Geom g, Phys p) {
    const int q = blockIdx.x;
    double c[3], v[3], w[3];
    load3(A.r, q, c);
    load3(A.v, q, v);
    load3(A.w, q, w);
    const Cube cube(c, A.half);
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < cube.count(); b += kPT) {
        int u[3];
        cube.at(b, g, u);
        const uint32_t s = site_of(u, g);
        const uint32_t fl = __ldg(flags + s);
        if ((fl & kSolid) || !(fl & kNbSolidMask)) continue;
        static_for<1, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            if (!(fl & (1u << Vel<i>::opp))) return;   // x + c_i is fluid
            const int t3[3] = {u[0] + Vel<i>::x, u[1] + Vel<i>::y, u[2] + Vel<i>::z};
            const uint32_t t = site_of(t3, g);
            if (A.owner[t] != q + 1) return;
            const double arm[3] = {min_image(((double)u[0] + 0.5 * Vel<i>::x) - c[0], g.nx),
                                   min_image(((double)u[1] + 0.5 * Vel<i>::y) - c[1], g.ny),
                                   min_image(((double)u[2] + 0.5 * Vel<i>::z) - c[2], g.nz)};
            double wa[3];
            cross(w, arm, wa);
            const double cu = 3.0 * (Vel<i>::x * (v[0] + wa[0]) + Vel<i>::y * (v[1] + wa[1]) +
                                     Vel<i>::z * (v[2] + wa[2]));
            float dA, dB;
            Store<S>::ld2(st + pidx(0, i, s), dA, dB);
            const double bA = 2.0 * (double)p.rho0[0] * wgt_d<i>() * cu;
            const double bB = 2.0 * (double)p.rho0[1] * wgt_d<i>() * cu;
            Store<S>::st2(st + pidx(0, Vel<i>::opp, t), dA - (float)bA, dB - (float)bB);
            if (!forces) return;
            const double ex = 2.0 * ((double)dA + wgt_d<i>() * (double)p.rho0[0]) - bA +
                              2.0 * ((double)dB + wgt_d<i>() * (double)p.rho0[1]) - bB;
            const double F[3] = {Vel<i>::x * ex, Vel<i>::y * ex, Vel<i>::z * ex};
            double Tq[3];
            cross(arm, F, Tq);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                acc[a] += F[a];
                acc[3 + a] += Tq[a];
            }
        });
    }
    if (!forces) return;
    block_sum(acc);
    if (threadIdx.x == 0)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            A.F[3 * q + a] = acc[a];
            A.T[3 * q + a] = acc[3 + a];
        }
}

// Leap-frog: v += F / m, r += v (wrapped into the box), w += T / I.
__global__ void sphere_update_kernel(Spheres A, Geom g) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= A.n || !(A.mass > 0.0)) return;
    const int n[3] = {g.nx, g.ny, g.nz};
    bool fast = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double v = __dadd_rn(A.v[3 * q + a], __ddiv_rn(A.F[3 * q + a], A.mass));
        double r = __dadd_rn(A.r[3 * q + a], v);
        // r mod n (the remainder of an exact division, then into [0, n))
        const double m = fmod(r, (double)n[a]);
        r = m < 0.0 ? __dadd_rn(m, (double)n[a]) : m;
        A.v[3 * q + a] = v;
        A.r[3 * q + a] = r;
        A.w[3 * q + a] = __dadd_rn(A.w[3 * q + a], __ddiv_rn(A.T[3 * q + a], A.inertia));
        fast = fast || fabs(v) > 1.0;
    }
    if (fast) atomicOr(A.err, 2);
}

// Re-meshing, first pass: nodes sphere q covered and no longer covers become
// fluid with f^eq(rho0^k, u_b) at the wall velocity there; the sphere loses
// that momentum (and its moment).
template <typename S>
__global__ void __launch_bounds__(kPT) sphere_uncover_kernel(S* __restrict__ st, Spheres A, Geom g, Phys p) {
    const int q = blockIdx.x;
    double c[3], v[3], w[3];
    load3(A.r, q, c);
    load3(A.v, q, v);
    load3(A.w, q, w);
    const Cube cube(c, A.half);
    const double R2 = __dmul_rn(A.radius, A.radius);
    const double r0 = (double)p.rho0[0] + (double)p.rho0[1];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < cube.count(); b += kPT) {
        int u[3];
        cube.at(b, g, u);
        const uint32_t s = site_of(u, g);
        if (A.owner[s] != q + 1) continue;
        const double arm[3] = {min_image((double)u[0] - c[0], g.nx), min_image((double)u[1] - c[1], g.ny),
                               min_image((double)u[2] - c[2], g.nz)};
        if (norm2(arm[0], arm[1], arm[2]) <= R2) continue;   // still covered
        A.owner[s] = 0;
        double ub[3];
        cross(w, arm, ub);
#pragma unroll
        for (int a = 0; a < 3; ++a) ub[a] += v[a];
        const float ux = (float)ub[0], uy = (float)ub[1], uz = (float)ub[2];
        const float uu = ux * ux + uy * uy + uz * uz;
        static_for<0, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            const float cu = Vel<i>::x * ux + Vel<i>::y * uy + Vel<i>::z * uz;
            const float e = cu * (3.0f + 4.5f * cu) - 1.5f * uu;
            Store<S>::st2(st + pidx(0, i, s), wgt<i>() * p.rho0[0] * e, wgt<i>() * p.rho0[1] * e);
        });
        double L[3];
        cross(arm, ub, L);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            acc[a] -= r0 * ub[a];
            acc[3 + a] -= r0 * L[a];
        }
    }
    block_sum(acc);
    if (threadIdx.x == 0 && A.mass > 0.0)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            A.v[3 * q + a] += acc[a] / A.mass;
            A.w[3 * q + a] += acc[3 + a] / A.inertia;
        }
}

// Re-meshing, second pass (and placement when !absorb): nodes sphere q now
// covers and did not take its fluid's momentum (and moment); their
// populations are cleared. A node held by another sphere or by the mask is
// an error.
template <typename S>
__global__ void __launch_bounds__(kPT) sphere_cover_kernel(S* __restrict__ st, const uint8_t* __restrict__ mask,
                                                          Spheres A, int absorb, Geom g) {
    const int q = blockIdx.x;
    double c[3];
    load3(A.r, q, c);
    const Cube cube(c, A.half);
    const double R2 = __dmul_rn(A.radius, A.radius);
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < cube.count(); b += kPT) {
        int u[3];
        cube.at(b, g, u);
        const uint32_t s = site_of(u, g);
        const double arm[3] = {min_image((double)u[0] - c[0], g.nx), min_image((double)u[1] - c[1], g.ny),
                               min_image((double)u[2] - c[2], g.nz)};
        if (norm2(arm[0], arm[1], arm[2]) > R2) continue;
        if (A.owner[s] == q + 1) continue;   // covered before
        if ((mask && mask[s]) || atomicCAS(A.owner + s, 0, q + 1) != 0) {
            atomicOr(A.err, 1);
            continue;
        }
        if (!absorb) continue;
        double m[3] = {0, 0, 0};
        static_for<1, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            float dA, dB;
            Store<S>::ld2(st + pidx(0, i, s), dA, dB);
            const double d = (double)dA + (double)dB;   // sum_i c_i w_i rho0 = 0
            m[0] += Vel<i>::x * d;
            m[1] += Vel<i>::y * d;
            m[2] += Vel<i>::z * d;
        });
        static_for<0, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            Store<S>::st2(st + pidx(0, i, s), 0.f, 0.f);
        });
        double L[3];
        cross(arm, m, L);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            acc[a] += m[a];
            acc[3 + a] += L[a];
        }
    }
    if (!absorb) return;
    block_sum(acc);
    if (threadIdx.x == 0 && A.mass > 0.0)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            A.v[3 * q + a] += acc[a] / A.mass;
            A.w[3 * q + a] += acc[3 + a] / A.inertia;
        }
}

// Solid flags (bit 0 solid, bit i: x - c_i solid) from the mask and the
// coverage: over the cube of every sphere widened by one (all sites whose
// flags a re-meshing can change), or over the whole grid when whole != 0.
__global__ void sphere_flags_kernel(uint32_t* __restrict__ flags, const uint8_t* __restrict__ mask, Spheres A,
                                    int whole, Geom g) {
    auto solid = [&](uint32_t s) { return (mask && mask[s]) || A.owner[s] != 0; };
    auto one = [&](int x, int y, int z) {
        PullIdx P;
        pull_indices(g, x, y, z, P);
        uint32_t f = solid((uint32_t)P.own) ? kSolid : 0u;
        static_for<1, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            if (solid((uint32_t)P.src[i])) f |= (1u << i);
        });
        flags[P.own] = f;
    };
    if (whole) {
        const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        if (s >= g.N) return;
        one((int)(s % g.nx), (int)((s / g.nx) % g.ny), (int)(s / g.plane));
        return;
    }
    const int q = blockIdx.x;
    double c[3];
    load3(A.r, q, c);
    const Cube cube(c, A.half + 1);
    for (int b = threadIdx.x; b < cube.count(); b += kPT) {
        int u[3];
        cube.at(b, g, u);
        one(u[0], u[1], u[2]);
    }
}

template <typename F32, typename F16, typename BF16>
cudaError_t by_prec(int prec, F32&& a, F16&& b, BF16&& c) {
    switch (prec) {
        case 0: a(); break;
        case 1: b(); break;
        case 2: c(); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sphere_links(int prec, void* state, const uint32_t* flags, const Spheres& S, bool forces,
                                const Geom& g, const Phys& p, cudaStream_t st) {
    if (S.n == 0) return cudaSuccess;
#define LBGB_LINKS(T) [&] { sphere_links_kernel<T><<<S.n, kPT, 0, st>>>((T*)state, flags, S, forces ? 1 : 0, g, p); }
    return by_prec(prec, LBGB_LINKS(float), LBGB_LINKS(__half), LBGB_LINKS(__nv_bfloat16));
#undef LBGB_LINKS
}

cudaError_t launch_sphere_move(int prec, void* state, uint32_t* flags, const uint8_t* mask, const Spheres& S,
                               const Geom& g, const Phys& p, cudaStream_t st) {
    if (S.n == 0 || !(S.mass > 0.0)) return cudaSuccess;   // fixed spheres never move
    sphere_update_kernel<<<(S.n + 127) / 128, 128, 0, st>>>(S, g);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
#define LBGB_MOVE(T)                                                                  \
    [&] {                                                                             \
        sphere_uncover_kernel<T><<<S.n, kPT, 0, st>>>((T*)state, S, g, p);            \
        sphere_cover_kernel<T><<<S.n, kPT, 0, st>>>((T*)state, mask, S, 1, g);        \
    }
    if ((e = by_prec(prec, LBGB_MOVE(float), LBGB_MOVE(__half), LBGB_MOVE(__nv_bfloat16))) != cudaSuccess) return e;
#undef LBGB_MOVE
    sphere_flags_kernel<<<S.n, kPT, 0, st>>>(flags, mask, S, 0, g);
    return cudaGetLastError();
}

cudaError_t launch_sphere_place(uint32_t* flags, const uint8_t* mask, const Spheres& S, const Geom& g,
                                cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(S.owner, 0, (size_t)g.N * sizeof(int), st);
    if (e != cudaSuccess) return e;
    if (S.n > 0) {
        sphere_cover_kernel<float><<<S.n, kPT, 0, st>>>(nullptr, mask, S, 0, g);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    sphere_flags_kernel<<<(unsigned)((g.N + 255) / 256), 256, 0, st>>>(flags, mask, S, 1, g);
    return cudaGetLastError();
}

}  // namespace lbgb
