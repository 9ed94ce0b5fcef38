// common.cuh -- per-site building blocks shared by the step, moment and
// reduction kernels.
//
// State in device memory: the POST-COLLISION populations g of the last step,
// stored as deviations d = g - w_i rho0^k in blocked SoA order (pidx below).
// One step is then a pull
// (Sec. 3 one-step two-grid scheme, two buffers, read one / write the other):
//   f_i(x) = g_i(x - c_i)         if x - c_i is fluid   (streaming, Eq. bgk)
//   f_i(x) = g_opp(i)(x)          if x - c_i is solid   (halfway bounce-back at
//                                                        rest, Eq. LADDFLBE)
// followed by densities, the Shan-Chen force, the velocity shift and BGK
// collision (Eq. bgk, Eq. LEQ), and a store of g(x).
#pragma once
#include <cstdint>
#include "lattice.cuh"
#include "store.cuh"
#include "vec2.cuh"

namespace lbgb {

struct Geom {
    int nx, ny, nz;
    int plane;       // nx * ny
    long long N;     // sites, s = x + nx (y + ny z)
};

// Blocked SoA storage: the site index s is cut into blocks of kBlk
// consecutive sites; a block holds velocity 0 of its sites, then velocity 1,
// ..., each as kBlk (A, B) component pairs, so that
//   element(k, i, s) = block(s) + i * 2 kBlk + 2 (s mod kBlk) + k.
// A warp's access to one velocity of 32 consecutive sites is one contiguous
// segment, both components of a velocity move as one vector access (they
// stream along the same c_i), and the offset of velocity i within a block is
// the constant i * 2 kBlk, so the 19 accesses of a node share one address
// and differ by immediates. Site indices are below 2^31 (checked at context
// creation): the split is an unsigned 32-bit shift and mask.
constexpr int kBlk = 64;
static_assert((kBlk & (kBlk - 1)) == 0, "kBlk must be a power of two");
__host__ __device__ __forceinline__ size_t blk_base(uint32_t s) {
    return (size_t)(s / (uint32_t)kBlk) * (size_t)(2 * Q * kBlk) + 2 * (size_t)(s % (uint32_t)kBlk);
}
__host__ __device__ __forceinline__ size_t pidx(int k, int i, uint32_t s) {
    return blk_base(s) + (size_t)i * (2 * kBlk) + (size_t)k;
}
// elements of one state (the last block is padded)
__host__ __device__ __forceinline__ size_t state_elems(long long N) {
    return (size_t)((N + kBlk - 1) / kBlk) * (size_t)(2 * Q * kBlk);
}

struct Phys {
    float tau;       // relaxation time
    float omega;     // 1 / tau
    float G;         // Shan-Chen coupling
    float g[3];      // body force
    float rho0[2];   // deviation base of components A, B
    int model;       // 0 Shan-Chen, 1 colour gradient
    float cg_inu[2]; // colour gradient: 1 / nu of the pure components
    float cg_sigma;  // colour gradient: surface tension
    float cg_beta;   // colour gradient: recolouring parameter
    int slots;       // state readers: 1 = every solid slot a fluid node pulls is written (pull it as is)
};

// solid-site flags: bit 0 = this node is solid; bit i (1..18) = node x - c_i
// is solid (so f_i(x) comes from bounce-back).
constexpr uint32_t kSolid = 1u;
// bits 1..Q-1: the pull source x - c_i of population i is solid
constexpr uint32_t kNbSolidMask = ((1u << Q) - 1u) & ~1u;

__device__ __forceinline__ int wrap_dec(int a, int n) { return a == 0 ? n - 1 : a - 1; }
__device__ __forceinline__ int wrap_inc(int a, int n) { return a == n - 1 ? 0 : a + 1; }

// Node x + c_i (periodic) of node (x, y, z), as a site index.
template <int i>
__device__ __forceinline__ long long nb_index(const Geom& g, int x, int y, int z) {
    const int xx = Vel<i>::x > 0 ? wrap_inc(x, g.nx) : (Vel<i>::x < 0 ? wrap_dec(x, g.nx) : x);
    const int yy = Vel<i>::y > 0 ? wrap_inc(y, g.ny) : (Vel<i>::y < 0 ? wrap_dec(y, g.ny) : y);
    const int zz = Vel<i>::z > 0 ? wrap_inc(z, g.nz) : (Vel<i>::z < 0 ? wrap_dec(z, g.nz) : z);
    return xx + (long long)g.nx * (yy + (long long)g.ny * zz);
}

// Tiling of the box step kernel: strips of kTileX columns (ncols of them),
// R bands of rows (band c covers rows [c ny / R, (c + 1) ny / R)), and
// z-chunks of zchunk planes. R == 0: no tiling.
constexpr int kTileX = 32;
struct TileMap {
    int ncols = 0, R = 0, zchunk = 0;
};
// band of row y: the largest c with c ny / R <= y (integer division)
__host__ __device__ __forceinline__ int band_of(int y, int ny, int R) {
    return (int)(((long long)(y + 1) * R - 1) / ny);
}
__host__ __device__ __forceinline__ int band_start(int c, int ny, int R) {
    return (int)(((long long)c * ny) / R);
}

// Bounce-back links grouped by (tile, source plane): list (b, z) is
// ent[start[b nz + z], start[b nz + z + 1]). An entry packs the source node's
// place in its tile and the velocity: lx | ly << 5 | i << 9 (lx < 32,
// ly < 16, 1 <= i < Q).
struct LinkTiles {
    const uint32_t* start = nullptr;
    const uint16_t* ent = nullptr;
};
__host__ __device__ __forceinline__ uint16_t link_entry(int lx, int ly, int i) {
    return (uint16_t)(lx | (ly << 5) | (i << 9));
}

// c_i by component for a velocity known only at run time: two bits per
// velocity holding c + 1, packed from the Vel table.
template <int AX, int I = 0>
__host__ __device__ constexpr unsigned long long packed_axis() {
    if constexpr (I == Q) {
        return 0ull;
    } else {
        constexpr int c = AX == 0 ? Vel<I>::x : (AX == 1 ? Vel<I>::y : Vel<I>::z);
        return ((unsigned long long)(c + 1) << (2 * I)) | packed_axis<AX, I + 1>();
    }
}
template <int AX>
__host__ __device__ __forceinline__ int vel_c(int i) {
    return (int)((packed_axis<AX>() >> (2 * i)) & 3ull) - 1;
}
// opposite of a moving velocity (the public order pairs 1-2, 3-4, ..., 17-18)
__host__ __device__ __forceinline__ int vel_opp(int i) { return ((i - 1) ^ 1) + 1; }

// Element offsets (component A of the pair) of a tile link's two slots:
// velocity i at the source node (x0 + lx, y0 + ly, z) and velocity opp(i) at
// the solid node x + c_i (periodic in x and y; the builder keeps only links
// whose target plane lies inside the source's z-chunk).
struct LinkSlots {
    size_t src, dst;
};
__device__ __forceinline__ LinkSlots tile_link_slots(uint32_t e, int x0, int y0, int z, const Geom& g) {
    const int i = (int)(e >> 9);
    const int x = x0 + (int)(e & 31u), y = y0 + (int)((e >> 5) & 15u);
    int tx = x + vel_c<0>(i), ty = y + vel_c<1>(i);
    tx = tx < 0 ? tx + g.nx : (tx >= g.nx ? tx - g.nx : tx);
    ty = ty < 0 ? ty + g.ny : (ty >= g.ny ? ty - g.ny : ty);
    const int tz = z + vel_c<2>(i);
    const uint32_t s = (uint32_t)x + (uint32_t)g.nx * ((uint32_t)y + (uint32_t)g.ny * (uint32_t)z);
    const uint32_t t = (uint32_t)tx + (uint32_t)g.nx * ((uint32_t)ty + (uint32_t)g.ny * (uint32_t)tz);
    return {pidx(0, i, s), pidx(0, vel_opp(i), t)};
}

// Site indices of the pull sources x - c_i for the 19 velocities.
struct PullIdx {
    int own;
    int src[Q];
};

__device__ __forceinline__ void pull_indices(const Geom& g, int x, int y, int z, PullIdx& P) {
    const int xm = wrap_dec(x, g.nx), xp = wrap_inc(x, g.nx);
    const int ym = wrap_dec(y, g.ny), yp = wrap_inc(y, g.ny);
    const int zm = wrap_dec(z, g.nz), zp = wrap_inc(z, g.nz);
    P.own = x + g.nx * (y + g.ny * z);
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        // source = x - c_i
        const int sx = Vel<i>::x == 1 ? xm : (Vel<i>::x == -1 ? xp : x);
        const int sy = Vel<i>::y == 1 ? ym : (Vel<i>::y == -1 ? yp : y);
        const int sz = Vel<i>::z == 1 ? zm : (Vel<i>::z == -1 ? zp : z);
        P.src[i] = sx + g.nx * (sy + g.ny * sz);
    });
}

// Pull the 38 deviations of node P.own into d[k][i].
template <typename S, bool MASK>
__device__ __forceinline__ void pull(const S* __restrict__ src, const Geom& g, const PullIdx& P,
                                     uint32_t flags, float (&d)[2][Q]) {
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        int idx = P.src[i];
        int pop = i;
        if constexpr (MASK && i != 0) {
            if (flags & (1u << i)) { idx = P.own; pop = Vel<i>::opp; }
        }
        Store<S>::ld2(src + pidx(0, pop, idx), d[0][i], d[1][i]);
    });
}

// Density deviations drho^k = rho^k - rho0^k = sum_i d_i^k and momentum
// j = sum_k sum_i c_i d_i^k (sum_i c_i w_i rho0 = 0, so the deviations carry
// the whole momentum), in velocity order starting from d_0. The momentum is
// summed over opposite pairs, c_i (d_i - d_opp(i)), whose differences are
// exact when the two are close.
//
// Two forms. With 16-bit storage the node work is bound by instruction issue,
// and the sums take both components at once as (A, B) pairs with the packed
// FP32 instructions (a component's momentum is summed on its own and the two
// are added last). With FP32 storage (bound by memory bandwidth, and
// scheduled best as it is) every sum is a scalar chain with A and B added
// per pair. Every kernel of one storage type takes the same form, so the
// kernels of one precision give the same bits.
template <typename S>
constexpr bool kPackedSums = sizeof(S) == 2;

__device__ __forceinline__ float2 dens_sum2(const float2 (&d)[Q]) {
    float2 s = d[0];
#pragma unroll
    for (int i = 1; i < Q; ++i) s = add2(s, d[i]);
    return s;
}
// one component: the same additions in the same order
__device__ __forceinline__ float dens_sum(const float (&d)[Q]) {
    float s = d[0];
#pragma unroll
    for (int i = 1; i < Q; ++i) s = __fadd_rn(s, d[i]);
    return s;
}

// c_i along axis a for a velocity known at compile time
template <int i, int a>
__host__ __device__ constexpr int vel_comp() {
    return a == 0 ? Vel<i>::x : (a == 1 ? Vel<i>::y : Vel<i>::z);
}
// first and second axes along which a velocity moves (diagonals move along two)
template <int i>
__host__ __device__ constexpr int vel_axis0() {
    return Vel<i>::x != 0 ? 0 : (Vel<i>::y != 0 ? 1 : 2);
}
template <int i>
__host__ __device__ constexpr int vel_axis1() {
    return (Vel<i>::x != 0 && Vel<i>::y != 0) ? 1 : 2;
}

template <bool PACKED>
__device__ __forceinline__ void momentum2(const float2 (&d)[Q], float (&j)[3]) {
    if constexpr (!PACKED) {
        j[0] = j[1] = j[2] = 0.f;
        static_for<0, 9>([&](auto M) {
            constexpr int i = 2 * decltype(M)::value + 1;   // (i, i + 1) are opposite
            const float diff = (d[i].x - d[i + 1].x) + (d[i].y - d[i + 1].y);
            if constexpr (Vel<i>::x != 0) j[0] += Vel<i>::x * diff;
            if constexpr (Vel<i>::y != 0) j[1] += Vel<i>::y * diff;
            if constexpr (Vel<i>::z != 0) j[2] += Vel<i>::z * diff;
        });
    } else {
        float2 J[3];
        static_for<0, 9>([&](auto M) {
            constexpr int i = 2 * decltype(M)::value + 1;
            // the odd member of each pair moves + along its first axis (public order)
            static_assert(vel_comp<i, vel_axis0<i>()>() == 1, "velocity order: odd members lead");
            const float2 diff = sub2(d[i], d[i + 1]);
            constexpr int a0 = vel_axis0<i>();
            if constexpr (Vel<i>::c2 == 1) {
                J[a0] = diff;   // the axis pairs come first (i = 1, 3, 5)
            } else {
                constexpr int a1 = vel_axis1<i>();
                J[a0] = add2(J[a0], diff);
                if constexpr (vel_comp<i, a1>() > 0) J[a1] = add2(J[a1], diff);
                else J[a1] = sub2(J[a1], diff);
            }
        });
#pragma unroll
        for (int a = 0; a < 3; ++a) j[a] = __fadd_rn(J[a].x, J[a].y);
    }
}

template <typename S>
__device__ __forceinline__ void momentum(const float (&d)[2][Q], float (&j)[3]) {
    float2 d2[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) d2[i] = make_float2(d[0][i], d[1][i]);
    momentum2<kPackedSums<S>>(d2, j);
}

template <typename S>
__device__ __forceinline__ void sums(const float (&d)[2][Q], float& dA, float& dB, float (&j)[3]) {
    dA = dens_sum(d[0]);
    dB = dens_sum(d[1]);
    momentum<S>(d, j);
}

// BGK arithmetic of storage type S: 16-bit storage (bound by instruction
// issue) takes the form with fewer operations (the pair's coefficients
// precomputed, c.u without an addition to zero: three fewer per pair and component);
// FP32 (bound by memory bandwidth) keeps the form that schedules faster
// there. Every kernel of one storage type uses the same form.
template <typename S>
constexpr bool kLeanBGK = sizeof(S) == 2;

// BGK collision with the Shan-Chen velocity shift, in deviation form, and
// store of the post-collision node.
//   SA, SB: sum_{i>=1} w_i psi^k(x + c_i) c_i for k = A, B.
// F^A = -G psi^A SB + rho^A g, so tau F^A / rho^A = tau (-G SB + g) at a
// fluid node (psi = rho there).
// Equilibrium deviation: f^eq_i - w_i rho0 = w_i [(rho - rho0) + rho (3 c.u
// + 4.5 (c.u)^2 - 1.5 u.u)] (Eq. LEQ with c_s^2 = 1/3); the stored value is
// (1 - omega) d_i + omega (f^eq_i - w_i rho0).
// With Z, a lane with zero set stores 0 in every slot (a solid node). Both
// components of a velocity are stored as one pair: component A's outputs are
// computed first (each replaces its input, which is dead after), then B's,
// each stored with its A partner.
// dget(k, i) gives the pulled deviation d_i^k.
template <typename S, bool Z = false, typename DGet>
__device__ __forceinline__ void collide_store_g(DGet&& dget, const Phys& p, float dA, float dB,
                                                const float (&j)[3], const float (&SA)[3],
                                                const float (&SB)[3], S* __restrict__ dst,
                                                const Geom& g, int own, bool zero = false) {
    const float rA = p.rho0[0] + dA, rB = p.rho0[1] + dB;
    // fast reciprocal (within 2 ulp): the correctly rounded division costs
    // about 5% of the step, and the parity bar is 1e-5
    const float inv = __fdividef(1.0f, rA + rB);
    const float up[3] = {j[0] * inv, j[1] * inv, j[2] * inv};
    const float om1 = 1.0f - p.omega;
    float gA[Q];
    S* out = dst + blk_base((uint32_t)own);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float (&Sk)[3] = (k == 0) ? SB : SA;
        const float rk = (k == 0) ? rA : rB;
        const float drk = (k == 0) ? dA : dB;
        float u[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) u[a] = up[a] + p.tau * (p.g[a] - p.G * Sk[a]);
        const float uu15 = 1.5f * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        auto put = [&](int i, float v) {
            if (k == 0) {
                gA[i] = v;
            } else {
                float a = gA[i], b = v;
                if (Z && zero) a = b = 0.f;
                Store<S>::st2(out + i * (2 * kBlk), a, b);
            }
        };
        if constexpr (kLeanBGK<S>) {
            // omega * f^eq deviation, split for an opposite pair (i, i+1) of
            // weight w into a part even in c, w (drho + rho (4.5 (c.u)^2 -
            // 1.5 u.u)) = a (c.u)^2 + e, and a part odd in c, 3 w rho c.u =
            // b c.u, with a = 4.5 w rho, b = 3 w rho, e = w (drho - 1.5 rho
            // u.u) (all times omega). The diagonal weight is half the axis
            // weight, so its three coefficients are the axis ones halved
            // (exactly).
            const float wr1 = p.omega * (1.0f / 18.0f) * rk;
            const float a1 = 4.5f * wr1, b1 = 3.0f * wr1;
            const float e1 = fmaf(-wr1, uu15, p.omega * (1.0f / 18.0f) * drk);
            const float a2 = 0.5f * a1, b2 = 0.5f * b1, e2 = 0.5f * e1;
            // rest population (weight 1/3 = 6 x 1/18): omega f^eq deviation 6 e
            put(0, fmaf(om1, dget(k, 0), 6.0f * e1));
            static_for<0, 9>([&](auto M) {
                constexpr int i = 2 * decltype(M)::value + 1;   // (i, i + 1) opposite
                // c.u from the nonzero components only (no addition to 0)
                constexpr int ax0 = vel_axis0<i>(), ax1 = vel_axis1<i>();
                float cu = vel_comp<i, ax0>() > 0 ? u[ax0] : -u[ax0];
                if constexpr (Vel<i>::c2 == 2) cu = vel_comp<i, ax1>() > 0 ? cu + u[ax1] : cu - u[ax1];
                constexpr bool axis = Vel<i>::c2 == 1;
                const float ca = axis ? a1 : a2, cb = axis ? b1 : b2, ce = axis ? e1 : e2;
                const float even = fmaf(ca, cu * cu, ce);
                put(i, fmaf(cb, cu, fmaf(om1, dget(k, i), even)));
                put(i + 1, fmaf(-cb, cu, fmaf(om1, dget(k, i + 1), even)));
            });
        } else {
            // omega * f^eq deviation, split for an opposite pair (i, i+1) into
            // a part even in c (w (drho + rho (4.5 (c.u)^2 - 1.5 u.u))) and a
            // part odd in c (3 w rho c.u)
            const float wr1 = p.omega * (1.0f / 18.0f) * rk, wd1 = p.omega * (1.0f / 18.0f) * drk;
            const float wr2 = p.omega * (1.0f / 36.0f) * rk, wd2 = p.omega * (1.0f / 36.0f) * drk;
            put(0, om1 * dget(k, 0) + p.omega * (1.0f / 3.0f) * (drk - rk * uu15));
            static_for<0, 9>([&](auto M) {
                constexpr int i = 2 * decltype(M)::value + 1;   // (i, i + 1) opposite
                float cu = 0.f;
                if constexpr (Vel<i>::x != 0) cu += Vel<i>::x * u[0];
                if constexpr (Vel<i>::y != 0) cu += Vel<i>::y * u[1];
                if constexpr (Vel<i>::z != 0) cu += Vel<i>::z * u[2];
                constexpr bool axis = Vel<i>::c2 == 1;
                const float wr = axis ? wr1 : wr2, wd = axis ? wd1 : wd2;
                const float even = wr * (4.5f * cu * cu - uu15) + wd;
                const float odd = 3.0f * wr * cu;
                put(i, om1 * dget(k, i) + (even + odd));
                put(i + 1, om1 * dget(k, i + 1) + (even - odd));
            });
        }
    }
}

template <typename S, bool Z = false>
__device__ __forceinline__ void collide_store(const float (&d)[2][Q], const Phys& p, float dA, float dB,
                                              const float (&j)[3], const float (&SA)[3],
                                              const float (&SB)[3], S* __restrict__ dst,
                                              const Geom& g, int own, bool zero = false) {
    collide_store_g<S, Z>([&](int k, int i) { return d[k][i]; }, p, dA, dB, j, SA, SB, dst, g, own, zero);
}

// Colour-gradient collision (Appendix: Eq. 1coll, BGK at the mixture
// viscosity; Eq. 2coll, the perturbation with A = 9 omega sigma / 4 and the
// table's B_i; Eq. 3coll, the recolouring) in deviation form, and store of the
// post-collision node. gt = grad Theta, Theta = (rho^A - rho^B) / rho. With
// f*_i = f_i^A,(2) + f_i^B,(2) = w_i (rho0^A + rho0^B) + D_i, the recoloured
// deviations are
//   d_i^A =  w_i e + (rho^A / rho) D_i + X_i,   d_i^B = -w_i e + (rho^B / rho) D_i - X_i,
// e = (rho^A rho0^B - rho0^A rho^B) / rho, X_i = beta (rho^A rho^B / rho) w_i cos(phi_i),
// which conserves the mass of each component and the total momentum.
template <typename S, typename DGet>
__device__ __forceinline__ void cg_collide_store_g(DGet&& dget, const Phys& p, float dA, float dB,
                                                   const float (&j)[3], const float (&gt)[3],
                                                   S* __restrict__ dst, int own) {
    // Every sum of products is written as explicit fused multiply-adds, so
    // that no kernel's compilation can contract it differently: the box and
    // the two-pass kernels give the same bits.
    const float rA = p.rho0[0] + dA, rB = p.rho0[1] + dB;
    const float rho = rA + rB, drho = dA + dB;
    const float inv = __fdividef(1.0f, rho);
    const float u[3] = {j[0] * inv, j[1] * inv, j[2] * inv};
    const float uu15 = 1.5f * fmaf(u[2], u[2], fmaf(u[1], u[1], u[0] * u[0]));
    const float inu = fmaf(rA, p.cg_inu[0], rB * p.cg_inu[1]) * inv;   // 1 / nu_bar
    const float omega = __fdividef(2.0f * inu, 6.0f + inu);             // 2 / (6 nu_bar + 1)
    const float om1 = 1.0f - omega;
    const float g2 = fmaf(gt[2], gt[2], fmaf(gt[1], gt[1], gt[0] * gt[0]));
    // 1 / |grad Theta|; 0 (no perturbation, no recolouring) where |grad Theta|
    // <= 1e-5: the direction of a gradient at the rounding level of the state
    // is undefined, and cos(phi_i) has no limit at grad Theta = 0
    const float q = g2 > 1e-10f ? rsqrtf(g2) : 0.f;
    const float gn = g2 * q;                           // |grad Theta|
    const float hA = 1.125f * omega * p.cg_sigma;     // A / 2
    const float kc = p.cg_beta * rA * rB * inv * q;   // beta rho^A rho^B / (rho |grad Theta|)
    const float e = fmaf(rA, p.rho0[1], -(p.rho0[0] * rB)) * inv;
    const float fa = rA * inv, fb = rB * inv;
    S* out = dst + blk_base((uint32_t)own);
    // The two components' BGK terms enter only through their sum D_i, so they
    // are added first, and each opposite pair's coefficients are formed once
    // per weight class (the diagonal ones are the axis ones halved, exactly):
    //   D_i = (1 - omega) (d_i^A + d_i^B) + E + a (c.u)^2 + P (c.gT)^2 + b c.u,
    // E = omega w (drho - 1.5 rho u.u) - 2 (A/2) B_i |gT|, a = 4.5 omega w rho,
    // P = 2 (A/2) w / |gT|, b = 3 omega w rho (gT = grad Theta); c.u and c.gT
    // change sign within a pair, the perturbation does not, and the
    // recolouring term X = beta rho^A rho^B / (rho |gT|) (w / |c|) c.gT flips.
    const float base = omega * fmaf(-rho, uu15, drho);   // omega (drho - 1.5 rho u.u)
    {   // rest velocity: c = 0, so no recolouring
        constexpr float w = 1.0f / 3.0f;
        const float D = fmaf(om1, dget(0, 0) + dget(1, 0), fmaf(w, base, hA * ((4.0f / 9.0f) * gn)));
        Store<S>::st2(out, fmaf(fa, D, w * e), fmaf(fb, D, -(w * e)));
    }
    const float orho = omega * rho;
    const float E1 = fmaf(-2.0f * hA * (1.0f / 54.0f), gn, (1.0f / 18.0f) * base);
    const float E2 = fmaf(-2.0f * hA * (1.0f / 27.0f), gn, (1.0f / 36.0f) * base);
    const float a1 = (4.5f / 18.0f) * orho, a2 = 0.5f * a1;
    const float b1 = (3.0f / 18.0f) * orho, b2 = 0.5f * b1;
    const float P1 = (2.0f / 18.0f) * hA * q, P2 = 0.5f * P1;
    const float X1 = kc * (1.0f / 18.0f), X2 = kc * (0.70710678f / 36.0f);   // w / |c|: 1/18, 1/(36 sqrt 2)
    const float we1 = (1.0f / 18.0f) * e, we2 = 0.5f * we1;
    static_for<0, 9>([&](auto M) {
        constexpr int i = 2 * decltype(M)::value + 1;   // (i, i + 1) opposite
        constexpr int ax0 = vel_axis0<i>(), ax1 = vel_axis1<i>();
        float cu = vel_comp<i, ax0>() > 0 ? u[ax0] : -u[ax0];
        float cg = vel_comp<i, ax0>() > 0 ? gt[ax0] : -gt[ax0];
        if constexpr (Vel<i>::c2 == 2) {
            cu = vel_comp<i, ax1>() > 0 ? cu + u[ax1] : cu - u[ax1];
            cg = vel_comp<i, ax1>() > 0 ? cg + gt[ax1] : cg - gt[ax1];
        }
        constexpr bool axis = Vel<i>::c2 == 1;
        const float Ec = axis ? E1 : E2, ac = axis ? a1 : a2, bc = axis ? b1 : b2;
        const float Pc = axis ? P1 : P2, Xc = axis ? X1 : X2, we = axis ? we1 : we2;
        const float even = fmaf(ac, cu * cu, fmaf(Pc, cg * cg, Ec));
        const float Di = fmaf(bc, cu, fmaf(om1, dget(0, i) + dget(1, i), even));
        const float Dj = fmaf(-bc, cu, fmaf(om1, dget(0, i + 1) + dget(1, i + 1), even));
        const float X = Xc * cg;
        Store<S>::st2(out + i * (2 * kBlk), fmaf(fa, Di, we) + X, fmaf(fb, Di, -we) - X);
        Store<S>::st2(out + (i + 1) * (2 * kBlk), fmaf(fa, Dj, we) - X, fmaf(fb, Dj, -we) + X);
    });
}

// Phase field Theta = (rho^A - rho^B) / rho from the density deviations.
__device__ __forceinline__ float phase_field(const Phys& p, float dA, float dB) {
    return __fdividef((p.rho0[0] - p.rho0[1]) + (dA - dB), (p.rho0[0] + p.rho0[1]) + (dA + dB));
}

// Per-node moments kept by the adjoint's recompute, 11 fields: drho^A,
// drho^B, j (3), S^A (3), S^B (3). Written at fluid nodes only, blocked like
// the populations: field c of site s at mom_base(s) + c * kBlk.
constexpr int kMom = 11;
__host__ __device__ __forceinline__ size_t mom_base(uint32_t s) {
    return (size_t)(s / (uint32_t)kBlk) * (size_t)(kMom * kBlk) + (size_t)(s % (uint32_t)kBlk);
}
__host__ __device__ __forceinline__ size_t mom_elems(long long N) {
    return (size_t)((N + kBlk - 1) / kBlk) * (size_t)(kMom * kBlk);
}
__device__ __forceinline__ void store_moments(float* __restrict__ mom, const Geom& g, long long own, float dA,
                                              float dB, const float (&j)[3], const float (&SA)[3],
                                              const float (&SB)[3]) {
    const float v[kMom] = {dA, dB, j[0], j[1], j[2], SA[0], SA[1], SA[2], SB[0], SB[1], SB[2]};
    float* m = mom + mom_base((uint32_t)own);
#pragma unroll
    for (int c = 0; c < kMom; ++c) m[c * kBlk] = v[c];
}

// Density deviations dpsi^k = psi^k - rho0^k of node (x, y, z): sum_i d_i^k at
// a fluid node, -rho0^k at a solid node (psi = 0 there). Since
// sum_{i>=1} w_i c_i = 0, the force sums S^k = sum_i w_i psi^k(x + c_i) c_i are
// the same sums over dpsi, without the rounding of rho0 + sum_i d_i.
template <typename S, bool MASK>
__device__ __forceinline__ float2 density_at(const S* __restrict__ src, const uint32_t* __restrict__ flags,
                                             const Geom& g, const Phys& p, int x, int y, int z) {
    PullIdx P;
    pull_indices(g, x, y, z, P);
    uint32_t fl = 0;
    if constexpr (MASK) {
        fl = __ldg(flags + P.own);
        if (fl & kSolid) return make_float2(-p.rho0[0], -p.rho0[1]);
    }
    float d[2][Q];
    pull<S, MASK>(src, g, P, p.slots ? 0u : fl, d);
    return make_float2(dens_sum(d[0]), dens_sum(d[1]));
}

// Shan-Chen neighbour sums S^k = sum_{i>=1} w_i psi^k(x + c_i) c_i, in a
// form factored by planes. For the column (x, y) of plane p (both components, .x = A,
// .y = B):
//   dx(p) = psi(x+1, y, p) - psi(x-1, y, p),   dy(p) = psi(x, y+1, p) - psi(x, y-1, p),
//   t(p)  = w1 psi(x, y, p) + w2 (psi(x+1, y, p) + psi(x-1, y, p) + psi(x, y+1, p) + psi(x, y-1, p)),
// with w1 = 1/18 (axis links) and w2 = 1/36 (diagonal links). Then, with the
// in-plane diagonals d_pm = psi(x+1, y-1, z) etc. of the node's plane z,
//   S_x = w1 dx(z) + w2 ((d_pp - d_mp) + (d_pm - d_mm)) + w2 (dx(z+1) + dx(z-1)),
//   S_y = w1 dy(z) + w2 ((d_pp - d_pm) + (d_mp - d_mm)) + w2 (dy(z+1) + dy(z-1)),
//   S_z = t(z+1) - t(z-1).
// A kernel marching in z computes the plane quantities of a column once and
// uses them for three nodes.
constexpr float kW1 = 1.0f / 18.0f, kW2 = 1.0f / 36.0f;

struct PlaneSums {
    float2 dx, dy, t;
};

// both components at once, with packed (A, B) instructions

__device__ __forceinline__ PlaneSums plane_sums(float2 c, float2 xp, float2 xm, float2 yp, float2 ym) {
    PlaneSums s;
    s.dx = sub2(xp, xm);
    s.dy = sub2(yp, ym);
    s.t = fma2(splat(kW1), c, mul2(splat(kW2), add2(add2(xp, xm), add2(yp, ym))));
    return s;
}

__device__ __forceinline__ void force_sums(const PlaneSums& lo, const PlaneSums& mid, const PlaneSums& hi,
                                           float2 pp, float2 mp, float2 pm, float2 mm, float (&SA)[3],
                                           float (&SB)[3]) {
    const float2 w1 = splat(kW1), w2 = splat(kW2);
    const float2 sx = fma2(w2, add2(hi.dx, lo.dx), fma2(w1, mid.dx, mul2(w2, add2(sub2(pp, mp), sub2(pm, mm)))));
    const float2 sy = fma2(w2, add2(hi.dy, lo.dy), fma2(w1, mid.dy, mul2(w2, add2(sub2(pp, pm), sub2(mp, mm)))));
    const float2 sz = sub2(hi.t, lo.t);
    SA[0] = sx.x;
    SB[0] = sx.y;
    SA[1] = sy.x;
    SB[1] = sy.y;
    SA[2] = sz.x;
    SB[2] = sz.y;
}

// plane quantities of plane dz (-1, 0, +1) from a lookup of dpsi(dx, dy, dz)
template <typename Look>
__device__ __forceinline__ PlaneSums plane_sums_at(Look&& psi, int dz) {
    return plane_sums(psi(0, 0, dz), psi(1, 0, dz), psi(-1, 0, dz), psi(0, 1, dz), psi(0, -1, dz));
}

// S^k from a lookup of dpsi(dx, dy, dz) (the 18 neighbours of the node).
// FACTORED: the plane form above with packed (A, B) instructions (16-bit
// storage, whose box kernel reuses the plane quantities); otherwise one
// multiply-add per link and component in velocity order (FP32, where it
// schedules faster). Every kernel of a storage type uses the same form, so
// the kernels of one precision give the same bits.
template <bool FACTORED, typename Look>
__device__ __forceinline__ void neighbour_sums(Look&& psi, float (&SA)[3], float (&SB)[3]) {
    if constexpr (FACTORED) {
        const PlaneSums lo = plane_sums_at(psi, -1), mid = plane_sums_at(psi, 0), hi = plane_sums_at(psi, 1);
        force_sums(lo, mid, hi, psi(1, 1, 0), psi(-1, 1, 0), psi(1, -1, 0), psi(-1, -1, 0), SA, SB);
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) SA[a] = SB[a] = 0.f;
        static_for<1, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            const float2 v = psi(Vel<i>::x, Vel<i>::y, Vel<i>::z);
            constexpr float w = wgt<i>();
            if constexpr (Vel<i>::x != 0) { SA[0] += (w * Vel<i>::x) * v.x; SB[0] += (w * Vel<i>::x) * v.y; }
            if constexpr (Vel<i>::y != 0) { SA[1] += (w * Vel<i>::y) * v.x; SB[1] += (w * Vel<i>::y) * v.y; }
            if constexpr (Vel<i>::z != 0) { SA[2] += (w * Vel<i>::z) * v.x; SB[2] += (w * Vel<i>::z) * v.y; }
        });
    }
}

// the form used by the kernels of storage type S
template <typename S>
constexpr bool kFactoredSums = sizeof(S) == 2;

}  // namespace lbgb
