// lb_particles.cu -- moving rigid spheres (Sec. 2): moving-wall halfway
// bounce-back at the links into a sphere (Eq. UPI, Eq. LADDFLBE), the
// momentum those links exchange summed in FP64 into each sphere's force and
// torque (Eq. FORCEPP, Eq. FORCEPARTEQ, Eq. TORQUEPARTEQ), the leap-frog
// update of Eq. PARDYN with the spheres' contact and lubrication forces, and
// re-meshing of the nodes a moved sphere leaves or reaches (the rule
// conserves the total momentum of fluid and spheres).
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

// minimum-image displacement along one axis of period n (general form)
__device__ __forceinline__ double min_image(double d, int n) {
    return __dsub_rn(d, __dmul_rn((double)n, rint(__ddiv_rn(d, (double)n))));
}

__device__ __forceinline__ double norm2(double a, double b, double c) {
    return __dadd_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)), __dmul_rn(c, c));
}

// The cube of sites of one sphere, centred on floor(c): site b of side^3
// has unwrapped coordinates u = lo + (bx, by, bz) and grid coordinates
// x = u + n m (m the wrap count). Its half-width keeps |u - c| below n / 2,
// so the minimum-image displacement of x from c is (x - c) - n m, rounded
// as that plain evaluation rounds it (no division).
struct Cube {
    int lo[3];
    int side;
    int base[3];    // floor(c)
    float frac[3];  // c - floor(c)
    __device__ Cube(const double* c, int half) {
        side = 2 * half + 1;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double f = floor(c[a]);
            base[a] = (int)f;
            frac[a] = (float)(c[a] - f);
            lo[a] = base[a] - half;
        }
    }
    // site (bx, by, bz) of the cube; u stays within one period of the grid
    // (0 <= floor(c) < n and half + 1 < n), so one conditional wrap gives x
    __device__ void site(int bx, int by, int bz, const Geom& g, int (&u)[3], int (&x)[3]) const {
        u[0] = lo[0] + bx;
        u[1] = lo[1] + by;
        u[2] = lo[2] + bz;
        const int n[3] = {g.nx, g.ny, g.nz};
#pragma unroll
        for (int a = 0; a < 3; ++a) x[a] = u[a] < 0 ? u[a] + n[a] : (u[a] >= n[a] ? u[a] - n[a] : u[a]);
    }
    // approximate squared distance from the centre (FP32, for shell tests)
    __device__ float dist2(const int (&u)[3], float (&d)[3]) const {
#pragma unroll
        for (int a = 0; a < 3; ++a) d[a] = (float)(u[a] - base[a]) - frac[a];
        return d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    }
};

// A walk over the cube's sites without a division per site: thread t of a
// block of nt threads visits the sites b = t, t + nt, t + 2 nt, ... of the
// side^3 cube (b = bx + side (by + side bz)); stepping adds nt in the same
// base-side digits.
struct CubeWalk {
    int side;
    int bx, by, bz;      // this thread's current site
    int dbx, dby, dbz;   // nt in those digits
    __device__ CubeWalk(const Cube& cube, int t, int nt) : side(cube.side) {
        split(t, bx, by, bz);
        split(nt, dbx, dby, dbz);
    }
    __device__ void split(int j, int& a, int& b, int& c) const {
        a = j % side;
        const int q = j / side;
        b = q % side;
        c = q / side;
    }
    __device__ bool valid() const { return bz < side; }
    __device__ void next() {
        bx += dbx;
        if (bx >= side) { bx -= side; ++by; }
        by += dby;
        if (by >= side) { by -= side; ++bz; }
        bz += dbz;
    }
};

// exact minimum-image displacement of grid coordinate x (unwrapped u) from c
__device__ __forceinline__ double disp(int x, int u, double c, int n) {
    const int m = (x - u) / n;
    return __dsub_rn(__dsub_rn((double)x, c), (double)(n * m));
}

// Is the site within radius of the centre? Far from the sphere's surface the
// FP32 distance decides; near it, the exact FP64 test (the oracle's rule).
// R2f = (float)R2, formed once by the caller (a conversion from FP64 per site
// would run on the FP64 pipe).
__device__ __forceinline__ bool covered(const int (&u)[3], const int (&x)[3], float r2f, const double* c, double R2,
                                        float R2f, const Geom& g) {
    if (r2f < 0.99f * R2f) return true;
    if (r2f > 1.01f * R2f) return false;
    return norm2(disp(x[0], u[0], c[0], g.nx), disp(x[1], u[1], c[1], g.ny), disp(x[2], u[2], c[2], g.nz)) <= R2;
}

// Has sphere q moved less than its margin since its last full re-meshing
// pass? Then no node can have changed (each node's distance to the centre
// changes by at most the displacement).
__device__ __forceinline__ bool within_margin(const Spheres& A, int q, const Geom& g) {
    const int n[3] = {g.nx, g.ny, g.nz};
    float d2 = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float d = (float)(A.r[3 * q + a] - A.ref[3 * q + a]);
        d -= (float)n[a] * rintf(d / (float)n[a]);
        d2 += d * d;
    }
    const float m = A.margin[q] - 1e-4f;   // FP32 slack
    return m > 0.f && d2 < m * m;
}

__device__ __forceinline__ uint32_t site_of(const int (&x)[3], const Geom& g) {
    return (uint32_t)x[0] + (uint32_t)g.nx * ((uint32_t)x[1] + (uint32_t)g.ny * (uint32_t)x[2]);
}

// This thread's nodes of a sphere's cube (its sites of the cube walk), eight
// steps at a time: cand(u, x, r2) picks the nodes to visit (it is called for
// every node),
// the owner of every picked node of the batch is loaded first -- independent
// loads whose DRAM round trips overlap, where one load per node in turn
// would wait for each -- and then body(u, x, r2, owner) runs for each.
// Another block writes an owner only for its own sphere's nodes, so a value
// read here either is this sphere's mark or says the node is not this
// sphere's.
template <typename Cand, typename Body>
__device__ __forceinline__ void cube_batches(const Cube& cube, const Geom& g, const int* owner, Cand&& cand,
                                             Body&& body) {
    constexpr int kB = 8;
    CubeWalk wk(cube, threadIdx.x, blockDim.x);
    while (wk.valid()) {
        const CubeWalk w0 = wk;
        int own[kB];
        bool ok[kB];
#pragma unroll
        for (int k = 0; k < kB; ++k) {
            ok[k] = false;
            own[k] = 0;
            if (wk.valid()) {
                int u[3], x[3];
                cube.site(wk.bx, wk.by, wk.bz, g, u, x);
                float df[3];
                const float r2 = cube.dist2(u, df);
                if (cand(u, x, r2)) {
                    ok[k] = true;
                    own[k] = __ldg(owner + site_of(x, g));
                }
                wk.next();
            }
        }
        CubeWalk w1 = w0;
#pragma unroll
        for (int k = 0; k < kB; ++k) {
            if (ok[k]) {
                int u[3], x[3];
                cube.site(w1.bx, w1.by, w1.bz, g, u, x);
                float df[3];
                const float r2 = cube.dist2(u, df);
                body(u, x, r2, own[k]);
            }
            w1.next();
        }
    }
}

template <typename T>
__device__ __forceinline__ void cross(const T (&a)[3], const T (&b)[3], T (&o)[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// Fixed-tree block sum of NV doubles per thread; thread 0 gets the totals.
template <int NV, int NT = kPT>
__device__ void block_sum(double (&v)[NV]) {
    __shared__ double red[NV][NT];
#pragma unroll
    for (int k = 0; k < NV; ++k) red[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int h = NT / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
#pragma unroll
            for (int k = 0; k < NV; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + h];
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = red[k][0];
}

// Exclusive prefix sum of v over the block's threads in thread order (block
// size a multiple of 32, at most 32 warps); *total gets the block's sum.
// wsum: one int per warp of shared memory. Ends with a barrier.
__device__ __forceinline__ int block_exclusive_scan(int v, int* wsum, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int t = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) wsum[lane] = t;   // inclusive warp totals
        if (lane == nw - 1) *total = t;
    }
    __syncthreads();
    return x - v + (warp > 0 ? wsum[warp - 1] : 0);
}

template <typename T>
__device__ __forceinline__ void load3(const double* a, int q, T (&o)[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) o[k] = (T)a[3 * q + k];
}

// Links from fluid nodes into sphere q: slot opp(i) of the covered node
// x + c_i takes g_i(x) - 2 rho0^k w_i (u_b . c_i) / c_s^2, and the link adds
// c_i sum_k (2 g_i^k(x) - 2 rho0^k w_i (u_b . c_i) / c_s^2) to the force and
// (r_b - r) x that to the torque. The exchanged momentum splits into the
// rest part c_i 2 w_i (rho0^A + rho0^B), large and cancelling over the
// surface, and a small deviation part. With 36 w_i integer and the link
// midpoint r_b = x + c_i / 2, the rest part's force and torque are exact
// integer sums of the link geometry, scaled once per sphere in FP64; the
// deviation part and the wall velocity are FP32 per link (as the state is),
// summed in FP64 across the block. A linked node is fluid (beyond R) with a
// neighbour inside (within R + sqrt 2): only that shell is visited (with a
// margin of 0.01 for the FP32 distances).
template <typename S>
__global__ void __launch_bounds__(kPT) sphere_links_kernel(S* __restrict__ st, const uint32_t* __restrict__ flags,
                                                          Spheres A, int forces, Geom g, Phys p) {
    const int q = blockIdx.x;
    double c[3];
    float v[3], w[3];
    load3(A.r, q, c);
    load3(A.v, q, v);
    load3(A.w, q, w);
    const Cube cube(c, A.half);
    const float lo2 = (float)((A.radius - 0.01) * (A.radius - 0.01));
    const float hi2 = (float)((A.radius + 1.4243) * (A.radius + 1.4243));
    int gF[3] = {0, 0, 0}, gT[3] = {0, 0, 0};   // sum 36 w_i c_i, sum 36 w_i (2 (u - base) + c_i) x c_i
    float dF[3] = {0.f, 0.f, 0.f}, dT[3] = {0.f, 0.f, 0.f};
    // the links of one fluid node (site s at x, unwrapped u, offset d from the centre)
    auto node = [&](const int (&u)[3], const int (&x)[3], const float (&d)[3], uint32_t s, uint32_t fl) {
        const int xm = wrap_dec(x[0], g.nx), xp = wrap_inc(x[0], g.nx);
        const int ym = wrap_dec(x[1], g.ny), yp = wrap_inc(x[1], g.ny);
        const int zm = wrap_dec(x[2], g.nz), zp = wrap_inc(x[2], g.nz);
        const int h0[3] = {2 * (u[0] - cube.base[0]), 2 * (u[1] - cube.base[1]), 2 * (u[2] - cube.base[2])};
        auto target = [&](auto I) -> uint32_t {   // site x + c_i
            constexpr int i = decltype(I)::value;
            constexpr int cx = Vel<i>::x, cy = Vel<i>::y, cz = Vel<i>::z;
            const int t3[3] = {cx > 0 ? xp : (cx < 0 ? xm : x[0]), cy > 0 ? yp : (cy < 0 ? ym : x[1]),
                               cz > 0 ? zp : (cz < 0 ? zm : x[2])};
            return site_of(t3, g);
        };
        // The node's links to this sphere, then their populations, each as a
        // batch of independent loads (the owner and population of one link
        // are a chain of two DRAM round trips; batched, the node's links
        // overlap theirs), then the slots and the force.
        uint32_t lmask = 0;
        static_for<1, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            if (fl & (1u << Vel<i>::opp))   // x + c_i is solid: is it this sphere?
                if (__ldg(A.owner + target(I)) == q + 1) lmask |= 1u << i;
        });
        float pA[Q], pB[Q];
        static_for<1, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            pA[i] = pB[i] = 0.f;
            if (lmask & (1u << i)) Store<S>::ld2(st + pidx(0, i, s), pA[i], pB[i]);
        });
        static_for<1, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int cx = Vel<i>::x, cy = Vel<i>::y, cz = Vel<i>::z;
            constexpr int w36 = Vel<i>::c2 == 1 ? 2 : 1;
            if (!(lmask & (1u << i))) return;
            const uint32_t t = target(I);
            const float arm[3] = {d[0] + 0.5f * cx, d[1] + 0.5f * cy, d[2] + 0.5f * cz};
            float wa[3];
            cross(w, arm, wa);
            const float cu = 3.0f * (cx * (v[0] + wa[0]) + cy * (v[1] + wa[1]) + cz * (v[2] + wa[2]));
            const float dA = pA[i], dB = pB[i];
            const float bA = 2.0f * p.rho0[0] * wgt<i>() * cu;
            const float bB = 2.0f * p.rho0[1] * wgt<i>() * cu;
            Store<S>::st2(st + pidx(0, Vel<i>::opp, t), dA - bA, dB - bB);
            if (!forces) return;
            const int h[3] = {h0[0] + cx, h0[1] + cy, h0[2] + cz};
            gF[0] += w36 * cx;
            gF[1] += w36 * cy;
            gF[2] += w36 * cz;
            gT[0] += w36 * (h[1] * cz - h[2] * cy);
            gT[1] += w36 * (h[2] * cx - h[0] * cz);
            gT[2] += w36 * (h[0] * cy - h[1] * cx);
            const float ex = 2.0f * (dA + dB) - (bA + bB);
            const float F[3] = {cx * ex, cy * ex, cz * ex};
            float Tq[3];
            cross(arm, F, Tq);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                dF[a] += F[a];
                dT[a] += Tq[a];
            }
        });
    };
    // In rounds: every thread screens kRound sites of its cube walk (in the
    // shell, fluid, with a solid neighbour; the flag loads as one batch) and
    // appends the nodes that pass to a shared list; then the block works the
    // list one node per thread, so that the link work (a few percent of the
    // cube's sites) runs on full warps.
    constexpr int kRound = 10;   // R = 5.5: 4913 sites, 20 a thread, two rounds
    __shared__ uint32_t lsite[kRound * kPT];   // walk index of each listed node
    __shared__ uint32_t lflag[kRound * kPT];
    __shared__ int nlist;
    __shared__ int wsum[kPT / 32];
    const int per_thread = (cube.side * cube.side * cube.side + (int)blockDim.x - 1) / (int)blockDim.x;
    const int rounds = (per_thread + kRound - 1) / kRound;
    CubeWalk wk(cube, threadIdx.x, blockDim.x);
    for (int round = 0; round < rounds; ++round) {
        uint32_t fl[kRound], idx[kRound];
        bool in[kRound];
#pragma unroll
        for (int k = 0; k < kRound; ++k) {
            in[k] = false;
            fl[k] = 0u;
            idx[k] = 0u;
            if (wk.valid()) {
                int u[3], x[3];
                cube.site(wk.bx, wk.by, wk.bz, g, u, x);
                float d[3];
                const float r2 = cube.dist2(u, d);
                if (r2 > lo2 && r2 <= hi2) {
                    in[k] = true;
                    idx[k] = (uint32_t)(wk.bx + cube.side * (wk.by + cube.side * wk.bz));
                    fl[k] = __ldg(flags + site_of(x, g));
                }
                wk.next();
            }
        }
        // each thread's passing sites go to the list in thread order (a block
        // scan of the counts), so that the work, and the force sums, are the
        // same from run to run
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < kRound; ++k) {
            in[k] = in[k] && !(fl[k] & kSolid) && (fl[k] & kNbSolidMask);
            cnt += in[k] ? 1 : 0;
        }
        int j = block_exclusive_scan(cnt, wsum, &nlist);
#pragma unroll
        for (int k = 0; k < kRound; ++k) {
            if (in[k]) {
                lsite[j] = idx[k];
                lflag[j] = fl[k];
                ++j;
            }
        }
        __syncthreads();
        const int n = nlist;
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const int b = (int)lsite[j];
            const int bx = b % cube.side, byz = b / cube.side;
            int u[3], x[3];
            cube.site(bx, byz % cube.side, byz / cube.side, g, u, x);
            float d[3];
            cube.dist2(u, d);
            node(u, x, d, site_of(x, g), lflag[j]);
        }
        __syncthreads();   // the list is read before the next round resets it
    }
    if (!forces) return;
    double acc[12];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        acc[a] = gF[a];
        acc[3 + a] = gT[a];
        acc[6 + a] = dF[a];
        acc[9 + a] = dT[a];
    }
    block_sum(acc);
    if (threadIdx.x == 0) {
        const double r36 = 2.0 * ((double)p.rho0[0] + (double)p.rho0[1]) / 36.0;
        const double fr[3] = {c[0] - cube.base[0], c[1] - cube.base[1], c[2] - cube.base[2]};
        const double Fr[3] = {r36 * acc[0], r36 * acc[1], r36 * acc[2]};
        double frF[3];
        cross(fr, Fr, frF);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            A.F[3 * q + a] = Fr[a] + acc[6 + a];
            A.T[3 * q + a] = 0.5 * r36 * acc[3 + a] - frF[a] + acc[9 + a];
        }
    }
}

// Pair forces: the contact repulsion k (2R + range - d)^(3/2) along the line
// of centres for every other sphere whose centre is d < 2R + range away
// (minimum image), and the normal lubrication force
// -(3/2) pi mu R^2 (1/h - 1/h_c) ((v_i - v_j) . n) n for gaps h = d - 2R
// below h_c (h clamped at 0.01), from the velocities before the update. One
// block per sphere, partners split over its threads in index order; an FP32
// distance test skips the far ones.
constexpr int kCT = 128;
__global__ void __launch_bounds__(kCT) sphere_contact_kernel(Spheres A, Geom g) {
    const int q = blockIdx.x;
    const int n[3] = {g.nx, g.ny, g.nz};
    const double reach = 2.0 * A.radius + A.contact_range;
    const double far = fmax(reach, 2.0 * A.radius + A.lub_cut);
    const float near2 = (float)((far + 0.5) * (far + 0.5));
    const double lub = 1.5 * 3.14159265358979323846 * A.mu * A.radius * A.radius;
    double c[3];
    load3(A.r, q, c);
    const float4 cq = A.rf[q];
    const float cf[3] = {cq.x, cq.y, cq.z};
    double F[3] = {0, 0, 0};
    for (int j = threadIdx.x; j < A.n; j += kCT) {
        if (j == q) continue;
        // FP32 screen on the FP32 centres (0 <= r < n, so one conditional
        // wrap gives the minimum image)
        const float4 cj = A.rf[j];
        const float cjf[3] = {cj.x, cj.y, cj.z};
        float e2 = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float d = cf[a] - cjf[a];
            const float h = 0.5f * (float)n[a];
            d = d > h ? d - (float)n[a] : (d < -h ? d + (float)n[a] : d);
            e2 += d * d;
        }
        if (e2 >= near2) continue;
        double d[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) d[a] = min_image(c[a] - A.r[3 * j + a], n[a]);
        const double dist = sqrt(norm2(d[0], d[1], d[2]));
        double f = 0.0;   // along n = d / dist
        if (A.contact_k != 0.0 && dist < reach) f += A.contact_k * pow(reach - dist, 1.5);
        const double h = dist - 2.0 * A.radius;
        if (A.lub_cut > 0.0 && h < A.lub_cut) {
            double vn = 0.0;
#pragma unroll
            for (int a = 0; a < 3; ++a) vn += (A.v[3 * q + a] - A.v[3 * j + a]) * d[a] / dist;
            f -= lub * (1.0 / fmax(h, 0.01) - 1.0 / A.lub_cut) * vn;
        }
        if (f == 0.0) continue;
#pragma unroll
        for (int a = 0; a < 3; ++a) F[a] += f * d[a] / dist;
    }
    block_sum<3, kCT>(F);
    if (threadIdx.x == 0)
#pragma unroll
        for (int a = 0; a < 3; ++a) A.Fc[3 * q + a] = F[a];
}

// Leap-frog: v += (F + F_c) / m, r += v (wrapped into the box), w += T / I.
__global__ void sphere_update_kernel(Spheres A, Geom g) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= A.n || !(A.mass > 0.0)) return;
    const int n[3] = {g.nx, g.ny, g.nz};
    bool fast = false;
    double v2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double v = __dadd_rn(A.v[3 * q + a],
                                   __ddiv_rn(__dadd_rn(A.F[3 * q + a], A.Fc[3 * q + a]), A.mass));
        double r = __dadd_rn(A.r[3 * q + a], v);
        // r mod n (the remainder of an exact division, then into [0, n))
        const double m = fmod(r, (double)n[a]);
        r = m < 0.0 ? __dadd_rn(m, (double)n[a]) : m;
        A.v[3 * q + a] = v;
        A.r[3 * q + a] = r;
        A.w[3 * q + a] = __dadd_rn(A.w[3 * q + a], __ddiv_rn(A.T[3 * q + a], A.inertia));
        fast = fast || fabs(v) > 1.0;
        v2 += v * v;
    }
    A.step[q] = __double2float_ru(sqrt(v2));
    A.rf[q] = make_float4((float)A.r[3 * q], (float)A.r[3 * q + 1], (float)A.r[3 * q + 2], 0.f);
    if (fast) atomicOr(A.err, 2);
}

// The flags a change of node x (grid coordinates) touches: its own solid
// bit, and bit j of x + c_j (whose neighbour x + c_j - c_j is x). Set when x
// becomes solid, cleared when it becomes fluid (a node that changes is never
// a mask node, and spheres share no node), with atomics since neighbouring
// changes share words.
__device__ __forceinline__ void flag_change(uint32_t* __restrict__ flags, const int (&x)[3], uint32_t s,
                                            bool solid, const Geom& g) {
    auto apply = [&](uint32_t t, uint32_t bit) {
        if (solid) atomicOr(flags + t, bit);
        else atomicAnd(flags + t, ~bit);
    };
    apply(s, kSolid);
    const int xm = wrap_dec(x[0], g.nx), xp = wrap_inc(x[0], g.nx);
    const int ym = wrap_dec(x[1], g.ny), yp = wrap_inc(x[1], g.ny);
    const int zm = wrap_dec(x[2], g.nz), zp = wrap_inc(x[2], g.nz);
    static_for<1, Q>([&](auto J) {
        constexpr int j = decltype(J)::value;
        constexpr int cx = Vel<j>::x, cy = Vel<j>::y, cz = Vel<j>::z;
        const int t3[3] = {cx > 0 ? xp : (cx < 0 ? xm : x[0]), cy > 0 ? yp : (cy < 0 ? ym : x[1]),
                           cz > 0 ? zp : (cz < 0 ? zm : x[2])};
        apply(site_of(t3, g), 1u << j);
    });
}

// Re-meshing, first pass: nodes sphere q covered and no longer covers become
// fluid with f^eq(rho0^k, u_b) at the wall velocity there; the sphere loses
// that momentum (and its moment).
template <typename S>
__global__ void __launch_bounds__(kPT) sphere_uncover_kernel(S* __restrict__ st, uint32_t* __restrict__ flags,
                                                            Spheres A, Geom g, Phys p) {
    const int q = blockIdx.x;
    double c[3], v[3], w[3];
    load3(A.r, q, c);
    load3(A.v, q, v);
    load3(A.w, q, w);
    const Cube cube(c, A.half);
    const double R2 = __dmul_rn(A.radius, A.radius);
    const float R2f = (float)R2;
    // The owners are the coverage at the centre before the last move (the
    // re-meshing of the previous step, or an earlier one within the margin),
    // which was the step's displacement away: only a node whose distance from
    // the surface now is at most that (plus slack for the FP32 distances) can
    // have changed.
    const float sd = A.step[q] + 1e-3f, Rf = (float)A.radius;
    const float in2 = Rf > sd ? (Rf - sd) * (Rf - sd) : -1.f;
    const float out2 = (Rf + sd) * (Rf + sd);
    const double r0 = (double)p.rho0[0] + (double)p.rho0[1];
    if (within_margin(A, q, g)) return;   // the whole block: no node changed
    __syncthreads();
    double acc[6] = {0, 0, 0, 0, 0, 0};
    bool changed = false;
    auto cand = [&](const int (&)[3], const int (&)[3], float r2) { return !(r2 < in2) && r2 <= out2; };
    cube_batches(cube, g, A.owner, cand, [&](const int (&u)[3], const int (&x)[3], float r2, int own) {
        if (own != q + 1) return;
        if (covered(u, x, r2, c, R2, R2f, g)) return;
        const uint32_t s = site_of(x, g);
        A.owner[s] = 0;
        changed = true;
        flag_change(flags, x, s, false, g);
        const double arm[3] = {disp(x[0], u[0], c[0], g.nx), disp(x[1], u[1], c[1], g.ny),
                               disp(x[2], u[2], c[2], g.nz)};
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
    });
    if (!__syncthreads_or(changed)) return;   // no node changed: nothing to exchange
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
__global__ void __launch_bounds__(kPT) sphere_cover_kernel(S* __restrict__ st, uint32_t* __restrict__ flags,
                                                          const uint8_t* __restrict__ mask, Spheres A, int absorb,
                                                          Geom g) {
    const int q = blockIdx.x;
    double c[3];
    load3(A.r, q, c);
    const Cube cube(c, A.half);
    if (absorb && within_margin(A, q, g)) return;
    const double R2 = __dmul_rn(A.radius, A.radius);
    const float R2f = (float)R2;
    const float Rf = (float)A.radius;
    // after a move only nodes within the step's displacement (plus slack) of
    // the surface can have become covered (the owners are the coverage before
    // it); a placement takes every node
    const float sd = A.step[q] + 1e-3f;
    const float in2 = absorb && Rf > sd ? (Rf - sd) * (Rf - sd) : -1.f;
    float margin = 1e30f;   // distance from the surface of the nearest node
    double acc[6] = {0, 0, 0, 0, 0, 0};
    bool changed = false;
    auto cand = [&](const int (&u)[3], const int (&x)[3], float r2) {
        margin = fminf(margin, fabsf(sqrtf(r2) - Rf));
        // covered now, and not already inside before the move
        return !(r2 < in2) && covered(u, x, r2, c, R2, R2f, g);
    };
    cube_batches(cube, g, A.owner, cand, [&](const int (&u)[3], const int (&x)[3], float, int own) {
        if (own == q + 1) return;   // covered before
        const uint32_t s = site_of(x, g);
        if ((mask && mask[s]) || atomicCAS(A.owner + s, 0, q + 1) != 0) {
            atomicOr(A.err, 1);
            return;
        }
        if (!absorb) return;   // a placement: the whole grid's flags follow
        changed = true;
        flag_change(flags, x, s, true, g);
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
        const double arm[3] = {disp(x[0], u[0], c[0], g.nx), disp(x[1], u[1], c[1], g.ny),
                               disp(x[2], u[2], c[2], g.nz)};
        double L[3];
        cross(arm, m, L);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            acc[a] += m[a];
            acc[3 + a] += L[a];
        }
    });
    // the margin of this centre (nodes beyond the cube are farther than its
    // half-width, which exceeds R + 1)
    __shared__ float mred[kPT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) margin = fminf(margin, __shfl_xor_sync(0xffffffffu, margin, o));
    if ((threadIdx.x & 31) == 0) mred[threadIdx.x >> 5] = margin;
    const bool any = __syncthreads_or(changed);   // also publishes mred
    if (threadIdx.x == 0) {
        float m = mred[0];
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) m = fminf(m, mred[k]);
        A.margin[q] = fminf(m, 1.0f);
#pragma unroll
        for (int a = 0; a < 3; ++a) A.ref[3 * q + a] = c[a];
        A.rf[q] = make_float4((float)c[0], (float)c[1], (float)c[2], 0.f);   // a placement sets it here
    }
    if (!absorb || !any) return;   // a placement, or no node changed: nothing to exchange
    block_sum(acc);
    if (threadIdx.x == 0 && A.mass > 0.0)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            A.v[3 * q + a] += acc[a] / A.mass;
            A.w[3 * q + a] += acc[3 + a] / A.inertia;
        }
}

// Solid flags (bit 0 solid, bit i: x - c_i solid) of the whole grid from the
// mask and the coverage (after a placement; a re-meshing updates the flags
// around the nodes it changes itself).
__global__ void sphere_flags_kernel(uint32_t* __restrict__ flags, const uint8_t* __restrict__ mask, Spheres A,
                                    Geom g) {
    auto solid = [&](uint32_t s) { return (mask && mask[s]) || A.owner[s] != 0; };
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.N) return;
    PullIdx P;
    pull_indices(g, (int)(s % g.nx), (int)((s / g.nx) % g.ny), (int)(s / g.plane), P);
    uint32_t f = solid((uint32_t)P.own) ? kSolid : 0u;
    static_for<1, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if (solid((uint32_t)P.src[i])) f |= (1u << i);
    });
    flags[P.own] = f;
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
    cudaError_t e = cudaSuccess;
    if (S.contact_k != 0.0 || S.lub_cut > 0.0) {   // else the pair forces stay zero
        Spheres T = S;
        T.mu = ((double)p.rho0[0] + (double)p.rho0[1]) * ((double)p.tau - 0.5) / 3.0;
        sphere_contact_kernel<<<S.n, kCT, 0, st>>>(T, g);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    sphere_update_kernel<<<(S.n + 127) / 128, 128, 0, st>>>(S, g);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
#define LBGB_MOVE(T)                                                                  \
    [&] {                                                                             \
        sphere_uncover_kernel<T><<<S.n, kPT, 0, st>>>((T*)state, flags, S, g, p);            \
        sphere_cover_kernel<T><<<S.n, kPT, 0, st>>>((T*)state, flags, mask, S, 1, g);        \
    }
    // the two passes update the flags around every node they change
    e = by_prec(prec, LBGB_MOVE(float), LBGB_MOVE(__half), LBGB_MOVE(__nv_bfloat16));
#undef LBGB_MOVE
    return e;
}

cudaError_t launch_sphere_place(uint32_t* flags, const uint8_t* mask, const Spheres& S, const Geom& g,
                                cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(S.owner, 0, (size_t)g.N * sizeof(int), st);
    if (e != cudaSuccess) return e;
    if (S.n > 0) {
        sphere_cover_kernel<float><<<S.n, kPT, 0, st>>>(nullptr, flags, mask, S, 0, g);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    sphere_flags_kernel<<<(unsigned)((g.N + 255) / 256), 256, 0, st>>>(flags, mask, S, g);
    return cudaGetLastError();
}

}  // namespace lbgb
