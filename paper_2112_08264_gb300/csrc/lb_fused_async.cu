// lb_fused_async.cu -- the fused step with an asynchronous copy pipeline.
//
// Same arithmetic as the register fused kernel (pull, densities, Shan-Chen
// force, velocity shift, BGK, store; Eq. bgk, Eq. LEQ, Eq. LADDFLBE at rest),
// restructured so that DRAM latency is hidden by copies in flight instead of
// resident warps:
//   - one block per SM owns a tile of 32 x TY x-y columns (TY chosen per grid
//     so that the number of tiles is close to a multiple of the SM count) and
//     marches along z;
//   - every thread copies, with cp.async, exactly the values it will read
//     later: the 38 pulled populations of its own node (streaming or
//     bounce-back source) and, for the first threads, of one node of the
//     one-node halo ring around the tile. A thread reads only its own copies,
//     so the shared-memory stages need no barrier; NST stages keep NST planes
//     of copies in flight;
//   - per plane, each thread turns its landed copies into density deviations
//     (own node and halo node) in a 4-plane ring, keeps its own populations in
//     registers, and after one barrier collides the previous plane with the 18
//     neighbour densities from the ring.
// Each copy fetches one velocity's (A, B) component pair: 8 bytes for FP32,
// one 4-byte word for FP16/BF16.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace lbgb {

namespace {

constexpr int kTX = 32;
static_assert(kTX == kTileX, "the bounce-back tile lists assume the box kernel's strip width");
constexpr int kMaxTY = 16;

__device__ __forceinline__ int wrap_any(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

__device__ __forceinline__ void cp_async4(uint32_t saddr, const void* gptr) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(saddr), "l"(gptr) : "memory");
}
__device__ __forceinline__ void cp_async8(uint32_t saddr, const void* gptr) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(saddr), "l"(gptr) : "memory");
}
// copy of one component pair (2 elements)
template <typename S>
__device__ __forceinline__ void cp_async_pair(uint32_t saddr, const S* gptr) {
    if constexpr (sizeof(S) == 4) cp_async8(saddr, gptr);
    else cp_async4(saddr, gptr);
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

struct Smem {
    unsigned char* stage;       // [nst][19][ns] component pairs
    float2* ring;               // [4][tymax + 2][kTX + 2]
    uint32_t* sflag;            // [nst][ns] flag words of the copied nodes
};

// Issue the copies of node (x, y, z) into slot `slot` of stage `st`; records
// its flag word. Solid nodes copy nothing.
template <typename S, bool MASK>
__device__ __forceinline__ void issue_node(const S* __restrict__ src, const uint32_t* __restrict__ flags,
                                           const Geom& g, const AsyncPlan& P, const Smem& sm, int st, int slot,
                                           int x, int y, int z) {
    PullIdx I;
    pull_indices(g, x, y, z, I);
    uint32_t fl = 0;
    if constexpr (MASK) {
        fl = __ldg(flags + I.own);
        sm.sflag[st * P.ns + slot] = fl;
        if (fl & kSolid) return;
    }
    constexpr int PB = 2 * (int)sizeof(S);
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(sm.stage + ((size_t)st * Q * P.ns + slot) * PB);
    static_for<0, Q>([&](auto II) {
        constexpr int i = decltype(II)::value;
        int idx = I.src[i];
        int pop = i;
        if constexpr (MASK && i != 0) {
            if (fl & (1u << i)) { idx = I.own; pop = Vel<i>::opp; }
        }
        cp_async_pair<S>(base + (uint32_t)(i * P.ns * PB), src + pidx(0, pop, idx));
    });
}

// Read the landed copies of a slot into d (deviations) and return the
// density deviations; solid nodes give (-rho0^A, -rho0^B).
template <typename S, bool MASK>
__device__ __forceinline__ float2 consume_node(const AsyncPlan& P, const Smem& sm, const Phys& p, int st, int slot,
                                               float (&d)[2][Q], bool& solid) {
    solid = false;
    if constexpr (MASK) {
        solid = (sm.sflag[st * P.ns + slot] & kSolid) != 0u;
        if (solid) return make_float2(-p.rho0[0], -p.rho0[1]);
    }
    const S* base = reinterpret_cast<const S*>(sm.stage) + ((size_t)st * Q * P.ns + slot) * 2;
#pragma unroll
    for (int i = 0; i < Q; ++i) Store<S>::lds2(base + (size_t)i * P.ns * 2, d[0][i], d[1][i]);
    return make_float2(dens_sum(d[0]), dens_sum(d[1]));
}

template <typename S, bool MASK>
__global__ void __launch_bounds__(kTX * kMaxTY, 1)
fused_async_kernel(const S* __restrict__ src, S* __restrict__ dst, const uint32_t* __restrict__ flags,
                   float* __restrict__ mom_out, Geom g, Phys p, AsyncPlan P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem sm;
    sm.stage = smem_raw;
    sm.ring = reinterpret_cast<float2*>(sm.stage + (size_t)P.nst * Q * P.ns * 2 * sizeof(S));
    sm.sflag = reinterpret_cast<uint32_t*>(sm.ring + 4 * (P.tymax + 2) * (kTX + 2));
    const int RW = kTX + 2, RH = P.tymax + 2;
    auto ring_at = [&](int slot, int ly, int lx) -> float2& { return sm.ring[(slot * RH + ly + 1) * RW + lx + 1]; };

    const int t = threadIdx.x, tx = t & 31, ty = t >> 5;
    const int cx = blockIdx.x % P.ncols, cy = blockIdx.x / P.ncols;
    const int x0 = cx * kTX;
    const int y0 = (int)(((long long)cy * g.ny) / P.R);
    const int y1 = (int)(((long long)(cy + 1) * g.ny) / P.R);
    const int TYt = y1 - y0;
    const int z0 = blockIdx.y * P.zchunk;
    const int z1 = min(z0 + P.zchunk, g.nz);
    if (z0 >= z1) return;   // uniform over the block
    const int L = (z1 - z0) + 2;   // planes z0 - 1 .. z1

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
    const int own_slot = t, halo_slot = P.threads + t;

    auto plane_of = [&](int e) { return wrap_any(z0 - 1 + e, g.nz); };
    auto issue = [&](int e) {
        if (e < L) {
            const int z = plane_of(e), st = e % P.nst;
            if (own_row) issue_node<S, MASK>(src, flags, g, P, sm, st, own_slot, gx, gy, z);
            if (has_halo) issue_node<S, MASK>(src, flags, g, P, sm, st, halo_slot, hgx, hgy, z);
        }
        cp_commit();   // one group per event, possibly empty, keeps the count uniform
    };

    for (int e = 0; e < P.nst; ++e) issue(e);

    float cur[2][Q], nxt[2][Q];
    bool solid_cur = true;
    for (int e = 0; e < L; ++e) {
        cp_wait_n(P.nst - 1);   // this thread's copies of event e have landed
        const int st = e % P.nst, slot = e & 3;
        bool solid_nxt = true;
        if (own_row) ring_at(slot, ty, tx) = consume_node<S, MASK>(P, sm, p, st, own_slot, nxt, solid_nxt);
        if (has_halo) {
            float dh[2][Q];
            bool sh;
            ring_at(slot, hly, hlx) = consume_node<S, MASK>(P, sm, p, st, halo_slot, dh, sh);
        }
        __syncthreads();   // ring of plane e complete (and every reader of it done)
        issue(e + P.nst);  // refill this thread's own slots of stage st
        if (e >= 2 && active) {
            const int z = plane_of(e - 1);
            const long long own = gx + (long long)g.nx * (gy + (long long)g.ny * z);
            const int sm_m = (e - 2) & 3, sm_c = (e - 1) & 3, sm_p = e & 3;
            if (!solid_cur) {
                float dA, dB, j[3];
                sums<S>(cur, dA, dB, j);
                float SA[3], SB[3];
                neighbour_sums<kFactoredSums<S>>(
                    [&](int dx, int dy, int dz) {
                        const int s = dz < 0 ? sm_m : (dz > 0 ? sm_p : sm_c);
                        return ring_at(s, ty + dy, tx + dx);
                    },
                    SA, SB);
                if (mom_out != nullptr) store_moments(mom_out, g, own, dA, dB, j, SA, SB);
                collide_store<S>(cur, p, dA, dB, j, SA, SB, dst, g, (int)own);
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

// ---------------------------------------------------------------------------
// Box variant (used when nx is a multiple of 4): per plane and velocity the
// block copies one box of rows -- the tile and its halo shifted by -c_i, both
// components -- in 16-byte chunks, cooperatively, each chunk's source wrapped
// periodically on its own (a chunk never straddles the wrap since nx and the
// tile origin are multiples of the chunk width, nor a storage block). A stage
// is laid out [box row][velocity][column][component], so the pulled pair of
// node (lx, ly) for velocity i sits at row ly + 1, column lx + PAD - c_ix: one
// shared-memory vector load at a compile-time offset from a per-node base.

template <typename S> struct BoxGeo {
    static constexpr int CS = 16 / (2 * (int)sizeof(S));   // sites per 16-byte chunk
    static constexpr int PAD = CS;                         // box columns left of the tile
    static constexpr int BW = kTX + 2 * PAD;               // box width (sites)
    static constexpr int CPR = BW / CS;                    // chunks per velocity and box row
    static constexpr int VS = 2 * BW;                      // velocity stride in a stage row (elements)
    // stage row stride (elements): the 19 boxes of a row, padded to 16 bytes
    // mod 128 so that the column-halo nodes of consecutive rows spread over
    // the banks
    static constexpr int ROW0B = Q * VS * (int)sizeof(S);
    static constexpr int ROW = (ROW0B + ((16 - ROW0B % 128) + 128) % 128) / (int)sizeof(S);
    static_assert((ROW * (int)sizeof(S)) % 16 == 0, "stage rows must stay 16-byte aligned");
};

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* gptr) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(gptr) : "memory");
}

// MODEL 0: Shan-Chen (the ring holds the density deviations psi - rho0);
// MODEL 1: colour gradient (the ring holds the phase field Theta, whose
// neighbour sums give grad Theta; no mask).
template <typename S, bool MASK, int MODEL = 0>
__global__ void __launch_bounds__(kTX * kMaxTY, 1)
fused_box_kernel(const S* __restrict__ src, S* __restrict__ dst, const uint32_t* __restrict__ flags,
                 float* __restrict__ mom_out, Geom g, Phys p, AsyncPlan P, LinkTiles LT) {
    constexpr bool CG = MODEL == 1;
    // what a node contributes to the ring: its density deviations, or Theta
    auto ring_val = [&](float2 d) -> float2 {
        if constexpr (CG) {
            const float t = phase_field(p, d.x, d.y);
            return make_float2(t, t);
        } else {
            return d;
        }
    };
    using B = BoxGeo<S>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int RH = P.tymax + 2, RW = kTX + 2;
    const size_t pop_bytes = (size_t)RH * B::ROW * sizeof(S);
    const size_t stage_bytes = pop_bytes + (MASK ? (size_t)RH * 40 * 4 : 0);
    auto stage_base = [&](int st) -> S* { return reinterpret_cast<S*>(smem_raw + (size_t)st * stage_bytes); };
    auto stage_flags = [&](int st) -> uint32_t* {
        return reinterpret_cast<uint32_t*>(smem_raw + (size_t)st * stage_bytes + pop_bytes);
    };
    float2* ring = reinterpret_cast<float2*>(smem_raw + (size_t)P.nst * stage_bytes);
    auto ring_at = [&](int slot, int ly, int lx) -> float2& { return ring[(slot * RH + ly + 1) * RW + lx + 1]; };

    const int t = threadIdx.x, tx = t & 31, ty = t >> 5;
    const int cx = blockIdx.x % P.ncols, cy = blockIdx.x / P.ncols;
    const int x0 = cx * kTX;
    const int y0 = (int)(((long long)cy * g.ny) / P.R);
    const int y1 = (int)(((long long)(cy + 1) * g.ny) / P.R);
    const int TYt = y1 - y0;
    const int z0 = blockIdx.y * P.zchunk;
    const int z1 = min(z0 + P.zchunk, g.nz);
    if (z0 >= z1) return;
    const int L = (z1 - z0) + 2;

    const bool own_row = ty < TYt;
    const int gx = wrap_any(x0 + tx, g.nx);
    const int gy = own_row ? y0 + ty : y0;
    const bool active = own_row && (x0 + tx < g.nx);
    // halo nodes go to the last threads (the first ones issue the copies)
    const int nh = 2 * RW + 2 * TYt;
    const int h = t - (P.threads - nh);
    const bool has_halo = h >= 0;
    int hlx = 0, hly = 0;
    if (h < RW) { hlx = h - 1; hly = -1; }
    else if (h < 2 * RW) { hlx = h - RW - 1; hly = TYt; }
    else if (h < 2 * RW + TYt) { hlx = -1; hly = h - 2 * RW; }
    else { hlx = kTX; hly = h - 2 * RW - TYt; }
    const int hgx = wrap_any(x0 + hlx, g.nx), hgy = wrap_any(y0 + hly, g.ny);

    auto plane_of = [&](int e) { return wrap_any(z0 - 1 + e, g.nz); };

    // In-tile bounce-back links (masked Shan-Chen grids): the links whose
    // source node lies in plane z0 + e - 3 are copied across two events --
    // event e fetches the entry after its first barrier and loads the source
    // slot after its collision; event e + 1 stores the target slot, after its
    // second barrier (FP32) or after its collision (16-bit storage; each
    // placement measured faster for its precision). By then every plane they
    // touch (z - 1, z, z + 1 of the tile, inside this z-chunk) was written by
    // this block before a barrier, and both slots are recent writes still in
    // L2. Thread t takes entry t of a list; a longer list's rest is copied in
    // one go at the store point. The list offsets of planes z0 .. z1 sit
    // after the ring.
    using LP = typename Store<S>::Pair;
    constexpr bool kLinks = MASK && MODEL == 0;
    constexpr bool kLateStore = sizeof(S) == 2;
    const bool links = kLinks && LT.ent != nullptr;
    uint32_t* lstart = reinterpret_cast<uint32_t*>(ring + 4 * RH * RW);
    if (links)
        for (int k = t; k <= z1 - z0; k += P.threads) lstart[k] = __ldg(LT.start + (size_t)blockIdx.x * g.nz + z0 + k);
    // the links of list plane zl beyond the first P.threads, or all from k0 on
    auto copy_links = [&](int zl, uint32_t k0) {
        const uint32_t a = lstart[zl], n = lstart[zl + 1] - a;
        for (uint32_t k = k0; k < n; k += (uint32_t)P.threads) {
            const LinkSlots ls = tile_link_slots(__ldg(LT.ent + a + k), x0, y0, z0 + zl, g);
            *reinterpret_cast<LP*>(dst + ls.dst) = __ldcg(reinterpret_cast<const LP*>(dst + ls.src));
        }
    };
    uint32_t lent = 0u, lent_p = 0u;
    bool lhave = false, lhave_p = false;
    LP lval{};
    // targets of list plane zl, whose sources were loaded one event earlier
    auto store_links = [&](int zl) {
        if (lhave_p) *reinterpret_cast<LP*>(dst + tile_link_slots(lent_p, x0, y0, z0 + zl, g).dst) = lval;
        copy_links(zl, (uint32_t)(t + P.threads));
    };

    // Copier thread t (< RH * CPR) owns chunk (row jr, column jc) of all 19
    // boxes. Its wrapped source offsets within a plane depend only on c_iy
    // and are computed once; on masked grids threads t < RH * 10 also copy
    // one 4-word chunk of the flag box.
    const bool copier = t < RH * B::CPR;
    const int jr = t / B::CPR, jc = t - (t / B::CPR) * B::CPR;
    const int xs_chunk = wrap_any(x0 - B::PAD + jc * B::CS, g.nx);
    const int yoff_m = wrap_any(y0 + jr, g.ny) * g.nx + xs_chunk;       // c_iy = -1
    const int yoff_0 = wrap_any(y0 - 1 + jr, g.ny) * g.nx + xs_chunk;   // c_iy =  0
    const int yoff_p = wrap_any(y0 - 2 + jr, g.ny) * g.nx + xs_chunk;   // c_iy = +1
    const int sdst = jr * B::ROW + jc * B::CS * 2;
    const bool fcopier = MASK && t < RH * 10;
    int foff = 0, fdst = 0;
    if (fcopier) {
        const int fr = t / 10, fc = t - (t / 10) * 10;
        foff = wrap_any(y0 - 1 + fr, g.ny) * g.nx + wrap_any(x0 - 4 + fc * 4, g.nx);
        fdst = fr * 40 + fc * 4;
    }

    // copies of event e (plane z, stage st) into the stage
    auto issue = [&](int e, int z, int st) {
        if (e < L) {
            if (copier) {
                // plane offsets for c_iz = -1, 0, +1 (source plane z - c_iz)
                const size_t pz_m = (size_t)wrap_inc(z, g.nz) * g.plane;
                const size_t pz_0 = (size_t)z * g.plane;
                const size_t pz_p = (size_t)wrap_dec(z, g.nz) * g.plane;
                const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(stage_base(st) + sdst);
                static_for<0, Q>([&](auto II) {
                    constexpr int i = decltype(II)::value;
                    const size_t pz = Vel<i>::z < 0 ? pz_m : (Vel<i>::z > 0 ? pz_p : pz_0);
                    const int yo = Vel<i>::y < 0 ? yoff_m : (Vel<i>::y > 0 ? yoff_p : yoff_0);
                    // a chunk starts at a multiple of CS sites and so lies inside one block
                    cp_async16(sbase + i * B::VS * (int)sizeof(S),
                               src + blk_base((uint32_t)(pz + yo)) + i * (2 * kBlk));
                });
            }
            if constexpr (MASK) {
                if (fcopier)
                    cp_async16((uint32_t)__cvta_generic_to_shared(stage_flags(st) + fdst),
                               flags + (size_t)z * g.plane + foff);
            }
        }
        cp_commit();
    };

    // pulled deviations of node (lx, ly) from stage st. A population whose
    // source node is solid was stored in that solid node's slot by the
    // write-side bounce-back, so every pull is the same box read.
    // (solid lanes read finite placeholders and report psi = 0)
    auto read_node = [&](int st, int lx, int ly, float (&d)[2][Q], uint32_t& fl) -> float2 {
        fl = MASK ? stage_flags(st)[(ly + 1) * 40 + lx + 4] : 0u;
        const S* nb = stage_base(st) + (ly + 1) * B::ROW + (lx + B::PAD) * 2;
        static_for<0, Q>([&](auto II) {
            constexpr int i = decltype(II)::value;
            Store<S>::lds2(nb + i * B::VS - 2 * Vel<i>::x, d[0][i], d[1][i]);
        });
        if (MASK && (fl & kSolid)) return make_float2(-p.rho0[0], -p.rho0[1]);
        return make_float2(dens_sum(d[0]), dens_sum(d[1]));
    };
    // density deviations of a node whose populations are not kept (16-bit
    // storage: both components summed at once)
    auto read_density = [&](int st, int lx, int ly) -> float2 {
        if constexpr (sizeof(S) == 2) {
            if (MASK && (stage_flags(st)[(ly + 1) * 40 + lx + 4] & kSolid)) return make_float2(-p.rho0[0], -p.rho0[1]);
            const S* nb = stage_base(st) + (ly + 1) * B::ROW + (lx + B::PAD) * 2;
            float2 d[Q];
            static_for<0, Q>([&](auto II) {
                constexpr int i = decltype(II)::value;
                d[i] = Store<S>::lds2v(nb + i * B::VS - 2 * Vel<i>::x);
            });
            return dens_sum2(d);
        } else {
            float d[2][Q];
            uint32_t fl;
            return read_node(st, lx, ly, d, fl);
        }
    };
    // 16-bit storage, own node: the pairs stay packed (one word per velocity)
    // until the collision; the momentum is taken here, from the same values
    auto read_node_packed = [&](int st, int lx, int ly, uint32_t (&w)[Q], float (&j)[3], uint32_t& fl) -> float2 {
        fl = MASK ? stage_flags(st)[(ly + 1) * 40 + lx + 4] : 0u;
        const S* nb = stage_base(st) + (ly + 1) * B::ROW + (lx + B::PAD) * 2;
        float2 d[Q];
        static_for<0, Q>([&](auto II) {
            if constexpr (sizeof(S) == 2) {
                constexpr int i = decltype(II)::value;
                w[i] = *reinterpret_cast<const uint32_t*>(nb + i * B::VS - 2 * Vel<i>::x);
                d[i] = Store<S>::unpack2(w[i]);
            }
        });
        momentum2<kPackedSums<S>>(d, j);
        if (MASK && (fl & kSolid)) return make_float2(-p.rho0[0], -p.rho0[1]);
        return dens_sum2(d);
    };

    // 16-bit storage (three or four stages fit): the copies of event
    // e + nst - 1 are issued right after the first barrier of event e, into
    // the stage read at event e - 1, so that the copier warps do that work
    // while the halo warps read their extra node. FP32 (two stages): they are
    // issued after the second barrier into the stage just read (event e + nst).
    constexpr bool early = sizeof(S) == 2;
    const int ahead = early ? P.nst - 1 : P.nst;   // events in flight
    // planes and stages advance by one per event; tracked incrementally
    const int zfirst = wrap_any(z0 - 1, g.nz);
    {
        int z = zfirst;
        for (int e = 0; e < ahead; ++e) {
            issue(e, z, e);
            z = wrap_inc(z, g.nz);
        }
    }
    int z_cur = zfirst, z_prev = zfirst, st_cur = 0;
    int z_iss = wrap_any(z0 - 1 + ahead, g.nz);   // plane of event e + ahead
    const int own_off = (ty + 1) * RW + tx + 1;   // this node's ring cell within a slot

    // own populations between their read (event e) and their collision
    // (event e + 1): floats for FP32, packed pair words and the momentum for
    // 16-bit storage (fewer live registers). Two holders swap roles on
    // alternate events (the loop is unrolled by two), so nothing is copied.
    constexpr bool packed = sizeof(S) == 2;
    struct Held {
        float d[2][packed ? 1 : Q];
        uint32_t w[packed ? Q : 1];
        float j[3];
        float2 dd;   // density deviations (16-bit colour gradient: the ring holds Theta)
        uint32_t fl;
    };
    Held h0, h1;
    h0.fl = h1.fl = kSolid;
    // 16-bit storage: plane quantities of the neighbour sums for this column,
    // planes e - 2, e - 1 (held) and e (computed once the ring of plane e is
    // complete); FP32 (fewer free registers) evaluates the same expressions
    // from the ring for each node
    PlaneSums ps_lo, ps_mid;
    ps_lo.dx = ps_lo.dy = ps_lo.t = ps_mid.dx = ps_mid.dy = ps_mid.t = make_float2(0.f, 0.f);
#pragma unroll
    for (int a = 0; a < 3; ++a) h0.j[a] = h1.j[a] = 0.f;

    auto event = [&](int e, Held& cur, Held& nxt) {
        cp_wait_n(ahead - 1);
        __syncthreads();   // every thread's chunks of event e are visible
        if constexpr (early) issue(e + ahead, z_iss, st_cur == 0 ? P.nst - 1 : st_cur - 1);
        if (kLinks && links && e >= 3) {   // entry of plane z0 + e - 3, used after the collision
            const uint32_t a = lstart[e - 3];
            lhave = (uint32_t)t < lstart[e - 2] - a;
            if (lhave) lent = __ldg(LT.ent + a + t);
        }
        const int slot = e & 3;
        nxt.fl = kSolid;
        if (own_row) {
            if constexpr (packed) {
                nxt.dd = read_node_packed(st_cur, tx, ty, nxt.w, nxt.j, nxt.fl);
                ring[slot * RH * RW + own_off] = ring_val(nxt.dd);
            } else {
                ring[slot * RH * RW + own_off] = ring_val(read_node(st_cur, tx, ty, nxt.d, nxt.fl));
            }
        }
        if (has_halo) ring_at(slot, hly, hlx) = ring_val(read_density(st_cur, hlx, hly));
        __syncthreads();   // ring of plane e complete; stage st_cur fully read
        if constexpr (!early) issue(e + ahead, z_iss, st_cur);
        if (kLinks && !kLateStore && links && e >= 4) store_links(e - 4);
        PlaneSums ps_hi;
        if constexpr (packed) {
            const float2* rn = ring + slot * RH * RW + own_off;
            if (own_row) ps_hi = plane_sums(rn[0], rn[1], rn[-1], rn[RW], rn[-RW]);
        }
        // Solid lanes run the same code and store zeros, so that every warp
        // stores whole sectors (a partly written sector costs a DRAM read);
        // the solid slots a fluid node pulls are filled afterwards by the
        // bounce-back pass. (The fl test on unmasked FP32 grids is always
        // true; it is kept because that form schedules measurably faster.)
        if (e >= 2 && active && (MASK || sizeof(S) != 4 || !(cur.fl & kSolid))) {
            const long long own = gx + (long long)g.nx * (gy + (long long)g.ny * z_prev);
            const float2* rc = ring + ((e - 1) & 3) * RH * RW + own_off;
            float dA, dB, j[3];
            if constexpr (!packed) {
                sums<S>(cur.d, dA, dB, j);
            } else {   // own density deviations are already in the ring (same sums)
                dA = CG ? cur.dd.x : rc[0].x;
                dB = CG ? cur.dd.y : rc[0].y;
#pragma unroll
                for (int a = 0; a < 3; ++a) j[a] = cur.j[a];
            }
            float SA[3], SB[3];
            if constexpr (packed) {
                force_sums(ps_lo, ps_mid, ps_hi, rc[RW + 1], rc[RW - 1], rc[1 - RW], rc[-1 - RW], SA, SB);
            } else {
                const float2* rm = ring + ((e - 2) & 3) * RH * RW + own_off;
                const float2* rp = ring + slot * RH * RW + own_off;
                neighbour_sums<kFactoredSums<S>>(
                    [&](int dx, int dy, int dz) {
                        const float2* r = dz < 0 ? rm : (dz > 0 ? rp : rc);
                        return r[dy * RW + dx];
                    },
                    SA, SB);
            }
            const bool solid = MASK && (cur.fl & kSolid);
            if constexpr (CG) {
                // grad Theta = (1 / c_s^2) sum_i w_i c_i Theta(x + c_i)
                const float gt[3] = {3.0f * SA[0], 3.0f * SA[1], 3.0f * SA[2]};
                if constexpr (packed)
                    cg_collide_store_g<S>(
                        [&](int k, int i) {
                            if constexpr (sizeof(S) == 2) return Store<S>::part(cur.w[i], k);
                            else return 0.f;
                        },
                        p, dA, dB, j, gt, dst, (int)own);
                else
                    cg_collide_store_g<S>([&](int k, int i) { return cur.d[k][i]; }, p, dA, dB, j, gt, dst,
                                          (int)own);
            } else {
                if (mom_out != nullptr && !solid) store_moments(mom_out, g, own, dA, dB, j, SA, SB);
                if constexpr (packed)
                    collide_store_g<S, MASK>(
                        [&](int k, int i) {
                            if constexpr (sizeof(S) == 2) return Store<S>::part(cur.w[i], k);
                            else return 0.f;
                        },
                        p, dA, dB, j, SA, SB, dst, g, (int)own, solid);
                else
                    collide_store<S, MASK>(cur.d, p, dA, dB, j, SA, SB, dst, g, (int)own, solid);
            }
        }
        if (kLinks && kLateStore && links && e >= 4) store_links(e - 4);
        if (kLinks && links && e >= 3) {   // sources of plane z0 + e - 3
            lhave_p = lhave;
            lent_p = lent;
            if (lhave) lval = __ldcg(reinterpret_cast<const LP*>(dst + tile_link_slots(lent, x0, y0, z0 + e - 3, g).src));
        }
        if constexpr (packed) {
            ps_lo = ps_mid;
            ps_mid = ps_hi;
        }
        z_prev = z_cur;
        z_cur = wrap_inc(z_cur, g.nz);
        z_iss = wrap_inc(z_iss, g.nz);
        st_cur = st_cur + 1 == P.nst ? 0 : st_cur + 1;
    };
    for (int e = 0; e < L; e += 2) {
        event(e, h0, h1);
        if (e + 1 < L) event(e + 1, h1, h0);
    }
    cp_wait<0>();
    if (kLinks && links) {
        __syncthreads();   // the last plane's stores are visible to the block
        if (L >= 4) store_links(L - 4);   // plane z1 - 2: sources loaded after the last collision
        copy_links(L - 3, (uint32_t)t);   // plane z1 - 1
    }
}

template <typename S, bool MASK, int MODEL = 0>
cudaError_t launch_box_t(const StepLaunch& L, cudaStream_t st) {
    const AsyncPlan& P = L.plan;
    auto kern = fused_box_kernel<S, MASK, MODEL>;
    static size_t configured = 0;
    if (configured < P.smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.smem);
        if (e != cudaSuccess) return e;
        // room for two resident blocks where the plan wants them
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        configured = P.smem;
    }
    dim3 grid(P.ncols * P.R, P.zsplit, 1);
    const LinkTiles lt = tiles_in_kernel(L) ? L.links.tiles : LinkTiles{};
    kern<<<grid, P.threads, P.smem, st>>>(static_cast<const S*>(L.src), static_cast<S*>(L.dst), L.flags, L.mom_out,
                                          L.g, L.p, P, lt);
    return cudaGetLastError();
}

template <typename S, bool MASK>
cudaError_t launch_t(const StepLaunch& L, cudaStream_t st) {
    const AsyncPlan& P = L.plan;
    auto kern = fused_async_kernel<S, MASK>;
    static size_t configured = 0;   // the attribute is per function
    if (configured < P.smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.smem);
        if (e != cudaSuccess) return e;
        configured = P.smem;
    }
    dim3 grid(P.ncols * P.R, P.zsplit, 1);
    kern<<<grid, P.threads, P.smem, st>>>(static_cast<const S*>(L.src), static_cast<S*>(L.dst), L.flags, L.mom_out,
                                          L.g, L.p, P);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fused_async(const StepLaunch& L, cudaStream_t st) {
    const bool m = L.flags != nullptr;
    if (L.p.model == 1) {   // colour gradient: periodic, box kernel only (the caller checks plan.box)
        switch (L.prec) {
            case 0: return launch_box_t<float, false, 1>(L, st);
            case 1: return launch_box_t<__half, false, 1>(L, st);
            case 2: return launch_box_t<__nv_bfloat16, false, 1>(L, st);
            default: return cudaErrorInvalidValue;
        }
    }
    if (L.plan.box) {
        switch (L.prec) {
            case 0: return m ? launch_box_t<float, true>(L, st) : launch_box_t<float, false>(L, st);
            case 1: return m ? launch_box_t<__half, true>(L, st) : launch_box_t<__half, false>(L, st);
            case 2: return m ? launch_box_t<__nv_bfloat16, true>(L, st) : launch_box_t<__nv_bfloat16, false>(L, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (L.prec) {
        case 0: return m ? launch_t<float, true>(L, st) : launch_t<float, false>(L, st);
        case 1: return m ? launch_t<__half, true>(L, st) : launch_t<__half, false>(L, st);
        case 2: return m ? launch_t<__nv_bfloat16, true>(L, st) : launch_t<__nv_bfloat16, false>(L, st);
        default: return cudaErrorInvalidValue;
    }
}

AsyncPlan plan_fused_async(int nx, int ny, int nz, int sm_count, int prec, bool masked, int model,
                           size_t smem_limit) {
    AsyncPlan best{};
    double best_cost = 1e300;
    const int ncols = (nx + kTX - 1) / kTX;
    const int esize = prec == 0 ? 4 : 2;
    // chunks of component pairs (2 or 4 sites) and of flag words (4 sites)
    const bool box = (nx % 4) == 0;
    const int cpr = prec == 0 ? BoxGeo<float>::CPR : BoxGeo<__half>::CPR;
    const size_t row_bytes = prec == 0 ? (size_t)BoxGeo<float>::ROW * 4 : (size_t)BoxGeo<__half>::ROW * 2;
    const int rmin = (ny + kMaxTY - 1) / kMaxTY;
    for (int R = rmin; R <= ny; ++R) {
        const int tymax = (ny + R - 1) / R;
        if (tymax < 4 && R > rmin && ny >= 4) break;
        const int threads = kTX * tymax;
        const int ns = threads + 2 * (kTX + 2) + 2 * tymax;
        if (threads < 2 * (kTX + 2) + 2 * tymax) continue;   // every halo node needs a thread
        if (box && threads < (tymax + 2) * cpr) continue;   // a chunk per copier thread
        const size_t stage = box ? (size_t)(tymax + 2) * row_bytes + (masked ? (size_t)(tymax + 2) * 40 * 4 : 0)
                                 : (size_t)Q * ns * 2 * esize + (masked ? (size_t)ns * 4 : 0);
        const size_t ring = (size_t)4 * (tymax + 2) * (kTX + 2) * 8;
        const long long bxy = (long long)ncols * R;
        const int zs_max = nz / 4 > 1 ? nz / 4 : 1;
        for (int zs = 1; zs <= zs_max; ++zs) {
            const int zchunk = (nz + zs - 1) / zs;
            // masked box kernel: the bounce-back list offsets of the chunk's planes
            const size_t lists = masked && box ? ((size_t)(zchunk + 1) * 4 + 15) / 16 * 16 : 0;
            if (smem_limit < ring + lists + 2 * stage) continue;
            int nst = (int)((smem_limit - ring - lists) / stage);
            nst = nst > 4 ? 4 : nst;
            const long long blocks = bxy * zs;
            const long long waves = (blocks + sm_count - 1) / sm_count;
            // per-block time ~ columns (own + 30% weight for halo nodes) x planes
            // (+2 halo planes), and blocks of few warps hide latency worse
            const double work = (tymax + 0.3 * (2.0 * (kTX + 2) + 2.0 * tymax) / kTX) * (zchunk + 2);
            const double cost = waves * work * (1.0 + 4.0 / tymax);
            if (cost < best_cost * (1 - 1e-9)) {
                best_cost = cost;
                best.ncols = ncols;
                best.R = R;
                best.tymax = tymax;
                best.zsplit = zs;
                best.zchunk = zchunk;
                best.nst = nst;
                best.threads = threads;
                best.ns = ns;
                best.smem = ring + lists + (size_t)nst * stage;
                best.box = box ? 1 : 0;
            }
            if (blocks >= sm_count) break;   // more z-splits only add halo planes
        }
    }
    // 16-bit storage on masked grids, for the colour gradient (the heavier
    // per-node work) and for BF16: where short tiles fill exactly one wave of
    // two resident blocks per SM (half of the SM's shared memory each), take
    // them instead, so that the two blocks' barriers interleave. Measured at
    // 256^3: colour gradient FP16 +0.7 % (with its lean collision; +19 %
    // before), masked FP16 +5.7 % (colloid mask, with the lean BGK), unmasked
    // Shan-Chen BF16 +1.1 %; unmasked Shan-Chen FP16 -0.4 %, FP32 -3 % and
    // masked FP32 (two stages each) -4 % (those keep one block of tall
    // tiles).
    if (esize == 2 && box && best.zsplit == 1 && (masked || model == 1 || prec == 2)) {
        const size_t half_limit = (smem_limit + 1024) / 2 - 1024;
        for (int R = best.R + 1; R <= ny && (long long)ncols * R <= 2LL * sm_count; ++R) {
            if ((long long)ncols * R != 2LL * sm_count) continue;
            const int tymax = (ny + R - 1) / R;
            const int threads = kTX * tymax;
            const int ns = threads + 2 * (kTX + 2) + 2 * tymax;
            if (threads < 2 * (kTX + 2) + 2 * tymax || threads < (tymax + 2) * cpr) continue;
            const size_t stage = (size_t)(tymax + 2) * row_bytes + (masked ? (size_t)(tymax + 2) * 40 * 4 : 0);
            const size_t ring = (size_t)4 * (tymax + 2) * (kTX + 2) * 8;
            const size_t lists = masked ? ((size_t)(nz + 1) * 4 + 15) / 16 * 16 : 0;
            if (half_limit < ring + lists + 3 * stage) continue;
            int nst = (int)((half_limit - ring - lists) / stage);
            nst = nst > 4 ? 4 : nst;
            best.R = R;
            best.tymax = tymax;
            best.zsplit = 1;
            best.zchunk = nz;
            best.nst = nst;
            best.threads = threads;
            best.ns = ns;
            best.smem = ring + lists + (size_t)nst * stage;
            break;
        }
    }
    return best;
}

}  // namespace lbgb
