// lb_noalloc.cu -- lb_moments_noalloc: densities and velocity of a caller's
// population field with no device allocation and no caller workspace.
//
// Who needs it: code that may not call cudaMalloc (or any allocator) on the
// device -- for example a host application whose device memory is owned by
// another framework's pool, a plugin running inside a process that forbids
// allocation after start-up, or a caller that only holds a population field
// (exported with lb_get_state or written by its own code) and the output
// buffers. Such a caller has no way to provide lb_create's workspace.
//
// The force sums of the velocity need the densities of neighbouring nodes,
// which a first kernel writes to scratch memory. That scratch lives in a
// file-scope __device__ array of fixed size (kMaxNodes nodes, 8 MiB), which
// every GPU that loads this library holds until the process exits. Host code
// cannot use the array's name as a device address, so the first call on each
// device looks the address up with cudaGetSymbolAddress (with that device
// current) and caches it; make that first call before any stream capture.
// Every call reuses the same array and leaves its contents behind; the density
// kernel rewrites every entry the moments kernel reads, so nothing has to be
// cleared. Calls that overlap on the GPU (on different streams, or from
// different threads) race on the array: serialise them.
#include <cmath>
#include <cstdio>
#include <mutex>

#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"
#include "lb.h"

namespace lbgb {
namespace {

constexpr long long kMaxNodes = 1LL << 20;   // 2 floats per node: 8 MiB
constexpr int kMaxDevices = 256;

static __device__ __align__(256) float g_psi_scratch[2 * kMaxNodes];

std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(float** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (g_scratch_ptr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_psi_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<float*>(g_scratch_ptr[dev]);
    return cudaSuccess;
}

__device__ __forceinline__ void node_xyz(long long s, const Geom& g, int& x, int& y, int& z) {
    x = (int)(s % g.nx);
    y = (int)((s / g.nx) % g.ny);
    z = (int)(s / g.plane);
}

// psi^k(s) = sum_i f_i^k(s) at fluid nodes, 0 at solid nodes.
__global__ void psi_kernel(const float* __restrict__ f, const uint8_t* __restrict__ mask,
                           float* __restrict__ psi, Geom g) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.N) return;
    const bool fluid = !(mask && mask[s]);
    float a = 0.f, b = 0.f;
    if (fluid)
        for (int i = 0; i < Q; ++i) {
            a += f[(size_t)i * g.N + s];
            b += f[(size_t)(Q + i) * g.N + s];
        }
    psi[s] = a;
    psi[g.N + s] = b;
}

// rho^k = sum_i f_i^k and u = (sum_k sum_i c_i f_i^k + (F^A + F^B)/2) / rho,
// F^A = -G psi^A sum_i w_i psi^B(x + c_i) c_i + rho^A g (and A <-> B).
// The momentum is summed over opposite pairs, c_i (f_i - f_opp(i)), whose
// differences are exact for the close values of a near-rest node. A node
// treated as fluid whose populations are all zero (a covered node of a state
// exported without its sphere coverage) has no velocity: u = 0 there.
__global__ void moments_from_f_kernel(const float* __restrict__ f, const uint8_t* __restrict__ mask,
                                      const float* __restrict__ psi, float* __restrict__ oA,
                                      float* __restrict__ oB, float* __restrict__ ou, Geom g, float G,
                                      float gx, float gy, float gz) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.N) return;
    if (mask && mask[s]) {
        if (oA) oA[s] = 0.f;
        if (oB) oB[s] = 0.f;
        if (ou) ou[s] = ou[g.N + s] = ou[2 * g.N + s] = 0.f;
        return;
    }
    int x, y, z;
    node_xyz(s, g, x, y, z);
    float rA = 0.f, rB = 0.f, j[3] = {0.f, 0.f, 0.f};
    float fa[Q], fb[Q];
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        fa[i] = f[(size_t)i * g.N + s];
        fb[i] = f[(size_t)(Q + i) * g.N + s];
        rA += fa[i];
        rB += fb[i];
    });
    static_for<0, 9>([&](auto M) {
        constexpr int i = 2 * decltype(M)::value + 1;   // (i, i + 1) are opposite
        const float diff = (fa[i] - fa[i + 1]) + (fb[i] - fb[i + 1]);
        if constexpr (Vel<i>::x != 0) j[0] += Vel<i>::x * diff;
        if constexpr (Vel<i>::y != 0) j[1] += Vel<i>::y * diff;
        if constexpr (Vel<i>::z != 0) j[2] += Vel<i>::z * diff;
    });
    if (oA) oA[s] = rA;
    if (oB) oB[s] = rB;
    if (!ou) return;
    float SA[3], SB[3];
    neighbour_sums<false>(
        [&](int dx, int dy, int dz) {
            const int xx = dx > 0 ? wrap_inc(x, g.nx) : (dx < 0 ? wrap_dec(x, g.nx) : x);
            const int yy = dy > 0 ? wrap_inc(y, g.ny) : (dy < 0 ? wrap_dec(y, g.ny) : y);
            const int zz = dz > 0 ? wrap_inc(z, g.nz) : (dz < 0 ? wrap_dec(z, g.nz) : z);
            const long long t = xx + (long long)g.nx * (yy + (long long)g.ny * zz);
            return make_float2(psi[t], psi[g.N + t]);
        },
        SA, SB);
    const float gv[3] = {gx, gy, gz};
    if (rA + rB == 0.f) {
        ou[s] = ou[g.N + s] = ou[2 * g.N + s] = 0.f;
        return;
    }
    const float inv = 1.0f / (rA + rB);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float F = -G * (rA * SB[a] + rB * SA[a]) + (rA + rB) * gv[a];
        ou[a * g.N + s] = (j[a] + 0.5f * F) * inv;
    }
}

}  // namespace
}  // namespace lbgb

extern "C" lb_status lb_moments_noalloc(int nx, int ny, int nz, float G, const double* body_force,
                                        const float* d_f, const uint8_t* d_mask, float* d_rhoA, float* d_rhoB,
                                        float* d_u, void* stream) {
    using namespace lbgb;
    if (nx < 3 || ny < 3 || nz < 3 || !d_f || !std::isfinite(G)) return LB_EINVAL;
    // each side alone within the limit first, so that the product cannot overflow
    const bool side_ok = nx <= kMaxNodes && ny <= kMaxNodes && nz <= kMaxNodes;
    const long long N = side_ok ? (long long)nx * ny * nz : kMaxNodes + 1;
    if (N > kMaxNodes) {   // beyond the static scratch
        char msg[160];
        std::snprintf(msg, sizeof msg,
                      "lb_moments_noalloc: nx*ny*nz = %d*%d*%d exceeds the static scratch limit of %lld nodes",
                      nx, ny, nz, kMaxNodes);
        record_error_text(msg);
        return LB_EINVAL;
    }
    float g3[3] = {0.f, 0.f, 0.f};
    if (body_force)
        for (int a = 0; a < 3; ++a) {
            if (!std::isfinite(body_force[a])) return LB_EINVAL;
            g3[a] = (float)body_force[a];
        }
    float* psi = nullptr;
    cudaError_t e = scratch_address(&psi);
    if (e != cudaSuccess) {
        record_error_text("lb_moments_noalloc: cudaGetSymbolAddress of the static scratch failed");
        return LB_ECUDA;
    }
    Geom g{};
    g.nx = nx; g.ny = ny; g.nz = nz;
    g.plane = nx * ny;
    g.N = N;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const unsigned nb = (unsigned)((N + 255) / 256);
    psi_kernel<<<nb, 256, 0, st>>>(d_f, d_mask, psi, g);
    if ((e = cudaGetLastError()) == cudaSuccess)
        moments_from_f_kernel<<<nb, 256, 0, st>>>(d_f, d_mask, psi, d_rhoA, d_rhoB, d_u, g, G, g3[0], g3[1], g3[2]);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "lb_moments_noalloc: %s", cudaGetErrorString(e));
        record_error_text(msg);
        return LB_ECUDA;
    }
    return LB_OK;
}
