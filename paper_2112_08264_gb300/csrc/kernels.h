// kernels.h -- host-side launchers of the device kernels (internal to the
// library; the public interface is include/lb.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"
#include "reduce.cuh"

namespace lbgb {

// One time step: src (post-collision state) -> dst.
struct StepLaunch {
    int prec;                 // 0 fp32, 1 fp16 deviation, 2 bf16 deviation
    int kernel;               // 0 fused, 1 two-pass
    const void* src;
    void* dst;
    const uint32_t* flags;    // nullptr = no solid nodes
    float* rho;               // density scratch (two-pass), 2N floats
    float* rho_out;           // optional: density deviations psi - rho0 of the source state, 2N
    Geom g;
    Phys p;
    int zsplit;               // fused: z-chunks per tile column
};

cudaError_t launch_step(const StepLaunch& L, cudaStream_t st);

// Fused-kernel launch geometry for a grid on a device with sm_count SMs.
void fused_geometry(int nx, int ny, int nz, int sm_count, int* tiles, int* zsplit, int* threads);

// Solid flags from a device mask (1 = solid).
cudaError_t launch_flags(const uint8_t* mask, uint32_t* flags, const Geom& g, cudaStream_t st);

// Internal state from a post-streaming population field: either the
// equilibrium of (rhoA, rhoB, u) (f == nullptr) or the given f (float,
// [k][i][s]). Inverse of the pull: g_j(y) = f_j(y + c_j) if y + c_j is fluid,
// else f_opp(j)(y).
cudaError_t launch_unstream(int prec, void* dst, const uint32_t* flags, const float* f,
                            const float* rhoA, const float* rhoB, const float* u, const Geom& g,
                            const Phys& p, cudaStream_t st);

// Post-streaming populations (float, [k][i][s]; 0 on solid nodes).
cudaError_t launch_get_state(int prec, const void* src, const uint32_t* flags, float* f, const Geom& g,
                             const Phys& p, cudaStream_t st);

// Density deviations psi - rho0 (into rho, 2N) and moments rhoA, rhoB, u.
cudaError_t launch_densities(int prec, const void* src, const uint32_t* flags, float* rho, const Geom& g,
                             const Phys& p, cudaStream_t st);
cudaError_t launch_moments(int prec, const void* src, const uint32_t* flags, const float* rho,
                           float* rhoA, float* rhoB, float* u, const Geom& g, const Phys& p,
                           cudaStream_t st);

// FP64 conserved totals: partials[kRedBlocks][kRedVals] then out[kRedVals] =
// {mass A, mass B, Px, Py, Pz, non-finite count}.
cudaError_t launch_stats(int prec, const void* src, const uint32_t* flags, double* partials, double* out,
                         const Geom& g, const Phys& p, cudaStream_t st);

// Checks of lb_init inputs over fluid nodes: out = {sum rhoA, sum rhoB,
// fluid count, bad count (rho <= 0 or not finite), 0, 0}.
cudaError_t launch_check_init(const float* rhoA, const float* rhoB, const float* u, const uint32_t* flags,
                              double* partials, double* out, const Geom& g, cudaStream_t st);

// Message returned by lb_last_error() (host code only).
void record_error_text(const char* msg);

}  // namespace lbgb
