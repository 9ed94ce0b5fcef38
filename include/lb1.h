/* lb1.h -- one-component D3Q19 BGK lattice-Boltzmann step (the paper's
 * single-fluid case, Sec. 5 "Single fluid": plain BGK, Eq. bgk with the
 * Eq. LEQ equilibrium, fused streaming; periodic grids).
 *
 * Same conventions as lb.h: plain pointers and sizes, no allocation (the
 * caller provides one device workspace), status codes (lb_status from lb.h),
 * all work asynchronous on the caller's stream unless stated. Populations are
 * stored as deviations d_i = f_i - w_i rho0 (FP32, FP16 or BF16, FP32
 * arithmetic), in blocks of 64 sites: element (i, s) at
 * (s / 64) * 19 * 64 + i * 64 + s mod 64. The state held is the
 * post-collision g of the last step; a step pulls f_i(x) = g_i(x - c_i),
 * computes rho, u = j / rho + tau g (body force g as a velocity shift) and
 * relaxes: g_i = f_i - (f_i - f_i^eq(rho, u)) / tau.
 */
#ifndef LB1_H
#define LB1_H

#include <stddef.h>
#include <stdint.h>

#include "lb.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb1_ctx lb1_ctx;

/* Bytes of device workspace for an nx x ny x nz grid with storage prec
 * (lb_precision): two population buffers and reduction scratch. Returns 0 for
 * invalid sizes (each >= 3, nx*ny*nz < 2^31) or precision. Host function. */
size_t lb1_workspace_bytes(int nx, int ny, int nz, int prec);

/* Create a context over the caller's workspace.
 *   tau          > 0.5, finite (nu = (tau - 1/2) / 3, Eq. viscosity).
 *   body_force   HOST pointer to 3 doubles (g), or NULL for 0.
 *   prec         lb_precision.
 *   d_workspace  device pointer, 256-byte aligned, ws_bytes >= lb1_workspace_bytes.
 *   stream       a cudaStream_t (NULL = legacy default stream).
 * nx must be a multiple of 4 (FP32) or 8 (16-bit storage): the step copies
 * 16-byte chunks of x rows. Errors: LB_EINVAL (sizes, parameters, alignment),
 * LB_ENOMEM (short workspace), LB_ECUDA. */
lb_status lb1_create(int nx, int ny, int nz, float tau, const double* body_force, int prec,
                     void* d_workspace, size_t ws_bytes, void* stream, lb1_ctx** out);

/* Initial state f_i = f_i^eq(rho, u) from DEVICE fields d_rho (N floats,
 * > 0) and d_u (3N floats SoA, or NULL = 0); rho0 = mean of d_rho.
 * LB_EINVAL if a density is <= 0 or an input is not finite. Synchronous. */
lb_status lb1_init(lb1_ctx* ctx, const float* d_rho, const float* d_u);

/* Advance n >= 1 steps (one kernel launch per step). */
lb_status lb1_step(lb1_ctx* ctx, int n);

/* DEVICE outputs: density rho (N floats) and velocity u = (j + rho g / 2) / rho
 * (3N floats SoA); either may be NULL. */
lb_status lb1_moments(lb1_ctx* ctx, float* d_rho, float* d_u);

/* FP64 totals of the state (mass, Px, Py, Pz) into HOST out4; synchronous. */
lb_status lb1_stats(lb1_ctx* ctx, double out4[4]);

/* Post-streaming populations f_i(x) into DEVICE d_f (19 N floats, [i][s], the
 * velocity order of lb.h). */
lb_status lb1_get_state(lb1_ctx* ctx, float* d_f);

/* Launch geometry of the step kernel (for reporting); any pointer may be NULL. */
lb_status lb1_launch_info(const lb1_ctx* ctx, int* blocks, int* threads);

void lb1_destroy(lb1_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LB1_H */
