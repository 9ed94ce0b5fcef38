// adjoint.h -- reverse-mode step (internal to the library).
//
// Forward map of one step on the post-streaming populations f:
//   f_{t+1} = P(C(f_t)),
// P = streaming with halfway bounce-back (a permutation of the fluid
// populations), C = the per-node BGK collision with the Shan-Chen velocity
// shift, which couples a node to its neighbours through the force sums
// S^k(x) = sum_{i>=1} w_i psi^k(x + c_i) c_i. With lambda_t = dL/df_t:
//   lambda_t = J_C(f_t)^T P^T lambda_{t+1},
// P^T = P^{-1} is the "unstream" gather mu_i(x) = lambda_i(x + c_i) if x + c_i
// is fluid, else lambda_opp(i)(x). J_C^T at a fluid node x, with
// v_k = u' + tau (g - G S^kbar), u' = j / rho, and the moments
// m0 = sum_i w_i mu_i, m1 = sum_i w_i mu_i c_i, M2 = sum_i w_i mu_i c_i c_i
// of the adjoint mu^k of component k:
//   E_k = omega (m0 + 3 m1.v + 4.5 v.M2.v - 1.5 |v|^2 m0)      (d/d rho_k)
//   V_k = omega rho_k (3 m1 + 9 M2 v - 3 m0 v)                  (d/d v_k)
//   W = (V_A + V_B) / rho,  q_k = E_k - W.u'
//   sigma^B = -tau G V_A,  sigma^A = -tau G V_B                 (d/d S^k)
//   lambda^k_i(x) = (1 - omega) mu^k_i + c_i.W + q_k
//                   + sum_{i'>=1} w_i' c_i'.sigma^k(x - c_i')
// and dL/dG accumulates -tau (V_A.S^B + V_B.S^A) over nodes and steps.
// The recompute keeps, per node, drho^A, drho^B, j, S^A and S^B (the forward
// step's own values), so the reverse step never pulls f_t.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace lbgb {

struct AdjointRun {
    int prec;
    int kernel;             // forward kernel used for the recompute
    const uint32_t* flags;
    Geom g;
    Phys p;
    int K;                  // checkpoint interval
    long long steps;        // recorded steps T
    size_t state_bytes;     // bytes of one stored state
    char* ckpt;             // checkpoint slots (slot m = state after m*K steps)
    char* seg;              // K states of the segment being reversed
    char* adj;              // adjoint buffers (adjoint_workspace_bytes)
    void* scratch;          // one state buffer the recompute may overwrite
    float* rho;             // density scratch, 2N
    double* red_part;       // kRedBlocks * kRedVals doubles
    double* red_out;
    int zsplit;
    AsyncPlan plan;         // forward (recompute) plan
    AsyncPlan adjplan;      // fused box adjoint plan; adjplan.box == 0: two-pass adjoint
    LinkList links;         // bounce-back links of the mask (recompute)
};

size_t adjoint_workspace_bytes(int nx, int ny, int nz, int K);

// Plan of the fused box adjoint (box = 0 when nx is not a multiple of 4).
AsyncPlan plan_adjoint_box(int nx, int ny, int nz, int sm_count, bool masked, size_t smem_limit);

cudaError_t run_adjoint(const AdjointRun& R, const float* dLA, const float* dLB, float* gA, float* gB,
                        double* gG, cudaStream_t st);

}  // namespace lbgb
