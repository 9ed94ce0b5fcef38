// reduce.cuh -- deterministic FP64 block reductions (fixed grid, fixed order).
#pragma once

namespace lbgb {

constexpr int kRedVals = 6;        // values reduced per block
constexpr int kRedBlocks = 1024;   // fixed block count, so the summation order is fixed

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of kRedVals doubles; thread 0 writes them to out.
__device__ __forceinline__ void block_sum_store(double (&v)[kRedVals], double* out) {
    __shared__ double sh[kRedVals][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < kRedVals; ++q) v[q] = warp_sum(v[q]);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < kRedVals; ++q) sh[q][warp] = v[q];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < kRedVals; ++q) {
            double t = lane < nw ? sh[q][lane] : 0.0;
            t = warp_sum(t);
            if (lane == 0) out[q] = t;
        }
    }
}

}  // namespace lbgb
