// store.cuh -- storage types of the populations.
//
// Populations are kept as deviations d = f - w_i rho0^k from the rest
// equilibrium at the base densities rho0^k, in FP32, FP16 or BF16. Loads go
// through the read-only (non-coherent) path and convert to FP32; stores
// convert with round-to-nearest-even and use the streaming (evict-first)
// hint, since a step never re-reads what it writes.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace lbgb {

template <typename S> struct Store;

template <> struct Store<float> {
    static constexpr int bytes = 4;
    static __device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ void st(float* p, float v) { __stcs(p, v); }
    static __device__ __forceinline__ float to_f(float v) { return v; }
};

template <> struct Store<__half> {
    static constexpr int bytes = 2;
    static __device__ __forceinline__ float ld(const __half* p) {
        return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(p))));
    }
    static __device__ __forceinline__ void st(__half* p, float v) {
        __stcs(reinterpret_cast<unsigned short*>(p), __half_as_ushort(__float2half_rn(v)));
    }
    static __device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
};

template <> struct Store<__nv_bfloat16> {
    static constexpr int bytes = 2;
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p) {
        return __bfloat162float(
            __ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short*>(p))));
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) {
        __stcs(reinterpret_cast<unsigned short*>(p), __bfloat16_as_ushort(__float2bfloat16_rn(v)));
    }
    static __device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
};

}  // namespace lbgb
