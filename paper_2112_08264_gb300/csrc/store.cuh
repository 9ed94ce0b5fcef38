// store.cuh -- storage types of the populations.
//
// Populations are kept as deviations d = f - w_i rho0^k from the rest
// equilibrium at the base densities rho0^k, in FP32, FP16 or BF16. Loads go
// through the read-only (non-coherent) path and convert to FP32; stores
// convert with round-to-nearest-even and use the streaming (evict-first)
// hint, since a step never re-reads what it writes. The two components of one
// velocity at one site are adjacent in memory (A first), and the *2 functions
// move such a pair as one 8-byte (FP32) or 4-byte (FP16/BF16) access.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace lbgb {

template <typename S> struct Store;

template <> struct Store<float> {
    static constexpr int bytes = 4;
    using Pair = float2;
    static __device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ void st(float* p, float v) { __stcs(p, v); }
    static __device__ __forceinline__ float to_f(float v) { return v; }
    static __device__ __forceinline__ void ld2(const float* p, float& a, float& b) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(p));
        a = v.x;
        b = v.y;
    }
    // plain load (shared memory)
    static __device__ __forceinline__ void lds2(const float* p, float& a, float& b) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        a = v.x;
        b = v.y;
    }
    static __device__ __forceinline__ void st2(float* p, float a, float b) {
        __stcs(reinterpret_cast<float2*>(p), make_float2(a, b));
    }
    // the pair as (A, B), from shared memory
    static __device__ __forceinline__ float2 lds2v(const float* p) { return *reinterpret_cast<const float2*>(p); }
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
    using Pair = unsigned int;
    static __device__ __forceinline__ void unpack(unsigned int w, float& a, float& b) {
        const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w));
        a = f.x;
        b = f.y;
    }
    // component k of a pair word (the conversion selects the half itself)
    static __device__ __forceinline__ float part(unsigned int w, int k) {
        const __half2 h = *reinterpret_cast<const __half2*>(&w);
        return k == 0 ? __low2float(h) : __high2float(h);
    }
    static __device__ __forceinline__ void ld2(const __half* p, float& a, float& b) {
        unpack(__ldg(reinterpret_cast<const unsigned int*>(p)), a, b);
    }
    static __device__ __forceinline__ void lds2(const __half* p, float& a, float& b) {
        unpack(*reinterpret_cast<const unsigned int*>(p), a, b);
    }
    // the pair word as (A, B)
    static __device__ __forceinline__ float2 unpack2(unsigned int w) {
        return __half22float2(*reinterpret_cast<const __half2*>(&w));
    }
    static __device__ __forceinline__ float2 lds2v(const __half* p) {
        return unpack2(*reinterpret_cast<const unsigned int*>(p));
    }
    static __device__ __forceinline__ void st2(__half* p, float a, float b) {
        const __half2 h = __floats2half2_rn(a, b);
        __stcs(reinterpret_cast<unsigned int*>(p), *reinterpret_cast<const unsigned int*>(&h));
    }
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
    using Pair = unsigned int;
    static __device__ __forceinline__ void unpack(unsigned int w, float& a, float& b) {
        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
        a = f.x;
        b = f.y;
    }
    // component k of a pair word (a bf16 is the upper half of its float)
    static __device__ __forceinline__ float part(unsigned int w, int k) {
        return __uint_as_float(k == 0 ? (w << 16) : (w & 0xffff0000u));
    }
    static __device__ __forceinline__ void ld2(const __nv_bfloat16* p, float& a, float& b) {
        unpack(__ldg(reinterpret_cast<const unsigned int*>(p)), a, b);
    }
    static __device__ __forceinline__ void lds2(const __nv_bfloat16* p, float& a, float& b) {
        unpack(*reinterpret_cast<const unsigned int*>(p), a, b);
    }
    // the pair word as (A, B)
    static __device__ __forceinline__ float2 unpack2(unsigned int w) {
        return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
    }
    static __device__ __forceinline__ float2 lds2v(const __nv_bfloat16* p) {
        return unpack2(*reinterpret_cast<const unsigned int*>(p));
    }
    static __device__ __forceinline__ void st2(__nv_bfloat16* p, float a, float b) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        __stcs(reinterpret_cast<unsigned int*>(p), *reinterpret_cast<const unsigned int*>(&h));
    }
};

}  // namespace lbgb
