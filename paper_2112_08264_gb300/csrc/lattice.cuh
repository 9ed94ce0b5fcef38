// lattice.cuh -- compile-time D3Q19 velocity set for the CUDA kernels.
//
// D3Q19 (Sec. 2 Method): rest, 6 velocities at distance 1, 12 at sqrt 2.
// Weights 1/3, 1/18, 1/36 by |c|^2 and c_s^2 = 1/3 (Appendix coefficient
// table; Eq. LEQ). Order = the library's public order (include/lb.h):
// 0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 diagonals in opposite pairs.
//
// Every velocity is a template specialisation so that loops written with
// static_for unroll into straight-line code in which c_i, w_i and the
// opposite index are literal constants (multiplications by 0 or +-1 fold).
#pragma once
#include <type_traits>

namespace lbgb {

constexpr int Q = 19;

template <int I> struct Vel;
#define LBGB_VEL(I, X, Y, Z, O)                                             \
    template <> struct Vel<I> {                                             \
        static constexpr int x = X, y = Y, z = Z, opp = O;                  \
        static constexpr int c2 = X * X + Y * Y + Z * Z;                    \
    };
LBGB_VEL(0, 0, 0, 0, 0)
LBGB_VEL(1, 1, 0, 0, 2)
LBGB_VEL(2, -1, 0, 0, 1)
LBGB_VEL(3, 0, 1, 0, 4)
LBGB_VEL(4, 0, -1, 0, 3)
LBGB_VEL(5, 0, 0, 1, 6)
LBGB_VEL(6, 0, 0, -1, 5)
LBGB_VEL(7, 1, 1, 0, 8)
LBGB_VEL(8, -1, -1, 0, 7)
LBGB_VEL(9, 1, -1, 0, 10)
LBGB_VEL(10, -1, 1, 0, 9)
LBGB_VEL(11, 1, 0, 1, 12)
LBGB_VEL(12, -1, 0, -1, 11)
LBGB_VEL(13, 1, 0, -1, 14)
LBGB_VEL(14, -1, 0, 1, 13)
LBGB_VEL(15, 0, 1, 1, 16)
LBGB_VEL(16, 0, -1, -1, 15)
LBGB_VEL(17, 0, 1, -1, 18)
LBGB_VEL(18, 0, -1, 1, 17)
#undef LBGB_VEL

template <int I>
__host__ __device__ constexpr float wgt() {
    return Vel<I>::c2 == 0 ? 1.0f / 3.0f : (Vel<I>::c2 == 1 ? 1.0f / 18.0f : 1.0f / 36.0f);
}

template <int I>
__host__ __device__ constexpr double wgt_d() {
    return Vel<I>::c2 == 0 ? 1.0 / 3.0 : (Vel<I>::c2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
}

template <int I> using IC = std::integral_constant<int, I>;

// static_for<B, E>(f) calls f(IC<B>{}), ..., f(IC<E-1>{}).
template <int B, int E, typename F>
__host__ __device__ __forceinline__ void static_for(F&& f) {
    if constexpr (B < E) {
        f(IC<B>{});
        static_for<B + 1, E>(f);
    }
}

}  // namespace lbgb
