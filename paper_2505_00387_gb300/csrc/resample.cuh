// Interpolation kernels of the time resamplers (the stretch S, its undoing
// U, their transposes, and the partial NMO), shared so every user evaluates
// bit-identical weights.
#pragma once

#include "internal.cuh"

namespace aahrt {

// Weights of the interpolation kernel at the taps of a position fl + x,
// x in [0, 1): tap t (input row fl + t) gets kern(x - t).  Keys' cubic
// convolution (a = -1/2) has taps t = -1..2 with the branch-free forms
//   c(x+1) = ((-x/2 + 1) x - 1/2) x,   c(x)   = (3x/2 - 5/2) x^2 + 1,
//   c(x-1) = ((-3x/2 + 2) x + 1/2) x,  c(x-2) = (x/2 - 1/2) x^2,
// linear interpolation taps t = 0, 1 with 1 - x and x.
template <int INTERP> struct Taps;
template <> struct Taps<AAHRT_INTERP_KEYS> { static constexpr int t0 = -1, n = 4; };
template <> struct Taps<AAHRT_INTERP_LINEAR> { static constexpr int t0 = 0, n = 2; };

template <int INTERP>
__device__ __forceinline__ float tap_weight(int t, float x) {
    if (INTERP == AAHRT_INTERP_LINEAR) return t == 0 ? __fadd_rn(1.0f, -x) : x;
    switch (t) {
        case -1: return __fmul_rn(__fmaf_rn(__fmaf_rn(-0.5f, x, 1.0f), x, -0.5f), x);
        case 0: return __fmaf_rn(__fmaf_rn(1.5f, x, -2.5f), __fmul_rn(x, x), 1.0f);
        case 1: return __fmul_rn(__fmaf_rn(__fmaf_rn(-1.5f, x, 2.0f), x, 0.5f), x);
        default: return __fmul_rn(__fmaf_rn(0.5f, x, -0.5f), __fmul_rn(x, x));
    }
}

}  // namespace aahrt
