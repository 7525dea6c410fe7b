// Per-trace arithmetic of the Fourier slice step (Algorithm 1 step 3,
// eqs. Inv_op / inv_GFST), shared by the forward and adjoint kernels so both
// use bit-identical phases, tap positions and kernel weights.
//
// For bin k the trace reads the q-spectrum of its azimuth slices at
// k_q = f_k r^2.  Along the curvature axis q_l = q0 + l dq this is the
// DTFT of the column at x = f_k dq r^2 cycles per sample, times the phase
// exp(-2 pi i f_k q0 r^2).  With the column centred at l = cq,
//
//   sum_l X_l e^{-2 pi i x l} = e^{-2 pi i x cq} sum_u phi(nos x - u) G[u mod nos]
//
// up to the spreading kernel's error, where G is the nos-point DFT of the
// deapodised, centred column and phi the exponential-of-semicircle kernel
// phi(z) = exp(beta (sqrt(1 - (2z/W)^2) - 1)), |z| <= W/2.  The total phase
// per bin is frac(k A) and the position frac(k B) (A, B: 0.64 fixed point),
// so both are exact integer products modulo 2^64.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

namespace aahrt {

struct TapSet {
    int u0;      // first grid point (may be negative; index mod nos)
    float z0;    // distance (grid units) from the first tap to the position
    float ph;    // phase in cycles, [-0.5, 0.5)
};

template <int W>
__host__ __device__ __forceinline__ TapSet trace_taps(unsigned long long A,
                                                      unsigned long long B,
                                                      unsigned k, int Lq) {
    const unsigned long long pa = (unsigned long long)k * A;
    const unsigned long long pb = (unsigned long long)k * B;
    const unsigned ptop = (unsigned)(pa >> 32);
    const unsigned xtop = (unsigned)(pb >> 32);
    TapSet t;
    t.ph = (float)(int)ptop * 2.3283064365386963e-10f;      // 2^-32
    const int iu = (int)(xtop >> (32 - Lq));                  // integer part of nos*x
    const float fy = (float)(unsigned)(xtop << Lq) * 2.3283064365386963e-10f;
    if (W & 1)
        t.u0 = iu - (W - 1) / 2 + (fy >= 0.5f ? 1 : 0);
    else
        t.u0 = iu - W / 2 + 1;
    t.z0 = (float)(iu - t.u0) + fy;
    return t;
}

// phi at the W taps u0 + i, i < W (distance z0 - i).
template <int W>
__host__ __device__ __forceinline__ void es_weights(float z0, float beta, float *phi) {
    const float inv = 2.0f / (float)W;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const float t = (z0 - (float)i) * inv;
        const float s = fmaxf(1.0f - t * t, 0.0f);
#ifdef __CUDA_ARCH__
        phi[i] = __expf(beta * (sqrtf(s) - 1.0f));
#else
        phi[i] = expf(beta * (sqrtf(s) - 1.0f));
#endif
    }
}

}  // namespace aahrt
