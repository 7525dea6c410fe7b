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
//
// Tap i of a trace sits at distance z_i = g + (W-1)/2 - i from the position,
// g in [-1/2, 1/2); phi_i(g) = phi(g + (W-1)/2 - i) is evaluated as a
// degree-(W+1) polynomial in g per tap (Horner), fitted on the host.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <utility>
#include <vector>

namespace aahrt {

constexpr int kPolyMaxW = 12;
constexpr int kPolyMaxD = kPolyMaxW + 1;

// c[d][i]: coefficient of g^d of tap i.
struct EsPoly {
    float c[kPolyMaxD + 1][kPolyMaxW];
};

struct TapSet {
    int u0;      // first grid point (may be negative; index mod nos)
    float g;     // centred offset of the position, [-1/2, 1/2)
    float ph;    // phase in cycles, [-1/2, 1/2)
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
    if (W & 1) {
        const bool up = fy >= 0.5f;
        t.u0 = iu - (W - 1) / 2 + (up ? 1 : 0);
        t.g = up ? fy - 1.0f : fy;
    } else {
        t.u0 = iu - W / 2 + 1;
        t.g = fy - 0.5f;
    }
    return t;
}

// phi at the W taps u0 + i, i < W.  The kernel is even and the taps sit
// symmetrically about the position (z_{W-1-i}(g) = -z_i(-g)), so tap W-1-i is
// tap i's polynomial at -g: with tap i's coefficients split into even and odd
// powers, phi_i = E(g^2) + g O(g^2) and phi_{W-1-i} = E(g^2) - g O(g^2), one
// pair of half-degree Horner sums per mirrored pair of taps.
template <int W>
__host__ __device__ __forceinline__ void es_weights(const EsPoly &P, float g, float *phi) {
    constexpr int D = W + 1;                 // polynomial degree
    constexpr int DE = D & ~1, DO = (D - 1) | 1;   // highest even / odd power
    const float g2 = g * g;
#pragma unroll
    for (int i = 0; i < (W + 1) / 2; ++i) {
        float e = P.c[DE][i], o = P.c[DO][i];
#pragma unroll
        for (int d = DE - 2; d >= 0; d -= 2) e = fmaf(e, g2, P.c[d][i]);
#pragma unroll
        for (int d = DO - 2; d >= 1; d -= 2) o = fmaf(o, g2, P.c[d][i]);
        phi[i] = fmaf(g, o, e);
        if (W - 1 - i != i) phi[W - 1 - i] = fmaf(-g, o, e);
    }
}

// exp(-2 pi i ph) as (cos, -sin) parts: returns c = cos(2 pi ph), s = sin(2 pi ph)
__host__ __device__ __forceinline__ void phase_cs(float ph, float *s, float *c) {
#ifdef __CUDA_ARCH__
    __sincosf(6.28318530717958647692f * ph, s, c);
#else
    *s = sinf(6.28318530717958647692f * ph);
    *c = cosf(6.28318530717958647692f * ph);
#endif
}

// Per-tap polynomial of the spreading kernel: phi_i(g) = phi(g + (W-1)/2 - i)
// for g in [-1/2, 1/2], interpolated at D+1 Chebyshev points (D = W+1) and
// written in the monomial basis of g (small Vandermonde solve in FP64).
inline void fit_es_poly(int W, double beta, EsPoly *P) {
    std::memset(P, 0, sizeof *P);
    const int D = W + 1;
    const int n = D + 1;
    std::vector<double> xs(n);
    for (int k = 0; k < n; ++k) xs[k] = 0.5 * std::cos(M_PI * (k + 0.5) / n);
    for (int i = 0; i < W; ++i) {
        std::vector<double> A((size_t)n * (n + 1));
        for (int r = 0; r < n; ++r) {
            double pw = 1.0;
            for (int c = 0; c < n; ++c) { A[r * (n + 1) + c] = pw; pw *= xs[r]; }
            const double z = xs[r] + 0.5 * (W - 1) - i;
            const double t = 2.0 * z / W;
            const double s = 1.0 - t * t;
            A[r * (n + 1) + n] = s > 0.0 ? std::exp(beta * (std::sqrt(s) - 1.0)) : 0.0;
        }
        for (int c = 0; c < n; ++c) {   // Gaussian elimination, partial pivoting
            int piv = c;
            for (int r = c + 1; r < n; ++r)
                if (std::fabs(A[r * (n + 1) + c]) > std::fabs(A[piv * (n + 1) + c])) piv = r;
            for (int q = 0; q <= n; ++q) std::swap(A[c * (n + 1) + q], A[piv * (n + 1) + q]);
            for (int r = 0; r < n; ++r) {
                if (r == c) continue;
                const double f = A[r * (n + 1) + c] / A[c * (n + 1) + c];
                for (int q = c; q <= n; ++q) A[r * (n + 1) + q] -= f * A[c * (n + 1) + q];
            }
        }
        for (int d = 0; d < n; ++d) P->c[d][i] = (float)(A[d * (n + 1) + n] / A[d * (n + 1) + d]);
    }
}

// Top 32 bits of a direct-sum phase k A + n_l k B (0.64 fixed point, mod 2^64)
// from 32-bit multiplies: with n' = n_l + 2^31 (0 <= n' < 2^32 since
// |n_l| <= 2^30) and A' = k A - 2^31 k B, the sum is A' + n' k B, whose top
// word is hi(A') + lo(n' hi(kB)) + hi(n' lo(kB)) up to the carry of the low
// words (at most 2^-32 cycle, dropped).  The forward and the adjoint evaluate
// it through the same code, so their phases agree bit for bit.
struct Phase32 {
    unsigned hiA, bh, bl, pad;
};

__host__ __device__ __forceinline__ Phase32 phase_consts(unsigned long long kA,
                                                         unsigned long long kB) {
    const unsigned long long ap = kA - (kB << 31);
    return Phase32{(unsigned)(ap >> 32), (unsigned)(kB >> 32), (unsigned)kB, 0u};
}

__host__ __device__ __forceinline__ unsigned umulhi32(unsigned a, unsigned b) {
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (unsigned)(((unsigned long long)a * b) >> 32);
#endif
}

__host__ __device__ __forceinline__ unsigned phase_top(unsigned np, const Phase32 &p) {
    return umulhi32(np, p.bl) + (np * p.bh + p.hiA);
}

}  // namespace aahrt
