// Block-cooperative in-place FFTs in shared memory.
//
// The textbook radix-2 Cooley-Tukey recursions, with up to four consecutive
// radix-2 stages fused into one register step (a "radix-2^A group" of
// R = 2^A elements per thread), one __syncthreads per fused step:
//
//   DIF (decimation in frequency): natural-order input, bit-reversed output.
//       stage s, half span h = N >> (s+1):
//         (a, c) -> (a + c, (a - c) * W_{2h}^o),  o = offset in the block.
//   DIT (decimation in time): bit-reversed input, natural-order output.
//       stage s, half span h = 1 << s:
//         (a, c) -> (a + c W_{2h}^o, a - c W_{2h}^o).
//
// W_n = exp(-2 pi i / n) for the forward transform and its conjugate for the
// inverse.  DIT with conjugated twiddles is the exact conjugate transpose of
// DIF (stages reversed, each butterfly transposed), so a forward DIF and an
// inverse DIT built from one twiddle table are adjoint to rounding.
//
// Shared-memory element i of a sequence lives at index i + (i >> 4): one pad
// slot per 16 elements keeps the small-stride steps free of bank conflicts.
#pragma once

#include <cuda_runtime.h>

namespace aahrt {

__host__ __device__ __forceinline__ int padi(int i) { return i + (i >> 4); }
__host__ __device__ __forceinline__ int padded_len(int n) { return n + (n >> 4); }

__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) {
    return make_float2(a.x + b.x, a.y + b.y);
}
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) {
    return make_float2(a.x - b.x, a.y - b.y);
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

__host__ __device__ __forceinline__ unsigned brev_bits(unsigned x, int L) {
#ifdef __CUDA_ARCH__
    return L ? (__brev(x) >> (32 - L)) : 0u;
#else
    unsigned r = 0;
    for (int i = 0; i < L; ++i) { r = (r << 1) | (x & 1u); x >>= 1; }
    return r;
#endif
}

template <typename T>
__host__ __device__ __forceinline__ T ldg_ro(const T *p) {
#ifdef __CUDA_ARCH__
    return __ldg(p);
#else
    return *p;
#endif
}

// One radix-2^A DIF group.  Sequence length N = 2^L, fused stages s..s+A-1,
// group index g < N >> A.  tw[m] = exp(-2 pi i m / N), m < N/2.
// INV = true uses conjugated twiddles (inverse transform).
template <int A, bool INV>
__host__ __device__ __forceinline__ void dif_group(float2 *p, int L, int s, int g,
                                                   const float2 *__restrict__ tw) {
    constexpr int R = 1 << A;
    const int lhs = L - s - A;                 // log2 of the smallest half span
    const int j = g & ((1 << lhs) - 1);
    const int base = ((g >> lhs) << (L - s)) | j;
    float2 v[R];
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = p[padi(base + (m << lhs))];
#pragma unroll
    for (int t = 0; t < A; ++t) {
        const int Mt = R >> (t + 1);
#pragma unroll
        for (int m = 0; m < R; ++m) {
            if (m & Mt) continue;
            const int o = j + ((m & (Mt - 1)) << lhs);
            const float2 a = v[m], c = v[m + Mt];
            v[m] = cadd(a, c);
            const float2 d = csub(a, c);
            if (o == 0) {
                v[m + Mt] = d;
            } else {
                const float2 w = ldg_ro(tw + (o << (s + t)));
                v[m + Mt] = INV ? cmulc(d, w) : cmul(d, w);
            }
        }
    }
#pragma unroll
    for (int m = 0; m < R; ++m) p[padi(base + (m << lhs))] = v[m];
}

// One radix-2^A DIT group (fused stages s..s+A-1 of the DIT recursion).
template <int A, bool INV>
__host__ __device__ __forceinline__ void dit_group(float2 *p, int L, int s, int g,
                                                   const float2 *__restrict__ tw) {
    constexpr int R = 1 << A;
    const int low = g & ((1 << s) - 1);
    const int base = ((g >> s) << (s + A)) | low;
    float2 v[R];
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = p[padi(base + (m << s))];
#pragma unroll
    for (int t = 0; t < A; ++t) {
        const int Mt = 1 << t;
#pragma unroll
        for (int m = 0; m < R; ++m) {
            if (m & Mt) continue;
            const int o = low + ((m & (Mt - 1)) << s);
            float2 c = v[m + Mt];
            if (o != 0) {
                const float2 w = ldg_ro(tw + (o << (L - 1 - (s + t))));
                c = INV ? cmulc(c, w) : cmul(c, w);
            }
            const float2 a = v[m];
            v[m] = cadd(a, c);
            v[m + Mt] = csub(a, c);
        }
    }
#pragma unroll
    for (int m = 0; m < R; ++m) p[padi(base + (m << s))] = v[m];
}

// Fused-step schedule: steps of 4 radix-2 stages, the remainder last.
__host__ __device__ __forceinline__ int fused_width(int L, int s) {
    const int r = L - s;
    return r >= 4 ? 4 : r;
}

#ifdef __CUDACC__
// nb sequences of length 2^L at buf + b*ld (ld in float2, padded layout
// inside each sequence).  Must be called by every thread of the block; ends
// with a __syncthreads.
template <bool INV>
__device__ void block_fft_dif(float2 *buf, int ld, int nb, int L,
                              const float2 *__restrict__ tw) {
    for (int s = 0; s < L;) {
        const int A = fused_width(L, s);
        const int ng = 1 << (L - A);
        const int total = ng * nb;
        for (int w = threadIdx.x; w < total; w += blockDim.x) {
            float2 *p = buf + (size_t)(w >> (L - A)) * ld;
            const int g = w & (ng - 1);
            switch (A) {
                case 4: dif_group<4, INV>(p, L, s, g, tw); break;
                case 3: dif_group<3, INV>(p, L, s, g, tw); break;
                case 2: dif_group<2, INV>(p, L, s, g, tw); break;
                default: dif_group<1, INV>(p, L, s, g, tw); break;
            }
        }
        s += A;
        __syncthreads();
    }
}

template <bool INV>
__device__ void block_fft_dit(float2 *buf, int ld, int nb, int L,
                              const float2 *__restrict__ tw) {
    for (int s = 0; s < L;) {
        const int A = fused_width(L, s);
        const int ng = 1 << (L - A);
        const int total = ng * nb;
        for (int w = threadIdx.x; w < total; w += blockDim.x) {
            float2 *p = buf + (size_t)(w >> (L - A)) * ld;
            const int g = w & (ng - 1);
            switch (A) {
                case 4: dit_group<4, INV>(p, L, s, g, tw); break;
                case 3: dit_group<3, INV>(p, L, s, g, tw); break;
                case 2: dit_group<2, INV>(p, L, s, g, tw); break;
                default: dit_group<1, INV>(p, L, s, g, tw); break;
            }
        }
        s += A;
        __syncthreads();
    }
}
#endif

// Host reference driver of the same groups (used by the CPU test harness).
template <bool DIF, bool INV>
inline void host_fft(float2 *p, int L, const float2 *tw) {
    for (int s = 0; s < L;) {
        const int A = fused_width(L, s);
        const int ng = 1 << (L - A);
        for (int g = 0; g < ng; ++g) {
            if (DIF) {
                switch (A) {
                    case 4: dif_group<4, INV>(p, L, s, g, tw); break;
                    case 3: dif_group<3, INV>(p, L, s, g, tw); break;
                    case 2: dif_group<2, INV>(p, L, s, g, tw); break;
                    default: dif_group<1, INV>(p, L, s, g, tw); break;
                }
            } else {
                switch (A) {
                    case 4: dit_group<4, INV>(p, L, s, g, tw); break;
                    case 3: dit_group<3, INV>(p, L, s, g, tw); break;
                    case 2: dit_group<2, INV>(p, L, s, g, tw); break;
                    default: dit_group<1, INV>(p, L, s, g, tw); break;
                }
            }
        }
        s += A;
    }
}

}  // namespace aahrt
