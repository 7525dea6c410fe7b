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
// inverse.  Inside a group the fused stages factor into a constant radix-2^A
// network and one layer of twiddles (post-twiddles for DIF, pre-twiddles for
// DIT) built from four exact table values.  DIT with conjugated twiddles is
// the exact conjugate transpose of DIF (stages reversed, each butterfly
// transposed), so a forward DIF and an inverse DIT from one table are
// adjoint to rounding.  The table holds exp(-2 pi i m / N) for m < N.
//
// Shared-memory element i of a sequence lives at index
// padi(i) = i + (i >> 4) + (i >> 8): the two pad terms keep every access
// pattern of the kernels (unit, 16- and 256-element strides, and the
// bit-reversed order of consecutive bins) free of bank conflicts.
// Sequences of a batch sit ld elements apart, ld = 1 modulo the bank count.
#pragma once

#include <cuda_runtime.h>

namespace aahrt {

__host__ __device__ __forceinline__ int padi(int i) { return i + (i >> 4) + (i >> 8); }
__host__ __device__ __forceinline__ int padded_len(int n) { return n > 0 ? padi(n - 1) + 1 : 0; }
// sequence stride of an interleaved (float2) batch: = 1 mod 16 float2
__host__ __device__ __forceinline__ int ld_interleaved(int n) {
    const int l = padded_len(n);
    return l + ((17 - (l & 15)) & 15);
}
// sequence stride of a split (re, im float planes) batch: = 1 mod 32 floats
__host__ __device__ __forceinline__ int ld_split(int n) {
    const int l = padded_len(n);
    return l + ((33 - (l & 31)) & 31);
}

__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) {
    return make_float2(a.x + b.x, a.y + b.y);
}
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) {
    return make_float2(a.x - b.x, a.y - b.y);
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
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

// Complex sequence stored interleaved (float2) with padded indexing.  ld/st
// take a logical index, ldp/stp an already padded one.
struct IBuf {
    float2 *p;
    __host__ __device__ __forceinline__ float2 ld(int i) const { return p[padi(i)]; }
    __host__ __device__ __forceinline__ void st(int i, float2 v) const { p[padi(i)] = v; }
    __host__ __device__ __forceinline__ float2 ldp(int j) const { return p[j]; }
    __host__ __device__ __forceinline__ void stp(int j, float2 v) const { p[j] = v; }
};
// Complex sequence stored as separate real and imaginary planes.
struct SBuf {
    float *re, *im;
    __host__ __device__ __forceinline__ float2 ld(int i) const { return ldp(padi(i)); }
    __host__ __device__ __forceinline__ void st(int i, float2 v) const { stp(padi(i), v); }
    __host__ __device__ __forceinline__ float2 ldp(int j) const { return make_float2(re[j], im[j]); }
    __host__ __device__ __forceinline__ void stp(int j, float2 v) const {
        re[j] = v.x;
        im[j] = v.y;
    }
};
// Batches: sequence b of the batch.
struct IBatch {
    float2 *base;
    int ld;
    __host__ __device__ __forceinline__ IBuf operator()(int b) const { return IBuf{base + (size_t)b * ld}; }
};
struct SBatch {
    float *re, *im;
    int ld;
    __host__ __device__ __forceinline__ SBuf operator()(int b) const {
        return SBuf{re + (size_t)b * ld, im + (size_t)b * ld};
    }
};

// Constant twiddle kappa_{T,r} = exp(-+ 2 pi i r / 2^(T+1)), r < 2^T, of the
// radix-2 stages inside a group (compile-time after unrolling).
template <bool INV>
__host__ __device__ __forceinline__ float2 kappa_mul(float2 c, int T, int r) {
    if (r == 0) return c;
    if (T == 1 || (T == 2 && r == 2) || (T == 3 && r == 4)) {      // -i (+i inverse)
        return INV ? make_float2(-c.y, c.x) : make_float2(c.y, -c.x);
    }
    const float h = 0.70710678118654752440f;
    if ((T == 2 && r == 1) || (T == 3 && r == 2)) {                  // exp(-+ i pi/4)
        return INV ? make_float2(h * (c.x - c.y), h * (c.x + c.y))
                   : make_float2(h * (c.x + c.y), h * (c.y - c.x));
    }
    if ((T == 2 && r == 3) || (T == 3 && r == 6)) {                  // exp(-+ 3 i pi/4)
        return INV ? make_float2(-h * (c.x + c.y), h * (c.x - c.y))
                   : make_float2(h * (c.y - c.x), -h * (c.x + c.y));
    }
    // T == 3, r odd: exp(-+ i pi r / 8)
    const float c8 = 0.92387953251128675613f, s8 = 0.38268343236508977173f;
    float wr, wi;
    switch (r) {
        case 1: wr = c8; wi = s8; break;
        case 3: wr = s8; wi = c8; break;
        case 5: wr = -s8; wi = c8; break;
        default: wr = -c8; wi = s8; break;   // r == 7
    }
    if (!INV) wi = -wi;
    return make_float2(c.x * wr - c.y * wi, c.x * wi + c.y * wr);
}

// w[r] = exp(-+ 2 pi i q r / 2^X) for r < 2^A from four exact table values
// (r = 1, 2, 4, 8) and products; tw holds exp(-2 pi i m / N), m < N, N = 2^L.
template <int A, bool INV>
__host__ __device__ __forceinline__ void group_twiddles(int q, int L, int X,
                                                        const float2 *__restrict__ tw,
                                                        float2 *w) {
    constexpr int R = 1 << A;
    const int N = 1 << L;
    const int sh = L - X;
    w[0] = make_float2(1.f, 0.f);
#pragma unroll
    for (int b = 0; b < A; ++b) {
        float2 t = ldg_ro(tw + ((((long long)q << b) << sh) & (N - 1)));
        if (INV) t.y = -t.y;
        w[1 << b] = t;
    }
#pragma unroll
    for (int r = 3; r < R; ++r) {
        if ((r & (r - 1)) == 0) continue;
        int hi = r;
        while (hi & (hi - 1)) hi &= hi - 1;      // highest set bit
        w[r] = cmul(w[hi], w[r - hi]);
    }
}

template <int A>
__host__ __device__ __forceinline__ int rev_bits_c(int m) {
    int r = 0;
#pragma unroll
    for (int i = 0; i < A; ++i) r |= ((m >> i) & 1) << (A - 1 - i);
    return r;
}

// Constant radix-2^A DIF network on v[0..2^A) (in place).
template <int A, bool INV>
__host__ __device__ __forceinline__ void dif_network(float2 *v) {
    constexpr int R = 1 << A;
#pragma unroll
    for (int t = 0; t < A; ++t) {
        const int Mt = R >> (t + 1);
        const int T = A - 1 - t;               // log2 Mt
#pragma unroll
        for (int m = 0; m < R; ++m) {
            if (m & Mt) continue;
            const float2 a = v[m], c = v[m + Mt];
            v[m] = cadd(a, c);
            v[m + Mt] = kappa_mul<INV>(csub(a, c), T, m & (Mt - 1));
        }
    }
}

// Constant radix-2^A DIT network on v[0..2^A) (in place).
template <int A, bool INV>
__host__ __device__ __forceinline__ void dit_network(float2 *v) {
    constexpr int R = 1 << A;
#pragma unroll
    for (int t = 0; t < A; ++t) {
        const int Mt = 1 << t;
#pragma unroll
        for (int m = 0; m < R; ++m) {
            if (m & Mt) continue;
            const float2 c = kappa_mul<INV>(v[m + Mt], t, m & (Mt - 1));
            const float2 a = v[m];
            v[m] = cadd(a, c);
            v[m + Mt] = csub(a, c);
        }
    }
}

// v[m] *= exp(-+ 2 pi i q rev_A(m) / 2^X), m >= 1 (nothing when q == 0).
template <int A, bool INV>
__host__ __device__ __forceinline__ void group_twiddle(float2 *v, int q, int L, int X,
                                                       const float2 *__restrict__ tw) {
    if (q == 0) return;
    constexpr int R = 1 << A;
    float2 w[R];
    group_twiddles<A, INV>(q, L, X, tw, w);
#pragma unroll
    for (int m = 1; m < R; ++m) v[m] = cmul(v[m], w[rev_bits_c<A>(m)]);
}

// One radix-2^A DIF group: fused stages s..s+A-1 of the DIF recursion for a
// sequence of N = 2^L, group index g < N >> A.  Written as the constant
// radix-2^A DIF network followed by the post-twiddles
// exp(-2 pi i j rev_A(m) / 2^(lhs+A)) of output m (j = offset of the group).
// INV = true conjugates every twiddle (inverse transform).
//
// The element indices base + (m << lhs) of a group split into disjoint bit
// fields, so padi(base + (m << lhs)) = padi(base) + padi(m << lhs): the
// caller passes off[m] = padi(m << lhs), computed once per fused step.
template <int A, bool INV, class B>
__host__ __device__ __forceinline__ void dif_group(const B &p, int L, int s, int g,
                                                   const float2 *__restrict__ tw,
                                                   const int *off) {
    constexpr int R = 1 << A;
    const int lhs = L - s - A;                 // log2 of the smallest half span
    const int j = g & ((1 << lhs) - 1);
    const int pb = padi(((g >> lhs) << (L - s)) | j);
    float2 v[R];
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = p.ldp(pb + off[m]);
    dif_network<A, INV>(v);
    group_twiddle<A, INV>(v, j, L, lhs + A, tw);
#pragma unroll
    for (int m = 0; m < R; ++m) p.stp(pb + off[m], v[m]);
}

// One radix-2^A DIT group (fused stages s..s+A-1 of the DIT recursion):
// pre-twiddles exp(-2 pi i low rev_A(m) / 2^(s+A)) on input m, then the
// constant radix-2^A DIT network.
template <int A, bool INV, class B>
__host__ __device__ __forceinline__ void dit_group(const B &p, int L, int s, int g,
                                                   const float2 *__restrict__ tw,
                                                   const int *off) {
    constexpr int R = 1 << A;
    const int low = g & ((1 << s) - 1);
    const int pb = padi(((g >> s) << (s + A)) | low);
    float2 v[R];
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = p.ldp(pb + off[m]);
    group_twiddle<A, INV>(v, low, L, s + A, tw);
    dit_network<A, INV>(v);
#pragma unroll
    for (int m = 0; m < R; ++m) p.stp(pb + off[m], v[m]);
}

// Fused-step schedule: steps of 4 radix-2 stages, the remainder last.
__host__ __device__ __forceinline__ int fused_width(int L, int s) {
    const int r = L - s;
    return r >= 4 ? 4 : r;
}

// off[m] = padi(m << sh) for m < 2^A: the padded offsets of a group's
// elements from its base (sh = lhs for DIF, s for DIT).
template <int A>
__host__ __device__ __forceinline__ void group_offsets(int sh, int *off) {
#pragma unroll
    for (int m = 0; m < (1 << A); ++m) off[m] = padi(m << sh);
}

// Twiddles of a group are exp(-+ 2 pi i q rev_A(m) / 2^X) with q the group
// index's low bits (q = j for DIF, q = low for DIT); a thread's groups in one
// step usually share q (whenever its group stride is a multiple of 2^qbits),
// so the twiddles are built once and reused while q stays the same.
template <bool DIF, bool INV, int A, bool HOIST, class Batch>
__host__ __device__ __forceinline__ void fft_step(const Batch &bt, int nb, int L, int s,
                                                  int w0, int dw,
                                                  const float2 *__restrict__ tw) {
    constexpr int R = 1 << A;
    int off[R];
    const int sh = DIF ? L - s - A : s;        // log2 of the element stride
    group_offsets<A>(sh, off);
    const int qmask = (1 << sh) - 1;           // twiddle index: low sh bits of g
    const int X = DIF ? L - s : s + A;
    const int total = nb << (L - A);
    float2 wt[R];
    int qcur = -1;
    for (int w = w0; w < total; w += dw) {
        const auto p = bt(w >> (L - A));
        const int g = w & ((1 << (L - A)) - 1);
        if (!HOIST) {
            if (DIF)
                dif_group<A, INV>(p, L, s, g, tw, off);
            else
                dit_group<A, INV>(p, L, s, g, tw, off);
            continue;
        }
        const int q = g & qmask;
        if (!HOIST || q != qcur) {
            if (q != 0) group_twiddles<A, INV>(q, L, X, tw, wt);
            qcur = q;
        }
        const int pb = DIF ? padi(((g >> sh) << (L - s)) | q) : padi(((g >> s) << (s + A)) | q);
        float2 v[R];
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = p.ldp(pb + off[m]);
        if (DIF) {
            dif_network<A, INV>(v);
            if (q != 0) {
#pragma unroll
                for (int m = 1; m < R; ++m) v[m] = cmul(v[m], wt[rev_bits_c<A>(m)]);
            }
        } else {
            if (q != 0) {
#pragma unroll
                for (int m = 1; m < R; ++m) v[m] = cmul(v[m], wt[rev_bits_c<A>(m)]);
            }
            dit_network<A, INV>(v);
        }
#pragma unroll
        for (int m = 0; m < R; ++m) p.stp(pb + off[m], v[m]);
    }
}

// Fused steps starting at stages s_begin .. s_end-1 (step starts are the
// multiples of 4) of nb sequences of length 2^L, groups w = w0, w0 + dw, ...
// of each step (one thread's share); the caller synchronises between steps
// through `sync`.
template <bool DIF, bool INV, bool HOIST, class Batch, class Sync>
__host__ __device__ __forceinline__ void fft_steps(const Batch &bt, int nb, int L, int w0,
                                                   int dw, const float2 *__restrict__ tw,
                                                   Sync sync, int s_begin = 0,
                                                   int s_end = 1 << 30) {
    for (int s = s_begin; s < L && s < s_end;) {
        const int A = fused_width(L, s);
        switch (A) {
            case 4: fft_step<DIF, INV, 4, HOIST>(bt, nb, L, s, w0, dw, tw); break;
            case 3: fft_step<DIF, INV, 3, HOIST>(bt, nb, L, s, w0, dw, tw); break;
            case 2: fft_step<DIF, INV, 2, HOIST>(bt, nb, L, s, w0, dw, tw); break;
            default: fft_step<DIF, INV, 1, HOIST>(bt, nb, L, s, w0, dw, tw); break;
        }
        s += A;
        sync();
    }
}

#ifdef __CUDACC__
struct BlockSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
// nb sequences of length 2^L (bt(b) gives sequence b).  Must be called by
// every thread of the block; ends with a __syncthreads.
// HOIST = true keeps a group's twiddles in registers across the thread's
// groups with the same twiddle index (more live registers).
template <bool DIF, bool INV, class Batch, bool HOIST = false>
__device__ void block_fft(const Batch &bt, int nb, int L, const float2 *__restrict__ tw,
                          int s_begin = 0, int s_end = 1 << 30) {
    fft_steps<DIF, INV, HOIST>(bt, nb, L, (int)threadIdx.x, (int)blockDim.x, tw, BlockSync{},
                               s_begin, s_end);
}
#endif

struct NoSync {
    __host__ __device__ void operator()() const {}
};
// Host driver of the same groups (used by the CPU test harness).
template <bool DIF, bool INV, class Batch>
inline void host_fft(const Batch &bt, int nb, int L, const float2 *tw) {
    fft_steps<DIF, INV, true>(bt, nb, L, 0, 1, tw, NoSync{});
}

}  // namespace aahrt
