// Time-axis stages of the AAHRT (Algorithms 1 and 2, steps 1-2 and 4-5):
//
//   r2c: X[k][c] = sum_n (G in)[n][c] exp(-2 pi i k n / Nfft), k < nbins
//        where G resamples each column: the time stretch S (model side,
//        Alg. 1 steps 1-2) or the transpose of its undoing, U^T (data side,
//        the adjoint's first two stages).
//   c2r: out[i][c] = sum_n G[i][n] H(X[.][c])[n] with the band-limited
//        Hermitian synthesis H(X)[n] = Re X_0 + 2 Re sum_{k>=1} X_k e^{+2 pi i k n/Nfft}
//        and G = U (data side, Alg. 1 steps 4-5) or S^T (model side, the
//        adjoint's last two stages).  Epilogues fuse the FISTA residual
//        r = d - L z and the soft-threshold/momentum update (eqs. ISTA, soft).
//
// One block owns up to 2*P adjacent columns; two real columns travel as
// the real and imaginary parts of one complex FFT of length Nfft held in
// shared memory (padded layout of fft.cuh).  Each thread resamples whole
// rows (all P pairs), so a row's weights are computed once per block.
//
// Resampling: output row o of S (or U) sits at position fl + fr on the input
// axis and reads input rows fl + t with weight kern(fr - t), t in the kernel's
// taps.  The transposed operators read, for output o, the contiguous source
// rows of a host-built table, in segments of equal tap t, and recompute the
// same weight from the source row's fr through the same function, so S and
// S^T (U and U^T) use bit-identical weights.
#include "fft.cuh"
#include "internal.cuh"
#include "resample.cuh"

namespace aahrt {

// Entry i of a resampler's row table, as its two raw words: a RowPos
// (fl, bits of fr) for S or U, a RowRange for S^T or U^T (sources lo, lo+1,
// ... in segments of decreasing tap t, largest t first; segment q, tap
// t0 + q, has (cnt >> 8q) & 255 rows).
template <bool TRANS>
__device__ __forceinline__ int2 row_entry(const DevResampler &rs, int i) {
    return __ldg(reinterpret_cast<const int2 *>(TRANS ? (const void *)(rs.rng + i)
                                                      : (const void *)(rs.pos + i)));
}

constexpr int kPackBatch = 8;   // spectrum loads in flight per thread (c2r pack)

// Threads of a time-kernel block: 256 while two blocks fit in one SM's shared
// memory, else 512 (one block per SM, e.g. the 8192-point frames of long
// traces), so an SM keeps 16 warps in flight either way.  Both run under the
// same 128-register cap.
static int time_threads(size_t smem) {
    return smem + 512 <= (size_t)kTimeSmemTwoBlocks ? kThreadsTime : kMaxThreadsTime;
}

// Asynchronous global -> shared copies (no registers held while in flight).
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n"); }
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Start copying nrow rows of 2P floats (row stride ld floats) into dst [row][2P].
template <int P>
__device__ __forceinline__ void prefetch_rows(float *dst, const float *src, int nrow, int ld) {
    constexpr int CB = P == 1 ? 8 : 16;            // bytes per copy
    constexpr int PER = (8 * P) / CB;              // copies per row
    for (int idx = threadIdx.x; idx < nrow * PER; idx += blockDim.x) {
        const int r = idx / PER, q = idx - r * PER;
        cp_async<CB>(dst + r * 2 * P + q * (CB / 4), src + (long long)r * ld + q * (CB / 4));
    }
}

template <int P>
struct Acc {
    float2 v[P];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int p = 0; p < P; ++p) v[p] = make_float2(0.f, 0.f);
    }
    // += w * (P complex values at row r of a row-major [row][P] float2 array)
    __device__ __forceinline__ void add_row(float w, const float2 *row) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const float2 x = row[p];
            v[p].x = fmaf(w, x.x, v[p].x);
            v[p].y = fmaf(w, x.y, v[p].y);
        }
    }
    // += w * (column p at padded position pr of P sequences ld apart)
    __device__ __forceinline__ void add_cols(float w, const float2 *sm, int ld, int pr) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const float2 x = sm[p * ld + pr];
            v[p].x = fmaf(w, x.x, v[p].x);
            v[p].y = fmaf(w, x.y, v[p].y);
        }
    }
};

// The r2c pipeline after its input rows are staged in shared memory
// (stg [row][2P] floats, sfr the source fractions of a transposed
// resampler; the caller synchronised): resample onto the frame, FFT, unpack.
// With a bound table (data side only: TRANS, ybd.max != nullptr) the unpack
// also raises ybd.max[cube][chunk] to the largest |re| + |im| it writes in
// each chunk of bins: the amplitude bound of the adjoint spread's fixed point.
struct YBound {
    unsigned *max;
    int nchunk, chunk_log;
};

template <int LP, int INTERP, bool TRANS>
__device__ __forceinline__ void r2c_core(float2 *sm, const float *stg, const float *sfr,
                                         const ColGroup &cg, const DevResampler &rs,
                                         int nrow_in, const float2 *__restrict__ tw, int L,
                                         int nbins, float2 *__restrict__ out,
                                         const YBound &ybd) {
    constexpr int P = 1 << LP;
    const int N = 1 << L;
    const int ld = ld_interleaved(N);
    // z_p[n] = sum_r G[n][r] (x_{2p} + i x_{2p+1})[r], one row n per thread
    const float2 *stg2 = reinterpret_cast<const float2 *>(stg);
    // the next row's table entry is loaded while this row is resampled
    int2 nxt = make_int2(0, 0);
    if ((int)threadIdx.x < rs.nrows)
        nxt = row_entry<TRANS>(rs, threadIdx.x);
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        Acc<P> acc;
        acc.zero();
        const int2 cur = nxt;
        if (n + (int)blockDim.x < rs.nrows)
            nxt = row_entry<TRANS>(rs, n + blockDim.x);
        if (n < rs.nrows) {
            if (!TRANS) {
                const RowPos ps{cur.x, __int_as_float(cur.y)};
#pragma unroll
                for (int q = 0; q < Taps<INTERP>::n; ++q) {
                    const int t = Taps<INTERP>::t0 + q;
                    const int r = ps.fl + t;
                    if (r < 0 || r >= nrow_in) continue;
                    acc.add_row(tap_weight<INTERP>(t, ps.fr), stg2 + r * P);
                }
            } else {
                const RowRange rg{cur.x, cur.y};
                int r = rg.lo;
#pragma unroll
                for (int q = Taps<INTERP>::n - 1; q >= 0; --q) {
                    const int t = Taps<INTERP>::t0 + q;
                    const int cnt = (rg.cnt >> (8 * q)) & 255;
                    for (int e = 0; e < cnt; ++e, ++r)
                        acc.add_row(tap_weight<INTERP>(t, sfr[r]), stg2 + r * P);
                }
            }
        }
#pragma unroll
        for (int p = 0; p < P; ++p) sm[p * ld + padi(n)] = acc.v[p];
    }
    __syncthreads();
    block_fft<true, false, IBatch, true>(IBatch{sm, ld}, P, L, tw);

    // unpack the two real spectra: A = (Z_k + conj Z_{N-k})/2, B = (Z_k - conj Z_{N-k})/(2i)
    float2 *dst = out + cg.spec_off;
    const int npair = (cg.ncol + 1) >> 1;
    const bool bound = TRANS && ybd.max != nullptr;
    __shared__ unsigned s_ymax[128];
    if (bound) {
        for (int c = threadIdx.x; c < ybd.nchunk; c += blockDim.x) s_ymax[c] = 0u;
        __syncthreads();
    }
    // rows 16-byte aligned (even row stride and offset): a column pair's A and
    // B leave as one 16-byte store
    const bool wide = ((cg.ld_spec | cg.spec_off) & 1) == 0;
    const int kend = ((P * nbins + blockDim.x - 1) / blockDim.x) * blockDim.x;
    for (int idx = threadIdx.x; idx < kend; idx += blockDim.x) {
        const int p = idx & (P - 1);
        const int k = idx >> LP;
        float amax = 0.f;
        if (idx < P * nbins && p < npair) {
            const float2 zk = sm[p * ld + padi(brev_bits(k, L))];
            const float2 zn = sm[p * ld + padi(brev_bits((N - k) & (N - 1), L))];
            const float2 A = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
            const float2 B = make_float2(0.5f * (zk.y + zn.y), -0.5f * (zk.x - zn.x));
            const long long o = (long long)k * cg.ld_spec + 2 * p;
            amax = fabsf(A.x) + fabsf(A.y);
            if (2 * p + 1 < cg.ncol) {
                if (wide)
                    *reinterpret_cast<float4 *>(dst + o) = make_float4(A.x, A.y, B.x, B.y);
                else {
                    dst[o] = A;
                    dst[o + 1] = B;
                }
                amax = fmaxf(amax, fabsf(B.x) + fabsf(B.y));
            } else {
                dst[o] = A;
            }
        }
        if (bound) {
            // a warp's 32 / P bins lie inside one chunk (chunks of >= 64 bins)
#pragma unroll
            for (int sh = 16; sh > 0; sh >>= 1)
                amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, sh));
            const int kw = (idx & ~31) >> LP;
            if ((threadIdx.x & 31) == 0 && kw < nbins && amax > 0.f)
                atomicMax(s_ymax + (kw >> ybd.chunk_log), __float_as_uint(amax));
        }
    }
    if (bound) {
        __syncthreads();
        // the table only grows within a launch, so a block whose maximum does
        // not exceed the value it reads needs no atomic
        unsigned *row = ybd.max + (long long)cg.cube * ybd.nchunk;
        for (int c = threadIdx.x; c < ybd.nchunk; c += blockDim.x) {
            const unsigned v = s_ymax[c];
            if (v > *(volatile unsigned *)(row + c)) atomicMax(row + c, v);
        }
    }
}

template <int LP, int INTERP, bool TRANS>
__global__ void __launch_bounds__(kMaxThreadsTime, 1)
r2c_kernel(const float *__restrict__ in, float2 *__restrict__ out,
           const ColGroup *__restrict__ groups, DevResampler rs, int nrow_in,
           const float2 *__restrict__ tw, int L, int nbins, YBound ybd) {
    constexpr int P = 1 << LP;
    extern __shared__ float4 smem_f4[];
    float2 *sm = reinterpret_cast<float2 *>(smem_f4);
    const ColGroup cg = groups[blockIdx.x];
    const int ld = ld_interleaved(1 << L);
    float *stg = reinterpret_cast<float *>(sm + P * ld);          // staged input [row][2P]
    float *sfr = stg + nrow_in * 2 * P;                           // source fractions (TRANS)

    // stage the block's input columns (independent, coalesced loads, a batch
    // of rounds in flight per thread)
    const float *src = in + cg.real_off;
    const int total = nrow_in * 2 * P;
    for (int base = threadIdx.x; base < total; base += kPackBatch * blockDim.x) {
        float v[kPackBatch];
#pragma unroll
        for (int u = 0; u < kPackBatch; ++u) {
            const int idx = base + u * blockDim.x;
            const int r = idx >> (LP + 1);
            const int c = idx & (2 * P - 1);
            v[u] = (idx < total && c < cg.ncol) ? __ldg(src + (long long)r * cg.ld_real + c) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kPackBatch; ++u)
            if (base + u * blockDim.x < total) stg[base + u * blockDim.x] = v[u];
    }
    if (TRANS)
        for (int idx = threadIdx.x; idx < rs.npos; idx += blockDim.x)
            sfr[idx] = __ldg(&rs.pos[idx].fr);
    __syncthreads();
    r2c_core<LP, INTERP, TRANS>(sm, stg, sfr, cg, rs, nrow_in, tw, L, nbins, out, ybd);
}

// The c2r pipeline of one column group.  With STAGE, the epilogue's real
// rows (the residual, or the new extrapolated point z of the FISTA update)
// also go to stg [row][2P] in shared memory for an r2c of the same columns
// (the residual is then not written to global memory).
template <int LP, int INTERP, bool TRANS, int EPI, bool STAGE>
__device__ __forceinline__ void c2r_core(float2 *sm, float *sfr, const float2 *__restrict__ in,
                                         float *__restrict__ out,
                                         const float *__restrict__ aux, const FistaArgs &fa,
                                         const ColGroup &cg, const DevResampler &rs, int n_in,
                                         const float2 *__restrict__ tw, int L, int nbins,
                                         float *stg) {
    constexpr int P = 1 << LP;
    const int N = 1 << L;
    const int half = N >> 1;
    const int ld = ld_interleaved(N);
    const float2 *src = in + cg.spec_off;
    const int npair = (cg.ncol + 1) >> 1;

    if (TRANS)
        for (int idx = threadIdx.x; idx < rs.npos; idx += blockDim.x)
            sfr[idx] = __ldg(&rs.pos[idx].fr);
    // pack Z = A + iB over the full frame, bit-reversed for the DIT pass;
    // kPackBatch rounds of loads are issued before any is used, so each
    // thread keeps that many spectrum reads in flight
    const int total = P * (half + 1);
    // rows 16-byte aligned: a column pair's A and B arrive as one 16-byte load
    const bool wide = ((cg.ld_spec | cg.spec_off) & 1) == 0;
    for (int base = threadIdx.x; base < total; base += kPackBatch * blockDim.x) {
        float2 A[kPackBatch], B[kPackBatch];
#pragma unroll
        for (int u = 0; u < kPackBatch; ++u) {
            const int idx = base + u * blockDim.x;
            const int p = idx & (P - 1);
            const int k = idx >> LP;
            A[u] = B[u] = make_float2(0.f, 0.f);
            if (idx < total && k < nbins && p < npair) {
                const long long o = (long long)k * cg.ld_spec + 2 * p;
                // the fused kernel rewrites the spectrum later: plain loads there
                if (wide && 2 * p + 1 < cg.ncol) {
                    const float4 *q4 = reinterpret_cast<const float4 *>(src + o);
                    const float4 v = STAGE ? *q4 : __ldg(q4);
                    A[u] = make_float2(v.x, v.y);
                    B[u] = make_float2(v.z, v.w);
                } else {
                    A[u] = STAGE ? src[o] : __ldg(src + o);
                    if (2 * p + 1 < cg.ncol) B[u] = STAGE ? src[o + 1] : __ldg(src + o + 1);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kPackBatch; ++u) {
            const int idx = base + u * blockDim.x;
            if (idx >= total) break;
            const int p = idx & (P - 1);
            const int k = idx >> LP;
            float2 a = A[u], b = B[u];
            if (k == 0) { a.y = 0.f; b.y = 0.f; }
            const float2 zk = make_float2(a.x - b.y, a.y + b.x);   // A + iB
            const float2 zn = make_float2(a.x + b.y, b.x - a.y);   // conj(A) + i conj(B)
            float2 *q = sm + p * ld;
            if (k == 0) {
                q[padi(0)] = zk;
            } else if (k == half) {
                q[padi(brev_bits(half, L))] = make_float2(0.f, 0.f);
            } else {
                q[padi(brev_bits(k, L))] = zk;
                q[padi(brev_bits(N - k, L))] = zn;
            }
        }
    }
    __syncthreads();
    block_fft<false, true, IBatch, true>(IBatch{sm, ld}, P, L, tw);
    if (STAGE && EPI != EPI_STORE) {
        // the epilogue's rows (d, or z) were prefetched into stg
        cp_async_wait_all();
        __syncthreads();
    }

    // resample the synthesized columns onto the output rows, one row per
    // thread; the next row's table entry is loaded while this one is done
    int2 nxt = make_int2(0, 0);
    if ((int)threadIdx.x < rs.nrows)
        nxt = row_entry<TRANS>(rs, threadIdx.x);
    for (int i = threadIdx.x; i < rs.nrows; i += blockDim.x) {
        Acc<P> acc;
        acc.zero();
        const int2 cur = nxt;
        if (i + (int)blockDim.x < rs.nrows)
            nxt = row_entry<TRANS>(rs, i + blockDim.x);
        const long long o = cg.real_off + (long long)i * cg.ld_real;
        const int nc = cg.ncol;
        // the FISTA update's m row is loaded first, its latency covered by
        // the resampling below
        float mo[2 * P];
        if (EPI == EPI_FISTA) {
#pragma unroll
            for (int c = 0; c < 2 * P; ++c) mo[c] = c < nc ? fa.m[o + c] : 0.f;
        }
        if (!TRANS) {
            const RowPos ps{cur.x, __int_as_float(cur.y)};
#pragma unroll
            for (int q = 0; q < Taps<INTERP>::n; ++q) {
                const int t = Taps<INTERP>::t0 + q;
                const int r = ps.fl + t;
                if (r < 0 || r >= n_in) continue;
                acc.add_cols(tap_weight<INTERP>(t, ps.fr), sm, ld, padi(r));
            }
        } else {
            const RowRange rg{cur.x, cur.y};
            int r = rg.lo;
#pragma unroll
            for (int q = Taps<INTERP>::n - 1; q >= 0; --q) {
                const int t = Taps<INTERP>::t0 + q;
                const int cnt = (rg.cnt >> (8 * q)) & 255;
                for (int e = 0; e < cnt; ++e, ++r)
                    acc.add_cols(tap_weight<INTERP>(t, sfr[r]), sm, ld, padi(r));
            }
        }
        float g2[2 * P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            g2[2 * p] = acc.v[p].x;
            g2[2 * p + 1] = acc.v[p].y;
        }
        if (EPI == EPI_STORE) {
#pragma unroll
            for (int c = 0; c < 2 * P; ++c)
                if (c < nc) out[o + c] = g2[c];
        } else if (EPI == EPI_RESIDUAL) {
            float dv[2 * P];
#pragma unroll
            for (int c = 0; c < 2 * P; ++c)
                dv[c] = c < nc ? (STAGE ? stg[i * 2 * P + c] : __ldg(aux + o + c)) : 0.f;
            if (STAGE) {
#pragma unroll
                for (int c = 0; c < 2 * P; ++c) stg[i * 2 * P + c] = c < nc ? dv[c] - g2[c] : 0.f;
            } else {
#pragma unroll
                for (int c = 0; c < 2 * P; ++c)
                    if (c < nc) out[o + c] = dv[c] - g2[c];
            }
        } else {
            // m+ = soft(z + gamma g, gamma lambda); z+ = m+ + beta (m+ - m)
            float gam = fa.gamma, th = fa.thresh;
            if (fa.cube_gt) {
                const float2 gt = __ldg(fa.cube_gt + cg.cube);
                gam = gt.x;
                th = gt.y;
            }
            float *__restrict__ mp = fa.m + o;
            float *__restrict__ zp = fa.z + o;
            float zo[2 * P];
#pragma unroll
            for (int c = 0; c < 2 * P; ++c)
                zo[c] = c < nc ? (STAGE ? stg[i * 2 * P + c] : zp[c]) : 0.f;
#pragma unroll
            for (int c = 0; c < 2 * P; ++c) {
                if (c >= nc) {
                    if (STAGE) stg[i * 2 * P + c] = 0.f;
                    continue;
                }
                const float mn = soft_threshold(fmaf(gam, g2[c], zo[c]), th);
                const float zn = fmaf(fa.beta, mn - mo[c], mn);
                mp[c] = mn;
                zp[c] = zn;
                if (STAGE) stg[i * 2 * P + c] = zn;
            }
        }
    }
}

template <int LP, int INTERP, bool TRANS, int EPI>
__global__ void __launch_bounds__(kMaxThreadsTime, 1)
c2r_kernel(const float2 *__restrict__ in, float *__restrict__ out,
           const float *__restrict__ aux, FistaArgs fa,
           const ColGroup *__restrict__ groups, DevResampler rs, int n_in,
           const float2 *__restrict__ tw, int L, int nbins) {
    constexpr int P = 1 << LP;
    extern __shared__ float4 smem_f4[];
    float2 *sm = reinterpret_cast<float2 *>(smem_f4);
    const ColGroup cg = groups[blockIdx.x];
    float *sfr = reinterpret_cast<float *>(sm + P * ld_interleaved(1 << L));
    c2r_core<LP, INTERP, TRANS, EPI, false>(sm, sfr, in, out, aux, fa, cg, rs, n_in, tw, L,
                                            nbins, nullptr);
}

// One FISTA half-iteration's two time stages on the same column group, fused:
// the synthesis c2r (with its epilogue: residual on the data side, FISTA
// update on the model side) stages its real rows in shared memory and the
// analysis r2c of the other direction transforms them in place of a round
// trip through global memory.  Data side: U H then U^T F (residual r = d - L z
// never stored); model side: S^T H with the update, then S F of the new z
// (the next iteration's first stage).  The spectrum is read and rewritten in
// place: a block touches only its own columns.
template <int LP, int INTERP, bool SYN_TRANS, int EPI>
__global__ void __launch_bounds__(kMaxThreadsTime, 1)
c2r_r2c_kernel(float2 *spec, const float *__restrict__ aux, FistaArgs fa,
               const ColGroup *__restrict__ groups, DevResampler rs_syn, int n_in,
               DevResampler rs_ana, int nrow_mid, const float2 *__restrict__ tw, int L,
               int nbins, YBound ybd) {
    constexpr int P = 1 << LP;
    constexpr bool ANA_TRANS = !SYN_TRANS;
    extern __shared__ float4 smem_f4[];
    float2 *sm = reinterpret_cast<float2 *>(smem_f4);
    const ColGroup cg = groups[blockIdx.x];
    float *stg = reinterpret_cast<float *>(sm + P * ld_interleaved(1 << L));   // [row][2P]
    float *sfr = stg + nrow_mid * 2 * P;
    // Prefetch the epilogue's state rows (the column group's slab of the
    // column-blocked d, or of z) into stg while the spectrum is packed and
    // transformed; the epilogue rewrites stg in place, element by element.
    prefetch_rows<P>(stg, (EPI == EPI_RESIDUAL ? aux : fa.z) + cg.real_off, rs_syn.nrows,
                     cg.ld_real);
    cp_async_commit();
    c2r_core<LP, INTERP, SYN_TRANS, EPI, true>(sm, sfr, spec, nullptr, aux, fa, cg, rs_syn, n_in,
                                               tw, L, nbins, stg);
    __syncthreads();
    if (ANA_TRANS) {
        for (int idx = threadIdx.x; idx < rs_ana.npos; idx += blockDim.x)
            sfr[idx] = __ldg(&rs_ana.pos[idx].fr);
        __syncthreads();
    }
    r2c_core<LP, INTERP, ANA_TRANS>(sm, stg, sfr, cg, rs_ana, nrow_mid, tw, L, nbins, spec, ybd);
}

// ------------------------------------------------------------- dispatch
template <int LP, int INTERP>
static void r2c_launch(bool model_side, int grid, size_t smem, cudaStream_t st, const float *in,
                       float2 *out, const ColGroup *cg, DevResampler rs, int nrow_in,
                       const float2 *tw, int L, int nbins, YBound ybd = YBound{}) {
    if (model_side)
        r2c_kernel<LP, INTERP, false><<<grid, time_threads(smem), smem, st>>>(in, out, cg, rs, nrow_in,
                                                                        tw, L, nbins, YBound{});
    else
        r2c_kernel<LP, INTERP, true><<<grid, time_threads(smem), smem, st>>>(in, out, cg, rs, nrow_in,
                                                                       tw, L, nbins, ybd);
}

// The bound table of the data spectrum, cleared for the analysis about to
// write Y (nothing for plans without one).
static cudaError_t ybound_reset(Plan &p, cudaStream_t st, YBound *yb) {
    *yb = YBound{p.ymax, p.nychunk, p.ychunk_log};
    if (!p.ymax) return cudaSuccess;
    return cudaMemsetAsync(p.ymax, 0, (size_t)p.ncube * p.nychunk * sizeof(unsigned), st);
}

template <int LP, int INTERP, int EPI>
static void c2r_launch(bool model_side, int grid, size_t smem, cudaStream_t st,
                       const float2 *in, float *out, const float *aux, FistaArgs fa,
                       const ColGroup *cg, DevResampler rs, int n_in, const float2 *tw, int L,
                       int nbins) {
    if (model_side)
        c2r_kernel<LP, INTERP, true, EPI><<<grid, time_threads(smem), smem, st>>>(
            in, out, aux, fa, cg, rs, n_in, tw, L, nbins);
    else
        c2r_kernel<LP, INTERP, false, EPI><<<grid, time_threads(smem), smem, st>>>(
            in, out, aux, fa, cg, rs, n_in, tw, L, nbins);
}

#define AAHRT_LP_SWITCH(LPV, STMT)                      \
    switch (LPV) {                                      \
        case 0: { constexpr int LPc = 0; STMT; } break; \
        case 1: { constexpr int LPc = 1; STMT; } break; \
        case 2: { constexpr int LPc = 2; STMT; } break; \
        default: { constexpr int LPc = 3; STMT; } break; \
    }
#define AAHRT_INTERP_SWITCH(IV, STMT)                                       \
    if ((IV) == AAHRT_INTERP_LINEAR) { constexpr int IPc = AAHRT_INTERP_LINEAR; STMT; } \
    else { constexpr int IPc = AAHRT_INTERP_KEYS; STMT; }

cudaError_t launch_r2c(Plan &p, bool model_side, const float *in, float2 *out,
                       cudaStream_t st, bool blocked) {
    const ColGroup *cg = model_side ? (blocked ? p.cg_model_blk : p.cg_model)
                                    : (blocked ? p.cg_data_blk : p.cg_data);
    const int n = model_side ? p.ncg_model : p.ncg_data;
    const DevResampler rs = model_side ? p.S : p.UT;
    const int nrow_in = model_side ? p.ntau : p.nt;
    const size_t smem = model_side ? p.smem_r2c_model : p.smem_r2c_data;
    const int stage = model_side ? 0 : 3;
    YBound yb{};
    if (!model_side) {
        const cudaError_t e = ybound_reset(p, st, &yb);
        if (e) return e;
    }
    prof_begin(p, stage, st);
    AAHRT_LP_SWITCH(p.lp, AAHRT_INTERP_SWITCH(p.interp, (r2c_launch<LPc, IPc>(
        model_side, n, smem, st, in, out, cg, rs, nrow_in, p.tw_t, p.L, p.nbins, yb))));
    prof_end(p, st);
    p.launches[stage]++;
    return cudaGetLastError();
}

cudaError_t launch_c2r(Plan &p, bool model_side, const float2 *in, float *out,
                       int epi, const float *aux, FistaArgs fa, cudaStream_t st, bool blocked) {
    const ColGroup *cg = model_side ? (blocked ? p.cg_model_blk : p.cg_model)
                                    : (blocked ? p.cg_data_blk : p.cg_data);
    const int n = model_side ? p.ncg_model : p.ncg_data;
    const DevResampler rs = model_side ? p.ST : p.U;
    const int n_in = p.ns;
    const size_t smem = model_side ? p.smem_c2r_model : p.smem_c2r_data;
    const int stage = model_side ? 5 : 2;
    prof_begin(p, stage, st);
    switch (epi) {
        case EPI_RESIDUAL:
            AAHRT_LP_SWITCH(p.lp, AAHRT_INTERP_SWITCH(p.interp, (c2r_launch<LPc, IPc, EPI_RESIDUAL>(
                model_side, n, smem, st, in, out, aux, fa, cg, rs, n_in, p.tw_t, p.L, p.nbins))));
            break;
        case EPI_FISTA:
            AAHRT_LP_SWITCH(p.lp, AAHRT_INTERP_SWITCH(p.interp, (c2r_launch<LPc, IPc, EPI_FISTA>(
                model_side, n, smem, st, in, out, aux, fa, cg, rs, n_in, p.tw_t, p.L, p.nbins))));
            break;
        default:
            AAHRT_LP_SWITCH(p.lp, AAHRT_INTERP_SWITCH(p.interp, (c2r_launch<LPc, IPc, EPI_STORE>(
                model_side, n, smem, st, in, out, aux, fa, cg, rs, n_in, p.tw_t, p.L, p.nbins))));
            break;
    }
    prof_end(p, st);
    p.launches[stage]++;
    return cudaGetLastError();
}

template <int LPc, int IPc>
static cudaError_t attrs_for(int max_smem) {
    cudaError_t e;
    if ((e = raise_smem_limit(r2c_kernel<LPc, IPc, false>, max_smem))) return e;
    if ((e = raise_smem_limit(r2c_kernel<LPc, IPc, true>, max_smem))) return e;
    if ((e = raise_smem_limit(c2r_kernel<LPc, IPc, false, EPI_STORE>, max_smem))) return e;
    if ((e = raise_smem_limit(c2r_kernel<LPc, IPc, true, EPI_STORE>, max_smem))) return e;
    if ((e = raise_smem_limit(c2r_kernel<LPc, IPc, false, EPI_RESIDUAL>, max_smem))) return e;
    if ((e = raise_smem_limit(c2r_kernel<LPc, IPc, true, EPI_RESIDUAL>, max_smem))) return e;
    if ((e = raise_smem_limit(c2r_kernel<LPc, IPc, false, EPI_FISTA>, max_smem))) return e;
    if ((e = raise_smem_limit(c2r_r2c_kernel<LPc, IPc, false, EPI_RESIDUAL>, max_smem))) return e;
    if ((e = raise_smem_limit(c2r_r2c_kernel<LPc, IPc, true, EPI_FISTA>, max_smem))) return e;
    return raise_smem_limit(c2r_kernel<LPc, IPc, true, EPI_FISTA>, max_smem);
}

// Fused data-side (residual) or model-side (FISTA update + next stretch)
// half-iteration on the column-blocked solver state, in place on the
// spectrum (see c2r_r2c_kernel).
cudaError_t launch_c2r_r2c(Plan &p, bool model_side, float2 *spec, const float *aux,
                           FistaArgs fa, cudaStream_t st) {
    const ColGroup *cg = model_side ? p.cg_model_blk : p.cg_data_blk;
    const int n = model_side ? p.ncg_model : p.ncg_data;
    const int stage = model_side ? 5 : 2;
    YBound yb{};
    if (!model_side) {
        const cudaError_t e = ybound_reset(p, st, &yb);
        if (e) return e;
    }
    prof_begin(p, stage, st);
    if (model_side) {
        AAHRT_LP_SWITCH(p.lp, AAHRT_INTERP_SWITCH(p.interp, (
            c2r_r2c_kernel<LPc, IPc, true, EPI_FISTA><<<n, time_threads(p.smem_fused_model),
                                                         p.smem_fused_model, st>>>(
                spec, nullptr, fa, cg, p.ST, p.ns, p.S, p.ntau, p.tw_t, p.L, p.nbins,
                YBound{}))));
    } else {
        AAHRT_LP_SWITCH(p.lp, AAHRT_INTERP_SWITCH(p.interp, (
            c2r_r2c_kernel<LPc, IPc, false, EPI_RESIDUAL><<<n, time_threads(p.smem_r2c_data),
                                                           p.smem_r2c_data,
                                                           st>>>(
                spec, aux, FistaArgs{}, cg, p.U, p.ns, p.UT, p.nt, p.tw_t, p.L, p.nbins, yb))));
    }
    prof_end(p, st);
    p.launches[stage]++;
    return cudaGetLastError();
}

cudaError_t set_time_kernel_attrs(int lp, int interp, int max_smem) {
    cudaError_t e = cudaSuccess;
    AAHRT_LP_SWITCH(lp, AAHRT_INTERP_SWITCH(interp, (e = attrs_for<LPc, IPc>(max_smem))));
    return e;
}

}  // namespace aahrt

namespace aahrt {

// The model's stretch S applied to data columns, then the FFT (the first two
// steps of the paper's velocity scan; needs ntau == nt).
cudaError_t launch_stretch_data(Plan &p, const float *d, float2 *Y, cudaStream_t st) {
    prof_begin(p, 3, st);
    AAHRT_LP_SWITCH(p.lp, AAHRT_INTERP_SWITCH(p.interp, (r2c_launch<LPc, IPc>(
        true, p.ncg_data, p.smem_r2c_model, st, d, Y, p.cg_data, p.S, p.nt, p.tw_t, p.L,
        p.nbins))));
    prof_end(p, st);
    p.launches[3]++;
    return cudaGetLastError();
}

// Hermitian synthesis and the stretch undone (U) on model columns (its last
// steps; ntau == nt).
cudaError_t launch_unstretch_model(Plan &p, const float2 *X, float *m, cudaStream_t st) {
    prof_begin(p, 5, st);
    AAHRT_LP_SWITCH(p.lp, AAHRT_INTERP_SWITCH(p.interp, (c2r_launch<LPc, IPc, EPI_STORE>(
        false, p.ncg_model, p.smem_c2r_data, st, X, m, nullptr, FistaArgs{}, p.cg_model, p.U,
        p.ns, p.tw_t, p.L, p.nbins))));
    prof_end(p, st);
    p.launches[5]++;
    return cudaGetLastError();
}

}  // namespace aahrt
