// Fourier slice stage of the AAHRT (Algorithm 1 step 3 and its exact
// transpose; eqs. Inv_op, inv_GFST and the theta factors of eq. thli).
//
// Forward, per bin k and trace h (scale = 1/Nfft folds the synthesis factor):
//   Y[k][h] = scale * sum_{s=0,1} w_s(h) * sum_l X[k][l][j_s(h)] exp(-2 pi i f_k q_l r_h^2)
// evaluated as a type-2 non-uniform DFT along q: the slice columns are
// deapodised, centred, DFT'd on an nos-point grid in shared memory, and each
// trace interpolates W grid points per slice with the spreading kernel.
// Adjoint: each trace spreads scale * conj(phase) * Y into the grid, the grid
// is inverse-DFT'd and deapodised: the transpose of the forward (same taps,
// weights, phases and twiddles).  The spread accumulates in 32-bit fixed
// point with native shared-memory integer atomics (real and imaginary parts in
// separate planes).  Each azimuth slice gets its own scale
// 2^30 / (Phi_max * scale * M * sum_h w_h) over the traces h that reach it,
// where M bounds |re y| + |im y| over the cube's bins in a chunk of 2^b bins
// (computed by the data-side analysis that wrote Y): no grid sum can exceed
// 2^30, and the rounding of each contribution stays near FP32 rounding of the
// slice's values.
//
// Work items are (cube, azimuth group, bin); a persistent grid pulls them
// from an atomic counter (reset by the launcher), largest groups first.
#include "fft.cuh"
#include "internal.cuh"
#include "slice_math.cuh"

namespace aahrt {

struct SliceArgs {
    const TraceGeo *__restrict__ geo;       // forward order (by slice, then r^2)
    const TraceGeo *__restrict__ geo_adj;   // adjoint order (by slice, then trace)
    const SliceGroup *__restrict__ groups;
    const int *__restrict__ slice_start;
    const float *__restrict__ dec;
    const float2 *__restrict__ tw;
    int *counter;
    long long total;
    int nbins, nq, ntheta, nos, Lq, cq, ngroup;
    float scale;
    float phimax;    // max over positions of sum_i phi_i (spread bound)
    const unsigned *__restrict__ ymax;   // [cube][chunk] max |re| + |im| of Y (float bits)
    const float *__restrict__ wsum;      // [cube][slice] azimuth weight reaching the slice
    int nychunk, ychunk_log;
    EsPoly poly;     // kernel-parameter (constant) bank: broadcast FMA operands
};

// a / d for 0 <= a < 2^20, d < 2^10, by a float reciprocal and one correction.
__device__ __forceinline__ int fast_div(int a, int d, float inv_d) {
    int q = __float2int_rz(((float)a + 0.5f) * inv_d);
    const int r = a - q * d;
    if (r < 0) --q;
    else if (r >= d) ++q;
    return q;
}

template <int W>
__global__ void __launch_bounds__(kThreadsSlice, 3)
slice_fwd_kernel(const SliceArgs a, const float2 *__restrict__ X, float2 *__restrict__ Y) {
    extern __shared__ float4 smem_f4[];
    float2 *G = reinterpret_cast<float2 *>(smem_f4);
    __shared__ long long s_item;
    const int ldg = ld_interleaved(a.nos);
    const int mask = a.nos - 1;
    const int extra = a.ngroup > 1 ? 1 : 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(a.counter, 1);
        __syncthreads();
        const long long item = s_item;
        if (item >= a.total) break;
        const int gi = (int)(item / a.nbins);
        const int k = (int)(item - (long long)gi * a.nbins);
        const SliceGroup g = a.groups[gi];
        const int ncolj = g.nj + extra;

        // First DIT step fused with the column load: element m of group g0
        // (bit-reversed position 16 g0 + m) is grid point
        // u = brev(16 g0 + m) = (brev4(m) << (Lq - 4)) | brev(g0), holding the
        // deapodised column entry l = (u + cq) mod nos when l < nq, else zero.
        {
            const float2 *Xk = X + g.x_off + (long long)k * a.nq * a.ntheta;
            const float inv_nc = 1.0f / (float)ncolj;
            const int items = (a.nos >> 4) * ncolj;
            int off0[16];
            group_offsets<4>(0, off0);
            for (int w = threadIdx.x; w < items; w += blockDim.x) {
                const int g0 = fast_div(w, ncolj, inv_nc);
                const int jj = w - g0 * ncolj;
                int j = g.ja + jj;
                if (j >= a.ntheta) j -= a.ntheta;
                const int ug = (int)brev_bits(g0, a.Lq - 4);
                float2 v[16];
#pragma unroll
                for (int m = 0; m < 16; ++m) {
                    const int u = (rev_bits_c<4>(m) << (a.Lq - 4)) | ug;
                    const int l = (u + a.cq) & mask;
                    v[m] = make_float2(0.f, 0.f);
                    if (l < a.nq) {
                        const float2 x = __ldg(Xk + (long long)l * a.ntheta + j);
                        const float dl = __ldg(a.dec + l);
                        v[m] = make_float2(x.x * dl, x.y * dl);
                    }
                }
                dit_network<4, false>(v);
                float2 *col = G + jj * ldg + padi(g0 << 4);
#pragma unroll
                for (int m = 0; m < 16; ++m) col[off0[m]] = v[m];
            }
        }
        __syncthreads();
        block_fft<false, false>(IBatch{G, ldg}, ncolj, a.Lq, a.tw, 4);

        // interpolate every owned trace
        const TraceGeo *geo = a.geo + g.geo_off;
        float2 *Yk = Y + g.y_off + (long long)k * g.ntr;
        // the next trace's record is loaded while this one is interpolated
        TraceGeo nxt{};
        if (g.f0 + (int)threadIdx.x < g.f1) nxt = geo[g.f0 + threadIdx.x];
        for (int t = g.f0 + threadIdx.x; t < g.f1; t += blockDim.x) {
            const TraceGeo tr = nxt;
            if (t + (int)blockDim.x < g.f1) nxt = geo[t + blockDim.x];
            const TapSet ts = trace_taps<W>(tr.A, tr.B, (unsigned)k, a.Lq);
            float phi[W];
            es_weights<W>(a.poly, ts.g, phi);
            const int jj0 = tr.j0 - g.ja;
            int jj1;
            if (extra) {
                jj1 = jj0 + 1;
            } else {
                jj1 = tr.j0 + 1;
                if (jj1 == a.ntheta) jj1 = 0;
            }
            const float2 *G0 = G + jj0 * ldg;
            const float2 *G1 = G + jj1 * ldg;
            float ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f;
#pragma unroll
            for (int i = 0; i < W; ++i) {
                const int u = padi((ts.u0 + i) & mask);
                const float2 g0 = G0[u], g1 = G1[u];
                ar = fmaf(phi[i], g0.x, ar);
                ai = fmaf(phi[i], g0.y, ai);
                br = fmaf(phi[i], g1.x, br);
                bi = fmaf(phi[i], g1.y, bi);
            }
            ar = fmaf(tr.w0, ar, tr.w1 * br);
            ai = fmaf(tr.w0, ai, tr.w1 * bi);
            float sn, cs;
            phase_cs(ts.ph, &sn, &cs);
            // times exp(-2 pi i ph) = cs - i sn
            Yk[tr.col] = make_float2(a.scale * (ar * cs + ai * sn), a.scale * (ai * cs - ar * sn));
        }
        __syncthreads();
    }
}

template <int W>
__device__ __forceinline__ void spread_trace(const SliceArgs &a, const SliceGroup &g,
                                             const TraceGeo &tr, float2 y, int k,
                                             int *Gre, int *Gim, int lds, int mask,
                                             const float *fx) {
    const TapSet ts = trace_taps<W>(tr.A, tr.B, (unsigned)k, a.Lq);
    float phi[W];
    es_weights<W>(a.poly, ts.g, phi);
    float sn, cs;
    phase_cs(ts.ph, &sn, &cs);
    // scale * y * exp(+2 pi i ph)
    const float vr = a.scale * (y.x * cs - y.y * sn);
    const float vi = a.scale * (y.x * sn + y.y * cs);
    const int jj0 = tr.j0 - g.ja;
    int j1 = tr.j0 + 1;
    if (j1 == a.ntheta) j1 = 0;
    const int jj1 = j1 - g.ja;
    const bool own0 = jj0 >= 0 && jj0 < g.nj;
    const bool own1 = jj1 >= 0 && jj1 < g.nj;
    const int c0 = own0 ? jj0 : 0, c1 = own1 ? jj1 : 0;
    const int o0 = c0 * lds, o1 = c1 * lds;
    const float f0 = tr.w0 * fx[c0], f1 = tr.w1 * fx[c1];
    const float ar = f0 * vr, ai = f0 * vi, br = f1 * vr, bi = f1 * vi;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const int u = padi((ts.u0 + i) & mask);
        if (own0) {
            atomicAdd(Gre + o0 + u, __float2int_rn(phi[i] * ar));
            atomicAdd(Gim + o0 + u, __float2int_rn(phi[i] * ai));
        }
        if (own1) {
            atomicAdd(Gre + o1 + u, __float2int_rn(phi[i] * br));
            atomicAdd(Gim + o1 + u, __float2int_rn(phi[i] * bi));
        }
    }
}

// First DIF step of the adjoint's inverse q-FFT fused with the conversion of
// the fixed-point grid: group j of column jj holds elements j + (m << (Lq-4));
// it reads them as integers, scales them back (1/fx of the column), applies
// the constant radix-16 network and the post-twiddles, and stores floats in
// place.
__device__ __forceinline__ void adj_first_step(const SliceArgs &a, const SliceGroup &g,
                                               float *smf, int lds, const float *ifx) {
    const int lhs = a.Lq - 4;
    const int ng = 1 << lhs;
    int off[16];
    group_offsets<4>(lhs, off);
    float *Gre = smf, *Gim = smf + g.nj * lds;
    const int *Ire = reinterpret_cast<const int *>(Gre);
    const int *Iim = reinterpret_cast<const int *>(Gim);
    // the column (slice) varies fastest across a warp's lanes: with the
    // column stride lds = 1 modulo the bank count, consecutive columns fall
    // in consecutive banks (at most 2-way conflicts, against 4-way when a warp
    // covered 4 columns x 8 groups)
    const float inv_nj = 1.0f / (float)g.nj;
    for (int w = threadIdx.x; w < ng * g.nj; w += blockDim.x) {
        const int j = fast_div(w, g.nj, inv_nj);
        const int jj = w - j * g.nj;
        const float f = ifx[jj];
        const int pb = jj * lds + padi(j);
        float2 v[16];
#pragma unroll
        for (int m = 0; m < 16; ++m)
            v[m] = make_float2((float)Ire[pb + off[m]] * f, (float)Iim[pb + off[m]] * f);
        dif_network<4, true>(v);
        group_twiddle<4, true>(v, j, a.Lq, a.Lq, a.tw);
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            Gre[pb + off[m]] = v[m].x;
            Gim[pb + off[m]] = v[m].y;
        }
    }
}

// Last DIF step (radix 2^A, no post-twiddles) fused with the deapodised
// output: output position p = (gg << A) + m is grid point u = brev(p), i.e.
// column entry l = (u + cq) mod nos, written when l < nq.
template <int A>
__device__ __forceinline__ void adj_last_step(const SliceArgs &a, const SliceGroup &g,
                                              const float *Gre, const float *Gim, int lds,
                                              int k, float2 *__restrict__ X) {
    constexpr int R = 1 << A;
    const int items = (1 << (a.Lq - A)) * g.nj;
    const float inv_nj = 1.0f / (float)g.nj;
    const int mask = a.nos - 1;
    int off[R];
    group_offsets<A>(0, off);
    float2 *Xk = X + g.x_off + (long long)k * a.nq * a.ntheta + g.ja;
    for (int w = threadIdx.x; w < items; w += blockDim.x) {
        const int gg = fast_div(w, g.nj, inv_nj);
        const int jj = w - gg * g.nj;
        const int base = gg << A;
        const int pb = jj * lds + padi(base);
        float2 v[R];
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = make_float2(Gre[pb + off[m]], Gim[pb + off[m]]);
        dif_network<A, true>(v);
#pragma unroll
        for (int m = 0; m < R; ++m) {
            const int l = ((int)brev_bits(base + m, a.Lq) + a.cq) & mask;
            if (l < a.nq) {
                const float dl = __ldg(a.dec + l);
                Xk[(long long)l * a.ntheta + jj] = make_float2(v[m].x * dl, v[m].y * dl);
            }
        }
    }
}

template <int W>
__global__ void __launch_bounds__(kThreadsSlice, 3)
slice_adj_kernel(const SliceArgs a, const float2 *__restrict__ Y, float2 *__restrict__ X) {
    extern __shared__ float4 smem_f4[];
    float *smf = reinterpret_cast<float *>(smem_f4);
    __shared__ long long s_item;
    __shared__ float s_fx[kMaxGroupSlices], s_ifx[kMaxGroupSlices];
    const int lds = ld_split(a.nos);
    const int mask = a.nos - 1;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(a.counter, 1);
        __syncthreads();
        const long long item = s_item;
        if (item >= a.total) break;
        const int gi = (int)(item / a.nbins);
        const int k = (int)(item - (long long)gi * a.nbins);
        const SliceGroup g = a.groups[gi];
        float *Gre = smf;
        float *Gim = smf + g.nj * lds;
        int *Ire = reinterpret_cast<int *>(Gre);
        int *Iim = reinterpret_cast<int *>(Gim);
        const TraceGeo *geo = a.geo_adj + g.geo_off;
        const float2 *Yk = Y + g.y_off + (long long)k * g.ntr;

        // zero the grid; per owned slice, the fixed-point scale from the
        // chunk's amplitude bound and the slice's total azimuth weight
        {
            const int nz4 = (2 * g.nj * lds) >> 2;
            float4 *z4 = reinterpret_cast<float4 *>(smf);
            for (int idx = threadIdx.x; idx < nz4; idx += blockDim.x)
                z4[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int idx = 4 * nz4 + threadIdx.x; idx < 2 * g.nj * lds; idx += blockDim.x)
                smf[idx] = 0.f;
        }
        {
            const float M = __uint_as_float(
                __ldg(a.ymax + (long long)g.cube * a.nychunk + (k >> a.ychunk_log)));
            const float *ws = a.wsum + (long long)g.cube * a.ntheta + g.ja;
            for (int jj = threadIdx.x; jj < g.nj; jj += blockDim.x) {
                const float bound = M * __ldg(ws + jj) * a.scale * a.phimax;
                s_fx[jj] = bound > 0.f ? 1073741824.0f / bound : 0.f;   // 2^30 / bound
                s_ifx[jj] = bound > 0.f ? bound * 9.3132257461547852e-10f : 0.f;   // 1/fx
            }
        }
        __syncthreads();

        // the next trace's record is loaded while this one is spread, and
        // this one's y at the top, ahead of the taps and weights
        for (int r = 0; r < 2; ++r) {
            const int t0 = r == 0 ? g.f0 : g.e0, t1 = r == 0 ? g.f1 : g.e1;
            TraceGeo nxt{};
            if (t0 + (int)threadIdx.x < t1) nxt = geo[t0 + threadIdx.x];
            for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
                const TraceGeo tr = nxt;
                const float2 y = __ldg(Yk + tr.col);
                if (t + (int)blockDim.x < t1) nxt = geo[t + blockDim.x];
                spread_trace<W>(a, g, tr, y, k, Ire, Iim, lds, mask, s_fx);
            }
        }
        __syncthreads();
        if (a.Lq >= 5) {
            adj_first_step(a, g, smf, lds, s_ifx);
            __syncthreads();
            const int s_last = 4 * ((a.Lq - 1) >> 2);
            block_fft<true, true>(SBatch{Gre, Gim, lds}, g.nj, a.Lq, a.tw, 4, s_last);
            switch (a.Lq - s_last) {
                case 4: adj_last_step<4>(a, g, Gre, Gim, lds, k, X); break;
                case 3: adj_last_step<3>(a, g, Gre, Gim, lds, k, X); break;
                case 2: adj_last_step<2>(a, g, Gre, Gim, lds, k, X); break;
                default: adj_last_step<1>(a, g, Gre, Gim, lds, k, X); break;
            }
        } else {
            // back to floating point, in place (slice jj sits in rows jj and nj + jj)
            for (int row = threadIdx.x >> 5; row < 2 * g.nj; row += kThreadsSlice / 32) {
                const float f = s_ifx[row < g.nj ? row : row - g.nj];
                float *rp = smf + row * lds;
                for (int u = threadIdx.x & 31; u < lds; u += 32)
                    rp[u] = (float)reinterpret_cast<int *>(rp)[u] * f;
            }
            __syncthreads();
            block_fft<true, true>(SBatch{Gre, Gim, lds}, g.nj, a.Lq, a.tw);
            float2 *Xk = X + g.x_off + (long long)k * a.nq * a.ntheta;
            const float inv_nj = 1.0f / (float)g.nj;
            for (int idx = threadIdx.x; idx < g.nj * a.nq; idx += blockDim.x) {
                const int l = fast_div(idx, g.nj, inv_nj);
                const int jj = idx - l * g.nj;
                const int u = padi(brev_bits((l - a.cq) & mask, a.Lq));
                const float dl = __ldg(a.dec + l);
                Xk[(long long)l * a.ntheta + g.ja + jj] =
                    make_float2(Gre[jj * lds + u] * dl, Gim[jj * lds + u] * dl);
            }
        }
        __syncthreads();
    }
}

// The spectrum bound table ymax from a given Y (for a slice adjoint whose
// input was not written by the data-side analysis): block (group, chunk)
// raises ymax[cube][chunk] to the largest |re| + |im| over the chunk's bins
// and the cube's traces.
__global__ void ybound_kernel(const SliceGroup *__restrict__ groups,
                              const float2 *__restrict__ Y, int nbins, int chunk_log,
                              int nchunk, unsigned *__restrict__ ymax) {
    const SliceGroup g = groups[blockIdx.x];
    const int k0 = blockIdx.y << chunk_log;
    const int k1 = min(nbins, k0 + (1 << chunk_log));
    const long long n = (long long)(k1 - k0) * g.ntr;
    const float2 *src = Y + g.y_off + (long long)k0 * g.ntr;
    float m = 0.f;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const float2 v = __ldg(src + i);
        m = fmaxf(m, fabsf(v.x) + fabsf(v.y));
    }
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, sh));
    if ((threadIdx.x & 31) == 0 && m > 0.f)
        atomicMax(ymax + (long long)g.cube * nchunk + blockIdx.y, __float_as_uint(m));
}

cudaError_t launch_ybound(Plan &p, const float2 *Y, cudaStream_t st) {
    if (!p.ymax || p.precision == 1 || p.slice_interp == AAHRT_SLICE_DIRECT) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(p.ymax, 0, (size_t)p.ncube * p.nychunk * sizeof(unsigned), st);
    if (e) return e;
    ybound_kernel<<<dim3(p.ngroups_total, p.nychunk), 256, 0, st>>>(
        p.groups, Y, p.nbins, p.ychunk_log, p.nychunk, p.ymax);
    return cudaGetLastError();
}

static SliceArgs make_args(const Plan &p, int counter_slot) {
    SliceArgs a;
    a.geo = p.geo;
    a.geo_adj = p.geo_adj;
    a.groups = p.groups;
    a.slice_start = p.slice_start;
    a.dec = p.dec;
    a.tw = p.tw_q;
    a.counter = p.counters + counter_slot;
    a.total = p.slice_items;
    a.nbins = p.nbins;
    a.nq = p.nq;
    a.ntheta = p.ntheta;
    a.nos = p.nos;
    a.Lq = p.Lq;
    a.cq = p.cq;
    a.ngroup = p.ngroup;
    a.scale = (float)(1.0 / p.nfft);
    a.phimax = (float)p.phimax;
    a.ymax = p.ymax;
    a.wsum = p.wsum;
    a.nychunk = p.nychunk;
    a.ychunk_log = p.ychunk_log;
    a.poly = p.poly;
    return a;
}

#define AAHRT_W_CASES(X) X(2) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12)

cudaError_t launch_slice(Plan &p, bool adjoint, const float2 *in, float2 *out,
                         cudaStream_t st, int *counter) {
    const int slot = adjoint ? 1 : 0;
    const int stage = adjoint ? 4 : 1;
    int *ctr = counter ? counter : p.counters + slot;
    cudaError_t e = cudaMemsetAsync(ctr, 0, sizeof(int), st);
    if (e) return e;
    if (p.precision == 1 || p.slice_interp == AAHRT_SLICE_DIRECT) {
        prof_begin(p, stage, st);
        e = p.precision == 1 ? launch_slice_tc(p, adjoint, in, out, st, ctr)
                             : launch_slice_direct(p, adjoint, in, out, st, ctr);
        prof_end(p, st);
        p.launches[stage]++;
        return e;
    }
    SliceArgs a = make_args(p, slot);
    a.counter = ctr;
    prof_begin(p, stage, st);
    if (!adjoint) {
        switch (p.w) {
#define AAHRT_CASE(WW)                                                              \
    case WW:                                                                       \
        slice_fwd_kernel<WW><<<p.slice_grid_fwd, kThreadsSlice, p.smem_sfwd, st>>>( \
            a, in, out);                                                           \
        break;
            AAHRT_W_CASES(AAHRT_CASE)
#undef AAHRT_CASE
            default: return cudaErrorInvalidValue;
        }
    } else {
        switch (p.w) {
#define AAHRT_CASE(WW)                                                              \
    case WW:                                                                       \
        slice_adj_kernel<WW><<<p.slice_grid_adj, kThreadsSlice, p.smem_sadj, st>>>( \
            a, in, out);                                                           \
        break;
            AAHRT_W_CASES(AAHRT_CASE)
#undef AAHRT_CASE
            default: return cudaErrorInvalidValue;
        }
    }
    prof_end(p, st);
    p.launches[stage]++;
    return cudaGetLastError();
}

// Dynamic shared memory attributes and persistent grid sizes for width w.
cudaError_t configure_slice_kernels(Plan &p, int num_sms, int max_smem) {
    cudaError_t e = cudaSuccess;
    int occ_f = 0, occ_a = 0;
    switch (p.w) {
#define AAHRT_CASE(WW)                                                                   \
    case WW:                                                                            \
        if ((e = raise_smem_limit(slice_fwd_kernel<WW>, max_smem))) return e;            \
        if ((e = raise_smem_limit(slice_adj_kernel<WW>, max_smem))) return e;            \
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(                          \
                 &occ_f, slice_fwd_kernel<WW>, kThreadsSlice, p.smem_sfwd)))             \
            return e;                                                                   \
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(                          \
                 &occ_a, slice_adj_kernel<WW>, kThreadsSlice, p.smem_sadj)))             \
            return e;                                                                   \
        break;
        AAHRT_W_CASES(AAHRT_CASE)
#undef AAHRT_CASE
        default: return cudaErrorInvalidValue;
    }
    if (occ_f < 1 || occ_a < 1) return cudaErrorInvalidConfiguration;
    const long long cap_f = (long long)occ_f * num_sms;
    const long long cap_a = (long long)occ_a * num_sms;
    p.slice_grid_fwd = (int)(p.slice_items < cap_f ? p.slice_items : cap_f);
    p.slice_grid_adj = (int)(p.slice_items < cap_a ? p.slice_items : cap_a);
    return cudaSuccess;
}

}  // namespace aahrt
