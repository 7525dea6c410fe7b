// Fourier slice stage of the AAHRT (Algorithm 1 step 3 and its exact
// transpose; eqs. Inv_op, inv_GFST and the theta factors of eq. thli).
//
// Forward, per bin k and trace h (scale = 1/Nfft folds the synthesis factor):
//   Y[k][h] = scale * sum_{s=0,1} w_s(h) * sum_l X[k][l][j_s(h)] exp(-2 pi i f_k q_l r_h^2)
// evaluated as a type-2 non-uniform DFT along q: the slice columns are
// deapodised, centred, DFT'd on an nos-point grid in shared memory, and each
// trace interpolates W grid points per slice with the spreading kernel.
// Adjoint: each trace spreads scale * conj(phase) * Y into the grid with
// shared-memory atomics, the grid is inverse-DFT'd and deapodised: the exact
// transpose of the forward (same taps, weights, phases and twiddles).
//
// Work items are (cube, azimuth group, bin); a persistent grid pulls them
// from an atomic counter (reset by the launcher), largest groups first.
#include "fft.cuh"
#include "internal.cuh"
#include "slice_math.cuh"

namespace aahrt {

struct SliceArgs {
    const TraceGeo *__restrict__ geo;
    const SliceGroup *__restrict__ groups;
    const float *__restrict__ dec;
    const float2 *__restrict__ tw;
    int *counter;
    long long total;
    int nbins, nq, ntheta, nos, Lq, cq, ngroup;
    float beta, scale;
};

template <int W>
__global__ void __launch_bounds__(kThreadsSlice)
slice_fwd_kernel(SliceArgs a, const float2 *__restrict__ X, float2 *__restrict__ Y) {
    extern __shared__ float2 G[];
    __shared__ long long s_item;
    const int ldg = padded_len(a.nos);
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

        // deapodised, centred columns into bit-reversed grid positions
        const float2 *Xk = X + g.x_off + (long long)k * a.nq * a.ntheta;
        for (int idx = threadIdx.x; idx < ncolj * a.nq; idx += blockDim.x) {
            const int jj = idx % ncolj;
            const int l = idx / ncolj;
            int j = g.ja + jj;
            if (j >= a.ntheta) j -= a.ntheta;
            const float2 x = __ldg(Xk + (long long)l * a.ntheta + j);
            const float dl = __ldg(a.dec + l);
            const int u = (l - a.cq) & mask;
            G[jj * ldg + padi(brev_bits(u, a.Lq))] = make_float2(x.x * dl, x.y * dl);
        }
        const int nz = a.nos - a.nq;
        for (int idx = threadIdx.x; idx < ncolj * nz; idx += blockDim.x) {
            const int jj = idx % ncolj;
            const int i = idx / ncolj;
            const int u = (a.nq - a.cq + i) & mask;
            G[jj * ldg + padi(brev_bits(u, a.Lq))] = make_float2(0.f, 0.f);
        }
        __syncthreads();
        block_fft_dit<false>(G, ldg, ncolj, a.Lq, a.tw);

        // interpolate every owned trace
        const TraceGeo *geo = a.geo + g.geo_off;
        float2 *Yk = Y + g.y_off + (long long)k * g.ntr;
        for (int t = g.f0 + threadIdx.x; t < g.f1; t += blockDim.x) {
            const TraceGeo tr = geo[t];
            const TapSet ts = trace_taps<W>(tr.A, tr.B, (unsigned)k, a.Lq);
            float phi[W];
            es_weights<W>(ts.z0, a.beta, phi);
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
            float ar = 0.f, ai = 0.f;
#pragma unroll
            for (int i = 0; i < W; ++i) {
                const int u = padi((ts.u0 + i) & mask);
                const float2 g0 = G0[u], g1 = G1[u];
                const float c0 = phi[i] * tr.w0, c1 = phi[i] * tr.w1;
                ar = fmaf(c0, g0.x, fmaf(c1, g1.x, ar));
                ai = fmaf(c0, g0.y, fmaf(c1, g1.y, ai));
            }
            float sn, cs;
            sincospif(2.0f * ts.ph, &sn, &cs);
            // times exp(-2 pi i ph) = cs - i sn
            Yk[tr.col] = make_float2(a.scale * (ar * cs + ai * sn), a.scale * (ai * cs - ar * sn));
        }
        __syncthreads();
    }
}

template <int W>
__device__ __forceinline__ void spread_trace(const SliceArgs &a, const SliceGroup &g,
                                             const TraceGeo &tr, const float2 *Yk,
                                             int k, float2 *G, int ldg, int mask) {
    const TapSet ts = trace_taps<W>(tr.A, tr.B, (unsigned)k, a.Lq);
    float phi[W];
    es_weights<W>(ts.z0, a.beta, phi);
    const float2 y = __ldg(Yk + tr.col);
    float sn, cs;
    sincospif(2.0f * ts.ph, &sn, &cs);
    // scale * y * exp(+2 pi i ph)
    const float vr = a.scale * (y.x * cs - y.y * sn);
    const float vi = a.scale * (y.x * sn + y.y * cs);
    const int jj0 = tr.j0 - g.ja;
    int j1 = tr.j0 + 1;
    if (j1 == a.ntheta) j1 = 0;
    const int jj1 = j1 - g.ja;
    const bool own0 = jj0 >= 0 && jj0 < g.nj;
    const bool own1 = jj1 >= 0 && jj1 < g.nj;
    float *G0 = reinterpret_cast<float *>(G + (own0 ? jj0 : 0) * ldg);
    float *G1 = reinterpret_cast<float *>(G + (own1 ? jj1 : 0) * ldg);
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const int u = 2 * padi((ts.u0 + i) & mask);
        if (own0) {
            const float c = phi[i] * tr.w0;
            atomicAdd(G0 + u, c * vr);
            atomicAdd(G0 + u + 1, c * vi);
        }
        if (own1) {
            const float c = phi[i] * tr.w1;
            atomicAdd(G1 + u, c * vr);
            atomicAdd(G1 + u + 1, c * vi);
        }
    }
}

template <int W>
__global__ void __launch_bounds__(kThreadsSlice)
slice_adj_kernel(SliceArgs a, const float2 *__restrict__ Y, float2 *__restrict__ X) {
    extern __shared__ float2 G[];
    __shared__ long long s_item;
    const int ldg = padded_len(a.nos);
    const int mask = a.nos - 1;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(a.counter, 1);
        __syncthreads();
        const long long item = s_item;
        if (item >= a.total) break;
        const int gi = (int)(item / a.nbins);
        const int k = (int)(item - (long long)gi * a.nbins);
        const SliceGroup g = a.groups[gi];

        for (int idx = threadIdx.x; idx < g.nj * ldg; idx += blockDim.x)
            G[idx] = make_float2(0.f, 0.f);
        __syncthreads();

        const TraceGeo *geo = a.geo + g.geo_off;
        const float2 *Yk = Y + g.y_off + (long long)k * g.ntr;
        for (int t = g.f0 + threadIdx.x; t < g.f1; t += blockDim.x)
            spread_trace<W>(a, g, geo[t], Yk, k, G, ldg, mask);
        for (int t = g.e0 + threadIdx.x; t < g.e1; t += blockDim.x)
            spread_trace<W>(a, g, geo[t], Yk, k, G, ldg, mask);
        __syncthreads();
        block_fft_dif<true>(G, ldg, g.nj, a.Lq, a.tw);

        float2 *Xk = X + g.x_off + (long long)k * a.nq * a.ntheta;
        for (int idx = threadIdx.x; idx < g.nj * a.nq; idx += blockDim.x) {
            const int jj = idx % g.nj;
            const int l = idx / g.nj;
            const int u = (l - a.cq) & mask;
            const float2 v = G[jj * ldg + padi(brev_bits(u, a.Lq))];
            const float dl = __ldg(a.dec + l);
            Xk[(long long)l * a.ntheta + g.ja + jj] = make_float2(v.x * dl, v.y * dl);
        }
        __syncthreads();
    }
}

static SliceArgs make_args(const Plan &p, int counter_slot) {
    SliceArgs a;
    a.geo = p.geo;
    a.groups = p.groups;
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
    a.beta = (float)p.beta;
    a.scale = (float)(1.0 / p.nfft);
    return a;
}

#define AAHRT_W_CASES(X) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12)

cudaError_t launch_slice(Plan &p, bool adjoint, const float2 *in, float2 *out,
                         cudaStream_t st) {
    const int slot = adjoint ? 1 : 0;
    const int stage = adjoint ? 4 : 1;
    cudaError_t e = cudaMemsetAsync(p.counters + slot, 0, sizeof(int), st);
    if (e) return e;
    const SliceArgs a = make_args(p, slot);
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
cudaError_t configure_slice_kernels(Plan &p, int num_sms) {
    cudaError_t e = cudaSuccess;
    int occ_f = 0, occ_a = 0;
    switch (p.w) {
#define AAHRT_CASE(WW)                                                                   \
    case WW:                                                                            \
        if ((e = cudaFuncSetAttribute(slice_fwd_kernel<WW>,                              \
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                                      (int)p.smem_sfwd)))                                \
            return e;                                                                   \
        if ((e = cudaFuncSetAttribute(slice_adj_kernel<WW>,                              \
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                                      (int)p.smem_sadj)))                                \
            return e;                                                                   \
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
