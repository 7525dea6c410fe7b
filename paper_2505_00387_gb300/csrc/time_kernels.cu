// Time-axis stages of the AAHRT (Algorithms 1 and 2, steps 1-2 and 4-5):
//
//   r2c: X[k][c] = sum_n (G in)[n][c] exp(-2 pi i k n / Nfft), k < nbins
//        where G is a sparse resampler applied to each column: the time
//        stretch S (model side, Alg. 1 steps 1-2) or the transpose of its
//        undoing U^T (data side, the adjoint's first two stages).
//   c2r: out[i][c] = sum_n G[i][n] H(X[.][c])[n] with the band-limited
//        Hermitian synthesis H(X)[n] = Re X_0 + 2 Re sum_{k>=1} X_k e^{+2 pi i k n/Nfft}
//        and G = U (data side, Alg. 1 steps 4-5) or S^T (model side, the
//        adjoint's last two stages).  Epilogues fuse the FISTA residual
//        r = d - L z and the soft-threshold/momentum update (eqs. ISTA, soft).
//
// One block owns up to 2*pairs adjacent columns; two real columns travel as
// the real and imaginary parts of one complex FFT of length Nfft held in
// shared memory (padded layout of fft.cuh).  The resampler rows are CSR
// (row pointer, input index, weight) shared by every column.
#include "fft.cuh"
#include "internal.cuh"

namespace aahrt {

__global__ void __launch_bounds__(kThreadsTime)
r2c_kernel(const float *__restrict__ in, float2 *__restrict__ out,
           const ColGroup *__restrict__ groups, DevCSR gat,
           const float2 *__restrict__ tw, int L, int nbins) {
    extern __shared__ float2 sm[];
    const ColGroup cg = groups[blockIdx.x];
    const int N = 1 << L;
    const int ld = padded_len(N);
    const int P = (cg.ncol + 1) >> 1;
    const float *src = in + cg.real_off;

    // gather: z_p[n] = sum_e val[e] * (src[col[e]][2p] + i src[col[e]][2p+1])
    for (int idx = threadIdx.x; idx < P * N; idx += blockDim.x) {
        const int p = idx % P;
        const int n = idx / P;
        float zr = 0.f, zi = 0.f;
        if (n < gat.nrows) {
            const int e0 = __ldg(gat.rowptr + n), e1 = __ldg(gat.rowptr + n + 1);
            const bool hasb = 2 * p + 1 < cg.ncol;
            for (int e = e0; e < e1; ++e) {
                const float wv = __ldg(gat.val + e);
                const float *rowp = src + (long long)__ldg(gat.col + e) * cg.ld_real + 2 * p;
                zr = fmaf(wv, __ldg(rowp), zr);
                if (hasb) zi = fmaf(wv, __ldg(rowp + 1), zi);
            }
        }
        sm[p * ld + padi(n)] = make_float2(zr, zi);
    }
    __syncthreads();
    block_fft_dif<false>(sm, ld, P, L, tw);

    // unpack the two real spectra: A = (Z_k + conj Z_{N-k})/2, B = (Z_k - conj Z_{N-k})/(2i)
    float2 *dst = out + cg.spec_off;
    for (int idx = threadIdx.x; idx < P * nbins; idx += blockDim.x) {
        const int p = idx % P;
        const int k = idx / P;
        const float2 zk = sm[p * ld + padi(brev_bits(k, L))];
        const float2 zn = sm[p * ld + padi(brev_bits((N - k) & (N - 1), L))];
        const float2 A = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
        const float2 B = make_float2(0.5f * (zk.y + zn.y), -0.5f * (zk.x - zn.x));
        const long long o = (long long)k * cg.ld_spec + 2 * p;
        dst[o] = A;
        if (2 * p + 1 < cg.ncol) dst[o + 1] = B;
    }
}

__device__ __forceinline__ float soft_threshold(float x, float t) {
    // x * max(1 - t/|x|, 0) of eq. soft, written without the division
    return copysignf(fmaxf(fabsf(x) - t, 0.f), x);
}

template <int EPI>
__global__ void __launch_bounds__(kThreadsTime)
c2r_kernel(const float2 *__restrict__ in, float *__restrict__ out,
           const float *__restrict__ aux, FistaArgs fa,
           const ColGroup *__restrict__ groups, DevCSR gat,
           const float2 *__restrict__ tw, int L, int nbins) {
    extern __shared__ float2 sm[];
    const ColGroup cg = groups[blockIdx.x];
    const int N = 1 << L;
    const int half = N >> 1;
    const int ld = padded_len(N);
    const int P = (cg.ncol + 1) >> 1;
    const float2 *src = in + cg.spec_off;

    // pack Z = A + iB over the full frame, bit-reversed for the DIT pass
    for (int idx = threadIdx.x; idx < P * (half + 1); idx += blockDim.x) {
        const int p = idx % P;
        const int k = idx / P;
        float2 zk = make_float2(0.f, 0.f), zn = zk;
        if (k < nbins) {
            const long long o = (long long)k * cg.ld_spec + 2 * p;
            float2 A = __ldg(src + o);
            float2 B = (2 * p + 1 < cg.ncol) ? __ldg(src + o + 1) : make_float2(0.f, 0.f);
            if (k == 0) { A.y = 0.f; B.y = 0.f; }
            zk = make_float2(A.x - B.y, A.y + B.x);   // A + iB
            zn = make_float2(A.x + B.y, B.x - A.y);   // conj(A) + i conj(B)
        }
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
    __syncthreads();
    block_fft_dit<true>(sm, ld, P, L, tw);

    // resample the synthesized columns onto the output rows
    for (int idx = threadIdx.x; idx < P * gat.nrows; idx += blockDim.x) {
        const int p = idx % P;
        const int i = idx / P;
        const int e0 = __ldg(gat.rowptr + i), e1 = __ldg(gat.rowptr + i + 1);
        float va = 0.f, vb = 0.f;
        for (int e = e0; e < e1; ++e) {
            const float wv = __ldg(gat.val + e);
            const float2 z = sm[p * ld + padi(__ldg(gat.col + e))];
            va = fmaf(wv, z.x, va);
            vb = fmaf(wv, z.y, vb);
        }
        const long long o = cg.real_off + (long long)i * cg.ld_real + 2 * p;
        const bool hasb = 2 * p + 1 < cg.ncol;
        if (EPI == EPI_STORE) {
            out[o] = va;
            if (hasb) out[o + 1] = vb;
        } else if (EPI == EPI_RESIDUAL) {
            out[o] = __ldg(aux + o) - va;
            if (hasb) out[o + 1] = __ldg(aux + o + 1) - vb;
        } else {
            // m+ = soft(z + gamma g, gamma lambda); z+ = m+ + beta (m+ - m)
            float g[2] = {va, vb};
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if (c == 1 && !hasb) break;
                const float mo = fa.m[o + c];
                const float zo = fa.z[o + c];
                const float mn = soft_threshold(fmaf(fa.gamma, g[c], zo), fa.thresh);
                fa.m[o + c] = mn;
                fa.z[o + c] = fmaf(fa.beta, mn - mo, mn);
            }
        }
    }
}

cudaError_t launch_r2c(Plan &p, bool model_side, const float *in, float2 *out,
                       cudaStream_t st) {
    const ColGroup *cg = model_side ? p.cg_model : p.cg_data;
    const int n = model_side ? p.ncg_model : p.ncg_data;
    const DevCSR gat = model_side ? p.S : p.UT;
    const int stage = model_side ? 0 : 3;
    prof_begin(p, stage, st);
    r2c_kernel<<<n, kThreadsTime, p.smem_r2c, st>>>(in, out, cg, gat, p.tw_t, p.L, p.nbins);
    prof_end(p, st);
    p.launches[stage]++;
    return cudaGetLastError();
}

cudaError_t launch_c2r(Plan &p, bool model_side, const float2 *in, float *out,
                       int epi, const float *aux, FistaArgs fa, cudaStream_t st) {
    const ColGroup *cg = model_side ? p.cg_model : p.cg_data;
    const int n = model_side ? p.ncg_model : p.ncg_data;
    const DevCSR gat = model_side ? p.ST : p.U;
    const int stage = model_side ? 5 : 2;
    prof_begin(p, stage, st);
    switch (epi) {
        case EPI_RESIDUAL:
            c2r_kernel<EPI_RESIDUAL><<<n, kThreadsTime, p.smem_c2r, st>>>(
                in, out, aux, fa, cg, gat, p.tw_t, p.L, p.nbins);
            break;
        case EPI_FISTA:
            c2r_kernel<EPI_FISTA><<<n, kThreadsTime, p.smem_c2r, st>>>(
                in, out, aux, fa, cg, gat, p.tw_t, p.L, p.nbins);
            break;
        default:
            c2r_kernel<EPI_STORE><<<n, kThreadsTime, p.smem_c2r, st>>>(
                in, out, aux, fa, cg, gat, p.tw_t, p.L, p.nbins);
            break;
    }
    prof_end(p, st);
    p.launches[stage]++;
    return cudaGetLastError();
}

cudaError_t set_time_kernel_attrs(size_t smem) {
    cudaError_t e;
    const int s = (int)smem;
    if ((e = cudaFuncSetAttribute(r2c_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, s)))
        return e;
    if ((e = cudaFuncSetAttribute(c2r_kernel<EPI_STORE>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, s)))
        return e;
    if ((e = cudaFuncSetAttribute(c2r_kernel<EPI_RESIDUAL>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, s)))
        return e;
    return cudaFuncSetAttribute(c2r_kernel<EPI_FISTA>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, s);
}

}  // namespace aahrt
