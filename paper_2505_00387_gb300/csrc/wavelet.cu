// Deconvolutive AAHRT (Sec. 4, eq. DecRT): R_w^{-1} = W R^{-1}, with W the
// linear convolution of every trace with a wavelet in time.  With the wavelet
// samples w[s] (s < nw) and sample `center` at lag zero:
//   (W x)[i]   = sum_s w[s] x[i - s + center]      (forward, after U)
//   (W^T y)[n] = sum_s w[s] y[n + s - center]      (adjoint, before U^T)
// traces zero outside [0, nt).  One block per data column group: its columns
// are staged in shared memory and every thread produces whole output rows.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace aahrt {

enum WavMode { WAV_CONV = 0, WAV_CONV_RESIDUAL = 1, WAV_CORR = 2 };

template <int MODE>
__global__ void __launch_bounds__(256)
wavelet_kernel(const float *__restrict__ in, float *__restrict__ out,
               const float *__restrict__ aux, const ColGroup *__restrict__ groups, int nt,
               const float *__restrict__ w, int nw, int center) {
    extern __shared__ float4 smem_f4[];
    float *sw = reinterpret_cast<float *>(smem_f4);   // nw wavelet samples
    float *sx = sw + ((nw + 3) & ~3);                 // nt rows x ncol
    const ColGroup cg = groups[blockIdx.x];
    const int nc = cg.ncol;
    for (int s = threadIdx.x; s < nw; s += blockDim.x) sw[s] = w[s];
    for (int idx = threadIdx.x; idx < nt * nc; idx += blockDim.x) {
        const int r = idx / nc, c = idx - r * nc;
        sx[idx] = __ldg(in + cg.real_off + (long long)r * cg.ld_real + c);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nt * nc; idx += blockDim.x) {
        const int i = idx / nc, c = idx - i * nc;
        float acc = 0.f;
        if (MODE == WAV_CORR) {
            // y[i + s - center] for s with 0 <= i + s - center < nt
            const int s0 = max(0, center - i), s1 = min(nw, nt - i + center);
            for (int s = s0; s < s1; ++s) acc = fmaf(sw[s], sx[(i + s - center) * nc + c], acc);
        } else {
            // x[i - s + center] for s with 0 <= i - s + center < nt
            const int s0 = max(0, i + center - nt + 1), s1 = min(nw, i + center + 1);
            for (int s = s0; s < s1; ++s) acc = fmaf(sw[s], sx[(i - s + center) * nc + c], acc);
        }
        const long long o = cg.real_off + (long long)i * cg.ld_real + c;
        out[o] = MODE == WAV_CONV_RESIDUAL ? __ldg(aux + o) - acc : acc;
    }
}

// Data-side column groups in the layout of the call (natural or blocked).
cudaError_t launch_wavelet(Plan &p, int mode, const float *in, float *out, const float *aux,
                           cudaStream_t st, bool blocked) {
    const ColGroup *groups = blocked ? p.cg_data_blk : p.cg_data;
    const size_t smem = (size_t)(((p.nw + 3) & ~3) + p.nt * 2 * p.pairs) * sizeof(float);
    const int grid = p.ncg_data;
    switch (mode) {
        case WAV_CONV:
            wavelet_kernel<WAV_CONV><<<grid, 256, smem, st>>>(in, out, aux, groups, p.nt, p.wav,
                                                               p.nw, p.wcenter);
            break;
        case WAV_CONV_RESIDUAL:
            wavelet_kernel<WAV_CONV_RESIDUAL><<<grid, 256, smem, st>>>(in, out, aux, groups, p.nt,
                                                                        p.wav, p.nw, p.wcenter);
            break;
        default:
            wavelet_kernel<WAV_CORR><<<grid, 256, smem, st>>>(in, out, aux, groups, p.nt, p.wav,
                                                               p.nw, p.wcenter);
            break;
    }
    return cudaGetLastError();
}

cudaError_t configure_wavelet_kernels(int max_smem) {
    cudaError_t e;
    if ((e = raise_smem_limit(wavelet_kernel<WAV_CONV>, max_smem))) return e;
    if ((e = raise_smem_limit(wavelet_kernel<WAV_CONV_RESIDUAL>, max_smem))) return e;
    return raise_smem_limit(wavelet_kernel<WAV_CORR>, max_smem);
}

}  // namespace aahrt

using namespace aahrt;

extern "C" int aahrt_plan_set_wavelet(aahrt_plan *plan, const float *w, int nw, int center) {
    if (!plan) return set_error(AAHRT_ERR_INVALID_ARG, "plan is NULL");
    Plan &p = *plan->p;
    DeviceGuard g(p.device);
    if (nw == 0) {
        p.nw = 0;
        p.wav_gen++;
        return AAHRT_OK;
    }
    if (!w || nw < 0 || nw > 4096 || center < 0 || center >= nw)
        return set_error(AAHRT_ERR_INVALID_ARG, "need a host wavelet of 1..4096 samples and "
                         "0 <= center < nw");
    for (int s = 0; s < nw; ++s)
        if (!std::isfinite(w[s])) return set_error(AAHRT_ERR_NONFINITE, "wavelet sample %d", s);
    int max_smem = 0;
    cudaError_t e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                           p.device);
    if (e) return cuda_fail(e, "device query");
    const size_t smem = (size_t)(((nw + 3) & ~3) + p.nt * 2 * p.pairs) * sizeof(float);
    if ((int)smem > max_smem)
        return set_error(AAHRT_ERR_UNSUPPORTED, "wavelet of %d samples does not fit", nw);
    if ((e = configure_wavelet_kernels(max_smem))) return cuda_fail(e, "kernel attributes");
    if ((e = cudaDeviceSynchronize())) return cuda_fail(e, "synchronise");
    if (p.wav) { cudaFree(p.wav); p.wav = nullptr; }
    if ((e = cudaMalloc((void **)&p.wav, nw * sizeof(float)))) return cuda_fail(e, "alloc wavelet");
    if ((e = cudaMemcpy(p.wav, w, nw * sizeof(float), cudaMemcpyHostToDevice)))
        return cuda_fail(e, "copy wavelet");
    if (!p.wtmp) {
        const long long n = std::max(p.data_len, p.dblk_len);
        if ((e = cudaMalloc((void **)&p.wtmp, n * sizeof(float))))
            return cuda_fail(e, "alloc wavelet workspace");
    }
    p.nw = nw;
    p.wcenter = center;
    p.wav_gen++;
    return AAHRT_OK;
}
