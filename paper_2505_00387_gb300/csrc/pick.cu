// Automatic anisotropic velocity picking (Sec. 3.3, eq. vel_est): the first
// moment of the Radon cube along q at every (tau, theta),
//   q_hat = sum_l q_l |M(tau, l, theta)| / sum_l |M(tau, l, theta)|,
// with the weight sum_l |M| returned beside it (q_hat = 0 where it is 0).
// One thread per (cube, tau, theta) walks the q axis; neighbouring threads
// read neighbouring azimuths (or gathers), so every load is coalesced.
#include <algorithm>

#include "internal.cuh"

namespace aahrt {

// m: ncube blocks of [ntau][nq][inner], inner = ntheta * G (G gathers
// fastest in tensor-core plans, else 1); out: [ncube][ntau][inner]
__global__ void pick_kernel(const float *__restrict__ m, float *__restrict__ qhat,
                            float *__restrict__ wsum, long long nout, int ntau, int nq,
                            int inner, const double *__restrict__ q) {
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < nout;
         o += (long long)gridDim.x * blockDim.x) {
        const long long row = o / inner;          // cube * ntau + tau
        const int c = (int)(o - row * inner);
        const float *col = m + row * (long long)nq * inner + c;
        double num = 0.0, den = 0.0;
        for (int l = 0; l < nq; ++l) {
            const double a = fabs((double)__ldg(col + (long long)l * inner));
            num += __ldg(q + l) * a;
            den += a;
        }
        qhat[o] = den > 0.0 ? (float)(num / den) : 0.f;
        if (wsum) wsum[o] = (float)den;
    }
}

}  // namespace aahrt

using namespace aahrt;

extern "C" int aahrt_pick_velocity(aahrt_plan *plan, const float *m, float *q_hat,
                                   float *weight, void *stream) {
    if (!plan) return set_error(AAHRT_ERR_INVALID_ARG, "plan is NULL");
    Plan &p = *plan->p;
    DeviceGuard g(p.device);
    int rc;
    if ((rc = check_dev_ptr(m, "m")) || (rc = check_dev_ptr(q_hat, "q_hat"))) return rc;
    if (weight && (rc = check_dev_ptr(weight, "weight"))) return rc;
    const int G = p.precision == AAHRT_PRECISION_SPLIT_BF16 ? p.ngather : 1;
    const int blocks = p.precision == AAHRT_PRECISION_SPLIT_BF16 ? 1 : p.ncube;
    const int inner = p.ntheta * G;
    const long long nout = (long long)blocks * p.ntau * inner;
    const int grid = (int)std::min<long long>((nout + 255) / 256, 152 * 16);
    pick_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(m, q_hat, weight, nout, p.ntau, p.nq,
                                                         inner, p.qv);
    p.launches[6]++;
    cudaError_t e = cudaGetLastError();
    return e ? cuda_fail(e, "pick launch") : AAHRT_OK;
}
