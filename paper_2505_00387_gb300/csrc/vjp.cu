// Derivative of the unrolled sparse solve (Sec. 4, eqs. ISTA and soft, with
// FISTA momentum): d_bar = (d m^n / d d)^T m_bar for the map d -> m^n of n
// iterations from m^0 = z^0 = 0 at a fixed step gamma and threshold
// t = gamma*lambda.
//
// Iteration k:  u_k = z_k + gamma L^T (d - L z_k),  m_{k+1} = soft(u_k, t),
//               z_{k+1} = (1 + beta_k) m_{k+1} - beta_k m_k.
// Reverse sweep with the cotangents a_m (of m_{k+1}) and a_z (of z_{k+1}):
//   c      = a_m + (1 + beta_k) a_z
//   u_bar  = c where |u_k| > t, else 0          (slope of the shrinkage)
//   s      = L u_bar;   d_bar += gamma s
//   a_z   <- u_bar - gamma L^T s
//   a_m   <- -beta_k a_z(old)
// The forward iterates are kept every `checkpoint` iterations; each segment
// is recomputed (bit-identically: every kernel of the operator is
// deterministic) to recover its u_k before its reverse sweep.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace aahrt {

static int ew_grid(long long n) {
    const long long b = (n + 255) / 256;
    return (int)std::max<long long>(1, std::min<long long>(b, 152 * 8));
}

// m+ = soft(z + gamma g, t); z+ = m+ + beta (m+ - m); u (optional) = z + gamma g.
// The same arithmetic as the solver's fused update.
__global__ void fista_step_kernel(float *__restrict__ m, float *__restrict__ z,
                                  const float *__restrict__ g, float *__restrict__ u_out,
                                  long long n, float gamma, float thresh, float beta) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float u = fmaf(gamma, g[i], z[i]);
        const float mn = soft_threshold(u, thresh);
        z[i] = fmaf(beta, mn - m[i], mn);
        m[i] = mn;
        if (u_out) u_out[i] = u;
    }
}

// u_bar = (a_m + (1 + beta) a_z) [|u| > t];  a_m <- -beta a_z
__global__ void vjp_mask_kernel(const float *__restrict__ u, float *__restrict__ am,
                                const float *__restrict__ az, float *__restrict__ ubar,
                                long long n, float beta, float thresh) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float a = az[i];
        const float c = fmaf(1.0f + beta, a, am[i]);
        ubar[i] = fabsf(u[i]) > thresh ? c : 0.f;
        am[i] = -beta * a;
    }
}

// y += a x
__global__ void axpy_kernel(float *__restrict__ y, const float *__restrict__ x, float a,
                            long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = fmaf(a, x[i], y[i]);
}

// a_z = u_bar - gamma g
__global__ void vjp_z_kernel(const float *__restrict__ ubar, const float *__restrict__ g,
                             float *__restrict__ az, float gamma, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        az[i] = fmaf(-gamma, g[i], ubar[i]);
}

namespace {

struct VjpBufs {
    float *wm, *wz, *g, *am, *az, *ub, *r;
    std::vector<float *> ckm, ckz, useg;
};

int ensure_vjp_ws(Plan &p, int nseg, int seg, VjpBufs *b) {
    const size_t ml = ((size_t)p.model_len + 63) & ~(size_t)63;   // 256-byte aligned slabs
    const size_t dl = ((size_t)p.data_len + 63) & ~(size_t)63;
    const size_t nmodel = 6 + 2 * (size_t)nseg + (size_t)seg;
    const size_t need = (nmodel * ml + dl) * sizeof(float);
    if (p.vjp_bytes < need) {
        if (p.vjp_ws) {
            cudaFree(p.vjp_ws);
            p.vjp_ws = nullptr;
            p.vjp_bytes = 0;
        }
        cudaError_t e = cudaMalloc((void **)&p.vjp_ws, need);
        if (e) {
            cudaGetLastError();
            return set_error(AAHRT_ERR_OOM, "derivative workspace of %zu bytes: %s", need,
                             cudaGetErrorString(e));
        }
        p.vjp_bytes = need;
    }
    float *q = p.vjp_ws;
    float **fixed[6] = {&b->wm, &b->wz, &b->g, &b->am, &b->az, &b->ub};
    for (float **f : fixed) { *f = q; q += ml; }
    b->ckm.resize(nseg);
    b->ckz.resize(nseg);
    b->useg.resize(seg);
    for (int s = 0; s < nseg; ++s) { b->ckm[s] = q; q += ml; b->ckz[s] = q; q += ml; }
    for (int s = 0; s < seg; ++s) { b->useg[s] = q; q += ml; }
    b->r = q;
    return AAHRT_OK;
}

// One forward iteration on (wm, wz), keeping u when u_out is non-null.
int forward_step(Plan &p, const float *d, VjpBufs &b, float gamma, float thresh, float beta,
                 float *u_out, cudaStream_t st) {
    int rc = apply_forward(p, b.wz, b.r, st, EPI_RESIDUAL, d);
    if (rc) return rc;
    if ((rc = apply_adjoint(p, b.r, b.g, st))) return rc;
    fista_step_kernel<<<ew_grid(p.model_len), 256, 0, st>>>(b.wm, b.wz, b.g, u_out, p.model_len,
                                                          gamma, thresh, beta);
    p.launches[6]++;
    cudaError_t e = cudaGetLastError();
    return e ? cuda_fail(e, "update launch") : AAHRT_OK;
}

int fista_vjp(Plan &p, const float *d, const float *m_bar, float lambda, float gamma, int iters,
              int ista, int checkpoint, float *m_out, float *d_bar, cudaStream_t st) {
    const long long nm = p.model_len, nd = p.data_len;
    const size_t mbytes = nm * sizeof(float);
    cudaError_t e;
    int rc;
    if (iters == 0) {
        if (m_out && (e = cudaMemsetAsync(m_out, 0, mbytes, st))) return cuda_fail(e, "memset");
        if ((e = cudaMemsetAsync(d_bar, 0, nd * sizeof(float), st))) return cuda_fail(e, "memset");
        return AAHRT_OK;
    }
    const int C = std::min(iters, checkpoint > 0 ? checkpoint : 10);
    const int nseg = (iters + C - 1) / C;
    const int last0 = (nseg - 1) * C;
    VjpBufs b;
    if ((rc = ensure_vjp_ws(p, nseg, C, &b))) return rc;

    std::vector<float> beta(iters, 0.f);
    if (!ista) {
        double t = 1.0;
        for (int k = 0; k < iters; ++k) {
            const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
            beta[k] = (float)((t - 1.0) / tn);
            t = tn;
        }
    }
    const float thresh = (float)((double)gamma * (double)lambda);

    // forward sweep: checkpoints at segment starts, u of the last segment kept
    if ((e = cudaMemsetAsync(b.wm, 0, mbytes, st)) || (e = cudaMemsetAsync(b.wz, 0, mbytes, st)))
        return cuda_fail(e, "memset");
    for (int k = 0; k < iters; ++k) {
        if (k % C == 0) {
            const int s = k / C;
            if ((e = cudaMemcpyAsync(b.ckm[s], b.wm, mbytes, cudaMemcpyDeviceToDevice, st)) ||
                (e = cudaMemcpyAsync(b.ckz[s], b.wz, mbytes, cudaMemcpyDeviceToDevice, st)))
                return cuda_fail(e, "checkpoint copy");
        }
        float *u = k >= last0 ? b.useg[k - last0] : nullptr;
        if ((rc = forward_step(p, d, b, gamma, thresh, beta[k], u, st))) return rc;
    }
    if (m_out && (e = cudaMemcpyAsync(m_out, b.wm, mbytes, cudaMemcpyDeviceToDevice, st)))
        return cuda_fail(e, "copy result");

    // reverse sweep
    if ((e = cudaMemcpyAsync(b.am, m_bar, mbytes, cudaMemcpyDeviceToDevice, st)) ||
        (e = cudaMemsetAsync(b.az, 0, mbytes, st)) ||
        (e = cudaMemsetAsync(d_bar, 0, nd * sizeof(float), st)))
        return cuda_fail(e, "init cotangents");
    for (int s = nseg - 1; s >= 0; --s) {
        const int k0 = s * C, k1 = std::min(iters, k0 + C);
        if (s != nseg - 1) {
            if ((e = cudaMemcpyAsync(b.wm, b.ckm[s], mbytes, cudaMemcpyDeviceToDevice, st)) ||
                (e = cudaMemcpyAsync(b.wz, b.ckz[s], mbytes, cudaMemcpyDeviceToDevice, st)))
                return cuda_fail(e, "checkpoint restore");
            for (int k = k0; k < k1; ++k)
                if ((rc = forward_step(p, d, b, gamma, thresh, beta[k], b.useg[k - k0], st)))
                    return rc;
        }
        for (int k = k1 - 1; k >= k0; --k) {
            vjp_mask_kernel<<<ew_grid(nm), 256, 0, st>>>(b.useg[k - k0], b.am, b.az, b.ub, nm,
                                                        beta[k], thresh);
            p.launches[6]++;
            if ((e = cudaGetLastError())) return cuda_fail(e, "mask launch");
            if ((rc = apply_forward(p, b.ub, b.r, st))) return rc;
            axpy_kernel<<<ew_grid(nd), 256, 0, st>>>(d_bar, b.r, gamma, nd);
            p.launches[6]++;
            if ((rc = apply_adjoint(p, b.r, b.g, st))) return rc;
            vjp_z_kernel<<<ew_grid(nm), 256, 0, st>>>(b.ub, b.g, b.az, gamma, nm);
            p.launches[6]++;
            if ((e = cudaGetLastError())) return cuda_fail(e, "cotangent launch");
        }
    }
    return AAHRT_OK;
}

}  // namespace
}  // namespace aahrt

using namespace aahrt;

extern "C" int aahrt_fista_vjp(aahrt_plan *plan, const float *d, const float *m_bar,
                               float lambda, float gamma, int iters, int ista, int checkpoint,
                               float *m_out, float *d_bar, void *stream) {
    if (!plan) return set_error(AAHRT_ERR_INVALID_ARG, "plan is NULL");
    Plan &p = *plan->p;
    DeviceGuard g(p.device);
    int rc;
    if ((rc = check_dev_ptr(d, "d")) || (rc = check_dev_ptr(m_bar, "m_bar")) ||
        (rc = check_dev_ptr(d_bar, "d_bar")))
        return rc;
    if (m_out && (rc = check_dev_ptr(m_out, "m_out"))) return rc;
    if (iters < 0) return set_error(AAHRT_ERR_INVALID_ARG, "iters must be >= 0");
    if (!(gamma > 0.f) || !std::isfinite(gamma))
        return set_error(AAHRT_ERR_INVALID_ARG, "gamma must be finite and > 0");
    if (!(lambda >= 0.f) || !std::isfinite(lambda))
        return set_error(AAHRT_ERR_INVALID_ARG, "lambda must be finite and >= 0");
    return fista_vjp(p, d, m_bar, lambda, gamma, iters, ista, checkpoint, m_out, d_bar,
                     (cudaStream_t)stream);
}
