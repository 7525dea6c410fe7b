// Curvature-range tools of Sec. 3.5 (eqs. q1-q3): the uniform-slowness
// curvature axis, the sample-count bound of eq. q3, and the partial NMO of
// the data by a reference curvature.
//
// Partial NMO.  In stretched time s = t^2 a hyperbola t^2 = tau^2 + q r^2 is
// the line s = tau^2 + q r^2; shifting the stretched trace by -q_ref r^2
// moves it to curvature q - q_ref.  On the time axis that is one resampling:
//   out(t_i, h) = sum_taps c(u - n) in(t_n, h),  u^2 = i^2 + q_ref r_h^2/dt^2,
// zero where u^2 < 0.  u is evaluated in float-float arithmetic: i^2 and
// c_h = q_ref r_h^2/dt^2 are exact (hi, lo) pairs, the sum is a two-sum, and
// one Newton step on the FP32 root recovers the fraction of a sample to about
// 1e-7 (a plain FP32 u of 1000 samples would lose 6e-5 of a sample).  The
// transpose gathers, for every input sample n, the outputs i whose taps reach
// n (recomputing their positions and weights bit-identically), so it needs no
// atomics and is deterministic.
#include <algorithm>
#include <cmath>

#include "internal.cuh"
#include "resample.cuh"

namespace aahrt {

struct PnArgs {
    const PnBlock *__restrict__ blk;
    const float2 *__restrict__ c;     // per trace (hi, lo) of q_ref r^2 / dt^2
    int nt;
};

__global__ void pn_coef_kernel(const double *__restrict__ rho, float2 *__restrict__ c,
                               long long n, double q_ref) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double v = q_ref * rho[i];
        const float hi = (float)v;
        c[i] = make_float2(hi, (float)(v - (double)hi));
    }
}

// Position u = sqrt(i^2 + c) of output row i as base + frac, frac in [0, 1);
// false where i^2 + c < 0 (the output is muted).
__device__ __forceinline__ bool pn_position(int i, float2 c, int *base, float *frac) {
    const int ii = i * i;
    const float a_hi = __int2float_rn(ii);
    const float a_lo = __int2float_rn(ii - __float2int_rn(a_hi));
    const float s = __fadd_rn(a_hi, c.x);                 // two-sum of a_hi + c.x
    const float bb = __fsub_rn(s, a_hi);
    const float err = __fadd_rn(__fsub_rn(a_hi, __fsub_rn(s, bb)), __fsub_rn(c.x, bb));
    const float t = __fadd_rn(__fadd_rn(err, a_lo), c.y);
    if (__fadd_rn(s, t) < 0.f) return false;
    const float u0 = sqrtf(fmaxf(s, 0.f));
    float corr = 0.f;
    if (u0 > 0.f) corr = __fadd_rn(__fmaf_rn(-u0, u0, s), t) / __fmul_rn(2.f, u0);
    const float fb = floorf(u0);
    float fr = __fadd_rn(__fsub_rn(u0, fb), corr);
    int b = (int)fb;
    if (fr < 0.f) {
        fr = __fadd_rn(fr, 1.f);
        --b;
    } else if (fr >= 1.f) {
        fr = __fsub_rn(fr, 1.f);
        ++b;
    }
    if (fr >= 1.f) fr = 0.99999994f;
    *base = b;
    *frac = fr;
    return true;
}

template <int INTERP>
__global__ void pnmo_kernel(const PnArgs a, const float *__restrict__ in, float *__restrict__ out) {
    const PnBlock b = a.blk[blockIdx.y];
    const long long n = (long long)a.nt * b.ld;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / b.ld);
        const int col = (int)(idx - (long long)i * b.ld);
        const float2 c = __ldg(a.c + b.r0 + col / b.rep);
        int base;
        float fr;
        float v = 0.f;
        if (pn_position(i, c, &base, &fr)) {
#pragma unroll
            for (int q = 0; q < Taps<INTERP>::n; ++q) {
                const int t = Taps<INTERP>::t0 + q;
                const int r = base + t;
                if (r >= 0 && r < a.nt)
                    v = fmaf(tap_weight<INTERP>(t, fr),
                             __ldg(in + b.off + (long long)r * b.ld + col), v);
            }
        }
        out[b.off + idx] = v;
    }
}

// largest i >= 0 with i^2 <= x (x may be negative: -1), by a float root and
// integer corrections
__device__ __forceinline__ int isqrt_floor(float x) {
    if (x < 0.f) return -1;
    int r = (int)sqrtf(x);
    while ((float)r * r > x) --r;
    while ((float)(r + 1) * (r + 1) <= x) ++r;
    return r;
}

template <int INTERP>
__global__ void pnmo_t_kernel(const PnArgs a, const float *__restrict__ in,
                              float *__restrict__ out) {
    constexpr int T0 = Taps<INTERP>::t0, TN = Taps<INTERP>::n;
    const PnBlock b = a.blk[blockIdx.y];
    const long long n = (long long)a.nt * b.ld;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(idx / b.ld);                 // input sample receiving
        const int col = (int)(idx - (long long)r * b.ld);
        const float2 c = __ldg(a.c + b.r0 + col / b.rep);
        const float cc = c.x + c.y;
        // outputs i read sample r when base_i + t = r for a tap t, i.e.
        // u_i in [r - T0 - TN + 1, r - T0 + 1); one sample of margin each side
        const float ulo = fmaxf((float)(r - T0 - TN), 0.f);
        const float uhi = (float)(r - T0 + 2);
        int ilo = isqrt_floor(ulo * ulo - cc) - 1;
        int ihi = isqrt_floor(uhi * uhi - cc) + 1;
        if (ilo < 0) ilo = 0;
        if (ihi > a.nt - 1) ihi = a.nt - 1;
        float v = 0.f;
        for (int i = ilo; i <= ihi; ++i) {
            int base;
            float fr;
            if (!pn_position(i, c, &base, &fr)) continue;
            const int t = r - base;
            if (t < T0 || t >= T0 + TN) continue;
            v = fmaf(tap_weight<INTERP>(t, fr), __ldg(in + b.off + (long long)i * b.ld + col), v);
        }
        out[b.off + idx] = v;
    }
}

}  // namespace aahrt

using namespace aahrt;

extern "C" int aahrt_q_axis_slowness(double pmin, double pmax, int nq, double *q) {
    if (!q) return set_error(AAHRT_ERR_INVALID_ARG, "q is NULL");
    if (nq < 1) return set_error(AAHRT_ERR_INVALID_ARG, "nq must be >= 1");
    if (!std::isfinite(pmin) || !std::isfinite(pmax))
        return set_error(AAHRT_ERR_NONFINITE, "pmin and pmax must be finite");
    const double step = nq > 1 ? (pmax - pmin) / (nq - 1) : 0.0;
    for (int l = 0; l < nq; ++l) {
        const double p = (nq > 1 && l == nq - 1) ? pmax : pmin + l * step;
        q[l] = p * p;
    }
    return AAHRT_OK;
}

extern "C" int aahrt_nq_required(double span, double fmax, double r2max, int *nq) {
    if (!nq) return set_error(AAHRT_ERR_INVALID_ARG, "nq is NULL");
    if (!std::isfinite(span) || !std::isfinite(fmax) || !std::isfinite(r2max))
        return set_error(AAHRT_ERR_NONFINITE, "span, fmax and r2max must be finite");
    if (span < 0.0 || fmax < 0.0 || r2max < 0.0)
        return set_error(AAHRT_ERR_INVALID_ARG, "span, fmax and r2max must be >= 0");
    const double n = std::ceil(span * fmax * r2max - 1e-12);
    if (!(n < 2147483647.0)) return set_error(AAHRT_ERR_INVALID_ARG, "sample count overflows");
    *nq = n < 1.0 ? 1 : (int)n;
    return AAHRT_OK;
}

extern "C" int aahrt_partial_nmo(aahrt_plan *plan, const float *in, float *out, double q_ref,
                                 int transpose, void *stream) {
    if (!plan) return set_error(AAHRT_ERR_INVALID_ARG, "plan is NULL");
    Plan &p = *plan->p;
    DeviceGuard g(p.device);
    int rc;
    if ((rc = check_dev_ptr(in, "in")) || (rc = check_dev_ptr(out, "out"))) return rc;
    if (transpose != 0 && transpose != 1)
        return set_error(AAHRT_ERR_INVALID_ARG, "transpose must be 0 or 1");
    if (!std::isfinite(q_ref)) return set_error(AAHRT_ERR_NONFINITE, "q_ref must be finite");
    const char *a0 = reinterpret_cast<const char *>(in), *b0 = reinterpret_cast<const char *>(out);
    const long long bytes = p.data_len * (long long)sizeof(float);
    if (a0 < b0 + bytes && b0 < a0 + bytes)
        return set_error(AAHRT_ERR_INVALID_ARG, "in and out overlap");
    if (p.nt >= 46341)
        return set_error(AAHRT_ERR_UNSUPPORTED, "nt too large for the partial NMO");
    cudaStream_t st = (cudaStream_t)stream;
    const int cgrid = (int)std::min<long long>((p.pn_ntr + 255) / 256, 1024);
    pn_coef_kernel<<<std::max(1, cgrid), 256, 0, st>>>(p.pn_rho, p.pn_c, p.pn_ntr, q_ref);
    cudaError_t e = cudaGetLastError();
    if (e) return cuda_fail(e, "partial NMO launch");
    PnArgs a{p.pn_blk, p.pn_c, p.nt};
    const long long per = (long long)p.nt * p.pn_ldmax;
    const dim3 grid((unsigned)std::max<long long>(1, std::min<long long>((per + 255) / 256, 2048)),
                    (unsigned)p.pn_nblk);
    const bool keys = p.interp == AAHRT_INTERP_KEYS;
    if (transpose) {
        if (keys) pnmo_t_kernel<AAHRT_INTERP_KEYS><<<grid, 256, 0, st>>>(a, in, out);
        else pnmo_t_kernel<AAHRT_INTERP_LINEAR><<<grid, 256, 0, st>>>(a, in, out);
    } else {
        if (keys) pnmo_kernel<AAHRT_INTERP_KEYS><<<grid, 256, 0, st>>>(a, in, out);
        else pnmo_kernel<AAHRT_INTERP_LINEAR><<<grid, 256, 0, st>>>(a, in, out);
    }
    p.launches[6] += 2;
    e = cudaGetLastError();
    return e ? cuda_fail(e, "partial NMO launch") : AAHRT_OK;
}
