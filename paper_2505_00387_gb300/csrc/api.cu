// C entry points of libaahrt (declared in include/aahrt.h) and the sparse
// solver of Sec. 4 (eqs. cost1, ISTA, soft) with FISTA momentum.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

namespace aahrt {

int build_plan(Plan **out, int ncube, int ndist, const aahrt_geom *geoms,
               const aahrt_opts *opts);
int autotune_plan(Plan **out, int ncube, int ndist, const aahrt_geom *geoms,
                  const aahrt_opts *opts);

static int make_plan(Plan **out, int ncube, int ndist, const aahrt_geom *geoms,
                     const aahrt_opts *opts) {
    if (opts && opts->autotune) return autotune_plan(out, ncube, ndist, geoms, opts);
    return build_plan(out, ncube, ndist, geoms, opts);
}
void free_plan(Plan *p);
void plan_info(const Plan &p, aahrt_plan_info *info);
int collect_profile(Plan &p);
const char *last_error_text();

// ---------------------------------------------------------- reductions
// Device scalars (Plan::scal, doubles): see the slot names below.
enum { SC_SUMSQ = 0, SC_L1 = 1, SC_DOT = 2, SC_ABSMAX = 3, SC_NORM2 = 4, SC_COUNT = 8 };

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// acc += sum f(x_i, y_i) in FP64: kind 0 = x^2, 1 = |x|, 2 = x*y
__global__ void reduce_kernel(const float *__restrict__ x, const float *__restrict__ y,
                              long long n, int kind, double *acc) {
    __shared__ double part[32];
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double a = x[i];
        s += kind == 0 ? a * a : (kind == 1 ? fabs(a) : a * (double)y[i]);
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
        s = warp_sum(s);
        if (threadIdx.x == 0) atomicAdd(acc, s);
    }
}

// max |x| as the bit pattern of a non-negative float (orders like an unsigned int)
__global__ void absmax_kernel(const float *__restrict__ x, long long n, unsigned *acc) {
    float mx = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        mx = fmaxf(mx, fabsf(x[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(acc, __float_as_uint(mx));
}

// y = x / sqrt(*ss)
__global__ void normalize_kernel(const float *__restrict__ x, float *__restrict__ y,
                                 long long n, const double *ss) {
    const float s = (float)(1.0 / sqrt(*ss));
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = x[i] * s;
}

// Per-cube (segmented) versions.  Cube c = blockIdx.y owns elements
// [c*seg, (c+1)*seg) when seg > 0, else [off[c], off[c+1]).
// kind 0: acc[c] += sum x^2; 1: += sum |x|; 2: += sum x*y; 3: max |x| (float bits)
__global__ void seg_reduce_kernel(const float *__restrict__ x, const float *__restrict__ y,
                                  long long seg, const long long *__restrict__ off, int kind,
                                  double *acc) {
    __shared__ double part[32];
    const int c = blockIdx.y;
    const long long b = seg > 0 ? c * seg : off[c];
    const long long e = seg > 0 ? b + seg : off[c + 1];
    double s = 0.0;
    float mx = 0.f;
    for (long long i = b + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < e;
         i += (long long)gridDim.x * blockDim.x) {
        const float a = x[i];
        if (kind == 3) mx = fmaxf(mx, fabsf(a));
        else s += kind == 0 ? (double)a * a : (kind == 1 ? fabs((double)a) : (double)a * y[i]);
    }
    if (kind == 3) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0)
            atomicMax(reinterpret_cast<unsigned *>(acc + c), __float_as_uint(mx));
        return;
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
        s = warp_sum(s);
        if (threadIdx.x == 0) atomicAdd(acc + c, s);
    }
}

// y = x / sqrt(ss[c]) on cube c's model block; a cube with ss = 0 gets the
// constant unit vector (a valid start of its power iteration).
__global__ void seg_normalize_kernel(const float *__restrict__ x, float *__restrict__ y,
                                     long long seg, const double *__restrict__ ss) {
    const int c = blockIdx.y;
    const double v = ss[c];
    const bool zero = !(v > 0.0);
    const float sc = zero ? 0.f : (float)(1.0 / sqrt(v));
    const float cst = (float)(1.0 / sqrt((double)seg));
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < seg;
         i += (long long)gridDim.x * blockDim.x) {
        const long long j = c * seg + i;
        y[j] = zero ? cst : x[j] * sc;
    }
}

static int reduce_grid(long long n) {
    long long b = (n + 255) / 256;
    return (int)std::max<long long>(1, std::min<long long>(b, 152 * 8));
}

static cudaError_t reduce(Plan &p, const float *x, const float *y, long long n, int kind,
                          int slot, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(p.scal + slot, 0, sizeof(double), st);
    if (e) return e;
    prof_begin(p, 6, st);
    reduce_kernel<<<reduce_grid(n), 256, 0, st>>>(x, y, n, kind, p.scal + slot);
    prof_end(p, st);
    p.launches[6]++;
    return cudaGetLastError();
}

// ------------------------------------------------------------ operators
// With a wavelet set (deconvolutive operator W L), the synthesis writes L m
// to the workspace and the time convolution produces d = W L m (or the
// residual dobs - W L m); the adjoint correlates first (W^T d).
int apply_forward(Plan &p, const float *m, float *d, cudaStream_t st, int epi,
                  const float *dobs, bool blocked) {
    cudaError_t e;
    if ((e = launch_r2c(p, true, m, p.X, st, blocked))) return cuda_fail(e, "stretch+FFT launch");
    if ((e = launch_slice(p, false, p.X, p.Y, st))) return cuda_fail(e, "slice launch");
    if (p.nw > 0) {
        if ((e = launch_c2r(p, false, p.Y, p.wtmp, EPI_STORE, nullptr, FistaArgs{}, st, blocked)))
            return cuda_fail(e, "inverse FFT+unstretch launch");
        prof_begin(p, 2, st);
        e = launch_wavelet(p, epi == EPI_RESIDUAL ? 1 : 0, p.wtmp, d, dobs, st, blocked);
        prof_end(p, st);
        p.launches[2]++;
        return e ? cuda_fail(e, "wavelet convolution launch") : AAHRT_OK;
    }
    if ((e = launch_c2r(p, false, p.Y, d, epi, dobs, FistaArgs{}, st, blocked)))
        return cuda_fail(e, "inverse FFT+unstretch launch");
    return AAHRT_OK;
}

int apply_adjoint(Plan &p, const float *d, float *m, cudaStream_t st, int epi, FistaArgs fa,
                  bool blocked) {
    cudaError_t e;
    if (p.nw > 0) {
        prof_begin(p, 3, st);
        e = launch_wavelet(p, 2, d, p.wtmp, nullptr, st, blocked);
        prof_end(p, st);
        p.launches[3]++;
        if (e) return cuda_fail(e, "wavelet correlation launch");
        d = p.wtmp;
    }
    if ((e = launch_r2c(p, false, d, p.Y, st, blocked)))
        return cuda_fail(e, "unstretch^T+FFT launch");
    if ((e = launch_slice(p, true, p.Y, p.X, st))) return cuda_fail(e, "slice adjoint launch");
    if ((e = launch_c2r(p, true, p.X, m, epi, nullptr, fa, st, blocked)))
        return cuda_fail(e, "inverse FFT+stretch^T launch");
    return AAHRT_OK;
}

// Copy between the row-major layout of the C ABI and the column-blocked
// layout [group][row][2*pairs] of the solver's internal arrays.
__global__ void reblock_kernel(const float *__restrict__ src, float *__restrict__ dst,
                               const ColGroup *__restrict__ nat,
                               const ColGroup *__restrict__ blk, int nrows, int lcpg,
                               int to_blocked) {
    const ColGroup a = nat[blockIdx.x], b = blk[blockIdx.x];
    const int cpg = 1 << lcpg;
    for (int idx = threadIdx.x; idx < nrows * cpg; idx += blockDim.x) {
        const int r = idx >> lcpg, c = idx & (cpg - 1);
        if (c >= a.ncol) continue;
        const long long io = a.real_off + (long long)r * a.ld_real + c;
        const long long ib = b.real_off + (long long)r * cpg + c;
        if (to_blocked) dst[ib] = src[io];
        else dst[io] = src[ib];
    }
}

static cudaError_t reblock(Plan &p, bool model_side, const float *src, float *dst,
                           bool to_blocked, cudaStream_t st) {
    const int n = model_side ? p.ncg_model : p.ncg_data;
    reblock_kernel<<<n, 256, 0, st>>>(src, dst, model_side ? p.cg_model : p.cg_data,
                                      model_side ? p.cg_model_blk : p.cg_data_blk,
                                      model_side ? p.ntau : p.nt, p.lp + 1,
                                      to_blocked ? 1 : 0);
    p.launches[6]++;
    return cudaGetLastError();
}

int check_dev_ptr(const void *ptr, const char *name) {
    if (!ptr) return set_error(AAHRT_ERR_INVALID_ARG, "%s is NULL", name);
    if (reinterpret_cast<uintptr_t>(ptr) & 15)
        return set_error(AAHRT_ERR_INVALID_ARG, "%s is not 16-byte aligned", name);
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, ptr);
    if (e) {
        cudaGetLastError();
        return set_error(AAHRT_ERR_INVALID_ARG, "%s: not a CUDA pointer", name);
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return set_error(AAHRT_ERR_INVALID_ARG, "%s is not device memory", name);
    return AAHRT_OK;
}

// Host or device?  Device pointers must be 16-byte aligned; host pointers
// (pinned or pageable) are staged through plan-owned device buffers.
static int classify_ptr(const void *ptr, const char *name, bool *is_host) {
    if (!ptr) return set_error(AAHRT_ERR_INVALID_ARG, "%s is NULL", name);
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, ptr);
    if (e) {
        cudaGetLastError();
        return set_error(AAHRT_ERR_INVALID_ARG, "%s: pointer query failed", name);
    }
    *is_host = !(at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
    if (!*is_host && (reinterpret_cast<uintptr_t>(ptr) & 15))
        return set_error(AAHRT_ERR_INVALID_ARG, "%s is not 16-byte aligned", name);
    if (*is_host && (reinterpret_cast<uintptr_t>(ptr) & 3))
        return set_error(AAHRT_ERR_INVALID_ARG, "%s is not 4-byte aligned", name);
    return AAHRT_OK;
}

static int ensure_staging(Plan &p) {
    cudaError_t e;
    if (!p.stage_m && (e = cudaMalloc((void **)&p.stage_m, p.model_len * sizeof(float))))
        return cuda_fail(e, "alloc staging buffer");
    if (!p.stage_d && (e = cudaMalloc((void **)&p.stage_d, p.data_len * sizeof(float))))
        return cuda_fail(e, "alloc staging buffer");
    return AAHRT_OK;
}

// Resolve (model, data) arguments: host inputs are copied in, host outputs
// get a device buffer that `finish` copies back.
struct Staged {
    const float *in_dev = nullptr;
    float *out_dev = nullptr;
    float *out_host = nullptr;
    long long out_len = 0;
};

static int stage_args(Plan &p, const float *in, long long in_len, bool in_is_model,
                      float *out, long long out_len, cudaStream_t st, Staged *s) {
    bool hin = false, hout = false;
    int rc;
    if ((rc = classify_ptr(in, "input", &hin)) || (rc = classify_ptr(out, "output", &hout)))
        return rc;
    if ((hin || hout) && (rc = ensure_staging(p))) return rc;
    s->in_dev = in;
    s->out_dev = out;
    if (hin) {
        float *buf = in_is_model ? p.stage_m : p.stage_d;
        cudaError_t e = cudaMemcpyAsync(buf, in, in_len * sizeof(float), cudaMemcpyHostToDevice, st);
        if (e) return cuda_fail(e, "copy input to device");
        s->in_dev = buf;
    }
    if (hout) {
        s->out_dev = in_is_model ? p.stage_d : p.stage_m;
        s->out_host = out;
        s->out_len = out_len;
    }
    return AAHRT_OK;
}

static int finish_args(const Staged &s, cudaStream_t st) {
    if (!s.out_host) return AAHRT_OK;
    cudaError_t e = cudaMemcpyAsync(s.out_host, s.out_dev, s.out_len * sizeof(float),
                                    cudaMemcpyDeviceToHost, st);
    return e ? cuda_fail(e, "copy output to host") : AAHRT_OK;
}

static int ensure_solver_ws(Plan &p) {
    cudaError_t e;
    if (!p.z && (e = cudaMalloc((void **)&p.z, p.model_len * sizeof(float))))
        return cuda_fail(e, "alloc solver workspace");
    if (!p.v && (e = cudaMalloc((void **)&p.v, p.model_len * sizeof(float))))
        return cuda_fail(e, "alloc solver workspace");
    if (!p.r && (e = cudaMalloc((void **)&p.r, p.data_len * sizeof(float))))
        return cuda_fail(e, "alloc solver workspace");
    if (!p.scal && (e = cudaMalloc((void **)&p.scal, SC_COUNT * sizeof(double))))
        return cuda_fail(e, "alloc solver workspace");
    float **mbufs[2] = {&p.zb, &p.mb};
    for (float **b : mbufs)
        if (!*b && (e = cudaMalloc((void **)b, p.mblk_len * sizeof(float))))
            return cuda_fail(e, "alloc solver workspace");
    float **dbufs[2] = {&p.rb, &p.db};
    for (float **b : dbufs)
        if (!*b && (e = cudaMalloc((void **)b, p.dblk_len * sizeof(float))))
            return cuda_fail(e, "alloc solver workspace");
    return AAHRT_OK;
}

static int read_scalars(Plan &p, double *h, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(h, p.scal, SC_COUNT * sizeof(double),
                                    cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    return e ? cuda_fail(e, "read solver scalars") : AAHRT_OK;
}

// The iterations proper, on the column-blocked state (mb, zb) and data (db):
// per iteration one forward with the residual fused (rb = db - L zb) and one
// adjoint with the shrinkage/momentum update fused.
static int run_iterations(Plan &p, int iters, float gamma, float thresh,
                          const std::vector<double> &betas, const float2 *cube_gt,
                          cudaStream_t st) {
    cudaError_t e;
    if (p.nw == 0 && p.smem_fused_model > 0 && p.smem_fused_data > 0 && iters > 0) {
        // Fused half-iterations: the stretch+FFT of z runs once up front, then
        // per iteration slice -> (synthesis + residual + U^T FFT) -> slice^T
        // -> (synthesis + update + stretch+FFT of the new z).  The same
        // arithmetic as the unfused sequence, without the residual and z
        // round trips; the last update skips the unused next stretch.
        if ((e = launch_r2c(p, true, p.zb, p.X, st, true)))
            return cuda_fail(e, "stretch+FFT launch");
        for (int it = 0; it < iters; ++it) {
            if ((e = launch_slice(p, false, p.X, p.Y, st))) return cuda_fail(e, "slice launch");
            if ((e = launch_c2r_r2c(p, false, p.Y, p.db, FistaArgs{}, st)))
                return cuda_fail(e, "fused data-side launch");
            if ((e = launch_slice(p, true, p.Y, p.X, st)))
                return cuda_fail(e, "slice adjoint launch");
            FistaArgs fa{p.mb, p.zb, gamma, thresh, (float)betas[it], cube_gt};
            if (it + 1 < iters) {
                if ((e = launch_c2r_r2c(p, true, p.X, nullptr, fa, st)))
                    return cuda_fail(e, "fused model-side launch");
            } else if ((e = launch_c2r(p, true, p.X, nullptr, EPI_FISTA, nullptr, fa, st, true))) {
                return cuda_fail(e, "inverse FFT+stretch^T launch");
            }
        }
        return AAHRT_OK;
    }
    for (int it = 0; it < iters; ++it) {
        int rc = apply_forward(p, p.zb, p.rb, st, EPI_RESIDUAL, p.db, true);
        if (rc) return rc;
        FistaArgs fa{p.mb, p.zb, gamma, thresh, (float)betas[it], cube_gt};
        rc = apply_adjoint(p, p.rb, nullptr, st, EPI_FISTA, fa, true);
        if (rc) return rc;
    }
    return AAHRT_OK;
}

enum { CA_SS = 0, CA_DOT = 1, CA_MAX = 2, CA_L1 = 3, CA_SLOTS = 4 };

static int ensure_cube_ws(Plan &p) {
    cudaError_t e;
    if (!p.cube_gt && (e = cudaMalloc((void **)&p.cube_gt, p.ncube * sizeof(float2))))
        return cuda_fail(e, "alloc per-cube scalars");
    if (!p.cube_acc &&
        (e = cudaMalloc((void **)&p.cube_acc, CA_SLOTS * p.ncube * sizeof(double))))
        return cuda_fail(e, "alloc per-cube scalars");
    if (!p.dseg) {
        std::vector<long long> off(p.ncube + 1);
        for (int c = 0; c < p.ncube; ++c) off[c] = p.data_off[c];
        off[p.ncube] = p.data_len;
        if ((e = cudaMalloc((void **)&p.dseg, off.size() * sizeof(long long))))
            return cuda_fail(e, "alloc per-cube scalars");
        if ((e = cudaMemcpy(p.dseg, off.data(), off.size() * sizeof(long long),
                            cudaMemcpyHostToDevice)))
            return cuda_fail(e, "upload cube offsets");
    }
    return AAHRT_OK;
}

// acc[slot][c] (re)computed over every cube's model (model = true) or data block
static cudaError_t seg_reduce(Plan &p, const float *x, const float *y, bool model, int kind,
                              int slot, cudaStream_t st) {
    double *acc = p.cube_acc + (size_t)slot * p.ncube;
    cudaError_t e = cudaMemsetAsync(acc, 0, p.ncube * sizeof(double), st);
    if (e) return e;
    const long long seg = model ? p.model_len / p.ncube : 0;
    const long long per = model ? seg : (p.data_len + p.ncube - 1) / p.ncube;
    const int gx = (int)std::max<long long>(1, std::min<long long>((per + 2047) / 2048, 64));
    seg_reduce_kernel<<<dim3(gx, p.ncube), 256, 0, st>>>(x, y, seg, p.dseg, kind, acc);
    p.launches[6]++;
    return cudaGetLastError();
}

static int read_cube_acc(Plan &p, std::vector<double> *h, cudaStream_t st) {
    h->resize((size_t)CA_SLOTS * p.ncube);
    cudaError_t e = cudaMemcpyAsync(h->data(), p.cube_acc, h->size() * sizeof(double),
                                    cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    return e ? cuda_fail(e, "read per-cube scalars") : AAHRT_OK;
}

static float acc_bits_to_float(double v) {
    unsigned bits;
    std::memcpy(&bits, &v, sizeof bits);
    float f;
    std::memcpy(&f, &bits, sizeof f);
    return f;
}

// Per-cube step and threshold: lambda_c = lambda_rel max|L^T d_c| (or the
// given value), gamma_c = 0.95 / (power estimate of ||L_c||^2) unless given.
static int cube_params(Plan &p, const float *d, float lambda, const aahrt_solve_opts &o,
                       std::vector<double> *gam, std::vector<double> *lam, cudaStream_t st) {
    const int nc = p.ncube;
    gam->assign(nc, 0.0);
    lam->assign(nc, (double)lambda);
    bool need_gamma = false;
    for (int c = 0; c < nc; ++c) {
        if (o.gamma > 0.0) (*gam)[c] = o.gamma;
        else if (o.cube_gamma && o.cube_gamma[c] > 0.0) (*gam)[c] = o.cube_gamma[c];
        else need_gamma = true;
        if (o.cube_lambda && !(o.lambda_rel > 0.0)) (*lam)[c] = o.cube_lambda[c];
    }
    if (!need_gamma && !(o.lambda_rel > 0.0)) return AAHRT_OK;
    int rc;
    cudaError_t e;
    std::vector<double> h;
    const long long seg = p.model_len / nc;
    const int gx = (int)std::max<long long>(1, std::min<long long>((seg + 2047) / 2048, 64));
    if ((rc = apply_adjoint(p, d, p.v, st))) return rc;
    if (o.lambda_rel > 0.0) {
        if ((e = seg_reduce(p, p.v, nullptr, true, 3, CA_MAX, st)))
            return cuda_fail(e, "absmax launch");
        if ((rc = read_cube_acc(p, &h, st))) return rc;
        for (int c = 0; c < nc; ++c)
            (*lam)[c] = o.lambda_rel * (double)acc_bits_to_float(h[(size_t)CA_MAX * nc + c]);
    }
    if (!need_gamma) return AAHRT_OK;
    const int piters = o.power_iters > 0 ? o.power_iters : 30;
    if ((e = seg_reduce(p, p.v, nullptr, true, 0, CA_SS, st))) return cuda_fail(e, "norm launch");
    seg_normalize_kernel<<<dim3(gx, nc), 256, 0, st>>>(p.v, p.v, seg, p.cube_acc + CA_SS * nc);
    p.launches[6]++;
    for (int it = 0; it < piters; ++it) {
        if ((rc = apply_forward(p, p.v, p.r, st))) return rc;
        if ((rc = apply_adjoint(p, p.r, p.z, st))) return rc;
        if ((e = seg_reduce(p, p.v, p.z, true, 2, CA_DOT, st)) ||
            (e = seg_reduce(p, p.z, nullptr, true, 0, CA_SS, st)))
            return cuda_fail(e, "power iteration launch");
        seg_normalize_kernel<<<dim3(gx, nc), 256, 0, st>>>(p.z, p.v, seg,
                                                          p.cube_acc + CA_SS * nc);
        p.launches[6]++;
    }
    if ((e = cudaGetLastError())) return cuda_fail(e, "power iteration");
    if ((rc = read_cube_acc(p, &h, st))) return rc;
    for (int c = 0; c < nc; ++c) {
        if ((*gam)[c] > 0.0) continue;
        const double s2 = h[(size_t)CA_DOT * nc + c];
        if (!(s2 > 0.0) || !std::isfinite(s2))
            return set_error(AAHRT_ERR_NONFINITE, "power iteration of cube %d gave %g", c, s2);
        (*gam)[c] = 0.95 / s2;
    }
    return AAHRT_OK;
}

static int solve(Plan &p, const float *d, float lambda, int iters, float *m,
                 const aahrt_solve_opts &o, aahrt_solve_info *info, cudaStream_t st) {
    int rc = ensure_solver_ws(p);
    if (rc) return rc;
    cudaError_t e;
    double gamma = o.gamma;
    double lam = lambda;
    double h[SC_COUNT];
    const bool per_cube = o.per_cube != 0;
    std::vector<double> cgam, clam;
    if (per_cube) {
        if ((rc = ensure_cube_ws(p))) return rc;
        if ((rc = cube_params(p, d, lambda, o, &cgam, &clam, st))) return rc;
        std::vector<float2> gt(p.ncube);
        for (int c = 0; c < p.ncube; ++c) {
            if (!(cgam[c] > 0.0) || !std::isfinite(cgam[c]) || !(clam[c] >= 0.0) ||
                !std::isfinite(clam[c]))
                return set_error(AAHRT_ERR_INVALID_ARG, "cube %d: gamma (%g) and lambda (%g) "
                                 "must be finite, gamma > 0, lambda >= 0", c, cgam[c], clam[c]);
            gt[c] = make_float2((float)cgam[c], (float)(cgam[c] * clam[c]));
        }
        if ((e = cudaMemcpyAsync(p.cube_gt, gt.data(), gt.size() * sizeof(float2),
                                 cudaMemcpyHostToDevice, st)) ||
            (e = cudaStreamSynchronize(st)))
            return cuda_fail(e, "upload per-cube scalars");
        for (int c = 0; c < p.ncube; ++c) {
            if (o.cube_gamma) o.cube_gamma[c] = cgam[c];
            if (o.cube_lambda) o.cube_lambda[c] = clam[c];
        }
        gamma = cgam[0];
        lam = clam[0];
    } else if (gamma <= 0.0 || o.lambda_rel > 0.0) {
        // L^T d, for lambda_rel * max|L^T d| and as the power iteration's start
        if ((rc = apply_adjoint(p, d, p.v, st))) return rc;
        if (o.lambda_rel > 0.0) {
            if ((e = cudaMemsetAsync(p.scal + SC_ABSMAX, 0, sizeof(double), st)))
                return cuda_fail(e, "memset");
            absmax_kernel<<<reduce_grid(p.model_len), 256, 0, st>>>(
                p.v, p.model_len, reinterpret_cast<unsigned *>(p.scal + SC_ABSMAX));
            p.launches[6]++;
            if ((e = cudaGetLastError())) return cuda_fail(e, "absmax launch");
            if ((rc = read_scalars(p, h, st))) return rc;
            unsigned bits;
            std::memcpy(&bits, &h[SC_ABSMAX], sizeof bits);
            float mx;
            std::memcpy(&mx, &bits, sizeof mx);
            lam = o.lambda_rel * (double)mx;
        }
        if (gamma <= 0.0) {
            const int piters = o.power_iters > 0 ? o.power_iters : 30;
            if ((e = reduce(p, p.v, nullptr, p.model_len, 0, SC_NORM2, st)))
                return cuda_fail(e, "norm launch");
            normalize_kernel<<<reduce_grid(p.model_len), 256, 0, st>>>(p.v, p.v, p.model_len,
                                                                       p.scal + SC_NORM2);
            p.launches[6]++;
            for (int it = 0; it < piters; ++it) {
                if ((rc = apply_forward(p, p.v, p.r, st))) return rc;
                if ((rc = apply_adjoint(p, p.r, p.z, st))) return rc;
                if ((e = reduce(p, p.v, p.z, p.model_len, 2, SC_DOT, st)))
                    return cuda_fail(e, "dot launch");
                if ((e = reduce(p, p.z, nullptr, p.model_len, 0, SC_NORM2, st)))
                    return cuda_fail(e, "norm launch");
                normalize_kernel<<<reduce_grid(p.model_len), 256, 0, st>>>(
                    p.z, p.v, p.model_len, p.scal + SC_NORM2);
                p.launches[6]++;
            }
            if ((e = cudaGetLastError())) return cuda_fail(e, "power iteration");
            if ((rc = read_scalars(p, h, st))) return rc;
            if (!(h[SC_DOT] > 0.0) || !std::isfinite(h[SC_DOT]))
                return set_error(AAHRT_ERR_NONFINITE, "power iteration gave %g", h[SC_DOT]);
            gamma = 0.95 / h[SC_DOT];
        }
    }
    if (!(gamma > 0.0) || !std::isfinite(gamma) || !(lam >= 0.0) || !std::isfinite(lam))
        return set_error(AAHRT_ERR_INVALID_ARG, "gamma (%g) and lambda (%g) must be finite, "
                         "gamma > 0, lambda >= 0", gamma, lam);

    // column-blocked copies: data, starting point m0 (warm) or 0, and z0 = m0
    if ((e = reblock(p, false, d, p.db, true, st))) return cuda_fail(e, "reblock data");
    if (o.warm_start) {
        if ((e = reblock(p, true, m, p.mb, true, st))) return cuda_fail(e, "reblock model");
    } else if ((e = cudaMemsetAsync(p.mb, 0, p.mblk_len * sizeof(float), st))) {
        return cuda_fail(e, "clear model");
    }
    if ((e = cudaMemcpyAsync(p.zb, p.mb, p.mblk_len * sizeof(float), cudaMemcpyDeviceToDevice,
                             st)))
        return cuda_fail(e, "copy model");

    std::vector<double> betas(std::max(iters, 1), 0.0);
    if (!o.ista) {
        double t = 1.0;
        for (int it = 0; it < iters; ++it) {
            const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
            betas[it] = (t - 1.0) / tn;
            t = tn;
        }
    }
    const float fg = (float)gamma, fth = (float)(gamma * lam);
    const float2 *cgt = per_cube ? p.cube_gt : nullptr;
    if (iters > 0) {
        if (o.use_graph && !p.profiling) {
            char key[256];
            if (per_cube)
                snprintf(key, sizeof key, "%d/cube/%d/w%d", iters, o.ista, p.wav_gen);
            else
                snprintf(key, sizeof key, "%d/%.9g/%.9g/%d/w%d", iters, (double)fg, (double)fth,
                         o.ista, p.wav_gen);
            if (!p.gexec || p.gkey != key) {
                if (p.gexec) { cudaGraphExecDestroy(p.gexec); p.gexec = nullptr; }
                cudaStream_t cs;
                if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)))
                    return cuda_fail(e, "capture stream");
                long long before[AAHRT_NSTAGES];
                std::memcpy(before, p.launches, sizeof before);
                cudaGraph_t graph = nullptr;
                e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
                if (!e) {
                    rc = run_iterations(p, iters, fg, fth, betas, cgt, cs);
                    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
                    if (!e) e = e2;
                }
                cudaStreamDestroy(cs);
                long long per = 0;
                for (int s = 0; s < AAHRT_NSTAGES; ++s) {
                    p.gstage[s] = p.launches[s] - before[s];
                    per += p.gstage[s];
                }
                std::memcpy(p.launches, before, sizeof before);
                if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
                if (e) { if (graph) cudaGraphDestroy(graph); return cuda_fail(e, "graph capture"); }
                e = cudaGraphInstantiate(&p.gexec, graph, 0);
                cudaGraphDestroy(graph);
                if (e) { p.gexec = nullptr; return cuda_fail(e, "graph instantiate"); }
                p.gkey = key;
                p.glaunches = per;
            }
            if ((e = cudaGraphLaunch(p.gexec, st))) return cuda_fail(e, "graph launch");
            // the kernels the captured sequence launches, per stage
            for (int s = 0; s < AAHRT_NSTAGES; ++s) p.launches[s] += p.gstage[s];
        } else {
            if ((rc = run_iterations(p, iters, fg, fth, betas, cgt, st))) return rc;
        }
    }

    if ((e = reblock(p, true, p.mb, m, false, st))) return cuda_fail(e, "reblock model");

    if (info && per_cube) {
        if ((rc = apply_forward(p, m, p.r, st, EPI_RESIDUAL, d))) return rc;
        if ((e = seg_reduce(p, p.r, nullptr, false, 0, CA_SS, st)) ||
            (e = seg_reduce(p, m, nullptr, true, 1, CA_L1, st)))
            return cuda_fail(e, "norm launch");
        std::vector<double> hc;
        if ((rc = read_cube_acc(p, &hc, st))) return rc;
        double ss = 0.0, l1 = 0.0, obj = 0.0;
        for (int c = 0; c < p.ncube; ++c) {
            const double sc = hc[(size_t)CA_SS * p.ncube + c], lc = hc[(size_t)CA_L1 * p.ncube + c];
            ss += sc;
            l1 += lc;
            obj += 0.5 * sc + clam[c] * lc;
        }
        info->iters = iters;
        info->gamma = gamma;
        info->lambda = lam;
        info->resid_norm = std::sqrt(ss);
        info->l1_norm = l1;
        info->objective = obj;
    } else if (info) {
        if ((rc = apply_forward(p, m, p.r, st, EPI_RESIDUAL, d))) return rc;
        if ((e = reduce(p, p.r, nullptr, p.data_len, 0, SC_SUMSQ, st)))
            return cuda_fail(e, "norm launch");
        if ((e = reduce(p, m, nullptr, p.model_len, 1, SC_L1, st)))
            return cuda_fail(e, "norm launch");
        if ((rc = read_scalars(p, h, st))) return rc;
        info->iters = iters;
        info->gamma = gamma;
        info->lambda = lam;
        info->resid_norm = std::sqrt(h[SC_SUMSQ]);
        info->l1_norm = h[SC_L1];
        info->objective = 0.5 * h[SC_SUMSQ] + lam * h[SC_L1];
    }
    return AAHRT_OK;
}

}  // namespace aahrt

using namespace aahrt;

extern "C" {

int aahrt_plan_create(aahrt_plan **out, const aahrt_geom *geom, const aahrt_opts *opts) {
    if (!out) return set_error(AAHRT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    const int G = (opts && opts->ngather > 0) ? opts->ngather : 1;
    Plan *p = nullptr;
    int rc = make_plan(&p, G, 1, geom, opts);
    if (rc) return rc;
    {
        DeviceGuard g(p->device);
        if ((rc = noalloc_prepare(p->device))) {
            free_plan(p);
            return rc;
        }
    }
    *out = new aahrt_plan{p};
    return AAHRT_OK;
}

int aahrt_plan_create_batched(aahrt_plan **out, int ncube, const aahrt_geom *geoms,
                              const aahrt_opts *opts) {
    if (!out) return set_error(AAHRT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (ncube < 1 || !geoms) return set_error(AAHRT_ERR_INVALID_ARG, "ncube < 1 or geoms NULL");
    if (opts && opts->ngather > 1)
        return set_error(AAHRT_ERR_INVALID_ARG, "ngather > 1 is for aahrt_plan_create");
    Plan *p = nullptr;
    int rc = make_plan(&p, ncube, ncube, geoms, opts);
    if (rc) return rc;
    {
        DeviceGuard g(p->device);
        if ((rc = noalloc_prepare(p->device))) {
            free_plan(p);
            return rc;
        }
    }
    *out = new aahrt_plan{p};
    return AAHRT_OK;
}

void aahrt_plan_destroy(aahrt_plan *plan) {
    if (!plan) return;
    free_plan(plan->p);
    delete plan;
}

int aahrt_plan_query(const aahrt_plan *plan, aahrt_plan_info *info) {
    if (!plan || !info) return set_error(AAHRT_ERR_INVALID_ARG, "plan or info is NULL");
    plan_info(*plan->p, info);
    return AAHRT_OK;
}

int aahrt_forward(aahrt_plan *plan, const float *m, float *d, void *stream) {
    if (!plan) return set_error(AAHRT_ERR_INVALID_ARG, "plan is NULL");
    Plan &p = *plan->p;
    DeviceGuard g(p.device);
    cudaStream_t st = (cudaStream_t)stream;
    Staged s;
    int rc = stage_args(p, m, p.model_len, true, d, p.data_len, st, &s);
    if (rc) return rc;
    if ((rc = apply_forward(p, s.in_dev, s.out_dev, st))) return rc;
    return finish_args(s, st);
}

int aahrt_adjoint(aahrt_plan *plan, const float *d, float *m, void *stream) {
    if (!plan) return set_error(AAHRT_ERR_INVALID_ARG, "plan is NULL");
    Plan &p = *plan->p;
    DeviceGuard g(p.device);
    cudaStream_t st = (cudaStream_t)stream;
    Staged s;
    int rc = stage_args(p, d, p.data_len, false, m, p.model_len, st, &s);
    if (rc) return rc;
    if ((rc = apply_adjoint(p, s.in_dev, s.out_dev, st))) return rc;
    return finish_args(s, st);
}

int aahrt_apply_stage(aahrt_plan *plan, int stage, const void *in, void *out, void *stream) {
    if (!plan) return set_error(AAHRT_ERR_INVALID_ARG, "plan is NULL");
    Plan &p = *plan->p;
    DeviceGuard g(p.device);
    int rc;
    if ((rc = check_dev_ptr(in, "in")) || (rc = check_dev_ptr(out, "out"))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    const float *fi = static_cast<const float *>(in);
    const float2 *ci = static_cast<const float2 *>(in);
    float *fo = static_cast<float *>(out);
    float2 *co = static_cast<float2 *>(out);
    switch (stage) {
        case 0: e = launch_r2c(p, true, fi, co, st); break;
        case 1: e = launch_slice(p, false, ci, co, st); break;
        case 2: e = launch_c2r(p, false, ci, fo, EPI_STORE, nullptr, FistaArgs{}, st); break;
        case 3: e = launch_r2c(p, false, fi, co, st); break;
        case 4:
            e = launch_ybound(p, ci, st);
            if (!e) e = launch_slice(p, true, ci, co, st);
            break;
        case 5: e = launch_c2r(p, true, ci, fo, EPI_STORE, nullptr, FistaArgs{}, st); break;
        default: return set_error(AAHRT_ERR_INVALID_ARG, "stage must be 0..5");
    }
    return e ? cuda_fail(e, "stage launch") : AAHRT_OK;
}

int aahrt_sparse_solve(aahrt_plan *plan, const float *d, float lambda, int iters, float *m,
                       const aahrt_solve_opts *opts, aahrt_solve_info *info, void *stream) {
    if (!plan) return set_error(AAHRT_ERR_INVALID_ARG, "plan is NULL");
    Plan &p = *plan->p;
    DeviceGuard g(p.device);
    int rc;
    if (iters < 0) return set_error(AAHRT_ERR_INVALID_ARG, "iters must be >= 0");
    aahrt_solve_opts o;
    std::memset(&o, 0, sizeof o);
    if (opts) o = *opts;
    if (!(o.lambda_rel > 0.0) && !(lambda >= 0.0 && std::isfinite(lambda)))
        return set_error(AAHRT_ERR_INVALID_ARG, "lambda must be finite and >= 0");
    if (o.lambda_rel < 0.0 || !std::isfinite(o.lambda_rel) || !std::isfinite(o.gamma))
        return set_error(AAHRT_ERR_INVALID_ARG, "lambda_rel and gamma must be finite");
    cudaStream_t st = (cudaStream_t)stream;
    bool hd = false, hm = false;
    if ((rc = classify_ptr(d, "d", &hd)) || (rc = classify_ptr(m, "m", &hm))) return rc;
    if ((hd || hm) && (rc = ensure_staging(p))) return rc;
    cudaError_t e;
    const float *dd = d;
    float *md = m;
    if (hd) {
        if ((e = cudaMemcpyAsync(p.stage_d, d, p.data_len * sizeof(float),
                                 cudaMemcpyHostToDevice, st)))
            return cuda_fail(e, "copy d to device");
        dd = p.stage_d;
    }
    if (hm) {
        md = p.stage_m;
        if (o.warm_start && (e = cudaMemcpyAsync(md, m, p.model_len * sizeof(float),
                                                 cudaMemcpyHostToDevice, st)))
            return cuda_fail(e, "copy m to device");
    }
    if ((rc = solve(p, dd, lambda, iters, md, o, info, st))) return rc;
    if (hm && (e = cudaMemcpyAsync(m, md, p.model_len * sizeof(float), cudaMemcpyDeviceToHost,
                                   st)))
        return cuda_fail(e, "copy m to host");
    return AAHRT_OK;
}

int aahrt_q_from_slowness(double pmin, double pmax, int nq, double *q0, double *dq) {
    if (!q0 || !dq || nq < 1 || !(pmin >= 0.0) || !(pmax > pmin) || !std::isfinite(pmax))
        return set_error(AAHRT_ERR_INVALID_ARG, "need 0 <= pmin < pmax, nq >= 1");
    *q0 = pmin * pmin;
    *dq = nq > 1 ? (pmax * pmax - pmin * pmin) / (nq - 1) : 0.0;
    return AAHRT_OK;
}

int aahrt_plan_set_profiling(aahrt_plan *plan, int on) {
    if (!plan) return set_error(AAHRT_ERR_INVALID_ARG, "plan is NULL");
    Plan &p = *plan->p;
    DeviceGuard g(p.device);
    if (on) {
        p.ev_used = 0;
        std::memset(p.prof_ms, 0, sizeof p.prof_ms);
        std::memset(p.launches, 0, sizeof p.launches);
    } else {
        int rc = collect_profile(p);
        if (rc) return rc;
    }
    p.profiling = on != 0;
    return AAHRT_OK;
}

int aahrt_plan_stage_times(aahrt_plan *plan, double *times_ms, long long *launches) {
    if (!plan) return set_error(AAHRT_ERR_INVALID_ARG, "plan is NULL");
    Plan &p = *plan->p;
    DeviceGuard g(p.device);
    int rc = collect_profile(p);
    if (rc) return rc;
    for (int s = 0; s < AAHRT_NSTAGES; ++s) {
        if (times_ms) times_ms[s] = p.prof_ms[s];
        if (launches) launches[s] = p.launches[s];
    }
    return AAHRT_OK;
}

int aahrt_plan_status(aahrt_plan *plan) {
    if (!plan) return set_error(AAHRT_ERR_INVALID_ARG, "plan is NULL");
    Plan &p = *plan->p;
    DeviceGuard g(p.device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e) return cuda_fail(e, "synchronise");
    int flag = 0;
    if ((e = cudaMemcpy(&flag, p.counters + kTcErrSlot, sizeof flag, cudaMemcpyDeviceToHost)))
        return cuda_fail(e, "read status");
    if (flag) {
        cudaMemset(p.counters + kTcErrSlot, 0, sizeof(int));
        return set_error(AAHRT_ERR_TIMEOUT, "a tensor-core kernel timed out waiting for its "
                         "matrix operations");
    }
    return AAHRT_OK;
}

int aahrt_plan_test_stall(aahrt_plan *plan, int on) {
    if (!plan) return set_error(AAHRT_ERR_INVALID_ARG, "plan is NULL");
    Plan &p = *plan->p;
    if (p.precision != AAHRT_PRECISION_SPLIT_BF16)
        return set_error(AAHRT_ERR_UNSUPPORTED, "only tensor-core plans wait on matrix operations");
    if (on != 0 && on != 1) return set_error(AAHRT_ERR_INVALID_ARG, "on must be 0 or 1");
    p.tc_stall = on != 0;
    if (p.gexec) {                 // a captured solve holds the old kernel arguments
        cudaGraphExecDestroy(p.gexec);
        p.gexec = nullptr;
        p.gkey.clear();
    }
    return AAHRT_OK;
}

const char *aahrt_status_string(int status) {
    switch (status) {
        case AAHRT_OK: return "success";
        case AAHRT_ERR_INVALID_ARG: return "invalid argument";
        case AAHRT_ERR_OOM: return "out of memory";
        case AAHRT_ERR_CUDA: return "CUDA error";
        case AAHRT_ERR_UNSUPPORTED: return "unsupported";
        case AAHRT_ERR_TIMEOUT: return "device wait timed out";
        case AAHRT_ERR_NONFINITE: return "non-finite value";
        default: return "unknown status";
    }
}

const char *aahrt_last_error(void) { return last_error_text(); }

}  // extern "C"
