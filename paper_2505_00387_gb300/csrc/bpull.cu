// The paper's velocity scan (Algorithm 2 with the B-coefficients of Sec. 3.4)
// for data on a regular offset grid: stretch the data time axis (the model's
// stretch S) and FFT it, then per bin f' and azimuth slice theta_j pull the
// data spectrum at (x, y) = +-sqrt(k/f') (cos theta_j, sin theta_j) by
// bilinear interpolation for every q-grid wavenumber k = k_u + n/dq
// (u < nos, all alias rings n inside the grid), with the centring phase
// exp(+2 pi i k q_c); inverse DFT along u onto the q axis in shared memory;
// Hermitian synthesis and the stretch undone (U) on the model columns.
#include <algorithm>
#include <cmath>

#include "fft.cuh"
#include "internal.cuh"

namespace aahrt {

struct PullArgs {
    const float2 *__restrict__ D;       // data spectrum [k][ntr]
    const SliceGroup *__restrict__ groups;
    const float2 *__restrict__ tw;
    int nbins, nq, ntheta, nos, Lq, cq, ngroup;
    int nx, ny;
    float x0, dx, y0, dy, r2max;
    double inv_nos_dq;      // 1 / (nos dq): wavenumber of grid step u
    double cfrac;           // q_c / (nos dq): centring phase per grid step, cycles
    double kscale;          // f_k = k * kscale
    float scale;            // 1 / Nfft
};

// bilinear (B-coefficient) read of the grid spectrum; zero outside
__device__ __forceinline__ float2 grid_read(const PullArgs &a, const float2 *Dk, float x,
                                           float y) {
    const float fx = (x - a.x0) / a.dx, fy = (y - a.y0) / a.dy;
    const float flx = floorf(fx), fly = floorf(fy);
    const int ix = (int)flx, iy = (int)fly;
    const float ax = fx - flx, ay = fy - fly;
    float2 v = make_float2(0.f, 0.f);
#pragma unroll
    for (int cx = 0; cx < 2; ++cx)
#pragma unroll
        for (int cy = 0; cy < 2; ++cy) {
            const int jx = ix + cx, jy = iy + cy;
            if (jx < 0 || jx >= a.nx || jy < 0 || jy >= a.ny) continue;
            const float w = (cx ? ax : 1.f - ax) * (cy ? ay : 1.f - ay);
            const float2 d = __ldg(Dk + (long long)jx * a.ny + jy);
            v.x = fmaf(w, d.x, v.x);
            v.y = fmaf(w, d.y, v.y);
        }
    return v;
}

__global__ void __launch_bounds__(256)
pull_kernel(const PullArgs a, float2 *__restrict__ X) {
    extern __shared__ float4 smem_f4[];
    float *smf = reinterpret_cast<float *>(smem_f4);
    const int gi = blockIdx.x % a.ngroup;
    const int k = blockIdx.x / a.ngroup;
    const SliceGroup g = a.groups[gi];
    const int lds = ld_split(a.nos);
    const int mask = a.nos - 1;
    float *Gre = smf, *Gim = smf + g.nj * lds;
    const float2 *Dk = a.D + (long long)k * a.nx * a.ny;
    const double f = k * a.kscale;
    for (int idx = threadIdx.x; idx < g.nj * a.nos; idx += blockDim.x) {
        const int jj = idx / a.nos, u = idx - jj * a.nos;
        float sr = 0.f, si = 0.f;
        if (k > 0) {
            const double th = (double)(g.ja + jj) / a.ntheta;     // theta / pi
            double sd, cd;
            sincospi(th, &sd, &cd);
            const float c = (float)cd, s = (float)sd;
            const double ph_u = (double)u * a.cfrac;
            const double ph_n = (double)a.nos * a.cfrac;
            for (int n = 0;; ++n) {
                const double kap = (double)(u + n * a.nos) * a.inv_nos_dq;
                const double r2 = kap / f;
                if (r2 > (double)a.r2max) break;
                const float r = (float)sqrt(r2);
                const float2 v0 = grid_read(a, Dk, r * c, r * s);
                const float2 v1 = grid_read(a, Dk, -r * c, -r * s);
                double ph = ph_u + n * ph_n;
                ph -= floor(ph);
                float ps, pc;
                sincospif((float)(2.0 * ph), &ps, &pc);
                const float vr = v0.x + v1.x, vi = v0.y + v1.y;
                sr += vr * pc - vi * ps;
                si += vr * ps + vi * pc;
            }
        }
        Gre[jj * lds + padi(u)] = sr;
        Gim[jj * lds + padi(u)] = si;
    }
    __syncthreads();
    block_fft<true, true>(SBatch{Gre, Gim, lds}, g.nj, a.Lq, a.tw);
    float2 *Xk = X + (long long)k * a.nq * a.ntheta;
    for (int idx = threadIdx.x; idx < g.nj * a.nq; idx += blockDim.x) {
        const int l = idx / g.nj, jj = idx - l * g.nj;
        const int p = jj * lds + padi(brev_bits((l - a.cq) & mask, a.Lq));
        Xk[(long long)l * a.ntheta + g.ja + jj] = make_float2(a.scale * Gre[p], a.scale * Gim[p]);
    }
}

cudaError_t launch_stretch_data(Plan &p, const float *d, float2 *Y, cudaStream_t st);
cudaError_t launch_unstretch_model(Plan &p, const float2 *X, float *m, cudaStream_t st);

}  // namespace aahrt

using namespace aahrt;

extern "C" int aahrt_velocity_scan_grid(aahrt_plan *plan, const aahrt_grid *grid,
                                        const float *d, float *m, void *stream) {
    if (!plan || !grid) return set_error(AAHRT_ERR_INVALID_ARG, "plan or grid is NULL");
    Plan &p = *plan->p;
    DeviceGuard g(p.device);
    int rc;
    if ((rc = check_dev_ptr(d, "d")) || (rc = check_dev_ptr(m, "m"))) return rc;
    if (p.precision != AAHRT_PRECISION_FP32 || p.ncube != 1 || p.ngather != 1)
        return set_error(AAHRT_ERR_UNSUPPORTED, "the grid scan needs a single-gather FP32 plan");
    if (p.ntau != p.nt || p.nq < 2)
        return set_error(AAHRT_ERR_UNSUPPORTED, "the grid scan needs ntau == nt and nq >= 2");
    if (p.qexplicit)
        return set_error(AAHRT_ERR_UNSUPPORTED, "the grid scan needs a uniform q axis (FFT "
                         "along q)");
    if (grid->nx < 1 || grid->ny < 1 || (long long)grid->nx * grid->ny != p.ntr[0] ||
        !(grid->dx > 0.0) || !(grid->dy > 0.0) || !std::isfinite(grid->x0) ||
        !std::isfinite(grid->y0))
        return set_error(AAHRT_ERR_INVALID_ARG, "grid must hold the plan's %d traces with "
                         "dx, dy > 0", p.ntr[0]);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    static int max_smem = 0;          // function attribute, process-wide
    if (!max_smem) {
        int mx = 0;
        if ((e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                        p.device)) ||
            (e = raise_smem_limit(pull_kernel, mx)))
            return cuda_fail(e, "pull kernel attributes");
        cudaFuncAttributes at;
        if ((e = cudaFuncGetAttributes(&at, pull_kernel))) return cuda_fail(e, "pull kernel attributes");
        max_smem = mx - (int)at.sharedSizeBytes;
    }
    // one group's split q grid (re and im planes of every owned slice)
    const size_t smem = (size_t)p.tgroup * ld_split(p.nos) * 2 * sizeof(float);
    if ((int)smem > max_smem)
        return set_error(AAHRT_ERR_UNSUPPORTED, "the grid scan's q grids (%zu bytes) exceed "
                         "shared memory; lower theta_group", smem);
    if ((e = launch_stretch_data(p, d, p.Y, st))) return cuda_fail(e, "stretch+FFT launch");
    PullArgs a;
    a.D = p.Y;
    a.groups = p.groups;
    a.tw = p.tw_q;
    a.nbins = p.nbins;
    a.nq = p.nq;
    a.ntheta = p.ntheta;
    a.nos = p.nos;
    a.Lq = p.Lq;
    a.cq = p.cq;
    a.ngroup = p.ngroup;
    a.nx = grid->nx;
    a.ny = grid->ny;
    a.x0 = (float)grid->x0;
    a.dx = (float)grid->dx;
    a.y0 = (float)grid->y0;
    a.dy = (float)grid->dy;
    const double xa = std::max(std::fabs(grid->x0), std::fabs(grid->x0 + (grid->nx - 1) * grid->dx));
    const double ya = std::max(std::fabs(grid->y0), std::fabs(grid->y0 + (grid->ny - 1) * grid->dy));
    a.r2max = (float)(xa * xa + ya * ya);
    a.inv_nos_dq = 1.0 / (p.nos * p.dq);
    a.cfrac = (p.q0 + p.cq * p.dq) / (p.nos * p.dq);
    a.kscale = 1.0 / (p.nfft * p.ds);
    a.scale = (float)(1.0 / p.nfft);
    prof_begin(p, 4, st);
    pull_kernel<<<p.nbins * p.ngroup, 256, smem, st>>>(a, p.X);
    prof_end(p, st);
    p.launches[4]++;
    if ((e = cudaGetLastError())) return cuda_fail(e, "pull launch");
    if ((e = launch_unstretch_model(p, p.X, m, st))) return cuda_fail(e, "unstretch launch");
    return AAHRT_OK;
}
