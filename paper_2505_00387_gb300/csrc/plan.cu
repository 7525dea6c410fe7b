// Plan construction of libaahrt: stretched-time sampling (Sec. 3.3 steps 1-2,
// eq. q3), azimuth binning of the traces (theta factors of eq. thli),
// resampler tables of the stretch S and its undoing U (Sec. 3.3: a local
// "spline" interpolation; here Keys' cubic convolution or linear), the
// spreading kernel of the q-slice, device workspace and work lists.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <vector>

#include "fft.cuh"
#include "internal.cuh"

namespace aahrt {

cudaError_t set_time_kernel_attrs(size_t smem);
cudaError_t configure_slice_kernels(Plan &p, int num_sms);

static thread_local char g_err[1024] = "";

int set_error(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    cudaGetLastError();  // clear a sticky launch error
    return set_error(e == cudaErrorMemoryAllocation ? AAHRT_ERR_OOM : AAHRT_ERR_CUDA,
                     "%s: %s", what, cudaGetErrorString(e));
}

const char *last_error_text() { return g_err; }

// ------------------------------------------------------------- helpers
static long long next_pow2(long long n) {
    long long p = 1;
    while (p < n) p <<= 1;
    return p;
}
static int ilog2(long long n) {
    int l = 0;
    while ((1LL << l) < n) ++l;
    return l;
}

// Keys' cubic convolution kernel, a = -1/2.
static double keys_kernel(double x) {
    const double a = -0.5;
    const double ax = std::fabs(x);
    if (ax <= 1.0) return (a + 2.0) * ax * ax * ax - (a + 3.0) * ax * ax + 1.0;
    if (ax < 2.0) return a * ax * ax * ax - 5.0 * a * ax * ax + 8.0 * a * ax - 4.0 * a;
    return 0.0;
}
static double linear_kernel(double x) {
    const double ax = std::fabs(x);
    return ax < 1.0 ? 1.0 - ax : 0.0;
}

struct HostCSR {
    std::vector<int> rowptr, col;
    std::vector<float> val;
    int nrows = 0;
};

// Interpolation rows at fractional positions pos[o] of an input axis of n_in
// samples; taps outside the axis (and exact zeros) are left out.
static HostCSR resampler(const std::vector<double> &pos, int n_in, int interp) {
    HostCSR c;
    c.nrows = (int)pos.size();
    c.rowptr.push_back(0);
    const int t0 = interp == AAHRT_INTERP_KEYS ? -1 : 0;
    const int t1 = interp == AAHRT_INTERP_KEYS ? 2 : 1;
    for (double u : pos) {
        const long long b = (long long)std::floor(u);
        for (int t = t0; t <= t1; ++t) {
            const long long i = b + t;
            if (i < 0 || i >= n_in) continue;
            const double wv = interp == AAHRT_INTERP_KEYS ? keys_kernel(u - (double)i)
                                                          : linear_kernel(u - (double)i);
            if (wv == 0.0) continue;
            c.col.push_back((int)i);
            c.val.push_back((float)wv);
        }
        c.rowptr.push_back((int)c.col.size());
    }
    return c;
}

// Exact transpose (same float weights) of a CSR with ncols columns.
static HostCSR transpose(const HostCSR &a, int ncols) {
    HostCSR t;
    t.nrows = ncols;
    t.rowptr.assign(ncols + 1, 0);
    for (int c : a.col) t.rowptr[c + 1]++;
    for (int i = 0; i < ncols; ++i) t.rowptr[i + 1] += t.rowptr[i];
    t.col.resize(a.col.size());
    t.val.resize(a.val.size());
    std::vector<int> fill(t.rowptr.begin(), t.rowptr.end() - 1);
    for (int r = 0; r < a.nrows; ++r)
        for (int e = a.rowptr[r]; e < a.rowptr[r + 1]; ++e) {
            const int d = fill[a.col[e]]++;
            t.col[d] = r;
            t.val[d] = a.val[e];
        }
    return t;
}

// Fourier transform of the spreading kernel phi(z) = exp(beta(sqrt(1-(2z/W)^2)-1)),
// |z| <= W/2: phihat(nu) = int phi(z) cos(2 pi nu z) dz, by the substitution
// z = (W/2) sin t, which turns it into the smooth integral of
// exp(beta (cos t - 1)) cos(pi nu W sin t) (W/2) cos t over [-pi/2, pi/2]
// (trapezoid rule; the integrand vanishes at both ends).
static double es_fourier(double nu, double beta, int W) {
    const int M = 4000;
    const double h = M_PI / M;
    double s = 0.0;
    for (int i = 1; i < M; ++i) {
        const double t = -0.5 * M_PI + i * h;
        s += std::exp(beta * (std::cos(t) - 1.0)) * std::cos(M_PI * nu * W * std::sin(t)) *
             std::cos(t);
    }
    return s * h * 0.5 * W;
}

static unsigned long long to_fixed64(double x) {
    double f = x - std::floor(x);  // [0, 1)
    double s = std::ldexp(f, 64);
    if (!(s < 18446744073709551616.0)) s = 0.0;
    return (unsigned long long)s;
}

struct CubeGeo {
    std::vector<TraceGeo> sorted;
    std::vector<int> start;  // start[j]: first sorted trace with j0 == j (size ntheta+1)
};

static CubeGeo bin_cube(const Plan &p, const double *hx, const double *hy, int ntr) {
    CubeGeo g;
    std::vector<TraceGeo> tr(ntr);
    const double dth = M_PI / p.ntheta;
    const double scale = 1.0 / (p.nfft * p.ds);
    for (int h = 0; h < ntr; ++h) {
        const double x = hx[h], y = hy[h];
        const double r2 = x * x + y * y;
        double th = 0.0;
        if (r2 > 0.0) {
            th = std::fmod(std::atan2(y, x), M_PI);
            if (th < 0.0) th += M_PI;
        }
        const double ph = th / dth;
        int j = (int)std::floor(ph);
        double fr = ph - j;
        if (j >= p.ntheta) { j -= p.ntheta; fr = 0.0; }
        if (j < 0) j = 0;
        if (j >= p.ntheta) j = p.ntheta - 1;
        TraceGeo t;
        t.A = to_fixed64((p.q0 + p.cq * p.dq) * r2 * scale);
        t.B = to_fixed64(p.dq * r2 * scale);
        t.w0 = (float)(1.0 - fr);
        t.w1 = (float)fr;
        t.j0 = j;
        t.col = h;
        tr[h] = t;
    }
    std::vector<int> idx(ntr);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(),
                     [&](int a, int b) { return tr[a].j0 < tr[b].j0; });
    g.sorted.resize(ntr);
    for (int i = 0; i < ntr; ++i) g.sorted[i] = tr[idx[i]];
    g.start.assign(p.ntheta + 1, 0);
    for (int i = 0; i < ntr; ++i) g.start[g.sorted[i].j0 + 1]++;
    for (int j = 0; j < p.ntheta; ++j) g.start[j + 1] += g.start[j];
    return g;
}

template <typename T>
static cudaError_t upload(T **dst, const std::vector<T> &src) {
    *dst = nullptr;
    if (src.empty()) return cudaSuccess;
    cudaError_t e = cudaMalloc((void **)dst, src.size() * sizeof(T));
    if (e) return e;
    return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

void free_plan(Plan *p) {
    if (!p) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p->device);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    void *ptrs[] = {p->tw_t, p->tw_q, p->dec, p->geo, p->groups, p->counters,
                    p->cg_model, p->cg_data, p->csr_i, p->csr_v, p->X, p->Y,
                    p->z, p->r, p->v, p->scal, p->stage_m, p->stage_d};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    cudaSetDevice(cur);
    delete p;
}

static int validate_geom(const aahrt_geom *g, int idx) {
    if (!g) return set_error(AAHRT_ERR_INVALID_ARG, "geometry %d is NULL", idx);
    if (g->nt < 4 || g->ntau < 4)
        return set_error(AAHRT_ERR_INVALID_ARG, "geometry %d: nt and ntau must be >= 4", idx);
    if (g->nq < 1 || g->ntheta < 1 || g->ntr < 1)
        return set_error(AAHRT_ERR_INVALID_ARG, "geometry %d: nq, ntheta, ntr must be >= 1", idx);
    if (!(g->dt > 0.0) || !std::isfinite(g->dt))
        return set_error(AAHRT_ERR_INVALID_ARG, "geometry %d: dt must be > 0", idx);
    if (!std::isfinite(g->q0) || !std::isfinite(g->dq) || (g->nq > 1 && !(g->dq > 0.0)))
        return set_error(AAHRT_ERR_INVALID_ARG, "geometry %d: q0/dq invalid", idx);
    if (!g->hx || !g->hy)
        return set_error(AAHRT_ERR_INVALID_ARG, "geometry %d: hx/hy are NULL", idx);
    if (g->nq > 1024)
        return set_error(AAHRT_ERR_UNSUPPORTED, "geometry %d: nq > 1024", idx);
    for (int h = 0; h < g->ntr; ++h)
        if (!std::isfinite(g->hx[h]) || !std::isfinite(g->hy[h]))
            return set_error(AAHRT_ERR_NONFINITE, "geometry %d: offset %d not finite", idx, h);
    return AAHRT_OK;
}

// Build a plan for ncube cubes.  geoms has ndist entries: ndist == ncube
// (independent cubes) or ndist == 1 (ncube gathers on one geometry).
int build_plan(Plan **out, int ncube, int ndist, const aahrt_geom *geoms,
               const aahrt_opts *opts_in) {
    if (!out) return set_error(AAHRT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (ncube < 1) return set_error(AAHRT_ERR_INVALID_ARG, "ncube must be >= 1");
    aahrt_opts opts;
    std::memset(&opts, 0, sizeof opts);
    if (opts_in) opts = *opts_in;
    for (int c = 0; c < ndist; ++c) {
        int rc = validate_geom(geoms + c, c);
        if (rc) return rc;
    }
    const aahrt_geom &g0 = geoms[0];
    for (int c = 1; c < ndist; ++c) {
        const aahrt_geom &g = geoms[c];
        if (g.nt != g0.nt || g.dt != g0.dt || g.ntau != g0.ntau || g.nq != g0.nq ||
            g.q0 != g0.q0 || g.dq != g0.dq || g.ntheta != g0.ntheta)
            return set_error(AAHRT_ERR_INVALID_ARG,
                             "cube %d: axes differ from cube 0 (nt, dt, ntau, nq, q0, dq, "
                             "ntheta must be shared)", c);
    }
    if (opts.interp_kind != AAHRT_INTERP_KEYS && opts.interp_kind != AAHRT_INTERP_LINEAR)
        return set_error(AAHRT_ERR_INVALID_ARG, "interp_kind must be 0 or 1");
    const int W = opts.spread_width ? opts.spread_width : 7;
    if (W < kMinW || W > kMaxW)
        return set_error(AAHRT_ERR_INVALID_ARG, "spread_width must be in [%d, %d]", kMinW, kMaxW);
    if (opts.sigma_t < 0.0 || (opts.sigma_t > 0.0 && opts.sigma_t < 1.0))
        return set_error(AAHRT_ERR_INVALID_ARG, "sigma_t must be 0 (default) or >= 1");
    if (opts.fmax < 0.0 || opts.theta_group < 0 || opts.ngather < 0)
        return set_error(AAHRT_ERR_INVALID_ARG, "fmax, theta_group, ngather must be >= 0");

    Plan *p = new Plan();
    cudaGetDevice(&p->device);
    p->nt = g0.nt;
    p->dt = g0.dt;
    p->ntau = g0.ntau;
    p->nq = g0.nq;
    p->q0 = g0.q0;
    p->dq = g0.nq > 1 ? g0.dq : 0.0;
    p->ntheta = g0.ntheta;
    p->interp = opts.interp_kind;
    p->w = W;
    p->sigma_t = opts.sigma_t > 0.0 ? opts.sigma_t : 2.0;
    p->fmax = opts.fmax;
    p->ncube = ncube;
    p->ngather = ndist == 1 ? ncube : 1;

    // ---------------------------------------------------- stretched time
    double r2max = 0.0;
    for (int c = 0; c < ndist; ++c)
        for (int h = 0; h < geoms[c].ntr; ++h)
            r2max = std::max(r2max, geoms[c].hx[h] * geoms[c].hx[h] + geoms[c].hy[h] * geoms[c].hy[h]);
    if (!(r2max > 0.0)) {
        free_plan(p);
        return set_error(AAHRT_ERR_INVALID_ARG, "all offsets are zero");
    }
    p->tmax = (p->nt - 1) * p->dt;
    const double qabs = std::max(std::fabs(p->q0), std::fabs(p->q0 + (p->nq - 1) * p->dq));
    p->rho = qabs * r2max / (p->tmax * p->tmax);
    const double want = std::ceil(p->sigma_t * p->nt * (1.0 + p->rho));
    if (!(want < 1e9)) {
        free_plan(p);
        return set_error(AAHRT_ERR_UNSUPPORTED, "FFT frame too long (rho = %g)", p->rho);
    }
    p->nfft = (int)next_pow2((long long)want);
    if (p->nfft > 16384) {
        free_plan(p);
        return set_error(AAHRT_ERR_UNSUPPORTED,
                         "FFT frame of %d samples exceeds 16384 (nt = %d, rho = %g)", p->nfft,
                         p->nt, p->rho);
    }
    p->L = ilog2(p->nfft);
    p->ns = (int)std::floor((p->nfft - 2) / (1.0 + p->rho)) + 1;
    p->ds = p->tmax * p->tmax / (p->ns - 1);
    p->kmax = p->nfft / 2 - 1;
    if (p->fmax > 0.0)
        p->kmax = std::min(p->kmax, (int)std::floor(p->fmax * p->nfft * p->ds));
    p->nbins = p->kmax + 1;
    p->pairs = std::max(1, std::min(8, 8192 / p->nfft));

    // ----------------------------------------------------- q spreading
    p->nos = (int)std::max(16LL, next_pow2(2LL * p->nq));
    p->Lq = ilog2(p->nos);
    p->cq = p->nq / 2;
    const double sigma_q = (double)p->nos / p->nq;
    p->beta = 0.97 * M_PI * W * (1.0 - 1.0 / (2.0 * sigma_q));
    std::vector<float> dec(p->nq);
    for (int l = 0; l < p->nq; ++l)
        dec[l] = (float)(1.0 / es_fourier((double)(l - p->cq) / p->nos, p->beta, W));

    // --------------------------------------------------- azimuth groups
    const int ldq = padded_len(p->nos);
    const size_t per_slice = (size_t)ldq * sizeof(float2);
    if (opts.theta_group > 0) {
        p->tgroup = std::min(opts.theta_group, p->ntheta);
    } else {
        const size_t budget = 80 * 1024;
        if (p->ntheta * per_slice <= budget) {
            p->tgroup = p->ntheta;
        } else {
            int t = (int)(budget / per_slice) - 1;
            if (t < 1) t = 1;
            const int ng = (p->ntheta + t - 1) / t;
            p->tgroup = (p->ntheta + ng - 1) / ng;
        }
    }
    p->ngroup = (p->ntheta + p->tgroup - 1) / p->tgroup;
    if (p->ngroup == 1) p->tgroup = p->ntheta;

    // ------------------------------------------------ per-cube geometry
    std::vector<CubeGeo> cg(ndist);
    for (int c = 0; c < ndist; ++c) cg[c] = bin_cube(*p, geoms[c].hx, geoms[c].hy, geoms[c].ntr);
    std::vector<long long> geo_off(ndist, 0);
    std::vector<TraceGeo> geo_all;
    for (int c = 0; c < ndist; ++c) {
        geo_off[c] = (long long)geo_all.size();
        geo_all.insert(geo_all.end(), cg[c].sorted.begin(), cg[c].sorted.end());
    }
    p->ntr.resize(ncube);
    p->data_off.resize(ncube);
    std::vector<long long> y_off(ncube);
    long long acc_tr = 0;
    for (int c = 0; c < ncube; ++c) {
        const int dc = ndist == 1 ? 0 : c;
        p->ntr[c] = geoms[dc].ntr;
        p->data_off[c] = acc_tr * p->nt;
        y_off[c] = acc_tr * p->nbins;
        acc_tr += p->ntr[c];
    }
    p->ntr_total = acc_tr;
    const long long C = (long long)p->nq * p->ntheta;
    p->cols_model = C;
    p->model_len = (long long)ncube * p->ntau * C;
    p->data_len = acc_tr * p->nt;
    p->x_len = (long long)ncube * p->nbins * C;
    p->y_len = acc_tr * p->nbins;

    std::vector<SliceGroup> groups;
    for (int c = 0; c < ncube; ++c) {
        const int dc = ndist == 1 ? 0 : c;
        const CubeGeo &G = cg[dc];
        for (int gi = 0; gi < p->ngroup; ++gi) {
            SliceGroup s;
            s.geo_off = geo_off[dc];
            s.x_off = (long long)c * p->nbins * C;
            s.y_off = y_off[c];
            s.ntr = p->ntr[c];
            s.ja = gi * p->tgroup;
            s.nj = std::min(p->tgroup, p->ntheta - s.ja);
            s.f0 = G.start[s.ja];
            s.f1 = G.start[s.ja + s.nj];
            if (p->ngroup > 1) {
                const int jp = (s.ja - 1 + p->ntheta) % p->ntheta;
                s.e0 = G.start[jp];
                s.e1 = G.start[jp + 1];
            } else {
                s.e0 = s.e1 = 0;
            }
            groups.push_back(s);
        }
    }
    std::stable_sort(groups.begin(), groups.end(), [](const SliceGroup &a, const SliceGroup &b) {
        return (a.f1 - a.f0 + a.e1 - a.e0) > (b.f1 - b.f0 + b.e1 - b.e0);
    });
    p->ngroups_total = (int)groups.size();
    p->slice_items = (long long)p->ngroups_total * p->nbins;

    // ------------------------------------------------- column groups
    const int cpg = 2 * p->pairs;
    std::vector<ColGroup> cgm, cgd;
    for (int c = 0; c < ncube; ++c)
        for (long long c0 = 0; c0 < C; c0 += cpg) {
            ColGroup q;
            q.real_off = (long long)c * p->ntau * C + c0;
            q.spec_off = (long long)c * p->nbins * C + c0;
            q.ld_real = (int)C;
            q.ld_spec = (int)C;
            q.ncol = (int)std::min<long long>(cpg, C - c0);
            q.pad_ = 0;
            cgm.push_back(q);
        }
    for (int c = 0; c < ncube; ++c)
        for (int h0 = 0; h0 < p->ntr[c]; h0 += cpg) {
            ColGroup q;
            q.real_off = p->data_off[c] + h0;
            q.spec_off = y_off[c] + h0;
            q.ld_real = p->ntr[c];
            q.ld_spec = p->ntr[c];
            q.ncol = std::min(cpg, p->ntr[c] - h0);
            q.pad_ = 0;
            cgd.push_back(q);
        }
    p->ncg_model = (int)cgm.size();
    p->ncg_data = (int)cgd.size();

    // ------------------------------------------------------ resamplers
    std::vector<double> upos(p->ns), vpos(p->nt);
    for (int n = 0; n < p->ns; ++n) upos[n] = std::sqrt(n * p->ds) / p->dt;
    for (int i = 0; i < p->nt; ++i) vpos[i] = (i * p->dt) * (i * p->dt) / p->ds;
    const HostCSR S = resampler(upos, p->ntau, p->interp);
    const HostCSR ST = transpose(S, p->ntau);
    const HostCSR U = resampler(vpos, p->ns, p->interp);
    const HostCSR UT = transpose(U, p->ns);
    std::vector<int> ci;
    std::vector<float> cv;
    size_t offs_i[4][3], offs_v[4];
    const HostCSR *all[4] = {&S, &ST, &U, &UT};
    for (int t = 0; t < 4; ++t) {
        offs_i[t][0] = ci.size();
        ci.insert(ci.end(), all[t]->rowptr.begin(), all[t]->rowptr.end());
        offs_i[t][1] = ci.size();
        ci.insert(ci.end(), all[t]->col.begin(), all[t]->col.end());
        offs_v[t] = cv.size();
        cv.insert(cv.end(), all[t]->val.begin(), all[t]->val.end());
        cv.push_back(0.f);  // keeps every table non-empty
    }

    // ------------------------------------------------------- twiddles
    auto twiddles = [](int N) {
        std::vector<float2> tw(std::max(1, N / 2));
        for (int m = 0; m < N / 2; ++m) {
            const double a = -2.0 * M_PI * m / N;
            tw[m] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
        if (N < 2) tw[0] = make_float2(1.f, 0.f);
        return tw;
    };

    // ------------------------------------------------------- device
    cudaError_t e;
    int num_sms = 0;
#define AAHRT_TRY(call, what)            \
    do {                                 \
        e = (call);                      \
        if (e) {                         \
            int rc = cuda_fail(e, what); \
            free_plan(p);                \
            return rc;                   \
        }                                \
    } while (0)
    AAHRT_TRY(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, p->device),
              "device query");
    AAHRT_TRY(upload(&p->tw_t, twiddles(p->nfft)), "upload twiddles");
    AAHRT_TRY(upload(&p->tw_q, twiddles(p->nos)), "upload twiddles");
    AAHRT_TRY(upload(&p->dec, dec), "upload deapodisation");
    AAHRT_TRY(upload(&p->geo, geo_all), "upload geometry");
    AAHRT_TRY(upload(&p->groups, groups), "upload work list");
    AAHRT_TRY(upload(&p->cg_model, cgm), "upload column groups");
    AAHRT_TRY(upload(&p->cg_data, cgd), "upload column groups");
    AAHRT_TRY(upload(&p->csr_i, ci), "upload resamplers");
    AAHRT_TRY(upload(&p->csr_v, cv), "upload resamplers");
    AAHRT_TRY(cudaMalloc((void **)&p->counters, 16 * sizeof(int)), "alloc counters");
    AAHRT_TRY(cudaMemset(p->counters, 0, 16 * sizeof(int)), "clear counters");
    DevCSR *dst[4] = {&p->S, &p->ST, &p->U, &p->UT};
    for (int t = 0; t < 4; ++t) {
        dst[t]->rowptr = p->csr_i + offs_i[t][0];
        dst[t]->col = p->csr_i + offs_i[t][1];
        dst[t]->val = p->csr_v + offs_v[t];
        dst[t]->nrows = all[t]->nrows;
    }
    AAHRT_TRY(cudaMalloc((void **)&p->X, std::max<long long>(1, p->x_len) * sizeof(float2)),
              "alloc X workspace");
    AAHRT_TRY(cudaMalloc((void **)&p->Y, std::max<long long>(1, p->y_len) * sizeof(float2)),
              "alloc Y workspace");

    p->smem_r2c = (size_t)p->pairs * padded_len(p->nfft) * sizeof(float2);
    p->smem_c2r = p->smem_r2c;
    p->smem_sfwd = (size_t)(p->tgroup + (p->ngroup > 1 ? 1 : 0)) * per_slice;
    p->smem_sadj = (size_t)p->tgroup * per_slice;
    int max_smem = 0;
    AAHRT_TRY(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                     p->device), "device query");
    if ((int)p->smem_r2c > max_smem || (int)p->smem_sfwd > max_smem) {
        free_plan(p);
        return set_error(AAHRT_ERR_UNSUPPORTED,
                         "shared memory per block (%zu / %zu bytes) exceeds %d; lower "
                         "theta_group", p->smem_r2c, p->smem_sfwd, max_smem);
    }
    AAHRT_TRY(set_time_kernel_attrs(p->smem_r2c), "kernel attributes");
    AAHRT_TRY(configure_slice_kernels(*p, num_sms), "slice kernel configuration");
#undef AAHRT_TRY
    *out = p;
    return AAHRT_OK;
}

void plan_info(const Plan &p, aahrt_plan_info *info) {
    std::memset(info, 0, sizeof *info);
    info->nfft = p.nfft;
    info->ns = p.ns;
    info->nbins = p.nbins;
    info->nq_os = p.nos;
    info->spread_width = p.w;
    info->theta_group = p.tgroup;
    info->ncube = p.ncube;
    info->ngather = p.ngather;
    info->ds = p.ds;
    info->rho = p.rho;
    info->beta = p.beta;
    info->model_len = p.model_len;
    info->data_len = p.data_len;
    info->xspec_len = p.x_len;
    info->yspec_len = p.y_len;
    info->workspace_bytes = (p.x_len + p.y_len) * (long long)sizeof(float2);
}

// ----------------------------------------------------------- profiling
void prof_begin(Plan &p, int stage, cudaStream_t st) {
    if (!p.profiling) return;
    const size_t i = p.ev_used;
    while (p.ev_pool.size() < 2 * i + 2) {
        cudaEvent_t ev;
        if (cudaEventCreate(&ev) != cudaSuccess) { p.profiling = false; return; }
        p.ev_pool.push_back(ev);
    }
    if (p.ev_stage.size() < i + 1) p.ev_stage.resize(i + 1);
    p.ev_stage[i] = stage;
    cudaEventRecord(p.ev_pool[2 * i], st);
}

void prof_end(Plan &p, cudaStream_t st) {
    if (!p.profiling) return;
    cudaEventRecord(p.ev_pool[2 * p.ev_used + 1], st);
    p.ev_used++;
}

int collect_profile(Plan &p) {
    for (size_t i = 0; i < p.ev_used; ++i) {
        cudaError_t e = cudaEventSynchronize(p.ev_pool[2 * i + 1]);
        if (e) return cuda_fail(e, "profiling event");
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, p.ev_pool[2 * i], p.ev_pool[2 * i + 1]);
        if (e) return cuda_fail(e, "profiling event");
        p.prof_ms[p.ev_stage[i]] += ms;
    }
    p.ev_used = 0;
    return AAHRT_OK;
}

}  // namespace aahrt
