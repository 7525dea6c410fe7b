// Plan construction of libaahrt: stretched-time sampling (Sec. 3.4 steps 1-2,
// eq. q3), azimuth binning of the traces (theta factors of eq. thli),
// resampler tables of the stretch S and its undoing U (Sec. 3.4: a local
// "spline" interpolation; here Keys' cubic convolution or linear), the
// spreading kernel of the q-slice, device workspace and work lists.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <vector>

#include "fft.cuh"
#include "internal.cuh"

namespace aahrt {

cudaError_t set_time_kernel_attrs(int lp, int interp, int max_smem);
cudaError_t configure_slice_kernels(Plan &p, int num_sms, int max_smem);

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

// Position of every output row of a resampler on its input axis.
static std::vector<RowPos> row_positions(const std::vector<double> &pos) {
    std::vector<RowPos> out(pos.size());
    for (size_t o = 0; o < pos.size(); ++o) {
        const double fl = std::floor(pos[o]);
        out[o].fl = (int)fl;
        out[o].fr = (float)(pos[o] - fl);
    }
    return out;
}

// Source ranges of the transpose: output o of the transpose collects every
// row r whose taps fl_r + t (t in [t0, t0 + ntap), inside [0, n_out)) include
// o.  Since fl_r is non-decreasing, the sources are contiguous and come in
// segments of decreasing t; the segment of tap t0 + q holds (cnt >> 8q) & 255
// rows.  Returns false if a range is not contiguous or a segment exceeds 255.
static bool transpose_ranges(const std::vector<RowPos> &pos, int n_out, int interp,
                             std::vector<RowRange> *rng) {
    const int t0 = interp == AAHRT_INTERP_KEYS ? -1 : 0;
    const int ntap = interp == AAHRT_INTERP_KEYS ? 4 : 2;
    std::vector<int> lo(n_out, 0), last(n_out, -2), total(n_out, 0);
    std::vector<std::array<int, 4>> seg(n_out, std::array<int, 4>{0, 0, 0, 0});
    for (int r = 0; r < (int)pos.size(); ++r)
        for (int q = 0; q < ntap; ++q) {
            const int o = pos[r].fl + t0 + q;
            if (o < 0 || o >= n_out) continue;
            if (total[o] == 0) lo[o] = r;
            else if (r != last[o] + 1) return false;
            last[o] = r;
            total[o]++;
            seg[o][q]++;
        }
    rng->resize(n_out);
    for (int o = 0; o < n_out; ++o) {
        unsigned packed = 0;
        for (int q = 0; q < ntap; ++q) {
            if (seg[o][q] > 255) return false;
            packed |= (unsigned)seg[o][q] << (8 * q);
        }
        (*rng)[o] = RowRange{lo[o], (int)packed};
    }
    return true;
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
    std::vector<TraceGeo> sorted;      // by slice, then r^2 (forward order)
    std::vector<TraceGeo> sorted_adj;  // by slice, then trace index (adjoint order)
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
        t.A = to_fixed64(p.qc * r2 * scale);
        t.B = to_fixed64(p.qeps * r2 * scale);
        t.w0 = (float)(1.0 - fr);
        t.w1 = (float)fr;
        t.j0 = j;
        t.col = h;
        tr[h] = t;
    }
    // Traces grouped by azimuth slice.  The forward slice kernel reads them
    // sorted by r^2 inside a slice: a trace's grid position at bin k is
    // frac(k B) with B ~ r^2, so one warp's consecutive traces read nearby or
    // evenly stepped grid points (broadcasts and fewer bank conflicts).  The
    // adjoint's atomics prefer the opposite (nearby positions collide on the
    // same words), so it gets the slices in the traces' own order.  Neither
    // order changes a result: each trace is independent in the forward, and
    // the adjoint's fixed-point sums are exact.
    std::vector<double> r2v(ntr);
    for (int h = 0; h < ntr; ++h) r2v[h] = hx[h] * hx[h] + hy[h] * hy[h];
    std::vector<int> idx(ntr);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
        return tr[a].j0 != tr[b].j0 ? tr[a].j0 < tr[b].j0 : r2v[a] < r2v[b];
    });
    g.start.assign(p.ntheta + 1, 0);
    for (int i = 0; i < ntr; ++i) g.start[tr[idx[i]].j0 + 1]++;
    for (int j = 0; j < p.ntheta; ++j) g.start[j + 1] += g.start[j];
    g.sorted.resize(ntr);
    for (int i = 0; i < ntr; ++i) g.sorted[i] = tr[idx[i]];
    std::vector<int> ida(ntr);
    std::iota(ida.begin(), ida.end(), 0);
    std::stable_sort(ida.begin(), ida.end(), [&](int a, int b) { return tr[a].j0 < tr[b].j0; });
    g.sorted_adj.resize(ntr);
    for (int i = 0; i < ntr; ++i) g.sorted_adj[i] = tr[ida[i]];
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
    void *ptrs[] = {p->tw_t, p->tw_q, p->dec, p->geo, p->groups, p->slice_start, p->counters,
                    p->cg_model, p->cg_data, p->cg_model_blk, p->cg_data_blk, p->posS,
                    p->posU, p->rngST, p->rngUT, p->X, p->Y, p->z, p->r, p->v, p->scal,
                    p->stage_m, p->stage_d, p->zb, p->mb, p->rb, p->db, p->vjp_ws,
                    p->cube_gt, p->cube_acc, p->dseg, p->tc_tiles, p->wav, p->wtmp,
                    p->qn, p->qv, p->pn_blk, p->pn_rho, p->pn_c, p->ymax, p->wsum,
                    p->geo_adj};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    cudaSetDevice(cur);
    delete p;
}

static int validate_geom(const aahrt_geom *g, int idx, bool q_explicit) {
    if (!g) return set_error(AAHRT_ERR_INVALID_ARG, "geometry %d is NULL", idx);
    if (g->nt < 4 || g->ntau < 4)
        return set_error(AAHRT_ERR_INVALID_ARG, "geometry %d: nt and ntau must be >= 4", idx);
    if (g->nq < 1 || g->ntheta < 1 || g->ntr < 1)
        return set_error(AAHRT_ERR_INVALID_ARG, "geometry %d: nq, ntheta, ntr must be >= 1", idx);
    if (!(g->dt > 0.0) || !std::isfinite(g->dt))
        return set_error(AAHRT_ERR_INVALID_ARG, "geometry %d: dt must be > 0", idx);
    if (!q_explicit &&
        (!std::isfinite(g->q0) || !std::isfinite(g->dq) || (g->nq > 1 && !(g->dq > 0.0))))
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
        int rc = validate_geom(geoms + c, c, opts.q_axis != nullptr);
        if (rc) return rc;
    }
    const aahrt_geom &g0 = geoms[0];
    for (int c = 1; c < ndist; ++c) {
        const aahrt_geom &g = geoms[c];
        const bool qdiff = opts.q_axis == nullptr && (g.q0 != g0.q0 || g.dq != g0.dq);
        if (g.nt != g0.nt || g.dt != g0.dt || g.ntau != g0.ntau || g.nq != g0.nq || qdiff ||
            g.ntheta != g0.ntheta)
            return set_error(AAHRT_ERR_INVALID_ARG,
                             "cube %d: axes differ from cube 0 (nt, dt, ntau, nq, q0, dq, "
                             "ntheta must be shared)", c);
    }
    if (opts.interp_kind != AAHRT_INTERP_KEYS && opts.interp_kind != AAHRT_INTERP_LINEAR)
        return set_error(AAHRT_ERR_INVALID_ARG, "interp_kind must be 0 or 1");
    int W = opts.spread_width;
    const bool lineark = opts.slice_interp == AAHRT_SLICE_LINEAR_K;
    if (opts.slice_interp != AAHRT_SLICE_SPREAD && !lineark &&
        opts.slice_interp != AAHRT_SLICE_DIRECT)
        return set_error(AAHRT_ERR_INVALID_ARG, "slice_interp must be 0, 1 or 2");
    const bool qexplicit = opts.q_axis != nullptr;
    if (qexplicit) {
        for (int l = 0; l < g0.nq; ++l)
            if (!std::isfinite(opts.q_axis[l]))
                return set_error(AAHRT_ERR_NONFINITE, "q_axis[%d] is not finite", l);
        if (lineark)
            return set_error(AAHRT_ERR_UNSUPPORTED, "the k-interpolation needs a uniform q "
                             "axis (FFT along q)");
    }
    if (lineark) {
        if (W != 0 && W != 2)
            return set_error(AAHRT_ERR_INVALID_ARG, "linear k-interpolation has 2 taps");
        W = 2;
    } else if (W != 0 && (W < kMinW || W > kMaxW)) {
        return set_error(AAHRT_ERR_INVALID_ARG, "spread_width must be in [%d, %d]", kMinW, kMaxW);
    }
    if (!(opts.sigma_q == 0.0 || (opts.sigma_q >= 1.0 && opts.sigma_q <= 16.0)))
        return set_error(AAHRT_ERR_INVALID_ARG, "sigma_q must be 0 (default 2) or in [1, 16]");
    if (opts.sigma_t < 0.0 || (opts.sigma_t > 0.0 && opts.sigma_t < 1.0))
        return set_error(AAHRT_ERR_INVALID_ARG, "sigma_t must be 0 (default) or >= 1");
    if (opts.fmax < 0.0 || opts.theta_group < 0 || opts.ngather < 0)
        return set_error(AAHRT_ERR_INVALID_ARG, "fmax, theta_group, ngather must be >= 0");
    if (opts.time_pairs != 0 && opts.time_pairs != 1 && opts.time_pairs != 2 &&
        opts.time_pairs != 4 && opts.time_pairs != 8)
        return set_error(AAHRT_ERR_INVALID_ARG, "time_pairs must be 0, 1, 2, 4 or 8");
    if (opts.precision != AAHRT_PRECISION_FP32 && opts.precision != AAHRT_PRECISION_SPLIT_BF16)
        return set_error(AAHRT_ERR_INVALID_ARG, "precision must be 0 or 1");
    // the tensor-core contraction serves gathers on one geometry, stored
    // gather-fastest: internally one cube whose columns are (column, gather)
    const bool tc = opts.precision == AAHRT_PRECISION_SPLIT_BF16;
    const int G_tc = tc ? ncube : 1;
    if (tc) {
        if (ndist != 1)
            return set_error(AAHRT_ERR_UNSUPPORTED,
                             "the tensor-core contraction needs gathers on one geometry");
        if (G_tc > 64 || g0.nq > 256)
            return set_error(AAHRT_ERR_UNSUPPORTED,
                             "the tensor-core contraction supports ngather <= 64, nq <= 256");
        if (lineark)
            return set_error(AAHRT_ERR_UNSUPPORTED,
                             "the tensor-core contraction evaluates the exact DFT along q");
        ncube = 1;
    }

    Plan *p = new Plan();
    cudaGetDevice(&p->device);
    p->nt = g0.nt;
    p->dt = g0.dt;
    p->ntau = g0.ntau;
    p->nq = g0.nq;
    p->q0 = qexplicit ? 0.0 : g0.q0;
    p->dq = (qexplicit || g0.nq < 2) ? 0.0 : g0.dq;
    p->ntheta = g0.ntheta;
    p->interp = opts.interp_kind;
    p->sigma_t = opts.sigma_t > 0.0 ? opts.sigma_t : 2.0;
    p->fmax = opts.fmax;
    p->ncube = ncube;
    p->ngather = tc ? G_tc : (ndist == 1 ? ncube : 1);
    p->precision = opts.precision;
    p->tc_gp = tc ? (G_tc + 7) / 8 * 8 : 0;

    // ---------------------------------------------------- stretched time
    double r2max = 0.0;
    for (int c = 0; c < ndist; ++c)
        for (int h = 0; h < geoms[c].ntr; ++h)
            r2max = std::max(r2max, geoms[c].hx[h] * geoms[c].hx[h] + geoms[c].hy[h] * geoms[c].hy[h]);
    if (opts.r2max != 0.0) {
        if (!(opts.r2max >= r2max) || !std::isfinite(opts.r2max)) {
            free_plan(p);
            return set_error(AAHRT_ERR_INVALID_ARG,
                             "opts.r2max %g is below the geometry's largest squared offset %g",
                             opts.r2max, r2max);
        }
        r2max = opts.r2max;
    }
    if (!(r2max > 0.0)) {
        free_plan(p);
        return set_error(AAHRT_ERR_INVALID_ARG, "all offsets are zero");
    }
    int rc_fail = AAHRT_OK;
    p->tmax = (p->nt - 1) * p->dt;
    if (qexplicit) {
        p->qexplicit = true;
        p->qaxis.assign(opts.q_axis, opts.q_axis + p->nq);
    } else {
        p->qaxis.resize(p->nq);
        for (int l = 0; l < p->nq; ++l) p->qaxis[l] = p->q0 + l * p->dq;
    }
    double qabs = 0.0;
    for (int l = 0; l < p->nq; ++l) qabs = std::max(qabs, std::fabs(p->qaxis[l]));
    p->rho = qabs * r2max / (p->tmax * p->tmax);
    const double want = std::ceil(p->sigma_t * p->nt * (1.0 + p->rho));
    if (!(want <= 16384.0)) {
        rc_fail = set_error(AAHRT_ERR_UNSUPPORTED,
                            "FFT frame of %.0f samples or more exceeds 16384 (nt = %d, rho = %g)",
                            want, p->nt, p->rho);
        free_plan(p);
        return rc_fail;
    }
    p->nfft = (int)next_pow2((long long)want);
    p->L = ilog2(p->nfft);
    p->ns = (int)std::floor((p->nfft - 2) / (1.0 + p->rho)) + 1;
    p->ds = p->tmax * p->tmax / (p->ns - 1);
    p->kmax = p->nfft / 2 - 1;
    if (p->fmax > 0.0)
        p->kmax = std::min(p->kmax, (int)std::floor(p->fmax * p->nfft * p->ds));
    p->nbins = p->kmax + 1;
    // column pairs per time block: 8192 / Nfft, at least 2 up to Nfft = 8192
    // (two pairs write whole 32-byte sectors of gathers-fastest spectra) when
    // their shared memory fits the device, 1 beyond
    p->pairs = opts.time_pairs > 0 ? opts.time_pairs
                                   : (p->nfft <= 8192 ? std::max(2, std::min(8, 8192 / p->nfft)) : 1);
    if (opts.time_pairs == 0 && p->pairs == 2 && 8192 / p->nfft < 2) {
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
        const size_t fftb2 = 2 * (size_t)ld_interleaved(p->nfft) * sizeof(float2);
        const size_t need = fftb2 + (size_t)std::max(p->ntau, p->nt) * 4 * sizeof(float) +
                            (size_t)std::max(p->ns, p->nt) * sizeof(float);
        if (need > (size_t)optin) p->pairs = 1;
    }
    p->lp = ilog2(p->pairs);

    // ----------------------------------------------------- q spreading
    const double sq = opts.sigma_q > 0.0 ? opts.sigma_q : 2.0;
    p->nos = (int)std::max(16LL, next_pow2((long long)std::ceil(sq * p->nq - 1e-9)));
    p->Lq = ilog2(p->nos);
    p->cq = p->nq / 2;
    p->slice_interp = (qexplicit && !tc) ? AAHRT_SLICE_DIRECT : opts.slice_interp;
    if (tc) p->slice_interp = AAHRT_SLICE_SPREAD;
    const bool direct = p->slice_interp == AAHRT_SLICE_DIRECT;
    // the curvature axis as q_c + n_l eps with integers n_l: the uniform axis
    // centred at l = cq, or an explicit one centred on its range with a
    // quantum eps of 2^-30 of its half-width (n_l exact to half a quantum)
    std::vector<long long> qn(p->nq);
    if (!qexplicit) {
        p->qc = p->q0 + p->cq * p->dq;
        p->qeps = p->dq;
        for (int l = 0; l < p->nq; ++l) qn[l] = l - p->cq;
    } else {
        const auto mm = std::minmax_element(p->qaxis.begin(), p->qaxis.end());
        p->qc = 0.5 * (*mm.first + *mm.second);
        const double half = 0.5 * (*mm.second - *mm.first);
        p->qeps = half > 0.0 ? std::ldexp(half, -30) : 1.0;
        for (int l = 0; l < p->nq; ++l)
            qn[l] = std::llround((p->qaxis[l] - p->qc) / p->qeps);
    }
    const double sigma_q = (double)p->nos / p->nq;
    if (!lineark && !direct && !tc && sigma_q < 1.25) {
        rc_fail = set_error(AAHRT_ERR_UNSUPPORTED, "the spreading kernel needs a q grid of at "
                            "least 1.25 nq points (sigma_q)");
        free_plan(p);
        return rc_fail;
    }
    if (W == 0) {
        // smallest width whose spreading error exp(-pi W sqrt(1 - 1/sigma))
        // is below 1e-6 (about 2e-6 measured for sigma = 2..2.6)
        W = (int)std::ceil(-std::log(1e-6) / (M_PI * std::sqrt(1.0 - 1.0 / sigma_q)));
        W = std::max(kMinW + 1, std::min(kMaxW, W));
    }
    p->w = W;
    p->beta = 0.97 * M_PI * W * (1.0 - 1.0 / (2.0 * sigma_q));
    std::vector<float> dec(p->nq);
    for (int l = 0; l < p->nq; ++l)
        dec[l] = lineark ? 1.0f
                         : (float)(1.0 / es_fourier((double)(l - p->cq) / p->nos, p->beta, W));

    // --------------------------------------------------- azimuth groups
    const size_t per_slice = (size_t)std::max(ld_interleaved(p->nos), ld_split(p->nos)) *
                             sizeof(float2);
    if (opts.theta_group > 0) {
        p->tgroup = std::min(opts.theta_group, p->ntheta);
    } else if (direct) {
        // the forward stages nq x (slices + 1) values, the adjoint two planes
        // of nq x slices accumulators beside its staged traces (32 bytes each)
        const int by_fwd = (int)(64 * 1024 / ((size_t)p->nq * sizeof(float2))) - 1;
        const int by_adj = (int)(48 * 1024 / (2 * (size_t)p->nq * sizeof(float2)));
        const int t = std::max(1, std::min(by_fwd, by_adj));
        const int ng = (p->ntheta + t - 1) / t;
        p->tgroup = (p->ntheta + ng - 1) / ng;
    } else {
        const size_t budget = 72 * 1024;      // three blocks per SM
        if (p->ntheta * per_slice <= budget) {
            p->tgroup = p->ntheta;
        } else {
            int t = (int)(budget / per_slice) - 1;
            if (t < 1) t = 1;
            const int ng = (p->ntheta + t - 1) / t;
            p->tgroup = (p->ntheta + ng - 1) / ng;
        }
    }
    if (p->tgroup > kMaxGroupSlices) p->tgroup = kMaxGroupSlices;
    p->ngroup = (p->ntheta + p->tgroup - 1) / p->tgroup;
    if (p->ngroup == 1) p->tgroup = p->ntheta;

    // ------------------------------------------------ per-cube geometry
    std::vector<CubeGeo> cg(ndist);
    for (int c = 0; c < ndist; ++c) cg[c] = bin_cube(*p, geoms[c].hx, geoms[c].hy, geoms[c].ntr);
    std::vector<long long> geo_off(ndist, 0);
    std::vector<TraceGeo> geo_all, geo_adj_all;
    std::vector<int> ss_all;
    for (int c = 0; c < ndist; ++c) {
        geo_off[c] = (long long)geo_all.size();
        geo_all.insert(geo_all.end(), cg[c].sorted.begin(), cg[c].sorted.end());
        geo_adj_all.insert(geo_adj_all.end(), cg[c].sorted_adj.begin(), cg[c].sorted_adj.end());
        ss_all.insert(ss_all.end(), cg[c].start.begin(), cg[c].start.end());
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
    p->model_len = (long long)ncube * p->ntau * C * G_tc;
    p->data_len = acc_tr * p->nt * G_tc;
    p->x_len = (long long)ncube * p->nbins * C * G_tc;
    p->y_len = acc_tr * p->nbins * G_tc;

    std::vector<SliceGroup> groups;
    for (int c = 0; c < ncube; ++c) {
        const int dc = ndist == 1 ? 0 : c;
        const CubeGeo &G = cg[dc];
        for (int gi = 0; gi < p->ngroup; ++gi) {
            SliceGroup s;
            s.cube = c;
            s.geo_off = geo_off[dc];
            s.ss_off = (long long)dc * (p->ntheta + 1);
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
    if (tc) {
        // Real columns (q, theta, gather) and (trace, gather), gather fastest;
        // spectra slice-major, X[j][k][l][g] and Y[j][k][i][g] (i = the trace's
        // rank inside slice j), so each (bin, slice) block is contiguous.  A
        // column group never straddles two (q, theta) or two traces.
        const int G = G_tc, J = p->ntheta, nq = p->nq;
        const long long nb = p->nbins;
        for (int l = 0; l < nq; ++l)
            for (int j = 0; j < J; ++j)
                for (int g0 = 0; g0 < G; g0 += cpg)
                    cgm.push_back(ColGroup{((long long)l * J + j) * G + g0,
                                           ((long long)j * nb * nq + l) * G + g0,
                                           (int)(C * G), nq * G, std::min(cpg, G - g0), 0});
        const CubeGeo &cg0 = cg[0];
        std::vector<int> rank(p->ntr[0]), slice(p->ntr[0]);
        for (int j = 0; j < J; ++j)
            for (int t = cg0.start[j]; t < cg0.start[j + 1]; ++t) {
                rank[cg0.sorted[t].col] = t - cg0.start[j];
                slice[cg0.sorted[t].col] = j;
            }
        for (int h = 0; h < p->ntr[0]; ++h) {
            const int j = slice[h];
            const int cnt = cg0.start[j + 1] - cg0.start[j];
            for (int g0 = 0; g0 < G; g0 += cpg)
                cgd.push_back(ColGroup{(long long)h * G + g0,
                                       (nb * cg0.start[j] + rank[h]) * G + g0,
                                       p->ntr[0] * G, cnt * G, std::min(cpg, G - g0), 0});
        }
    }
    for (int c = 0; c < (tc ? 0 : ncube); ++c)
        for (long long c0 = 0; c0 < C; c0 += cpg) {
            ColGroup q;
            q.real_off = (long long)c * p->ntau * C + c0;
            q.spec_off = (long long)c * p->nbins * C + c0;
            q.ld_real = (int)C;
            q.ld_spec = (int)C;
            q.ncol = (int)std::min<long long>(cpg, C - c0);
            q.cube = c;
            cgm.push_back(q);
        }
    for (int c = 0; c < (tc ? 0 : ncube); ++c)
        for (int h0 = 0; h0 < p->ntr[c]; h0 += cpg) {
            ColGroup q;
            q.real_off = p->data_off[c] + h0;
            q.spec_off = y_off[c] + h0;
            q.ld_real = p->ntr[c];
            q.ld_spec = p->ntr[c];
            q.ncol = std::min(cpg, p->ntr[c] - h0);
            q.cube = c;
            cgd.push_back(q);
        }
    p->ncg_model = (int)cgm.size();
    p->ncg_data = (int)cgd.size();
    std::vector<ColGroup> cgmb = cgm, cgdb = cgd;
    for (size_t gi = 0; gi < cgmb.size(); ++gi) {
        cgmb[gi].real_off = (long long)gi * p->ntau * cpg;
        cgmb[gi].ld_real = cpg;
    }
    for (size_t gi = 0; gi < cgdb.size(); ++gi) {
        cgdb[gi].real_off = (long long)gi * p->nt * cpg;
        cgdb[gi].ld_real = cpg;
    }
    p->mblk_len = (long long)p->ncg_model * p->ntau * cpg;
    p->dblk_len = (long long)p->ncg_data * p->nt * cpg;

    // ------------------------------------------------------ resamplers
    std::vector<double> upos(p->ns), vpos(p->nt);
    for (int n = 0; n < p->ns; ++n) upos[n] = std::sqrt(n * p->ds) / p->dt;
    for (int i = 0; i < p->nt; ++i) vpos[i] = (i * p->dt) * (i * p->dt) / p->ds;
    const std::vector<RowPos> posS = row_positions(upos), posU = row_positions(vpos);
    std::vector<RowRange> rngST, rngUT;
    if (!transpose_ranges(posS, p->ntau, p->interp, &rngST) ||
        !transpose_ranges(posU, p->ns, p->interp, &rngUT)) {
        rc_fail = set_error(AAHRT_ERR_UNSUPPORTED, "resampler transpose is not banded");
        free_plan(p);
        return rc_fail;
    }
    if (lineark) {
        // two taps at grid points u0, u0 + 1 with g = a - 1/2: 1/2 - g and 1/2 + g
        std::memset(&p->poly, 0, sizeof p->poly);
        p->poly.c[0][0] = 0.5f;
        p->poly.c[1][0] = -1.0f;
        p->poly.c[0][1] = 0.5f;
        p->poly.c[1][1] = 1.0f;
    } else {
        fit_es_poly(W, p->beta, &p->poly);
    }
    {   // bound on the summed kernel weights of one trace, with margin
        double mx = 0.0;
        for (int s = 0; s <= 2000; ++s) {
            const double g = -0.5 + s / 2000.0;
            double sum = 0.0;
            for (int i = 0; i < W; ++i) {
                double v = 0.0;
                for (int d = W + 1; d >= 0; --d) v = v * g + p->poly.c[d][i];
                sum += std::fabs(v);
            }
            mx = std::max(mx, sum);
        }
        p->phimax = 1.05 * mx;
    }

    // ------------------------------------------------------- twiddles
    auto twiddles = [](int N) {
        std::vector<float2> tw(std::max(1, N));
        for (int m = 0; m < N; ++m) {
            const double a = -2.0 * M_PI * m / N;
            tw[m] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
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
    AAHRT_TRY(upload(&p->geo_adj, geo_adj_all), "upload geometry");
    AAHRT_TRY(upload(&p->groups, groups), "upload work list");
    AAHRT_TRY(upload(&p->slice_start, ss_all), "upload slice table");
    if (!tc) {
        // spectrum bound tables of the adjoint spread (see ymax, wsum)
        p->ychunk_log = 6;
        while ((p->nbins >> p->ychunk_log) > 128) ++p->ychunk_log;
        p->nychunk = (p->nbins + (1 << p->ychunk_log) - 1) >> p->ychunk_log;
        std::vector<float> ws((size_t)ncube * p->ntheta);
        for (int c = 0; c < ncube; ++c) {
            const CubeGeo &G = cg[ndist == 1 ? 0 : c];
            std::vector<double> acc(p->ntheta, 0.0);
            for (const TraceGeo &t : G.sorted) {
                acc[t.j0] += t.w0;
                acc[(t.j0 + 1) % p->ntheta] += t.w1;
            }
            for (int j = 0; j < p->ntheta; ++j)   // rounded up: a bound
                ws[(size_t)c * p->ntheta + j] = (float)(acc[j] * (1.0 + 1e-6));
        }
        AAHRT_TRY(upload(&p->wsum, ws), "upload slice weights");
        AAHRT_TRY(cudaMalloc((void **)&p->ymax, (size_t)ncube * p->nychunk * sizeof(unsigned)),
                  "alloc spectrum bound");
        AAHRT_TRY(cudaMemset(p->ymax, 0, (size_t)ncube * p->nychunk * sizeof(unsigned)),
                  "clear spectrum bound");
    }
    AAHRT_TRY(upload(&p->cg_model, cgm), "upload column groups");
    AAHRT_TRY(upload(&p->cg_data, cgd), "upload column groups");
    AAHRT_TRY(upload(&p->cg_model_blk, cgmb), "upload column groups");
    AAHRT_TRY(upload(&p->cg_data_blk, cgdb), "upload column groups");
    AAHRT_TRY(upload(&p->posS, posS), "upload resamplers");
    AAHRT_TRY(upload(&p->posU, posU), "upload resamplers");
    AAHRT_TRY(upload(&p->rngST, rngST), "upload resamplers");
    AAHRT_TRY(upload(&p->rngUT, rngUT), "upload resamplers");
    AAHRT_TRY(upload(&p->qn, qn), "upload curvature axis");
    AAHRT_TRY(upload(&p->qv, p->qaxis), "upload curvature axis");
    {   // partial NMO: data blocks and r^2/dt^2 of every trace of every geometry
        std::vector<PnBlock> blk;
        std::vector<double> rho;
        std::vector<long long> r0(ndist);
        for (int c = 0; c < ndist; ++c) {
            r0[c] = (long long)rho.size();
            for (int h = 0; h < geoms[c].ntr; ++h)
                rho.push_back((geoms[c].hx[h] * geoms[c].hx[h] + geoms[c].hy[h] * geoms[c].hy[h]) /
                              (p->dt * p->dt));
        }
        if (tc) {
            blk.push_back(PnBlock{0, 0, geoms[0].ntr * G_tc, G_tc});
        } else {
            for (int c = 0; c < ncube; ++c)
                blk.push_back(PnBlock{p->data_off[c], r0[ndist == 1 ? 0 : c], p->ntr[c], 1});
        }
        p->pn_nblk = (int)blk.size();
        p->pn_ldmax = 0;
        for (const PnBlock &b : blk) p->pn_ldmax = std::max(p->pn_ldmax, b.ld);
        p->pn_ntr = (long long)rho.size();
        AAHRT_TRY(upload(&p->pn_blk, blk), "upload data blocks");
        AAHRT_TRY(upload(&p->pn_rho, rho), "upload offsets");
        AAHRT_TRY(cudaMalloc((void **)&p->pn_c, rho.size() * sizeof(float2)), "alloc offsets");
    }
    AAHRT_TRY(cudaMalloc((void **)&p->counters, 16 * sizeof(int)), "alloc counters");
    AAHRT_TRY(cudaMemset(p->counters, 0, 16 * sizeof(int)), "clear counters");
    p->S = DevResampler{p->posS, nullptr, p->ns, p->ns};
    p->ST = DevResampler{p->posS, p->rngST, p->ntau, p->ns};
    p->U = DevResampler{p->posU, nullptr, p->nt, p->nt};
    p->UT = DevResampler{p->posU, p->rngUT, p->ns, p->nt};
    AAHRT_TRY(cudaMalloc((void **)&p->X, std::max<long long>(1, p->x_len) * sizeof(float2)),
              "alloc X workspace");
    AAHRT_TRY(cudaMalloc((void **)&p->Y, std::max<long long>(1, p->y_len) * sizeof(float2)),
              "alloc Y workspace");

    const size_t fftb = (size_t)p->pairs * ld_interleaved(p->nfft) * sizeof(float2);
    p->smem_r2c_model = fftb + (size_t)p->ntau * 2 * p->pairs * sizeof(float);
    p->smem_r2c_data = fftb + (size_t)p->nt * 2 * p->pairs * sizeof(float) +
                       (size_t)p->nt * sizeof(float);
    p->smem_c2r_data = fftb;
    p->smem_c2r_model = fftb + (size_t)p->ns * sizeof(float);
    // fused FISTA half-iterations: the synthesis' source fractions (S^T has
    // ns of them) beside the analysis' staged rows
    p->smem_fused_model = p->smem_r2c_model + (size_t)p->ns * sizeof(float);
    p->smem_fused_data = p->smem_r2c_data;
    const size_t smem_r2c = std::max(p->smem_r2c_model, p->smem_r2c_data);
    const size_t smem_c2r = std::max(p->smem_c2r_model, p->smem_c2r_data);
    if (direct) {
        int most = 32;
        for (const SliceGroup &s : groups) most = std::max(most, s.f1 - s.f0 + s.e1 - s.e0);
        const size_t base = direct_smem_adj(p->tgroup, p->nq, 0);
        const size_t budget = 72 * 1024;
        const int room = base < budget ? (int)((budget - base) / 32) : 0;
        p->direct_chunk = std::max(64, std::min(most, room));
        p->smem_sfwd = direct_smem_fwd(p->tgroup, p->ngroup > 1 ? 1 : 0, p->nq);
        p->smem_sadj = direct_smem_adj(p->tgroup, p->nq, p->direct_chunk);
    } else {
        p->smem_sfwd = (size_t)(p->tgroup + (p->ngroup > 1 ? 1 : 0)) * ld_interleaved(p->nos) *
                       sizeof(float2);
        p->smem_sadj = (size_t)p->tgroup * ld_split(p->nos) * 2 * sizeof(float);
    }
    int max_smem = 0;
    AAHRT_TRY(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                     p->device), "device query");
    // the time kernels hold 512 bytes of static shared memory (the spectrum
    // bound of the data-side unpack) beside their dynamic buffers
    const int max_time = max_smem - 512;
    if ((int)smem_r2c > max_time || (int)smem_c2r > max_time || (int)p->smem_sfwd > max_smem ||
        (int)p->smem_sadj > max_smem) {
        rc_fail = set_error(AAHRT_ERR_UNSUPPORTED,
                            "shared memory per block (%zu / %zu bytes) exceeds %d; lower "
                            "theta_group or time_pairs", smem_r2c, p->smem_sfwd, max_smem);
        free_plan(p);
        return rc_fail;
    }
    if ((int)p->smem_fused_model > max_time) p->smem_fused_model = 0;
    if ((int)p->smem_fused_data > max_time) p->smem_fused_data = 0;
    // The dynamic shared memory limit is a property of each kernel function,
    // shared by every plan of the process: raise it to the device maximum once
    // so no plan lowers it under another.
    AAHRT_TRY(set_time_kernel_attrs(p->lp, p->interp, max_smem), "kernel attributes");
    if (tc) {
        std::vector<int4> tiles;
        for (int j = 0; j < p->ntheta; ++j)
            for (int t0 = ss_all[j]; t0 < ss_all[j + 1]; t0 += 128)
                tiles.push_back(make_int4(j, t0, std::min(t0 + 128, ss_all[j + 1]), 0));
        p->tc_ntiles = (int)tiles.size();
        AAHRT_TRY(upload(&p->tc_tiles, tiles), "upload row tiles");
        AAHRT_TRY(configure_tc_kernels(*p, num_sms, max_smem), "tensor-core kernel configuration");
    } else if (direct) {
        AAHRT_TRY(configure_direct_kernels(*p, num_sms, max_smem), "direct kernel configuration");
    } else {
        AAHRT_TRY(configure_slice_kernels(*p, num_sms, max_smem), "slice kernel configuration");
    }
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
    info->time_pairs = p.pairs;
    info->autotuned = p.autotuned ? 1 : 0;
    info->tune_ms = p.tune_ms;
    info->precision = p.precision;
    info->slice_interp = p.slice_interp;
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
