/*
 * aahrt.h -- C ABI of the GB300 azimuthally anisotropic hyperbolic Radon
 * transform (AAHRT) library, libaahrt.so.
 *
 * The operator (Sec. 3 of Mokhtari & Gholami, "Fast Azimuthally Anisotropic
 * 3D Radon Transform by Generalized Fourier Slice Theorem"):
 *
 *   d = L m,   L = S^{-1} F1^{-1} P F2 S                       (eq. axb2)
 *
 * maps a Radon model m(tau, q, theta) -- intercept time, curvature
 * q = squared slowness, azimuth -- to a CMP cube d(t, trace) through the
 * hyperbolic basis of eq. Inverse, computed by Algorithm 1 (time stretch
 * t' = t^2, FFT, Fourier slice k_q = f' r^2 / theta = atan(y/x) of eq.
 * inv_GFST, inverse FFT, stretch undone).  aahrt_adjoint applies the exact
 * transpose L^T (the velocity stack of Sec. 3.2 / Algorithm 2, built as a
 * true transpose of every stage) and aahrt_sparse_solve minimises
 * 1/2||d - L m||^2 + lambda ||m||_1 (eq. cost1) by forward-backward splitting
 * (eq. ISTA with the shrinkage of eq. soft), optionally with FISTA momentum.
 *
 * Discretisation (fixed at plan creation):
 *   tau_i = i*dt (i < ntau), t_i = i*dt (i < nt), q_l = q0 + l*dq (l < nq;
 *   or explicit values, opts.q_axis),
 *   theta_j = j*pi/ntheta (j < ntheta); a trace at offset (hx, hy) has
 *   r^2 = hx^2 + hy^2 and axial azimuth atan2(hy, hx) mod pi, and reads the
 *   two neighbouring azimuth slices with linear weights (theta factors of
 *   eq. thli).  Stretched time is sampled inside an FFT frame of Nfft samples
 *   (Nfft = power of two >= sigma_t*nt*(1+rho), rho = |q|max r^2max/tmax^2),
 *   bins 0..K (K = Nfft/2-1, Nyquist excluded).  The DFT along q read at the
 *   non-uniform k_q is evaluated by an exponential-of-semicircle spreading
 *   kernel of `spread_width` taps on a 2x-or-more oversampled q grid (the
 *   paper's step 3 uses linear interpolation; this is its accurate form).
 *
 * Memory layout (all float32, caller-owned):
 *   model  m[g][tau][q][theta]   theta fastest, g = gather (ngather > 1) or
 *                                cube (batched plans), each block contiguous
 *   data   d[g][t][trace]        trace fastest
 * The model and data buffers of aahrt_forward, aahrt_adjoint and
 * aahrt_sparse_solve may be device memory (16-byte aligned) or host memory
 * (pinned or pageable, 4-byte aligned); host buffers are copied through
 * device staging buffers the plan allocates on first use, inside the call's
 * stream order (with pageable memory the copies synchronise the host).
 * Spectra of aahrt_apply_stage must be device memory.  Buffers of one call
 * must not overlap.  Every call is stream-ordered on `stream` (a
 * cudaStream_t; NULL is the legacy default stream) and returns without
 * synchronising, except where stated.  The plan's workspace is reused by
 * every call: calls on one plan must be serialised on one stream (or
 * ordered by the caller).
 *
 * Errors: every int-returning function returns AAHRT_OK (0) or a negative
 * AAHRT_ERR_* code; no function exits, throws or traps.  The text of the
 * most recent error of the calling thread is aahrt_last_error().
 */
#ifndef AAHRT_H
#define AAHRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status */
#define AAHRT_OK 0
#define AAHRT_ERR_INVALID_ARG -1   /* bad size, pointer, alignment or option */
#define AAHRT_ERR_OOM -2           /* device or host allocation failed */
#define AAHRT_ERR_CUDA -3          /* a CUDA runtime call or launch failed */
#define AAHRT_ERR_UNSUPPORTED -4   /* valid request this build cannot serve */
#define AAHRT_ERR_TIMEOUT -5       /* a bounded device wait ran out */
#define AAHRT_ERR_NONFINITE -6     /* NaN/Inf met where a finite value is needed */

#define AAHRT_INTERP_KEYS 0        /* Keys cubic convolution, a = -1/2 (default) */
#define AAHRT_INTERP_LINEAR 1      /* linear interpolation */

/* Slice-step arithmetic.
 * AAHRT_PRECISION_FP32: the non-uniform DFT along q by an exponential-of-
 *   semicircle spreading kernel on an oversampled q grid, FP32 on the CUDA
 *   cores (about 2e-6 relative to the exact operator).
 * AAHRT_PRECISION_SPLIT_BF16: for ngather gathers on one geometry (plans of
 *   aahrt_plan_create; ngather <= 64, nq <= 256), the slice step of every bin
 *   and azimuth slice is a direct complex contraction over q (traces) with
 *   the exact phases exp(-+2 pi i f_k q_l r^2), run on the tensor cores with
 *   every FP32 operand split into two bf16 parts (three products, FP32
 *   accumulation; about 1e-5 relative).  Its model and data buffers hold the
 *   gathers fastest: m[tau][q][theta][g], d[t][trace][g]. */
/* Slice-step interpolation of the FP32 path.
 * AAHRT_SLICE_SPREAD: exponential-of-semicircle spreading kernel with
 *   deapodisation (the accurate non-uniform DFT along q, default).
 * AAHRT_SLICE_LINEAR_K: the paper's own step 3 (A-coefficients of eq. thli):
 *   FFT of the centred, zero-padded q columns and linear interpolation
 *   between the two neighbouring k samples, no deapodisation (second-order
 *   in the k spacing: about 30 % error at sigma_q = 1, 8 % at 2 on smooth
 *   events; see the design notes).  The adjoint is its exact transpose. */
/* AAHRT_SLICE_DIRECT: the DFT along q summed directly at k_q = f_k r^2
 *   with exact phases (64-bit fixed-point phase arguments, FP32 sums on the
 *   CUDA cores; about 1e-6 relative): O(nq) work per bin and trace instead
 *   of the spreading kernel's O(W), for any curvature axis.  Plans with an
 *   explicit opts.q_axis always use it (slice_interp 0 or 2). */
#define AAHRT_SLICE_SPREAD 0
#define AAHRT_SLICE_LINEAR_K 1
#define AAHRT_SLICE_DIRECT 2

#define AAHRT_PRECISION_FP32 0
#define AAHRT_PRECISION_SPLIT_BF16 1

typedef struct aahrt_plan aahrt_plan;

/* Axes and trace geometry of one CMP cube.  hx, hy: host arrays of ntr
 * offsets in metres, copied at plan creation (the caller keeps ownership).
 * dt in seconds, q0 and dq in s^2/m^2.  Requires nt >= 4, ntau >= 4,
 * nq >= 1, ntheta >= 1, ntr >= 1, dt > 0, dq > 0 when nq > 1 (q0 and dq are
 * not read when opts.q_axis is given), and at least one nonzero offset. */
typedef struct {
    int nt;
    double dt;
    int ntau;
    int nq;
    double q0;
    double dq;
    int ntheta;
    int ntr;
    const double *hx;
    const double *hy;
} aahrt_geom;

/* Options; a zero-initialised struct selects every default. */
typedef struct {
    int interp_kind;    /* AAHRT_INTERP_KEYS (0) or AAHRT_INTERP_LINEAR */
    int spread_width;   /* q-spreading kernel taps, 4..12; 0 = smallest width
                           with ~1e-6 spreading error for the plan's q
                           oversampling (7 at 2x, 6 at 2.56x) */
    int theta_group;    /* azimuth slices per slice-kernel block; 0 = automatic */
    int ngather;        /* gathers sharing this geometry; 0 = 1 */
    double sigma_t;     /* FFT frame oversampling of the time axis; 0 = 2 */
    double fmax;        /* highest kept stretched frequency in 1/s^2; 0 = all */
    int time_pairs;     /* column pairs per time-kernel block (1, 2, 4 or 8);
                           0 = automatic (8192 / Nfft clamped to [2, 8] up to
                           Nfft = 8192, 1 beyond) */
    int autotune;       /* 1: pick spread_width, theta_group and time_pairs
                           at plan creation (see aahrt_plan_create); fields
                           set explicitly above are kept */
    int precision;      /* AAHRT_PRECISION_FP32 (0) or AAHRT_PRECISION_SPLIT_BF16 */
    int slice_interp;   /* AAHRT_SLICE_SPREAD (0) or AAHRT_SLICE_LINEAR_K */
    double sigma_q;     /* q grid oversampling: the grid has max(16,
                           next_pow2(ceil(sigma_q nq))) points; 0 = 2; the
                           spreading kernel needs >= 1.25 nq points */
    const double *q_axis;  /* NULL: the uniform axis q_l = q0 + l dq of the
                           geometry.  Else a host array of nq finite
                           curvatures in s^2/m^2 (any order, copied; q0 and
                           dq are then ignored), for instance the uniform-
                           slowness axis of aahrt_q_axis_slowness: the slice
                           step is the direct sum over these q_l (a type-3
                           DFT along q; AAHRT_SLICE_DIRECT, or the tensor-core
                           contraction).  Not available with
                           AAHRT_SLICE_LINEAR_K or the pull scan. */
    double r2max;       /* largest squared offset (m^2) the stretched-time
                           plan is sized for (Sec. 3.4's no-wrap padding,
                           through rho = |q|max r2max / tmax^2); 0 = the
                           geometry's own.  A cube planned alone with the
                           r2max of a batch gets the batch's time plan (Nfft,
                           Ns, ds) and so the same operator.  Values below the
                           geometry's own are refused (AAHRT_ERR_INVALID_ARG). */
} aahrt_opts;

/* What a plan chose (filled by aahrt_plan_query). */
typedef struct {
    int nfft;           /* FFT frame length along stretched time */
    int ns;             /* stretched samples s_n = n*ds, n < ns */
    int nbins;          /* kept frequency bins K+1 */
    int nq_os;          /* oversampled q grid of the spreading kernel */
    int spread_width;
    int theta_group;
    int ncube;          /* cubes of a batched plan (1 otherwise) */
    int ngather;
    double ds;          /* stretched sampling interval, s^2 */
    double rho;         /* |q|max r^2max / tmax^2 */
    double beta;        /* spreading kernel shape parameter */
    long long model_len;     /* floats of one m buffer (all gathers/cubes) */
    long long data_len;      /* floats of one d buffer */
    long long xspec_len;     /* complex values of a model spectrum X[g][k][q][theta] */
    long long yspec_len;     /* complex values of a data spectrum Y[g][k][trace] */
    long long workspace_bytes;
    int time_pairs;          /* column pairs per time-kernel block */
    int autotuned;           /* 1 if the autotuner chose the tiles above */
    double tune_ms;          /* autotuner: best forward+adjoint time of its trial batch */
    int precision;           /* AAHRT_PRECISION_* of the slice step */
    int slice_interp;        /* AAHRT_SLICE_* the FP32 slice step runs */
} aahrt_plan_info;

/* Create a plan on the current CUDA device: validates the geometry,
 * computes the stretched-time sampling (Sec. 3.4, steps 1-2) and the trace
 * azimuth binning (eq. thli), and allocates the device workspace.  With
 * opts->ngather = G > 1 the plan serves G gathers on this one geometry,
 * stored back to back in m and d.  On success *out owns device memory until
 * aahrt_plan_destroy.
 *
 * Autotuning (opts->autotune = 1; not part of the paper's method): the
 * spreading width is the smallest whose measured forward error against the
 * widest kernel (12 taps) on a seeded random model stays below 2e-6
 * relative, then every candidate (theta_group, time_pairs) pair is built and
 * timed (median of 3 forward+adjoint pairs, CUDA events) on a trial batch of
 * at most 16 of the cubes or gathers, and the fastest is kept.  Explicitly
 * set fields are not tuned.  Tuning synchronises the device and needs room
 * for two plans of the trial batch at once. */
int aahrt_plan_create(aahrt_plan **out, const aahrt_geom *geom,
                      const aahrt_opts *opts);

/* Create one plan for ncube independent CMP cubes of different fold and
 * azimuth coverage.  All cubes must share nt, dt, ntau, nq, q0, dq (unless
 * opts.q_axis gives the axis) and ntheta; they share one stretched-time sampling built from the largest
 * offset of the whole batch.  m holds the cubes' models back to back,
 * d their data back to back (cube c has geoms[c].ntr traces). */
int aahrt_plan_create_batched(aahrt_plan **out, int ncube,
                              const aahrt_geom *geoms, const aahrt_opts *opts);

void aahrt_plan_destroy(aahrt_plan *plan);

int aahrt_plan_query(const aahrt_plan *plan, aahrt_plan_info *info);

/* d = L m (Algorithm 1; eq. axb2).  m: model_len floats, d: data_len floats,
 * both device memory; d is overwritten. */
int aahrt_forward(aahrt_plan *plan, const float *m, float *d, void *stream);

/* m = L^T d, the exact transpose of aahrt_forward (Sec. 3.2 / Algorithm 2
 * as a true adjoint).  m is overwritten. */
int aahrt_adjoint(aahrt_plan *plan, const float *d, float *m, void *stream);

/* One stage of the operator pair on caller buffers (for stage-by-stage
 * checks and custom pipelines).  Spectra are interleaved complex float32
 * (re, im), bins k = 0..nbins-1 with f_k = k/(nfft*ds):
 *   stage 0  X = F S m          m (model_len) -> X (xspec_len), X[g][k][q][theta]
 *   stage 1  Y = P X / nfft     X -> Y (yspec_len), Y[g][k][trace]  (Fourier slice)
 *   stage 2  d = U H Y          Y -> d (data_len)
 *   stage 3  Y = F U^T d        d -> Y
 *   stage 4  X = P^H Y / nfft   Y -> X  (exact transpose of stage 1)
 *   stage 5  m = S^T H X        X -> m
 * F: DFT along stretched time (Alg. 1 step 2); H: band-limited Hermitian
 * synthesis x_n = Re X_0 + 2 Re sum_{k>=1} X_k e^{+2 pi i k n/nfft} (so
 * H/nfft is the paper's F1^{-1}, step 4); S, U: the stretch and its undoing
 * (steps 1 and 5).  forward = 2 o 1 o 0, adjoint = 5 o 4 o 3.
 * Plans of AAHRT_PRECISION_SPLIT_BF16 keep their spectra slice-major with
 * the gathers fastest: X[theta][k][q][g] and Y[j][k][i][g], where block j
 * holds the traces whose first azimuth slice is j (i = rank of the trace
 * among them, in input order). */
int aahrt_apply_stage(aahrt_plan *plan, int stage, const void *in, void *out,
                      void *stream);

/* Options of the sparse solve; zero-initialised = defaults. */
typedef struct {
    int ista;            /* 0 (default): FISTA momentum; 1: plain ISTA (eq. ISTA) */
    int warm_start;      /* 1: m holds the starting model on entry; else m0 = 0 */
    int power_iters;     /* power iterations for gamma when gamma <= 0; 0 = 30 */
    int use_graph;       /* 1: capture the iterations in a CUDA graph; 0 = eager */
    double gamma;        /* step length; <= 0: 0.95 / (power estimate of ||L||^2) */
    double lambda_rel;   /* > 0: lambda = lambda_rel * max|L^T d| (lambda ignored) */
    int per_cube;        /* 1: every cube of a batched plan (every gather of a
                            multi-gather plan) is an independent problem with
                            its own step and threshold; the power iteration
                            and max|L^T d| are then taken per cube */
    double *cube_gamma;  /* per_cube: NULL or host array [ncube]; entries > 0 are
                            used as that cube's step, the others (and all when
                            NULL, or when gamma > 0: gamma for every cube) are
                            estimated; on return holds the steps used */
    double *cube_lambda; /* per_cube: NULL or host array [ncube]; on entry the
                            cube's lambda (lambda_rel > 0 overrides), on return
                            the lambda used; NULL: lambda (or lambda_rel) for all */
} aahrt_solve_opts;

typedef struct {
    int iters;           /* iterations run */
    double gamma;        /* step length used */
    double lambda;       /* lambda used */
    double resid_norm;   /* ||d - L m||_2 of the result, FP64 accumulation */
    double l1_norm;      /* ||m||_1 of the result */
    double objective;    /* 1/2 resid_norm^2 + lambda * l1_norm */
} aahrt_solve_info;

/* Sparse Radon transform (eq. cost1): iters iterations of
 *   m <- soft(z + gamma L^T (d - L z), gamma*lambda)   (eqs. ISTA, soft)
 * with z = m (ISTA) or the FISTA extrapolation of m.  d: data_len floats;
 * m: model_len floats, in/out.  opts and info may be NULL.  When info is
 * non-NULL, gamma/lambda must be estimated, or per_cube is set, the call
 * synchronises the stream.  For batched and multi-gather plans one gamma and
 * one lambda serve every cube unless opts->per_cube is set; then info holds
 * cube 0's gamma and lambda, the residual and l1 norms over all cubes and
 * the sum of the cubes' objectives. */
int aahrt_sparse_solve(aahrt_plan *plan, const float *d, float lambda,
                       int iters, float *m, const aahrt_solve_opts *opts,
                       aahrt_solve_info *info, void *stream);

/* A regular offset grid: trace ix * ny + iy sits at (x0 + ix dx, y0 + iy dy). */
typedef struct {
    int nx, ny;
    double x0, dx, y0, dy;
} aahrt_grid;

/* The paper's own velocity scan (Algorithm 2 with the B-coefficients of
 * Sec. 3.4), for data recorded on a regular offset grid: the data time axis
 * is stretched by interpolation and FFT'd; at every bin f' and azimuth slice
 * theta_j the spectrum is read by bilinear interpolation at
 * (x, y) = +-sqrt(k/f') (cos theta_j, sin theta_j) for every q-grid
 * wavenumber k (all alias rings k + n/dq that stay inside the grid; both
 * antipodal points, no Jacobian factor, bin 0 set to zero), inverse-DFT'd
 * along k onto the q axis (centred on q_c = q0 + (nq/2) dq, with the phase
 * exp(+2 pi i k q_c)), synthesised along f' (1/Nfft) and unstretched.  It is
 * the paper's approximation of the velocity stack, not L^T (compare
 * aahrt_adjoint).  The plan: single gather, AAHRT_PRECISION_FP32, ntau == nt,
 * nq >= 2, ntr == nx * ny (its own offsets set only the stretched-time
 * sampling); the q grid has nq_os points (opts.sigma_q).  d: data_len floats
 * in grid trace order; m: model_len floats.  Device memory, stream-ordered;
 * uses the plan's spectra workspace. */
int aahrt_velocity_scan_grid(aahrt_plan *plan, const aahrt_grid *grid,
                             const float *d, float *m, void *stream);

/* Automatic anisotropic velocity picking (Sec. 3.3, eq. vel_est): for a
 * Radon model m (model_len floats, the plan's layout) writes, at every
 * (tau, theta) of every cube or gather, the squared-slowness estimate
 *   q_hat = sum_l q_l |m(tau, q_l, theta)| / sum_l |m(tau, q_l, theta)|
 * (v^-2; the paper's ratio of q-moments with |m| as weights) and, when
 * weight is non-NULL, the weight sum_l |m| (q_hat = 0 where it is 0).
 * q_hat and weight hold model_len / nq floats: [g][tau][theta], or
 * [tau][theta][g] for AAHRT_PRECISION_SPLIT_BF16 plans.  Device memory,
 * 16-byte aligned; FP64 accumulation; stream-ordered. */
int aahrt_pick_velocity(aahrt_plan *plan, const float *m, float *q_hat,
                        float *weight, void *stream);

/* Deconvolutive AAHRT (Sec. 4, eq. DecRT): after this call the plan's
 * operator is W L, W the linear convolution of every trace with the wavelet
 * in time (the band-limited wavelet replaces the Dirac pulse of the basis
 * functions), truncated to the trace length:
 *   (W x)[i] = sum_s w[s] x[i - s + center],  x = 0 outside [0, nt),
 * and the adjoint L^T W^T.  aahrt_forward, aahrt_adjoint, aahrt_sparse_solve,
 * aahrt_fista_vjp and aahrt_forward_noalloc all use it; aahrt_apply_stage
 * does not.  w: host array of nw (1..4096) finite samples, center in
 * [0, nw); nw = 0 restores the plain operator.  Synchronises the device
 * (allocates the wavelet and a data-sized workspace on first use). */
int aahrt_plan_set_wavelet(aahrt_plan *plan, const float *w, int nw, int center);

/* Derivative of the unrolled sparse solve (configuration of Sec. 4 used as a
 * differentiable layer).  With m^n(d) the result of `iters` iterations of
 * aahrt_sparse_solve from m^0 = 0 at the given gamma and lambda (FISTA, or
 * ISTA when ista != 0), computes the vector-Jacobian product
 *   d_bar = (d m^n / d d)^T m_bar
 * and, when m_out is non-NULL, m^n itself.  The shrinkage of eq. soft has
 * slope 1 where |z + gamma g| > gamma*lambda and 0 elsewhere (its kink is
 * given slope 0).  gamma (> 0) and lambda (>= 0) are fixed inputs here:
 * their estimation from d (power iteration, lambda_rel) is not
 * differentiated.  The forward iterates are checkpointed every `checkpoint`
 * iterations (<= 0: 10) and each segment is recomputed before its reverse
 * sweep, so one call costs about 3*iters operator pairs and holds
 * 2*ceil(iters/checkpoint) + checkpoint + 6 model-sized buffers and one
 * data-sized buffer of plan-owned workspace (grown on demand, freed with the
 * plan; growing it synchronises the device).
 * d (data_len), m_bar (model_len), d_bar (data_len) and m_out (model_len):
 * device memory, 16-byte aligned, not overlapping.  Stream-ordered, no
 * synchronisation otherwise. */
int aahrt_fista_vjp(aahrt_plan *plan, const float *d, const float *m_bar,
                    float lambda, float gamma, int iters, int ista,
                    int checkpoint, float *m_out, float *d_bar, void *stream);

/* Uniform curvature axis for a slowness range: q0 = pmin^2 and
 * dq = (pmax^2 - pmin^2)/(nq - 1) (curvature is squared slowness, Sec. 2). */
int aahrt_q_from_slowness(double pmin, double pmax, int nq, double *q0,
                          double *dq);

/* Uniform-slowness curvature axis (non-uniform in q): q[l] = p_l^2 with
 * p_l = pmin + l (pmax - pmin)/(nq - 1) (p_0 = pmin when nq = 1), for
 * opts.q_axis.  q: host array of nq doubles.  Requires finite pmin, pmax
 * and nq >= 1. */
int aahrt_q_axis_slowness(double pmin, double pmax, int nq, double *q);

/* Curvature sampling bound of Sec. 3.5 (eqs. q1-q3).  k_q = f' r^2 is never
 * negative, so a uniform q step dq reads it without aliasing over a whole
 * period 1/dq when dq <= 1/(fmax r2max); a range of width span (2 q_max for
 * the paper's axis [-q_max, q_max], eq. q3) then needs
 *   *nq = max(1, ceil(span fmax r2max))
 * samples.  fmax: highest stretched-time frequency inverted (1/s^2; a plan's
 * is (nbins - 1)/(nfft ds)), r2max: largest squared offset (m^2).  A partial
 * NMO by q_ref = (q_a + q_b)/2 (aahrt_partial_nmo) turns a range [q_a, q_b]
 * into one of width q_b - q_a centred on zero.  Requires span, fmax,
 * r2max >= 0 and finite, and a count below 2^31. */
int aahrt_nq_required(double span, double fmax, double r2max, int *nq);

/* Partial NMO of the data by a reference curvature q_ref (Sec. 3.5): in
 * stretched time s = t^2 every trace is shifted by -q_ref r^2, which moves a
 * hyperbola of curvature q to q - q_ref; it is applied on the time axis in
 * one resampling with the plan's interpolation kernel:
 *   out(t_i, h) = sum_taps c(u - n) in(t_n, h),  u = sqrt(t_i^2 + q_ref r_h^2)/dt,
 * zero where t_i^2 + q_ref r_h^2 < 0 and taps outside [0, nt) taken as 0.
 * transpose = 1 applies the exact transpose of that map instead (a gather
 * over the output samples whose taps reach each input sample; no atomics).
 * The inverse of the map is the map with -q_ref (up to interpolation and the
 * muted zone).  in and out: data_len floats of device memory in the plan's
 * data layout (every trace of every cube or gather), 16-byte aligned, not
 * overlapping.  q_ref must be finite.  Stream-ordered. */
int aahrt_partial_nmo(aahrt_plan *plan, const float *in, float *out, double q_ref,
                      int transpose, void *stream);

/* Per-stage device time.  While profiling is on, every stage launch of the
 * plan is bracketed by CUDA events on its stream and, at
 * aahrt_plan_stage_times (which synchronises on those events), the elapsed
 * milliseconds are summed per stage:
 *   0 stretch+FFT (model side)   1 Fourier slice forward
 *   2 inverse FFT+unstretch      3 unstretch^T+FFT (data side)
 *   4 Fourier slice adjoint      5 inverse FFT+stretch^T
 *   6 solver updates and norms
 * times_ms[7] and launches[7] receive the totals since profiling was
 * turned on (either may be NULL).  Turning profiling on clears them. */
#define AAHRT_NSTAGES 7
int aahrt_plan_set_profiling(aahrt_plan *plan, int on);
int aahrt_plan_stage_times(aahrt_plan *plan, double *times_ms,
                           long long *launches);

/* d = L m like aahrt_forward, for callers that must not allocate device
 * memory during the call (for example code whose device heap is owned by an
 * external memory manager, or loops that forbid allocation on their hot
 * path).  The paper has no counterpart: it concerns memory management only.
 * Scratch (spectra and a work counter) comes from one array of
 * AAHRT_NOALLOC_SCRATCH_BYTES in device memory, shared by all plans and held
 * on every device it was committed on until the process exits; the call
 * allocates nothing.  The array is committed, and its address looked up
 * (cudaGetSymbolAddress), when a plan is created on a device
 * (aahrt_plan_create / aahrt_plan_create_batched, which fail if that fails):
 * the call itself loads nothing.  After a cudaDeviceReset, create a new plan
 * before calling this again (old plans are invalid after a reset).  m and d
 * must be device memory.  Plans whose spectra need more than the array
 * (aahrt_plan_info xspec_len + yspec_len complex values, plus 256 bytes) get
 * AAHRT_ERR_UNSUPPORTED.  Every call shares the array, which keeps the last
 * call's contents; calls whose kernels overlap on the GPU race on it and
 * must be serialised. */
#define AAHRT_NOALLOC_SCRATCH_BYTES (16u << 20)
int aahrt_forward_noalloc(aahrt_plan *plan, const float *m, float *d, void *stream);

/* Synchronises the plan's device and reports device-side failures of its
 * kernels since the last call: AAHRT_ERR_TIMEOUT if a tensor-core kernel
 * gave up waiting for its matrix unit (every such wait is bounded by 1 s of
 * device time; the kernel then releases its tensor memory and returns, its
 * output incomplete), else AAHRT_OK.  The flag is cleared. */
int aahrt_plan_status(aahrt_plan *plan);

/* Test hook for the failure path above: while on, the plan's tensor-core
 * kernels issue no matrix operations, so their bounded waits run out (after
 * 20 ms of device time instead of the normal 1 s limit), the kernels record
 * the timeout, release their tensor memory and return, and the next
 * aahrt_plan_status reports AAHRT_ERR_TIMEOUT.  Outputs computed meanwhile
 * are invalid.  Plans of other precisions get AAHRT_ERR_UNSUPPORTED.  Not for
 * production use. */
int aahrt_plan_test_stall(aahrt_plan *plan, int on);

const char *aahrt_status_string(int status);
const char *aahrt_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* AAHRT_H */
