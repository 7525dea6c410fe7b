// Internal structures of libaahrt: plan, device tables and stage launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "aahrt.h"
#include "slice_math.cuh"

namespace aahrt {

constexpr int kThreadsTime = 256;
constexpr int kMaxThreadsTime = 512;
// dynamic shared memory of a time-kernel block up to which two blocks fit on
// one SM (228 KB per SM, 1 KB reserved per block, 512 bytes static)
constexpr int kTimeSmemTwoBlocks = 112 * 1024;
constexpr int kThreadsSlice = 256;
constexpr int kMinW = 4;
constexpr int kMaxW = 12;
constexpr int kMaxGroupSlices = 256;   // azimuth slices one slice-kernel block may own

// One trace, in azimuth-sorted order within its cube (32 bytes).
//   A: phase per frequency bin, 0.64 fixed point of frac((q0 + cq*dq) r^2 / (Nfft ds))
//   B: q-grid position per bin, 0.64 fixed point of frac(dq r^2 / (Nfft ds))
// so that bin k has phase frac(k*A) and position frac(k*B) (exact modular
// integer products; no floating-point range reduction on the device).
struct TraceGeo {
    unsigned long long A;
    unsigned long long B;
    float w0, w1;     // weights of slices j0 and (j0 + 1) mod ntheta
    int j0;           // first azimuth slice
    int col;          // trace index within its cube = data column
};
static_assert(sizeof(TraceGeo) == 32, "TraceGeo must be 32 bytes");

// Work unit of the slice kernels: one cube and one group of azimuth slices
// (all bins of the unit are separate work items).
struct SliceGroup {
    long long geo_off;  // first TraceGeo of the cube
    long long x_off;    // complex offset of the cube's X[k][q][theta] block
    long long y_off;    // complex offset of the cube's Y[k][trace] block
    int ntr;            // traces of the cube (Y row length)
    int ja, nj;         // owned slices [ja, ja + nj)
    int f0, f1;         // traces with j0 in the owned slices
    int e0, e1;         // traces with j0 == ja - 1 (mod ntheta), adjoint only
    long long ss_off;   // offset of the cube's slice-start table (ntheta + 1 ints)
    int cube;           // cube index (row of the spectrum bound tables)
};

// Data block of the partial NMO: nt rows of ld floats starting at float
// offset off; column c of a row belongs to trace r0 + c / rep (rep = gathers
// stored fastest, else 1).
struct PnBlock {
    long long off;
    long long r0;
    int ld;
    int rep;
};

// Column group of the time-axis kernels (at most 2*pairs columns).
struct ColGroup {
    long long real_off;  // float offset of the group's first column in the
                         // real (time-domain) array, row 0
    long long spec_off;  // complex offset of its first column in the spectrum
    int ld_real, ld_spec;  // row strides (elements)
    int ncol;
    int cube;            // cube (or gather) the columns belong to
};

// Resampler tables.  Output row o of the stretch S (or its undoing U) sits
// at position fl + fr of the input axis; the transposed operator reads, for
// output o, the contiguous source rows lo .. lo + cnt - 1.
struct RowPos {
    int fl;
    float fr;
};
struct RowRange {
    int lo;
    int cnt;
};
struct DevResampler {
    const RowPos *pos;      // per output row (S, U) or per source row (S^T, U^T)
    const RowRange *rng;    // per output row of a transposed operator, else null
    int nrows;              // output rows
    int npos;               // entries of pos
};

enum C2REpilogue { EPI_STORE = 0, EPI_RESIDUAL = 1, EPI_FISTA = 2 };

struct FistaArgs {
    float *m;        // current iterate (in/out)
    float *z;        // extrapolated point (in/out)
    float gamma;
    float thresh;    // gamma * lambda
    float beta;      // momentum weight (t_k - 1)/t_{k+1}
    const float2 *cube_gt;   // per-cube (gamma, thresh) overriding the two above, or null
};

// x * max(1 - t/|x|, 0) of eq. soft, written without the division
__device__ __forceinline__ float soft_threshold(float x, float t) {
    return copysignf(fmaxf(fabsf(x) - t, 0.f), x);
}

struct Plan {
    int device = 0;
    // axes
    int nt = 0, ntau = 0, nq = 0, ntheta = 0;
    double dt = 0, q0 = 0, dq = 0;
    int interp = AAHRT_INTERP_KEYS;
    int w = 7;
    double sigma_t = 2.0, fmax = 0.0;
    int ncube = 1;          // cubes (independent geometries or gathers)
    int ngather = 1;        // gathers per distinct geometry
    std::vector<int> ntr;   // traces per cube
    std::vector<long long> data_off;   // float offset of cube c in d
    long long ntr_total = 0;
    // stretched-time plan
    double tmax = 0, rho = 0, ds = 0;
    int nfft = 0, L = 0, ns = 0, kmax = 0, nbins = 0;
    int pairs = 1;          // column pairs per time-kernel block
    // q spreading
    int nos = 0, Lq = 0, cq = 0;
    double beta = 0;
    int tgroup = 0, ngroup = 1;   // slices per group, groups per cube
    long long model_len = 0, data_len = 0, cols_model = 0;
    // device tables
    float2 *tw_t = nullptr, *tw_q = nullptr;
    float *dec = nullptr;
    TraceGeo *geo = nullptr;
    SliceGroup *groups = nullptr;
    int *slice_start = nullptr;    // per distinct geometry: first sorted trace of each slice
    TraceGeo *geo_adj = nullptr;   // the same traces in the adjoint slice kernel's order
    // Amplitude bound of the data spectrum for the adjoint spread's
    // fixed-point scale: ymax[cube][chunk] = max |re| + |im| of Y over the
    // chunk's 2^ychunk_log bins (float bits; written by the data-side
    // analysis that produces Y, cleared before it), and wsum[cube][j] = the
    // total azimuth weight of the traces that reach slice j.
    unsigned *ymax = nullptr;
    float *wsum = nullptr;
    int nychunk = 0, ychunk_log = 6;
    int ngroups_total = 0;
    long long slice_items = 0;
    int *counters = nullptr;       // work counters of the persistent kernels
    ColGroup *cg_model = nullptr, *cg_data = nullptr;
    // the same column groups over column-blocked arrays [group][row][2*pairs]
    // (the solver's internal state), every group's rows one contiguous slab
    ColGroup *cg_model_blk = nullptr, *cg_data_blk = nullptr;
    int ncg_model = 0, ncg_data = 0;
    long long mblk_len = 0, dblk_len = 0;
    RowPos *posS = nullptr, *posU = nullptr;       // resampler tables
    RowRange *rngST = nullptr, *rngUT = nullptr;
    DevResampler S{}, ST{}, U{}, UT{};
    EsPoly poly{};                 // Horner coefficients of the spreading kernel
    double phimax = 0;             // bound on sum_i phi_i over positions
    int lp = 0;                    // log2(pairs)
    int slice_grid_fwd = 0, slice_grid_adj = 0;
    size_t smem_r2c_model = 0, smem_r2c_data = 0, smem_c2r_model = 0, smem_c2r_data = 0;
    size_t smem_sfwd = 0, smem_sadj = 0;
    size_t smem_fused_model = 0;   // fused model half-iteration (0: not available)
    size_t smem_fused_data = 0;    // fused data half-iteration (0: not available)
    // workspace
    float2 *X = nullptr, *Y = nullptr;
    long long x_len = 0, y_len = 0;
    // solver workspace (allocated on first solve)
    float *z = nullptr, *r = nullptr, *v = nullptr;
    float *zb = nullptr, *mb = nullptr, *rb = nullptr, *db = nullptr;   // column-blocked
    double *scal = nullptr;        // device scalars of the solver
    float *stage_m = nullptr, *stage_d = nullptr;   // staging of host buffers
    float *vjp_ws = nullptr;       // workspace of the unrolled-solve derivative
    size_t vjp_bytes = 0;
    float2 *cube_gt = nullptr;     // per-cube (gamma, gamma*lambda) of a per-cube solve
    double *cube_acc = nullptr;    // per-cube FP64 accumulators [slot][ncube]
    long long *dseg = nullptr;     // data offsets of the cubes (ncube + 1 entries)
    // tensor-core direct contraction (precision 1): gathers stored fastest
    int precision = 0;
    int slice_interp = 0;          // AAHRT_SLICE_SPREAD, _LINEAR_K or _DIRECT
    // curvature axis: q_l = qc + qn[l] * qeps exactly (qn integer); the
    // uniform axis has qc = q0 + cq dq, qeps = dq, qn[l] = l - cq
    bool qexplicit = false;        // opts.q_axis given (non-uniform q)
    std::vector<double> qaxis;     // q_l (host)
    double qc = 0, qeps = 0;
    long long *qn = nullptr;       // device [nq]
    double *qv = nullptr;          // device [nq], q_l
    int direct_chunk = 0;          // traces the direct adjoint stages per pass
    // partial NMO: data blocks and per-trace r^2 / dt^2
    PnBlock *pn_blk = nullptr;
    int pn_nblk = 0, pn_ldmax = 0;
    double *pn_rho = nullptr;      // [traces of every distinct geometry]
    float2 *pn_c = nullptr;        // per trace q_ref r^2/dt^2 as (hi, lo)
    long long pn_ntr = 0;
    int tc_gp = 0;                 // gathers padded to a multiple of 8
    int4 *tc_tiles = nullptr;      // forward row tiles {slice, first, end, 0}
    bool tc_stall = false;         // test hook: tensor-core kernels issue no MMAs
    int tc_ntiles = 0;
    // deconvolutive operator: wavelet convolved with every trace in time
    float *wav = nullptr;          // nw samples (device)
    int nw = 0, wcenter = 0;
    int wav_gen = 0;               // bumped whenever the wavelet changes
    float *wtmp = nullptr;         // data-sized workspace of the convolution
    // tiles
    bool autotuned = false;
    double tune_ms = 0;
    // cached graph of the last solve
    cudaGraphExec_t gexec = nullptr;
    std::string gkey;
    long long glaunches = 0;
    long long gstage[AAHRT_NSTAGES] = {0};   // its launches per stage
    // accounting
    long long launches[AAHRT_NSTAGES] = {0};
    bool profiling = false;
    double prof_ms[AAHRT_NSTAGES] = {0};
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> ev_stage;     // stage of pending pair i (events 2i, 2i+1)
    size_t ev_used = 0;
    long long bytes = 0;
};

// Raise a kernel's dynamic shared memory limit to what the device allows
// beside the kernel's static shared memory.
template <typename F>
inline cudaError_t raise_smem_limit(F *func, int max_smem) {
    cudaFuncAttributes at;
    cudaError_t e = cudaFuncGetAttributes(&at, func);
    if (e) return e;
    return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                max_smem - (int)at.sharedSizeBytes);
}

// error state
int set_error(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

// stage launchers (stream-ordered, no synchronisation)
cudaError_t launch_r2c(Plan &p, bool model_side, const float *in, float2 *out,
                       cudaStream_t st, bool blocked = false);
cudaError_t launch_c2r(Plan &p, bool model_side, const float2 *in, float *out,
                       int epi, const float *aux, FistaArgs fa, cudaStream_t st,
                       bool blocked = false);
cudaError_t launch_slice(Plan &p, bool adjoint, const float2 *in, float2 *out,
                         cudaStream_t st, int *counter = nullptr);
// fused synthesis + analysis of one FISTA half-iteration (column-blocked state)
cudaError_t launch_c2r_r2c(Plan &p, bool model_side, float2 *spec, const float *aux,
                           FistaArgs fa, cudaStream_t st);
cudaError_t launch_slice_tc(Plan &p, bool adjoint, const float2 *in, float2 *out,
                            cudaStream_t st, int *counter);
// direct sum of the DFT along q (any curvature axis)
cudaError_t launch_slice_direct(Plan &p, bool adjoint, const float2 *in, float2 *out,
                                cudaStream_t st, int *counter);
cudaError_t configure_direct_kernels(Plan &p, int num_sms, int max_smem);
size_t direct_smem_fwd(int tgroup, int extra, int nq);
size_t direct_smem_adj(int tgroup, int nq, int chunk);
cudaError_t configure_tc_kernels(Plan &p, int num_sms, int max_smem);
// time convolution of the data columns with the plan's wavelet: mode 0 out = W in,
// 1 out = aux - W in, 2 out = W^T in
cudaError_t launch_wavelet(Plan &p, int mode, const float *in, float *out, const float *aux,
                           cudaStream_t st, bool blocked);
// device error flag of the tensor-core kernels (a timed-out wait), in Plan::counters
constexpr int kTcErrSlot = 8;

// profiling brackets around a stage launch
void prof_begin(Plan &p, int stage, cudaStream_t st);
void prof_end(Plan &p, cudaStream_t st);

// pointer checks of the C ABI
int check_dev_ptr(const void *ptr, const char *name);

// Makes the plan's device current for the scope of a C entry point.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// Resolves and caches the allocation-free forward's scratch address on
// device `dev` (current); called at plan creation (noalloc.cu).
int noalloc_prepare(int dev);

// Spectrum bound table of the slice adjoint computed from a given Y (when Y
// does not come from the data-side analysis, which writes the table itself).
cudaError_t launch_ybound(Plan &p, const float2 *Y, cudaStream_t st);

// operator application used by the C ABI and the solver
int apply_forward(Plan &p, const float *m, float *d, cudaStream_t st,
                  int epi = EPI_STORE, const float *dobs = nullptr, bool blocked = false);
int apply_adjoint(Plan &p, const float *d, float *m, cudaStream_t st,
                  int epi = EPI_STORE, FistaArgs fa = FistaArgs{}, bool blocked = false);

}  // namespace aahrt

// The opaque handle of the C ABI.
struct aahrt_plan {
    aahrt::Plan *p;
};
