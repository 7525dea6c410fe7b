// Plan autotuner (not part of the paper's method): chooses the spreading
// width by measured accuracy and the slice/time kernel tiles by measured time
// on a trial batch of the plan's cubes, then builds the full plan with them.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace aahrt {

int build_plan(Plan **out, int ncube, int ndist, const aahrt_geom *geoms,
               const aahrt_opts *opts);
void free_plan(Plan *p);

namespace {

// x[i] = uniform in [-1, 1) from a 64-bit integer hash of (seed, i)
// (the finaliser of the SplitMix64 generator).
__global__ void fill_random_kernel(float *x, long long n, unsigned long long seed) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        x[i] = (float)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
    }
}

// acc[0] += sum (a - b)^2, acc[1] += sum b^2
__global__ void diff_norm_kernel(const float *__restrict__ a, const float *__restrict__ b,
                                 long long n, double *acc) {
    double s0 = 0.0, s1 = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double d = (double)a[i] - (double)b[i];
        s0 += d * d;
        s1 += (double)b[i] * b[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc, s0);
        atomicAdd(acc + 1, s1);
    }
}

int grid_for(long long n) {
    return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 8));
}

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
};

struct Trial {
    int ncube, ndist;
    std::vector<aahrt_geom> geoms;
};

// At most 16 cubes, evenly spaced, always including the cube with the largest
// offset (it fixes the stretched-time frame of the whole batch).
Trial trial_batch(int ncube, int ndist, const aahrt_geom *geoms) {
    Trial t;
    const int nt = std::min(ncube, 16);
    if (ndist == 1) {
        t.ncube = nt;
        t.ndist = 1;
        t.geoms.push_back(geoms[0]);
        return t;
    }
    int cmax = 0;
    double r2max = -1.0;
    for (int c = 0; c < ncube; ++c)
        for (int h = 0; h < geoms[c].ntr; ++h) {
            const double r2 = geoms[c].hx[h] * geoms[c].hx[h] + geoms[c].hy[h] * geoms[c].hy[h];
            if (r2 > r2max) { r2max = r2; cmax = c; }
        }
    std::vector<int> pick;
    for (int i = 0; i < nt; ++i) pick.push_back((int)((long long)i * ncube / nt));
    if (std::find(pick.begin(), pick.end(), cmax) == pick.end()) pick.back() = cmax;
    std::sort(pick.begin(), pick.end());
    pick.erase(std::unique(pick.begin(), pick.end()), pick.end());
    for (int c : pick) t.geoms.push_back(geoms[c]);
    t.ncube = t.ndist = (int)t.geoms.size();
    return t;
}

// Median time (ms) of 3 forward+adjoint pairs after one warm-up pair.
int time_pair(Plan &p, const float *m, float *d, float *g, cudaStream_t st, double *ms) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) || cudaEventCreate(&e1)) return cuda_fail(cudaGetLastError(), "event");
    std::vector<float> t;
    int rc = AAHRT_OK;
    for (int r = 0; r < 4 && !rc; ++r) {
        cudaEventRecord(e0, st);
        rc = apply_forward(p, m, d, st);
        if (!rc) rc = apply_adjoint(p, d, g, st);
        cudaEventRecord(e1, st);
        cudaError_t e = cudaEventSynchronize(e1);
        if (!rc && e) rc = cuda_fail(e, "tuning run");
        float x = 0.f;
        cudaEventElapsedTime(&x, e0, e1);
        if (r > 0) t.push_back(x);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return AAHRT_OK;
}

}  // namespace

int autotune_plan(Plan **out, int ncube, int ndist, const aahrt_geom *geoms,
                  const aahrt_opts *opts_in) {
    aahrt_opts base;
    std::memset(&base, 0, sizeof base);
    if (opts_in) base = *opts_in;
    base.autotune = 0;
    const Trial tb = trial_batch(ncube, ndist, geoms);
    base.ngather = tb.ndist == 1 ? tb.ncube : 0;
    cudaStream_t st = nullptr;
    cudaError_t e;
    int rc;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)))
        return cuda_fail(e, "tuning stream");
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } sg{st};
    auto make = [&](const aahrt_opts &o, Plan **p) {
        return build_plan(p, tb.ncube, tb.ndist, tb.geoms.data(), &o);
    };

    // reference plan (widest kernel) fixes the buffer sizes of the trial batch
    Plan *ref = nullptr;
    aahrt_opts o = base;
    const bool lineark = base.slice_interp == AAHRT_SLICE_LINEAR_K;
    // the direct sum (explicit q axes) and the tensor-core contraction have
    // no spreading kernel to size
    const bool no_width = base.slice_interp == AAHRT_SLICE_DIRECT || base.q_axis != nullptr ||
                          base.precision == AAHRT_PRECISION_SPLIT_BF16;
    if (!lineark && !no_width) o.spread_width = kMaxW;
    if ((rc = make(o, &ref))) return rc;
    const long long nm = ref->model_len, nd = ref->data_len;
    DevBuf bm, bd, bd2, bg, bacc;
    if ((e = cudaMalloc(&bm.p, nm * sizeof(float))) || (e = cudaMalloc(&bd.p, nd * sizeof(float))) ||
        (e = cudaMalloc(&bd2.p, nd * sizeof(float))) || (e = cudaMalloc(&bg.p, nm * sizeof(float))) ||
        (e = cudaMalloc(&bacc.p, 2 * sizeof(double)))) {
        free_plan(ref);
        cudaGetLastError();
        return set_error(AAHRT_ERR_OOM, "autotuner buffers: %s", cudaGetErrorString(e));
    }
    float *m = (float *)bm.p, *d = (float *)bd.p, *d2 = (float *)bd2.p, *g = (float *)bg.p;
    double *acc = (double *)bacc.p;
    fill_random_kernel<<<grid_for(nm), 256, 0, st>>>(m, nm, 0x5eed0001ull);
    rc = apply_forward(*ref, m, d, st);
    free_plan(ref);
    if (rc) return rc;

    // spreading width: smallest with measured relative error <= 2e-6
    int W = base.spread_width;
    if (W == 0 && !lineark && !no_width) {
        W = kMaxW;
        for (int w = kMinW + 1; w < kMaxW; ++w) {
            Plan *pw = nullptr;
            o = base;
            o.spread_width = w;
            if ((rc = make(o, &pw))) return rc;
            rc = apply_forward(*pw, m, d2, st);
            free_plan(pw);
            if (rc) return rc;
            double h[2] = {0, 0};
            if ((e = cudaMemsetAsync(acc, 0, 2 * sizeof(double), st))) return cuda_fail(e, "memset");
            diff_norm_kernel<<<grid_for(nd), 256, 0, st>>>(d2, d, nd, acc);
            if ((e = cudaMemcpyAsync(h, acc, sizeof h, cudaMemcpyDeviceToHost, st)) ||
                (e = cudaStreamSynchronize(st)))
                return cuda_fail(e, "tuning accuracy");
            if (std::sqrt(h[0] / std::max(h[1], 1e-300)) <= 2e-6) {
                W = w;
                break;
            }
        }
    }

    // tiles: theta_group x time_pairs, timed
    const int nth = geoms[0].ntheta;
    std::vector<int> tgs, tps;
    if (base.theta_group > 0) {
        tgs.push_back(base.theta_group);
    } else {
        tgs.push_back(0);
        for (int div = 1; div <= 6; ++div) {
            const int t = (nth + div - 1) / div;
            if (t >= 1 && std::find(tgs.begin(), tgs.end(), t) == tgs.end()) tgs.push_back(t);
        }
    }
    if (base.time_pairs > 0) {
        tps.push_back(base.time_pairs);
    } else {
        for (int t : {1, 2, 4, 8}) tps.push_back(t);
    }
    double best = 1e300;
    int best_tg = 0, best_tp = 0;
    for (int tg : tgs)
        for (int tp : tps) {
            Plan *pc = nullptr;
            o = base;
            o.spread_width = W;
            o.theta_group = tg;
            o.time_pairs = tp;
            if (make(o, &pc)) continue;          // candidate does not fit (shared memory)
            double ms = 0;
            rc = time_pair(*pc, m, d2, g, st, &ms);
            free_plan(pc);
            if (rc) return rc;
            if (ms < best) {
                best = ms;
                best_tg = tg;
                best_tp = tp;
            }
        }
    if (best >= 1e300) return set_error(AAHRT_ERR_UNSUPPORTED, "autotuner: no candidate fits");

    aahrt_opts fin;
    std::memset(&fin, 0, sizeof fin);
    if (opts_in) fin = *opts_in;
    fin.autotune = 0;
    fin.spread_width = W;
    fin.theta_group = best_tg;
    fin.time_pairs = best_tp;
    Plan *p = nullptr;
    if ((rc = build_plan(&p, ncube, ndist, geoms, &fin))) return rc;
    p->autotuned = true;
    p->tune_ms = best;
    *out = p;
    return AAHRT_OK;
}

}  // namespace aahrt
