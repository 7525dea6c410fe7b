// Fourier slice stage as a direct sum of the DFT along q (Algorithm 1 step 3
// and its exact transpose; eqs. Inv_op, inv_GFST and the theta factors of
// eq. thli), for any curvature axis -- in particular a uniform slowness axis,
// whose curvatures q_l = p_l^2 are not uniform (a type-3 DFT along q):
//
//   Y[k][h] = scale * sum_s w_s(h) sum_l X[k][l][j_s(h)] exp(-2 pi i f_k q_l r_h^2)
//   X^[k][l][j] = scale * sum_h w_j(h) exp(+2 pi i f_k q_l r_h^2) Y^[k][h]
//
// The phase in cycles is f_k q_l r_h^2 = k A_h + n_l k B_h with the axis
// written as q_l = q_c + n_l eps (integer n_l), A_h = q_c r_h^2/(Nfft ds) and
// B_h = eps r_h^2/(Nfft ds) in 0.64 fixed point: the products wrap modulo
// 2^64, so the fraction of a cycle is exact up to the rounding of A_h and B_h;
// per term only its top 32 bits are formed, from two 32-bit multiply-adds.
//
// Work items are (cube, azimuth group, bin) as in the spreading kernels.
// Forward: the item's slice columns of X[k] are staged in shared memory and
// each thread sums one trace over l (in four interleaved partial sums).
// Adjoint: the item's traces (y, weights, phase constants) are staged in
// chunks; each lane owns one (first slice, curvature) pair -- consecutive
// lanes take consecutive pairs, so a warp reads one or two traces at a time
// (shared-memory broadcast) -- evaluates every phase once and sums it with
// weight w0 (for that slice) and w1 (for the next) into two accumulator
// planes; each accumulator has one writer, so the order of the sums is fixed
// (no atomics).
#include <algorithm>

#include "internal.cuh"
#include "slice_math.cuh"

namespace aahrt {

constexpr int kDirectLanes = 4;   // interleaved partial sums per output (fixed below)

struct DirectArgs {
    const TraceGeo *__restrict__ geo;
    const SliceGroup *__restrict__ groups;
    const int *__restrict__ slice_start;
    const long long *__restrict__ qn;
    int *counter;
    long long total;
    int nbins, nq, ntheta, ngroup, tgroup, chunk;
    float scale;
};

// (cos, sin) of 2 pi t 2^-32 for a signed fraction t of a cycle
__device__ __forceinline__ void cis32(unsigned t, float *c, float *s) {
    __sincosf((float)(int)t * 1.4629180792671596e-9f, s, c);   // 2 pi / 2^32
}

size_t direct_smem_fwd(int tgroup, int extra, int nq) {
    return (size_t)(tgroup + extra) * nq * sizeof(float2) + (size_t)(nq + 1) / 2 * 8;
}

// chunk staged traces of 32 bytes ((y re, y im, w0, w1) and the phase
// constants), two accumulator planes nq x tgroup (w0 and w1 parts), then the
// n' table
size_t direct_smem_adj(int tgroup, int nq, int chunk) {
    return 2 * (size_t)tgroup * nq * sizeof(float2) + (size_t)nq * sizeof(unsigned) +
           (size_t)chunk * (sizeof(float4) + sizeof(Phase32));
}

__global__ void __launch_bounds__(kThreadsSlice, 3)
direct_fwd_kernel(const DirectArgs a, const float2 *__restrict__ X, float2 *__restrict__ Y) {
    extern __shared__ float4 smem_f4[];
    __shared__ long long s_item;
    const int extra = a.ngroup > 1 ? 1 : 0;
    float2 *Xs = reinterpret_cast<float2 *>(smem_f4);          // [jj][l]
    unsigned *s_np = reinterpret_cast<unsigned *>(Xs + (size_t)(a.tgroup + extra) * a.nq);
    for (int l = threadIdx.x; l < a.nq; l += blockDim.x)
        s_np[l] = (unsigned)((unsigned long long)a.qn[l] + 0x80000000ull);
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(a.counter, 1);
        __syncthreads();
        const long long item = s_item;
        if (item >= a.total) break;
        const int gi = (int)(item / a.nbins);
        const int k = (int)(item - (long long)gi * a.nbins);
        const SliceGroup g = a.groups[gi];
        const int ncol = g.nj + extra;
        // stage X[k][l][ja + jj] (slice index mod ntheta) as Xs[jj][l], so a
        // trace walks its slices' curvatures at unit stride
        const float2 *Xk = X + g.x_off + (long long)k * a.nq * a.ntheta;
        for (int idx = threadIdx.x; idx < a.nq * ncol; idx += blockDim.x) {
            const int l = idx / ncol;
            const int jj = idx - l * ncol;
            int j = g.ja + jj;
            if (j >= a.ntheta) j -= a.ntheta;
            Xs[jj * a.nq + l] = __ldg(Xk + (long long)l * a.ntheta + j);
        }
        __syncthreads();

        const TraceGeo *geo = a.geo + g.geo_off;
        float2 *Yk = Y + g.y_off + (long long)k * g.ntr;
        for (int t = g.f0 + threadIdx.x; t < g.f1; t += blockDim.x) {
            const TraceGeo tr = geo[t];
            const int jj0 = tr.j0 - g.ja;
            int jj1;
            if (extra) {
                jj1 = jj0 + 1;
            } else {
                jj1 = tr.j0 + 1;
                if (jj1 == a.ntheta) jj1 = 0;
            }
            const Phase32 ph = phase_consts((unsigned long long)k * tr.A,
                                            (unsigned long long)k * tr.B);
            const float2 *X0 = Xs + jj0 * a.nq;
            const float2 *X1 = Xs + jj1 * a.nq;
            // curvature l goes to partial sum l mod kDirectLanes; the partial
            // sums (fewer terms each: smaller rounding of the random-phase
            // sum) are added in a fixed order at the end
            float ar[kDirectLanes], ai[kDirectLanes];
#pragma unroll
            for (int u = 0; u < kDirectLanes; ++u) ar[u] = ai[u] = 0.f;
            for (int l = 0; l < a.nq; l += kDirectLanes) {
#pragma unroll
                for (int u = 0; u < kDirectLanes; ++u) {
                    if (l + u < a.nq) {
                        float c, s;
                        cis32(phase_top(s_np[l + u], ph), &c, &s);
                        const float2 x0 = X0[l + u], x1 = X1[l + u];
                        const float vr = fmaf(tr.w0, x0.x, tr.w1 * x1.x);
                        const float vi = fmaf(tr.w0, x0.y, tr.w1 * x1.y);
                        // v * exp(-2 pi i ph) = v (c - i s)
                        ar[u] = fmaf(vr, c, fmaf(vi, s, ar[u]));
                        ai[u] = fmaf(vi, c, fmaf(-vr, s, ai[u]));
                    }
                }
            }
            const float sr = (ar[0] + ar[1]) + (ar[2] + ar[3]);
            const float si = (ai[0] + ai[1]) + (ai[2] + ai[3]);
            Yk[tr.col] = make_float2(a.scale * sr, a.scale * si);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreadsSlice, 3)
direct_adj_kernel(const DirectArgs a, const float2 *__restrict__ Y, float2 *__restrict__ X) {
    extern __shared__ float4 smem_f4[];
    __shared__ long long s_item;
    float4 *s_y = smem_f4;                                                  // [chunk]
    Phase32 *s_ph = reinterpret_cast<Phase32 *>(s_y + a.chunk);            // phase constants
    float2 *acc0 = reinterpret_cast<float2 *>(s_ph + a.chunk);             // [l][nj], w0 parts
    float2 *acc1 = acc0 + (size_t)a.tgroup * a.nq;                          // [l][nj], w1 parts
    unsigned *s_np = reinterpret_cast<unsigned *>(acc1 + (size_t)a.tgroup * a.nq);
    for (int l = threadIdx.x; l < a.nq; l += blockDim.x)
        s_np[l] = (unsigned)((unsigned long long)a.qn[l] + 0x80000000ull);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool several = a.ngroup > 1;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(a.counter, 1);
        __syncthreads();
        const long long item = s_item;
        if (item >= a.total) break;
        const int gi = (int)(item / a.nbins);
        const int k = (int)(item - (long long)gi * a.nbins);
        const SliceGroup g = a.groups[gi];
        const TraceGeo *geo = a.geo + g.geo_off;
        const float2 *Yk = Y + g.y_off + (long long)k * g.ntr;
        const int *ss = a.slice_start + g.ss_off;
        const int nf = g.f1 - g.f0, ntot = nf + (g.e1 - g.e0);
        for (int idx = threadIdx.x; idx < a.nq * g.nj; idx += blockDim.x) {
            acc0[idx] = make_float2(0.f, 0.f);
            acc1[idx] = make_float2(0.f, 0.f);
        }
        // Source slice s of the item: s < nj holds the traces whose first
        // slice is ja + s (weight w0 into slice s, w1 into slice s + 1: the
        // next group's when s + 1 = nj, slice 0 when one group owns them all);
        // s = nj is the e-range (slice ja - 1), whose w1 lands on slice 0.
        // Each trace's phases are evaluated once for both weights.
        const int nsrc = g.nj + (several ? 1 : 0);
        for (int c0 = 0; c0 < ntot; c0 += a.chunk) {
            const int cn = min(a.chunk, ntot - c0);
            for (int i = threadIdx.x; i < cn; i += blockDim.x) {
                const int p = c0 + i;
                const int t = p < nf ? g.f0 + p : g.e0 + (p - nf);
                const TraceGeo tr = geo[t];
                const float2 y = __ldg(Yk + tr.col);
                s_y[i] = make_float4(a.scale * y.x, a.scale * y.y, tr.w0, tr.w1);
                s_ph[i] = phase_consts((unsigned long long)k * tr.A, (unsigned long long)k * tr.B);
            }
            __syncthreads();
            // lanes take the (source slice, curvature) pairs in order, 32 per
            // warp; a warp straddles at most a few slices (their trace
            // ranges differ; the lanes of each read the same trace)
            for (int pb = warp * 32; pb < nsrc * a.nq; pb += kThreadsSlice) {
                const int pidx = pb + lane;
                const bool live = pidx < nsrc * a.nq;
                const int sj = live ? pidx / a.nq : 0;
                const int l = live ? pidx - sj * a.nq : 0;
                const unsigned np = s_np[l];
                int ra, rb;
                if (sj < g.nj) {
                    ra = ss[g.ja + sj] - g.f0;
                    rb = ss[g.ja + sj + 1] - g.f0;
                } else {
                    ra = nf;
                    rb = ntot;
                }
                int lo = max(ra, c0) - c0, hi = min(rb, c0 + cn) - c0;
                if (!live) hi = lo;
                float ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f;
                for (int i = lo; i < hi; ++i) {
                    const float4 v = s_y[i];
                    const Phase32 ph = s_ph[i];
                    float c, s;
                    cis32(phase_top(np, ph), &c, &s);     // the forward's phase, bit for bit
                    // scale y exp(+2 pi i (k A + n_l k B))
                    const float zr = fmaf(v.x, c, -v.y * s);
                    const float zi = fmaf(v.x, s, v.y * c);
                    ar = fmaf(v.z, zr, ar);
                    ai = fmaf(v.z, zi, ai);
                    br = fmaf(v.w, zr, br);
                    bi = fmaf(v.w, zi, bi);
                }
                if (live && lo < hi) {
                    if (sj < g.nj) {
                        float2 &o = acc0[l * g.nj + sj];
                        o.x += ar;
                        o.y += ai;
                    }
                    int s1 = sj + 1;
                    if (sj == g.nj) s1 = 0;                    // e-range -> slice 0
                    else if (s1 == g.nj) s1 = several ? -1 : 0;
                    if (s1 >= 0) {
                        float2 &o = acc1[l * g.nj + s1];
                        o.x += br;
                        o.y += bi;
                    }
                }
            }
            __syncthreads();
        }
        float2 *Xk = X + g.x_off + (long long)k * a.nq * a.ntheta + g.ja;
        for (int idx = threadIdx.x; idx < a.nq * g.nj; idx += blockDim.x) {
            const int l = idx / g.nj;
            const int jj = idx - l * g.nj;
            const float2 u = acc0[idx], v = acc1[idx];
            Xk[(long long)l * a.ntheta + jj] = make_float2(u.x + v.x, u.y + v.y);
        }
        __syncthreads();
    }
}

cudaError_t configure_direct_kernels(Plan &p, int num_sms, int max_smem) {
    if ((int)p.smem_sfwd > max_smem || (int)p.smem_sadj > max_smem)
        return cudaErrorInvalidConfiguration;
    cudaError_t e;
    if ((e = raise_smem_limit(direct_fwd_kernel, max_smem))) return e;
    if ((e = raise_smem_limit(direct_adj_kernel, max_smem))) return e;
    int occ_f = 0, occ_a = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_f, direct_fwd_kernel,
                                                           kThreadsSlice, p.smem_sfwd)))
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_a, direct_adj_kernel,
                                                           kThreadsSlice, p.smem_sadj)))
        return e;
    if (occ_f < 1 || occ_a < 1) return cudaErrorInvalidConfiguration;
    p.slice_grid_fwd = (int)std::min<long long>(p.slice_items, (long long)occ_f * num_sms);
    p.slice_grid_adj = (int)std::min<long long>(p.slice_items, (long long)occ_a * num_sms);
    return cudaSuccess;
}

cudaError_t launch_slice_direct(Plan &p, bool adjoint, const float2 *in, float2 *out,
                                cudaStream_t st, int *counter) {
    DirectArgs a;
    a.geo = p.geo;
    a.groups = p.groups;
    a.slice_start = p.slice_start;
    a.qn = p.qn;
    a.counter = counter;
    a.total = p.slice_items;
    a.nbins = p.nbins;
    a.nq = p.nq;
    a.ntheta = p.ntheta;
    a.ngroup = p.ngroup;
    a.tgroup = p.tgroup;
    a.chunk = p.direct_chunk;
    a.scale = (float)(1.0 / p.nfft);
    if (adjoint)
        direct_adj_kernel<<<p.slice_grid_adj, kThreadsSlice, p.smem_sadj, st>>>(a, in, out);
    else
        direct_fwd_kernel<<<p.slice_grid_fwd, kThreadsSlice, p.smem_sfwd, st>>>(a, in, out);
    return cudaGetLastError();
}

}  // namespace aahrt
