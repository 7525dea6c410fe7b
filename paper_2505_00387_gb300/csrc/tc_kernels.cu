// Fourier slice stage as a direct complex contraction on the tensor cores,
// for gathers that share one geometry (Algorithm 1 step 3 / its transpose,
// eqs. Inv_op, inv_GFST, theta factors of eq. thli).
//
// With G gathers stored gather-fastest in slice-major spectra
// (X[j][k][l][g], Y[j][k][i][g] with i the trace's rank inside slice j, so
// every (bin, slice) block is contiguous), the slice step of bin k for the
// traces h whose first azimuth slice is j is
//   Y[h][g] = scale * sum_s w_s(h) sum_l E[h][l] X[l][j_s][g],
//   E[h][l] = exp(-2 pi i f_k q_l r_h^2),  j_0 = j, j_1 = j + 1 (mod ntheta),
// a complex GEMM (traces x q) * (q x 2G) per (k, j); the adjoint of slice j,
//   X^[l][j][g] = scale * sum_h w_j(h) conj(E[h][l]) Y^[h][g],
// is a complex GEMM (q x traces) * (traces x G) over the traces of slices j
// (weight w0) and j - 1 (weight w1).  No spreading kernel and no q-FFT: the
// DFT along q is evaluated exactly at k_q = f_k r^2.
//
// Complex products become real GEMMs with interleaved real/imaginary K:
//   A'[m][2p] = Re A[m][p], A'[m][2p+1] = Im A[m][p]
//   B'[n][2p], B'[n][2p+1] = (Re B, -Im B) for real-part columns n,
//                            (Im B,  Re B) for imaginary-part columns,
// and every FP32 operand is split into bf16 hi + lo parts:
//   A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi   (FP32 accumulation in TMEM).
// The phase arguments are range-reduced exactly in 64-bit fixed point.
//
// One CTA per SM (persistent, items from an atomic counter); all 16 warps
// build the bf16 operand tiles of a K chunk (64 K-elements) in shared memory
// (128-byte swizzled K-major layout) while the tensor core works on the
// previous chunk (two stages, mbarrier-tracked tcgen05.commit); thread 0
// issues the MMAs; accumulators live in TMEM and are read back by all warps.
#include <algorithm>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace aahrt {

using namespace tc;

constexpr int kTcThreads = 512;
constexpr uint32_t kTileA = 128u * 128u;     // one 128-row x 64-element bf16 tile
constexpr uint32_t kTcWait = 1u << 24;       // mbarrier polls before giving up
constexpr int kTcMaxGp = 64;

struct TcArgs {
    const TraceGeo *__restrict__ geo;     // traces sorted by first slice
    const int *__restrict__ ss;           // first sorted trace of each slice (ntheta + 1)
    const int4 *__restrict__ tiles;       // forward row tiles {j, t0, t1, 0}
    int *counter;
    int *err;
    long long total;
    const long long *__restrict__ qn;     // explicit axis: q_l = q_c + qn[l] eps, else null
    unsigned long long wait_ns;           // device time a wait may take before giving up
    int stall;                            // test hook: issue no matrix operations
    int ntiles, nbins, nq, ntheta, G, Gp, ntr, cq;
    float scale;
};

__device__ __forceinline__ unsigned char *align1024(unsigned char *p) {
    return (unsigned char *)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
}

// (a, b) -> bf16x2 hi parts and bf16x2 lo parts (a - hi_a, b - hi_b); one
// packed conversion each way
__device__ __forceinline__ void split2(float a, float b, uint32_t *hi, uint32_t *lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    *hi = *reinterpret_cast<const uint32_t *>(&h);
    *lo = *reinterpret_cast<const uint32_t *>(&l);
}

// 8 floats -> hi and lo bf16 chunks (16 bytes each)
__device__ __forceinline__ void split8(const float *v, uint4 *hi, uint4 *lo) {
    split2(v[0], v[1], &hi->x, &lo->x);
    split2(v[2], v[3], &hi->y, &lo->y);
    split2(v[4], v[5], &hi->z, &lo->z);
    split2(v[6], v[7], &hi->w, &lo->w);
}

// 16-byte chunk c (K-elements 8c .. 8c+7) of row r of a swizzled tile
__device__ __forceinline__ void st_chunk(unsigned char *tile, int r, int c, uint4 v) {
    *reinterpret_cast<uint4 *>(tile + r * 128 + ((((unsigned)c ^ (unsigned)r) & 7u) << 4)) = v;
}

// exp(sgn * 2 pi i x), x a fixed-point fraction of a cycle (2^-64 units)
__device__ __forceinline__ float2 cis_fixed(unsigned long long x, float sgn) {
    const float f = (float)(int)(unsigned)(x >> 32) * 2.3283064365386963e-10f;   // [-1/2, 1/2)
    float s, c;
    __sincosf(6.28318530717958647692f * f, &s, &c);     // |angle| <= pi
    return make_float2(c, sgn * s);
}

__device__ __forceinline__ float2 cmul2(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Eight consecutive q samples l0 .. l0+7 of exp(sgn 2 pi i f_k q_l r^2) (zero
// for l >= nq): the phase of l is k*A + (l - cq)*k*B in fixed point.
__device__ __forceinline__ void phases8(const TraceGeo &tr, unsigned k, int l0, int cq, int nq,
                                        float sgn, float wgt, float2 *e) {
    const unsigned long long kb = (unsigned long long)k * tr.B;
    const unsigned long long p0 =
        (unsigned long long)k * tr.A + (unsigned long long)(long long)(l0 - cq) * kb;
    float2 z = cis_fixed(p0, sgn);
    z.x *= wgt;
    z.y *= wgt;
    const float2 st = cis_fixed(kb, sgn);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        e[i] = l0 + i < nq ? z : make_float2(0.f, 0.f);
        z = cmul2(z, st);
    }
}

// The same eight samples on an explicit (non-uniform) curvature axis: the
// phase of l is k*A + qn[l]*k*B, one rotation per sample.
__device__ __forceinline__ void phases8_axis(const TraceGeo &tr, unsigned k, int l0,
                                             const long long *qn, int nq, float sgn, float wgt,
                                             float2 *e) {
    const unsigned long long ka = (unsigned long long)k * tr.A;
    const unsigned long long kb = (unsigned long long)k * tr.B;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int l = l0 + i;
        if (l < nq) {
            const float2 z = cis_fixed(ka + (unsigned long long)__ldg(qn + l) * kb, sgn);
            e[i] = make_float2(z.x * wgt, z.y * wgt);
        } else {
            e[i] = make_float2(0.f, 0.f);
        }
    }
}

struct TcState {
    uint32_t tm;            // TMEM base
    uint32_t mbar[2];
    uint32_t ncommit[2];
    bool failed;
};

__device__ __forceinline__ void tc_begin(TcState &s, uint64_t *mbar, uint32_t *tmem_slot) {
    const int warp = threadIdx.x >> 5;
    if (warp == 0) tmem_alloc(smem_u32(tmem_slot), 256);
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&mbar[0]), 1);
        mbar_init(smem_u32(&mbar[1]), 1);
        mbar_fence_init();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    s.tm = *tmem_slot;
    s.mbar[0] = smem_u32(&mbar[0]);
    s.mbar[1] = smem_u32(&mbar[1]);
    s.ncommit[0] = s.ncommit[1] = 0;
    s.failed = false;
}

// wait for the latest commit on buffer b
__device__ __forceinline__ void tc_wait(TcState &s, int b, int *err, unsigned long long ns) {
    if (s.ncommit[b] == 0 || s.failed) return;
    if (!mbar_wait(s.mbar[b], (s.ncommit[b] - 1) & 1u, kTcWait, ns)) {
        s.failed = true;
        if ((threadIdx.x & 31) == 0) atomicExch(err, 1);
    }
}

__device__ __forceinline__ void tc_end(TcState &s) {
    fence_before_sync();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) tmem_dealloc(s.tm, 256);
}

// Fetch the next work item (uniform); -1 when done or after a timeout.
__device__ __forceinline__ long long tc_next(const TcArgs &a, TcState &s, long long *slot) {
    fence_before_sync();
    if (threadIdx.x == 0) *slot = (long long)atomicAdd(a.counter, 1);
    const int any_failed = __syncthreads_or(s.failed ? 1 : 0);
    fence_after_sync();
    const long long item = *slot;
    __syncthreads();            // every thread has read the slot before it is rewritten
    if (any_failed) s.failed = true;
    if (any_failed || item >= a.total) return -1;
    return item;
}

// After a timeout: give the MMAs already issued a bounded chance to finish
// before the TMEM is released.
__device__ __forceinline__ void tc_drain(TcState &s, unsigned long long ns) {
    if (!s.failed) return;
    for (int b = 0; b < 2; ++b)
        if (s.ncommit[b] > 0) mbar_wait(s.mbar[b], (s.ncommit[b] - 1) & 1u, kTcWait, ns);
}

// ------------------------------------------------------------- forward
__global__ void __launch_bounds__(kTcThreads, 1)
slice_fwd_tc_kernel(const TcArgs a, const float2 *__restrict__ X, float2 *__restrict__ Y) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = align1024(smem_raw);
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ long long s_item;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Gp = a.Gp, N = 4 * Gp;
    const uint32_t bbytes = (uint32_t)N * 128u;
    const uint32_t stage_bytes = 2 * kTileA + 2 * bbytes;
    const uint32_t idesc = idesc_bf16_f32(128, N);
    const int nch = (a.nq + 31) >> 5;
    const int J = a.ntheta;
    TcState s;
    tc_begin(s, mbar, &tmem_slot);

    for (;;) {
        const long long item = tc_next(a, s, &s_item);
        if (item < 0) break;
        const int k = (int)(item / a.ntiles);
        const int4 tile = a.tiles[item - (long long)k * a.ntiles];
        const int j = tile.x, t0 = tile.y, t1 = tile.z;
        const int jn = j + 1 == J ? 0 : j + 1;
        const long long blk = (long long)a.nq * a.G;          // one (bin, slice) block of X
        const float2 *Xj = X + ((long long)j * a.nbins + k) * blk;
        const float2 *Xn = X + ((long long)jn * a.nbins + k) * blk;

        for (int c = 0; c < nch; ++c) {
            const int b = c & 1;
            if (c >= 2) tc_wait(s, b, a.err, a.wait_ns);
            unsigned char *ahi = sm + b * stage_bytes, *alo = ahi + kTileA;
            unsigned char *bhi = alo + kTileA, *blo = bhi + bbytes;
            // A: E[h][l] for 128 traces x 32 q samples, (Re, Im) interleaved
            for (int u = tid; u < 128 * 4; u += kTcThreads) {
                const int r = u >> 2, lb = u & 3;
                const int t = t0 + r;
                float2 e[8];
                if (t < t1) {
                    const TraceGeo tr = a.geo[t];
                    if (a.qn)
                        phases8_axis(tr, (unsigned)k, 32 * c + 8 * lb, a.qn, a.nq, -1.f, 1.f, e);
                    else
                        phases8(tr, (unsigned)k, 32 * c + 8 * lb, a.cq, a.nq, -1.f, 1.f, e);
                } else {
#pragma unroll
                    for (int i = 0; i < 8; ++i) e[i] = make_float2(0.f, 0.f);
                }
                uint4 h0, l0, h1, l1;
                split8(reinterpret_cast<const float *>(e), &h0, &l0);
                split8(reinterpret_cast<const float *>(e) + 8, &h1, &l1);
                st_chunk(ahi, r, 2 * lb, h0);
                st_chunk(ahi, r, 2 * lb + 1, h1);
                st_chunk(alo, r, 2 * lb, l0);
                st_chunk(alo, r, 2 * lb + 1, l1);
            }
            // B: rows (part, slice, g), K = the chunk's q samples
            for (int u = tid; u < 8 * Gp; u += kTcThreads) {
                const int g = u % Gp;
                const int rest = u / Gp;
                const int sl = rest & 1, lb = rest >> 1;
                const float2 *Xs = sl ? Xn : Xj;
                const int l0 = 32 * c + 8 * lb;
                float vr[16], vi[16];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int l = l0 + i;
                    float2 x = make_float2(0.f, 0.f);
                    if (l < a.nq && g < a.G) x = __ldg(Xs + (long long)l * a.G + g);
                    vr[2 * i] = x.x;
                    vr[2 * i + 1] = -x.y;
                    vi[2 * i] = x.y;
                    vi[2 * i + 1] = x.x;
                }
                const int nre = sl * Gp + g, nim = 2 * Gp + sl * Gp + g;
                uint4 h0, lo0, h1, lo1;
                split8(vr, &h0, &lo0);
                split8(vr + 8, &h1, &lo1);
                st_chunk(bhi, nre, 2 * lb, h0);
                st_chunk(bhi, nre, 2 * lb + 1, h1);
                st_chunk(blo, nre, 2 * lb, lo0);
                st_chunk(blo, nre, 2 * lb + 1, lo1);
                split8(vi, &h0, &lo0);
                split8(vi + 8, &h1, &lo1);
                st_chunk(bhi, nim, 2 * lb, h0);
                st_chunk(bhi, nim, 2 * lb + 1, h1);
                st_chunk(blo, nim, 2 * lb, lo0);
                st_chunk(blo, nim, 2 * lb + 1, lo1);
            }
            fence_async_smem();
            __syncthreads();
            if (tid == 0 && !a.stall) {
                fence_after_sync();
                const uint32_t a_hi = smem_u32(ahi), a_lo = smem_u32(alo);
                const uint32_t b_hi = smem_u32(bhi), b_lo = smem_u32(blo);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    mma_bf16(s.tm, sw128_desc(a_hi + 32 * t), sw128_desc(b_hi + 32 * t), idesc,
                             (c > 0 || t > 0) ? 1u : 0u);
                    mma_bf16(s.tm, sw128_desc(a_hi + 32 * t), sw128_desc(b_lo + 32 * t), idesc, 1u);
                    mma_bf16(s.tm, sw128_desc(a_lo + 32 * t), sw128_desc(b_hi + 32 * t), idesc, 1u);
                }
                mma_commit(s.mbar[b]);
            }
            s.ncommit[b]++;
        }
        tc_wait(s, (nch - 1) & 1, a.err, a.wait_ns);
        fence_after_sync();
        if (s.failed) continue;

        // epilogue: Y[h][g] = scale (w0 P[h][g, j] + w1 P[h][g, j+1])
        const int q = warp & 3, quarter = warp >> 2;
        const int r = 32 * q + lane;
        const int t = t0 + r;
        const bool valid = t < t1;
        TraceGeo tr{};
        if (valid) tr = a.geo[t];
        const uint32_t lanebase = s.tm + ((uint32_t)(32 * q) << 16);
        const int s0 = a.ss[j], cnt = a.ss[j + 1] - s0;
        float2 *Yrow = Y + ((long long)a.nbins * s0 + (long long)k * cnt + (valid ? t - s0 : 0)) * a.G;
        for (int gb = 16 * quarter; gb < Gp; gb += 64) {
            float re0[16], re1[16], im0[16], im1[16];
            tmem_ld16(lanebase + gb, re0);
            tmem_ld16(lanebase + Gp + gb, re1);
            tmem_ld16(lanebase + 2 * Gp + gb, im0);
            tmem_ld16(lanebase + 3 * Gp + gb, im1);
            if (valid) {
                const float w0 = a.scale * tr.w0, w1 = a.scale * tr.w1;
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (gb + i < a.G)
                        Yrow[gb + i] = make_float2(fmaf(w0, re0[i], w1 * re1[i]),
                                                   fmaf(w0, im0[i], w1 * im1[i]));
            }
        }
    }
    tc_drain(s, a.wait_ns);
    tc_end(s);
}

// ------------------------------------------------------------- adjoint
__global__ void __launch_bounds__(kTcThreads, 1)
slice_adj_tc_kernel(const TcArgs a, const float2 *__restrict__ Yh, float2 *__restrict__ Xh) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = align1024(smem_raw);
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ long long s_item;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Gp = a.Gp, N = 2 * Gp;
    const uint32_t bbytes = (uint32_t)N * 128u;
    const uint32_t stage_bytes = 4 * kTileA + 2 * bbytes;
    const uint32_t idesc = idesc_bf16_f32(128, N);
    const int nmt = a.nq > 128 ? 2 : 1;
    const int J = a.ntheta;
    TcState s;
    tc_begin(s, mbar, &tmem_slot);

    for (;;) {
        const long long item = tc_next(a, s, &s_item);
        if (item < 0) break;
        const int k = (int)(item / J);
        const int j = (int)(item - (long long)k * J);
        const int jm = j == 0 ? J - 1 : j - 1;
        const int a0 = a.ss[j], n1 = a.ss[j + 1] - a0;      // weight w0
        const int b0 = a.ss[jm], n2 = a.ss[jm + 1] - b0;    // weight w1
        const int ntot = n1 + n2;
        const int nch = (ntot + 31) >> 5;
        // slice blocks of Y^: slice j (weight w0) and slice j - 1 (weight w1)
        const float2 *Ya = Yh + ((long long)a.nbins * a0 + (long long)k * n1) * a.G;
        const float2 *Yb = Yh + ((long long)a.nbins * b0 + (long long)k * n2) * a.G;

        for (int c = 0; c < nch; ++c) {
            const int b = c & 1;
            if (c >= 2) tc_wait(s, b, a.err, a.wait_ns);
            unsigned char *st0 = sm + b * stage_bytes;
            unsigned char *bhi = st0 + 4 * kTileA, *blo = bhi + bbytes;
            // A: w conj(E)[l][h], rows l (two M-tiles), K = 32 traces
            {
                const int hh = lane;
                const int p = 32 * c + hh;
                TraceGeo tr{};
                float wgt = 0.f;
                const bool have = p < ntot;
                if (have) {
                    tr = a.geo[p < n1 ? a0 + p : b0 + (p - n1)];
                    wgt = p < n1 ? tr.w0 : tr.w1;
                }
                for (int lb = warp; lb < 16 * nmt; lb += kTcThreads / 32) {
                    const int l0 = 8 * lb;
                    const int mt = l0 >> 7;
                    unsigned char *ahi = st0 + (2 * mt) * kTileA, *alo = ahi + kTileA;
                    float2 e[8];
                    if (have) {
                        if (a.qn)
                            phases8_axis(tr, (unsigned)k, l0, a.qn, a.nq, 1.f, wgt, e);
                        else
                            phases8(tr, (unsigned)k, l0, a.cq, a.nq, 1.f, wgt, e);
                    } else {
#pragma unroll
                        for (int i = 0; i < 8; ++i) e[i] = make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int r = (l0 & 127) + i;
                        uint32_t h, lo;
                        split2(e[i].x, e[i].y, &h, &lo);
                        const uint32_t off = sw128_offset((uint32_t)r, (uint32_t)(2 * hh));
                        *reinterpret_cast<uint32_t *>(ahi + off) = h;
                        *reinterpret_cast<uint32_t *>(alo + off) = lo;
                    }
                }
            }
            // B: rows (part, g), K = 32 traces x (Re, Im); one unit is one
            // 16-byte chunk (4 traces) of a row pair, so 8 Gp units
            for (int u = tid; u < 8 * Gp; u += kTcThreads) {
                const int g = u % Gp, tq = u / Gp;
                float vr[8], vi[8];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int p = 32 * c + 4 * tq + i;
                    float2 y = make_float2(0.f, 0.f);
                    if (p < ntot && g < a.G)
                        y = __ldg(p < n1 ? Ya + (long long)p * a.G + g
                                         : Yb + (long long)(p - n1) * a.G + g);
                    vr[2 * i] = y.x;
                    vr[2 * i + 1] = -y.y;
                    vi[2 * i] = y.y;
                    vi[2 * i + 1] = y.x;
                }
                uint4 h, lo;
                split8(vr, &h, &lo);
                st_chunk(bhi, g, tq, h);
                st_chunk(blo, g, tq, lo);
                split8(vi, &h, &lo);
                st_chunk(bhi, Gp + g, tq, h);
                st_chunk(blo, Gp + g, tq, lo);
            }
            fence_async_smem();
            __syncthreads();
            if (tid == 0 && !a.stall) {
                fence_after_sync();
                const uint32_t b_hi = smem_u32(bhi), b_lo = smem_u32(blo);
                for (int mt = 0; mt < nmt; ++mt) {
                    const uint32_t a_hi = smem_u32(st0 + (2 * mt) * kTileA);
                    const uint32_t a_lo = a_hi + kTileA;
                    const uint32_t d = s.tm + (uint32_t)(mt * N);
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        mma_bf16(d, sw128_desc(a_hi + 32 * t), sw128_desc(b_hi + 32 * t), idesc,
                                 (c > 0 || t > 0) ? 1u : 0u);
                        mma_bf16(d, sw128_desc(a_hi + 32 * t), sw128_desc(b_lo + 32 * t), idesc,
                                 1u);
                        mma_bf16(d, sw128_desc(a_lo + 32 * t), sw128_desc(b_hi + 32 * t), idesc,
                                 1u);
                    }
                }
                mma_commit(s.mbar[b]);
            }
            s.ncommit[b]++;
        }
        if (nch > 0) tc_wait(s, (nch - 1) & 1, a.err, a.wait_ns);
        fence_after_sync();
        if (s.failed) continue;

        // epilogue: X^[l][j][g] = scale * accumulator (zero without traces)
        const int q = warp & 3, mt = (warp >> 2) & 1, half = warp >> 3;
        if (mt < nmt) {
            const int l = 128 * mt + 32 * q + lane;
            const uint32_t base = s.tm + ((uint32_t)(32 * q) << 16) + (uint32_t)(mt * N);
            float2 *Xrow = Xh + (((long long)j * a.nbins + k) * a.nq + (l < a.nq ? l : 0)) * a.G;
            for (int gb = 16 * half; gb < Gp; gb += 32) {
                float re[16], im[16];
                if (nch > 0) {
                    tmem_ld16(base + gb, re);
                    tmem_ld16(base + Gp + gb, im);
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i) re[i] = im[i] = 0.f;
                }
                if (l < a.nq) {
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (gb + i < a.G)
                            Xrow[gb + i] = make_float2(a.scale * re[i], a.scale * im[i]);
                }
            }
        }
    }
    tc_drain(s, a.wait_ns);
    tc_end(s);
}

// ------------------------------------------------------------- host side
static TcArgs tc_args(const Plan &p, bool adjoint, int *counter) {
    TcArgs a;
    a.geo = p.geo;
    a.ss = p.slice_start;
    a.tiles = p.tc_tiles;
    a.counter = counter;
    a.err = p.counters + kTcErrSlot;
    a.ntiles = p.tc_ntiles;
    a.total = adjoint ? (long long)p.nbins * p.ntheta : (long long)p.nbins * p.tc_ntiles;
    a.nbins = p.nbins;
    a.nq = p.nq;
    a.ntheta = p.ntheta;
    a.G = p.ngather;
    a.Gp = p.tc_gp;
    a.ntr = p.ntr[0];
    a.cq = p.cq;
    a.qn = p.qexplicit ? p.qn : nullptr;
    a.stall = p.tc_stall ? 1 : 0;
    a.wait_ns = p.tc_stall ? 20000000ull : 1000000000ull;   // 20 ms under the test hook, else 1 s
    a.scale = (float)(1.0 / p.nfft);
    return a;
}

size_t tc_smem_bytes(int Gp, bool adjoint) {
    const size_t b = (size_t)(adjoint ? 2 * Gp : 4 * Gp) * 128;
    const size_t stage = (adjoint ? 4 : 2) * (size_t)kTileA + 2 * b;
    return 2 * stage + 1024;
}

cudaError_t configure_tc_kernels(Plan &p, int num_sms, int max_smem) {
    if (p.tc_gp < 8 || p.tc_gp > kTcMaxGp || (p.tc_gp & 7)) return cudaErrorInvalidValue;
    const size_t sf = tc_smem_bytes(p.tc_gp, false), sa = tc_smem_bytes(p.tc_gp, true);
    if ((int)sf > max_smem || (int)sa > max_smem) return cudaErrorInvalidConfiguration;
    cudaError_t e;
    if ((e = raise_smem_limit(slice_fwd_tc_kernel, max_smem))) return e;
    if ((e = raise_smem_limit(slice_adj_tc_kernel, max_smem))) return e;
    p.smem_sfwd = sf;
    p.smem_sadj = sa;
    const long long items_f = (long long)p.nbins * p.tc_ntiles;
    const long long items_a = (long long)p.nbins * p.ntheta;
    p.slice_grid_fwd = (int)std::min<long long>(items_f, num_sms);
    p.slice_grid_adj = (int)std::min<long long>(items_a, num_sms);
    return cudaSuccess;
}

cudaError_t launch_slice_tc(Plan &p, bool adjoint, const float2 *in, float2 *out,
                            cudaStream_t st, int *counter) {
    const TcArgs a = tc_args(p, adjoint, counter);
    if (adjoint)
        slice_adj_tc_kernel<<<p.slice_grid_adj, kTcThreads, p.smem_sadj, st>>>(a, in, out);
    else
        slice_fwd_tc_kernel<<<p.slice_grid_fwd, kTcThreads, p.smem_sfwd, st>>>(a, in, out);
    return cudaGetLastError();
}

}  // namespace aahrt
