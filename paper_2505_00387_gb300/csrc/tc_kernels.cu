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
// One CTA of 16 warps per SM (persistent), warp-specialized: producer warps
// build the bf16 operand tiles of each K chunk (64 K-elements) in shared
// memory (128-byte swizzled K-major layout) into a ring of two stages, one
// thread issues the MMAs and commits each stage back to the producers through
// an mbarrier, and epilogue warps read a finished accumulator out of TMEM
// while the tensor core fills the other of two accumulator buffers.
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

// The two B-operand rows of complex values: the real-part row holds
// (Re, -Im) and the imaginary-part row (Im, Re).  One hi/lo split of
// (Re, Im) gives both: negate the high half, or swap the halves (bf16
// negation is exact, so this equals splitting the negated value).
__device__ __forceinline__ void split_cplx(float re, float im, uint32_t *rhi, uint32_t *rlo,
                                           uint32_t *ihi, uint32_t *ilo) {
    uint32_t h, l;
    split2(re, im, &h, &l);
    *rhi = h ^ 0x80000000u;
    *rlo = l ^ 0x80000000u;
    *ihi = __byte_perm(h, 0, 0x1032);
    *ilo = __byte_perm(l, 0, 0x1032);
}

// a / d for 0 <= a < 2^20, d < 2^10, by a float reciprocal and one correction
__device__ __forceinline__ int tc_div(int a, int d, float inv_d) {
    int q = __float2int_rz(((float)a + 0.5f) * inv_d);
    const int r = a - q * d;
    if (r < 0) --q;
    else if (r >= d) ++q;
    return q;
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

// ------------------------------------------------------ pipeline roles
// Warp 0 allocates the TMEM (two accumulator buffers of 256 columns) and
// its lane 0 issues the MMAs; warps 1..11 build the operand tiles into a
// ring of two shared-memory stages; warps 12..15 (one per TMEM lane quarter)
// drain a finished accumulator to global memory while the tensor core fills
// the other.  Four kinds of mbarrier hand the stages and accumulators
// around:
//   full[s]   producers -> MMA    (stage s written; one arrival per producer thread)
//   empty[s]  MMA -> producers    (tcgen05.commit: the MMAs reading stage s are done)
//   accf[b]   MMA -> epilogue     (tcgen05.commit after an item's last chunk)
//   acce[b]   epilogue -> MMA     (accumulator b read out; one arrival per epilogue warp)
// Items are dealt round-robin (item = block + i * grid), so every role walks
// the same sequence without sharing a counter.  Every wait is bounded; a
// wait that runs out sets the error flag and the block's abort flag, which
// ends every role's loop, and the MMA thread waits (bounded) for its last
// commit before the TMEM is released.
constexpr int kTcProdWarp0 = 1;
constexpr int kTcProdWarps = 11;
constexpr int kTcProdThreads = 32 * kTcProdWarps;
constexpr int kTcEpiWarp0 = 12;          // warps 12..15: TMEM lane quarters 0..3
constexpr uint32_t kTcTmemCols = 512;    // two accumulators of 256 columns

struct TcBars {
    uint64_t full[2], empty[2], accf[2], acce[2];
};

__device__ __forceinline__ void tc_setup(TcBars *bars, uint32_t *tmem_slot, int *abort) {
    const int warp = threadIdx.x >> 5;
    if (warp == 0) tmem_alloc(smem_u32(tmem_slot), kTcTmemCols);
    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(&bars->full[i]), kTcProdThreads);
            mbar_init(smem_u32(&bars->empty[i]), 1);
            mbar_init(smem_u32(&bars->accf[i]), 1);
            mbar_init(smem_u32(&bars->acce[i]), 4);
        }
        *abort = 0;
        mbar_fence_init();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
}

__device__ __forceinline__ void tc_fail(const TcArgs &a, volatile int *abort) {
    *abort = 1;
    atomicExch(a.err, 1);
}

// wait on barrier `bar` for the phase of the given parity; false on timeout
// or abort (recording a timeout)
__device__ __forceinline__ bool tc_wait_bar(const TcArgs &a, uint64_t *bar, uint32_t parity,
                                            volatile int *abort) {
    if (*abort) return false;
    if (mbar_wait_or_abort(smem_u32(bar), parity, kTcWait, a.wait_ns, abort)) return true;
    tc_fail(a, abort);
    return false;
}

// ------------------------------------------------------------- forward
// Item = (bin k, row tile of <= 128 traces of slice j); K chunks of 32 q
// samples (64 interleaved bf16 K-elements); accumulator 128 x 4Gp.
__global__ void __launch_bounds__(kTcThreads, 1)
slice_fwd_tc_kernel(const TcArgs a, const float2 *__restrict__ X, float2 *__restrict__ Y) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = align1024(smem_raw);
    __shared__ TcBars bars;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort;
    volatile int *abort = &s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Gp = a.Gp, N = 4 * Gp;
    const uint32_t bbytes = (uint32_t)N * 128u;
    const uint32_t stage_bytes = 2 * kTileA + 2 * bbytes;
    const int nch = (a.nq + 31) >> 5;
    const int J = a.ntheta;
    tc_setup(&bars, &tmem_slot, &s_abort);
    const uint32_t tm = tmem_slot;

    if (warp == 0) {
        // ---------------------------------------------------------- MMA
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(128, N);
            uint32_t cc = 0, last_bar = 0, last_par = 0;
            bool issued = false;
            int it = 0;
            for (long long item = blockIdx.x; item < a.total; item += gridDim.x, ++it) {
                const int ab = it & 1;
                if (!tc_wait_bar(a, &bars.acce[ab], ((it >> 1) & 1) ^ 1, abort)) break;
                fence_after_sync();
                const uint32_t d = tm + (uint32_t)(ab * N);
                bool ok = true;
                for (int c = 0; c < nch; ++c, ++cc) {
                    const int st = cc & 1;
                    if (!tc_wait_bar(a, &bars.full[st], (cc >> 1) & 1, abort)) { ok = false; break; }
                    fence_after_sync();
                    if (!a.stall) {
                        unsigned char *ahi = sm + st * stage_bytes, *alo = ahi + kTileA;
                        unsigned char *bhi = alo + kTileA, *blo = bhi + bbytes;
                        const uint32_t a_hi = smem_u32(ahi), a_lo = smem_u32(alo);
                        const uint32_t b_hi = smem_u32(bhi), b_lo = smem_u32(blo);
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            mma_bf16(d, sw128_desc(a_hi + 32 * t), sw128_desc(b_hi + 32 * t),
                                     idesc, (c > 0 || t > 0) ? 1u : 0u);
                            mma_bf16(d, sw128_desc(a_hi + 32 * t), sw128_desc(b_lo + 32 * t),
                                     idesc, 1u);
                            mma_bf16(d, sw128_desc(a_lo + 32 * t), sw128_desc(b_hi + 32 * t),
                                     idesc, 1u);
                        }
                        mma_commit(smem_u32(&bars.empty[st]));
                        issued = true;
                        last_bar = smem_u32(&bars.empty[st]);
                        last_par = (cc >> 1) & 1;
                    }
                }
                if (!ok) break;
                if (!a.stall) {
                    mma_commit(smem_u32(&bars.accf[ab]));
                    last_bar = smem_u32(&bars.accf[ab]);
                    last_par = (it >> 1) & 1;
                }
            }
            // the TMEM is released only after the MMAs issued have finished
            if (issued) mbar_wait(last_bar, last_par, kTcWait, a.wait_ns);
        }
    } else if (warp < kTcEpiWarp0) {
        // ---------------------------------------------------- producers
        const int pid = tid - 32 * kTcProdWarp0;
        const float inv_gp = 1.0f / (float)Gp;
        uint32_t cc = 0;
        for (long long item = blockIdx.x; item < a.total && !*abort; item += gridDim.x) {
            const int k = (int)(item / a.ntiles);
            const int4 tile = a.tiles[item - (long long)k * a.ntiles];
            const int j = tile.x, t0 = tile.y, t1 = tile.z;
            const int jn = j + 1 == J ? 0 : j + 1;
            const long long blk = (long long)a.nq * a.G;      // one (bin, slice) block of X
            const float2 *Xj = X + ((long long)j * a.nbins + k) * blk;
            const float2 *Xn = X + ((long long)jn * a.nbins + k) * blk;
            for (int c = 0; c < nch; ++c, ++cc) {
                const int st = cc & 1;
                if (!tc_wait_bar(a, &bars.empty[st], ((cc >> 1) & 1) ^ 1, abort)) break;
                unsigned char *ahi = sm + st * stage_bytes, *alo = ahi + kTileA;
                unsigned char *bhi = alo + kTileA, *blo = bhi + bbytes;
                for (int u = pid; u < 128 * 4 + 8 * Gp; u += kTcProdThreads) {
                    if (u < 128 * 4) {
                        // A: E[h][l] for 128 traces x 32 q samples, (Re, Im) interleaved
                        const int r = u >> 2, lb = u & 3;
                        const int t = t0 + r;
                        float2 e[8];
                        if (t < t1) {
                            const TraceGeo tr = a.geo[t];
                            if (a.qn)
                                phases8_axis(tr, (unsigned)k, 32 * c + 8 * lb, a.qn, a.nq, -1.f,
                                             1.f, e);
                            else
                                phases8(tr, (unsigned)k, 32 * c + 8 * lb, a.cq, a.nq, -1.f, 1.f,
                                        e);
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
                    } else {
                        // B: rows (part, slice, g), K = the chunk's q samples
                        const int v = u - 128 * 4;
                        const int rest = tc_div(v, Gp, inv_gp);
                        const int g = v - rest * Gp;
                        const int sl = rest & 1, lb = rest >> 1;
                        const float2 *Xs = sl ? Xn : Xj;
                        const int l0 = 32 * c + 8 * lb;
                        uint32_t rh[8], rl[8], ih[8], il[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int l = l0 + i;
                            float2 x = make_float2(0.f, 0.f);
                            if (l < a.nq && g < a.G) x = __ldg(Xs + (long long)l * a.G + g);
                            split_cplx(x.x, x.y, &rh[i], &rl[i], &ih[i], &il[i]);
                        }
                        const int nre = sl * Gp + g, nim = 2 * Gp + sl * Gp + g;
                        st_chunk(bhi, nre, 2 * lb, make_uint4(rh[0], rh[1], rh[2], rh[3]));
                        st_chunk(bhi, nre, 2 * lb + 1, make_uint4(rh[4], rh[5], rh[6], rh[7]));
                        st_chunk(blo, nre, 2 * lb, make_uint4(rl[0], rl[1], rl[2], rl[3]));
                        st_chunk(blo, nre, 2 * lb + 1, make_uint4(rl[4], rl[5], rl[6], rl[7]));
                        st_chunk(bhi, nim, 2 * lb, make_uint4(ih[0], ih[1], ih[2], ih[3]));
                        st_chunk(bhi, nim, 2 * lb + 1, make_uint4(ih[4], ih[5], ih[6], ih[7]));
                        st_chunk(blo, nim, 2 * lb, make_uint4(il[0], il[1], il[2], il[3]));
                        st_chunk(blo, nim, 2 * lb + 1, make_uint4(il[4], il[5], il[6], il[7]));
                    }
                }
                fence_async_smem();     // this thread's tile writes -> the tensor core
                mbar_arrive(smem_u32(&bars.full[st]));
            }
        }
    } else {
        // ----------------------------------------------------- epilogue
        // Y[h][g] = scale (w0 P[h][g, j] + w1 P[h][g, j+1])
        const int q = warp & 3;
        int it = 0;
        for (long long item = blockIdx.x; item < a.total; item += gridDim.x, ++it) {
            const int ab = it & 1;
            if (!tc_wait_bar(a, &bars.accf[ab], (it >> 1) & 1, abort)) break;
            fence_after_sync();
            const int k = (int)(item / a.ntiles);
            const int4 tile = a.tiles[item - (long long)k * a.ntiles];
            const int j = tile.x, t0 = tile.y, t1 = tile.z;
            const int r = 32 * q + lane;
            const int t = t0 + r;
            const bool valid = t < t1;
            TraceGeo tr{};
            if (valid) tr = a.geo[t];
            const uint32_t lanebase = tm + ((uint32_t)(32 * q) << 16) + (uint32_t)(ab * N);
            const int s0 = a.ss[j], cnt = a.ss[j + 1] - s0;
            float2 *Yrow =
                Y + ((long long)a.nbins * s0 + (long long)k * cnt + (valid ? t - s0 : 0)) * a.G;
            const float w0 = a.scale * tr.w0, w1 = a.scale * tr.w1;
            for (int gb = 0; gb < Gp; gb += 16) {
                float re0[16], re1[16], im0[16], im1[16];
                tmem_ld16(lanebase + gb, re0);
                tmem_ld16(lanebase + Gp + gb, re1);
                tmem_ld16(lanebase + 2 * Gp + gb, im0);
                tmem_ld16(lanebase + 3 * Gp + gb, im1);
                if (valid) {
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (gb + i < a.G)
                            Yrow[gb + i] = make_float2(fmaf(w0, re0[i], w1 * re1[i]),
                                                       fmaf(w0, im0[i], w1 * im1[i]));
                }
            }
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bars.acce[ab]));
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tm, kTcTmemCols);
}

// ------------------------------------------------------------- adjoint
// Item = (bin k, slice j); M = q (nmt tiles of 128), K = the traces of
// slices j (weight w0) and j - 1 (weight w1) in chunks of 32; accumulator
// nmt x (128 x 2Gp).
__global__ void __launch_bounds__(kTcThreads, 1)
slice_adj_tc_kernel(const TcArgs a, const float2 *__restrict__ Yh, float2 *__restrict__ Xh) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = align1024(smem_raw);
    __shared__ TcBars bars;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort;
    volatile int *abort = &s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Gp = a.Gp, N = 2 * Gp;
    const uint32_t bbytes = (uint32_t)N * 128u;
    const uint32_t stage_bytes = 4 * kTileA + 2 * bbytes;
    const int nmt = a.nq > 128 ? 2 : 1;
    const int J = a.ntheta;
    const int acc_cols = 2 * N;          // columns per accumulator buffer (room for two M tiles)
    tc_setup(&bars, &tmem_slot, &s_abort);
    const uint32_t tm = tmem_slot;

    if (warp == 0) {
        // ---------------------------------------------------------- MMA
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(128, N);
            uint32_t cc = 0, last_bar = 0, last_par = 0;
            bool issued = false;
            int it = 0;
            for (long long item = blockIdx.x; item < a.total; item += gridDim.x, ++it) {
                const int ab = it & 1;
                const int k = (int)(item / J);
                const int j = (int)(item - (long long)k * J);
                const int jm = j == 0 ? J - 1 : j - 1;
                const int ntot = (a.ss[j + 1] - a.ss[j]) + (a.ss[jm + 1] - a.ss[jm]);
                const int nch = (ntot + 31) >> 5;
                if (!tc_wait_bar(a, &bars.acce[ab], ((it >> 1) & 1) ^ 1, abort)) break;
                fence_after_sync();
                bool ok = true;
                for (int c = 0; c < nch; ++c, ++cc) {
                    const int st = cc & 1;
                    if (!tc_wait_bar(a, &bars.full[st], (cc >> 1) & 1, abort)) { ok = false; break; }
                    fence_after_sync();
                    if (!a.stall) {
                        unsigned char *st0 = sm + st * stage_bytes;
                        const uint32_t b_hi = smem_u32(st0 + 4 * kTileA);
                        const uint32_t b_lo = b_hi + bbytes;
                        for (int mt = 0; mt < nmt; ++mt) {
                            const uint32_t a_hi = smem_u32(st0 + (2 * mt) * kTileA);
                            const uint32_t a_lo = a_hi + kTileA;
                            const uint32_t d = tm + (uint32_t)(ab * acc_cols + mt * N);
#pragma unroll
                            for (int t = 0; t < 4; ++t) {
                                mma_bf16(d, sw128_desc(a_hi + 32 * t), sw128_desc(b_hi + 32 * t),
                                         idesc, (c > 0 || t > 0) ? 1u : 0u);
                                mma_bf16(d, sw128_desc(a_hi + 32 * t), sw128_desc(b_lo + 32 * t),
                                         idesc, 1u);
                                mma_bf16(d, sw128_desc(a_lo + 32 * t), sw128_desc(b_hi + 32 * t),
                                         idesc, 1u);
                            }
                        }
                        mma_commit(smem_u32(&bars.empty[st]));
                        issued = true;
                        last_bar = smem_u32(&bars.empty[st]);
                        last_par = (cc >> 1) & 1;
                    }
                }
                if (!ok) break;
                if (!a.stall) {
                    // with no chunk (no traces) the commit arrives at once
                    mma_commit(smem_u32(&bars.accf[ab]));
                    issued = true;
                    last_bar = smem_u32(&bars.accf[ab]);
                    last_par = (it >> 1) & 1;
                }
            }
            if (issued) mbar_wait(last_bar, last_par, kTcWait, a.wait_ns);
        }
    } else if (warp < kTcEpiWarp0) {
        // ---------------------------------------------------- producers
        const int pid = tid - 32 * kTcProdWarp0;
        const float inv_gp = 1.0f / (float)Gp;
        const int na = 32 * 16 * nmt;    // A units: (trace, 8-q group)
        uint32_t cc = 0;
        for (long long item = blockIdx.x; item < a.total && !*abort; item += gridDim.x) {
            const int k = (int)(item / J);
            const int j = (int)(item - (long long)k * J);
            const int jm = j == 0 ? J - 1 : j - 1;
            const int a0 = a.ss[j], n1 = a.ss[j + 1] - a0;      // weight w0
            const int b0 = a.ss[jm], n2 = a.ss[jm + 1] - b0;    // weight w1
            const int ntot = n1 + n2;
            const int nch = (ntot + 31) >> 5;
            const float2 *Ya = Yh + ((long long)a.nbins * a0 + (long long)k * n1) * a.G;
            const float2 *Yb = Yh + ((long long)a.nbins * b0 + (long long)k * n2) * a.G;
            for (int c = 0; c < nch; ++c, ++cc) {
                const int st = cc & 1;
                if (!tc_wait_bar(a, &bars.empty[st], ((cc >> 1) & 1) ^ 1, abort)) break;
                unsigned char *st0 = sm + st * stage_bytes;
                unsigned char *bhi = st0 + 4 * kTileA, *blo = bhi + bbytes;
                for (int u = pid; u < na + 8 * Gp; u += kTcProdThreads) {
                    if (u < na) {
                        // A: w conj(E)[l][h], rows l (M tiles), K = 32 traces
                        const int hh = u & 31, lb = u >> 5;
                        const int p = 32 * c + hh;
                        const int l0 = 8 * lb;
                        const int mt = l0 >> 7;
                        unsigned char *ahi = st0 + (2 * mt) * kTileA, *alo = ahi + kTileA;
                        float2 e[8];
                        if (p < ntot) {
                            const TraceGeo tr = a.geo[p < n1 ? a0 + p : b0 + (p - n1)];
                            const float wgt = p < n1 ? tr.w0 : tr.w1;
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
                    } else {
                        // B: rows (part, g), K = 32 traces x (Re, Im); one unit is
                        // one 16-byte chunk (4 traces) of a row pair
                        const int v = u - na;
                        const int tq = tc_div(v, Gp, inv_gp);
                        const int g = v - tq * Gp;
                        uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int p = 32 * c + 4 * tq + i;
                            float2 y = make_float2(0.f, 0.f);
                            if (p < ntot && g < a.G)
                                y = __ldg(p < n1 ? Ya + (long long)p * a.G + g
                                                 : Yb + (long long)(p - n1) * a.G + g);
                            split_cplx(y.x, y.y, &rh[i], &rl[i], &ih[i], &il[i]);
                        }
                        st_chunk(bhi, g, tq, make_uint4(rh[0], rh[1], rh[2], rh[3]));
                        st_chunk(blo, g, tq, make_uint4(rl[0], rl[1], rl[2], rl[3]));
                        st_chunk(bhi, Gp + g, tq, make_uint4(ih[0], ih[1], ih[2], ih[3]));
                        st_chunk(blo, Gp + g, tq, make_uint4(il[0], il[1], il[2], il[3]));
                    }
                }
                fence_async_smem();
                mbar_arrive(smem_u32(&bars.full[st]));
            }
        }
    } else {
        // ----------------------------------------------------- epilogue
        // X^[l][j][g] = scale * accumulator (zero without traces)
        const int q = warp & 3;
        int it = 0;
        for (long long item = blockIdx.x; item < a.total; item += gridDim.x, ++it) {
            const int ab = it & 1;
            if (!tc_wait_bar(a, &bars.accf[ab], (it >> 1) & 1, abort)) break;
            fence_after_sync();
            const int k = (int)(item / J);
            const int j = (int)(item - (long long)k * J);
            const int jm = j == 0 ? J - 1 : j - 1;
            const int ntot = (a.ss[j + 1] - a.ss[j]) + (a.ss[jm + 1] - a.ss[jm]);
            for (int mt = 0; mt < nmt; ++mt) {
                const int l = 128 * mt + 32 * q + lane;
                const uint32_t base = tm + ((uint32_t)(32 * q) << 16) +
                                      (uint32_t)(ab * acc_cols + mt * N);
                float2 *Xrow =
                    Xh + (((long long)j * a.nbins + k) * a.nq + (l < a.nq ? l : 0)) * a.G;
                for (int gb = 0; gb < Gp; gb += 16) {
                    float re[16], im[16];
                    if (ntot > 0) {
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
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bars.acce[ab]));
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tm, kTcTmemCols);
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
