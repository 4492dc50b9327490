// rqb_chol.cu -- blocked multi-CTA Cholesky of wide panel Gram matrices.
//
// CholeskyQR (Sec. 4.3, lines (3)/(3') of Fig. randQB_b) factors the FP64
// Gram matrix G = Y^T Y of a panel, G = R^T R.  For bp <= 128 the single-CTA
// kernel of rqb_kernels.cu holds G in shared memory; a 256-wide Gram needs
// n^3/3 = 5.6 M FP64 multiply-adds, which one SM (two FP64 FMAs per clock on
// this part) needs about 1.4 ms for.  Here the factorization G = L L^T is
// blocked in 32 x 32 tiles and spread over many CTAs:
//   panel k   every CTA factors the diagonal tile G_kk and inverts L_kk (the
//             whole CTA on the tile in shared memory, one barrier per pivot);
//             CTA 0 stores L_kk and L_kk^{-1}, the others the 8-row strips of
//             L_ik = G_ik L_kk^{-T} below it (and FP32 copies of both when
//             R^{-1} is formed in FP32)
//   update k  G_ij -= L_ik L_jk^T for every tile k < j <= i, one CTA per
//             8-row strip
// R = L^T in FP64.  Each panel also keeps L_kk^{-1}, from which R^{-1} =
// (L^{-1})^T is formed by block forward substitution in the output type.
// An FP32 factorization of up to 256 columns instead holds the whole Gram in
// one CTA's shared memory (k_chol_f32_cta): FP32 has the SM's full FMA rate,
// and the chain of launches, not the arithmetic, bounds the tiled scheme.
#include <cuda_runtime.h>

#include <algorithm>

#include "rqb_engine.h"
#include "rqb_internal.cuh"

namespace rqb {
namespace {

constexpr int kNb = 32;     // tile
constexpr int kStrip = 8;   // rows per CTA in the solves and updates

// Padding rows/columns >= p become the identity; dG = diagonal of G (the
// reference for the relative pivot test); L (when given) cleared; Gf (when
// given) = G rounded to FP32.
__global__ void k_chol_init(double* __restrict__ G, int bp, int p, double* __restrict__ dG,
                            double* __restrict__ L, const int* __restrict__ skip, float* __restrict__ Gf) {
    pdl_trigger();
    pdl_wait();
    if (skip && *skip) return;   // the near-identity expansion gave the factor
    const int total = bp * bp;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int r = e % bp, c = e / bp;
        double g;
        if (r >= p || c >= p) {
            g = (r == c) ? 1.0 : 0.0;
            G[e] = g;
        } else {
            g = G[e];
        }
        if (L) L[e] = 0.0;
        if (Gf) Gf[e] = (float)g;
        if (r == c) dG[r] = g;
    }
}

// 1 / sqrt(d) for d > 0 in FP64: an FP32 estimate refined by two Newton
// steps y <- y (3 - d y^2) / 2 (each about squares the relative error:
// 2^-22 -> 2^-43 -> below the FP64 rounding): a few dependent FP64
// multiply-adds instead of an FP64 square root and division.  The FP32 argument of the estimate and the widening of its result
// are built from the IEEE-754 fields with integer operations (binary64 ->
// binary32 by truncating the significand, binary32 -> binary64 exactly), which
// keeps the FP64 pipe -- a few lanes per clock on this part -- for the Newton
// steps.  Pivots whose binary32 image would not be a normal number take the
// FP64 library route.
__device__ __forceinline__ double rsqrt_fp64(double d) {
    const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
    const int e = (int)(hi >> 20);   // sign and biased exponent (sign 0 for d > 0)
    if (e < 1023 - 120 || e > 1023 + 120) return 1.0 / sqrt(d);
    const float df = __uint_as_float(((uint32_t)(e - 1023 + 127) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
    const uint32_t fb = __float_as_uint(rsqrtf(df));
    double y = __hiloint2double((int)((((fb >> 23) + (1023 - 127)) << 20) | ((fb & 0x7fffffu) >> 3)),
                                (int)(fb << 29));
    const double h = 0.5 * d;
#pragma unroll
    for (int it = 0; it < 2; ++it) y = y * fma(-h, y * y, 1.5);
    return y;
}

// 1 / d for d > 0 in FP64 by the same construction: the FP32 estimate
// refined by two Newton steps y <- y + y (1 - d y) (2^-22 -> 2^-44 -> below
// the FP64 rounding), two dependent FP64 operations per step.
__device__ __forceinline__ double rcp_fp64(double d) {
    const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
    const int e = (int)(hi >> 20);
    if (e < 1023 - 120 || e > 1023 + 120) return 1.0 / d;
    const float df = __uint_as_float(((uint32_t)(e - 1023 + 127) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
    const uint32_t fb = __float_as_uint(__frcp_rn(df));
    double y = __hiloint2double((int)((((fb >> 23) + (1023 - 127)) << 20) | ((fb & 0x7fffffu) >> 3)),
                                (int)(fb << 29));
#pragma unroll
    for (int it = 0; it < 2; ++it) y = fma(y, fma(-d, y, 1.0), y);
    return y;
}

// rcp_fp64 and rsqrt_fp64 over an array, for the test that holds them to
// their error bounds (entry point rqb_fp64_recip_selftest).
__global__ void k_recip_selftest(const double* __restrict__ x, int64_t count, double* __restrict__ rcp,
                                 double* __restrict__ rsq) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        rcp[i] = rcp_fp64(x[i]);
        rsq[i] = rsqrt_fp64(x[i]);
    }
}

template <typename W>
__global__ void __launch_bounds__(256) k_chol_panel(const double* __restrict__ G, double* __restrict__ L,
                                                    double* __restrict__ Linv, float* __restrict__ Lf,
                                                    float* __restrict__ Lif, int bp, int k,
                                                    const double* __restrict__ dG, double tol, DevState* st,
                                                    const int* __restrict__ skip) {
    pdl_trigger();
    pdl_wait();
    if (skip && *skip) return;   // the near-identity expansion gave the factor
    __shared__ W D[kNb][kNb + 1];    // L_kk (lower)
    __shared__ W Di[kNb][kNb + 1];   // L_kk^{-1} (lower)
    __shared__ W inv[kNb];
    __shared__ int fail;
    const int tid = threadIdx.x;
    const int k0 = k * kNb;
    // strip CTAs: row `srow` of G_ik is loaded before the factorization so
    // that the loads overlap it (thread (rr, c) needs all 32 entries of its row)
    const bool strip = blockIdx.x > 0;
    const int bi = strip ? (blockIdx.x - 1) / (kNb / kStrip) : 0, sq = strip ? (blockIdx.x - 1) % (kNb / kStrip) : 0;
    const int srow = (k + 1 + bi) * kNb + sq * kStrip + (tid >> 5);
    W gv[kNb];
    if (strip) {
#pragma unroll
        for (int t = 0; t < kNb; ++t) gv[t] = (W)G[srow + (int64_t)(k0 + t) * bp];
    }
    {
        // The tile in shared memory, one barrier per pivot.  The elimination
        // runs unscaled: D keeps the Schur complements and Di the unscaled
        // rows of L^{-1} (step j subtracts D[r][j] D[c][j] / pivot_j and
        // D[r][j] Di[j][c] / pivot_j).  Thread 0 owns the serial chain: it
        // updates D[j+1][j+1] and takes the next pivot at once, while six
        // other warps update the other active entries, so the chain never
        // queues behind a warp's elimination work.  The factors are scaled by pivot^{-1/2} at the end.  A pivot
        // that fails the test sets `fail` without stopping the chain (the
        // factorization is then reported and discarded).  FP64 keeps the
        // FP64 pipes of all four SM sub-partitions busy; FP32 (the second
        // CholeskyQR pass) is bound by the chain and the barriers.
        __shared__ W invp[kNb];
        __shared__ W thr[kNb];
        for (int e = tid; e < kNb * kNb; e += 256) {
            const int r = e & (kNb - 1), c = e / kNb;
            D[r][c] = (r >= c) ? (W)G[(k0 + r) + (int64_t)(k0 + c) * bp] : W(0);
            Di[r][c] = (r == c) ? W(1) : W(0);
        }
        if (tid < kNb) thr[tid] = (W)(tol * dG[k0 + tid]);
        if (tid == 0) fail = 0;
        __syncthreads();
        // the chain needs 1 / pivot only (the elimination runs unscaled);
        // pivot^{-1/2} for the final scaling is formed after the loop
        auto take_pivot = [&](int j, W d) {
            if constexpr (sizeof(W) == 8) {
                invp[j] = rcp_fp64(d);
            } else {
                // FP32: the hardware estimate and one Newton step
                const float y = __frcp_rn(d);
                invp[j] = fmaf(y, fmaf(-d, y, 1.f), y);
            }
            if (!(d > thr[j]) || !isfinite(d)) fail = 1;   // issued after the chain's operations
        };
        if (tid == 0) take_pivot(0, D[0][0]);
        __syncthreads();
        // workers: the six warps of sub-partitions 1..3 (warp w runs on
        // sub-partition w % 4), so the chain of thread 0 has sub-partition 0's
        // pipes alone.  Worker warp u owns the columns c = u (mod 6) of D and
        // of Di, lane r their row r: a thread's active entries at step j
        // share one multiplier D[r][j] / pivot_j, and all its operands are
        // conflict-free or broadcast shared-memory reads.
        const int wid = tid >> 5, lane = tid & 31;
        const int u = (wid & 3) ? ((wid >> 2) * 3 + (wid & 3) - 1) : -1;
        for (int j = 0; j < kNb; ++j) {
            const W ip = invp[j];
            if (tid == 0) {
                if (j + 1 < kNb) {
                    const W l = D[j + 1][j];
                    const W nv = fma(-(l * ip), l, D[j + 1][j + 1]);
                    D[j + 1][j + 1] = nv;
                    take_pivot(j + 1, nv);
                }
            } else if (u >= 0 && lane > j) {
                const int r = lane;
                const W a = D[r][j] * ip;
                // this thread's columns c = u + 6 i: every operand is read
                // before the first update is stored, so the six updates
                // overlap instead of running as a chain of dependent accesses
                W x[6], y[6];
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    const int c = u + 6 * i;
                    if (c < kNb) {
                        x[i] = (c > j) ? D[c][j] : Di[j][c];
                        y[i] = (c > j) ? D[r][c] : Di[r][c];
                    }
                }
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    const int c = u + 6 * i;
                    if (c < kNb) {
                        const W v = fma(-a, x[i], y[i]);
                        if (c > j) {
                            // the trailing triangle j < c <= r; its one entry in
                            // row j + 1, (j+1, j+1), is thread 0's
                            if (r >= c && r != j + 1) D[r][c] = v;
                        } else {
                            Di[r][c] = v;
                        }
                    }
                }
            }
            __syncthreads();
        }
        if (tid < kNb) {   // D[c][c] holds pivot c
            const W d = D[tid][tid];
            if constexpr (sizeof(W) == 8) {
                inv[tid] = rsqrt_fp64(d);
            } else {
                const float y = rsqrtf(d);
                inv[tid] = y * fmaf(-0.5f * d, y * y, 1.5f);
            }
        }
        __syncthreads();
        for (int e = tid; e < kNb * kNb; e += 256) {
            const int r = e & (kNb - 1), c = e / kNb;
            if (r >= c) {
                D[r][c] *= inv[c];
                Di[r][c] *= inv[r];
            }
        }
        __syncthreads();
    }
    if (!strip) {
        for (int e = tid; e < kNb * kNb; e += 256) {
            const int r = e & (kNb - 1), c = e / kNb;
            if (r >= c) {
                const int64_t o = (k0 + r) + (int64_t)(k0 + c) * bp;
                L[o] = (double)D[r][c];
                Linv[o] = (double)Di[r][c];
                if (Lf) {
                    Lf[o] = (float)D[r][c];
                    Lif[o] = (float)Di[r][c];
                }
            }
        }
        if (tid == 0 && fail) record_error(st, RQB_ERR_BREAKDOWN);
        return;
    }
    // strip sq of tile row i: L_ik(rows) = G_ik(rows) L_kk^{-T}
    const int c = tid & 31;
    W s = W(0);
#pragma unroll
    for (int t = 0; t < kNb; ++t) s += gv[t] * Di[c][t];
    L[srow + (int64_t)(k0 + c) * bp] = (double)s;
    if (Lf) Lf[srow + (int64_t)(k0 + c) * bp] = (float)s;
}

// G_ij -= L_ik L_jk^T on the 8-row strip (blockIdx.x % 4) of tile pair
// (i, j), k < j <= i < nblk, pairs enumerated column by column.
template <typename W>
__global__ void __launch_bounds__(256) k_chol_update(double* __restrict__ G, const double* __restrict__ L, int bp,
                                                     int k, int nblk, const int* __restrict__ skip) {
    pdl_trigger();
    pdl_wait();
    if (skip && *skip) return;   // the near-identity expansion gave the factor
    __shared__ W Lj[kNb][kNb + 1];
    int pair = blockIdx.x / (kNb / kStrip);
    const int q = blockIdx.x % (kNb / kStrip);
    int j = k + 1;
    while (pair >= nblk - j) {
        pair -= nblk - j;
        ++j;
    }
    const int i = j + pair;
    const int k0 = k * kNb;
    const int tid = threadIdx.x;
    for (int e = tid; e < kNb * kNb; e += 256) {
        const int c = e & (kNb - 1), t = e / kNb;
        Lj[c][t] = (W)L[(j * kNb + c) + (int64_t)(k0 + t) * bp];
    }
    __syncthreads();
    const int rr = tid >> 5, c = tid & 31;
    const int row = i * kNb + q * kStrip + rr;
    W s = W(0);
#pragma unroll 8
    for (int t = 0; t < kNb; ++t) s += (W)L[row + (int64_t)(k0 + t) * bp] * Lj[c][t];
    G[row + (int64_t)(j * kNb + c) * bp] -= (double)s;
}

// ---------------------------------------------------------------------------
// FP32 factor of a Gram of at most 256 columns on one CTA.  The lower 32 x 32
// tiles of G (FP32) stay in shared memory, each stored by columns with a
// stride of kTs floats; for each tile column k: the diagonal tile is
// factored by one warp in registers (tile_factor_warp, L_kk^{-1} alongside),
// the tiles below it are solved,
// L_ik = G_ik L_kk^{-T}, and the trailing tiles updated, G_ij -= L_ik L_jk^T
// (k < j <= i), each by a 64-thread group with 4 x 4 outputs per thread fed
// by 16-byte shared-memory reads and packed FP32 FMAs.  No launch and no
// global round trip separates the tile columns, which a chain of panel and
// update kernels pays for at every tile.
constexpr int kTs = 36;                // column stride of a tile in shared memory (floats)
constexpr int kTileF = kNb * kTs;      // floats per tile
constexpr int kCtaThreads = 512;

__host__ __device__ constexpr int tri_tile(int i, int j) { return i * (i + 1) / 2 + j; }

size_t chol_f32_cta_smem(int bp) {
    const int nblk = bp / kNb;
    return sizeof(float) * (size_t)(nblk * (nblk + 1) / 2 + 1) * kTileF;
}

// Tile number t -> (i, j), j <= i, in the order of tri_tile.
__device__ __forceinline__ void tile_ij(int t, int* i, int* j) {
    int a = 0;
    while ((a + 1) * (a + 2) / 2 <= t) ++a;
    *i = a;
    *j = t - a * (a + 1) / 2;
}

// The diagonal tile's factor on one warp, without block barriers: lane r
// holds row r of the tile (d[c] = D(r, c)) and of its inverse (w[c]), both in
// registers.  Unscaled elimination: step j takes pivot D(j, j) from lane j
// and, for r > j, subtracts D(r, j) / pivot_j times column j's entries D(c, j)
// (c > j, from lane c) from D(r, c), and times row j of the inverse (from
// lane j) from w; rows are scaled by pivot^{-1/2} at the end.  thr: this
// lane's pivot threshold; a pivot at or below it, or not finite, sets *fail.
// Entries above the diagonal are read and updated but not used, and are
// stored as zeros.
__device__ __forceinline__ void tile_factor_warp(float* __restrict__ D, float* __restrict__ Di, float thr, int lane,
                                                 int* fail) {
    float d[kNb], w[kNb];
#pragma unroll
    for (int c = 0; c < kNb; ++c) {
        d[c] = D[c * kTs + lane];
        w[c] = (c == lane) ? 1.f : 0.f;
    }
    bool bad = false;
#pragma unroll
    for (int j = 0; j < kNb; ++j) {
        const float pj = __shfl_sync(0xffffffffu, d[j], j);
        const float y = __frcp_rn(pj);
        const float ip = fmaf(y, fmaf(-pj, y, 1.f), y);
        if (lane == j && (!(pj > thr) || !isfinite(pj))) bad = true;
        const float a = (lane > j) ? d[j] * ip : 0.f;
#pragma unroll
        for (int c = j + 1; c < kNb; ++c) d[c] = fmaf(-a, __shfl_sync(0xffffffffu, d[j], c), d[c]);
#pragma unroll
        for (int c = 0; c <= j; ++c) w[c] = fmaf(-a, __shfl_sync(0xffffffffu, w[c], j), w[c]);
    }
    float dd = 0.f;
#pragma unroll
    for (int c = 0; c < kNb; ++c) dd = (c == lane) ? d[c] : dd;
    const float yy = rsqrtf(dd);
    const float inv = yy * fmaf(-0.5f * dd, yy * yy, 1.5f);
#pragma unroll
    for (int c = 0; c < kNb; ++c) {
        const float ic = __shfl_sync(0xffffffffu, inv, c);
        D[c * kTs + lane] = (lane >= c) ? d[c] * ic : 0.f;
        Di[c * kTs + lane] = (lane >= c) ? w[c] * inv : 0.f;
    }
    if (bad) *fail = 1;
}

// Gf: bp x bp (ld bp, FP32, lower triangle read); writes the lower tiles of
// L to Lf and the diagonal tiles of L^{-1} (that is, L_kk^{-1}) to Lif, both
// bp x bp ld bp; a pivot at or below tol * dG or not finite records
// RQB_ERR_BREAKDOWN (the factorization then runs on and is discarded).
__global__ void __launch_bounds__(kCtaThreads, 1)
k_chol_f32_cta(const float* __restrict__ Gf, int bp, const double* __restrict__ dG, double tol,
               float* __restrict__ Lf, float* __restrict__ Lif, DevState* st, const int* __restrict__ skip) {
    pdl_trigger();
    pdl_wait();
    if (skip && *skip) return;   // the near-identity expansion gave the factor
    extern __shared__ __align__(16) float csm[];
    const int nblk = bp / kNb, ntile = nblk * (nblk + 1) / 2;
    float* T = csm;                               // tile (i, j) at T + tri_tile(i, j) kTileF, (r, c) at [c kTs + r]
    float* Di = csm + (size_t)ntile * kTileF;     // L_kk^{-1} of the current column, same layout
    __shared__ int fail;
    __shared__ float thrs[8 * kNb];   // pivot thresholds tol * dG, all columns
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    for (int r = tid; r < bp; r += kCtaThreads) thrs[r] = (float)(tol * dG[r]);
    for (int e = tid; e < ntile * kNb * (kNb / 4); e += kCtaThreads) {
        const int v = e & 7, c = (e >> 3) & 31, t = e >> 8;
        int i, j;
        tile_ij(t, &i, &j);
        cp_async16(T + (size_t)t * kTileF + c * kTs + 4 * v, Gf + (size_t)(i * kNb + 4 * v) + (size_t)(j * kNb + c) * bp,
                   16);
    }
    cp_async_commit();
    if (tid == 0) fail = 0;
    cp_async_wait<0>();
    __syncthreads();
    for (int k = 0; k < nblk; ++k) {
        const int k0 = k * kNb;
        if (wid == 0) tile_factor_warp(T + (size_t)tri_tile(k, k) * kTileF, Di, thrs[k0 + lane], lane, &fail);
        __syncthreads();
        for (int e = tid; e < kNb * (kNb / 4); e += kCtaThreads) {
            const int v = e & 7, c = e >> 3;
            *reinterpret_cast<float4*>(Lif + (size_t)(k0 + 4 * v) + (size_t)(k0 + c) * bp) =
                *reinterpret_cast<const float4*>(Di + c * kTs + 4 * v);
        }
        // L_ik = G_ik L_kk^{-T}: each half of the CTA takes every other tile
        // i > k, thread (r, columns 4 cg .. 4 cg + 3); a half's named barrier
        // orders its reads of a tile before its stores to it (the halves
        // never share a tile)
        {
            const int half = tid >> 8, r = tid & 31, cg = (tid >> 5) & 7;
            for (int i = k + 1 + half; i < nblk; i += 2) {
                float* Tik = T + (size_t)tri_tile(i, k) * kTileF;
                float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
                for (int t = 0; t < kNb; ++t) {
                    const float g = Tik[t * kTs + r];
                    const float4 l = *reinterpret_cast<const float4*>(Di + t * kTs + 4 * cg);
                    acc[0] = fmaf(g, l.x, acc[0]);
                    acc[1] = fmaf(g, l.y, acc[1]);
                    acc[2] = fmaf(g, l.z, acc[2]);
                    acc[3] = fmaf(g, l.w, acc[3]);
                }
                asm volatile("bar.sync %0, %1;" ::"r"(1 + half), "r"(kCtaThreads / 2) : "memory");
#pragma unroll
                for (int q = 0; q < 4; ++q) Tik[(4 * cg + q) * kTs + r] = acc[q];
            }
        }
        __syncthreads();
        // G_ij -= L_ik L_jk^T, k < j <= i: group g of 64 threads per tile pair,
        // thread (rb, cb) rows 4 rb .. 4 rb + 3, columns 4 cb .. 4 cb + 3
        const int mrem = nblk - 1 - k, npair = mrem * (mrem + 1) / 2;
        const int g = tid >> 6, l = tid & 63, rb = l & 7, cb = l >> 3;
        for (int pr = g; pr < npair; pr += kCtaThreads / 64) {
            int jj = 0, rem = pr;
            while (rem >= mrem - jj) {
                rem -= mrem - jj;
                ++jj;
            }
            const int j = k + 1 + jj, i = j + rem;
            const float* Li = T + (size_t)tri_tile(i, k) * kTileF;
            const float* Lj = T + (size_t)tri_tile(j, k) * kTileF;
            float* Tij = T + (size_t)tri_tile(i, j) * kTileF;
            float2 acc[4][2];
#pragma unroll
            for (int a = 0; a < 4; ++a) acc[a][0] = acc[a][1] = make_float2(0.f, 0.f);
#pragma unroll 8
            for (int t = 0; t < kNb; ++t) {
                const float4 a = *reinterpret_cast<const float4*>(Li + t * kTs + 4 * rb);
                const float4 b = *reinterpret_cast<const float4*>(Lj + t * kTs + 4 * cb);
                const float2 b01 = make_float2(b.x, b.y), b23 = make_float2(b.z, b.w);
                const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float2 aa = make_float2(av[q], av[q]);
                    acc[q][0] = __ffma2_rn(aa, b01, acc[q][0]);
                    acc[q][1] = __ffma2_rn(aa, b23, acc[q][1]);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {   // column 4 cb + q, rows 4 rb .. 4 rb + 3
                float4* dst = reinterpret_cast<float4*>(Tij + (4 * cb + q) * kTs + 4 * rb);
                float4 v = *dst;
                const int h = q >> 1;
                v.x -= (q & 1) ? acc[0][h].y : acc[0][h].x;
                v.y -= (q & 1) ? acc[1][h].y : acc[1][h].x;
                v.z -= (q & 1) ? acc[2][h].y : acc[2][h].x;
                v.w -= (q & 1) ? acc[3][h].y : acc[3][h].x;
                *dst = v;
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < ntile * kNb * (kNb / 4); e += kCtaThreads) {
        const int v = e & 7, c = (e >> 3) & 31, t = e >> 8;
        int i, j;
        tile_ij(t, &i, &j);
        *reinterpret_cast<float4*>(Lf + (size_t)(i * kNb + 4 * v) + (size_t)(j * kNb + c) * bp) =
            *reinterpret_cast<const float4*>(T + (size_t)t * kTileF + c * kTs + 4 * v);
    }
    if (tid == 0 && fail) record_error(st, RQB_ERR_BREAKDOWN);
}

// R = L^T (FP64, column-major, upper) from the FP32 L of k_chol_f32_cta
// (lower triangle of Lf read).
__global__ void k_chol_transpose_f32(const float* __restrict__ Lf, int bp, double* __restrict__ R,
                                     const int* __restrict__ skip) {
    pdl_trigger();
    pdl_wait();
    if (skip && *skip) return;   // the near-identity expansion gave the factor
    const int total = bp * bp;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int r = e % bp, c = e / bp;
        R[e] = (r <= c) ? (double)Lf[c + (int64_t)r * bp] : 0.0;
    }
}

// R = L^T (FP64, column-major, upper).
__global__ void k_chol_transpose(const double* __restrict__ L, int bp, double* __restrict__ R,
                                 const int* __restrict__ skip) {
    pdl_trigger();
    pdl_wait();
    if (skip && *skip) return;   // the near-identity expansion gave the factor
    const int total = bp * bp;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int r = e % bp, c = e / bp;
        R[e] = (r <= c) ? L[c + (int64_t)r * bp] : 0.0;
    }
}

// Rinv = R^{-1} for upper-triangular R (FP64, column-major): with L = R^T,
// warp w of CTA b computes column c = b * 8 + w of L^{-1} by forward
// substitution down the column (row c of R^{-1}), with L staged in shared
// memory in working type W, columns packed (column t holds rows t .. bp-1).
template <typename T, typename W>
__global__ void __launch_bounds__(256) k_upper_inverse(const double* __restrict__ R, int bp, T* __restrict__ Rinv) {
    extern __shared__ __align__(16) unsigned char inv_smem[];
    W* Ls = reinterpret_cast<W*>(inv_smem);
    W* xs = Ls + (size_t)bp * (bp + 1) / 2;                  // 8 x bp
    auto off = [bp](int t) { return (size_t)t * bp - (size_t)t * (t - 1) / 2; };
    // R[t + r bp] = L[r][t]; flat loop over R for coalesced reads
    for (int e = threadIdx.x; e < bp * bp; e += 256) {
        const int t = e % bp, r = e / bp;
        if (r >= t) Ls[off(t) + (r - t)] = (W)R[e];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * 8 + warp;
    if (c >= bp) return;
    W* x = xs + (size_t)warp * bp;
    for (int r = lane; r < bp; r += 32) x[r] = (r == c) ? W(1) : W(0);
    __syncwarp();
    for (int t = c; t < bp; ++t) {
        const W* Lt = Ls + off(t);          // L[t..bp-1][t]
        const W xt = x[t] / Lt[0];
        __syncwarp();
        for (int r = t + 1 + lane; r < bp; r += 32) x[r] -= Lt[r - t] * xt;
        if (lane == 0) x[t] = xt;
        __syncwarp();
    }
    for (int r = lane; r < bp; r += 32) Rinv[c + (int64_t)r * bp] = (T)((r >= c) ? x[r] : W(0));
}

// Rinv = R^{-1} = (L^{-1})^T from the tiles of L and the inverses of its
// diagonal tiles (written by the panels): CTA j forms column block j of
// X = L^{-1} down the block rows, X_jj = L_jj^{-1} and
// X_ij = -L_ii^{-1} sum_{j <= t < i} L_it X_tj (block forward substitution),
// in working type W with the block row of L staged in shared memory, and
// stores it transposed.
template <typename T, typename W>
__global__ void __launch_bounds__(256) k_linv_blocked(const double* __restrict__ L, const double* __restrict__ Linv,
                                                      int bp, T* __restrict__ Rinv, const int* __restrict__ skip) {
    pdl_trigger();
    pdl_wait();
    if (skip && *skip) return;   // the near-identity expansion gave the factor
    extern __shared__ __align__(16) unsigned char linv_smem[];
    W* X = reinterpret_cast<W*>(linv_smem);          // bp x 32, column block j of L^{-1}, ld bp
    W* Lr = X + (size_t)bp * kNb;                     // 32 x bp block row of L, ld 33 (row-padded)
    W* S = Lr + (size_t)bp * (kNb + 1);               // 32 x 32 partial sum, ld 33
    W* Di = S + (size_t)kNb * (kNb + 1);              // 32 x 32 L_ii^{-1}, ld 33
    const int j = blockIdx.x, nblk = bp / kNb;
    const int tid = threadIdx.x;
    const int j0 = j * kNb;
    for (int e = tid; e < bp * kNb; e += 256) {
        const int r = e % bp, c = e / bp;
        X[r + (size_t)c * bp] = (r >= j0 && r < j0 + kNb && r - j0 >= c) ? (W)Linv[r + (int64_t)(j0 + c) * bp] : W(0);
    }
    const int r = tid & 31, cg = tid >> 5;    // output row r, columns cg + 8 q
    for (int i = j + 1; i < nblk; ++i) {
        const int i0 = i * kNb, len = i0 - j0;
        __syncthreads();     // X rows of block i-1 complete; Lr, Di free
        for (int e = tid; e < kNb * len; e += 256) {
            const int rr = e & (kNb - 1), t = e >> 5;
            Lr[t * (kNb + 1) + rr] = (W)L[(i0 + rr) + (int64_t)(j0 + t) * bp];
        }
        for (int e = tid; e < kNb * kNb; e += 256) {
            const int rr = e & (kNb - 1), t = e >> 5;
            Di[t * (kNb + 1) + rr] = (W)Linv[(i0 + rr) + (int64_t)(i0 + t) * bp];
        }
        __syncthreads();
        W acc[4] = {W(0), W(0), W(0), W(0)};
        for (int t0 = 0; t0 < len; t0 += kNb) {
#pragma unroll 8
            for (int t = t0; t < t0 + kNb; ++t) {
                const W l = Lr[t * (kNb + 1) + r];
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[q] += l * X[(j0 + t) + (size_t)(cg + 8 * q) * bp];
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) S[r + (cg + 8 * q) * (kNb + 1)] = acc[q];
        __syncthreads();
        W out[4] = {W(0), W(0), W(0), W(0)};
#pragma unroll 8
        for (int t = 0; t < kNb; ++t) {
            const W dv = (t <= r) ? Di[t * (kNb + 1) + r] : W(0);
#pragma unroll
            for (int q = 0; q < 4; ++q) out[q] += dv * S[t + (cg + 8 * q) * (kNb + 1)];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) X[(i0 + r) + (size_t)(cg + 8 * q) * bp] = -out[q];
    }
    __syncthreads();
    // Rinv(c, r) = X(r, c): row j0 + c of Rinv, columns r >= j0
    for (int e = tid; e < bp * kNb; e += 256) {
        const int c = e % kNb, rr = e / kNb;
        Rinv[(j0 + c) + (int64_t)rr * bp] = (T)X[rr + (size_t)c * bp];
    }
}

// Rinv = R^{-1} = (L^{-1})^T in FP32, by the block forward substitution of
// k_linv_blocked, from the FP32 copies of L and of the diagonal-tile inverses
// that the panels write (no FP64 loads or conversions).  CTA j forms column
// block j of X = L^{-1}; the block row of L and L_ii^{-1} of step i + 1 are
// copied by cp.async while step i multiplies.  X and the step's partial sum S
// are row-major with rows padded to 36 floats, and thread (r, g) owns row r,
// columns 4g .. 4g + 3, so that each operand of a multiply-add is one 16-byte
// broadcast read or one conflict-free 4-byte read.
constexpr int kXs = 36;   // padded row of X and S (floats)

__global__ void __launch_bounds__(256) k_linv_f32(const float* __restrict__ Lf, const float* __restrict__ Lif, int bp,
                                                  float* __restrict__ Rinv, const int* __restrict__ skip) {
    pdl_trigger();
    pdl_wait();
    if (skip && *skip) return;   // the near-identity expansion gave the factor
    extern __shared__ __align__(16) unsigned char linvf_smem[];
    float* X = reinterpret_cast<float*>(linvf_smem);   // bp x 36
    float* Lr = X + (size_t)bp * kXs;                  // [2][bp][32]: Lr[t][rr] = L(i0 + rr, j0 + t)
    float* Dv = Lr + 2 * (size_t)bp * kNb;             // [2][32][32]: Dv[t][rr] = L_ii^{-1}(rr, t)
    float* S = Dv + 2 * kNb * kNb;                      // 32 x 36
    const int j = blockIdx.x, nblk = bp / kNb, tid = threadIdx.x, j0 = j * kNb;
    auto issue = [&](int i, int b) {
        const int i0 = i * kNb, len = i0 - j0;
        float* lr = Lr + (size_t)b * bp * kNb;
        for (int e = tid; e < len * 8; e += 256) {   // 8 vectors of 4 rows per column
            const int t = e >> 3, v = (e & 7) * 4;
            cp_async16(lr + t * kNb + v, Lf + (i0 + v) + (int64_t)(j0 + t) * bp, 16);
        }
        float* dv = Dv + b * kNb * kNb;
        for (int e = tid; e < kNb * 8; e += 256) {
            const int t = e >> 3, v = (e & 7) * 4;
            cp_async16(dv + t * kNb + v, Lif + (i0 + v) + (int64_t)(i0 + t) * bp, 16);
        }
        cp_async_commit();
    };
    if (j + 1 < nblk) issue(j + 1, 0);
    for (int e = tid; e < bp * kNb; e += 256) {
        const int c = e % kNb, r = e / kNb;
        X[r * kXs + c] = (r >= j0 && r < j0 + kNb && r - j0 >= c) ? Lif[r + (int64_t)(j0 + c) * bp] : 0.f;
    }
    const int r = tid & 31, g = tid >> 5;   // row r, columns 4g .. 4g + 3
    for (int i = j + 1; i < nblk; ++i) {
        const int b = (i - j - 1) & 1, i0 = i * kNb, len = i0 - j0;
        cp_async_wait<0>();
        __syncthreads();   // step i's operands landed; X rows of block i - 1 and S are complete / free
        if (i + 1 < nblk) issue(i + 1, b ^ 1);
        const float* lr = Lr + (size_t)b * bp * kNb;
        const float* dv = Dv + b * kNb * kNb;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 8
        for (int t = 0; t < len; ++t) {
            const float l = lr[t * kNb + r];
            const float4 x = *reinterpret_cast<const float4*>(X + (j0 + t) * kXs + 4 * g);
            acc.x = fmaf(l, x.x, acc.x);
            acc.y = fmaf(l, x.y, acc.y);
            acc.z = fmaf(l, x.z, acc.z);
            acc.w = fmaf(l, x.w, acc.w);
        }
        *reinterpret_cast<float4*>(S + r * kXs + 4 * g) = acc;
        __syncthreads();
        float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 8
        for (int t = 0; t < kNb; ++t) {
            const float d = (t <= r) ? dv[t * kNb + r] : 0.f;
            const float4 sv = *reinterpret_cast<const float4*>(S + t * kXs + 4 * g);
            out.x = fmaf(d, sv.x, out.x);
            out.y = fmaf(d, sv.y, out.y);
            out.z = fmaf(d, sv.z, out.z);
            out.w = fmaf(d, sv.w, out.w);
        }
        *reinterpret_cast<float4*>(X + (i0 + r) * kXs + 4 * g) = make_float4(-out.x, -out.y, -out.z, -out.w);
    }
    __syncthreads();
    // Rinv(j0 + c, rr) = X(rr, c)
    for (int e = tid; e < bp * kNb; e += 256) {
        const int c = e % kNb, rr = e / kNb;
        Rinv[(j0 + c) + (int64_t)rr * bp] = X[rr * kXs + c];
    }
}

// Second CholeskyQR pass on a near-identity Gram (Sec. 4.3): after the first
// pass, G = Y1^T Y1 = I + E with E of the order of that pass's rounding.
// With U the upper triangle of E and its diagonal halved (U + U^T = E),
// R = I + U gives R^T R = I + E + U^T U, so R is the Cholesky factor of G up
// to O(||E||^2), and R^{-1} = I - U up to O(||E||^2).  When ||E||_F <= tau,
// with tau^2 below the working precision's unit roundoff, the factor is taken
// from this expansion (in FP64, from G's own entries) and the elimination is
// skipped; FP32 factors up to ||E||_F = 2e-2 take the expansion iterated to
// convergence (k_near_id_step); otherwise the elimination runs as before.
// Rows and columns >= p are the identity.

// part[b] = sum of (G_rc - delta_rc)^2 over CTA b's share of the p x p block.
__global__ void __launch_bounds__(256) k_near_id_norm(const double* __restrict__ G, int bp, int p,
                                                      double* __restrict__ part) {
    pdl_trigger();
    pdl_wait();
    __shared__ double sh[8];
    double acc = 0.0;
    const int total = p * p;
    for (int e = blockIdx.x * 256 + threadIdx.x; e < total; e += gridDim.x * 256) {
        const int r = e % p, c = e / p;
        const double d = G[r + (int64_t)c * bp] - (r == c ? 1.0 : 0.0);
        acc = fma(d, d, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sh[w];
        part[blockIdx.x] = t;
    }
}

// Every CTA sums the parts in order and takes the same decision:
//   ||E||_F^2 <= tau2:  first order, the CTAs write their share of R = I + U
//                       (FP64) and R^{-1} = I - U (T); *skip = 1, *iter = 0;
//   <= tau2i:           the iterated expansion (k_near_id_step): the CTAs
//                       write E (FP32) to Ef and the first iterate U to X;
//                       *skip = 1, *iter = 1;
//   else:               *skip = 0, *iter = 0 (the elimination runs).
template <typename T>
__global__ void __launch_bounds__(256) k_near_id_apply(const double* __restrict__ G, int bp, int p,
                                                       const double* __restrict__ part, double tau2, double tau2i,
                                                       double* __restrict__ R, T* __restrict__ Rinv,
                                                       float* __restrict__ Ef, float* __restrict__ X,
                                                       int* __restrict__ skip, int* __restrict__ iter,
                                                       DevState* st) {
    pdl_trigger();
    pdl_wait();
    __shared__ int mode;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < kNearIdParts; ++b) t += part[b];
        mode = (t <= tau2) ? 1 : (t <= tau2i) ? 2 : 0;   // 0 for a NaN norm
        if (blockIdx.x == 0) {
            *skip = mode != 0;
            // steps of the iterated route for a 2e-9 error (e = ||E||_F,
            // ||X|| <= e / sqrt(2), the map contracting by sqrt(2) e): s
            // fixed-point steps after X_1 leave (sqrt(2) e)^s e^2 / 2, and the
            // series to (-X)^(s+1) leaves (e / sqrt(2))^(s+2) (in numpy the
            // worst of rank-one, rank-four, diagonal and dense E at these
            // thresholds was 5e-11)
            const double e = sqrt(t);
            const int nx = (e <= 1.4e-3) ? 1 : (e <= 6.7e-3) ? 2 : 3;
            const int nz = (e <= 1.7e-3) ? 1 : (e <= 9.4e-3) ? 2 : 3;
            *iter = (mode == 2) ? (nx | (nz << 4)) : 0;
            if (mode != 0 && st) atomicAdd(&st->near_id, 1);
        }
    }
    __syncthreads();
    if (mode == 0) return;
    const int total = bp * bp;
    for (int e = blockIdx.x * 256 + threadIdx.x; e < total; e += gridDim.x * 256) {
        const int r = e % bp, c = e / bp;
        const bool in = r < p && c < p;
        double u = 0.0;                      // U_rc
        if (in) {
            if (r < c) u = G[e];
            else if (r == c) u = 0.5 * (G[e] - 1.0);
        }
        if (mode == 1) {
            const double id = (r == c) ? 1.0 : 0.0;
            R[e] = (r <= c) ? id + u : 0.0;
            Rinv[e] = (T)((r <= c) ? id - u : 0.0);
        } else {
            Ef[e] = in ? (float)(G[e] - (r == c ? 1.0 : 0.0)) : 0.f;
            X[e] = (float)u;
            if (r > c) {   // the steps write the upper triangles only
                R[e] = 0.0;
                Rinv[e] = T(0);
            }
        }
    }
}

// One step of the iterated expansion on the 32 x 32 tiles (I, J), I <= J, of
// bp x bp upper-triangular FP32 matrices (column-major), one tile per CTA; it
// runs only when *iter is set.
//   MODE 0, the fixed point X = Phi(E - X^T X) of R = I + X (Phi: the upper
//          triangle with the diagonal halved): Out = Phi(Ef - In^T In); the
//          last step also writes R = I + Out (FP64) and Z = I - Out.
//   MODE 1, R^{-1} = sum_j (-X)^j by Horner: Out = I - X In; the last step
//          also writes Rinv = Out.
// From X_1 = Phi(E) the k-th iterate is within ||E||^(k+1) / 2 of the exact
// X (the map contracts by about ||E||), and j terms of the series leave
// ||X||^(j+1): at ||E||_F <= 2e-2, X_4 and four terms are within 2e-9.  The
// apply kernel sets how many steps of each kind a panel needs for that.
template <int MODE, typename T>
__global__ void __launch_bounds__(256) k_near_id_step(const float* __restrict__ Ef, const float* __restrict__ Xa,
                                                      const float* __restrict__ Xb, const float* __restrict__ In,
                                                      float* __restrict__ Out, int bp, int k,
                                                      double* __restrict__ R, float* __restrict__ Z,
                                                      T* __restrict__ Rinv, const int* __restrict__ iter) {
    pdl_trigger();
    pdl_wait();
    // *iter: fixed-point steps in bits 0..3, series steps in bits 4..7 (0:
    // the iterated route is off); this launch is step k of its kind
    const int nsteps = (MODE == 0) ? (*iter & 15) : ((*iter >> 4) & 15);
    if (k >= nsteps) return;
    const bool last = (k == nsteps - 1);
    // the final fixed-point iterate is in Xb after one or three steps, in Xa after two
    const float* X = ((*iter & 15) == 2) ? Xa : Xb;
    // all the operand tiles of this output tile are loaded at once (up to
    // 2 x 8 tiles, every load in flight together), then multiplied
    extern __shared__ float nis[];
    constexpr int kT = kNb * (kNb + 1);   // one padded 32 x 33 tile
    int J = 0;
    while ((J + 1) * (J + 2) / 2 <= (int)blockIdx.x) ++J;
    const int I = (int)blockIdx.x - J * (J + 1) / 2;
    const int tid = threadIdx.x, lr = tid & 31, lc = (tid >> 5) * 4;
    // MODE 0: sum over l of In(l, i) In(l, j), l <= i; MODE 1: X(i, l) In(l, j), i <= l <= j
    const int L0 = (MODE == 0) ? 0 : I, L1 = (MODE == 0) ? I : J, nL = L1 - L0 + 1;
    float* As = nis;              // tile L: As[L][l][r]
    float* Bs = nis + nL * kT;    // tile L: Bs[L][l][c]
    for (int e = tid; e < nL * kNb * kNb; e += 256) {
        const int L = L0 + e / (kNb * kNb), a = e & 31, b2 = (e >> 5) & 31;
        float* at = As + (L - L0) * kT;
        if (MODE == 0) at[a * (kNb + 1) + b2] = In[(L * kNb + a) + (int64_t)(I * kNb + b2) * bp];
        else at[b2 * (kNb + 1) + a] = X[(I * kNb + a) + (int64_t)(L * kNb + b2) * bp];
        Bs[(L - L0) * kT + a * (kNb + 1) + b2] = In[(L * kNb + a) + (int64_t)(J * kNb + b2) * bp];
    }
    __syncthreads();
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int L = 0; L < nL; ++L) {
        const float* at = As + L * kT;
        const float* bt = Bs + L * kT;
#pragma unroll 8
        for (int l = 0; l < kNb; ++l) {
            const float av = at[l * (kNb + 1) + lr];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fmaf(av, bt[l * (kNb + 1) + lc + q], acc[q]);
        }
    }
    const int i = I * kNb + lr;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = J * kNb + lc + q;
        const int64_t o = i + (int64_t)j * bp;
        float v;
        if (MODE == 0) v = (i < j) ? Ef[o] - acc[q] : (i == j) ? 0.5f * (Ef[o] - acc[q]) : 0.f;
        else v = (i <= j) ? ((i == j) ? 1.f : 0.f) - acc[q] : 0.f;
        Out[o] = v;
        if (last) {
            if (MODE == 0) {
                R[o] = (i <= j) ? ((i == j) ? 1.0 : 0.0) + (double)v : 0.0;
                Z[o] = (i <= j) ? ((i == j) ? 1.f : 0.f) - v : 0.f;
            } else {
                Rinv[o] = (T)v;
            }
        }
    }
}

}  // namespace

// Rinv (T) = R^{-1} for an upper-triangular FP64 R (bp x bp, column-major);
// the substitution runs in T.
template <typename T>
cudaError_t upper_inverse(Ctx& cx, const double* R, int bp, T* Rinv) {
    using W = T;
    const size_t smem = sizeof(W) * ((size_t)bp * (bp + 1) / 2 + 8 * (size_t)bp);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    cudaError_t ea = smem_limit(k_upper_inverse<T, W>, 200 * 1024);
    if (ea != cudaSuccess) return ea;
    k_upper_inverse<T, W><<<(bp + 7) / 8, 256, smem, cx.stream>>>(R, bp, Rinv);
    cx.launches++;
    return cudaGetLastError();
}

// G (bp x bp, FP64, overwritten) = R^T R; R (FP64) and Rinv (T).  scratch:
// 2 bp^2 + bp doubles (L, the inverses of its diagonal tiles, and the
// diagonal of G), plus bp^2 doubles' room for their FP32 copies when T is
// float.  fp64: working precision of the factorization (FP32 serves the
// second CholeskyQR pass, whose Gram is I + O(u kappa), and the first pass
// of the tensor-core handles); the factors are stored in FP64 either way;
// R^{-1} is formed in T.  FP32 factors of up to 256 columns run on one CTA
// (k_chol_f32_cta), the others as the chain of panel and update kernels.
template <typename T>
cudaError_t chol_inv_blocked(Ctx& cx, double* G, int bp, int p, double* R, T* Rinv, double tol, double* scratch,
                             size_t scratch_doubles, bool fp64, const int* skip) {
    constexpr bool f32 = sizeof(T) == 4;
    const size_t need = 2 * (size_t)bp * bp + bp + (f32 ? (size_t)bp * bp : 0);
    if (bp % kNb != 0 || scratch_doubles < need) return cudaErrorInvalidValue;
    double* L = scratch;
    double* Linv = scratch + (size_t)bp * bp;
    double* dG = Linv + (size_t)bp * bp;
    float* Lf = f32 ? reinterpret_cast<float*>(dG + bp) : nullptr;   // 16-byte aligned: bp % 32 == 0
    float* Lif = f32 ? Lf + (size_t)bp * bp : nullptr;
    const int nblk = bp / kNb;
    cudaError_t e;
    if (f32 && !fp64 && nblk <= 8) {
        // FP32 factor on one CTA (k_chol_f32_cta); G in FP32 where L would sit
        float* Gf = reinterpret_cast<float*>(L);
        const size_t smem = chol_f32_cta_smem(bp);
        if ((e = smem_limit(k_chol_f32_cta, (int)smem)) != cudaSuccess) return e;
        e = launch_pdl(k_chol_init, dim3(std::max(1, bp * bp / 256)), dim3(256), 0, cx.stream, G, bp, p, dG,
                       static_cast<double*>(nullptr), skip, Gf);
        if (e != cudaSuccess) return e;
        cx.launches++;
        e = launch_pdl(k_chol_f32_cta, dim3(1), dim3(kCtaThreads), smem, cx.stream, static_cast<const float*>(Gf), bp,
                       static_cast<const double*>(dG), tol, Lf, Lif, cx.st, skip);
        if (e != cudaSuccess) return e;
        cx.launches++;
        e = launch_pdl(k_chol_transpose_f32, dim3(std::max(1, bp * bp / 256)), dim3(256), 0, cx.stream,
                       static_cast<const float*>(Lf), bp, R, skip);
        if (e != cudaSuccess) return e;
        cx.launches++;
    } else {
        e = launch_pdl(k_chol_init, dim3(std::max(1, bp * bp / 256)), dim3(256), 0, cx.stream, G, bp, p, dG, L, skip,
                       static_cast<float*>(nullptr));
        if (e != cudaSuccess) return e;
        cx.launches++;
        for (int k = 0; k < nblk; ++k) {
            const int below = nblk - k - 1;
            const dim3 gp(1 + below * (kNb / kStrip));
            e = fp64 ? launch_pdl(k_chol_panel<double>, gp, dim3(256), 0, cx.stream, G, L, Linv, Lf, Lif, bp, k, dG,
                                  tol, cx.st, skip)
                     : launch_pdl(k_chol_panel<float>, gp, dim3(256), 0, cx.stream, G, L, Linv, Lf, Lif, bp, k, dG,
                                  tol, cx.st, skip);
            if (e != cudaSuccess) return e;
            cx.launches++;
            if (below > 0) {
                const int pairs = below * (below + 1) / 2;
                const dim3 gu(pairs * (kNb / kStrip));
                e = fp64 ? launch_pdl(k_chol_update<double>, gu, dim3(256), 0, cx.stream, G, L, bp, k, nblk, skip)
                         : launch_pdl(k_chol_update<float>, gu, dim3(256), 0, cx.stream, G, L, bp, k, nblk, skip);
                if (e != cudaSuccess) return e;
                cx.launches++;
            }
        }
        e = launch_pdl(k_chol_transpose, dim3(std::max(1, bp * bp / 256)), dim3(256), 0, cx.stream, L, bp, R, skip);
        if (e != cudaSuccess) return e;
        cx.launches++;
    }
    if constexpr (f32) {
        const size_t smem = sizeof(float) * ((size_t)bp * kXs + 2 * (size_t)bp * kNb + 2 * kNb * kNb + kNb * kXs);
        if (smem > 200 * 1024) return cudaErrorInvalidValue;
        cudaError_t ea = smem_limit(k_linv_f32, 200 * 1024);
        if (ea != cudaSuccess) return ea;
        e = launch_pdl(k_linv_f32, dim3(nblk), dim3(256), smem, cx.stream, Lf, Lif, bp, Rinv, skip);
        if (e != cudaSuccess) return e;
    } else {
        const size_t smem = sizeof(T) * ((size_t)bp * kNb + (size_t)bp * (kNb + 1) + 2 * (size_t)kNb * (kNb + 1));
        cudaError_t ea = smem_limit(k_linv_blocked<T, T>, 200 * 1024);
        if (ea != cudaSuccess) return ea;
        e = launch_pdl(k_linv_blocked<T, T>, dim3(nblk), dim3(256), smem, cx.stream, L, Linv, bp, Rinv, skip);
        if (e != cudaSuccess) return e;
    }
    cx.launches++;
    return cudaGetLastError();
}

// The norm's parts, then the decision and the first-order factor (kNearIdParts
// CTAs each), then for FP32 factors the iterated route's six steps.
template <typename T>
cudaError_t near_identity(Ctx& cx, const double* G, int bp, int p, double* R, T* Rinv, double tau, double* work,
                          int* skip) {
    cudaError_t e = launch_pdl(k_near_id_norm, dim3(kNearIdParts), dim3(256), 0, cx.stream, G, bp, p, work);
    if (e != cudaSuccess) return e;
    cx.launches++;
    // the iterated route for FP32 factors (whose tau leaves most tensor-core
    // panels above it): up to three fixed-point steps and three series steps
    // on the FP32 work matrices after the parts and the flags (the steps a
    // panel does not need return at once)
    constexpr bool kIter = sizeof(T) == 4;
    const double tau_i = kIter ? 2e-2 : 0.0;
    const size_t sq = (size_t)bp * bp;
    float* fw = reinterpret_cast<float*>(work + kNearIdParts + 2);
    float *Ef = fw, *Xa = fw + sq, *Xb = fw + 2 * sq, *Za = fw + 3 * sq, *Zb = fw + 4 * sq;
    int* iter = skip + 1;
    e = launch_pdl(k_near_id_apply<T>, dim3(kNearIdParts), dim3(256), 0, cx.stream, G, bp, p,
                   static_cast<const double*>(work), tau * tau, tau_i * tau_i, R, Rinv, Ef, Xa, skip, iter, cx.st);
    if (e != cudaSuccess) return e;
    cx.launches++;
    if constexpr (kIter) {
        const int nblk = bp / kNb;
        const dim3 gt(nblk * (nblk + 1) / 2);
        // up to 2 x nblk padded operand tiles per CTA
        const size_t smem = sizeof(float) * 2 * (size_t)nblk * kNb * (kNb + 1);
        if ((e = smem_limit(k_near_id_step<0, T>, (int)smem)) != cudaSuccess) return e;
        if ((e = smem_limit(k_near_id_step<1, T>, (int)smem)) != cudaSuccess) return e;
        const float* X0in[3] = {Xa, Xb, Xa};
        float* X0out[3] = {Xb, Xa, Xb};
        for (int k = 0; k < 3; ++k) {
            e = launch_pdl(k_near_id_step<0, T>, gt, dim3(256), smem, cx.stream, static_cast<const float*>(Ef),
                           static_cast<const float*>(nullptr), static_cast<const float*>(nullptr), X0in[k], X0out[k],
                           bp, k, R, Za, static_cast<T*>(nullptr), static_cast<const int*>(iter));
            if (e != cudaSuccess) return e;
            cx.launches++;
        }
        const float* Zin[3] = {Za, Zb, Za};
        float* Zout[3] = {Zb, Za, Zb};
        for (int k = 0; k < 3; ++k) {
            e = launch_pdl(k_near_id_step<1, T>, gt, dim3(256), smem, cx.stream, static_cast<const float*>(nullptr),
                           static_cast<const float*>(Xa), static_cast<const float*>(Xb), Zin[k], Zout[k], bp, k,
                           static_cast<double*>(nullptr), static_cast<float*>(nullptr), Rinv,
                           static_cast<const int*>(iter));
            if (e != cudaSuccess) return e;
            cx.launches++;
        }
    }
    return cudaGetLastError();
}

template cudaError_t upper_inverse<float>(Ctx&, const double*, int, float*);
template cudaError_t upper_inverse<double>(Ctx&, const double*, int, double*);
template cudaError_t chol_inv_blocked<float>(Ctx&, double*, int, int, double*, float*, double, double*, size_t, bool,
                                             const int*);
template cudaError_t chol_inv_blocked<double>(Ctx&, double*, int, int, double*, double*, double, double*, size_t,
                                              bool, const int*);
template cudaError_t near_identity<float>(Ctx&, const double*, int, int, double*, float*, double, double*, int*);
template cudaError_t near_identity<double>(Ctx&, const double*, int, int, double*, double*, double, double*, int*);

}  // namespace rqb

extern "C" int rqb_fp64_recip_selftest(const double* x, int64_t count, double* rcp, double* rsq, void* stream) {
    if (!x || !rcp || !rsq || count < 1) return RQB_ERR_INVALID;
    const int blocks = (int)std::min<int64_t>((count + 255) / 256, 1024);
    rqb::k_recip_selftest<<<blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(x, count, rcp, rsq);
    return cudaGetLastError() == cudaSuccess ? RQB_OK : RQB_ERR_CUDA;
}
