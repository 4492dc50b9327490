// rqb_batched.cu -- randQB_b for many independent FP32 matrices of uneven
// sizes (block size b <= 32), grouped by block index.
//
// All matrices advance through the blocks of Fig. randQB_b together: block i
// of every still-active matrix is one sequence of grouped launches, each of
// which covers the tiles of all active matrices (work-item tables built once
// on the host), so a large matrix spreads over many SMs while small ones fill
// the rest of the GPU.  Per block i:
//   line (2)   Omega_i: every matrix uses global columns i b .. i b + 31 of one
//              Omega (its first n_t rows), drawn once per block
//   line (3)   Y = A Omega_1 (block 1; later blocks come out of the update)
//   (3), (3')  CholeskyQR2 with re-projection: exact FP32 Gram promoted to
//              FP64 and FP64 Cholesky per matrix (one CTA each), Y R^-1 and
//              Y - Qbar C on 128-row tiles, C = Qbar^T Y on 128-column tiles
//              with FP64 accumulation
//   line (4)   B_i = Q_i^T A^(i-1) on 128-column tiles, ||B_i||^2 (FP64)
//   line (6)   per-matrix test on E_i outside the FP32 rounding band, else on
//              the direct ||A^(i)||^2 of the update
//   line (5)   A^(i) = A^(i-1) - Q_i B_i fused with the next block's sketch
// The per-matrix state (k, E, flags, status) lives on the device; the items of
// finished matrices return at once.  The whole batch is one instantiated CUDA
// graph: a prologue, then a WHILE node whose body is one block of every
// matrix, its condition (some matrix still active) set on the device at the
// end of each block, so no host round trip happens between blocks.  The graph
// is kept by the handle and relaunched while the batch shape is the same.
// The projection's tile width (128 or 256 columns per work item) is picked by
// an autotuner per batch class.  Partial sums are combined per matrix in a
// fixed order, so results are bitwise repeatable.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "rqb_engine.h"
#include "rqb_gemm_simt.cuh"

namespace rqb {
namespace batched {

constexpr int NT = 256;          // threads per CTA
constexpr int BP = 32;           // padded block width (b <= 32)
constexpr int TR = 128;          // rows per row item
constexpr int TC = 256;          // columns per projection item
constexpr int TCR = 128;         // columns per re-projection item
constexpr int KCH = 32;          // reduction chunk of the grouped products

struct Smem {
    double G[BP][BP + 1];        // Gram / Cholesky work (FP64)
    float Rinv[BP][BP + 1];      // R^{-1}
    double red[NT / 32];
    double scal[8];
    int ival[4];
};

__device__ __forceinline__ double cta_sum(double v, Smem& s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s.red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < NT / 32; ++w) t += s.red[w];
    __syncthreads();
    return t;   // every thread gets the same value
}



// Per-matrix descriptors (built on the host) and device state.
struct GMat {
    const float* A;      // caller's matrix (ld lda)
    float* W;            // residual A^(i) (ld ldw)
    float* Q;            // m x kcap output (ld ldq)
    float* B;            // kcap x n output (ld ldb)
    float* Y;            // m x BP panel (ld ldw)
    float* Y1;           // m x BP panel scratch (ld ldw)
    float* Cc;           // kcap x BP re-projection coefficients (ld kcap)
    float* Rinv;         // BP x BP, row-major
    int64_t m, n, lda, ldw, ldq, ldb, kcap;
    double eps2;
    int rows_begin, rows_end;   // items of this matrix in the row table
    int proj_begin, proj_end;   // ... in the projection table
};

struct GState {
    double normA2, E, tau, D;
    int64_t k;           // columns of Q done before the current block
    int64_t knext;       // k + p once the current block is accepted
    int p;               // width of the current block
    int active;          // still factoring
    int pending;         // the current block's update must run
    int flag;            // stop decision of the current block (StopFlag)
    int status;
    int blocks;
};

struct Item {
    int t;               // matrix
    int tile;            // row tile (rows 128 tile ..) or column tile
};

// Cholesky of s.G (p x p valid, identity beyond): G = L L^T with L and L^{-1}
// formed together in shared memory (right-looking; at step j the pivot column
// of L and row j of L^{-1} are scaled by 1 / l_jj, then the trailing part of L
// is updated and column j eliminated from the rows of L^{-1} below j, all
// entries in parallel).  s.Rinv = R^{-1} = (L^{-1})^T (FP32) for R = L^T.
// Returns false (CTA-uniform) on a pivot <= tol * G_jj.
__device__ bool cta_chol_inv(Smem& s, int p, double tol) {
    const int tid = threadIdx.x;
    __shared__ double diag0[BP];
    __shared__ double L[BP][BP + 1];
    __shared__ double Li[BP][BP + 1];
    __shared__ double inv[BP];
    __shared__ int fail;
    for (int r = tid; r < BP; r += NT) diag0[r] = (r < p) ? s.G[r][r] : 1.0;
    for (int e = tid; e < BP * BP; e += NT) {
        const int r = e / BP, c = e % BP;
        double v = (r < p && c < p) ? s.G[r][c] : (r == c ? 1.0 : 0.0);
        L[r][c] = (r >= c) ? v : 0.0;
        Li[r][c] = (r == c) ? 1.0 : 0.0;
    }
    if (tid == 0) fail = 0;
    __syncthreads();
    for (int j = 0; j < BP; ++j) {
        if (tid == 0) {
            double d = L[j][j];
            if (!(d > tol * diag0[j]) || !isfinite(d)) {
                fail = 1;
                d = 1.0;
            }
            const double l = sqrt(d);
            L[j][j] = l;
            inv[j] = 1.0 / l;
        }
        __syncthreads();
        const double ij = inv[j];
        if (tid < BP) {
            if (tid > j) L[tid][j] *= ij;
        } else if (tid < 2 * BP) {
            if (tid - BP <= j) Li[j][tid - BP] *= ij;
        }
        __syncthreads();
        for (int e = tid; e < BP * BP; e += NT) {
            const int r = e % BP, c = e / BP;
            if (c > j && r >= c) L[r][c] -= L[r][j] * L[c][j];
            else if (r > j && c <= j) Li[r][c] -= L[r][j] * Li[j][c];
        }
        __syncthreads();
    }
    if (fail) return false;
    for (int e = tid; e < BP * BP; e += NT) {
        const int r = e / BP, c = e % BP;
        s.Rinv[r][c] = (float)Li[c][r];   // R^{-1} = (L^{-1})^T, upper
    }
    __syncthreads();
    return true;
}


// ---------------------------------------------------------------------------
// Row items: 128-row tiles, output 128 x BP.  Thread (ty, tx) owns rows
// ty*4 .. +3 and columns tx*4 .. +3 of the tile.

// acc += X(r0 .. r0+127, 0 .. K) C(0 .. K, 0 .. BP), X column-major (ld ldx),
// C(k, j) = C[k * csk + j * csj]; sq (if non-null) += sum of the squares of
// the X entries this thread loaded.
__device__ __forceinline__ void rows_product(float (&acc)[4][4], int64_t rows, int64_t r0, int64_t K, const float* X,
                                             int64_t ldx, const float* C, int64_t csk, int64_t csj,
                                             float (*Xs)[TR + 4], float (*Cs)[BP + 4], double* sq) {
    const int tid = threadIdx.x, ty = tid >> 3, tx = tid & 7;
    const bool vec = ((reinterpret_cast<uintptr_t>(X) & 15u) == 0) && (ldx % 4 == 0);
    for (int64_t k0 = 0; k0 < K; k0 += KCH) {
        __syncthreads();
        float sqf = 0.f;
        for (int v = tid; v < KCH * (TR / 4); v += NT) {
            const int kk = v / (TR / 4), rr = (v % (TR / 4)) * 4;
            const int64_t k = k0 + kk, r = r0 + rr;
            float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k < K && r < rows) {
                const float* src = X + r + k * ldx;
                if (vec && r + 4 <= rows) {
                    x = *reinterpret_cast<const float4*>(src);
                } else {
                    x.x = src[0];
                    if (r + 1 < rows) x.y = src[1];
                    if (r + 2 < rows) x.z = src[2];
                    if (r + 3 < rows) x.w = src[3];
                }
            }
            *reinterpret_cast<float4*>(&Xs[kk][rr]) = x;
            sqf = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, sqf))));
        }
        if (sq) *sq += (double)sqf;
        for (int e = tid; e < KCH * BP; e += NT) {
            const int kk = e / BP, j = e % BP;
            const int64_t k = k0 + kk;
            Cs[kk][j] = (k < K) ? C[k * csk + (int64_t)j * csj] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < KCH; ++kk) {
            const float4 a = *reinterpret_cast<const float4*>(&Xs[kk][ty * 4]);
            const float4 b = *reinterpret_cast<const float4*>(&Cs[kk][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
    }
}

// Out(r, j) = sub ? Out(r, j) - acc : acc for rows < `rows`, columns < BP;
// columns >= ncols are written as zero.
__device__ __forceinline__ void rows_store(const float (&acc)[4][4], int64_t rows, int64_t r0, float* Out, int64_t ldo,
                                           int ncols, bool sub) {
    const int tid = threadIdx.x, ty = tid >> 3, tx = tid & 7;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t r = r0 + ty * 4 + i;
        if (r >= rows) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = tx * 4 + j;
            float* o = Out + r + (int64_t)c * ldo;
            *o = (c < ncols) ? (sub ? *o - acc[i][j] : acc[i][j]) : 0.f;
        }
    }
}

__device__ __forceinline__ double block_sum_d(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < NT / 32; ++w) t += red[w];
    return t;
}

// Rows r .. r + 3 of one column: src points at row r, rem = rows left (m - r);
// a 16-byte load when vec (aligned column, ld a multiple of 4) and rem >= 4.
__device__ __forceinline__ float4 load_rows4(const float* src, int64_t rem, bool valid, bool vec) {
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!valid || rem <= 0) return x;
    if (vec && rem >= 4) return *reinterpret_cast<const float4*>(src);
    x.x = src[0];
    if (rem > 1) x.y = src[1];
    if (rem > 2) x.z = src[2];
    if (rem > 3) x.w = src[3];
    return x;
}

__device__ __forceinline__ bool vec_ok(const float* p, int64_t ld) {
    return ((reinterpret_cast<uintptr_t>(p) & 15u) == 0) && (ld % 4 == 0);
}

enum RowOp { kRowSketch0 = 0, kRowMulR1 = 1, kRowSubQC = 2, kRowMulR2 = 3 };

// kRowSketch0  Y = A Omega_1 (columns >= p zero), part = ||A tile||_F^2
// kRowMulR1    Y1 = Y R^-1
// kRowSubQC    Y1 -= Qbar C (k > 0)
// kRowMulR2    Q_i = Y1 R^-1 (columns k .. k + p of Q)
template <int OP>
__global__ void __launch_bounds__(NT) k_rows(const GMat* __restrict__ mats, const GState* __restrict__ st,
                                             const Item* __restrict__ items, int b, const float* __restrict__ Om,
                                             double* __restrict__ part) {
    __shared__ __align__(16) float Xs[KCH][TR + 4];
    __shared__ __align__(16) float Cs[KCH][BP + 4];
    __shared__ double red[NT / 32];
    const Item it = items[blockIdx.x];
    const GMat& d = mats[it.t];
    const int64_t r0 = (int64_t)it.tile * TR;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    if (OP == kRowSketch0) {
        const int p = (int)min((int64_t)b, d.kcap);
        double sq = 0.0;
        rows_product(acc, d.m, r0, d.n, d.A, d.lda, Om, BP, 1, Xs, Cs, &sq);
        rows_store(acc, d.m, r0, d.Y, d.ldw, p, false);
        const double t = block_sum_d(sq, red);
        if (threadIdx.x == 0) part[blockIdx.x] = t;
        return;
    }
    const GState s = st[it.t];
    if (!s.active) return;
    if (OP == kRowMulR1) {
        rows_product(acc, d.m, r0, BP, d.Y, d.ldw, d.Rinv, BP, 1, Xs, Cs, nullptr);
        rows_store(acc, d.m, r0, d.Y1, d.ldw, BP, false);
    } else if (OP == kRowSubQC) {
        if (s.k == 0) return;
        rows_product(acc, d.m, r0, s.k, d.Q, d.ldq, d.Cc, 1, d.kcap, Xs, Cs, nullptr);
        rows_store(acc, d.m, r0, d.Y1, d.ldw, BP, true);
    } else {
        rows_product(acc, d.m, r0, BP, d.Y1, d.ldw, d.Rinv, BP, 1, Xs, Cs, nullptr);
        // Q has kcap columns: only the p columns of this block are written
        const int tid = threadIdx.x, ty = tid >> 3, tx = tid & 7;
        float* Qi = d.Q + s.k * d.ldq;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t r = r0 + ty * 4 + i;
            if (r >= d.m) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = tx * 4 + j;
                if (c < s.p) Qi[r + (int64_t)c * d.ldq] = acc[i][j];
            }
        }
    }
}

// Line (5) fused with the next sketch on one 128-row tile:
//   W(rows, :) = Wsrc(rows, :) - Q_i(rows, :) B_i,  Y(rows, :) = W(rows, :) Omega_{i+1}
// column chunk by column chunk; part = ||W(rows, :)||_F^2.  Wsrc is A in the
// first block.  Runs for matrices whose block i was accepted or is ambiguous.
// 128 threads; thread (ty, tx) owns rows ty*8 .. +7 and columns tx + 8 j
// (j < 4) of both products: the element-wise update then reads and writes its
// 8 contiguous rows of a column with conflict-free 16-byte accesses.  The
// next column chunk is loaded into registers while the current one is used.
constexpr int NTU = 128;

__global__ void __launch_bounds__(NTU) k_rows_update(const GMat* __restrict__ mats, const GState* __restrict__ st,
                                                     const Item* __restrict__ items, int b, const int* __restrict__ blk,
                                                     const float* __restrict__ Om_next, double* __restrict__ part) {
    // B_i and Omega_{i+1} chunks are stored so that a thread's four strided
    // columns tx + 8 j (j < 4) are one 16-byte word: entry (t, c) of a row
    // sits at [(c % 8) * 4 + c / 8] (rows padded to 36 floats)
    __shared__ __align__(16) float Qs[BP][TR + 4];    // Qs[t][r] = Q_i(r0 + r, t)
    __shared__ __align__(16) float Bs[BP][36];        // B_i(t, c0 + c) at Bs[t][(c % 8) * 4 + c / 8]
    __shared__ __align__(16) float Ws[KCH][TR + 4];   // Ws[c][r] = W(r0 + r, c0 + c)
    __shared__ __align__(16) float Os[KCH][36];       // Omega_{i+1}(c0 + c, j) at Os[c][(j % 8) * 4 + j / 8]
    __shared__ double red[NTU / 32];
    const Item it = items[blockIdx.x];
    const GState s = st[it.t];
    if (!s.pending) return;
    const GMat& d = mats[it.t];
    const int first = (*blk == 0) ? 1 : 0;   // block 1 reads A itself
    const int tid = threadIdx.x, ty = tid >> 3, tx = tid & 7;
    const int64_t m = d.m, n = d.n, r0 = (int64_t)it.tile * TR;
    const float* Wsrc = first ? d.A : d.W;
    const int64_t ldws = first ? d.lda : d.ldw;
    const bool vsrc = vec_ok(Wsrc, ldws);
    const float* Qi = d.Q + s.k * d.ldq;
    const float* Bi = d.B + s.k;
    const int p = s.p;
    const int pn = (int)max((int64_t)0, min((int64_t)b, d.kcap - s.knext));
    for (int v = tid; v < BP * (TR / 4); v += NTU) {
        const int t = v / (TR / 4), rr = (v % (TR / 4)) * 4;
        const int64_t r = r0 + rr;
        *reinterpret_cast<float4*>(&Qs[t][rr]) = load_rows4(Qi + r + (int64_t)t * d.ldq, m - r, t < p, true);
    }
    constexpr int WQ = KCH * (TR / 4) / NTU;   // float4 of W per thread (8)
    constexpr int SQ = KCH * BP / NTU;         // B_i and Omega entries per thread (8)
    float4 wr[WQ];
    float br[SQ], orr[SQ];
    auto load = [&](int64_t c0) {
#pragma unroll
        for (int u = 0; u < SQ; ++u) {
            const int e = tid + u * NTU, c = e / BP, t = e % BP;
            const int64_t cc = c0 + c;
            br[u] = (t < p && cc < n) ? Bi[t + cc * d.ldb] : 0.f;
            orr[u] = (cc < n) ? Om_next[cc * BP + t] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < WQ; ++u) {
            const int v = tid + u * NTU, c = v / (TR / 4), rr = (v % (TR / 4)) * 4;
            const int64_t cc = c0 + c, r = r0 + rr;
            wr[u] = load_rows4(Wsrc + r + cc * ldws, m - r, cc < n, vsrc);
        }
    };
    float2 yacc[4][4];   // (rows 2i, 2i + 1) x column j, for the packed FMAs
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) yacc[i][j] = make_float2(0.f, 0.f);
    double sq = 0.0;
    load(0);
    for (int64_t c0 = 0; c0 < n; c0 += KCH) {
        __syncthreads();
#pragma unroll
        for (int u = 0; u < SQ; ++u) {
            const int e = tid + u * NTU, c = e / BP, t = e % BP;
            Bs[t][(c & 7) * 4 + (c >> 3)] = br[u];
            Os[c][(t & 7) * 4 + (t >> 3)] = orr[u];
        }
#pragma unroll
        for (int u = 0; u < WQ; ++u) {
            const int v = tid + u * NTU, c = v / (TR / 4), rr = (v % (TR / 4)) * 4;
            *reinterpret_cast<float4*>(&Ws[c][rr]) = wr[u];
        }
        __syncthreads();
        if (c0 + KCH < n) load(c0 + KCH);
        // P = Q_i(tile) B_i(:, chunk)
        float2 pacc2[4][4];   // (rows 2i, 2i + 1) x column j
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) pacc2[i][j] = make_float2(0.f, 0.f);
#pragma unroll 8
        for (int t = 0; t < BP; ++t) {
            const float4 a0 = *reinterpret_cast<const float4*>(&Qs[t][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&Qs[t][ty * 8 + 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float4 b4 = *reinterpret_cast<const float4*>(&Bs[t][tx * 4]);
            const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
            fma_tile_f32x2_rows<8, 4>(pacc2, av, bv);
        }
        float pacc[8][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                pacc[2 * i][j] = pacc2[i][j].x;
                pacc[2 * i + 1][j] = pacc2[i][j].y;
            }
        // W = Wsrc - P on this thread's entries: shared copy, global store, ||W||^2
        float sqf = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = tx + 8 * j;
            const int64_t cc = c0 + c;
            float* ws = &Ws[c][ty * 8];
            const float4 w0 = *reinterpret_cast<const float4*>(ws);
            const float4 w1 = *reinterpret_cast<const float4*>(ws + 4);
            float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                w[i] -= pacc[i][j];
                if (cc >= n || r0 + ty * 8 + i >= m) w[i] = 0.f;
                sqf = fmaf(w[i], w[i], sqf);
            }
            *reinterpret_cast<float4*>(ws) = make_float4(w[0], w[1], w[2], w[3]);
            *reinterpret_cast<float4*>(ws + 4) = make_float4(w[4], w[5], w[6], w[7]);
            if (cc < n) {
                const int64_t r = r0 + ty * 8;
                float* dst = d.W + r + cc * d.ldw;
                if (r + 8 <= m) {   // ldw % 4 == 0: two aligned 16-byte stores
                    *reinterpret_cast<float4*>(dst) = make_float4(w[0], w[1], w[2], w[3]);
                    *reinterpret_cast<float4*>(dst + 4) = make_float4(w[4], w[5], w[6], w[7]);
                } else {
                    for (int i = 0; i < 8; ++i)
                        if (r + i < m) dst[i] = w[i];
                }
            }
        }
        sq += (double)sqf;
        __syncthreads();
        // Y += W(tile, chunk) Omega_{i+1}(chunk, :)
#pragma unroll 8
        for (int c = 0; c < KCH; ++c) {
            const float4 a0 = *reinterpret_cast<const float4*>(&Ws[c][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&Ws[c][ty * 8 + 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float4 o4 = *reinterpret_cast<const float4*>(&Os[c][tx * 4]);
            const float ov[4] = {o4.x, o4.y, o4.z, o4.w};
            fma_tile_f32x2_rows<8, 4>(yacc, av, ov);
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t r = r0 + ty * 8 + i;
        if (r >= m) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = tx + 8 * j;
            const float y = (i & 1) ? yacc[i >> 1][j].y : yacc[i >> 1][j].x;
            d.Y[r + (int64_t)c * d.ldw] = (c < pn) ? y : 0.f;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if ((tid & 31) == 0) red[tid >> 5] = sq;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < NTU / 32; ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

// ---------------------------------------------------------------------------
// Column items: out(j, c) for j < BP and W columns c of the item, reduced over
// the m rows:
//   kColProject  B_i(j, c) = sum_r Q_i(r, j) Wsrc(r, c), 256 columns per item,
//                part = ||B_i tile||^2
//   kColReproj   C(c, j)   = sum_r Qbar(r, c) Y1(r, j), 128 columns per item,
//                FP32 partials promoted to FP64 every 128 rows
// Thread (jg, ct) owns j = jg*JT .. +JT-1 and the four columns 4 ct .. +3
// (JT = W / 32): per chunk row one broadcast 16-byte read of P and one
// 16-byte read of V feed 4 JT multiply-adds.  The 16-byte groups of a V row
// are permuted by (row / 4) % 8 so that both the transposing stores of the
// staged chunk and the 16-byte reads are free of bank conflicts.
enum ColOp { kColProject = 0, kColReproj = 1 };

__device__ __forceinline__ int vs_col(int r, int c) {   // physical column of V entry (r, c)
    return ((((c >> 2) ^ ((r >> 2) & 7))) << 2) | (c & 3);
}

template <int OP, int W>
__global__ void __launch_bounds__(NT) k_cols(const GMat* __restrict__ mats, const GState* __restrict__ st,
                                             const Item* __restrict__ items, const int* __restrict__ blk,
                                             double* __restrict__ part) {
    // W: columns per item (the projection's is picked by the autotuner)
    constexpr int JT = W / 32;                           // j per thread (8 or 4)
    constexpr int NCT = W / 4;                           // column threads
    static_assert((BP / JT) * NCT == NT, "thread map");
    __shared__ __align__(16) float Ps[KCH][BP + 4];   // Ps[r][j]: Q_i or Y1 rows of the chunk
    __shared__ __align__(16) float Vs[KCH][W];        // Vs[r][vs_col(r, c)]: Wsrc or Qbar columns of the item
    __shared__ double red[NT / 32];
    const Item it = items[blockIdx.x];
    const GState s = st[it.t];
    if (!s.active) return;
    if (OP == kColReproj && s.k == 0) return;
    const GMat& d = mats[it.t];
    const int first = (*blk == 0) ? 1 : 0;   // block 1 projects A itself
    const int64_t c0 = (int64_t)it.tile * W;
    const int64_t ncols = (OP == kColProject) ? d.n : s.k;
    if (c0 >= ncols) return;
    const float* P = (OP == kColProject) ? d.Q + s.k * d.ldq : d.Y1;
    const int64_t ldp = (OP == kColProject) ? d.ldq : d.ldw;
    const int pw = (OP == kColProject) ? s.p : BP;
    const float* V = (OP == kColProject) ? (first ? d.A : d.W) : d.Q;
    const int64_t ldv = (OP == kColProject) ? (first ? d.lda : d.ldw) : d.ldq;
    const int64_t m = d.m;
    const int tid = threadIdx.x, jg = tid / NCT, ct = tid % NCT;
    float acc[JT][4];
    float2 accp[JT][2];   // acc as column pairs, for the packed FMAs
    double acc2[OP == kColReproj ? JT : 1][4];
#pragma unroll
    for (int i = 0; i < JT; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = 0.f;
    zero_tile_f32x2<JT, 4>(accp);
    if (OP == kColReproj) {
#pragma unroll
        for (int i = 0; i < (OP == kColReproj ? JT : 1); ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc2[i][q] = 0.0;
    }
    // staging: float4 e of a chunk covers rows 4 (e % 8) .. +3 of column e / 8;
    // the next chunk is loaded into registers while the current one is used
    constexpr int VQ = (KCH / 4) * W / NT;
    const bool pvec = vec_ok(P, ldp), vvec = vec_ok(V, ldv);
    float4 pr, vr[VQ];
    auto load = [&](int64_t r0) {
        {
            const int j = tid / (KCH / 4), rq = (tid % (KCH / 4)) * 4;
            pr = load_rows4(P + (r0 + rq) + (int64_t)j * ldp, m - r0 - rq, j < pw, pvec);
        }
#pragma unroll
        for (int u = 0; u < VQ; ++u) {
            const int e = tid + u * NT, c = e / (KCH / 4), rq = (e % (KCH / 4)) * 4;
            const int64_t cc = c0 + c;
            vr[u] = load_rows4(V + (r0 + rq) + cc * ldv, m - r0 - rq, cc < ncols, vvec);
        }
    };
    load(0);
    int chunk = 0;
    for (int64_t r0 = 0; r0 < m; r0 += KCH) {
        __syncthreads();
        {
            const int j = tid / (KCH / 4), rq = (tid % (KCH / 4)) * 4;
            Ps[rq][j] = pr.x; Ps[rq + 1][j] = pr.y; Ps[rq + 2][j] = pr.z; Ps[rq + 3][j] = pr.w;
        }
#pragma unroll
        for (int u = 0; u < VQ; ++u) {
            const int e = tid + u * NT, c = e / (KCH / 4), rq = (e % (KCH / 4)) * 4;
            const int pc = vs_col(rq, c);   // rows rq .. rq + 3 share the permutation
            Vs[rq][pc] = vr[u].x; Vs[rq + 1][pc] = vr[u].y; Vs[rq + 2][pc] = vr[u].z; Vs[rq + 3][pc] = vr[u].w;
        }
        __syncthreads();
        if (r0 + KCH < m) load(r0 + KCH);
#pragma unroll 4
        for (int rr = 0; rr < KCH; ++rr) {
            float a[JT];
#pragma unroll
            for (int h = 0; h < JT; h += 4) {   // warp-uniform: broadcast
                const float4 a4 = *reinterpret_cast<const float4*>(&Ps[rr][jg * JT + h]);
                a[h] = a4.x; a[h + 1] = a4.y; a[h + 2] = a4.z; a[h + 3] = a4.w;
            }
            const float4 v4 = *reinterpret_cast<const float4*>(&Vs[rr][vs_col(rr, 4 * ct)]);
            const float v[4] = {v4.x, v4.y, v4.z, v4.w};
            fma_tile_f32x2<JT, 4>(accp, a, v);
        }
        if (OP == kColReproj && (++chunk == 4 || r0 + KCH >= m)) {
            chunk = 0;
            unpack_tile_f32x2<JT, 4>(accp, acc);
            zero_tile_f32x2<JT, 4>(accp);
#pragma unroll
            for (int i = 0; i < (OP == kColReproj ? JT : 1); ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    acc2[i][q] += (double)acc[i][q];
                    acc[i][q] = 0.f;
                }
        }
    }
    if (OP == kColProject) unpack_tile_f32x2<JT, 4>(accp, acc);
    double sq = 0.0;
#pragma unroll
    for (int i = 0; i < JT; ++i) {
        const int j = jg * JT + i;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t cc = c0 + 4 * ct + q;
            if (cc >= ncols) continue;
            if (OP == kColProject) {
                if (j < s.p) {
                    const float bv = acc[i][q];
                    d.B[(s.k + j) + cc * d.ldb] = bv;
                    sq += (double)bv * (double)bv;
                }
            } else {
                d.Cc[cc + (int64_t)j * d.kcap] = (float)acc2[OP == kColReproj ? i : 0][q];
            }
        }
    }
    if (OP == kColProject) {
        const double t = block_sum_d(sq, red);
        if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
}

// Exact Gram partials of one 128-row tile of Y (SRC = 0) or Y1 (SRC = 1):
// gpart[item][r][c] = sum over the tile's rows of Y(., r) Y(., c), products
// split exactly and summed with TwoSum in FP32 pairs, promoted to FP64.
// Thread (ti, tj) of a 16 x 16 grid owns entries (2 ti .. +1, 2 tj .. +1).
template <int SRC>
__global__ void __launch_bounds__(NT) k_rows_gram(const GMat* __restrict__ mats, const GState* __restrict__ st,
                                                  const Item* __restrict__ items, double* __restrict__ gpart) {
    __shared__ float Ys[TR][BP + 1];
    const Item it = items[blockIdx.x];
    const GState s = st[it.t];
    if (!s.active) return;
    const GMat& d = mats[it.t];
    const float* Y = (SRC == 0) ? d.Y : d.Y1;
    const int64_t r0 = (int64_t)it.tile * TR;
    const int tid = threadIdx.x;
    for (int e = tid; e < TR * BP; e += NT) {
        const int j = e / TR, rr = e % TR;
        const int64_t r = r0 + rr;
        Ys[rr][j] = (r < d.m) ? Y[r + (int64_t)j * d.ldw] : 0.f;
    }
    __syncthreads();
    const int ti = tid >> 4, tj = tid & 15;
    float hi[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, lo[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 4
    for (int rr = 0; rr < TR; ++rr) {
        const float a0 = Ys[rr][ti * 2], a1 = Ys[rr][ti * 2 + 1];
        const float b0 = Ys[rr][tj * 2], b1 = Ys[rr][tj * 2 + 1];
        exact_fma_acc(a0, b0, hi[0][0], lo[0][0]);
        exact_fma_acc(a0, b1, hi[0][1], lo[0][1]);
        exact_fma_acc(a1, b0, hi[1][0], lo[1][0]);
        exact_fma_acc(a1, b1, hi[1][1], lo[1][1]);
    }
    double* g = gpart + (size_t)blockIdx.x * (BP * BP);
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) g[(ti * 2 + i) * BP + tj * 2 + j] = (double)hi[i][j] + (double)lo[i][j];
}

// ---------------------------------------------------------------------------
// Matrix items: one CTA per matrix.
//   kMatInit    ||A||^2 from the first sketch's partials; state of block 1
//   kMatPanel1  Gram of Y from its tiles' exact partials (fixed order), FP64
//               Cholesky, R^-1 (first CholeskyQR pass)
//   kMatPanel2  the same for Y1 (second pass)
//   kMatStop    E_i -= ||B_i||^2 and the decision of line (6)
//   kMatDirect  inside the band: the direct ||A^(i)||^2 of the update decides;
//               advance to the next block
enum MatOp { kMatInit = 0, kMatPanel1 = 1, kMatPanel2 = 2, kMatStop = 3, kMatDirect = 4 };

template <int OP>
__global__ void __launch_bounds__(NT, 1) k_mat(const GMat* __restrict__ mats, GState* __restrict__ st, int b,
                                               const double* __restrict__ rows_part,
                                               const double* __restrict__ proj_part,
                                               const double* __restrict__ gpart) {
    __shared__ Smem s;
    const int t = blockIdx.x;
    const GMat& d = mats[t];
    GState g = st[t];
    const double tau_rel = 32.0 * 5.9604644775390625e-08;   // FP32 rounding band of E
    if (OP == kMatInit) {
        if (threadIdx.x == 0) {
            double nrm = 0.0;
            for (int i = d.rows_begin; i < d.rows_end; ++i) nrm += rows_part[i];
            g.normA2 = nrm;
            g.E = nrm;
            g.tau = tau_rel * nrm;
            g.D = -1.0;
            g.k = 0;
            g.knext = 0;
            g.p = (int)min((int64_t)b, d.kcap);
            g.pending = 0;
            g.flag = kContinue;
            g.blocks = 0;
            g.active = isfinite(nrm) ? 1 : 0;
            g.status = isfinite(nrm) ? RQB_NOT_CONVERGED : RQB_ERR_NONFINITE;
            if (isfinite(nrm) && nrm <= d.eps2) {
                // ||A||_F <= eps already: the empty factorization (k = 0)
                g.active = 0;
                g.status = RQB_OK;
            }
            st[t] = g;
        }
        return;
    }
    if (!g.active) return;
    if (OP == kMatPanel1 || OP == kMatPanel2) {
        for (int e = threadIdx.x; e < BP * BP; e += NT) {
            double acc = 0.0;
            for (int i = d.rows_begin; i < d.rows_end; ++i) acc += gpart[(size_t)i * (BP * BP) + e];
            s.G[e / BP][e % BP] = acc;
        }
        __syncthreads();
        const bool ok = cta_chol_inv(s, g.p, 1e-14);
        if (!ok) {
            if (threadIdx.x == 0) {
                g.status = RQB_ERR_BREAKDOWN;
                g.active = 0;
                g.pending = 0;
                st[t] = g;
            }
            return;
        }
        for (int e = threadIdx.x; e < BP * BP; e += NT) d.Rinv[e] = s.Rinv[e / BP][e % BP];
        return;
    }
    if (threadIdx.x != 0) return;
    if (OP == kMatStop) {
        double nb = 0.0;
        for (int i = d.proj_begin; i < d.proj_end; ++i) nb += proj_part[i];
        g.E -= nb;
        g.blocks += 1;
        g.knext = g.k + g.p;
        g.flag = (g.E <= d.eps2 - g.tau) ? kStop : (g.E > d.eps2 + g.tau) ? kContinue : kAmbiguous;
        if (g.flag == kStop) {
            g.status = RQB_OK;
            g.active = 0;
            g.pending = 0;
            g.k = g.knext;
        } else if (g.flag == kContinue && g.knext >= d.kcap) {
            g.active = 0;             // rank cap reached: RQB_NOT_CONVERGED
            g.pending = 0;
            g.k = g.knext;
        } else {
            g.pending = 1;
        }
        st[t] = g;
        return;
    }
    // kMatDirect
    if (!g.pending) return;
    double dn = 0.0;
    for (int i = d.rows_begin; i < d.rows_end; ++i) dn += rows_part[i];
    g.D = dn;
    g.k = g.knext;
    g.pending = 0;
    if (g.flag == kAmbiguous && dn <= d.eps2) {
        g.status = RQB_OK;
        g.active = 0;
    } else if (g.k >= d.kcap) {
        g.active = 0;
    } else {
        g.p = (int)min((int64_t)b, d.kcap - g.k);
    }
    st[t] = g;
}

// Omega (n_max x BP, row-major): global columns col0 .. col0 + b - 1, zero
// beyond b, with col0 = 0 (no blk) or (*blk + 1) b, the next block's.
__global__ void k_omega_rows(int64_t n_max, const int* __restrict__ blk, int b, uint64_t seed,
                             float* __restrict__ Om) {
    const int64_t col0 = blk ? (int64_t)(*blk + 1) * b : 0;
    const int64_t total = n_max * BP;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / BP;
        const int c = (int)(e % BP);
        Om[e] = (c < b) ? gaussian_f32(seed, r, col0 + c) : 0.f;
    }
}

// End of a block of the device-side loop: advance the block index and keep
// the loop (the graph's WHILE node) running while a matrix is still active
// and fewer than max_blocks blocks have run; every matrix is done after
// max_blocks blocks (k reaches its cap), so the loop always ends.
__global__ void k_advance(int* __restrict__ blk, const GState* __restrict__ st, int count, int max_blocks,
                          cudaGraphConditionalHandle loop) {
    __shared__ int sh[NT / 32];
    int c = 0;
    for (int t = threadIdx.x; t < count; t += NT) c += st[t].active;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < NT / 32; ++w) tot += sh[w];
        const int next = *blk + 1;
        *blk = next;
        cudaGraphSetConditional(loop, (tot > 0 && next < max_blocks) ? 1u : 0u);
    }
}

}  // namespace batched
}  // namespace rqb

namespace rqb {
namespace batched {

static size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

static int grow(void** buf, size_t* bytes, size_t need) {
    if (need <= *bytes) return RQB_OK;
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *bytes = 0;
    if (alloc_should_fail()) return RQB_ERR_OOM;
    if (cudaMalloc(buf, need) != cudaSuccess) {
        cudaGetLastError();
        return RQB_ERR_OOM;
    }
    *bytes = need;
    return RQB_OK;
}

namespace {

struct Tables {
    const GMat* mats;
    GState* st;
    const Item* rows;
    const Item* proj;
    const Item* reproj;
    int nrows, nproj, nreproj, count;
    double* rows_part;
    double* proj_part;
    double* gpart;       // BP x BP exact Gram partial per row item
    float* Om[2];        // Omega_1, and the next block's Omega
    int64_t n_max;
    int* blk;            // 0-based index of the block being run
    int max_blocks;
};

// The launches of one block of every active matrix; the block index is read
// on the device (T.blk), so the same launches serve every block.
template <int PW>
void launch_block(cudaStream_t cs, const Tables& T, int b, uint64_t seed, cudaGraphConditionalHandle loop) {
    float* Om_next = T.Om[1];
    k_rows_gram<0><<<T.nrows, NT, 0, cs>>>(T.mats, T.st, T.rows, T.gpart);
    k_mat<kMatPanel1><<<T.count, NT, 0, cs>>>(T.mats, T.st, b, T.rows_part, T.proj_part, T.gpart);
    k_rows<kRowMulR1><<<T.nrows, NT, 0, cs>>>(T.mats, T.st, T.rows, b, nullptr, nullptr);
    // line (3'): both kernels return at once for a matrix with k = 0
    k_cols<kColReproj, TCR><<<T.nreproj, NT, 0, cs>>>(T.mats, T.st, T.reproj, T.blk, nullptr);
    k_rows<kRowSubQC><<<T.nrows, NT, 0, cs>>>(T.mats, T.st, T.rows, b, nullptr, nullptr);
    k_rows_gram<1><<<T.nrows, NT, 0, cs>>>(T.mats, T.st, T.rows, T.gpart);
    k_mat<kMatPanel2><<<T.count, NT, 0, cs>>>(T.mats, T.st, b, T.rows_part, T.proj_part, T.gpart);
    k_rows<kRowMulR2><<<T.nrows, NT, 0, cs>>>(T.mats, T.st, T.rows, b, nullptr, nullptr);
    k_cols<kColProject, PW><<<T.nproj, NT, 0, cs>>>(T.mats, T.st, T.proj, T.blk, T.proj_part);
    k_mat<kMatStop><<<T.count, NT, 0, cs>>>(T.mats, T.st, b, T.rows_part, T.proj_part, T.gpart);
    const int64_t tot = T.n_max * BP;
    k_omega_rows<<<(int)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, cs>>>(T.n_max, T.blk, b, seed, Om_next);
    k_rows_update<<<T.nrows, NTU, 0, cs>>>(T.mats, T.st, T.rows, b, T.blk, Om_next, T.rows_part);
    k_mat<kMatDirect><<<T.count, NT, 0, cs>>>(T.mats, T.st, b, T.rows_part, T.proj_part, T.gpart);
    k_advance<<<1, NT, 0, cs>>>(T.blk, T.st, T.count, T.max_blocks, loop);
}
constexpr int kBlockLaunches = 14;   // kernels per block in launch_block
constexpr int kPrologueLaunches = 3;

}  // namespace

// The factorization of one batch shape as one instantiated graph: a prologue
// (Omega_1, the first sketch with ||A||^2, the initial state, block index 0)
// followed by a WHILE node whose body is launch_block, so that the whole
// batch runs from one cudaGraphLaunch with no host round trip.  Kept by the
// handle and reused while the shape, the workspace and the launch
// parameters are the same; the descriptors and item tables it reads are
// rewritten in device memory before every launch.
struct GraphCache {
    // key
    const void* work = nullptr;
    int64_t count = 0, nrows = 0, nproj = 0, nreproj = 0, n_max = 0, b = 0;
    int max_blocks = 0, pw = 0, device = -1;
    uint64_t seed = 0;
    // graph
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;        // capture stream (the caller's may be the legacy one)
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    // autotuned projection widths, by batch class
    std::vector<std::pair<std::string, int>> tuned;
    bool tuned_loaded = false;
    void drop_graph() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        work = nullptr;
    }
    ~GraphCache() {
        drop_graph();
        if (cap) cudaStreamDestroy(cap);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

void release_cache(void* cache) { delete static_cast<GraphCache*>(cache); }

namespace {

template <int PW>
int build_graph(GraphCache& G, const Tables& T, int b, uint64_t seed) {
    cudaGraph_t g = nullptr, pro = nullptr;
    cudaGraphNode_t npro = nullptr, nloop = nullptr;
    cudaGraphConditionalHandle loop = 0;
    int rc = RQB_OK;
    do {
        if (cudaGraphCreate(&g, 0) != cudaSuccess) { rc = RQB_ERR_CUDA; break; }
        // prologue, captured on the private stream
        if (cudaStreamBeginCapture(G.cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { rc = RQB_ERR_CUDA; break; }
        const int64_t tot = T.n_max * BP;
        k_omega_rows<<<(int)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, G.cap>>>(T.n_max, nullptr, b, seed,
                                                                                       T.Om[0]);
        k_rows<kRowSketch0><<<T.nrows, NT, 0, G.cap>>>(T.mats, T.st, T.rows, b, T.Om[0], T.rows_part);
        k_mat<kMatInit><<<T.count, NT, 0, G.cap>>>(T.mats, T.st, b, T.rows_part, T.proj_part, T.gpart);
        cudaMemsetAsync(T.blk, 0, sizeof(int), G.cap);
        const cudaError_t le = cudaGetLastError();
        if (cudaStreamEndCapture(G.cap, &pro) != cudaSuccess || !pro || le != cudaSuccess) { rc = RQB_ERR_CUDA; break; }
        if (cudaGraphAddChildGraphNode(&npro, g, nullptr, 0, pro) != cudaSuccess) { rc = RQB_ERR_CUDA; break; }
        // the block loop: a WHILE node, its condition set by k_advance
        if (cudaGraphConditionalHandleCreate(&loop, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
            rc = RQB_ERR_CUDA; break;
        }
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = loop;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        if (cudaGraphAddNode(&nloop, g, &npro, nullptr, 1, &cp) != cudaSuccess) { rc = RQB_ERR_CUDA; break; }
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        if (cudaStreamBeginCaptureToGraph(G.cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
            cudaSuccess) { rc = RQB_ERR_CUDA; break; }
        launch_block<PW>(G.cap, T, b, seed, loop);
        const cudaError_t le2 = cudaGetLastError();
        cudaGraph_t same = nullptr;
        if (cudaStreamEndCapture(G.cap, &same) != cudaSuccess || le2 != cudaSuccess) { rc = RQB_ERR_CUDA; break; }
        if (cudaGraphInstantiate(&G.exec, g, 0) != cudaSuccess) { G.exec = nullptr; rc = RQB_ERR_CUDA; break; }
    } while (0);
    if (pro) cudaGraphDestroy(pro);
    if (g) cudaGraphDestroy(g);
    if (rc != RQB_OK) cudaGetLastError();
    return rc;
}

// Batch class of the autotuner: the number of matrices and the sizes, on a
// coarse grid, with b.
std::string batch_class(int64_t count, const int64_t* m, const int64_t* n, int64_t b) {
    int64_t mx_m = 0, mx_n = 0;
    double mn = 0.0;
    for (int64_t t = 0; t < count; ++t) {
        mx_m = std::max(mx_m, m[t]);
        mx_n = std::max(mx_n, n[t]);
        mn += (double)m[t] * (double)n[t];
    }
    char buf[128];
    std::snprintf(buf, sizeof(buf), "c%lld_m%lld_n%lld_mn%lld_b%lld", (long long)count,
                  (long long)((mx_m + 255) / 256), (long long)((mx_n + 127) / 128),
                  (long long)std::llround(std::log2(std::max(mn, 1.0)) * 4.0), (long long)b);
    return std::string(buf);
}

}  // namespace

// Autotuner of the projection's column tile (128 or 256 columns of A per
// work item): the first batch of a class is run with each width and timed on
// the device; the faster width is kept for the class in the handle and, when
// the environment variable RQB_AUTOTUNE_CACHE names a file, appended to that
// file and read back by later processes.  Both widths give the same results
// bit for bit (each B_i entry is one thread's sum over the rows in the same
// order).
static void tune_load(GraphCache& G) {
    if (G.tuned_loaded) return;
    G.tuned_loaded = true;
    const char* path = std::getenv("RQB_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = std::fopen(path, "r");
    if (!f) return;
    char key[256];
    int w = 0;
    while (std::fscanf(f, "batched_projection_width %255s %d\n", key, &w) == 2)
        if (w == 128 || w == 256) G.tuned.emplace_back(std::string(key), w);
    std::fclose(f);
}

static int tune_lookup(const GraphCache& G, const std::string& key) {
    for (auto it = G.tuned.rbegin(); it != G.tuned.rend(); ++it)
        if (it->first == key) return it->second;
    return 0;
}

static void tune_store(GraphCache& G, const std::string& key, int w) {
    G.tuned.emplace_back(key, w);
    const char* path = std::getenv("RQB_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "batched_projection_width %s %d\n", key.c_str(), w);
    std::fclose(f);
}

namespace {

// Host-side layout of one batch for a projection width pw.
struct Layout {
    std::vector<GMat> d;
    std::vector<Item> rows, proj, reproj;
    size_t work_bytes = 0, out_bytes = 0;
    size_t oDesc, oSt, oRows, oProj, oRep, oRp, oPp, oGp, oBlk, oOm0, oOm1;
    std::vector<size_t> oW, qoff, boff;
    int64_t n_max = 1, max_blocks = 1;
};

void make_layout(Layout& L, int pw, int64_t count, const void* const* A, const int64_t* m, const int64_t* n,
                 const int64_t* lda, const double* eps, int64_t b, int64_t max_rank) {
    // largest matrices first: their items are scheduled first in every launch
    std::vector<int> order((size_t)count);
    for (int64_t t = 0; t < count; ++t) order[(size_t)t] = (int)t;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return m[x] * n[x] > m[y] * n[y]; });
    L.d.assign((size_t)count, GMat{});
    L.qoff.assign((size_t)count, 0);
    L.boff.assign((size_t)count, 0);
    size_t total = 0;
    for (int64_t t = 0; t < count; ++t) {
        const int64_t r = std::min(m[t], n[t]);
        const int64_t kc = (max_rank > 0 && max_rank < r) ? max_rank : r;
        GMat& x = L.d[(size_t)t];
        x.A = static_cast<const float*>(A[t]);
        x.m = m[t]; x.n = n[t]; x.lda = lda[t]; x.kcap = kc;
        x.ldq = ((m[t] + 3) / 4) * 4;
        x.ldb = ((kc + 3) / 4) * 4;
        x.ldw = ((m[t] + 3) / 4) * 4;
        x.eps2 = eps[t] * eps[t];
        L.qoff[(size_t)t] = total; total = al256(total + sizeof(float) * (size_t)x.ldq * (size_t)kc);
        L.boff[(size_t)t] = total; total = al256(total + sizeof(float) * (size_t)x.ldb * (size_t)n[t]);
        L.n_max = std::max(L.n_max, n[t]);
        L.max_blocks = std::max(L.max_blocks, (kc + b - 1) / b);
    }
    L.out_bytes = total;
    L.rows.clear(); L.proj.clear(); L.reproj.clear();
    for (int t : order) {
        GMat& x = L.d[(size_t)t];
        x.rows_begin = (int)L.rows.size();
        for (int64_t i = 0; i < (x.m + TR - 1) / TR; ++i) L.rows.push_back(Item{t, (int)i});
        x.rows_end = (int)L.rows.size();
        x.proj_begin = (int)L.proj.size();
        for (int64_t i = 0; i < (x.n + pw - 1) / pw; ++i) L.proj.push_back(Item{t, (int)i});
        x.proj_end = (int)L.proj.size();
        for (int64_t i = 0; i < (x.kcap + TCR - 1) / TCR; ++i) L.reproj.push_back(Item{t, (int)i});
    }
    // work layout: descriptors, state, item tables, partials, block index,
    // Omega x 2, then per matrix W, Y, Y1, Cc, Rinv
    size_t w = 0;
    L.oDesc = w; w = al256(w + sizeof(GMat) * (size_t)count);
    L.oSt = w; w = al256(w + sizeof(GState) * (size_t)count);
    L.oRows = w; w = al256(w + sizeof(Item) * L.rows.size());
    L.oProj = w; w = al256(w + sizeof(Item) * L.proj.size());
    L.oRep = w; w = al256(w + sizeof(Item) * L.reproj.size());
    L.oRp = w; w = al256(w + sizeof(double) * L.rows.size());
    L.oPp = w; w = al256(w + sizeof(double) * L.proj.size());
    L.oGp = w; w = al256(w + sizeof(double) * BP * BP * L.rows.size());
    L.oBlk = w; w = al256(w + sizeof(int));
    L.oOm0 = w; w = al256(w + sizeof(float) * (size_t)L.n_max * BP);
    L.oOm1 = w; w = al256(w + sizeof(float) * (size_t)L.n_max * BP);
    L.oW.assign((size_t)count, 0);
    for (int64_t t = 0; t < count; ++t) {
        const GMat& x = L.d[(size_t)t];
        L.oW[(size_t)t] = w;
        w = al256(w + sizeof(float) * (size_t)x.ldw * (size_t)x.n);          // W
        w = al256(w + sizeof(float) * (size_t)x.ldw * BP);                    // Y
        w = al256(w + sizeof(float) * (size_t)x.ldw * BP);                    // Y1
        w = al256(w + sizeof(float) * (size_t)x.kcap * BP);                   // Cc
        w = al256(w + sizeof(float) * BP * BP);                               // Rinv
    }
    L.work_bytes = w;
}

// Runs the batch with projection width pw through the cached (or a new)
// graph; on success *ms is the device time of the graph and *iters the
// number of blocks the loop ran.
int run_batch(GraphCache& G, Layout& L, int pw, int64_t count, int64_t b, uint64_t seed, cudaStream_t stream,
              int device, void** outbuf, size_t* outbytes, void** workbuf, size_t* workbytes,
              std::vector<GState>& outs, float* ms, int* iters) {
    int rc = grow(outbuf, outbytes, L.out_bytes);
    if (rc != RQB_OK) return rc;
    rc = grow(workbuf, workbytes, L.work_bytes);
    if (rc != RQB_OK) return rc;
    char* ob = static_cast<char*>(*outbuf);
    char* wb = static_cast<char*>(*workbuf);
    for (int64_t t = 0; t < count; ++t) {
        GMat& x = L.d[(size_t)t];
        x.Q = reinterpret_cast<float*>(ob + L.qoff[(size_t)t]);
        x.B = reinterpret_cast<float*>(ob + L.boff[(size_t)t]);
        char* p = wb + L.oW[(size_t)t];
        x.W = reinterpret_cast<float*>(p); p += al256(sizeof(float) * (size_t)x.ldw * (size_t)x.n);
        x.Y = reinterpret_cast<float*>(p); p += al256(sizeof(float) * (size_t)x.ldw * BP);
        x.Y1 = reinterpret_cast<float*>(p); p += al256(sizeof(float) * (size_t)x.ldw * BP);
        x.Cc = reinterpret_cast<float*>(p); p += al256(sizeof(float) * (size_t)x.kcap * BP);
        x.Rinv = reinterpret_cast<float*>(p);
    }
    Tables T;
    T.mats = reinterpret_cast<const GMat*>(wb + L.oDesc);
    T.st = reinterpret_cast<GState*>(wb + L.oSt);
    T.rows = reinterpret_cast<const Item*>(wb + L.oRows);
    T.proj = reinterpret_cast<const Item*>(wb + L.oProj);
    T.reproj = reinterpret_cast<const Item*>(wb + L.oRep);
    T.nrows = (int)L.rows.size();
    T.nproj = (int)L.proj.size();
    T.nreproj = (int)L.reproj.size();
    T.count = (int)count;
    T.rows_part = reinterpret_cast<double*>(wb + L.oRp);
    T.proj_part = reinterpret_cast<double*>(wb + L.oPp);
    T.gpart = reinterpret_cast<double*>(wb + L.oGp);
    T.blk = reinterpret_cast<int*>(wb + L.oBlk);
    T.Om[0] = reinterpret_cast<float*>(wb + L.oOm0);
    T.Om[1] = reinterpret_cast<float*>(wb + L.oOm1);
    T.n_max = L.n_max;
    T.max_blocks = (int)L.max_blocks;

    if (!G.cap && cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking) != cudaSuccess) return RQB_ERR_CUDA;
    if (!G.e0 && cudaEventCreate(&G.e0) != cudaSuccess) return RQB_ERR_CUDA;
    if (!G.e1 && cudaEventCreate(&G.e1) != cudaSuccess) return RQB_ERR_CUDA;
    const bool same = G.exec && G.work == wb && G.count == count && G.nrows == T.nrows && G.nproj == T.nproj &&
                      G.nreproj == T.nreproj && G.n_max == T.n_max && G.b == b && G.max_blocks == T.max_blocks &&
                      G.pw == pw && G.seed == seed && G.device == device;
    if (!same) {
        G.drop_graph();
        rc = (pw == 128) ? build_graph<128>(G, T, (int)b, seed) : build_graph<256>(G, T, (int)b, seed);
        if (rc != RQB_OK) return rc;
        G.work = wb; G.count = count; G.nrows = T.nrows; G.nproj = T.nproj; G.nreproj = T.nreproj;
        G.n_max = T.n_max; G.b = b; G.max_blocks = T.max_blocks; G.pw = pw; G.seed = seed; G.device = device;
    }
    // descriptors and item tables for this call, then the whole factorization
    if (cudaMemcpyAsync(wb + L.oDesc, L.d.data(), sizeof(GMat) * (size_t)count, cudaMemcpyHostToDevice, stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(wb + L.oRows, L.rows.data(), sizeof(Item) * L.rows.size(), cudaMemcpyHostToDevice, stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(wb + L.oProj, L.proj.data(), sizeof(Item) * L.proj.size(), cudaMemcpyHostToDevice, stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(wb + L.oRep, L.reproj.data(), sizeof(Item) * L.reproj.size(), cudaMemcpyHostToDevice,
                        stream) != cudaSuccess)
        return RQB_ERR_CUDA;
    int blk = 0;
    outs.resize((size_t)count);
    if (cudaEventRecord(G.e0, stream) != cudaSuccess || cudaGraphLaunch(G.exec, stream) != cudaSuccess ||
        cudaEventRecord(G.e1, stream) != cudaSuccess ||
        cudaMemcpyAsync(outs.data(), wb + L.oSt, sizeof(GState) * (size_t)count, cudaMemcpyDeviceToHost, stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(&blk, T.blk, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return RQB_ERR_CUDA;
    float t_ms = 0.f;
    cudaEventElapsedTime(&t_ms, G.e0, G.e1);
    *ms = t_ms;
    *iters = blk;
    return RQB_OK;
}

}  // namespace

int factor_batched(cudaStream_t stream, int num_sms, int64_t count, const void* const* A, const int64_t* m,
                   const int64_t* n, const int64_t* lda, const double* eps, int64_t b, uint64_t seed, int64_t max_rank,
                   const void** Q, int64_t* ldq, const void** B, int64_t* ldb, int64_t* k, int* status, void** outbuf,
                   size_t* outbytes, void** workbuf, size_t* workbytes, void** cache, float* ms, int* launches,
                   int* proj_width) {
    (void)num_sms;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return RQB_ERR_CUDA;
    if (!*cache) {
        *cache = new (std::nothrow) GraphCache();
        if (!*cache) return RQB_ERR_OOM;
    }
    GraphCache& G = *static_cast<GraphCache*>(*cache);
    tune_load(G);
    const std::string cls = batch_class(count, m, n, b);
    int pw = tune_lookup(G, cls);
    std::vector<GState> outs;
    Layout L;
    float t_ms = 0.f;
    int iters = 0;
    int rc = RQB_OK;
    if (pw == 0) {
        // first batch of this class: run both widths, keep the faster
        float best = 0.f;
        for (int cand : {256, 128}) {
            make_layout(L, cand, count, A, m, n, lda, eps, b, max_rank);
            rc = run_batch(G, L, cand, count, b, seed, stream, device, outbuf, outbytes, workbuf, workbytes, outs,
                           &t_ms, &iters);
            if (rc != RQB_OK) return rc;
            if (pw == 0 || t_ms < best) {
                best = t_ms;
                pw = cand;
            }
        }
        tune_store(G, cls, pw);
        if (pw != 128) {
            // the outputs of the last run (width 128) are those of the kept
            // width too; the graph of the kept width is built for the next call
            make_layout(L, pw, count, A, m, n, lda, eps, b, max_rank);
            rc = run_batch(G, L, pw, count, b, seed, stream, device, outbuf, outbytes, workbuf, workbytes, outs,
                           &t_ms, &iters);
        }
    } else {
        make_layout(L, pw, count, A, m, n, lda, eps, b, max_rank);
        rc = run_batch(G, L, pw, count, b, seed, stream, device, outbuf, outbytes, workbuf, workbytes, outs, &t_ms,
                       &iters);
    }
    if (rc != RQB_OK) return rc;
    if (ms) *ms = t_ms;
    if (launches) *launches = kPrologueLaunches + kBlockLaunches * iters;
    if (proj_width) *proj_width = pw;
    for (int64_t t = 0; t < count; ++t) {
        Q[t] = L.d[(size_t)t].Q; ldq[t] = L.d[(size_t)t].ldq;
        B[t] = L.d[(size_t)t].B; ldb[t] = L.d[(size_t)t].ldb;
        k[t] = outs[(size_t)t].k; status[t] = outs[(size_t)t].status;
    }
    return RQB_OK;
}

}  // namespace batched
}  // namespace rqb
