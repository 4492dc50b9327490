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
// finished matrices return at once.  Blocks are launched in chunks of eight,
// each chunk captured into one CUDA graph; the host reads the number of
// active matrices between chunks.  Partial sums are combined per matrix in a
// fixed order, so results are bitwise repeatable.
#include <algorithm>
#include <cstring>
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
                                                     const Item* __restrict__ items, int b, int first,
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
    float yacc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) yacc[i][j] = 0.f;
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
        float pacc[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) pacc[i][j] = 0.f;
#pragma unroll 8
        for (int t = 0; t < BP; ++t) {
            const float4 a0 = *reinterpret_cast<const float4*>(&Qs[t][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&Qs[t][ty * 8 + 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float4 b4 = *reinterpret_cast<const float4*>(&Bs[t][tx * 4]);
            const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) pacc[i][j] = fmaf(av[i], bv[j], pacc[i][j]);
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
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) yacc[i][j] = fmaf(av[i], ov[j], yacc[i][j]);
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t r = r0 + ty * 8 + i;
        if (r >= m) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = tx + 8 * j;
            d.Y[r + (int64_t)c * d.ldw] = (c < pn) ? yacc[i][j] : 0.f;
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

template <int OP>
__global__ void __launch_bounds__(NT) k_cols(const GMat* __restrict__ mats, const GState* __restrict__ st,
                                             const Item* __restrict__ items, int first, double* __restrict__ part) {
    constexpr int W = (OP == kColProject) ? TC : TCR;   // columns per item
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
    double acc2[OP == kColReproj ? JT : 1][4];
#pragma unroll
    for (int i = 0; i < JT; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = 0.f;
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
#pragma unroll
            for (int i = 0; i < JT; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[i][q] = fmaf(a[i], v[q], acc[i][q]);
        }
        if (OP == kColReproj && (++chunk == 4 || r0 + KCH >= m)) {
            chunk = 0;
#pragma unroll
            for (int i = 0; i < (OP == kColReproj ? JT : 1); ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    acc2[i][q] += (double)acc[i][q];
                    acc[i][q] = 0.f;
                }
        }
    }
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

// Omega (n_max x BP, row-major): global columns col0 .. col0 + b - 1, zero beyond b.
__global__ void k_omega_rows(int64_t n_max, int64_t col0, int b, uint64_t seed, float* __restrict__ Om) {
    const int64_t total = n_max * BP;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / BP;
        const int c = (int)(e % BP);
        Om[e] = (c < b) ? gaussian_f32(seed, r, col0 + c) : 0.f;
    }
}

__global__ void k_count_active(const GState* __restrict__ st, int count, int* __restrict__ out) {
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
        *out = tot;
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
    if (cudaMalloc(buf, need) != cudaSuccess) {
        cudaGetLastError();
        return RQB_ERR_OOM;
    }
    *bytes = need;
    return RQB_OK;
}

namespace {

constexpr int kChunk = 8;   // blocks per captured graph

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
    float* Om[2];
    int64_t n_max;
};

// The launches of block i (0-based) of every active matrix.
cudaError_t launch_block(cudaStream_t cs, const Tables& T, int i, int b, uint64_t seed, int* launches) {
    const int first = (i == 0) ? 1 : 0;
    const float* Om = T.Om[i & 1];
    float* Om_next = T.Om[(i + 1) & 1];
    k_rows_gram<0><<<T.nrows, NT, 0, cs>>>(T.mats, T.st, T.rows, T.gpart);
    k_mat<kMatPanel1><<<T.count, NT, 0, cs>>>(T.mats, T.st, b, T.rows_part, T.proj_part, T.gpart);
    k_rows<kRowMulR1><<<T.nrows, NT, 0, cs>>>(T.mats, T.st, T.rows, b, Om, nullptr);
    int nl = 3;
    if (i > 0) {
        k_cols<kColReproj><<<T.nreproj, NT, 0, cs>>>(T.mats, T.st, T.reproj, first, nullptr);
        k_rows<kRowSubQC><<<T.nrows, NT, 0, cs>>>(T.mats, T.st, T.rows, b, Om, nullptr);
        nl += 2;
    }
    k_rows_gram<1><<<T.nrows, NT, 0, cs>>>(T.mats, T.st, T.rows, T.gpart);
    k_mat<kMatPanel2><<<T.count, NT, 0, cs>>>(T.mats, T.st, b, T.rows_part, T.proj_part, T.gpart);
    k_rows<kRowMulR2><<<T.nrows, NT, 0, cs>>>(T.mats, T.st, T.rows, b, Om, nullptr);
    k_cols<kColProject><<<T.nproj, NT, 0, cs>>>(T.mats, T.st, T.proj, first, T.proj_part);
    k_mat<kMatStop><<<T.count, NT, 0, cs>>>(T.mats, T.st, b, T.rows_part, T.proj_part, T.gpart);
    const int64_t tot = T.n_max * BP;
    k_omega_rows<<<(int)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, cs>>>(T.n_max, (int64_t)(i + 1) * b, b,
                                                                                 seed, Om_next);
    k_rows_update<<<T.nrows, NTU, 0, cs>>>(T.mats, T.st, T.rows, b, first, Om_next, T.rows_part);
    k_mat<kMatDirect><<<T.count, NT, 0, cs>>>(T.mats, T.st, b, T.rows_part, T.proj_part, T.gpart);
    nl += 8;
    *launches += nl;
    return cudaGetLastError();
}

}  // namespace

int factor_batched(cudaStream_t stream, int num_sms, int64_t count, const void* const* A, const int64_t* m,
                   const int64_t* n, const int64_t* lda, const double* eps, int64_t b, uint64_t seed, int64_t max_rank,
                   const void** Q, int64_t* ldq, const void** B, int64_t* ldb, int64_t* k, int* status, void** outbuf,
                   size_t* outbytes, void** workbuf, size_t* workbytes, float* ms, int* launches) {
    (void)num_sms;
    // largest matrices first: their items are scheduled first in every launch
    std::vector<int> order((size_t)count);
    for (int64_t t = 0; t < count; ++t) order[(size_t)t] = (int)t;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return m[x] * n[x] > m[y] * n[y]; });

    // outputs: Q_t (ldq x kcap), B_t (ldb x n) per matrix
    std::vector<GMat> d((size_t)count);
    std::vector<size_t> qoff((size_t)count), boff((size_t)count);
    size_t total = 0;
    int64_t n_max = 1, max_blocks = 1;
    for (int64_t t = 0; t < count; ++t) {
        const int64_t r = std::min(m[t], n[t]);
        const int64_t kc = (max_rank > 0 && max_rank < r) ? max_rank : r;
        GMat& x = d[(size_t)t];
        x.A = static_cast<const float*>(A[t]);
        x.m = m[t]; x.n = n[t]; x.lda = lda[t]; x.kcap = kc;
        x.ldq = ((m[t] + 3) / 4) * 4;
        x.ldb = ((kc + 3) / 4) * 4;
        x.ldw = ((m[t] + 3) / 4) * 4;
        x.eps2 = eps[t] * eps[t];
        qoff[(size_t)t] = total; total = al256(total + sizeof(float) * (size_t)x.ldq * (size_t)kc);
        boff[(size_t)t] = total; total = al256(total + sizeof(float) * (size_t)x.ldb * (size_t)n[t]);
        n_max = std::max(n_max, n[t]);
        max_blocks = std::max(max_blocks, (kc + b - 1) / b);
    }
    int rc = grow(outbuf, outbytes, total);
    if (rc != RQB_OK) return rc;
    char* ob = static_cast<char*>(*outbuf);
    // work items, in decreasing matrix size
    std::vector<Item> rows, proj, reproj;
    for (int t : order) {
        GMat& x = d[(size_t)t];
        x.Q = reinterpret_cast<float*>(ob + qoff[(size_t)t]);
        x.B = reinterpret_cast<float*>(ob + boff[(size_t)t]);
        x.rows_begin = (int)rows.size();
        for (int64_t i = 0; i < (x.m + TR - 1) / TR; ++i) rows.push_back(Item{t, (int)i});
        x.rows_end = (int)rows.size();
        x.proj_begin = (int)proj.size();
        for (int64_t i = 0; i < (x.n + TC - 1) / TC; ++i) proj.push_back(Item{t, (int)i});
        x.proj_end = (int)proj.size();
        for (int64_t i = 0; i < (x.kcap + TCR - 1) / TCR; ++i) reproj.push_back(Item{t, (int)i});
    }
    // work layout: descriptors, state, item tables, partials, Omega x 2,
    // then per matrix W, Y, Y1, Cc, Rinv
    size_t w = 0;
    const size_t oDesc = w; w = al256(w + sizeof(GMat) * (size_t)count);
    const size_t oSt = w; w = al256(w + sizeof(GState) * (size_t)count);
    const size_t oRows = w; w = al256(w + sizeof(Item) * rows.size());
    const size_t oProj = w; w = al256(w + sizeof(Item) * proj.size());
    const size_t oRep = w; w = al256(w + sizeof(Item) * reproj.size());
    const size_t oRp = w; w = al256(w + sizeof(double) * rows.size());
    const size_t oPp = w; w = al256(w + sizeof(double) * proj.size());
    const size_t oGp = w; w = al256(w + sizeof(double) * BP * BP * rows.size());
    const size_t oCnt = w; w = al256(w + sizeof(int));
    const size_t oOm0 = w; w = al256(w + sizeof(float) * (size_t)n_max * BP);
    const size_t oOm1 = w; w = al256(w + sizeof(float) * (size_t)n_max * BP);
    std::vector<size_t> oW((size_t)count);
    for (int64_t t = 0; t < count; ++t) {
        const GMat& x = d[(size_t)t];
        oW[(size_t)t] = w;
        w = al256(w + sizeof(float) * (size_t)x.ldw * (size_t)x.n);          // W
        w = al256(w + sizeof(float) * (size_t)x.ldw * BP);                    // Y
        w = al256(w + sizeof(float) * (size_t)x.ldw * BP);                    // Y1
        w = al256(w + sizeof(float) * (size_t)x.kcap * BP);                   // Cc
        w = al256(w + sizeof(float) * BP * BP);                               // Rinv
    }
    rc = grow(workbuf, workbytes, w);
    if (rc != RQB_OK) return rc;
    char* wb = static_cast<char*>(*workbuf);
    for (int64_t t = 0; t < count; ++t) {
        GMat& x = d[(size_t)t];
        char* p = wb + oW[(size_t)t];
        x.W = reinterpret_cast<float*>(p); p += al256(sizeof(float) * (size_t)x.ldw * (size_t)x.n);
        x.Y = reinterpret_cast<float*>(p); p += al256(sizeof(float) * (size_t)x.ldw * BP);
        x.Y1 = reinterpret_cast<float*>(p); p += al256(sizeof(float) * (size_t)x.ldw * BP);
        x.Cc = reinterpret_cast<float*>(p); p += al256(sizeof(float) * (size_t)x.kcap * BP);
        x.Rinv = reinterpret_cast<float*>(p);
    }
    Tables T;
    T.mats = reinterpret_cast<const GMat*>(wb + oDesc);
    T.st = reinterpret_cast<GState*>(wb + oSt);
    T.rows = reinterpret_cast<const Item*>(wb + oRows);
    T.proj = reinterpret_cast<const Item*>(wb + oProj);
    T.reproj = reinterpret_cast<const Item*>(wb + oRep);
    T.nrows = (int)rows.size();
    T.nproj = (int)proj.size();
    T.nreproj = (int)reproj.size();
    T.count = (int)count;
    T.rows_part = reinterpret_cast<double*>(wb + oRp);
    T.proj_part = reinterpret_cast<double*>(wb + oPp);
    T.gpart = reinterpret_cast<double*>(wb + oGp);
    T.Om[0] = reinterpret_cast<float*>(wb + oOm0);
    T.Om[1] = reinterpret_cast<float*>(wb + oOm1);
    T.n_max = n_max;
    int* dcount = reinterpret_cast<int*>(wb + oCnt);

    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return RQB_ERR_CUDA;
    cudaEvent_t e0 = nullptr, e1 = nullptr, dep = nullptr;
    int nl = 0;
    rc = RQB_OK;
    do {
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
            cudaEventCreateWithFlags(&dep, cudaEventDisableTiming) != cudaSuccess) { rc = RQB_ERR_CUDA; break; }
        // order after earlier work on the caller's stream
        if (cudaEventRecord(dep, stream) != cudaSuccess || cudaStreamWaitEvent(cs, dep, 0) != cudaSuccess) {
            rc = RQB_ERR_CUDA; break;
        }
        if (cudaMemcpyAsync(wb + oDesc, d.data(), sizeof(GMat) * (size_t)count, cudaMemcpyHostToDevice, cs) !=
                cudaSuccess ||
            cudaMemcpyAsync(wb + oRows, rows.data(), sizeof(Item) * rows.size(), cudaMemcpyHostToDevice, cs) !=
                cudaSuccess ||
            cudaMemcpyAsync(wb + oProj, proj.data(), sizeof(Item) * proj.size(), cudaMemcpyHostToDevice, cs) !=
                cudaSuccess ||
            cudaMemcpyAsync(wb + oRep, reproj.data(), sizeof(Item) * reproj.size(), cudaMemcpyHostToDevice, cs) !=
                cudaSuccess) { rc = RQB_ERR_CUDA; break; }
        if (cudaEventRecord(e0, cs) != cudaSuccess) { rc = RQB_ERR_CUDA; break; }
        // block 1's sketch and the initial state
        const int64_t tot = n_max * BP;
        k_omega_rows<<<(int)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, cs>>>(n_max, 0, (int)b, seed,
                                                                                     T.Om[0]);
        k_rows<kRowSketch0><<<T.nrows, NT, 0, cs>>>(T.mats, T.st, T.rows, (int)b, T.Om[0], T.rows_part);
        k_mat<kMatInit><<<T.count, NT, 0, cs>>>(T.mats, T.st, (int)b, T.rows_part, T.proj_part, T.gpart);
        nl += 3;
        if (cudaGetLastError() != cudaSuccess) { rc = RQB_ERR_CUDA; break; }
        // blocks in chunks of kChunk, each chunk one captured graph
        for (int i0 = 0; i0 < (int)max_blocks && rc == RQB_OK; i0 += kChunk) {
            const int i1 = std::min<int>((int)max_blocks, i0 + kChunk);
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { rc = RQB_ERR_CUDA; break; }
            cudaError_t le = cudaSuccess;
            for (int i = i0; i < i1 && le == cudaSuccess; ++i) le = launch_block(cs, T, i, (int)b, seed, &nl);
            if (le == cudaSuccess) k_count_active<<<1, NT, 0, cs>>>(T.st, T.count, dcount);
            if (cudaStreamEndCapture(cs, &graph) != cudaSuccess || !graph || le != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                rc = RQB_ERR_CUDA;
                break;
            }
            nl += 1;
            int active = 0;
            if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess || cudaGraphLaunch(exec, cs) != cudaSuccess ||
                cudaMemcpyAsync(&active, dcount, sizeof(int), cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
                cudaStreamSynchronize(cs) != cudaSuccess)
                rc = RQB_ERR_CUDA;
            if (exec) cudaGraphExecDestroy(exec);
            cudaGraphDestroy(graph);
            if (rc == RQB_OK && active == 0) break;
        }
        if (rc != RQB_OK) break;
        if (cudaEventRecord(e1, cs) != cudaSuccess) { rc = RQB_ERR_CUDA; break; }
        std::vector<GState> outs((size_t)count);
        if (cudaMemcpyAsync(outs.data(), wb + oSt, sizeof(GState) * (size_t)count, cudaMemcpyDeviceToHost, cs) !=
                cudaSuccess ||
            cudaStreamSynchronize(cs) != cudaSuccess) { rc = RQB_ERR_CUDA; break; }
        float t_ms = 0.f;
        cudaEventElapsedTime(&t_ms, e0, e1);
        if (ms) *ms = t_ms;
        if (launches) *launches = nl;
        for (int64_t t = 0; t < count; ++t) {
            Q[t] = d[(size_t)t].Q; ldq[t] = d[(size_t)t].ldq;
            B[t] = d[(size_t)t].B; ldb[t] = d[(size_t)t].ldb;
            k[t] = outs[(size_t)t].k; status[t] = outs[(size_t)t].status;
        }
    } while (0);
    if (rc != RQB_OK) cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (dep) cudaEventDestroy(dep);
    cudaStreamDestroy(cs);
    return rc;
}

}  // namespace batched
}  // namespace rqb
