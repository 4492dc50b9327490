// rqb_batched.cu -- randQB_b for many independent matrices of uneven sizes in
// one persistent launch (FP32, block size b <= 32).
//
// Each CTA repeatedly takes the next matrix from a device work counter (the
// host orders the matrices by decreasing m n, so the largest start first) and
// runs the whole of Fig. randQB_b on it with CTA-level tile routines:
//   line (2)  Omega_i into an L2-resident per-CTA buffer (Philox + Box-Muller)
//   line (3)  Y = A Omega_i (first block; later blocks from the fused pass)
//   (3), (3') CholeskyQR2 with re-projection, Gram in FP32 pairs promoted to
//             FP64, Cholesky in FP64
//   line (4)  B_i = Q_i^T A, ||B_i||^2 in FP64
//   line (6)  stop on E_i <= eps^2 outside the FP32 rounding band, else on
//             the direct ||A^(i)||^2 of the fused pass
//   line (5)  A - Q_i B_i fused with the next block's sketch
// Nothing waits on another CTA, so there is no inter-CTA synchronisation.
#include <algorithm>
#include <cstring>
#include <vector>

#include "rqb_engine.h"
#include "rqb_gemm_simt.cuh"

namespace rqb {
namespace batched {

constexpr int NT = 256;          // threads per CTA
constexpr int BP = 32;           // padded block width
constexpr int RB = 256;          // rows per row tile
constexpr int KC = 16;           // reduction chunk

struct MatDesc {
    const float* A;
    float* W;        // residual copy (ld ldw)
    float* Q;        // m x kcap (ld ldq)
    float* B;        // kcap x n (ld ldb)
    int64_t m, n, lda, ldw, ldq, ldb, kcap;
    double eps2;
};

struct MatOut {
    int64_t k;
    int32_t status;
    int32_t blocks;
    double normA2;
    double E;
};

struct Smem {
    float tA[KC][RB + 4];        // X chunk: KC reduction rows x RB outputs
    float tB[KC][BP + 4];        // C chunk: KC x BP
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

// Out (rows x nout, ld ldo) = alpha * X (rows x K) * C (K x BP) + beta * Yin,
// C(k, j) = C[k * csk + j * csj].  Thread (ty, tx): rows ty*8..+7, cols tx*4..+3
// of each 256-row tile.  Optionally ||X||_F^2 into *nrm (FP64, CTA-uniform).
__device__ void cta_nn(Smem& s, int64_t rows, int64_t K, const float* X, int64_t ldx, const float* C, int64_t csk,
                       int64_t csj, float* Out, int64_t ldo, int nout, float alpha, float beta, const float* Yin,
                       int64_t ldyin, double* nrm) {
    const int tid = threadIdx.x, ty = tid >> 3, tx = tid & 7;
    double nacc = 0.0;
    const bool want_norm = (nrm != nullptr);
    for (int64_t r0 = 0; r0 < rows; r0 += RB) {
        float acc[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        for (int64_t k0 = 0; k0 < K; k0 += KC) {
            // X chunk: KC columns x RB rows (column-major runs of RB rows)
            float sq = 0.f;
            for (int v = tid; v < KC * RB; v += NT) {
                const int kk = v / RB, rr = v % RB;
                const int64_t r = r0 + rr, k = k0 + kk;
                const float x = (r < rows && k < K) ? X[r + k * ldx] : 0.f;
                s.tA[kk][rr] = x;
                sq = fmaf(x, x, sq);
            }
            if (want_norm) nacc += (double)sq;
            for (int v = tid; v < KC * BP; v += NT) {
                const int kk = v / BP, j = v % BP;
                const int64_t k = k0 + kk;
                s.tB[kk][j] = (k < K) ? C[k * csk + j * csj] : 0.f;
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < KC; ++kk) {
                float a[8], b[4];
#pragma unroll
                for (int i = 0; i < 8; ++i) a[i] = s.tA[kk][ty * 8 + i];
#pragma unroll
                for (int j = 0; j < 4; ++j) b[j] = s.tB[kk][tx * 4 + j];
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t r = r0 + ty * 8 + i;
            if (r >= rows) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = tx * 4 + j;
                if (c >= nout) continue;
                float v = alpha * acc[i][j];
                if (beta != 0.f) v = fmaf(beta, Yin[r + (int64_t)c * ldyin], v);
                Out[r + (int64_t)c * ldo] = v;
            }
        }
    }
    __syncthreads();   // Out is read by the next routine
    if (nrm) {
        const double t = cta_sum(nacc, s);
        if (threadIdx.x == 0) *nrm = t;
        __syncthreads();
    }
}

// Out (P x BP, FP64, ld ldo) = X^T Y over `rows` rows; X rows x P (ld ldx),
// Y rows x BP (ld ldy).  FP32 products summed over 128-row chunks, promoted
// to FP64 after each chunk.  Thread (ty, tx): P entries ty*8..+7 of each 256-wide
// P tile, columns tx*4..+3.
__device__ void cta_tn(Smem& s, int64_t rows, int64_t P, const float* X, int64_t ldx, const float* Y, int64_t ldy,
                       double* Out, int64_t ldo) {
    const int tid = threadIdx.x, ty = tid >> 3, tx = tid & 7;
    for (int64_t p0 = 0; p0 < P; p0 += RB) {
        double acc2[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc2[i][j] = 0.0;
        float acc[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        int chunk = 0;
        for (int64_t k0 = 0; k0 < rows; k0 += KC) {
            for (int v = tid; v < KC * RB; v += NT) {
                const int pp = v / KC, kk = v % KC;      // column-major runs of KC rows
                const int64_t pc = p0 + pp, r = k0 + kk;
                s.tA[kk][pp] = (pc < P && r < rows) ? X[r + pc * ldx] : 0.f;
            }
            for (int v = tid; v < KC * BP; v += NT) {
                const int j = v / KC, kk = v % KC;
                const int64_t r = k0 + kk;
                s.tB[kk][j] = (r < rows) ? Y[r + (int64_t)j * ldy] : 0.f;
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < KC; ++kk) {
                float a[8], b[4];
#pragma unroll
                for (int i = 0; i < 8; ++i) a[i] = s.tA[kk][ty * 8 + i];
#pragma unroll
                for (int j = 0; j < 4; ++j) b[j] = s.tB[kk][tx * 4 + j];
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
            }
            if (++chunk == 8 || k0 + KC >= rows) {   // promote every 128 rows
                chunk = 0;
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) { acc2[i][j] += (double)acc[i][j]; acc[i][j] = 0.f; }
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t pc = p0 + ty * 8 + i;
            if (pc >= P) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) Out[pc + (int64_t)(tx * 4 + j) * ldo] = acc2[i][j];
        }
    }
    __syncthreads();
}

// s.G (BP x BP, FP64) = Y^T Y over `rows` rows with error-free FP32
// accumulation (exact products, TwoSum into an FP32 pair, promoted to FP64
// every 256 rows).  Thread (ti, tj): entries ti*2..+1 x tj*2..+1.
__device__ void cta_gram_exact(Smem& s, int64_t rows, const float* Y, int64_t ldy) {
    const int tid = threadIdx.x, ti = tid >> 4, tj = tid & 15;
    constexpr int CH = 120;   // CH x (BP + 1) floats fit in tA (KC x (RB + 4))
    static_assert(CH * (BP + 1) <= KC * (RB + 4), "Gram staging must fit in tA");
    float (*tY)[BP + 1] = reinterpret_cast<float (*)[BP + 1]>(&s.tA[0][0]);
    double acc2[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int64_t r0 = 0; r0 < rows; r0 += CH) {
        for (int v = tid; v < CH * BP; v += NT) {
            const int j = v / CH, rr = v % CH;
            const int64_t r = r0 + rr;
            tY[rr][j] = (r < rows) ? Y[r + (int64_t)j * ldy] : 0.f;
        }
        __syncthreads();
        float hi[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, lo[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
        for (int rr = 0; rr < CH; ++rr) {
            const float a0 = tY[rr][ti * 2], a1 = tY[rr][ti * 2 + 1];
            const float b0 = tY[rr][tj * 2], b1 = tY[rr][tj * 2 + 1];
            exact_fma_acc(a0, b0, hi[0][0], lo[0][0]);
            exact_fma_acc(a0, b1, hi[0][1], lo[0][1]);
            exact_fma_acc(a1, b0, hi[1][0], lo[1][0]);
            exact_fma_acc(a1, b1, hi[1][1], lo[1][1]);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) acc2[i][j] += (double)hi[i][j] + (double)lo[i][j];
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) s.G[ti * 2 + i][tj * 2 + j] = acc2[i][j];
    __syncthreads();
}

// Cholesky of s.G (p x p valid, identity beyond), then s.Rinv = R^{-1} (FP32).
// Returns false (CTA-uniform) on a pivot <= tol * G_jj.
__device__ bool cta_chol_inv(Smem& s, int p, double tol) {
    const int tid = threadIdx.x;
    __shared__ double diag0[BP];
    for (int r = tid; r < BP; r += NT) diag0[r] = (r < p) ? s.G[r][r] : 1.0;
    // identity beyond p
    for (int e = tid; e < BP * BP; e += NT) {
        const int r = e / BP, c = e % BP;
        if (r >= p || c >= p) s.G[r][c] = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    bool ok = true;
    for (int j = 0; j < p; ++j) {
        const double d = s.G[j][j];
        if (!(d > tol * diag0[j]) || !isfinite(d)) { ok = false; break; }
        const double invd = 1.0 / d;
        for (int e = tid; e < BP * BP; e += NT) {     // upper triangle r <= c, both > j
            const int r = e / BP, c = e % BP;
            if (r > j && c >= r && c < p) s.G[r][c] -= s.G[j][r] * s.G[j][c] * invd;
        }
        __syncthreads();
    }
    if (!ok) return false;
    // R[r][c] = G[r][c] / sqrt(d_r) (upper), stored back in s.G
    __shared__ double rd[BP];
    for (int r = tid; r < BP; r += NT) rd[r] = sqrt(s.G[r][r]);
    __syncthreads();
    for (int e = tid; e < BP * BP; e += NT) {
        const int r = e / BP, c = e % BP;
        double v = 0.0;
        if (c > r) v = s.G[r][c] / rd[r];
        else if (c == r) v = rd[r];
        s.G[r][c] = v;   // each entry read and written by its own thread
    }
    __syncthreads();
    // inverse: thread c < BP solves R x = e_c (column c of R^{-1})
    if (tid < BP) {
        const int c = tid;
        double x[BP];
#pragma unroll
        for (int r = 0; r < BP; ++r) x[r] = (r == c) ? 1.0 : 0.0;
        for (int t = c; t >= 0; --t) {
            const double xt = x[t] / s.G[t][t];
            x[t] = xt;
            for (int r = 0; r < t; ++r) x[r] -= s.G[r][t] * xt;
        }
        for (int r = 0; r < BP; ++r) s.Rinv[r][c] = (r <= c) ? (float)x[r] : 0.f;
    }
    __syncthreads();
    return true;
}

// Omega_i (n x BP, row-major, columns >= p zero): global columns col0 .. col0 + p - 1.
__device__ void cta_omega(int64_t n, int64_t col0, int p, uint64_t seed, float* Om) {
    for (int64_t e = threadIdx.x; e < n * BP; e += NT) {
        const int64_t r = e / BP;
        const int c = (int)(e % BP);
        Om[e] = (c < p) ? gaussian_f32(seed, r, col0 + c) : 0.f;
    }
    __syncthreads();
}

// Line (5) fused with line (3) of the next block:  Wdst = Wsrc - Q_i B_i over the
// whole matrix and Y (m x BP) = Wdst Omega; returns ||Wdst||_F^2 (CTA-uniform).
// Per 256-row tile: Q_i rows staged in shared memory; per KC-column chunk the
// rank-p update is formed (thread: rows ty*8..+7, columns tx*2..+1 of the
// chunk), written back, staged transposed and multiplied by the Omega chunk.
__device__ double cta_downdate_sketch(Smem& s, float (*Qs)[RB + 4], float (*Bs)[KC + 1], int64_t m, int64_t n, int p,
                                      const float* Wsrc, int64_t ldws, const float* Qi, int64_t ldq, const float* Bi,
                                      int64_t ldb, const float* Om, float* Wdst, int64_t ldwd, float* Y) {
    const int tid = threadIdx.x, ty = tid >> 3, tx = tid & 7;
    double nacc = 0.0;
    for (int64_t r0 = 0; r0 < m; r0 += RB) {
        for (int v = tid; v < BP * RB; v += NT) {
            const int t = v / RB, rr = v % RB;
            const int64_t r = r0 + rr;
            Qs[t][rr] = (t < p && r < m) ? Qi[r + (int64_t)t * ldq] : 0.f;
        }
        float yacc[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) yacc[i][j] = 0.f;
        for (int64_t c0 = 0; c0 < n; c0 += KC) {
            for (int v = tid; v < BP * KC; v += NT) {
                const int cc = v / BP, t = v % BP;
                const int64_t c = c0 + cc;
                Bs[t][cc] = (t < p && c < n) ? Bi[t + c * ldb] : 0.f;
            }
            for (int v = tid; v < KC * BP; v += NT) {
                const int cc = v / BP, j = v % BP;
                const int64_t c = c0 + cc;
                s.tB[cc][j] = (c < n) ? Om[c * BP + j] : 0.f;
            }
            __syncthreads();
            float pacc[8][2];
#pragma unroll
            for (int i = 0; i < 8; ++i) { pacc[i][0] = 0.f; pacc[i][1] = 0.f; }
            for (int t = 0; t < BP; ++t) {
                const float b0 = Bs[t][tx * 2], b1 = Bs[t][tx * 2 + 1];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float a = Qs[t][ty * 8 + i];
                    pacc[i][0] = fmaf(a, b0, pacc[i][0]);
                    pacc[i][1] = fmaf(a, b1, pacc[i][1]);
                }
            }
            float sq = 0.f;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int cc = tx * 2 + j;
                const int64_t c = c0 + cc;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int rr = ty * 8 + i;
                    const int64_t r = r0 + rr;
                    float w = 0.f;
                    if (r < m && c < n) {
                        w = Wsrc[r + c * ldws] - pacc[i][j];
                        Wdst[r + c * ldwd] = w;
                    }
                    sq = fmaf(w, w, sq);
                    s.tA[cc][rr] = w;
                }
            }
            nacc += (double)sq;
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < KC; ++kk) {
                float a[8], b[4];
#pragma unroll
                for (int i = 0; i < 8; ++i) a[i] = s.tA[kk][ty * 8 + i];
#pragma unroll
                for (int j = 0; j < 4; ++j) b[j] = s.tB[kk][tx * 4 + j];
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) yacc[i][j] = fmaf(a[i], b[j], yacc[i][j]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t r = r0 + ty * 8 + i;
            if (r >= m) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) Y[r + (int64_t)(tx * 4 + j) * m] = yacc[i][j];
        }
        __syncthreads();
    }
    return cta_sum(nacc, s);
}

// B_i (p x n, written into B at row offset, ld ldb) = Q_i^T W; returns ||B_i||^2.
// Thread (ty, tx): W columns ty*8..+7 of each 256-column tile, rows tx*4..+3 of B_i.
__device__ double cta_project(Smem& s, int64_t m, int64_t n, int p, const float* Qi, int64_t ldq, const float* W,
                              int64_t ldw, float* Bi, int64_t ldb) {
    const int tid = threadIdx.x, ty = tid >> 3, tx = tid & 7;
    double nb = 0.0;
    for (int64_t c0 = 0; c0 < n; c0 += RB) {
        float acc[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        for (int64_t k0 = 0; k0 < m; k0 += KC) {
            for (int v = tid; v < KC * RB; v += NT) {
                const int cc = v / KC, kk = v % KC;
                const int64_t c = c0 + cc, r = k0 + kk;
                s.tA[kk][cc] = (c < n && r < m) ? W[r + c * ldw] : 0.f;
            }
            for (int v = tid; v < KC * BP; v += NT) {
                const int j = v / KC, kk = v % KC;
                const int64_t r = k0 + kk;
                s.tB[kk][j] = (j < p && r < m) ? Qi[r + (int64_t)j * ldq] : 0.f;
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < KC; ++kk) {
                float a[8], b[4];
#pragma unroll
                for (int i = 0; i < 8; ++i) a[i] = s.tA[kk][ty * 8 + i];
#pragma unroll
                for (int j = 0; j < 4; ++j) b[j] = s.tB[kk][tx * 4 + j];
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t c = c0 + ty * 8 + i;
            if (c >= n) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int t = tx * 4 + j;
                if (t >= p) continue;
                Bi[t + c * ldb] = acc[i][j];
                nb += (double)acc[i][j] * (double)acc[i][j];
            }
        }
    }
    return cta_sum(nb, s);
}

// Per-CTA global scratch for the matrix being factored.
struct SlotBuf {
    float* Om;   // n_max x BP row-major
    float* Y;    // m_max x BP
    float* Y1;   // m_max x BP
    float* W;    // m_max x n_max residual (ld m)
    float* Cc;   // kcap_max x BP
    double* Cd;  // kcap_max x BP
};

// Lines (3), (3'): Qout (p columns) from Y (BP columns, zero beyond p) and
// Qbar (kprev columns): CholeskyQR, re-projection, CholeskyQR.
__device__ bool cta_panel(Smem& s, int64_t m, int p, const float* Y, float* Y1, const float* Qbar, int64_t kprev,
                          int64_t ldq, double* Cd, float* Cc, float* Qout) {
    cta_gram_exact(s, m, Y, m);
    if (!cta_chol_inv(s, p, 1e-14)) return false;
    cta_nn(s, m, BP, Y, m, &s.Rinv[0][0], BP + 1, 1, Y1, m, BP, 1.f, 0.f, nullptr, 0, nullptr);
    if (kprev > 0) {
        cta_tn(s, m, kprev, Qbar, ldq, Y1, m, Cd, kprev);
        for (int64_t e = threadIdx.x; e < kprev * BP; e += NT) Cc[e] = (float)Cd[e];
        __syncthreads();
        cta_nn(s, m, kprev, Qbar, ldq, Cc, 1, kprev, Y1, m, BP, -1.f, 1.f, Y1, m, nullptr);
    }
    cta_gram_exact(s, m, Y1, m);
    if (!cta_chol_inv(s, p, 1e-14)) return false;
    cta_nn(s, m, BP, Y1, m, &s.Rinv[0][0], BP + 1, 1, Qout, ldq, p, 1.f, 0.f, nullptr, 0, nullptr);
    return true;
}

__global__ void __launch_bounds__(NT, 1)
k_batched(const MatDesc* __restrict__ descs, const int* __restrict__ order, int count, const SlotBuf* __restrict__ slots,
          MatOut* __restrict__ outs, int b, uint64_t seed, int* counter) {
    extern __shared__ __align__(16) float dyn[];
    float (*Qs)[RB + 4] = reinterpret_cast<float (*)[RB + 4]>(dyn);
    float (*Bs)[KC + 1] = reinterpret_cast<float (*)[KC + 1]>(dyn + BP * (RB + 4));
    __shared__ Smem s;
    __shared__ int cur;
    const SlotBuf sl = slots[blockIdx.x];
    const double tau_rel = 32.0 * 5.9604644775390625e-08;   // FP32 rounding band of E
    for (;;) {
        if (threadIdx.x == 0) cur = atomicAdd(counter, 1);
        __syncthreads();
        const int idx = cur;
        __syncthreads();
        if (idx >= count) break;
        const int t = order[idx];
        const MatDesc d = descs[t];
        const int64_t m = d.m, n = d.n, kcap = d.kcap;
        int p = (int)min((int64_t)b, kcap);
        cta_omega(n, 0, p, seed, sl.Om);
        cta_nn(s, m, n, d.A, d.lda, sl.Om, BP, 1, sl.Y, m, BP, 1.f, 0.f, nullptr, 0, &s.scal[0]);
        const double N0 = s.scal[0];
        double E = N0;
        const double tau = tau_rel * N0;
        int64_t k = 0;
        int blocks = 0, status = RQB_NOT_CONVERGED;
        const float* Wsrc = d.A;
        int64_t ldws = d.lda;
        if (!isfinite(N0)) status = RQB_ERR_NONFINITE;
        while (status == RQB_NOT_CONVERGED) {
            p = (int)min((int64_t)b, kcap - k);
            float* Qi = d.Q + k * d.ldq;
            float* Bi = d.B + k;
            if (!cta_panel(s, m, p, sl.Y, sl.Y1, d.Q, k, d.ldq, sl.Cd, sl.Cc, Qi)) {
                status = RQB_ERR_BREAKDOWN;
                break;
            }
            const double nb = cta_project(s, m, n, p, Qi, d.ldq, Wsrc, ldws, Bi, d.ldb);
            E -= nb;
            k += p;
            ++blocks;
            const int flag = (E <= d.eps2 - tau) ? kStop : (E > d.eps2 + tau) ? kContinue : kAmbiguous;
            if (flag == kStop) { status = RQB_OK; break; }
            if (flag == kContinue && k >= kcap) break;
            const int pn = (int)min((int64_t)b, max((int64_t)0, kcap - k));
            cta_omega(n, k, pn, seed, sl.Om);
            const double D = cta_downdate_sketch(s, Qs, Bs, m, n, p, Wsrc, ldws, Qi, d.ldq, Bi, d.ldb, sl.Om, sl.W, m,
                                                 sl.Y);
            Wsrc = sl.W;
            ldws = m;
            if (flag == kAmbiguous && D <= d.eps2) { status = RQB_OK; break; }
            if (k >= kcap) break;
        }
        if (threadIdx.x == 0) {
            MatOut o;
            o.k = k; o.status = status; o.blocks = blocks; o.normA2 = N0; o.E = E;
            outs[t] = o;
        }
        __syncthreads();
    }
}

constexpr size_t kDynSmem = sizeof(float) * ((size_t)BP * (RB + 4) + (size_t)BP * (KC + 1));

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

int factor_batched(cudaStream_t stream, int num_sms, int64_t count, const void* const* A, const int64_t* m,
                   const int64_t* n, const int64_t* lda, const double* eps, int64_t b, uint64_t seed, int64_t max_rank,
                   const void** Q, int64_t* ldq, const void** B, int64_t* ldb, int64_t* k, int* status, void** outbuf,
                   size_t* outbytes, void** workbuf, size_t* workbytes, float* ms, int* launches) {
    // output layout and sizes
    std::vector<MatDesc> d((size_t)count);
    std::vector<size_t> qoff((size_t)count), boff((size_t)count);
    size_t total = 0;
    int64_t m_max = 1, n_max = 1, kcap_max = 1;
    for (int64_t t = 0; t < count; ++t) {
        const int64_t r = std::min(m[t], n[t]);
        const int64_t kc = (max_rank > 0 && max_rank < r) ? max_rank : r;
        MatDesc& x = d[(size_t)t];
        x.A = static_cast<const float*>(A[t]);
        x.m = m[t]; x.n = n[t]; x.lda = lda[t]; x.kcap = kc;
        x.ldq = ((m[t] + 3) / 4) * 4;
        x.ldb = ((kc + 3) / 4) * 4;
        x.ldw = m[t];
        x.eps2 = eps[t] * eps[t];
        qoff[(size_t)t] = total; total = al256(total + sizeof(float) * (size_t)x.ldq * (size_t)kc);
        boff[(size_t)t] = total; total = al256(total + sizeof(float) * (size_t)x.ldb * (size_t)n[t]);
        m_max = std::max(m_max, m[t]); n_max = std::max(n_max, n[t]); kcap_max = std::max(kcap_max, kc);
    }
    int rc = grow(outbuf, outbytes, total);
    if (rc != RQB_OK) return rc;
    char* ob = static_cast<char*>(*outbuf);
    for (int64_t t = 0; t < count; ++t) {
        d[(size_t)t].Q = reinterpret_cast<float*>(ob + qoff[(size_t)t]);
        d[(size_t)t].B = reinterpret_cast<float*>(ob + boff[(size_t)t]);
        d[(size_t)t].W = nullptr;
    }
    // work layout: descriptors, order, outputs, counter, slot table, slot arrays
    const int nslots = std::max(1, num_sms);
    size_t w = 0;
    const size_t oDesc = w; w = al256(w + sizeof(MatDesc) * (size_t)count);
    const size_t oOrder = w; w = al256(w + sizeof(int) * (size_t)count);
    const size_t oOuts = w; w = al256(w + sizeof(MatOut) * (size_t)count);
    const size_t oCnt = w; w = al256(w + sizeof(int));
    const size_t oSlots = w; w = al256(w + sizeof(SlotBuf) * (size_t)nslots);
    const size_t per_slot = al256(sizeof(float) * (size_t)n_max * BP) + 2 * al256(sizeof(float) * (size_t)m_max * BP) +
                            al256(sizeof(float) * (size_t)m_max * (size_t)n_max) +
                            al256(sizeof(float) * (size_t)kcap_max * BP) + al256(sizeof(double) * (size_t)kcap_max * BP);
    const size_t oSlotData = w; w += per_slot * (size_t)nslots;
    rc = grow(workbuf, workbytes, w);
    if (rc != RQB_OK) return rc;
    char* wb = static_cast<char*>(*workbuf);
    std::vector<SlotBuf> sl((size_t)nslots);
    for (int i = 0; i < nslots; ++i) {
        char* p = wb + oSlotData + per_slot * (size_t)i;
        sl[(size_t)i].Om = reinterpret_cast<float*>(p); p += al256(sizeof(float) * (size_t)n_max * BP);
        sl[(size_t)i].Y = reinterpret_cast<float*>(p); p += al256(sizeof(float) * (size_t)m_max * BP);
        sl[(size_t)i].Y1 = reinterpret_cast<float*>(p); p += al256(sizeof(float) * (size_t)m_max * BP);
        sl[(size_t)i].W = reinterpret_cast<float*>(p); p += al256(sizeof(float) * (size_t)m_max * (size_t)n_max);
        sl[(size_t)i].Cc = reinterpret_cast<float*>(p); p += al256(sizeof(float) * (size_t)kcap_max * BP);
        sl[(size_t)i].Cd = reinterpret_cast<double*>(p);
    }
    // largest matrices first (longest-processing-time order)
    std::vector<int> order((size_t)count);
    for (int64_t t = 0; t < count; ++t) order[(size_t)t] = (int)t;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return m[x] * n[x] > m[y] * n[y]; });
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return RQB_ERR_CUDA;
    cudaEvent_t e0 = nullptr, e1 = nullptr, dep = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    rc = RQB_OK;
    do {
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
            cudaEventCreateWithFlags(&dep, cudaEventDisableTiming) != cudaSuccess) { rc = RQB_ERR_CUDA; break; }
        // order after earlier work on the caller's stream
        if (cudaEventRecord(dep, stream) != cudaSuccess || cudaStreamWaitEvent(cs, dep, 0) != cudaSuccess) {
            rc = RQB_ERR_CUDA; break;
        }
        if (cudaMemcpyAsync(wb + oDesc, d.data(), sizeof(MatDesc) * (size_t)count, cudaMemcpyHostToDevice, cs) !=
                cudaSuccess ||
            cudaMemcpyAsync(wb + oOrder, order.data(), sizeof(int) * (size_t)count, cudaMemcpyHostToDevice, cs) !=
                cudaSuccess ||
            cudaMemcpyAsync(wb + oSlots, sl.data(), sizeof(SlotBuf) * (size_t)nslots, cudaMemcpyHostToDevice, cs) !=
                cudaSuccess) { rc = RQB_ERR_CUDA; break; }
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDynSmem);
            attr = true;
        }
        // one launch (counter reset + persistent kernel) captured into a graph
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { rc = RQB_ERR_CUDA; break; }
        cudaMemsetAsync(wb + oCnt, 0, sizeof(int), cs);
        k_batched<<<nslots, NT, kDynSmem, cs>>>(reinterpret_cast<const MatDesc*>(wb + oDesc),
                                                reinterpret_cast<const int*>(wb + oOrder), (int)count,
                                                reinterpret_cast<const SlotBuf*>(wb + oSlots),
                                                reinterpret_cast<MatOut*>(wb + oOuts), (int)b, seed,
                                                reinterpret_cast<int*>(wb + oCnt));
        if (cudaStreamEndCapture(cs, &graph) != cudaSuccess || !graph) { rc = RQB_ERR_CUDA; break; }
        if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) { rc = RQB_ERR_CUDA; break; }
        if (cudaEventRecord(e0, cs) != cudaSuccess || cudaGraphLaunch(exec, cs) != cudaSuccess ||
            cudaEventRecord(e1, cs) != cudaSuccess) { rc = RQB_ERR_CUDA; break; }
        std::vector<MatOut> outs((size_t)count);
        if (cudaMemcpyAsync(outs.data(), wb + oOuts, sizeof(MatOut) * (size_t)count, cudaMemcpyDeviceToHost, cs) !=
                cudaSuccess ||
            cudaStreamSynchronize(cs) != cudaSuccess) { rc = RQB_ERR_CUDA; break; }
        float t_ms = 0.f;
        cudaEventElapsedTime(&t_ms, e0, e1);
        if (ms) *ms = t_ms;
        if (launches) *launches = 2;
        for (int64_t t = 0; t < count; ++t) {
            Q[t] = d[(size_t)t].Q; ldq[t] = d[(size_t)t].ldq;
            B[t] = d[(size_t)t].B; ldb[t] = d[(size_t)t].ldb;
            k[t] = outs[(size_t)t].k; status[t] = outs[(size_t)t].status;
        }
    } while (0);
    if (rc != RQB_OK) cudaGetLastError();
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (dep) cudaEventDestroy(dep);
    cudaStreamDestroy(cs);
    return rc;
}

}  // namespace batched
}  // namespace rqb
