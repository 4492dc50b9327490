// rqb_kernels.cu -- SIMT kernels of the randQB_b hot path and their launchers.
//
// Steps of Fig. randQB_b and the kernels that carry them:
//   line (2)   Omega_i = randn(n, b)             k_omega
//   line (3)   A Omega_i (first block)           k_gemm_nn (+ ||A||_F^2 on the same read)
//   line (3)/(3') orth + re-projection           CholeskyQR2: k_gemm_tn (FP64 Gram),
//                                                k_cholesky (FP64), k_tri_inverse,
//                                                k_gemm_nn (Y R^{-1}, Y - Qbar C)
//   line (4)   B_i = Q_i^T A                     k_gemm_tn + k_reduce_split (+ ||B_i||^2)
//   line (5)   A = A - Q_i B_i, fused with line (3) of block i+1:
//                                                k_downdate_sketch (+ ||A^(i)||_F^2)
//   line (6)   stop test                         k_stop_after_b / k_stop_direct
#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>
#include <cstdio>

#include "rqb_engine.h"
#include "rqb_gemm_simt.cuh"

#ifndef RQB_NN_PIPE_BK_F32
#define RQB_NN_PIPE_BK_F32 8
#endif
#ifndef RQB_NN_PIPE_ST_F32
#define RQB_NN_PIPE_ST_F32 4
#endif

namespace rqb {

// ---------------------------------------------------------------------------
// line (2): Omega entries; out[r * rs + c * cs] for r < n, c < ncols_pad,
// columns c >= ncols are zero (padding of the block to the tile width).
template <typename T>
__global__ void k_omega(int64_t n, int64_t col0, int ncols, int ncols_pad, uint64_t seed,
                        T* __restrict__ out, int64_t rs, int64_t cs) {
    pdl_trigger();
    pdl_wait();
    const int64_t total = n * (int64_t)ncols_pad;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r, c;
        if (rs == 1) { r = e % n; c = e / n; }       // column-major target: walk rows
        else { c = e % ncols_pad; r = e / ncols_pad; }
        const T v = (c < ncols) ? gaussian<T>(seed, r, col0 + c) : T(0);
        out[r * rs + c * cs] = v;
    }
}

template <typename T>
cudaError_t launch_omega(Ctx& cx, int64_t n, int64_t col0, int ncols, int ncols_pad, uint64_t seed,
                         T* out, int64_t rs, int64_t cs) {
    const int64_t total = n * (int64_t)ncols_pad;
    int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)cx.num_sms * 8);
    if (blocks < 1) blocks = 1;
    {
        const cudaError_t le_ = launch_pdl(k_omega<T>, dim3(blocks), dim3(256), 0, cx.stream, n, col0, ncols,
                                           ncols_pad, seed, out, rs, cs);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Deterministic block reduction of one double per thread (fixed tree).
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < NT / 32; ++w) r += sh[w];
    }
    __syncthreads();
    return r;  // valid in thread 0
}

// Sum of squares of an m x n matrix (FP64 accumulation), one partial per CTA.
template <typename T>
__global__ void __launch_bounds__(256) k_sumsq(int64_t m, int64_t n, const T* __restrict__ X, int64_t ldx,
                                               double* __restrict__ part) {
    pdl_trigger();
    pdl_wait();
    // one warp per column at a time (coalesced rows); FP32 or BF16 data: each square
    // is split exactly into p + e (e = fma(v, v, -p)) and summed with
    // compensated FP32 adds, promoted to FP64 every 64 rows per lane
    __shared__ double sh[8];
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5), nw = (int64_t)gridDim.x * 8;
    double acc = 0.0;
    for (int64_t c = gw; c < n; c += nw) {
        const T* col = X + c * ldx;
        if constexpr (sizeof(T) == 8) {
            for (int64_t r = lane; r < m; r += 32) {
                const double v = (double)col[r];
                acc = fma(v, v, acc);
            }
        } else if (sizeof(T) == 2 && (ldx & 7) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0) {
            // BF16 with 16-byte aligned columns: eight values per lane and
            // load; a BF16 square is exact in FP32, summed with TwoSum
            const int64_t m8 = m & ~(int64_t)7;
            for (int64_t r0 = 0; r0 < m; r0 += 32 * 8 * 16) {
                float hi = 0.f, lo = 0.f;
                const int64_t r1 = r0 + 32 * 8 * 16 < m ? r0 + 32 * 8 * 16 : m;
                for (int64_t r = r0 + 8 * lane; r < r1; r += 32 * 8) {
                    float v[8];
                    if (r + 8 <= m8) {
                        const uint4 u = __ldcs(reinterpret_cast<const uint4*>(col + r));
                        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            v[2 * i] = __uint_as_float(w[i] << 16);
                            v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 8; ++i) v[i] = (r + i < m) ? static_cast<float>(col[r + i]) : 0.f;
                    }
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float p2 = __fmul_rn(v[i], v[i]);
                        const float t = __fadd_rn(hi, p2);
                        const float bp = __fsub_rn(t, hi);
                        lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(p2, bp)));
                        hi = t;
                    }
                }
                acc += (double)hi + (double)lo;
            }
        } else {
            for (int64_t r0 = 0; r0 < m; r0 += 32 * 64) {
                float hi = 0.f, lo = 0.f;
                const int64_t r1 = r0 + 32 * 64 < m ? r0 + 32 * 64 : m;
                for (int64_t r = r0 + lane; r < r1; r += 32) {
                    const float v = static_cast<float>(col[r]);
                    const float p2 = __fmul_rn(v, v);     // rounded square, never contracted
                    const float e2 = fmaf(v, v, -p2);     // its exact error
                    const float t = __fadd_rn(hi, p2);    // TwoSum(hi, p2)
                    const float bp = __fsub_rn(t, hi);
                    lo += __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(p2, bp)) + e2;
                    hi = t;
                }
                acc += (double)hi + (double)lo;
            }
        }
    }
    const double s = block_sum<256>(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// Sum `count` doubles in a fixed order into *out (single CTA).
__global__ void __launch_bounds__(256) k_sum_doubles(const double* __restrict__ part, int count,
                                                     double* __restrict__ out) {
    pdl_trigger();
    pdl_wait();
    __shared__ double sh[8];
    double acc = 0.0;
    for (int i = threadIdx.x; i < count; i += 256) acc += part[i];
    const double s = block_sum<256>(acc, sh);
    if (threadIdx.x == 0) *out = s;
}

cudaError_t launch_sum_doubles(Ctx& cx, const double* part, int count, double* out) {
    {
        const cudaError_t le_ = launch_pdl(k_sum_doubles, dim3(1), dim3(256), 0, cx.stream, part, count, out);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sumsq(Ctx& cx, int64_t m, int64_t n, const T* X, int64_t ldx, double* part, int part_cap,
                         double* out) {
    int blocks = std::min<int>(part_cap, cx.num_sms * 4);
    blocks = (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (m * n + 255) / 256));
    {
        const cudaError_t le_ = launch_pdl(k_sumsq<T>, dim3(blocks), dim3(256), 0, cx.stream, m, n, X, ldx, part);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    return launch_sum_doubles(cx, part, blocks, out);
}

// ---------------------------------------------------------------------------
// Split reduction: out(r, c) = sum_z part[z](r, c) (FP64 sum in z order), for
// r < rows, c < cols; optional sum of squares of the stored outputs, one
// partial per CTA.
template <typename TP, typename TO>
__global__ void __launch_bounds__(256)
k_reduce_split(int64_t rows, int64_t cols, int splits, const TP* __restrict__ part, int64_t ldp,
               int64_t zstride, TO* out, int64_t ldo, double* __restrict__ sq_part, double alpha, double beta,
               const TO* Yin, int64_t ldyin, int sym) {
    pdl_trigger();
    pdl_wait();
    __shared__ double sh[8];
    double sq = 0.0;
    const int64_t total = rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < total; e += (int64_t)gridDim.x * 256) {
        const int64_t r = e % rows, c = e / rows;
        // sym: the upper triangle is the mirror of the lower one
        const int64_t pe = (sym && r < c) ? c + r * ldp : r + c * ldp;
        // partials summed in their own precision, in split order (FP32
        // partials: 2^-24 per term, far below the product's own rounding;
        // FP64 partials: the FP64-accumulated Grams and coefficients)
        TP acc = TP(0);
#pragma unroll 4
        for (int z = 0; z < splits; ++z) acc += part[z * zstride + pe];
        double s = (double)acc;
        if (alpha != 1.0) s *= alpha;
        if (beta != 0.0) s += beta * (double)Yin[r + c * ldyin];
        const TO v = (TO)s;
        out[r + c * ldo] = v;
        sq += (double)v * (double)v;
    }
    if (sq_part) {
        const double t = block_sum<256>(sq, sh);
        if (threadIdx.x == 0) sq_part[blockIdx.x] = t;
    }
}

// The FP32 case with alpha = 1, beta = 0 and aligned columns of a multiple
// of four rows: four consecutive rows per thread (16-byte loads and stores,
// 32-bit index arithmetic), the same FP32 sums in split order, and no FP64
// work unless ||out||^2 is asked for.
__global__ void __launch_bounds__(256)
k_reduce_split4(int rows, int cols, int splits, const float* __restrict__ part, int64_t ldp, int64_t zstride,
                float* __restrict__ out, int64_t ldo, double* __restrict__ sq_part) {
    pdl_trigger();
    pdl_wait();
    __shared__ double sh[8];
    double sq = 0.0;
    const int rq = rows / 4;
    const int total = rq * cols;
    for (int e = blockIdx.x * 256 + threadIdx.x; e < total; e += gridDim.x * 256) {
        const int r = (e % rq) * 4, c = e / rq;
        const float* p = part + r + (int64_t)c * ldp;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
        for (int z = 0; z < splits; ++z) {
            const float4 v = *reinterpret_cast<const float4*>(p + z * zstride);
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
        *reinterpret_cast<float4*>(out + r + (int64_t)c * ldo) = acc;
        if (sq_part) {
            sq = fma((double)acc.x, (double)acc.x, sq);
            sq = fma((double)acc.y, (double)acc.y, sq);
            sq = fma((double)acc.z, (double)acc.z, sq);
            sq = fma((double)acc.w, (double)acc.w, sq);
        }
    }
    if (sq_part) {
        const double t = block_sum<256>(sq, sh);
        if (threadIdx.x == 0) sq_part[blockIdx.x] = t;
    }
}

template <typename TP, typename TO>
cudaError_t launch_reduce_split(Ctx& cx, int64_t rows, int64_t cols, int splits, const TP* part, int64_t ldp,
                                int64_t zstride, TO* out, int64_t ldo, double* sq_part, int sq_cap,
                                double* sq_out, double alpha, double beta, const TO* Yin, int64_t ldyin, int sym) {
    bool vec4 = false;
    if constexpr (std::is_same<TP, float>::value && std::is_same<TO, float>::value)
        vec4 = alpha == 1.0 && beta == 0.0 && !sym && rows % 4 == 0 && ldp % 4 == 0 && zstride % 4 == 0 &&
               ldo % 4 == 0 && (uintptr_t)part % 16 == 0 && (uintptr_t)out % 16 == 0 && rows * cols < (1LL << 31);
    const int64_t work = vec4 ? rows / 4 * cols : rows * cols;
    int blocks = std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, (int64_t)cx.num_sms * 8));
    if (sq_part) blocks = std::min(blocks, sq_cap);
    if constexpr (std::is_same<TP, float>::value && std::is_same<TO, float>::value) {
        if (vec4) {
            const cudaError_t le_ = launch_pdl(k_reduce_split4, dim3(blocks), dim3(256), 0, cx.stream, (int)rows,
                                               (int)cols, splits, part, ldp, zstride, out, ldo, sq_part);
            if (le_ != cudaSuccess) return le_;
        }
    }
    if (!vec4) {
        const cudaError_t le_ = launch_pdl(k_reduce_split<TP, TO>, dim3(blocks), dim3(256), 0, cx.stream, rows, cols,
                                           splits, part, ldp, zstride, out, ldo, sq_part, alpha, beta, Yin, ldyin,
                                           sym);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !sq_part) return e;
    return launch_sum_doubles(cx, sq_part, blocks, sq_out);
}

// ---------------------------------------------------------------------------
// CholeskyQR factor of the panel Gram matrix: G (bp x bp, FP64, symmetric;
// only rows/cols < p are meaningful) = R^T R with R upper triangular and
// diag(R) > 0; rows/cols >= p are set to the identity.  One CTA of 256
// threads, working precision W (FP64 for the first CholeskyQR pass, whose Gram
// may be ill-conditioned; FP32 for the second, whose Gram is I + O(u kappa)).
// The upper triangle is kept row-major and packed (row r holds columns
// r .. bp-1), in shared memory when it fits, else in a global scratch.
// Thread (ty, tx) of a 16 x 16 grid owns the entries (r, c) with r = ty,
// c = tx (mod 16); step j subtracts S[j][r] S[j][c] / d_j from each owned
// S[r][c] (j < r <= c) using the unscaled pivot row, so a step needs one
// barrier; rows are scaled by d_j^{-1/2} at the end.  A pivot <= tol * G_jj
// records RQB_ERR_BREAKDOWN.
__device__ __forceinline__ int64_t packed_row(int r, int bp) { return (int64_t)r * bp - (int64_t)r * (r + 1) / 2; }

template <typename W>
__global__ void __launch_bounds__(256)
k_cholesky(const double* __restrict__ G, int bp, int p, double* __restrict__ R, int in_smem, void* scratch,
           double tol, DevState* st, const int* __restrict__ skip) {
    pdl_trigger();
    pdl_wait();
    if (skip && *skip) return;   // the near-identity expansion gave the factor
    extern __shared__ __align__(16) unsigned char chol_smem[];
    __shared__ double refd[256];
    __shared__ double rdiag[256];
    W* S = in_smem ? reinterpret_cast<W*>(chol_smem) : reinterpret_cast<W*>(scratch);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    for (int r = tid; r < p; r += 256) refd[r] = G[r + (int64_t)r * bp];
    for (int r = ty; r < p; r += 16) {
        W* Sr = S + packed_row(r, bp);
        for (int c = r + ((tx - r) % 16 + 16) % 16; c < p; c += 16) Sr[c] = (W)G[r + (int64_t)c * bp];
    }
    __syncthreads();
    bool bad = false;
    for (int j = 0; j < p; ++j) {
        const W* Sj = S + packed_row(j, bp);
        const W d = Sj[j];
        if (!((double)d > tol * refd[j]) || !isfinite((double)d)) { bad = true; break; }   // uniform
        const W invd = W(1) / d;
        for (int r = j + 1 + ((ty - (j + 1)) % 16 + 16) % 16; r < p; r += 16) {
            const W f = Sj[r] * invd;
            W* Sr = S + packed_row(r, bp);
            for (int c = r + ((tx - r) % 16 + 16) % 16; c < p; c += 16) Sr[c] -= f * Sj[c];
        }
        __syncthreads();
    }
    if (bad) {
        if (tid == 0) record_error(st, RQB_ERR_BREAKDOWN);
        return;
    }
    // R (column-major, FP64): R[r][c] = S[r][c] / sqrt(d_r), identity beyond p.
    for (int r = tid; r < p; r += 256) rdiag[r] = sqrt((double)S[packed_row(r, bp) + r]);
    __syncthreads();
    for (int e = tid; e < bp * bp; e += 256) {
        const int r = e % bp, c = e / bp;
        double v = 0.0;
        if (r < p && c < p) {
            if (r < c) v = (double)S[packed_row(r, bp) + c] / rdiag[r];
            else if (r == c) v = rdiag[r];
        } else if (r == c) {
            v = 1.0;
        }
        R[e] = v;
    }
}

// Rinv (bp x bp, type T, column-major) = R^{-1} for upper-triangular R (FP64).
// One warp per column c solves R x = e_c by column-oriented back substitution
// (x_t = x_t / R_tt, then x_r -= R_rt x_t for r < t), warp-synchronous, with
// the CTA's leading block of R and the reciprocal diagonal in shared memory.
template <typename T>
__global__ void __launch_bounds__(128)
k_tri_inverse(const double* __restrict__ R, int bp, T* __restrict__ Rinv, int staged_cols,
              const int* __restrict__ skip) {
    pdl_trigger();
    pdl_wait();
    if (skip && *skip) return;   // the near-identity expansion gave the factor
    extern __shared__ __align__(16) double dsm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cmax = min(bp - 1, (int)blockIdx.x * 4 + 3);
    const int c = blockIdx.x * 4 + warp;
    double* invd = dsm;                  // bp
    double* xs = dsm + bp;               // 4 x bp
    double* Rs = dsm + 5 * bp;           // columns 0..cmax of R (ld bp), when staged
    const bool staged = (cmax < staged_cols);
    for (int t = threadIdx.x; t <= cmax; t += 128) invd[t] = 1.0 / R[t + (int64_t)t * bp];
    if (staged)
        for (int e = threadIdx.x; e < (cmax + 1) * bp; e += 128) Rs[e] = R[e];
    __syncthreads();
    if (c >= bp) return;
    const double* Rc = staged ? Rs : R;
    double* x = xs + warp * bp;
    for (int r = lane; r <= c; r += 32) x[r] = (r == c) ? 1.0 : 0.0;
    __syncwarp();
    for (int t = c; t >= 0; --t) {
        const double xt = x[t] * invd[t];
        for (int r = lane; r < t; r += 32) x[r] -= Rc[r + (int64_t)t * bp] * xt;
        __syncwarp();
        if (lane == 0) x[t] = xt;
        __syncwarp();
    }
    for (int r = lane; r < bp; r += 32) Rinv[r + (int64_t)c * bp] = (T)((r <= c) ? x[r] : 0.0);
}

// ---------------------------------------------------------------------------
// Stopping test (line (6)).  After B_i:  E -= ||B_i||^2 and
//   E <= eps2 - tau  -> stop;  E > eps2 + tau -> continue;  else ambiguous
// (decided on the direct norm after the downdate).  tau is the rounding band
// of E in the working precision.
__global__ void k_set_norm(DevState* st, const double* nrm) {
    pdl_trigger();
    pdl_wait();
    const double v = *nrm;
    st->normA2 = v;
    st->E = v;
    st->flag = kContinue;
    if (!isfinite(v)) record_error(st, RQB_ERR_NONFINITE);
}

__global__ void k_stop_after_b(DevState* st, const double* nb2, double eps2, double tau_rel, int fixed) {
    pdl_trigger();
    pdl_wait();
    const double tau = tau_rel * st->normA2;
    const double b2 = *nb2;
    st->normB2 = b2;
    st->E -= b2;
    st->D = -1.0;
    if (!isfinite(b2)) record_error(st, RQB_ERR_NONFINITE);
    const double E = st->E;
    if (fixed) st->flag = kContinue;
    else if (E <= eps2 - tau) st->flag = kStop;
    else if (E > eps2 + tau) st->flag = kContinue;
    else st->flag = kAmbiguous;
}

// always = 0: decide only when the downdate test was ambiguous; always = 1:
// decide on the direct norm whenever the downdate test did not stop.
__global__ void k_stop_direct(DevState* st, const double* d2, double eps2, int always) {
    pdl_trigger();
    pdl_wait();
    const double d = *d2;
    st->D = d;
    if (st->flag == kAmbiguous || (always && st->flag != kStop)) st->flag = (d <= eps2) ? kStop : kContinue;
}

cudaError_t launch_set_norm(Ctx& cx, const double* nrm) {
    {
        const cudaError_t le_ = launch_pdl(k_set_norm, dim3(1), dim3(1), 0, cx.stream, cx.st, nrm);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    return cudaGetLastError();
}
cudaError_t launch_stop_after_b(Ctx& cx, const double* nb2, double eps2, double tau_rel, int fixed) {
    {
        const cudaError_t le_ = launch_pdl(k_stop_after_b, dim3(1), dim3(1), 0, cx.stream, cx.st, nb2, eps2, tau_rel,
                                           fixed);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    return cudaGetLastError();
}
cudaError_t launch_stop_direct(Ctx& cx, const double* d2, double eps2, bool always) {
    {
        const cudaError_t le_ = launch_pdl(k_stop_direct, dim3(1), dim3(1), 0, cx.stream, cx.st, d2, eps2,
                                           always ? 1 : 0);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// line (5) fused with line (3) of the next block.  CTA (x, z) owns rows
// [x BM, x BM + BM) and the column range of split z.  Per column chunk of BC
// columns:  Wn = Wsrc - Q_i B_i (GEMM 1, K = bp), stored to Wdst and, transposed,
// to shared memory; then Yacc += Wn Omega_next(chunk, :) (GEMM 2, K = BC).
// Also ||Wn||_F^2 (FP64 partial per CTA).
template <typename T, int BM, int BN>
struct DDCfg {
    static constexpr int TM = SimtTile<T>::TM, TN = SimtTile<T>::TN;
    static constexpr int NT = (BM / TM) * (BN / TN);
    static constexpr int BC = 2 * NT * TM / BM;          // chunk columns: GEMM 1 thread tile TM x 2
    static constexpr int TN1 = BM * BC / (NT * TM);      // == 2
    static constexpr size_t SMEM = sizeof(T) * ((size_t)BN * BM + (size_t)BN * BC + (size_t)BC * BM +
                                                (size_t)BC * BN);
    static_assert(TN1 == 2, "GEMM 1 tile");
};

template <typename T, int BM, int BN>
__global__ void __launch_bounds__(DDCfg<T, BM, BN>::NT)
k_downdate_sketch(int64_t m, int64_t n, int p, int64_t csplit,
                  const T* Wsrc, int64_t ldws, const T* __restrict__ Qi, int64_t ldq,
                  const T* __restrict__ Bi, int64_t ldb, const T* __restrict__ Om /* n x BN row-major */,
                  T* Wdst, int64_t ldwd, T* __restrict__ Ypart, int64_t ldyp, int64_t yzstride,
                  double* __restrict__ nrm_part) {
    using C = DDCfg<T, BM, BN>;
    constexpr int TM = C::TM, TN = C::TN, NT = C::NT, BC = C::BC, V = Vec16<T>::N;
    constexpr int HM = TM / 2, HN = TN / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Qs = reinterpret_cast<T*>(smem_raw);   // [BN][BM]  Qs[t*BM + r] = Q(r0 + r, t)
    T* Bs = Qs + BN * BM;                      // [BN][BC]  Bs[t*BC + c] = B(t, c0 + c)
    T* Ws = Bs + BN * BC;                      // [BC][BM]  Ws[c*BM + r] = Wn(r0 + r, c0 + c)
    T* Os = Ws + BC * BM;                      // [BC][BN]  Os[c*BN + j] = Omega(c0 + c, j)
    __shared__ double red[NT / 32];

    const int tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * BM;
    const int64_t cbeg = (int64_t)blockIdx.z * csplit;
    const int64_t cend = (cbeg + csplit < n) ? cbeg + csplit : n;

    // stage Q_i rows of this tile (once)
    for (int v = tid; v < BN * (BM / V); v += NT) {
        const int t = v / (BM / V), rr = (v % (BM / V)) * V;
        const int64_t r = r0 + rr;
        T tmp[V];
        if (t < p && r < m) ldg_run<T>(tmp, Qi + r + (int64_t)t * ldq, m - r);
        else {
#pragma unroll
            for (int i = 0; i < V; ++i) tmp[i] = T(0);
        }
#pragma unroll
        for (int i = 0; i < V; ++i) Qs[t * BM + rr + i] = tmp[i];
    }

    // GEMM 2 (Y) thread tile
    const int tx = tid % (BN / TN), ty = tid / (BN / TN);
    // GEMM 1 (downdate) thread tile: TM rows x 2 columns (c = tx1, BC/2 + tx1)
    const int tx1 = tid % (BC / 2), ty1 = tid / (BC / 2);

    T yacc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) yacc[i][j] = T(0);
    float2 yacq[TM][TN / 2];   // FP32: yacc as column pairs, for the packed FMAs
    if constexpr (sizeof(T) == 4) zero_tile_f32x2<TM, TN>(yacq);
    double nrm = 0.0;

    for (int64_t c0 = cbeg; c0 < cend; c0 += BC) {
        __syncthreads();   // previous chunk's readers of Bs/Ws/Os are done (and Qs staged)
        // B_i chunk: column c of B is p contiguous entries
        for (int v = tid; v < BC * (BN / V); v += NT) {
            const int cc = v / (BN / V), tt = (v % (BN / V)) * V;
            const int64_t c = c0 + cc;
            T tmp[V];
            if (c < cend && tt < p) ldg_run<T>(tmp, Bi + tt + c * ldb, p - tt);
            else {
#pragma unroll
                for (int i = 0; i < V; ++i) tmp[i] = T(0);
            }
#pragma unroll
            for (int i = 0; i < V; ++i) Bs[(tt + i) * BC + cc] = tmp[i];
        }
        // Omega chunk rows (row-major, BN per row)
        for (int v = tid; v < BC * (BN / V); v += NT) {
            const int cc = v / (BN / V), jj = (v % (BN / V)) * V;
            const int64_t c = c0 + cc;
            T tmp[V];
            if (c < cend) ldg_run<T>(tmp, Om + c * BN + jj, BN - jj);
            else {
#pragma unroll
                for (int i = 0; i < V; ++i) tmp[i] = T(0);
            }
#pragma unroll
            for (int i = 0; i < V; ++i) Os[cc * BN + jj + i] = tmp[i];
        }
        __syncthreads();

        // GEMM 1: P = Q_tile * B_chunk
        T pacc[TM][2];
#pragma unroll
        for (int i = 0; i < TM; ++i) { pacc[i][0] = T(0); pacc[i][1] = T(0); }
        for (int t = 0; t < BN; ++t) {
            T a0[HM], a1[HM];
            lds_vec<T, HM>(a0, &Qs[t * BM + ty1 * HM]);
            lds_vec<T, HM>(a1, &Qs[t * BM + BM / 2 + ty1 * HM]);
            const T b0 = Bs[t * BC + tx1], b1 = Bs[t * BC + BC / 2 + tx1];
#pragma unroll
            for (int i = 0; i < HM; ++i) {
                pacc[i][0] = fma(a0[i], b0, pacc[i][0]);
                pacc[i][1] = fma(a0[i], b1, pacc[i][1]);
                pacc[HM + i][0] = fma(a1[i], b0, pacc[HM + i][0]);
                pacc[HM + i][1] = fma(a1[i], b1, pacc[HM + i][1]);
            }
        }
        // Wn = Wsrc - P; store to Wdst and Ws; accumulate ||Wn||^2
        T part_sq = T(0);
#pragma unroll
        for (int jc = 0; jc < 2; ++jc) {
            const int cc = (jc == 0) ? tx1 : (BC / 2 + tx1);
            const int64_t c = c0 + cc;
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                const int rr = (g == 0) ? ty1 * HM : (BM / 2 + ty1 * HM);
                const int64_t r = r0 + rr;
                T w[HM];
                if (c < cend && r < m) {
                    const T* src = Wsrc + r + c * ldws;
                    if (r + HM <= m && aligned16(src) && HM * sizeof(T) == 16) {
                        lds_vec<T, HM>(w, src);   // aligned 16-byte global load
                    } else {
#pragma unroll
                        for (int i = 0; i < HM; ++i) w[i] = (r + i < m) ? src[i] : T(0);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < HM; ++i) w[i] = T(0);
                }
#pragma unroll
                for (int i = 0; i < HM; ++i) {
                    w[i] -= pacc[g * HM + i][jc];
                    if (!(c < cend && r + i < m)) w[i] = T(0);
                    part_sq = fma(w[i], w[i], part_sq);
                    Ws[cc * BM + rr + i] = w[i];
                }
                if (c < cend && r < m) {
                    T* dst = Wdst + r + c * ldwd;
                    if (r + HM <= m && aligned16(dst) && HM * sizeof(T) == 16) {
                        using VT = typename VecH<T, HM>::type;
                        *reinterpret_cast<VT*>(dst) = *reinterpret_cast<const VT*>(w);
                    } else {
#pragma unroll
                        for (int i = 0; i < HM; ++i)
                            if (r + i < m) dst[i] = w[i];
                    }
                }
            }
        }
        nrm += (double)part_sq;
        __syncthreads();

        // GEMM 2: Yacc += Wn(chunk) * Omega(chunk, :)
#pragma unroll 4
        for (int kk = 0; kk < BC; ++kk) {
            T a[TM], b[TN], a0[HM], a1[HM], b0[HN], b1[HN];
            lds_vec<T, HM>(a0, &Ws[kk * BM + ty * HM]);
            lds_vec<T, HM>(a1, &Ws[kk * BM + BM / 2 + ty * HM]);
            lds_vec<T, HN>(b0, &Os[kk * BN + tx * HN]);
            lds_vec<T, HN>(b1, &Os[kk * BN + BN / 2 + tx * HN]);
#pragma unroll
            for (int i = 0; i < HM; ++i) { a[i] = a0[i]; a[HM + i] = a1[i]; }
#pragma unroll
            for (int j = 0; j < HN; ++j) { b[j] = b0[j]; b[HN + j] = b1[j]; }
            if constexpr (sizeof(T) == 4) {
                fma_tile_f32x2<TM, TN>(yacq, a, b);
            } else {
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) yacc[i][j] = fma(a[i], b[j], yacc[i][j]);
            }
        }
    }
    if constexpr (sizeof(T) == 4) unpack_tile_f32x2<TM, TN>(yacq, yacc);

    // Y partial of this split
    T* yout = Ypart + (int64_t)blockIdx.z * yzstride;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t r = r0 + ((i < HM) ? (ty * HM + i) : (BM / 2 + ty * HM + (i - HM)));
        if (r >= m) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int c = (j < HN) ? (tx * HN + j) : (BN / 2 + tx * HN + (j - HN));
            yout[r + (int64_t)c * ldyp] = yacc[i][j];
        }
    }
    // ||Wn||^2 partial
    double v = nrm;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < NT / 32; ++w) s += red[w];
        nrm_part[blockIdx.x + (int64_t)gridDim.x * blockIdx.z] = s;
    }
}

// ---------------------------------------------------------------------------
// Launch configuration helpers
static int choose_splits(int64_t tiles, int64_t kdim, int64_t kmin, int max_splits, int slots) {
    // Largest wave efficiency ctas / (waves * slots); a larger split count is
    // taken only when it improves the efficiency by more than 1 % (relative),
    // so grids smaller than one wave grow until the reduction length per split
    // reaches kmin, and full grids keep the fewest splits.
    int best = 1;
    double best_eff = -1.0;
    for (int s = 1; s <= max_splits; ++s) {
        if (s > 1 && kdim / s < kmin) break;
        const int64_t ctas = tiles * s;
        const int64_t waves = (ctas + slots - 1) / slots;
        const double eff = (double)ctas / (double)(waves * slots);
        if (eff > best_eff * 1.01) { best_eff = eff; best = s; }
    }
    return best;
}

template <typename K>
static int occupancy(K kernel, int threads, size_t dyn_smem) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, dyn_smem) != cudaSuccess || nb < 1)
        nb = 1;
    return nb;
}

// Tile table ---------------------------------------------------------------
// NN: float BM = 128 (64 for BN = 256), BN = bp; double BM = 64, BN = min(bp, 128).
template <typename T> struct NNTile;
template <> struct NNTile<float> { static constexpr int BK = 8; };
template <> struct NNTile<double> { static constexpr int BK = 8; };

// Pipelined NN (row-major C, cp.async-fed): reduction chunk and stage count.
template <typename T> struct NNPipeCfg;
template <> struct NNPipeCfg<float> { static constexpr int BK = RQB_NN_PIPE_BK_F32, ST = RQB_NN_PIPE_ST_F32; };
template <> struct NNPipeCfg<double> { static constexpr int BK = 8, ST = 4; };

template <typename T, int BM, int BN, bool ROWC>
static cudaError_t nn_launch(Ctx& cx, const NNArgs<T>& a) {
    using G = GemmNN<T, BM, BN, NNTile<T>::BK, ROWC>;
    using P = GemmNNPipe<T, BM, BN, NNPipeCfg<T>::BK, NNPipeCfg<T>::ST>;
    using KernT = void (*)(int64_t, int64_t, int64_t, int, int, const T*, int64_t, const T*, int64_t, int64_t, T*,
                           int64_t, int64_t, const T*, int64_t, T, T, double*);
    using KernP = void (*)(int64_t, int64_t, int64_t, int, int, const T*, int64_t, const T*, int64_t, T*, int64_t,
                           int64_t, const T*, int64_t, T, T, double*);
    KernT kern = k_gemm_nn<T, BM, BN, NNTile<T>::BK, ROWC>;
    KernP kernp = k_gemm_nn_pipe<T, BM, BN, NNPipeCfg<T>::BK, NNPipeCfg<T>::ST>;
    constexpr int V = Vec16<T>::N;
    // the pipelined kernel needs 16-byte aligned vectors of X and of C's rows
    const bool pipe = ROWC && ((uintptr_t)a.X % 16 == 0) && ((uintptr_t)a.C % 16 == 0) && (a.ldx % V == 0) &&
                      (a.csk % V == 0);
    int threads = pipe ? P::NT : G::NT;
    size_t dsmem = pipe ? P::SMEM : 0;
    if (pipe) {
        // the FP64 64 x 128 tile's 48 KB of dynamic shared memory plus the
        // kernel's static reduction buffer exceed the default limit
        cudaError_t e = smem_limit(kernp, (int)P::SMEM);
        if (e != cudaSuccess) return e;
    }
    const int64_t kalign = pipe ? NNPipeCfg<T>::BK : NNTile<T>::BK;
    const int64_t mt = (a.m + BM - 1) / BM;
    const int nt = (std::max(a.nc, a.nout) + BN - 1) / BN;
    const int slots = cx.num_sms * (pipe ? occupancy(kernp, threads, dsmem) : occupancy(kern, threads, dsmem));
    // FP64 pipes are 64x slower than FP32 ones on this part: spread FP64
    // products over more CTAs by splitting shorter reductions
    constexpr int64_t kmin = (sizeof(T) == 8) ? 64 : 256;
    bool allow_split = a.allow_split && a.part;
    int splits = 1;
    if (allow_split) {
        const int64_t per = a.m * (int64_t)nt * BN;
        int64_t maxs = std::min<int64_t>(32, (int64_t)(a.part_cap / (size_t)std::max<int64_t>(per, 1)));
        if (a.nrm_part) maxs = std::min<int64_t>(maxs, a.nrm_cap / std::max<int64_t>(mt, 1));
        splits = choose_splits(mt * nt, a.K, kmin, (int)std::max<int64_t>(1, maxs), slots);
    }
    int64_t ks = (a.K + splits - 1) / splits;
    ks = ((ks + kalign - 1) / kalign) * kalign;
    if (ks < kalign) ks = kalign;
    splits = (int)std::max<int64_t>(1, (a.K + ks - 1) / ks);
    if (a.nrm_part && mt * splits > a.nrm_cap) return cudaErrorInvalidValue;
    dim3 grid((unsigned)mt, (unsigned)nt, (unsigned)splits);
    // one split: the product goes straight to Out; else a partial per split (m x nt*BN, ld = m)
    const bool one = (splits == 1);
    T* out = one ? a.Out : a.part;
    const int nout = one ? a.nout : nt * BN;
    const int64_t ldo = one ? a.ldo : a.m, zs = one ? 0 : a.m * (int64_t)nt * BN;
    const T* yin = one ? a.Yin : nullptr;
    const int64_t ldyin = one ? a.ldyin : 0;
    const T alpha = one ? a.alpha : T(1), beta = one ? a.beta : T(0);
    if (pipe)
        kernp<<<grid, threads, dsmem, cx.stream>>>(a.m, a.K, ks, a.nc, nout, a.X, a.ldx, a.C, a.csk, out, ldo, zs, yin,
                                                   ldyin, alpha, beta, a.nrm_part);
    else
        kern<<<grid, threads, dsmem, cx.stream>>>(a.m, a.K, ks, a.nc, nout, a.X, a.ldx, a.C, a.csk, a.csj, out, ldo,
                                                  zs, yin, ldyin, alpha, beta, a.nrm_part);
    cx.launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (a.nrm_part) {
        e = launch_sum_doubles(cx, a.nrm_part, (int)(mt * splits), a.nrm_out);
        if (e != cudaSuccess) return e;
    }
    if (splits == 1) return cudaSuccess;
    return launch_reduce_split<T, T>(cx, a.m, a.nout, splits, a.part, a.m, a.m * (int64_t)nt * BN, a.Out, a.ldo,
                                     nullptr, 0, nullptr, (double)a.alpha, (double)a.beta, a.Yin, a.ldyin);
}

template <typename T>
cudaError_t gemm_nn(Ctx& cx, const NNArgs<T>& a) {
    const bool rowc = a.c_rowmajor;
    const int bp = std::max(a.nc, a.nout);
#define RQB_NN(BM_, BN_) return rowc ? nn_launch<T, BM_, BN_, true>(cx, a) : nn_launch<T, BM_, BN_, false>(cx, a)
    if constexpr (sizeof(T) == 4) {
        if (bp <= 32) { RQB_NN(128, 32); }
        if (bp <= 64) { RQB_NN(128, 64); }
        if (bp <= 128) { RQB_NN(128, 128); }
        RQB_NN(64, 256);
    } else {
        if (bp <= 32) { RQB_NN(64, 32); }
        if (bp <= 64) { RQB_NN(64, 64); }
        RQB_NN(64, 128);
    }
#undef RQB_NN
}

// TN ----------------------------------------------------------------------
template <typename T, typename Acc, int BP, int BQ, int BK, int TP, int TQ, int PROMOTE, bool COMP = false>
static cudaError_t tn_launch(Ctx& cx, int64_t m, int pn, int64_t qn, const T* X, int64_t ldx, const T* Y,
                             int64_t ldy, Acc* part, size_t part_cap_elems, int max_splits, int* splits_out,
                             int64_t kmin = 512, int sym = 0) {
    auto kern = k_gemm_tn<T, Acc, BP, BQ, BK, TP, TQ, PROMOTE, COMP>;
    constexpr int NT = (BP / TP) * (BQ / TQ);
    const int pt = (pn + BP - 1) / BP;
    const int64_t qt = (qn + BQ - 1) / BQ;
    const int slots = cx.num_sms * occupancy(kern, NT, 0);
    const int64_t per = (int64_t)pn * qn;
    if ((size_t)per > part_cap_elems) return cudaErrorInvalidValue;
    int maxs = (int)std::min<int64_t>(max_splits, (int64_t)(part_cap_elems / (size_t)std::max<int64_t>(per, 1)));
    maxs = std::max(1, maxs);
    // tiles that do work (the lower triangle of tiles for a Gram)
    const int64_t work_tiles = sym ? (int64_t)pt * (pt + 1) / 2 : (int64_t)pt * qt;
    int splits = choose_splits(work_tiles, m, kmin, maxs, slots);
    int64_t rs = (m + splits - 1) / splits;
    rs = ((rs + BK - 1) / BK) * BK;
    splits = (int)std::max<int64_t>(1, (m + rs - 1) / rs);
    dim3 grid((unsigned)pt, (unsigned)qt, (unsigned)splits);
    kern<<<grid, NT, 0, cx.stream>>>(m, pn, qn, rs, X, ldx, Y, ldy, part, pn, per, sym);
    cx.launches++;
    *splits_out = splits;
    return cudaGetLastError();
}

// Out (pn x qn, type TO, ld ldo) = X^T Y; optional ||Out||^2 into *sq_out.
template <typename T>
cudaError_t gemm_tn(Ctx& cx, int64_t m, int pn, int64_t qn, const T* X, int64_t ldx, const T* Y, int64_t ldy,
                    T* Out, int64_t ldo, T* part, size_t part_cap_elems, double* sq_part, int sq_cap,
                    double* sq_out) {
    int splits = 1;
    cudaError_t e;
    constexpr int64_t kmin = (sizeof(T) == 8) ? 64 : 512;
    if constexpr (sizeof(T) == 4) {
        if (pn <= 32) e = tn_launch<T, T, 32, 128, 16, 8, 8, 0>(cx, m, pn, qn, X, ldx, Y, ldy, part, part_cap_elems, 64, &splits, kmin);
        else if (pn <= 64) e = tn_launch<T, T, 64, 128, 16, 8, 8, 0>(cx, m, pn, qn, X, ldx, Y, ldy, part, part_cap_elems, 64, &splits, kmin);
        else e = tn_launch<T, T, 128, 128, 16, 8, 8, 0>(cx, m, pn, qn, X, ldx, Y, ldy, part, part_cap_elems, 64, &splits, kmin);
    } else {
        if (pn <= 32) e = tn_launch<T, T, 32, 64, 8, 4, 4, 0>(cx, m, pn, qn, X, ldx, Y, ldy, part, part_cap_elems, 64, &splits, kmin);
        else e = tn_launch<T, T, 64, 64, 8, 4, 4, 0>(cx, m, pn, qn, X, ldx, Y, ldy, part, part_cap_elems, 64, &splits, kmin);
    }
    if (e != cudaSuccess) return e;
    return launch_reduce_split<T, T>(cx, pn, qn, splits, part, pn, (int64_t)pn * qn, Out, ldo, sq_part, sq_cap,
                                     sq_out, 1.0, 0.0, nullptr, 0);
}

// Out (pn x qn, FP64, ld ldo) = X^T Y with FP64 accumulation across chunks.
// sym: X and Y are the same matrix (a Gram matrix): only the lower triangle
// of tiles is computed and the upper one mirrored.
template <typename T>
cudaError_t gemm_tn_f64acc(Ctx& cx, int64_t m, int pn, int64_t qn, const T* X, int64_t ldx, const T* Y,
                           int64_t ldy, double* Out, int64_t ldo, double* part, size_t part_cap_elems, bool exact,
                           bool sym) {
    int splits = 1;
    cudaError_t e;
    const int sy = (sym && X == Y && ldx == ldy && pn == qn) ? 1 : 0;
    if constexpr (sizeof(T) == 4) {
        if (exact)
            e = tn_launch<T, double, 64, 64, 16, 4, 4, 16, true>(cx, m, pn, qn, X, ldx, Y, ldy, part,
                                                                 part_cap_elems, 128, &splits, 128, sy);
        else
            e = tn_launch<T, double, 64, 64, 16, 4, 4, 8>(cx, m, pn, qn, X, ldx, Y, ldy, part, part_cap_elems, 128,
                                                          &splits, 256, sy);
    } else {
        e = tn_launch<T, double, 64, 64, 8, 4, 4, 0>(cx, m, pn, qn, X, ldx, Y, ldy, part, part_cap_elems, 128, &splits,
                                                     32, sy);
    }
    if (e != cudaSuccess) return e;
    return launch_reduce_split<double, double>(cx, pn, qn, splits, part, pn, (int64_t)pn * qn, Out, ldo, nullptr,
                                               0, nullptr, 1.0, 0.0, nullptr, 0, sy);
}

// Cholesky + inverse -------------------------------------------------------
// fp64_factor: FP64 Cholesky (first CholeskyQR pass); else FP32 (second pass).
template <typename T>
cudaError_t chol_inv(Ctx& cx, double* G, int bp, int p, double* R, T* Rinv, bool fp64_factor, double* scratch,
                     size_t scratch_doubles, bool second_pass) {
    for (const void* k : {reinterpret_cast<const void*>(k_cholesky<double>),
                          reinterpret_cast<const void*>(k_cholesky<float>),
                          reinterpret_cast<const void*>(k_tri_inverse<T>)}) {
        cudaError_t ea = smem_limit_once(k, 200 * 1024);
        if (ea != cudaSuccess) return ea;
    }
    // relative pivot below which a panel column counts as dependent: rounding
    // of the panel itself leaves pivots of order u^2 (1e-32 for FP64 data,
    // 4e-15 for FP32 data); CholeskyQR2 with an FP64 Gram handles anything above
    const double tol = (sizeof(T) == 8) ? 1e-15 : 1e-14;
    const size_t sq = (size_t)bp * bp;
    const size_t packed = (size_t)bp * (bp + 1) / 2;
    if (scratch_doubles < sq) return cudaErrorInvalidValue;
    // second pass: the near-identity expansion first; its work sits past the
    // 3 bp^2 + bp doubles the elimination uses of scratch.  First order drops
    // O(||G - I||^2): tau^2 = 2^-56 for an FP64 factor, 1e-8 for an FP32 one,
    // both below the unit roundoff; FP32 factors up to ||G - I||_F = 2e-2
    // take the iterated expansion
    int* skip = nullptr;
    if (second_pass) {
        const size_t at = 3 * sq + (size_t)bp;
        if (scratch_doubles < at + kNearIdWork(bp)) return cudaErrorInvalidValue;
        skip = reinterpret_cast<int*>(scratch + at + kNearIdParts);
        const double tau = fp64_factor ? 0x1p-28 : 1e-4;
        cudaError_t en = near_identity<T>(cx, G, bp, p, R, Rinv, tau, scratch + at, skip);
        if (en != cudaSuccess) return en;
    }
    // a Gram of 128 or more columns: blocked over many CTAs (one CTA's shared
    // memory does not hold a wide FP64 one, and one SM's FP64 rate bounds it)
    if (bp >= 128)
        return chol_inv_blocked<T>(cx, G, bp, p, R, Rinv, tol, scratch, scratch_doubles, fp64_factor, skip);
    if (fp64_factor) {
        const int in_smem = (sizeof(double) * packed <= 200 * 1024) ? 1 : 0;
        {
            const cudaError_t le_ = launch_pdl(k_cholesky<double>, dim3(1), dim3(256),
                                               in_smem ? sizeof(double) * packed : 0, cx.stream, G, bp, p, R, in_smem,
                                               scratch, tol, cx.st, static_cast<const int*>(skip));
            if (le_ != cudaSuccess) return le_;
        }
    } else {
        const int in_smem = (sizeof(float) * packed <= 200 * 1024) ? 1 : 0;
        {
            const cudaError_t le_ = launch_pdl(k_cholesky<float>, dim3(1), dim3(256),
                                               in_smem ? sizeof(float) * packed : 0, cx.stream, G, bp, p, R, in_smem,
                                               scratch, tol, cx.st, static_cast<const int*>(skip));
            if (le_ != cudaSuccess) return le_;
        }
    }
    cx.launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // stage columns 0..cmax of R when (cmax + 1) * bp + 5 bp doubles <= 200 KB
    const int staged_cols = (int)std::min<int64_t>(bp, (200 * 1024 / 8) / bp - 5);
    const int cmax_all = std::min(bp, staged_cols);
    const size_t smem2 = sizeof(double) * (size_t)(5 * bp + (int64_t)bp * std::max(cmax_all, 1));
    {
        const cudaError_t le_ = launch_pdl(k_tri_inverse<T>, dim3((bp + 3) / 4), dim3(128), smem2, cx.stream, R, bp,
                                           Rinv, staged_cols, static_cast<const int*>(skip));
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    return cudaGetLastError();
}

// Upper-triangular inverse of a kdim x kdim FP64 matrix (entries below the
// diagonal are ignored), result in T.
template <typename T>
cudaError_t tri_inverse(Ctx& cx, const double* R, int kdim, T* Rinv) {
    cudaError_t ea = smem_limit(k_tri_inverse<T>, 200 * 1024);
    if (ea != cudaSuccess) return ea;
    const int staged_cols = (int)std::min<int64_t>(kdim, std::max<int64_t>(0, (200 * 1024 / 8) / kdim - 5));
    const int cmax_all = std::min(kdim, staged_cols);
    const size_t smem2 = sizeof(double) * (size_t)(5 * (int64_t)kdim + (int64_t)kdim * std::max(cmax_all, 1));
    if (smem2 > 200 * 1024) return cudaErrorInvalidValue;
    {
        const cudaError_t le_ = launch_pdl(k_tri_inverse<T>, dim3((kdim + 3) / 4), dim3(128), smem2, cx.stream, R,
                                           kdim, Rinv, staged_cols, static_cast<const int*>(nullptr));
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    return cudaGetLastError();
}

template <typename T>
__global__ void k_to_double(int64_t rows, int64_t cols, const T* __restrict__ src, int64_t lds,
                            double* __restrict__ dst, int64_t ldd) {
    pdl_trigger();
    pdl_wait();
    const int64_t total = rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e % rows, c = e / rows;
        dst[r + c * ldd] = (double)src[r + c * lds];
    }
}

template <typename T>
cudaError_t launch_to_double(Ctx& cx, int64_t rows, int64_t cols, const T* src, int64_t lds, double* dst,
                             int64_t ldd) {
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((rows * cols + 255) / 256, cx.num_sms * 4));
    {
        const cudaError_t le_ = launch_pdl(k_to_double<T>, dim3(blocks), dim3(256), 0, cx.stream, rows, cols, src, lds,
                                           dst, ldd);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    return cudaGetLastError();
}

// Downdate + sketch ---------------------------------------------------------
template <typename T, int BM, int BN>
static cudaError_t dd_launch(Ctx& cx, int64_t m, int64_t n, int p, const T* Wsrc, int64_t ldws, const T* Qi,
                             int64_t ldq, const T* Bi, int64_t ldb, const T* Om, T* Wdst, int64_t ldwd, T* Y,
                             int64_t ldy, T* part, size_t part_cap_elems, double* nrm_part, int nrm_cap,
                             double* nrm_out) {
    using C = DDCfg<T, BM, BN>;
    auto kern = k_downdate_sketch<T, BM, BN>;
    cudaError_t ea = smem_limit(kern, (int)C::SMEM);
    if (ea != cudaSuccess) return ea;
    const int64_t mt = (m + BM - 1) / BM;
    const int slots = cx.num_sms * occupancy(kern, C::NT, C::SMEM);
    const int64_t per = m * (int64_t)BN;
    if ((size_t)per > part_cap_elems || mt > nrm_cap) return cudaErrorInvalidValue;
    int maxs = (int)std::min<int64_t>(64, (int64_t)(part_cap_elems / (size_t)per));
    maxs = std::min<int64_t>(maxs, nrm_cap / std::max<int64_t>(mt, 1));
    maxs = std::max(1, maxs);
    int splits = choose_splits(mt, n, 4 * C::BC, maxs, slots);
    int64_t cs = (n + splits - 1) / splits;
    cs = ((cs + C::BC - 1) / C::BC) * C::BC;
    splits = (int)std::max<int64_t>(1, (n + cs - 1) / cs);
    dim3 grid((unsigned)mt, 1, (unsigned)splits);
    kern<<<grid, C::NT, C::SMEM, cx.stream>>>(m, n, p, cs, Wsrc, ldws, Qi, ldq, Bi, ldb, Om, Wdst, ldwd, part, m,
                                              per, nrm_part);
    cx.launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_sum_doubles(cx, nrm_part, (int)(mt * splits), nrm_out);
    if (e != cudaSuccess) return e;
    return launch_reduce_split<T, T>(cx, m, BN, splits, part, m, per, Y, ldy, nullptr, 0, nullptr, 1.0, 0.0, nullptr,
                                     0);
}

template <typename T>
cudaError_t downdate_sketch(Ctx& cx, int64_t m, int64_t n, int p, int bp, const T* Wsrc, int64_t ldws,
                            const T* Qi, int64_t ldq, const T* Bi, int64_t ldb, const T* Om, T* Wdst,
                            int64_t ldwd, T* Y, int64_t ldy, T* part, size_t part_cap_elems, double* nrm_part,
                            int nrm_cap, double* nrm_out) {
    if constexpr (sizeof(T) == 4) {
        if (bp == 32) return dd_launch<T, 128, 32>(cx, m, n, p, Wsrc, ldws, Qi, ldq, Bi, ldb, Om, Wdst, ldwd, Y, ldy, part, part_cap_elems, nrm_part, nrm_cap, nrm_out);
        if (bp == 64) return dd_launch<T, 128, 64>(cx, m, n, p, Wsrc, ldws, Qi, ldq, Bi, ldb, Om, Wdst, ldwd, Y, ldy, part, part_cap_elems, nrm_part, nrm_cap, nrm_out);
        if (bp == 128) return dd_launch<T, 128, 128>(cx, m, n, p, Wsrc, ldws, Qi, ldq, Bi, ldb, Om, Wdst, ldwd, Y, ldy, part, part_cap_elems, nrm_part, nrm_cap, nrm_out);
        if (bp == 256) return dd_launch<T, 64, 256>(cx, m, n, p, Wsrc, ldws, Qi, ldq, Bi, ldb, Om, Wdst, ldwd, Y, ldy, part, part_cap_elems, nrm_part, nrm_cap, nrm_out);
    } else {
        if (bp == 32) return dd_launch<T, 64, 32>(cx, m, n, p, Wsrc, ldws, Qi, ldq, Bi, ldb, Om, Wdst, ldwd, Y, ldy, part, part_cap_elems, nrm_part, nrm_cap, nrm_out);
        if (bp == 64) return dd_launch<T, 64, 64>(cx, m, n, p, Wsrc, ldws, Qi, ldq, Bi, ldb, Om, Wdst, ldwd, Y, ldy, part, part_cap_elems, nrm_part, nrm_cap, nrm_out);
        if (bp == 128) return dd_launch<T, 64, 128>(cx, m, n, p, Wsrc, ldws, Qi, ldq, Bi, ldb, Om, Wdst, ldwd, Y, ldy, part, part_cap_elems, nrm_part, nrm_cap, nrm_out);
    }
    return cudaErrorInvalidValue;
}

// Explicit instantiations ---------------------------------------------------
#define RQB_INST(T)                                                                                              \
    template cudaError_t launch_omega<T>(Ctx&, int64_t, int64_t, int, int, uint64_t, T*, int64_t, int64_t);       \
    template cudaError_t launch_sumsq<T>(Ctx&, int64_t, int64_t, const T*, int64_t, double*, int, double*);       \
    template cudaError_t gemm_nn<T>(Ctx&, const NNArgs<T>&);                                                      \
    template cudaError_t gemm_tn<T>(Ctx&, int64_t, int, int64_t, const T*, int64_t, const T*, int64_t, T*,        \
                                    int64_t, T*, size_t, double*, int, double*);                                 \
    template cudaError_t gemm_tn_f64acc<T>(Ctx&, int64_t, int, int64_t, const T*, int64_t, const T*, int64_t,    \
                                           double*, int64_t, double*, size_t, bool, bool);                        \
    template cudaError_t chol_inv<T>(Ctx&, double*, int, int, double*, T*, bool, double*, size_t, bool);         \
    template cudaError_t downdate_sketch<T>(Ctx&, int64_t, int64_t, int, int, const T*, int64_t, const T*,        \
                                            int64_t, const T*, int64_t, const T*, T*, int64_t, T*, int64_t, T*,   \
                                            size_t, double*, int, double*);                                       \
    template cudaError_t launch_reduce_split<double, T>(Ctx&, int64_t, int64_t, int, const double*, int64_t,      \
                                                        int64_t, T*, int64_t, double*, int, double*, double,      \
                                                        double, const T*, int64_t, int);

RQB_INST(float)
RQB_INST(double)
template cudaError_t launch_sumsq<__nv_bfloat16>(Ctx&, int64_t, int64_t, const __nv_bfloat16*, int64_t, double*, int,
                                                 double*);
template cudaError_t tri_inverse<float>(Ctx&, const double*, int, float*);
template cudaError_t tri_inverse<double>(Ctx&, const double*, int, double*);
template cudaError_t launch_to_double<float>(Ctx&, int64_t, int64_t, const float*, int64_t, double*, int64_t);
template cudaError_t launch_to_double<double>(Ctx&, int64_t, int64_t, const double*, int64_t, double*, int64_t);
#undef RQB_INST

}  // namespace rqb
