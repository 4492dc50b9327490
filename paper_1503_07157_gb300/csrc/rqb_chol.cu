// rqb_chol.cu -- blocked multi-CTA Cholesky of wide panel Gram matrices.
//
// CholeskyQR (Sec. 4.3, lines (3)/(3') of Fig. randQB_b) factors the FP64
// Gram matrix G = Y^T Y of a panel, G = R^T R.  For bp <= 128 the single-CTA
// kernel of rqb_kernels.cu holds G in shared memory; a 256-wide Gram needs
// n^3/3 = 5.6 M FP64 multiply-adds, which one SM (two FP64 FMAs per clock on
// this part) needs about 1.4 ms for.  Here the factorization G = L L^T is
// blocked in 32 x 32 tiles and spread over many CTAs:
//   panel k   every CTA factors the diagonal tile G_kk and inverts L_kk in
//             shared memory; CTA 0 stores L_kk, the others the 8-row strips
//             of L_ik = G_ik L_kk^{-T} below it
//   update k  G_ij -= L_ik L_jk^T for every tile k < j <= i, one CTA per
//             8-row strip
// R = L^T in FP64; R^{-1} = (L^{-1})^T is formed in the output type from L
// staged (packed, lower) in shared memory, one warp per column.
#include <cuda_runtime.h>

#include <algorithm>

#include "rqb_engine.h"
#include "rqb_internal.cuh"

namespace rqb {
namespace {

constexpr int kNb = 32;     // tile
constexpr int kStrip = 8;   // rows per CTA in the solves and updates

// Padding rows/columns >= p become the identity; dG = diagonal of G (the
// reference for the relative pivot test); L cleared.
__global__ void k_chol_init(double* __restrict__ G, int bp, int p, double* __restrict__ dG,
                            double* __restrict__ L) {
    const int total = bp * bp;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int r = e % bp, c = e / bp;
        if (r >= p || c >= p) G[e] = (r == c) ? 1.0 : 0.0;
        L[e] = 0.0;
        if (r == c) dG[r] = (r < p) ? G[e] : 1.0;
    }
}

__global__ void __launch_bounds__(256) k_chol_panel(const double* __restrict__ G, double* __restrict__ L, int bp,
                                                    int k, const double* __restrict__ dG, double tol,
                                                    DevState* st) {
    __shared__ double D[kNb][kNb + 1];    // G_kk -> L_kk (lower)
    __shared__ double Di[kNb][kNb + 1];   // L_kk^{-1} (lower)
    __shared__ int fail;
    const int tid = threadIdx.x;
    const int k0 = k * kNb;
    for (int e = tid; e < kNb * kNb; e += 256) {
        const int r = e & (kNb - 1), c = e / kNb;
        D[r][c] = (r >= c) ? G[(k0 + r) + (int64_t)(k0 + c) * bp] : 0.0;
    }
    if (tid == 0) fail = 0;
    __syncthreads();
    for (int j = 0; j < kNb; ++j) {
        if (tid == 0) {
            double d = D[j][j];
            if (!(d > tol * dG[k0 + j]) || !isfinite(d)) {
                fail = 1;
                d = 1.0;
            }
            D[j][j] = sqrt(d);
        }
        __syncthreads();
        if (tid > j && tid < kNb) D[tid][j] /= D[j][j];
        __syncthreads();
        for (int e = tid; e < kNb * kNb; e += 256) {
            const int r = e & (kNb - 1), c = e / kNb;
            if (c > j && r >= c) D[r][c] -= D[r][j] * D[c][j];
        }
        __syncthreads();
    }
    if (blockIdx.x == 0) {
        for (int e = tid; e < kNb * kNb; e += 256) {
            const int r = e & (kNb - 1), c = e / kNb;
            if (r >= c) L[(k0 + r) + (int64_t)(k0 + c) * bp] = D[r][c];
        }
        if (tid == 0 && fail) record_error(st, RQB_ERR_BREAKDOWN);
        return;
    }
    // L_kk^{-1}: thread c solves column c by forward substitution
    if (tid < kNb) {
        const int c = tid;
        for (int r = 0; r < c; ++r) Di[r][c] = 0.0;
        Di[c][c] = 1.0 / D[c][c];
        for (int r = c + 1; r < kNb; ++r) {
            double s = 0.0;
            for (int t = c; t < r; ++t) s += D[r][t] * Di[t][c];
            Di[r][c] = -s / D[r][r];
        }
    }
    __syncthreads();
    // strip q of tile row i: L_ik(rows) = G_ik(rows) L_kk^{-T}
    const int bi = (blockIdx.x - 1) / (kNb / kStrip), q = (blockIdx.x - 1) % (kNb / kStrip);
    const int rr = tid >> 5, c = tid & 31;
    const int row = (k + 1 + bi) * kNb + q * kStrip + rr;
    double s = 0.0;
#pragma unroll 8
    for (int t = 0; t < kNb; ++t) s += G[row + (int64_t)(k0 + t) * bp] * Di[c][t];
    L[row + (int64_t)(k0 + c) * bp] = s;
}

// G_ij -= L_ik L_jk^T on the 8-row strip (blockIdx.x % 4) of tile pair
// (i, j), k < j <= i < nblk, pairs enumerated column by column.
__global__ void __launch_bounds__(256) k_chol_update(double* __restrict__ G, const double* __restrict__ L, int bp,
                                                     int k, int nblk) {
    __shared__ double Lj[kNb][kNb + 1];
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
        Lj[c][t] = L[(j * kNb + c) + (int64_t)(k0 + t) * bp];
    }
    __syncthreads();
    const int rr = tid >> 5, c = tid & 31;
    const int row = i * kNb + q * kStrip + rr;
    double s = 0.0;
#pragma unroll 8
    for (int t = 0; t < kNb; ++t) s += L[row + (int64_t)(k0 + t) * bp] * Lj[c][t];
    G[row + (int64_t)(j * kNb + c) * bp] -= s;
}

// R = L^T (FP64, column-major, upper).
__global__ void k_chol_transpose(const double* __restrict__ L, int bp, double* __restrict__ R) {
    const int total = bp * bp;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int r = e % bp, c = e / bp;
        R[e] = (r <= c) ? L[c + (int64_t)r * bp] : 0.0;
    }
}

// Rinv = (L^{-1})^T: warp w of CTA b computes column c = b * 8 + w of L^{-1}
// by forward substitution down the column, with L staged in shared memory
// (type W, columns packed: column t holds rows t .. bp-1).
template <typename T, typename W>
__global__ void __launch_bounds__(256) k_lower_inverse(const double* __restrict__ L, int bp, T* __restrict__ Rinv) {
    extern __shared__ __align__(16) unsigned char inv_smem[];
    W* Ls = reinterpret_cast<W*>(inv_smem);
    W* xs = Ls + (size_t)bp * (bp + 1) / 2;                  // 8 x bp
    auto off = [bp](int t) { return (size_t)t * bp - (size_t)t * (t - 1) / 2; };
    for (int t = 0; t < bp; ++t)
        for (int r = t + threadIdx.x; r < bp; r += 256) Ls[off(t) + (r - t)] = (W)L[r + (int64_t)t * bp];
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

}  // namespace

// G (bp x bp, FP64, overwritten) = R^T R; R (FP64) and Rinv (T).  scratch:
// bp * bp + bp doubles (L and the diagonal of G).
template <typename T>
cudaError_t chol_inv_blocked(Ctx& cx, double* G, int bp, int p, double* R, T* Rinv, double tol, double* scratch,
                             size_t scratch_doubles) {
    if (bp % kNb != 0 || scratch_doubles < (size_t)bp * bp + bp) return cudaErrorInvalidValue;
    using W = T;   // inverse in the output precision
    const size_t inv_smem = sizeof(W) * ((size_t)bp * (bp + 1) / 2 + 8 * (size_t)bp);
    if (inv_smem > 200 * 1024) return cudaErrorInvalidValue;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_lower_inverse<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    double* L = scratch;
    double* dG = scratch + (size_t)bp * bp;
    const int nblk = bp / kNb;
    k_chol_init<<<std::max(1, bp * bp / 256), 256, 0, cx.stream>>>(G, bp, p, dG, L);
    cx.launches++;
    for (int k = 0; k < nblk; ++k) {
        const int below = nblk - k - 1;
        k_chol_panel<<<1 + below * (kNb / kStrip), 256, 0, cx.stream>>>(G, L, bp, k, dG, tol, cx.st);
        cx.launches++;
        if (below > 0) {
            const int pairs = below * (below + 1) / 2;
            k_chol_update<<<pairs * (kNb / kStrip), 256, 0, cx.stream>>>(G, L, bp, k, nblk);
            cx.launches++;
        }
    }
    k_chol_transpose<<<std::max(1, bp * bp / 256), 256, 0, cx.stream>>>(L, bp, R);
    cx.launches++;
    k_lower_inverse<T, W><<<(bp + 7) / 8, 256, inv_smem, cx.stream>>>(L, bp, Rinv);
    cx.launches++;
    return cudaGetLastError();
}

template cudaError_t chol_inv_blocked<float>(Ctx&, double*, int, int, double*, float*, double, double*, size_t);
template cudaError_t chol_inv_blocked<double>(Ctx&, double*, int, int, double*, double*, double, double*, size_t);

}  // namespace rqb
