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
// R = L^T in FP64; R^{-1} is formed in the output type from R staged
// (packed) in shared memory, one warp per column.
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

template <typename W>
__global__ void __launch_bounds__(256) k_chol_panel(const double* __restrict__ G, double* __restrict__ L, int bp,
                                                    int k, const double* __restrict__ dG, double tol,
                                                    DevState* st) {
    __shared__ W D[kNb][kNb + 1];    // G_kk -> L_kk (lower)
    __shared__ W Di[kNb][kNb + 1];   // I -> L_kk^{-1} (lower)
    __shared__ W inv[kNb];
    __shared__ int fail;
    const int tid = threadIdx.x;
    const int k0 = k * kNb;
    for (int e = tid; e < kNb * kNb; e += 256) {
        const int r = e & (kNb - 1), c = e / kNb;
        D[r][c] = (r >= c) ? (W)G[(k0 + r) + (int64_t)(k0 + c) * bp] : W(0);
        Di[r][c] = (r == c) ? W(1) : W(0);
    }
    if (tid == 0) fail = 0;
    __syncthreads();
    // step j: pivot; scale column j of L and row j of L^{-1} by 1 / l_jj;
    // update the trailing part of L and eliminate column j from the rows of
    // L^{-1} below j (forward substitution applied to all columns at once)
    for (int j = 0; j < kNb; ++j) {
        if (tid == 0) {
            W d = D[j][j];
            if (!((double)d > tol * dG[k0 + j]) || !isfinite((double)d)) {
                fail = 1;
                d = W(1);
            }
            const W l = sqrt(d);
            D[j][j] = l;
            inv[j] = W(1) / l;
        }
        __syncthreads();
        const W ij = inv[j];
        if (tid < kNb) {
            if (tid > j) D[tid][j] *= ij;
        } else if (tid < 2 * kNb) {
            if (tid - kNb <= j) Di[j][tid - kNb] *= ij;
        }
        __syncthreads();
        for (int e = tid; e < kNb * kNb; e += 256) {
            const int r = e & (kNb - 1), c = e / kNb;
            if (c > j && r >= c) D[r][c] -= D[r][j] * D[c][j];
            else if (r > j && c <= j) Di[r][c] -= D[r][j] * Di[j][c];
        }
        __syncthreads();
    }
    if (blockIdx.x == 0) {
        for (int e = tid; e < kNb * kNb; e += 256) {
            const int r = e & (kNb - 1), c = e / kNb;
            if (r >= c) L[(k0 + r) + (int64_t)(k0 + c) * bp] = (double)D[r][c];
        }
        if (tid == 0 && fail) record_error(st, RQB_ERR_BREAKDOWN);
        return;
    }
    // strip q of tile row i: L_ik(rows) = G_ik(rows) L_kk^{-T}
    const int bi = (blockIdx.x - 1) / (kNb / kStrip), q = (blockIdx.x - 1) % (kNb / kStrip);
    const int rr = tid >> 5, c = tid & 31;
    const int row = (k + 1 + bi) * kNb + q * kStrip + rr;
    W s = W(0);
#pragma unroll 8
    for (int t = 0; t < kNb; ++t) s += (W)G[row + (int64_t)(k0 + t) * bp] * Di[c][t];
    L[row + (int64_t)(k0 + c) * bp] = (double)s;
}

// G_ij -= L_ik L_jk^T on the 8-row strip (blockIdx.x % 4) of tile pair
// (i, j), k < j <= i < nblk, pairs enumerated column by column.
template <typename W>
__global__ void __launch_bounds__(256) k_chol_update(double* __restrict__ G, const double* __restrict__ L, int bp,
                                                     int k, int nblk) {
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

// R = L^T (FP64, column-major, upper).
__global__ void k_chol_transpose(const double* __restrict__ L, int bp, double* __restrict__ R) {
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

}  // namespace

// Rinv (T) = R^{-1} for an upper-triangular FP64 R (bp x bp, column-major);
// the substitution runs in T.
template <typename T>
cudaError_t upper_inverse(Ctx& cx, const double* R, int bp, T* Rinv) {
    using W = T;
    const size_t smem = sizeof(W) * ((size_t)bp * (bp + 1) / 2 + 8 * (size_t)bp);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_upper_inverse<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    k_upper_inverse<T, W><<<(bp + 7) / 8, 256, smem, cx.stream>>>(R, bp, Rinv);
    cx.launches++;
    return cudaGetLastError();
}

// G (bp x bp, FP64, overwritten) = R^T R; R (FP64) and Rinv (T).  scratch:
// bp * bp + bp doubles (L and the diagonal of G).  fp64: working precision
// of the factorization (FP32 serves the second CholeskyQR pass, whose Gram
// is I + O(u kappa)); the factors are stored in FP64 either way.
template <typename T>
cudaError_t chol_inv_blocked(Ctx& cx, double* G, int bp, int p, double* R, T* Rinv, double tol, double* scratch,
                             size_t scratch_doubles, bool fp64) {
    if (bp % kNb != 0 || scratch_doubles < (size_t)bp * bp + bp) return cudaErrorInvalidValue;
    double* L = scratch;
    double* dG = scratch + (size_t)bp * bp;
    const int nblk = bp / kNb;
    k_chol_init<<<std::max(1, bp * bp / 256), 256, 0, cx.stream>>>(G, bp, p, dG, L);
    cx.launches++;
    for (int k = 0; k < nblk; ++k) {
        const int below = nblk - k - 1;
        if (fp64)
            k_chol_panel<double><<<1 + below * (kNb / kStrip), 256, 0, cx.stream>>>(G, L, bp, k, dG, tol, cx.st);
        else
            k_chol_panel<float><<<1 + below * (kNb / kStrip), 256, 0, cx.stream>>>(G, L, bp, k, dG, tol, cx.st);
        cx.launches++;
        if (below > 0) {
            const int pairs = below * (below + 1) / 2;
            if (fp64)
                k_chol_update<double><<<pairs * (kNb / kStrip), 256, 0, cx.stream>>>(G, L, bp, k, nblk);
            else
                k_chol_update<float><<<pairs * (kNb / kStrip), 256, 0, cx.stream>>>(G, L, bp, k, nblk);
            cx.launches++;
        }
    }
    k_chol_transpose<<<std::max(1, bp * bp / 256), 256, 0, cx.stream>>>(L, bp, R);
    cx.launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return upper_inverse<T>(cx, R, bp, Rinv);
}

template cudaError_t upper_inverse<float>(Ctx&, const double*, int, float*);
template cudaError_t upper_inverse<double>(Ctx&, const double*, int, double*);
template cudaError_t chol_inv_blocked<float>(Ctx&, double*, int, int, double*, float*, double, double*, size_t, bool);
template cudaError_t chol_inv_blocked<double>(Ctx&, double*, int, int, double*, double*, double, double*, size_t,
                                              bool);

}  // namespace rqb
