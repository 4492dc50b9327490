// rqb_gemm_simt.cuh -- register-blocked SIMT GEMM tiles for the tall-skinny
// products of randQB_b (FP32 and FP64 pipes).
//
// Two shapes cover every product of Fig. randQB_b:
//   NN:  Out (m x N) = alpha * X (m x K) * C (K x N) + beta * Yin
//        -- the sketch A Omega (line (3)), Q_i = Y R^{-1}, Y - Qbar C (line (3'))
//   TN:  Out (P x Q) = X^T (P x m) * Y (m x Q), a reduction over the m rows
//        -- B_i = Q_i^T A (line (4)), Gram matrices and Qbar^T Y of the panel
// Both split the reduction dimension over gridDim.z; each split writes its
// own partial (deterministic two-stage reduction, no float atomics).
//
// Every global access is bounds-checked per element or per 16-byte vector
// (a vector is used only when it is aligned and entirely in range).
#pragma once

#include "rqb_internal.cuh"

namespace rqb {

// Thread tile: float threads own 8 x 8 outputs, double threads 4 x 4; each
// thread's rows are two groups of TM/2 contiguous rows, BM/2 apart, and its
// columns two groups of TN/2, BN/2 apart (conflict-free vector smem reads).
template <typename T> struct SimtTile;
template <> struct SimtTile<float> { static constexpr int TM = 8, TN = 8; };
template <> struct SimtTile<double> { static constexpr int TM = 4, TN = 4; };

// Packed FP32 multiply-adds (two per instruction on this part's FP32 pipe):
// acc2[i][jp] += (a[i] a[i]) * (b[2jp] b[2jp+1]), each lane an IEEE
// binary32 fused multiply-add rounded to nearest, so the results are bit for
// bit those of fmaf in the same order.  Half the FMA instructions leave issue
// slots to the loads of the issue-bound SIMT products.
template <int TM, int TN>
__device__ __forceinline__ void fma_tile_f32x2(float2 (&acc2)[TM][TN / 2], const float (&a)[TM],
                                               const float (&b)[TN]) {
    float2 bp[TN / 2];
#pragma unroll
    for (int j = 0; j < TN / 2; ++j) bp[j] = make_float2(b[2 * j], b[2 * j + 1]);
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const float2 aa = make_float2(a[i], a[i]);
#pragma unroll
        for (int j = 0; j < TN / 2; ++j) acc2[i][j] = __ffma2_rn(aa, bp[j], acc2[i][j]);
    }
}
// The same with the pairs along rows: accr[ip][j] += (a[2ip] a[2ip+1]) *
// (b[j] b[j]).
template <int TM, int TN>
__device__ __forceinline__ void fma_tile_f32x2_rows(float2 (&accr)[TM / 2][TN], const float (&a)[TM],
                                                    const float (&b)[TN]) {
#pragma unroll
    for (int j = 0; j < TN; ++j) {
        const float2 bb = make_float2(b[j], b[j]);
#pragma unroll
        for (int i = 0; i < TM / 2; ++i) accr[i][j] = __ffma2_rn(make_float2(a[2 * i], a[2 * i + 1]), bb, accr[i][j]);
    }
}

template <int TM, int TN>
__device__ __forceinline__ void zero_tile_f32x2(float2 (&acc2)[TM][TN / 2]) {
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN / 2; ++j) acc2[i][j] = make_float2(0.f, 0.f);
}
template <int TM, int TN, typename T>
__device__ __forceinline__ void unpack_tile_f32x2(const float2 (&acc2)[TM][TN / 2], T (&acc)[TM][TN]) {
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN / 2; ++j) {
            acc[i][2 * j] = (T)acc2[i][j].x;
            acc[i][2 * j + 1] = (T)acc2[i][j].y;
        }
}

template <typename T, int H> struct VecH;   // H contiguous elements
template <> struct VecH<float, 4> { using type = float4; };
template <> struct VecH<float, 2> { using type = float2; };
template <> struct VecH<double, 2> { using type = double2; };

template <typename T, int H>
__device__ __forceinline__ void lds_vec(T (&dst)[H], const T* src) {
    using V = typename VecH<T, H>::type;
    const V v = *reinterpret_cast<const V*>(src);
    const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
    for (int i = 0; i < H; ++i) dst[i] = e[i];
}

// Load V16 consecutive elements p[0..V16) of a contiguous run whose valid
// length from p is `valid` (<= 0: all zeros).  Uses one 16-byte load when the
// run is complete and p is aligned.
template <typename T>
__device__ __forceinline__ void ldg_run(T* dst, const T* p, int64_t valid) {
    constexpr int V = Vec16<T>::N;
    if (valid >= V && aligned16(p)) {
        using VT = typename Vec16<T>::type;
        const VT v = __ldg(reinterpret_cast<const VT*>(p));
        const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
        for (int i = 0; i < V; ++i) dst[i] = e[i];
    } else {
#pragma unroll
        for (int i = 0; i < V; ++i) dst[i] = (i < valid) ? __ldg(p + i) : T(0);
    }
}

// ---------------------------------------------------------------------------
// NN: Out[z] (rows r0.., cols) = alpha * sum_{k in split z} X(r,k) C(k,j) + beta * Yin(r,j)
// C(k, j) = C[k * csk + j * csj]; C_ROWMAJOR selects csj == 1 (else csk == 1).
// Columns j >= nc read C as zero; only columns j < nout and rows r < m are written.
template <typename T, int BM, int BN, int BK, bool C_ROWMAJOR>
struct GemmNN {
    static constexpr int TM = SimtTile<T>::TM, TN = SimtTile<T>::TN;
    static constexpr int NT = (BM / TM) * (BN / TN);
    static constexpr int V = Vec16<T>::N;
    static constexpr int XVEC = BM * BK / V;   // 16-byte vectors per X tile
    static constexpr int CVEC = BK * BN / V;
    static_assert(XVEC % NT == 0 || NT % XVEC == 0, "X tile split");
    static constexpr int XPER = (XVEC + NT - 1) / NT;
    static constexpr int CPER = (CVEC + NT - 1) / NT;
    static constexpr int SMEM_ELEMS = 2 * BK * (BM + BN);
};

template <typename T, int BM, int BN, int BK, bool C_ROWMAJOR>
__global__ void __launch_bounds__(GemmNN<T, BM, BN, BK, C_ROWMAJOR>::NT,
                                  (sizeof(T) == 4 && GemmNN<T, BM, BN, BK, C_ROWMAJOR>::NT >= 256) ? 2 : 1)
k_gemm_nn(int64_t m, int64_t K, int64_t ksplit, int nc, int nout,
          const T* __restrict__ X, int64_t ldx,
          const T* __restrict__ C, int64_t csk, int64_t csj,
          T* Out, int64_t ldo, int64_t out_zstride,
          const T* Yin, int64_t ldyin, T alpha, T beta, double* __restrict__ nrm_part) {
    using G = GemmNN<T, BM, BN, BK, C_ROWMAJOR>;
    constexpr int TM = G::TM, TN = G::TN, NT = G::NT, V = G::V;
    constexpr int HM = TM / 2, HN = TN / 2;
    __shared__ __align__(16) T As[2][BK][BM];
    __shared__ __align__(16) T Bs[2][BK][BN];

    const int tid = threadIdx.x;
    const int tx = tid % (BN / TN), ty = tid / (BN / TN);
    const int64_t r0 = (int64_t)blockIdx.x * BM;
    const int j0 = blockIdx.y * BN;
    const int64_t kbeg = (int64_t)blockIdx.z * ksplit;
    const int64_t kend = (kbeg + ksplit < K) ? kbeg + ksplit : K;

    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
    // FP32 tiles of up to 128 x 64: acc as column pairs for the packed FMAs
    // (the larger tiles keep scalar FMAs: their pairs would not fit the
    // registers of two CTAs per SM)
    constexpr bool kPackNN = (sizeof(T) == 4) && (BN <= 64);
    float2 accq[TM][TN / 2];
    if constexpr (kPackNN) zero_tile_f32x2<TM, TN>(accq);

    T xa[G::XPER][V];
    T cb[G::CPER][V];
    // ||X||_F^2 of the tiles this CTA reads (only the blockIdx.y == 0 column
    // of CTAs counts, so every element of X is counted once)
    const bool do_norm = (nrm_part != nullptr) && (blockIdx.y == 0);
    double nacc = 0.0;

    // X tile: vector v covers rows rr..rr+V of column kk (BM/V vectors per column)
    auto load_x = [&](int64_t k0) {
#pragma unroll
        for (int t = 0; t < G::XPER; ++t) {
            const int v = tid + t * NT;
            if (v < G::XVEC) {
                const int kk = v / (BM / V);
                const int rr = (v % (BM / V)) * V;
                const int64_t k = k0 + kk, r = r0 + rr;
                if (k < kend && r < m) ldg_run<T>(xa[t], X + r + k * ldx, m - r);
                else {
#pragma unroll
                    for (int i = 0; i < V; ++i) xa[t][i] = T(0);
                }
                if (do_norm) {
                    T sq = T(0);
#pragma unroll
                    for (int i = 0; i < V; ++i) sq = fma(xa[t][i], xa[t][i], sq);
                    nacc += (double)sq;
                }
            }
        }
    };
    auto store_x = [&](int buf) {
#pragma unroll
        for (int t = 0; t < G::XPER; ++t) {
            const int v = tid + t * NT;
            if (v < G::XVEC) {
                const int kk = v / (BM / V);
                const int rr = (v % (BM / V)) * V;
#pragma unroll
                for (int i = 0; i < V; ++i) As[buf][kk][rr + i] = xa[t][i];
            }
        }
    };
    auto load_c = [&](int64_t k0) {
#pragma unroll
        for (int t = 0; t < G::CPER; ++t) {
            const int v = tid + t * NT;
            if (v < G::CVEC) {
                if (C_ROWMAJOR) {   // vector along j
                    const int kk = v / (BN / V);
                    const int jj = (v % (BN / V)) * V;
                    const int64_t k = k0 + kk;
                    const int j = j0 + jj;
                    if (k < kend && j < nc) ldg_run<T>(cb[t], C + k * csk + j, nc - j);
                    else {
#pragma unroll
                        for (int i = 0; i < V; ++i) cb[t][i] = T(0);
                    }
                } else {            // vector along k
                    const int jj = v / (BK / V);
                    const int kk = (v % (BK / V)) * V;
                    const int64_t k = k0 + kk;
                    const int j = j0 + jj;
                    if (k < kend && j < nc) ldg_run<T>(cb[t], C + k + (int64_t)j * csj, kend - k);
                    else {
#pragma unroll
                        for (int i = 0; i < V; ++i) cb[t][i] = T(0);
                    }
                }
            }
        }
    };
    auto store_c = [&](int buf) {
#pragma unroll
        for (int t = 0; t < G::CPER; ++t) {
            const int v = tid + t * NT;
            if (v < G::CVEC) {
                if (C_ROWMAJOR) {
                    const int kk = v / (BN / V);
                    const int jj = (v % (BN / V)) * V;
#pragma unroll
                    for (int i = 0; i < V; ++i) Bs[buf][kk][jj + i] = cb[t][i];
                } else {
                    const int jj = v / (BK / V);
                    const int kk = (v % (BK / V)) * V;
#pragma unroll
                    for (int i = 0; i < V; ++i) Bs[buf][kk + i][jj] = cb[t][i];
                }
            }
        }
    };

    int buf = 0;
    if (kbeg < kend) {
        load_x(kbeg);
        load_c(kbeg);
        store_x(0);
        store_c(0);
    }
    __syncthreads();
    for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
        const bool more = (k0 + BK < kend);
        if (more) {
            load_x(k0 + BK);
            load_c(k0 + BK);
        }
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM], b[TN];
            T a0[HM], a1[HM], b0[HN], b1[HN];
            lds_vec<T, HM>(a0, &As[buf][kk][ty * HM]);
            lds_vec<T, HM>(a1, &As[buf][kk][BM / 2 + ty * HM]);
            lds_vec<T, HN>(b0, &Bs[buf][kk][tx * HN]);
            lds_vec<T, HN>(b1, &Bs[buf][kk][BN / 2 + tx * HN]);
#pragma unroll
            for (int i = 0; i < HM; ++i) { a[i] = a0[i]; a[HM + i] = a1[i]; }
#pragma unroll
            for (int j = 0; j < HN; ++j) { b[j] = b0[j]; b[HN + j] = b1[j]; }
            if constexpr (kPackNN) {
                fma_tile_f32x2<TM, TN>(accq, a, b);
            } else {
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
        }
        if (more) {
            store_x(buf ^ 1);
            store_c(buf ^ 1);
        }
        __syncthreads();
        buf ^= 1;
    }
    if constexpr (kPackNN) unpack_tile_f32x2<TM, TN>(accq, acc);

    if (nrm_part != nullptr) {   // uniform per CTA
        __shared__ double red[NT / 32];
        double v = nacc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0) red[tid >> 5] = v;
        __syncthreads();
        if (tid == 0 && do_norm) {
            double t = 0.0;
            for (int w = 0; w < NT / 32; ++w) t += red[w];
            nrm_part[blockIdx.x + (int64_t)gridDim.x * blockIdx.z] = t;
        }
    }

    // epilogue
    T* out = Out + (int64_t)blockIdx.z * out_zstride;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t r = r0 + ((i < HM) ? (ty * HM + i) : (BM / 2 + ty * HM + (i - HM)));
        if (r >= m) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int c = j0 + ((j < HN) ? (tx * HN + j) : (BN / 2 + tx * HN + (j - HN)));
            if (c >= nout) continue;
            T v = alpha * acc[i][j];
            if (beta != T(0)) v = fma(beta, Yin[r + (int64_t)c * ldyin], v);
            out[r + (int64_t)c * ldo] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// NN with a row-major C, fed by cp.async: the X and C tiles of the next
// ST - 1 reduction chunks are in flight while the current one is multiplied,
// so the loads need no staging registers and their latency is covered by
// several chunks of FMAs instead of one.  Same contract as k_gemm_nn with
// C_ROWMAJOR, plus: X, C 16-byte aligned, ldx and csk multiples of 16 bytes
// (the host checks).  Elements outside the matrices are zero-filled by the
// copy itself (src-size below 16 bytes).
template <typename T, int BM, int BN, int BK, int ST>
struct GemmNNPipe {
    static constexpr int TM = SimtTile<T>::TM, TN = SimtTile<T>::TN;
    static constexpr int NT = (BM / TM) * (BN / TN);
    static constexpr int V = Vec16<T>::N;
    static constexpr int XVEC = BM * BK / V, CVEC = BK * BN / V;
    static constexpr int XPER = (XVEC + NT - 1) / NT, CPER = (CVEC + NT - 1) / NT;
    static constexpr size_t SMEM = sizeof(T) * (size_t)ST * BK * (BM + BN);
    static constexpr int MINB = (sizeof(T) == 4 && NT >= 256) ? 2 : 1;
};

template <typename T, int BM, int BN, int BK, int ST>
__global__ void __launch_bounds__(GemmNNPipe<T, BM, BN, BK, ST>::NT, GemmNNPipe<T, BM, BN, BK, ST>::MINB)
k_gemm_nn_pipe(int64_t m, int64_t K, int64_t ksplit, int nc, int nout,
               const T* __restrict__ X, int64_t ldx, const T* __restrict__ C, int64_t csk,
               T* Out, int64_t ldo, int64_t out_zstride,
               const T* Yin, int64_t ldyin, T alpha, T beta, double* __restrict__ nrm_part) {
    using G = GemmNNPipe<T, BM, BN, BK, ST>;
    constexpr int TM = G::TM, TN = G::TN, NT = G::NT, V = G::V;
    constexpr int HM = TM / 2, HN = TN / 2;
    extern __shared__ __align__(16) unsigned char nn_smem[];
    T* As = reinterpret_cast<T*>(nn_smem);   // [ST][BK][BM]
    T* Bs = As + (size_t)ST * BK * BM;        // [ST][BK][BN]

    const int tid = threadIdx.x;
    const int tx = tid % (BN / TN), ty = tid / (BN / TN);
    const int64_t r0 = (int64_t)blockIdx.x * BM;
    const int j0 = blockIdx.y * BN;
    const int64_t kbeg = (int64_t)blockIdx.z * ksplit;
    const int64_t kend = (kbeg + ksplit < K) ? kbeg + ksplit : K;
    const int64_t nch = (kend > kbeg) ? (kend - kbeg + BK - 1) / BK : 0;

    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
    // FP32 tiles of 128 rows: the accumulators as pairs for the packed FMAs
    // (the 64 x 256 tile keeps scalar FMAs, its pairs would spill)
    constexpr bool kPackP = (sizeof(T) == 4) && (BM == 128);
    float2 acc2[TM][TN / 2];
    if constexpr (kPackP) zero_tile_f32x2<TM, TN>(acc2);
    const bool do_norm = (nrm_part != nullptr) && (blockIdx.y == 0);
    double nacc = 0.0;

    // chunk c (K columns kbeg + c*BK ..) into stage c % ST
    auto issue = [&](int64_t c) {
        const int s = (int)(c % ST);
        const int64_t k0 = kbeg + c * BK;
#pragma unroll
        for (int t = 0; t < G::XPER; ++t) {
            const int v = tid + t * NT;
            if (v < G::XVEC) {
                const int kk = v / (BM / V), rr = (v % (BM / V)) * V;
                const int64_t k = k0 + kk, r = r0 + rr;
                int64_t valid = (k < kend) ? m - r : 0;
                valid = valid < 0 ? 0 : (valid > V ? V : valid);
                const T* src = (valid > 0) ? X + r + k * ldx : X;
                cp_async16(As + ((size_t)s * BK + kk) * BM + rr, src, (int)(valid * sizeof(T)));
            }
        }
#pragma unroll
        for (int t = 0; t < G::CPER; ++t) {
            const int v = tid + t * NT;
            if (v < G::CVEC) {
                const int kk = v / (BN / V), jj = (v % (BN / V)) * V;
                const int64_t k = k0 + kk;
                const int j = j0 + jj;
                int valid = (k < kend) ? nc - j : 0;
                valid = valid < 0 ? 0 : (valid > V ? V : valid);
                const T* src = (valid > 0) ? C + k * csk + j : C;
                cp_async16(Bs + ((size_t)s * BK + kk) * BN + jj, src, valid * (int)sizeof(T));
            }
        }
    };

#pragma unroll
    for (int s = 0; s < ST - 1; ++s) {
        if (s < nch) issue(s);
        cp_async_commit();
    }
    for (int64_t c = 0; c < nch; ++c) {
        cp_async_wait<ST - 2>();
        __syncthreads();   // chunk c landed for every thread; stage (c - 1) % ST is free
        if (c + ST - 1 < nch) issue(c + ST - 1);
        cp_async_commit();
        const T* as = As + (size_t)(c % ST) * BK * BM;
        const T* bs = Bs + (size_t)(c % ST) * BK * BN;
        if (do_norm) {   // this thread's own vectors of the X chunk, each element once
#pragma unroll
            for (int t = 0; t < G::XPER; ++t) {
                const int v = tid + t * NT;
                if (v < G::XVEC) {
                    const int kk = v / (BM / V), rr = (v % (BM / V)) * V;
                    T xv[V];
                    lds_vec<T, V>(xv, as + kk * BM + rr);
                    T sq = T(0);
#pragma unroll
                    for (int i = 0; i < V; ++i) sq = fma(xv[i], xv[i], sq);
                    nacc += (double)sq;
                }
            }
        }
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM], b[TN];
            T a0[HM], a1[HM], b0[HN], b1[HN];
            lds_vec<T, HM>(a0, as + kk * BM + ty * HM);
            lds_vec<T, HM>(a1, as + kk * BM + BM / 2 + ty * HM);
            lds_vec<T, HN>(b0, bs + kk * BN + tx * HN);
            lds_vec<T, HN>(b1, bs + kk * BN + BN / 2 + tx * HN);
#pragma unroll
            for (int i = 0; i < HM; ++i) { a[i] = a0[i]; a[HM + i] = a1[i]; }
#pragma unroll
            for (int j = 0; j < HN; ++j) { b[j] = b0[j]; b[HN + j] = b1[j]; }
            if constexpr (kPackP) {
                fma_tile_f32x2<TM, TN>(acc2, a, b);
            } else {
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
        }
    }
    cp_async_wait<0>();
    if constexpr (kPackP) unpack_tile_f32x2<TM, TN>(acc2, acc);

    if (nrm_part != nullptr) {   // uniform per CTA
        __shared__ double red[NT / 32];
        double v = nacc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0) red[tid >> 5] = v;
        __syncthreads();
        if (tid == 0 && do_norm) {
            double t = 0.0;
            for (int w = 0; w < NT / 32; ++w) t += red[w];
            nrm_part[blockIdx.x + (int64_t)gridDim.x * blockIdx.z] = t;
        }
    }

    T* out = Out + (int64_t)blockIdx.z * out_zstride;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t r = r0 + ((i < HM) ? (ty * HM + i) : (BM / 2 + ty * HM + (i - HM)));
        if (r >= m) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int c = j0 + ((j < HN) ? (tx * HN + j) : (BN / 2 + tx * HN + (j - HN)));
            if (c >= nout) continue;
            T v = alpha * acc[i][j];
            if (beta != T(0)) v = fma(beta, Yin[r + (int64_t)c * ldyin], v);
            out[r + (int64_t)c * ldo] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// TN: Out[z] (p x q) = sum over rows r of split z of X(r, p) * Y(r, q).
// X is m x pn (ldx), Y is m x qn (ldy); rows >= m and columns beyond pn/qn
// read as zero; outputs with p < pn, q < qn are written, type Acc.
// With PROMOTE > 0 (Acc = double, T = float) the FP32 tile accumulators are
// added into FP64 accumulators every PROMOTE row-chunks of BK rows.
// With COMP (T = float) every product is formed exactly as a pair
// (a*b, fma(a, b, -a*b)) and summed with TwoSum into an unevaluated FP32 pair
// (Knuth's error-free transformations), so the FP64 result carries about
// 2^-46 relative error instead of 2^-24: the accuracy the Gram matrix of an
// ill-conditioned panel needs before its Cholesky factorisation.
__device__ __forceinline__ void exact_fma_acc(float a, float b, float& hi, float& lo) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    const float s = __fadd_rn(hi, p);
    const float bv = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(p, bv));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
}

template <typename T, typename Acc, int BP, int BQ, int BK, int TP, int TQ, int PROMOTE, bool COMP = false>
__global__ void __launch_bounds__((BP / TP) * (BQ / TQ), ((BP / TP) * (BQ / TQ) >= 256 && TP * TQ == 64) ? 2 : 1)
k_gemm_tn(int64_t m, int pn, int64_t qn, int64_t rsplit,
          const T* __restrict__ X, int64_t ldx,
          const T* __restrict__ Y, int64_t ldy,
          Acc* __restrict__ Out, int64_t ldo, int64_t out_zstride, int sym) {
    // sym (X = Y, a Gram matrix): tiles strictly above the diagonal are left
    // to the reduction, which reads their mirror image
    if (sym && (int64_t)blockIdx.x * BP + BP <= (int64_t)blockIdx.y * BQ) return;
    constexpr int NT = (BP / TP) * (BQ / TQ);
    constexpr int V = Vec16<T>::N;
    constexpr int HP = TP / 2, HQ = TQ / 2;
    constexpr int XVEC = BP * BK / V, YVEC = BQ * BK / V;
    constexpr int XPER = (XVEC + NT - 1) / NT, YPER = (YVEC + NT - 1) / NT;
    constexpr int PAD = 4;   // breaks the 4-way bank conflict of the transposed stores
    __shared__ __align__(16) T Xs[2][BK][BP + PAD];
    __shared__ __align__(16) T Ys[2][BK][BQ + PAD];

    const int tid = threadIdx.x;
    const int tq = tid % (BQ / TQ), tp = tid / (BQ / TQ);
    const int p0 = blockIdx.x * BP;
    const int64_t q0 = (int64_t)blockIdx.y * BQ;
    const int64_t rbeg = (int64_t)blockIdx.z * rsplit;
    const int64_t rend = (rbeg + rsplit < m) ? rbeg + rsplit : m;

    T acc[TP][TQ];
    T lo[TP][TQ];
    Acc acc2[TP][TQ];
#pragma unroll
    for (int i = 0; i < TP; ++i)
#pragma unroll
        for (int j = 0; j < TQ; ++j) { acc[i][j] = T(0); lo[i][j] = T(0); acc2[i][j] = Acc(0); }
    // FP32 without COMP: the running sums as pairs for the packed FMAs
    constexpr bool kPacked = (sizeof(T) == 4) && !COMP && (TP % 2 == 0);
    float2 accp[(TP + 1) / 2][TQ];
    if constexpr (kPacked) {
#pragma unroll
        for (int i = 0; i < (TP + 1) / 2; ++i)
#pragma unroll
            for (int j = 0; j < TQ; ++j) accp[i][j] = make_float2(0.f, 0.f);
    }

    T xa[XPER][V], ya[YPER][V];
    // vector v: column cc = v / (BK/V), rows kk..kk+V
    auto load = [&](int64_t rr0) {
#pragma unroll
        for (int t = 0; t < XPER; ++t) {
            const int v = tid + t * NT;
            if (v < XVEC) {
                const int cc = v / (BK / V), kk = (v % (BK / V)) * V;
                const int p = p0 + cc;
                const int64_t r = rr0 + kk;
                if (p < pn && r < rend) ldg_run<T>(xa[t], X + r + (int64_t)p * ldx, rend - r);
                else {
#pragma unroll
                    for (int i = 0; i < V; ++i) xa[t][i] = T(0);
                }
            }
        }
#pragma unroll
        for (int t = 0; t < YPER; ++t) {
            const int v = tid + t * NT;
            if (v < YVEC) {
                const int cc = v / (BK / V), kk = (v % (BK / V)) * V;
                const int64_t q = q0 + cc;
                const int64_t r = rr0 + kk;
                if (q < qn && r < rend) ldg_run<T>(ya[t], Y + r + q * ldy, rend - r);
                else {
#pragma unroll
                    for (int i = 0; i < V; ++i) ya[t][i] = T(0);
                }
            }
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int t = 0; t < XPER; ++t) {
            const int v = tid + t * NT;
            if (v < XVEC) {
                const int cc = v / (BK / V), kk = (v % (BK / V)) * V;
#pragma unroll
                for (int i = 0; i < V; ++i) Xs[buf][kk + i][cc] = xa[t][i];
            }
        }
#pragma unroll
        for (int t = 0; t < YPER; ++t) {
            const int v = tid + t * NT;
            if (v < YVEC) {
                const int cc = v / (BK / V), kk = (v % (BK / V)) * V;
#pragma unroll
                for (int i = 0; i < V; ++i) Ys[buf][kk + i][cc] = ya[t][i];
            }
        }
    };

    int buf = 0;
    if (rbeg < rend) {
        load(rbeg);
        store(0);
    }
    __syncthreads();
    int chunk = 0;
    for (int64_t rr0 = rbeg; rr0 < rend; rr0 += BK) {
        const bool more = (rr0 + BK < rend);
        if (more) load(rr0 + BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TP], b[TQ];
            T a0[HP], a1[HP], b0[HQ], b1[HQ];
            lds_vec<T, HP>(a0, &Xs[buf][kk][tp * HP]);
            lds_vec<T, HP>(a1, &Xs[buf][kk][BP / 2 + tp * HP]);
            lds_vec<T, HQ>(b0, &Ys[buf][kk][tq * HQ]);
            lds_vec<T, HQ>(b1, &Ys[buf][kk][BQ / 2 + tq * HQ]);
#pragma unroll
            for (int i = 0; i < HP; ++i) { a[i] = a0[i]; a[HP + i] = a1[i]; }
#pragma unroll
            for (int j = 0; j < HQ; ++j) { b[j] = b0[j]; b[HQ + j] = b1[j]; }
            if constexpr (COMP) {
#pragma unroll
                for (int i = 0; i < TP; ++i)
#pragma unroll
                    for (int j = 0; j < TQ; ++j) exact_fma_acc(a[i], b[j], acc[i][j], lo[i][j]);
            } else if constexpr (kPacked) {
                fma_tile_f32x2_rows<TP, TQ>(accp, a, b);
            } else {
#pragma unroll
                for (int i = 0; i < TP; ++i)
#pragma unroll
                    for (int j = 0; j < TQ; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
        }
        if (PROMOTE > 0 && ++chunk == PROMOTE) {
            chunk = 0;
            if constexpr (kPacked) {
#pragma unroll
                for (int i = 0; i < TP / 2; ++i)
#pragma unroll
                    for (int j = 0; j < TQ; ++j) {
                        acc[2 * i][j] = accp[i][j].x;
                        acc[2 * i + 1][j] = accp[i][j].y;
                        accp[i][j] = make_float2(0.f, 0.f);
                    }
            }
#pragma unroll
            for (int i = 0; i < TP; ++i)
#pragma unroll
                for (int j = 0; j < TQ; ++j) {
                    acc2[i][j] += (Acc)acc[i][j];
                    if (COMP) acc2[i][j] += (Acc)lo[i][j];
                    acc[i][j] = T(0);
                    lo[i][j] = T(0);
                }
        }
        if (more) store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
    if constexpr (kPacked) {
#pragma unroll
        for (int i = 0; i < TP / 2; ++i)
#pragma unroll
            for (int j = 0; j < TQ; ++j) {
                acc[2 * i][j] = accp[i][j].x;
                acc[2 * i + 1][j] = accp[i][j].y;
            }
    }

    Acc* out = Out + (int64_t)blockIdx.z * out_zstride;
#pragma unroll
    for (int i = 0; i < TP; ++i) {
        const int p = p0 + ((i < HP) ? (tp * HP + i) : (BP / 2 + tp * HP + (i - HP)));
        if (p >= pn) continue;
#pragma unroll
        for (int j = 0; j < TQ; ++j) {
            const int64_t q = q0 + ((j < HQ) ? (tq * HQ + j) : (BQ / 2 + tq * HQ + (j - HQ)));
            if (q >= qn) continue;
            Acc v = (PROMOTE > 0) ? (acc2[i][j] + (Acc)acc[i][j]) : (Acc)acc[i][j];
            if (COMP) v += (Acc)lo[i][j];
            out[p + q * ldo] = v;
        }
    }
}

}  // namespace rqb

