// rqb_svd.cu -- low-rank SVD from a QB factorization (Sec. 2 "Computing the
// low rank SVD"): the full SVD of the small k x n factor B = U_hat D V_hat^T
// gives A ~ Q B = (Q U_hat) D V_hat^T, truncated to the leading r triplets.
//
// On the GPU: G = B B^T (k x k, FP64 sums of exact products), its symmetric
// eigendecomposition G = W diag(lambda) W^T by cyclic Jacobi in FP64 (one
// kernel per round of disjoint rotations in round-robin order, every pair of
// indices met once per sweep), D = sqrt(lambda) in descending order, U_hat = W,
// U_r = Q W_r and V_r^T = D_r^-1 W_r^T B.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "rqb_engine.h"

namespace rqb {
namespace {

// dst (cols x rows, ld ldd) = src^T (src rows x cols, ld lds); 32 x 32 tiles.
template <typename T>
__global__ void k_transpose(int64_t rows, int64_t cols, const T* __restrict__ src, int64_t lds, T* __restrict__ dst,
                            int64_t ldd) {
    __shared__ T tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int i = ty; i < 32; i += 8) {
        const int64_t r = r0 + tx, c = c0 + i;
        if (r < rows && c < cols) tile[i][tx] = src[r + c * lds];
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        const int64_t c = c0 + tx, r = r0 + i;
        if (r < rows && c < cols) dst[c + r * ldd] = tile[tx][i];
    }
}

// Gp (kk x kk, ld kk) = G (k x k, ld ldg) padded with zeros; W = I.
__global__ void k_jacobi_init(const double* __restrict__ G, int64_t ldg, int k, int kk, double* __restrict__ Gp,
                              double* __restrict__ W) {
    const int64_t total = (int64_t)kk * kk;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % kk), j = (int)(e / kk);
        Gp[e] = (i < k && j < k) ? G[i + (int64_t)j * ldg] : 0.0;
        W[e] = (i == j) ? 1.0 : 0.0;
    }
}

// Round-robin schedule on kk (even) indices: index 0 stays at seat 0, the
// others rotate through seats 1 .. kk-1; round r pairs seat s with seat
// kk-1-s, so the kk-1 rounds of a sweep meet every pair exactly once.
__device__ __forceinline__ int seat_player(int seat, int round, int kk) {
    return seat == 0 ? 0 : (seat - 1 + round) % (kk - 1) + 1;
}
__device__ __forceinline__ void pair_of(int u, int round, int kk, int* p, int* q) {
    const int a = seat_player(u, round, kk), b = seat_player(kk - 1 - u, round, kk);
    *p = a < b ? a : b;
    *q = a < b ? b : a;
}

// Rotation J = [c s; -s c] on (p, q) that zeroes G'_pq of G' = J^T G J
// (the symmetric 2 x 2 Schur decomposition: tau = (g_qq - g_pp) / (2 g_pq),
// t the smaller root of t^2 + 2 tau t - 1 = 0).  Skipped (J = I, returns
// false) when g_pq is below 1e-15 sqrt(|g_pp g_qq|) -- the relative test that
// keeps small eigenvalues of a positive definite G accurate -- or below the
// absolute floor.
__device__ __forceinline__ bool rotation(const double* __restrict__ G, int kk, int p, int q, double floor, double* c,
                                         double* s) {
    const double gpq = G[p + (int64_t)q * kk];
    const double gpp = G[p + (int64_t)p * kk], gqq = G[q + (int64_t)q * kk];
    if (fabs(gpq) <= floor || fabs(gpq) <= 1e-15 * sqrt(fabs(gpp) * fabs(gqq))) {
        *c = 1.0;
        *s = 0.0;
        return false;
    }
    const double tau = (gqq - gpp) / (2.0 * gpq);
    double t;
    if (fabs(tau) > 1e150) t = 0.5 / tau;
    else t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
    const double cc = 1.0 / sqrt(1.0 + t * t);
    *c = cc;
    *s = t * cc;
    return true;
}

// One round: Gout = J^T Gin J (each thread one 2 x 2 block of index pairs
// (u, v)) and W <- W J (each thread one row of one pair); *applied counts
// the rotations of the round that were not skipped.
__global__ void __launch_bounds__(256) k_jacobi_round(const double* __restrict__ Gin, double* __restrict__ Gout,
                                                      double* __restrict__ W, int kk, int round, double floor,
                                                      unsigned int* __restrict__ applied) {
    const int h = kk / 2;
    const int64_t nblk = (int64_t)h * h, total = nblk + (int64_t)kk * h;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        if (e < nblk) {
            const int u = (int)(e % h), v = (int)(e / h);
            int pu, qu, pv, qv;
            pair_of(u, round, kk, &pu, &qu);
            pair_of(v, round, kk, &pv, &qv);
            double cu, su, cv, sv;
            const bool ru = rotation(Gin, kk, pu, qu, floor, &cu, &su);
            rotation(Gin, kk, pv, qv, floor, &cv, &sv);
            if (u == v && ru) atomicAdd(applied, 1u);
            const double x00 = Gin[pu + (int64_t)pv * kk], x10 = Gin[qu + (int64_t)pv * kk];
            const double x01 = Gin[pu + (int64_t)qv * kk], x11 = Gin[qu + (int64_t)qv * kk];
            // Y = X J_v, then Z = J_u^T Y
            const double y00 = cv * x00 - sv * x01, y01 = sv * x00 + cv * x01;
            const double y10 = cv * x10 - sv * x11, y11 = sv * x10 + cv * x11;
            double z00 = cu * y00 - su * y10, z01 = cu * y01 - su * y11;
            double z10 = su * y00 + cu * y10, z11 = su * y01 + cu * y11;
            if (u == v) {
                z01 = 0.0;
                z10 = 0.0;
            }
            Gout[pu + (int64_t)pv * kk] = z00;
            Gout[qu + (int64_t)pv * kk] = z10;
            Gout[pu + (int64_t)qv * kk] = z01;
            Gout[qu + (int64_t)qv * kk] = z11;
        } else {
            const int64_t f = e - nblk;
            const int i = (int)(f % kk), v = (int)(f / kk);
            int pv, qv;
            pair_of(v, round, kk, &pv, &qv);
            double cv, sv;
            rotation(Gin, kk, pv, qv, floor, &cv, &sv);
            const double wp = W[i + (int64_t)pv * kk], wq = W[i + (int64_t)qv * kk];
            W[i + (int64_t)pv * kk] = cv * wp - sv * wq;
            W[i + (int64_t)qv * kk] = sv * wp + cv * wq;
        }
    }
}

// part[2 b] = sum of squares of the off-diagonal entries, part[2 b + 1] = of
// the diagonal ones, over the columns of CTA b; then summed in CTA order.
__global__ void __launch_bounds__(256) k_offdiag(const double* __restrict__ G, int kk, double* __restrict__ part) {
    __shared__ double so[8], sd[8];
    double off = 0.0, dia = 0.0;
    for (int j = blockIdx.x; j < kk; j += gridDim.x)
        for (int i = threadIdx.x; i < kk; i += blockDim.x) {
            const double g = G[i + (int64_t)j * kk];
            if (i == j) dia += g * g;
            else off += g * g;
        }
    for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_xor_sync(0xffffffffu, off, o);
        dia += __shfl_xor_sync(0xffffffffu, dia, o);
    }
    if ((threadIdx.x & 31) == 0) { so[threadIdx.x >> 5] = off; sd[threadIdx.x >> 5] = dia; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, d = 0.0;
        for (int w = 0; w < 8; ++w) { a += so[w]; d += sd[w]; }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = d;
    }
}

__global__ void k_offdiag_sum(const double* __restrict__ part, int count, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double a = 0.0, d = 0.0;
        for (int b = 0; b < count; ++b) { a += part[2 * b]; d += part[2 * b + 1]; }
        out[0] = a;
        out[1] = d;
    }
}

__global__ void k_diag(const double* __restrict__ G, int kk, double* __restrict__ d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kk) d[i] = G[i + (int64_t)i * kk];
}

// Wr (k x r, ld k, type T) = columns perm[0 .. r) of W (kk x kk), first k rows.
template <typename T>
__global__ void k_gather_cols(const double* __restrict__ W, int kk, int k, const int* __restrict__ perm, int r,
                              T* __restrict__ Wr) {
    const int64_t total = (int64_t)k * r;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % k), c = (int)(e / k);
        Wr[e] = (T)W[i + (int64_t)perm[c] * kk];
    }
}

// Vt (r x n, ld ldv) = diag(1 / sigma) Vt; rows with sigma = 0 become zero.
template <typename T>
__global__ void k_scale_rows(T* __restrict__ Vt, int64_t ldv, int r, int64_t n, const double* __restrict__ sigma) {
    const int64_t total = (int64_t)r * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % r);
        const int64_t j = e / r;
        const double s = sigma[i];
        Vt[i + j * ldv] = s > 0.0 ? (T)((double)Vt[i + j * ldv] / s) : T(0);
    }
}

int grid_for(int64_t work, int sms) { return (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 8LL * sms)); }

}  // namespace

size_t svd_scratch_bytes(int64_t m, int64_t n, int k, int r) {
    const int64_t kk = k + (k & 1);
    const size_t g = sizeof(double) * (size_t)kk * kk;
    const size_t gram_part = sizeof(double) * (size_t)k * k * 8;
    const size_t part = (size_t)8 * (size_t)r * n;     // T partials of V^T (at most 8 bytes each)
    return 3 * g + gram_part + part + (size_t)8 * n * k + (size_t)8 * k * r + sizeof(double) * (kk + 2 + 2 * 1024) +
           sizeof(int) * (size_t)kk + sizeof(double) * (size_t)r + 16 * 256;
}

template <typename T>
int svd_lowrank(Ctx& cx, int64_t m, int64_t n, int k, int r, const T* Q, int64_t ldq, const T* B, int64_t ldb,
                T* U, int64_t ldu, double* S_host, T* Vt, int64_t ldvt, void* scratch, size_t scratch_bytes,
                int* sweeps_out) {
    if (k < 1 || r < 1 || r > k) return RQB_ERR_INVALID;
    if (scratch_bytes < svd_scratch_bytes(m, n, k, r)) return RQB_ERR_INVALID;
    const int kk = k + (k & 1);
    char* p = static_cast<char*>(scratch);
    auto take = [&](size_t bytes) { char* o = p; p += (bytes + 255) & ~(size_t)255; return o; };
    double* G = reinterpret_cast<double*>(take(sizeof(double) * (size_t)kk * kk));
    double* G0 = reinterpret_cast<double*>(take(sizeof(double) * (size_t)kk * kk));
    double* G1 = reinterpret_cast<double*>(take(sizeof(double) * (size_t)kk * kk));
    double* W = G;   // the unpadded Gram is no longer needed once padded into G0
    double* gpart = reinterpret_cast<double*>(take(sizeof(double) * (size_t)k * k * 8));
    T* part = reinterpret_cast<T*>(take((size_t)8 * (size_t)r * n));
    T* Bt = reinterpret_cast<T*>(take((size_t)8 * n * k));
    T* Wr = reinterpret_cast<T*>(take((size_t)8 * k * r));
    double* dvals = reinterpret_cast<double*>(take(sizeof(double) * (kk + 2)));
    double* opart = reinterpret_cast<double*>(take(sizeof(double) * 2 * 1024));
    int* perm = reinterpret_cast<int*>(take(sizeof(int) * (size_t)kk));
    unsigned int* applied = reinterpret_cast<unsigned int*>(take(sizeof(unsigned int) * 2));
    double* sig = reinterpret_cast<double*>(take(sizeof(double) * (size_t)r));
    cudaError_t e;
#define SVD_CK(call)                                  \
    do {                                              \
        if ((e = (call)) != cudaSuccess) {            \
            cudaGetLastError();                       \
            return e == cudaErrorMemoryAllocation ? RQB_ERR_OOM : RQB_ERR_CUDA; \
        }                                             \
    } while (0)

    // G = B B^T = (B^T)^T B^T with exact products and FP64 sums
    {
        dim3 grid((unsigned)((k + 31) / 32), (unsigned)((n + 31) / 32));
        k_transpose<T><<<grid, 256, 0, cx.stream>>>(k, n, B, ldb, Bt, n);
        cx.launches++;
        SVD_CK(cudaGetLastError());
        SVD_CK(gemm_tn_f64acc<T>(cx, n, k, k, Bt, n, Bt, n, G, k, gpart, (size_t)k * k * 8, true, true));
    }
    k_jacobi_init<<<grid_for((int64_t)kk * kk, cx.num_sms), 256, 0, cx.stream>>>(G, k, k, kk, G0, G1);
    cx.launches++;
    SVD_CK(cudaGetLastError());
    // W lives in G's storage from here on (G1 holds the identity written by init)
    SVD_CK(cudaMemcpyAsync(W, G1, sizeof(double) * (size_t)kk * kk, cudaMemcpyDeviceToDevice, cx.stream));

    // scale of G for the absolute rotation floor: ||diag(G)||_2
    const int ogrid = std::min(kk, 1024);
    double host_od[2] = {0.0, 0.0};
    k_offdiag<<<ogrid, 256, 0, cx.stream>>>(G0, kk, opart);
    k_offdiag_sum<<<1, 32, 0, cx.stream>>>(opart, ogrid, dvals);
    cx.launches += 2;
    SVD_CK(cudaMemcpyAsync(host_od, dvals, 2 * sizeof(double), cudaMemcpyDeviceToHost, cx.stream));
    SVD_CK(cudaStreamSynchronize(cx.stream));
    if (!std::isfinite(host_od[0]) || !std::isfinite(host_od[1])) return RQB_ERR_NONFINITE;
    const double floor = 1e-18 * std::sqrt(host_od[1]);

    // cyclic Jacobi: two sweeps (an even number of rounds) per check, so the
    // current matrix is back in G0 at every check; converged once a sweep
    // applies no rotation
    const int rounds = kk - 1;
    const int64_t work = (int64_t)(kk / 2) * (kk / 2) + (int64_t)kk * (kk / 2);
    const int rgrid = grid_for(work, cx.num_sms);
    int sweeps = 0;
    unsigned int host_applied[2] = {1u, 1u};
    for (; sweeps < 60 && kk > 1;) {
        SVD_CK(cudaMemsetAsync(applied, 0, 2 * sizeof(unsigned int), cx.stream));
        for (int s2 = 0; s2 < 2; ++s2)
            for (int rd = 0; rd < rounds; ++rd) {
                const int q = s2 * rounds + rd;
                const double* gin = (q & 1) ? G1 : G0;
                double* gout = (q & 1) ? G0 : G1;
                k_jacobi_round<<<rgrid, 256, 0, cx.stream>>>(gin, gout, W, kk, rd, floor, applied + s2);
                cx.launches++;
            }
        SVD_CK(cudaGetLastError());
        sweeps += 2;
        SVD_CK(cudaMemcpyAsync(host_applied, applied, 2 * sizeof(unsigned int), cudaMemcpyDeviceToHost, cx.stream));
        SVD_CK(cudaStreamSynchronize(cx.stream));
        if (host_applied[0] == 0 || host_applied[1] == 0) break;
    }
    if (sweeps_out) *sweeps_out = sweeps;

    // eigenvalues, descending; the padding index (k when k is odd) is left out
    std::vector<double> lam(kk);
    k_diag<<<(kk + 255) / 256, 256, 0, cx.stream>>>(G0, kk, dvals);
    cx.launches++;
    SVD_CK(cudaMemcpyAsync(lam.data(), dvals, sizeof(double) * kk, cudaMemcpyDeviceToHost, cx.stream));
    SVD_CK(cudaStreamSynchronize(cx.stream));
    std::vector<int> order(k);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lam[a] > lam[b]; });
    std::vector<double> s(r);
    for (int i = 0; i < r; ++i) s[i] = std::sqrt(std::max(lam[order[i]], 0.0));
    SVD_CK(cudaMemcpyAsync(perm, order.data(), sizeof(int) * r, cudaMemcpyHostToDevice, cx.stream));
    SVD_CK(cudaMemcpyAsync(sig, s.data(), sizeof(double) * r, cudaMemcpyHostToDevice, cx.stream));
    k_gather_cols<T><<<grid_for((int64_t)k * r, cx.num_sms), 256, 0, cx.stream>>>(W, kk, k, perm, r, Wr);
    cx.launches++;
    SVD_CK(cudaGetLastError());

    // U_r = Q W_r
    {
        NNArgs<T> a;
        a.m = m; a.K = k; a.nc = r; a.nout = r;
        a.X = Q; a.ldx = ldq;
        a.C = Wr; a.csk = 1; a.csj = k; a.c_rowmajor = false;
        a.Out = U; a.ldo = ldu;
        SVD_CK(gemm_nn<T>(cx, a));
    }
    // V_r^T = D_r^-1 W_r^T B
    SVD_CK(gemm_tn<T>(cx, k, r, n, Wr, k, B, ldb, Vt, ldvt, part, (size_t)r * n, nullptr, 0, nullptr));
    k_scale_rows<T><<<grid_for((int64_t)r * n, cx.num_sms), 256, 0, cx.stream>>>(Vt, ldvt, r, n, sig);
    cx.launches++;
    SVD_CK(cudaGetLastError());
    SVD_CK(cudaStreamSynchronize(cx.stream));
    for (int i = 0; i < r; ++i) S_host[i] = s[i];
#undef SVD_CK
    return RQB_OK;
}

template int svd_lowrank<float>(Ctx&, int64_t, int64_t, int, int, const float*, int64_t, const float*, int64_t,
                                float*, int64_t, double*, float*, int64_t, void*, size_t, int*);
template int svd_lowrank<double>(Ctx&, int64_t, int64_t, int, int, const double*, int64_t, const double*, int64_t,
                                 double*, int64_t, double*, double*, int64_t, void*, size_t, int*);

}  // namespace rqb
