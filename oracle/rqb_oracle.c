/*
 * rqb_oracle.c -- CPU FP64 oracle for blocked randomized QB (randQB_b).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this library.  It shares nothing with the CUDA
 * library and is never called by it.
 *
 * Every routine is written to be checked against the paper by eye:
 *   - matrix products are plain sums over the contraction index, in increasing
 *     index order, one output element per sum (OpenMP only splits the set of
 *     output columns between threads, which does not change any sum);
 *   - orth() is an unpivoted Householder QR (Sec. 2.4), sign-normalised so that
 *     diag(R) >= 0;
 *   - randQB_b follows Fig. randQB_b lines (1)-(8) in order; randQB_pb follows
 *     Fig. randQB_pb lines (1)-(13).
 * Compile with -ffp-contract=off so that no multiply-add is fused.
 */
#include "rqb_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11).  One round maps (x0, x1, x2, x3) with key (k0, k1) to
 * (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0)); between
 * rounds the key is advanced by the Weyl increments (W0, W1).                */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += ORC_PHILOX_W0;
            k1 += ORC_PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Entry (r, c) of the Gaussian matrix: the Philox block with counter
 * (r, c/2, stream, 0) and key (seed low word, seed high word) gives two
 * uniforms u1, u2 in (0, 1); Box-Muller turns them into the pair
 * sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2), of which column c takes the first
 * entry when c is even and the second when c is odd. */
/* Round x to 11 significant bits (the TF32 format: 10 fraction bits), to
 * nearest with ties away from zero: with x = f 2^e, 1/2 <= |f| < 1, the
 * result is round(f 2^11) 2^(e - 11).  Exact in binary64. */
double orc_round_tf32(double x) {
    if (x == 0.0 || !isfinite(x)) return x;
    int e;
    double f = frexp(x, &e);
    double s = ldexp(fabs(f), 11);
    double r = floor(s + 0.5);
    return ldexp(f < 0 ? -r : r, e - 11);
}

/* Round x to 8 significant bits (the BF16 format: 7 fraction bits), to
 * nearest with ties to even: with x = f 2^e, 1/2 <= |f| < 1, the result is
 * rint(f 2^8) 2^(e - 8) (rint rounds half to even).  Exact in binary64. */
double orc_round_bf16(double x) {
    if (x == 0.0 || !isfinite(x)) return x;
    int e;
    double f = frexp(x, &e);
    double r = rint(ldexp(fabs(f), 8));
    return ldexp(f < 0 ? -r : r, e - 8);
}

/* y[i] = orc_round_bf16(x[i]) for i < count (x and y may alias). */
void orc_round_bf16_n(const double* x, double* y, int64_t count) {
    for (int64_t i = 0; i < count; ++i) y[i] = orc_round_bf16(x[i]);
}

static double orc_omega_entry(uint64_t seed, uint32_t stream, int64_t r, int64_t c, int prec) {
    const double PI = 3.14159265358979323846;
    uint32_t ctr[4] = {(uint32_t)r, (uint32_t)(c >> 1), stream, 0u};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    if (prec == 32 || prec == 19 || prec == 8) {
        /* binary32 evaluation: 23-bit uniforms (j + 1/2) 2^-23, exact in float;
         * prec 19 then rounds the binary32 value to TF32, prec 8 to BF16 */
        float u1 = ((float)(x[0] >> 9) + 0.5f) * 0x1p-23f;
        float u2 = ((float)(x[2] >> 9) + 0.5f) * 0x1p-23f;
        double rad = sqrt(-2.0 * log((double)u1));
        double ang = 2.0 * PI * (double)u2;
        double z = (c & 1) ? rad * sin(ang) : rad * cos(ang);
        if (prec == 19) return orc_round_tf32((double)(float)z);
        if (prec == 8) return orc_round_bf16((double)(float)z);
        return (double)(float)z;
    }
    /* binary64: 53-bit uniforms ((x0 >> 5) 2^26 + (x1 >> 6) + 1/2) 2^-53 */
    double u1 = ((double)(x[0] >> 5) * 67108864.0 + (double)(x[1] >> 6) + 0.5) * 0x1p-53;
    double u2 = ((double)(x[2] >> 5) * 67108864.0 + (double)(x[3] >> 6) + 0.5) * 0x1p-53;
    double rad = sqrt(-2.0 * log(u1));
    double ang = 2.0 * PI * u2;
    return (c & 1) ? rad * sin(ang) : rad * cos(ang);
}

void orc_omega(uint64_t seed, uint32_t stream, int64_t n, int64_t col0,
               int64_t ncols, int prec, double* out, int64_t ldo) {
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < ncols; ++c)
        for (int64_t r = 0; r < n; ++r)
            out[r + c * ldo] = orc_omega_entry(seed, stream, r, col0 + c, prec);
}

/* ------------------------------------------------------------------------ */
/* Plain dense products (column-major).                                      */

/* Z (m x p) = X (m x q) * Y (q x p) */
static void mm_nn(int64_t m, int64_t p, int64_t q, const double* X, int64_t ldx,
                  const double* Y, int64_t ldy, double* Z, int64_t ldz) {
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < p; ++c) {
        double* z = Z + c * ldz;
        for (int64_t r = 0; r < m; ++r) z[r] = 0.0;
        for (int64_t t = 0; t < q; ++t) {
            const double y = Y[t + c * ldy];
            const double* x = X + t * ldx;
            for (int64_t r = 0; r < m; ++r) z[r] += x[r] * y;
        }
    }
}

/* Z (p x q) = X^T Y with X m x p and Y m x q */
static void mm_tn(int64_t m, int64_t p, int64_t q, const double* X, int64_t ldx,
                  const double* Y, int64_t ldy, double* Z, int64_t ldz) {
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < q; ++c) {
        const double* y = Y + c * ldy;
        for (int64_t i = 0; i < p; ++i) {
            const double* x = X + i * ldx;
            double s = 0.0;
            for (int64_t r = 0; r < m; ++r) s += x[r] * y[r];
            Z[i + c * ldz] = s;
        }
    }
}

/* Sum of squares of an m x n matrix, columns in order, rows in order. */
static double frob2(int64_t m, int64_t n, const double* X, int64_t ldx) {
    double s = 0.0;
    for (int64_t c = 0; c < n; ++c)
        for (int64_t r = 0; r < m; ++r) s += X[r + c * ldx] * X[r + c * ldx];
    return s;
}

/* ------------------------------------------------------------------------ */
/* orth(): unpivoted Householder QR, thin Q, diag(R) >= 0 (Sec. 2.4).         */
void orc_orth(const double* Y, int64_t m, int64_t p, int64_t ldy,
              double* Q, int64_t ldq, double* R, int64_t ldr) {
    double* Wk = (double*)malloc(sizeof(double) * (size_t)m * (size_t)p);
    double* V = (double*)calloc((size_t)m * (size_t)p, sizeof(double));
    double* tau = (double*)calloc((size_t)p, sizeof(double));
    double* Rl = (double*)calloc((size_t)p * (size_t)p, sizeof(double));
    for (int64_t c = 0; c < p; ++c)
        for (int64_t r = 0; r < m; ++r) Wk[r + c * m] = Y[r + c * ldy];

    /* Reduce to upper-triangular form: reflector j maps Wk[j:, j] to alpha e_j. */
    for (int64_t j = 0; j < p; ++j) {
        double* x = Wk + j + j * m;
        int64_t len = m - j;
        double nx = 0.0;
        for (int64_t r = 0; r < len; ++r) nx += x[r] * x[r];
        nx = sqrt(nx);
        double* v = V + j + j * m;
        if (nx == 0.0) {        /* zero column: no reflection, R_jj = 0 */
            tau[j] = 0.0;
            continue;
        }
        double alpha = (x[0] >= 0.0) ? -nx : nx;  /* avoids cancellation in v0 */
        for (int64_t r = 0; r < len; ++r) v[r] = x[r];
        v[0] = x[0] - alpha;
        double vv = 0.0;
        for (int64_t r = 0; r < len; ++r) vv += v[r] * v[r];
        tau[j] = 2.0 / vv;
        for (int64_t c = j; c < p; ++c) {
            double* w = Wk + j + c * m;
            double s = 0.0;
            for (int64_t r = 0; r < len; ++r) s += v[r] * w[r];
            s *= tau[j];
            for (int64_t r = 0; r < len; ++r) w[r] -= s * v[r];
        }
    }
    for (int64_t c = 0; c < p; ++c)
        for (int64_t r = 0; r <= c; ++r) Rl[r + c * p] = Wk[r + c * m];

    /* Q = H_0 H_1 ... H_{p-1} [I_p; 0], applied from the last reflector back. */
    for (int64_t c = 0; c < p; ++c) {
        for (int64_t r = 0; r < m; ++r) Q[r + c * ldq] = 0.0;
        Q[c + c * ldq] = 1.0;
    }
    for (int64_t j = p - 1; j >= 0; --j) {
        if (tau[j] == 0.0) continue;
        const double* v = V + j + j * m;
        int64_t len = m - j;
        for (int64_t c = 0; c < p; ++c) {
            double* q = Q + j + c * ldq;
            double s = 0.0;
            for (int64_t r = 0; r < len; ++r) s += v[r] * q[r];
            s *= tau[j];
            for (int64_t r = 0; r < len; ++r) q[r] -= s * v[r];
        }
    }
    /* Sign convention: flip column j of Q and row j of R where R_jj < 0. */
    for (int64_t j = 0; j < p; ++j) {
        if (Rl[j + j * p] < 0.0) {
            for (int64_t r = 0; r < m; ++r) Q[r + j * ldq] = -Q[r + j * ldq];
            for (int64_t c = j; c < p; ++c) Rl[j + c * p] = -Rl[j + c * p];
        }
    }
    if (R) {
        for (int64_t c = 0; c < p; ++c)
            for (int64_t r = 0; r < p; ++r) R[r + c * ldr] = Rl[r + c * p];
    }
    free(Wk); free(V); free(tau); free(Rl);
}

/* ------------------------------------------------------------------------ */
void orc_sketch(const double* A, int64_t m, int64_t n, int64_t lda,
                uint64_t seed, int64_t col0, int64_t p, int omega_prec,
                double* Y, int64_t ldy) {
    double* Om = (double*)malloc(sizeof(double) * (size_t)n * (size_t)p);
    orc_omega(seed, 0u, n, col0, p, omega_prec, Om, n);
    mm_nn(m, p, n, A, lda, Om, n, Y, ldy);
    free(Om);
}

/* Lines (3') of Fig. randQB_b applied to an already orthonormalised Q_i:
 * Q_i <- orth(Q_i - Qbar (Qbar^T Q_i)). */
static void reproject_orth(double* Qi, int64_t m, int64_t p,
                           const double* Qbar, int64_t kprev, int64_t ldqb) {
    if (kprev > 0) {
        double* C = (double*)malloc(sizeof(double) * (size_t)kprev * (size_t)p);
        double* P = (double*)malloc(sizeof(double) * (size_t)m * (size_t)p);
        mm_tn(m, kprev, p, Qbar, ldqb, Qi, m, C, kprev);   /* C = Qbar^T Q_i  */
        mm_nn(m, p, kprev, Qbar, ldqb, C, kprev, P, m);    /* P = Qbar C      */
        for (int64_t c = 0; c < p; ++c)
            for (int64_t r = 0; r < m; ++r) Qi[r + c * m] -= P[r + c * m];
        free(C); free(P);
    }
    double* T = (double*)malloc(sizeof(double) * (size_t)m * (size_t)p);
    orc_orth(Qi, m, p, m, T, m, NULL, 0);
    memcpy(Qi, T, sizeof(double) * (size_t)m * (size_t)p);
    free(T);
}

void orc_orth_reproject(const double* Y, int64_t m, int64_t p, int64_t ldy,
                        const double* Qbar, int64_t kprev, int64_t ldqb,
                        double* Qi, int64_t ldqi) {
    double* T = (double*)malloc(sizeof(double) * (size_t)m * (size_t)p);
    orc_orth(Y, m, p, ldy, T, m, NULL, 0);                 /* line (3)  */
    reproject_orth(T, m, p, Qbar, kprev, ldqb);             /* line (3') */
    for (int64_t c = 0; c < p; ++c)
        for (int64_t r = 0; r < m; ++r) Qi[r + c * ldqi] = T[r + c * m];
    free(T);
}

/* ------------------------------------------------------------------------ */
int orc_randqb_b(const double* A, int64_t m, int64_t n, int64_t lda,
                 double eps, int64_t b, uint64_t seed, int64_t max_rank,
                 int fixed_rank, int power, int skip_inner_orth, int omega_prec,
                 double* Q, int64_t ldq, double* B, int64_t ldb,
                 orc_qb_result* res) {
    return orc_randqb_b_store(A, m, n, lda, eps, b, seed, max_rank, fixed_rank, power, skip_inner_orth,
                              omega_prec, 64, Q, ldq, B, ldb, res);
}

int orc_randqb_b_store(const double* A, int64_t m, int64_t n, int64_t lda,
                       double eps, int64_t b, uint64_t seed, int64_t max_rank,
                       int fixed_rank, int power, int skip_inner_orth, int omega_prec,
                       int storage_prec, double* Q, int64_t ldq, double* B, int64_t ldb,
                       orc_qb_result* res) {
    if (m <= 0 || n <= 0 || b <= 0 || lda < m || eps < 0.0 || power < 0 || !res) return -1;
    if (storage_prec != 64 && storage_prec != 16) return -1;
    const int64_t rmax = (m < n) ? m : n;
    int64_t kcap = (max_rank <= 0 || max_rank > rmax) ? rmax : max_rank;
    if (ldq < m || ldb < kcap) return -1;

    /* A^(0) = A (eq. def0); the working copy W is downdated in place. */
    double* W = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n);
    for (int64_t c = 0; c < n; ++c)
        for (int64_t r = 0; r < m; ++r) W[r + c * m] = A[r + c * lda];
    const double normA2 = frob2(m, n, W, m);
    double E = normA2;
    const double eps2 = eps * eps;
    /* ||A||_F <= eps already (e.g. A = 0): the empty factorization, k = 0,
     * meets the tolerance of Sec. 1.1; the figure's first panel would be the
     * orthonormalisation of a zero (or negligible) sketch. */
    if (!fixed_rank && normA2 <= eps2) {
        res->k = 0;
        res->blocks = 0;
        res->normA2 = normA2;
        res->status = 0;
        free(W);
        return 0;
    }

    double* Om = (double*)malloc(sizeof(double) * (size_t)n * (size_t)b);
    double* Y = (double*)malloc(sizeof(double) * (size_t)m * (size_t)b);
    double* Qi = (double*)malloc(sizeof(double) * (size_t)m * (size_t)b);
    double* Z = (double*)malloc(sizeof(double) * (size_t)n * (size_t)b);
    double* Zq = (double*)malloc(sizeof(double) * (size_t)n * (size_t)b);
    double* Bi = (double*)malloc(sizeof(double) * (size_t)b * (size_t)n);

    int64_t k = 0, blocks = 0;
    int converged = 0;
    while (k < kcap) {
        /* Last block is shrunk so that k never exceeds the cap. */
        const int64_t bi = (kcap - k < b) ? (kcap - k) : b;
        /* (2) Omega_i = randn(n, b): global columns k .. k + bi - 1. */
        orc_omega(seed, 0u, n, k, bi, omega_prec, Om, n);
        /* (3) Q_i = orth(A Omega_i), with A the current (downdated) matrix. */
        mm_nn(m, bi, n, W, m, Om, n, Y, m);
        if (power > 0 && skip_inner_orth) {
            /* Sec. 5.4 variant: Y = A (A^* Y) repeated P times, then one orth. */
            for (int pw = 0; pw < power; ++pw) {
                mm_tn(m, n, bi, W, m, Y, m, Z, n);
                mm_nn(m, bi, n, W, m, Z, n, Y, m);
            }
            orc_orth(Y, m, bi, m, Qi, m, NULL, 0);
        } else {
            orc_orth(Y, m, bi, m, Qi, m, NULL, 0);
            /* Fig. randQB_pb lines (4)-(7): Q_i = orth(A^* Q_i); Q_i = orth(A Q_i). */
            for (int pw = 0; pw < power; ++pw) {
                mm_tn(m, n, bi, W, m, Qi, m, Z, n);
                orc_orth(Z, n, bi, n, Zq, n, NULL, 0);
                mm_nn(m, bi, n, W, m, Zq, n, Y, m);
                orc_orth(Y, m, bi, m, Qi, m, NULL, 0);
            }
        }
        /* (3') Q_i = orth(Q_i - sum_j Q_j Q_j^* Q_i) against the stored blocks. */
        reproject_orth(Qi, m, bi, Q, k, ldq);
        /* (4) B_i = Q_i^* A. */
        mm_tn(m, bi, n, Qi, m, W, m, Bi, bi);
        /* Stopping quantity E_i = ||A||^2 - sum_j ||B_j||^2 (Sec. 4.2 with
         * Prop. 4.1(b)). */
        E -= frob2(bi, n, Bi, bi);
        /* (5) A = A - Q_i B_i. */
#pragma omp parallel for schedule(static)
        for (int64_t c = 0; c < n; ++c) {
            for (int64_t r = 0; r < m; ++r) {
                double s = 0.0;
                for (int64_t t = 0; t < bi; ++t) s += Qi[r + t * m] * Bi[t + c * bi];
                W[r + c * m] -= s;
            }
        }
        /* a residual stored in BF16 is rounded after every downdate */
        if (storage_prec == 16) {
#pragma omp parallel for schedule(static)
            for (int64_t c = 0; c < n; ++c)
                for (int64_t r = 0; r < m; ++r) W[r + c * m] = orc_round_bf16(W[r + c * m]);
        }
        /* (8) Q = [Q_1 ... Q_i], B = [B_1; ...; B_i]. */
        for (int64_t c = 0; c < bi; ++c)
            for (int64_t r = 0; r < m; ++r) Q[r + (k + c) * ldq] = Qi[r + c * m];
        for (int64_t c = 0; c < n; ++c)
            for (int64_t r = 0; r < bi; ++r) B[k + r + c * ldb] = Bi[r + c * bi];
        const double Dcur = frob2(m, n, W, m);
        if (blocks < res->max_blocks) {
            if (res->E) res->E[blocks] = E;
            if (res->D) res->D[blocks] = Dcur;
        }
        k += bi;
        blocks += 1;
        /* (6) stop once the residual norm is within tolerance: E_i (exact
         * arithmetic: E_i = ||A^(i)||^2); a rounded residual no longer follows
         * E_i, so the stored residual's own norm decides. */
        if (!fixed_rank && ((storage_prec == 64) ? E : Dcur) <= eps2) {
            converged = 1;
            break;
        }
    }
    res->k = k;
    res->blocks = blocks;
    res->normA2 = normA2;
    res->status = (fixed_rank || converged) ? 0 : 1;
    free(W); free(Om); free(Y); free(Qi); free(Z); free(Zq); free(Bi);
    return 0;
}

/* ------------------------------------------------------------------------ */
int orc_randqb(const double* A, int64_t m, int64_t n, int64_t lda, int64_t l,
               uint64_t seed, int omega_prec, double* Q, int64_t ldq,
               double* B, int64_t ldb) {
    if (m <= 0 || n <= 0 || l <= 0 || l > m || lda < m || ldq < m || ldb < l) return -1;
    double* Om = (double*)malloc(sizeof(double) * (size_t)n * (size_t)l);
    double* Y = (double*)malloc(sizeof(double) * (size_t)m * (size_t)l);
    orc_omega(seed, 0u, n, 0, l, omega_prec, Om, n);        /* (1) */
    mm_nn(m, l, n, A, lda, Om, n, Y, m);
    orc_orth(Y, m, l, m, Q, ldq, NULL, 0);                   /* (2) */
    mm_tn(m, l, n, Q, ldq, A, lda, B, ldb);                  /* (3) */
    free(Om); free(Y);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One-sided Jacobi: rotate column pairs of a working copy until all pairs are
 * orthogonal; the column norms are then the singular values.               */
int orc_svd_values(const double* A, int64_t m, int64_t n, int64_t lda, double* sigma) {
    int transpose = (m < n);
    int64_t rows = transpose ? n : m, cols = transpose ? m : n;
    double* U = (double*)malloc(sizeof(double) * (size_t)rows * (size_t)cols);
    for (int64_t c = 0; c < cols; ++c)
        for (int64_t r = 0; r < rows; ++r)
            U[r + c * rows] = transpose ? A[c + r * lda] : A[r + c * lda];
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int64_t i = 0; i < cols - 1; ++i) {
            for (int64_t j = i + 1; j < cols; ++j) {
                double* ui = U + i * rows;
                double* uj = U + j * rows;
                double a = 0.0, bb = 0.0, g = 0.0;
                for (int64_t r = 0; r < rows; ++r) {
                    a += ui[r] * ui[r];
                    bb += uj[r] * uj[r];
                    g += ui[r] * uj[r];
                }
                if (g == 0.0) continue;
                double rel = fabs(g) / sqrt(a * bb);
                if (rel > off) off = rel;
                if (rel < 1e-15) continue;
                double zeta = (bb - a) / (2.0 * g);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                for (int64_t r = 0; r < rows; ++r) {
                    double x = ui[r], y = uj[r];
                    ui[r] = cs * x - sn * y;
                    uj[r] = sn * x + cs * y;
                }
            }
        }
        if (off < 1e-15) break;
    }
    for (int64_t c = 0; c < cols; ++c) {
        double s = 0.0;
        for (int64_t r = 0; r < rows; ++r) s += U[r + c * rows] * U[r + c * rows];
        sigma[c] = sqrt(s);
    }
    /* insertion sort, decreasing */
    for (int64_t i = 1; i < cols; ++i) {
        double v = sigma[i];
        int64_t j = i - 1;
        while (j >= 0 && sigma[j] < v) { sigma[j + 1] = sigma[j]; --j; }
        sigma[j + 1] = v;
    }
    free(U);
    return 0;
}

/* Low-rank SVD from Q (m x k) and B (k x n) (Sec. 2, computing the low rank
 * SVD): the full SVD B = Uh D Vh^T, then U_r = Q Uh(:, 1:r), S = D(1:r) and
 * Vt = Vh(:, 1:r)^T.  B's SVD by one-sided (Hestenes) Jacobi on X = B^T
 * (n x k): column rotations X J make the columns of X orthogonal, so
 * B^T = (X J) J^T, sigma_i = ||(X J)_i||, Vh_i = (X J)_i / sigma_i and Uh = J.
 * Needs k <= n.  S in decreasing order; a zero sigma gives a zero Vt row. */
int orc_rsvd(const double* Q, int64_t m, int64_t k, int64_t ldq, const double* B, int64_t n, int64_t ldb,
             int64_t r, double* U, int64_t ldu, double* S, double* Vt, int64_t ldvt) {
    if (k < 1 || r < 1 || r > k || k > n || ldq < m || ldb < k || ldu < m || ldvt < r) return -1;
    double* X = (double*)malloc(sizeof(double) * (size_t)n * (size_t)k);
    double* J = (double*)malloc(sizeof(double) * (size_t)k * (size_t)k);
    double* sig = (double*)malloc(sizeof(double) * (size_t)k);
    int64_t* ord = (int64_t*)malloc(sizeof(int64_t) * (size_t)k);
    for (int64_t c = 0; c < k; ++c)
        for (int64_t j = 0; j < n; ++j) X[j + c * n] = B[c + j * ldb];
    for (int64_t c = 0; c < k; ++c)
        for (int64_t i = 0; i < k; ++i) J[i + c * k] = (i == c) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int64_t i = 0; i < k - 1; ++i) {
            for (int64_t j = i + 1; j < k; ++j) {
                double* xi = X + i * n;
                double* xj = X + j * n;
                double a = 0.0, bb = 0.0, g = 0.0;
                for (int64_t t = 0; t < n; ++t) {
                    a += xi[t] * xi[t];
                    bb += xj[t] * xj[t];
                    g += xi[t] * xj[t];
                }
                if (g == 0.0) continue;
                double rel = fabs(g) / sqrt(a * bb);
                if (rel > off) off = rel;
                if (rel < 1e-15) continue;
                double zeta = (bb - a) / (2.0 * g);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                for (int64_t q = 0; q < n; ++q) {
                    double x = xi[q], y = xj[q];
                    xi[q] = cs * x - sn * y;
                    xj[q] = sn * x + cs * y;
                }
                double* ji = J + i * k;
                double* jj = J + j * k;
                for (int64_t q = 0; q < k; ++q) {
                    double x = ji[q], y = jj[q];
                    ji[q] = cs * x - sn * y;
                    jj[q] = sn * x + cs * y;
                }
            }
        }
        if (off < 1e-15) break;
    }
    for (int64_t c = 0; c < k; ++c) {
        double s2 = 0.0;
        for (int64_t t = 0; t < n; ++t) s2 += X[t + c * n] * X[t + c * n];
        sig[c] = sqrt(s2);
        ord[c] = c;
    }
    /* insertion sort of the indices by decreasing sigma (stable) */
    for (int64_t i = 1; i < k; ++i) {
        int64_t v = ord[i];
        int64_t j = i - 1;
        while (j >= 0 && sig[ord[j]] < sig[v]) { ord[j + 1] = ord[j]; --j; }
        ord[j + 1] = v;
    }
    for (int64_t c = 0; c < r; ++c) {
        const int64_t o = ord[c];
        S[c] = sig[o];
        for (int64_t i = 0; i < m; ++i) {
            double acc = 0.0;
            for (int64_t t = 0; t < k; ++t) acc += Q[i + t * ldq] * J[t + o * k];
            U[i + c * ldu] = acc;
        }
        for (int64_t j = 0; j < n; ++j) Vt[c + j * ldvt] = sig[o] > 0.0 ? X[j + o * n] / sig[o] : 0.0;
    }
    free(X); free(J); free(sig); free(ord);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Derivative of the fixed-rank map A -> X = Q Q^T A, Q = orth(A Omega) with
 * Omega (n x k, the first k global columns) held fixed.  Q Q^T is the
 * orthogonal projector P onto R(Y), Y = A Omega, whatever the blocking
 * (Sec. 4.1, Prop. 4.1(c)).  Differentiating P = Y (Y^T Y)^{-1} Y^T gives
 *   dL/dA = P G + (I - P)(G A^T + A G^T) Y^{+T} Omega^T,
 * and with Y = Q R, R = Q^T A Omega = B Omega, Y^{+T} = Q R^{-T}, A^T Q = B^T:
 *   dL/dA = Q (Q^T G) + (I - Q Q^T)(G B^T + A (G^T Q)) R^{-T} Omega^T.
 * G = dL/dX (m x n); Q (m x k) and B (k x n) are the forward's factors. */

/* X (k x nrhs) = M^{-1} Rhs for a k x k matrix M: Gaussian elimination with
 * partial pivoting (no structure of M assumed). */
static int solve_left(const double* M, int64_t k, const double* Rhs, int64_t nrhs, double* X) {
    double* Lu = (double*)malloc(sizeof(double) * (size_t)k * (size_t)k);
    memcpy(Lu, M, sizeof(double) * (size_t)k * (size_t)k);
    memcpy(X, Rhs, sizeof(double) * (size_t)k * (size_t)nrhs);
    int ok = 1;
    for (int64_t c = 0; c < k && ok; ++c) {
        int64_t p = c;
        for (int64_t r = c + 1; r < k; ++r)
            if (fabs(Lu[r + c * k]) > fabs(Lu[p + c * k])) p = r;
        if (Lu[p + c * k] == 0.0) { ok = 0; break; }
        if (p != c) {
            for (int64_t j = 0; j < k; ++j) { double t = Lu[c + j * k]; Lu[c + j * k] = Lu[p + j * k]; Lu[p + j * k] = t; }
            for (int64_t j = 0; j < nrhs; ++j) { double t = X[c + j * k]; X[c + j * k] = X[p + j * k]; X[p + j * k] = t; }
        }
        for (int64_t r = c + 1; r < k; ++r) {
            const double f = Lu[r + c * k] / Lu[c + c * k];
            for (int64_t j = c; j < k; ++j) Lu[r + j * k] -= f * Lu[c + j * k];
            for (int64_t j = 0; j < nrhs; ++j) X[r + j * k] -= f * X[c + j * k];
        }
    }
    if (ok) {
        for (int64_t j = 0; j < nrhs; ++j)
            for (int64_t r = k - 1; r >= 0; --r) {
                double s = X[r + j * k];
                for (int64_t t = r + 1; t < k; ++t) s -= Lu[r + t * k] * X[t + j * k];
                X[r + j * k] = s / Lu[r + r * k];
            }
    }
    free(Lu);
    return ok ? 0 : -1;
}

int orc_qqta_adjoint(const double* A, int64_t m, int64_t n, int64_t lda, const double* Q, int64_t ldq,
                     const double* B, int64_t ldb, int64_t k, uint64_t seed, int omega_prec,
                     const double* G, int64_t ldg, double* dA, int64_t ldda) {
    if (k <= 0 || k > m || k > n) return -1;
    double* Om = (double*)malloc(sizeof(double) * (size_t)n * (size_t)k);
    double* R = (double*)malloc(sizeof(double) * (size_t)k * (size_t)k);
    double* QtG = (double*)malloc(sizeof(double) * (size_t)k * (size_t)n);
    double* Bt = (double*)malloc(sizeof(double) * (size_t)n * (size_t)k);
    double* M1 = (double*)malloc(sizeof(double) * (size_t)m * (size_t)k);
    double* GtQ = (double*)malloc(sizeof(double) * (size_t)n * (size_t)k);
    double* T1 = (double*)malloc(sizeof(double) * (size_t)m * (size_t)k);
    double* QtM = (double*)malloc(sizeof(double) * (size_t)k * (size_t)k);
    double* M1t = (double*)malloc(sizeof(double) * (size_t)k * (size_t)m);
    double* Nt = (double*)malloc(sizeof(double) * (size_t)k * (size_t)m);
    double* Omt = (double*)malloc(sizeof(double) * (size_t)k * (size_t)n);
    double* T2 = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n);
    orc_omega(seed, 0u, n, 0, k, omega_prec, Om, n);
    mm_nn(k, k, n, B, ldb, Om, n, R, k);                       /* R = B Omega            */
    mm_tn(m, k, n, Q, ldq, G, ldg, QtG, k);                    /* Q^T G                  */
    mm_nn(m, n, k, Q, ldq, QtG, k, dA, ldda);                  /* dA = Q (Q^T G)         */
    for (int64_t c = 0; c < k; ++c)
        for (int64_t r = 0; r < n; ++r) Bt[r + c * n] = B[c + r * ldb];
    mm_nn(m, k, n, G, ldg, Bt, n, M1, m);                      /* M1 = G B^T             */
    mm_tn(m, n, k, G, ldg, Q, ldq, GtQ, n);                    /* G^T Q                  */
    mm_nn(m, k, n, A, lda, GtQ, n, T1, m);                     /* A (G^T Q)              */
    for (int64_t c = 0; c < k; ++c)
        for (int64_t r = 0; r < m; ++r) M1[r + c * m] += T1[r + c * m];
    mm_tn(m, k, k, Q, ldq, M1, m, QtM, k);                     /* Q^T M1                 */
    mm_nn(m, k, k, Q, ldq, QtM, k, T1, m);
    for (int64_t c = 0; c < k; ++c)
        for (int64_t r = 0; r < m; ++r) M1[r + c * m] -= T1[r + c * m];   /* (I - QQ^T) M1 */
    /* N = M1 R^{-T}  <=>  R N^T = M1^T */
    for (int64_t c = 0; c < k; ++c)
        for (int64_t r = 0; r < m; ++r) M1t[c + r * k] = M1[r + c * m];
    int rc = solve_left(R, k, M1t, m, Nt);
    if (rc == 0) {
        for (int64_t c = 0; c < n; ++c)
            for (int64_t r = 0; r < k; ++r) Omt[r + c * k] = Om[c + r * n];
        /* T2 = N Omega^T with N = Nt^T (m x k) */
        double* Nm = T1;
        for (int64_t c = 0; c < k; ++c)
            for (int64_t r = 0; r < m; ++r) Nm[r + c * m] = Nt[c + r * k];
        mm_nn(m, n, k, Nm, m, Omt, k, T2, m);
        for (int64_t c = 0; c < n; ++c)
            for (int64_t r = 0; r < m; ++r) dA[r + c * ldda] += T2[r + c * m];
    }
    free(Om); free(R); free(QtG); free(Bt); free(M1); free(GtQ); free(T1); free(QtM);
    free(M1t); free(Nt); free(Omt); free(T2);
    return rc;
}
