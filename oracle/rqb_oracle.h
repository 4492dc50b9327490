/*
 * rqb_oracle.h -- CPU FP64 oracle for the blocked randomized QB scheme of
 * Martinsson & Voronin, "A randomized blocked algorithm for efficiently
 * computing rank-revealing factorizations of matrices" (arXiv:1503.07157).
 *
 * TEST INFRASTRUCTURE.  This library is the slow, obviously-correct reference
 * that the GPU path is checked against.  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or constant with the CUDA library under
 * paper_1503_07157_gb300/csrc, and the CUDA library never calls it.
 *
 * Conventions: every matrix is column-major with an explicit leading
 * dimension; every floating-point computation is IEEE binary64 unless a
 * function says otherwise.
 */
#ifndef RQB_ORACLE_H
#define RQB_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), written from its published round
 * definition.  ctr: 4 words, key: 2 words, out: 4 words. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* x rounded to 11 significant bits (TF32: 10 fraction bits), to nearest,
 * ties away from zero. */
double orc_round_tf32(double x);

/* x rounded to 8 significant bits (BF16: 7 fraction bits), to nearest, ties
 * to even. */
double orc_round_bf16(double x);
/* elementwise orc_round_bf16 of count values (x and y may alias) */
void orc_round_bf16_n(const double* x, double* y, int64_t count);

/* Gaussian test matrix Omega (Fig. randQB_b, line (2): Omega_i = randn(n, b)).
 * Writes the n x ncols block whose first column is global column col0 of the
 * infinite Gaussian matrix defined by (seed, stream).  Entry (r, c) depends
 * only on (seed, stream, r, c), so a block is a slice of one fixed Omega as in
 * eq. (OmegaBlock).  prec = 64: Box-Muller in binary64 from 53-bit uniforms.
 * prec = 32: the binary32 evaluation (23-bit uniforms, result rounded to
 * float, returned widened to double).  prec = 19: the prec-32 value rounded
 * to TF32 by orc_round_tf32, so that a tensor-core product with Omega as an
 * operand is exact; prec = 8: rounded to BF16 by orc_round_bf16.  out is
 * n x ncols, leading dim ldo. */
void orc_omega(uint64_t seed, uint32_t stream, int64_t n, int64_t col0,
               int64_t ncols, int prec, double* out, int64_t ldo);

/* orth() of Sec. 2.4: thin Householder QR of the m x p matrix Y (m >= p),
 * returning the m x p orthonormal factor with the sign convention diag(R) >= 0
 * (unique when Y has full column rank).  R (p x p, upper) is optional. */
void orc_orth(const double* Y, int64_t m, int64_t p, int64_t ldy,
              double* Q, int64_t ldq, double* R, int64_t ldr);

/* Result record of orc_randqb_b. */
typedef struct {
    int64_t k;          /* rank reached (multiple of b except a capped block) */
    int64_t blocks;     /* number of blocks s */
    int32_t status;     /* 0 converged, 1 reached the rank cap without E <= eps^2 */
    int32_t pad;
    double normA2;      /* ||A||_F^2 */
    /* per-block trajectories, capacity max_blocks entries each */
    double* E;          /* running downdate ||A||^2 - sum_j ||B_j||^2 after block i */
    double* D;          /* direct ||A^(i)||_F^2 after the downdate of block i */
    int64_t max_blocks;
} orc_qb_result;

/* randQB_b (Fig. randQB_b) and its power form randQB_pb (Fig. randQB_pb).
 *   A      m x n input (not modified; the oracle downdates a private copy)
 *   eps    absolute Frobenius tolerance: stop once E_i <= eps^2
 *   b      block size
 *   seed   Omega seed; block i uses global columns (i-1)b .. ib-1
 *   max_rank  rank cap (<= min(m, n)); 0 means min(m, n)
 *   fixed_rank  nonzero: ignore eps and run until k = max_rank (Sec. 4.1)
 *   power  P of randQB_pb (0 gives randQB_b)
 *   skip_inner_orth  nonzero: the Sec. 5.4 variant that applies the powers
 *          without the intermediate orth() calls
 *   omega_prec  64, 32, 19 or 8, see orc_omega
 *   Q      m x max_rank output, leading dim ldq
 *   B      max_rank x n output, leading dim ldb
 * Returns 0 on success, -1 on invalid arguments. */
int orc_randqb_b(const double* A, int64_t m, int64_t n, int64_t lda,
                 double eps, int64_t b, uint64_t seed, int64_t max_rank,
                 int fixed_rank, int power, int skip_inner_orth, int omega_prec,
                 double* Q, int64_t ldq, double* B, int64_t ldb,
                 orc_qb_result* res);

/* orc_randqb_b with the residual stored in a narrower format: storage_prec
 * 64 is orc_randqb_b; 16 rounds the residual to BF16 (orc_round_bf16) after
 * every downdate (line (5)), as a path that keeps A^(i) in BF16 does, and
 * then stops on the stored residual's norm D_i <= eps^2 (line (6)), since a
 * rounded residual no longer satisfies ||A^(i)||^2 = E_i. */
int orc_randqb_b_store(const double* A, int64_t m, int64_t n, int64_t lda,
                       double eps, int64_t b, uint64_t seed, int64_t max_rank,
                       int fixed_rank, int power, int skip_inner_orth, int omega_prec,
                       int storage_prec, double* Q, int64_t ldq, double* B, int64_t ldb,
                       orc_qb_result* res);

/* Unblocked randQB (Fig. randQB): Omega = the first l global columns,
 * Q = orth(A Omega), B = Q^T A.  Q is m x l, B is l x n. */
int orc_randqb(const double* A, int64_t m, int64_t n, int64_t lda, int64_t l,
               uint64_t seed, int omega_prec, double* Q, int64_t ldq,
               double* B, int64_t ldb);

/* Singular values of a small m x n matrix by one-sided (Hestenes) Jacobi,
 * sorted in decreasing order; sigma has min(m, n) entries. */
int orc_svd_values(const double* A, int64_t m, int64_t n, int64_t lda, double* sigma);

/* Low-rank SVD from a QB factorization (Sec. 2): B = Uh D Vh^T by one-sided
 * Jacobi on B^T; U = Q Uh(:, 1:r) (m x r), S = D(1:r) decreasing, Vt =
 * Vh(:, 1:r)^T (r x n).  Needs 1 <= r <= k <= n.  Returns 0, or -1 on bad
 * arguments. */
int orc_rsvd(const double* Q, int64_t m, int64_t k, int64_t ldq, const double* B, int64_t n, int64_t ldb,
             int64_t r, double* U, int64_t ldu, double* S, double* Vt, int64_t ldvt);

/* One step of the blocked scheme, exposed for step-level checks:
 *   orc_sketch:  Y = A Omega(:, col0 : col0 + p), Y is m x p.
 *   orc_orth_reproject: lines (3) and (3') of Fig. randQB_b,
 *          Q_i = orth(Y); Q_i = orth(Q_i - Qbar Qbar^T Q_i), Qbar m x kprev. */
void orc_sketch(const double* A, int64_t m, int64_t n, int64_t lda,
                uint64_t seed, int64_t col0, int64_t p, int omega_prec,
                double* Y, int64_t ldy);
void orc_orth_reproject(const double* Y, int64_t m, int64_t p, int64_t ldy,
                        const double* Qbar, int64_t kprev, int64_t ldqb,
                        double* Qi, int64_t ldqi);

/* Gradient of L(X) with respect to A for the fixed-rank map X = Q Q^T A,
 * Q = orth(A Omega) with Omega (first k global columns of the Gaussian matrix)
 * held fixed: dA = Q (Q^T G) + (I - Q Q^T)(G B^T + A (G^T Q)) R^{-T} Omega^T,
 * R = B Omega, from differentiating the projector onto R(A Omega).
 * Q (m x k), B (k x n) are the forward's factors; G = dL/dX (m x n).
 * Returns 0, or -1 when R is singular or k is out of range. */
int orc_qqta_adjoint(const double* A, int64_t m, int64_t n, int64_t lda, const double* Q, int64_t ldq,
                     const double* B, int64_t ldb, int64_t k, uint64_t seed, int omega_prec,
                     const double* G, int64_t ldg, double* dA, int64_t ldda);

/* Number of OpenMP threads the oracle's parallel loops use (1 without OpenMP). */
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
