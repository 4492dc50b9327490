/*
 * rqb.h -- C ABI of the GB300 library for the blocked randomized QB scheme
 * (randQB_b) of Martinsson & Voronin, "A randomized blocked algorithm for
 * efficiently computing rank-revealing factorizations of matrices"
 * (arXiv:1503.07157).
 *
 * Problem (Sec. 1.1 eq. (1); Sec. 1.2): given an m x n matrix A and a tolerance
 * eps, find an orthonormal Q (m x k) and B = Q^T A (k x n) with
 * ||A - Q B||_F <= eps, building Q and B b columns/rows at a time as in
 * Fig. randQB_b:
 *   (2)  Omega_i = randn(n, b)
 *   (3)  Q_i = orth(A Omega_i)
 *   (3') Q_i = orth(Q_i - sum_{j<i} Q_j Q_j^T Q_i)
 *   (4)  B_i = Q_i^T A
 *   (5)  A = A - Q_i B_i
 *   (6)  stop once ||A||_F <= eps
 *
 * Conventions for every entry point:
 *   - matrices are column-major; a leading dimension is in elements and must
 *     be >= the row count;
 *   - pointers are DEVICE pointers unless the name ends in _host;
 *   - the element type of A, Q, B, Y, Omega is given by the handle's dtype:
 *     RQB_F64 -> double, RQB_F32 -> float (BF16 input: Q, B, Y are float);
 *   - every call returns an rqb_status; no exception crosses the ABI; the last
 *     status is also kept in the handle (rqb_get_stats);
 *   - all work is enqueued on the handle's stream (cfg.stream, a
 *     cudaStream_t; NULL = the legacy default stream).  Calls that return
 *     results to the host (k, stop decisions) synchronise that stream.
 *     The library's small kernels use programmatic dependent launches (each
 *     waits for the kernel before it in the stream before touching memory);
 *     the environment variable RQB_PDL=0, read once per process, launches
 *     everything ordinarily, with bit-identical results.
 *   - Omega entry (r, c) is a function of (seed, r, c) only: Philox4x32-10
 *     (Salmon et al., SC'11) at counter (r, c/2, 0, 0) with key (seed low
 *     word, seed high word) gives two uniforms u1, u2 in (0, 1) and
 *     Box-Muller gives sqrt(-2 ln u1) cos(2 pi u2) for even c and
 *     sqrt(-2 ln u1) sin(2 pi u2) for odd c.  FP64 handles use 53-bit uniforms
 *     and binary64 arithmetic; FP32 and BF16 handles use 23-bit uniforms and
 *     binary32 arithmetic.  Block i uses global columns (i-1) b .. i b - 1, so
 *     the blocks slice one fixed Omega (eq. OmegaBlock).
 */
#ifndef RQB_H
#define RQB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RQB_OK = 0,
    RQB_ERR_INVALID = 1,     /* bad size, leading dimension, pointer or config */
    RQB_ERR_NONFINITE = 2,   /* NaN or Inf in A (detected through ||A||_F^2)   */
    RQB_ERR_BREAKDOWN = 3,   /* Gram matrix of a panel not positive definite   */
    RQB_ERR_OOM = 4,         /* device or pinned-host allocation failed        */
    RQB_ERR_TIMEOUT = 5,     /* a bounded device wait gave up                  */
    RQB_ERR_CUDA = 6,        /* a CUDA runtime call failed                     */
    RQB_NOT_CONVERGED = 7,   /* k reached max_rank with ||A - QB||_F > eps;
                                Q, B and k are still valid                      */
    RQB_ERR_UNSUPPORTED = 8, /* valid request this build cannot serve          */
    RQB_ERR_SCRATCH_LIMIT = 9 /* request exceeds the fixed scratch of
                                 rqb_sketch_noalloc                              */
} rqb_status;

typedef enum { RQB_F64 = 0, RQB_F32 = 1, RQB_BF16 = 2 } rqb_dtype;

/* Arithmetic of the n- and m-long products (sketch, B = Q^T A, downdate).
 * NATIVE: the dtype's own arithmetic on the SIMT pipes (FP64 or FP32).
 * TF32X3 (FP32 handles): tensor-core products with FP32 operands split into
 *   TF32 hi + lo parts (2 or 3 MMA passes), FP32 accumulation.
 * BF16 (BF16 handles; NATIVE means the same there): A and the downdated
 *   residual are stored in BF16 and the products run on BF16 tensor-core
 *   MMAs with FP32 accumulation -- W Omega exactly (Omega rounded to BF16),
 *   Q_i^T W and Q_i B_i with Q_i and B_i split into BF16 hi + lo parts.  Each
 *   downdate rounds the new residual to BF16 (nearest even).  Q, B and Y are
 *   FP32.
 * Panel Gram matrices, Cholesky factors, re-projection coefficients and the
 * Frobenius downdate are accumulated in FP64 in every mode. */
typedef enum { RQB_PREC_NATIVE = 0, RQB_PREC_TF32X3 = 1, RQB_PREC_BF16 = 2 } rqb_prec;

typedef struct {
    int32_t dtype;       /* rqb_dtype                                           */
    int32_t prec;        /* rqb_prec                                            */
    int64_t max_rank;    /* rank cap; 0 = min(m, n)                             */
    int32_t fixed_rank;  /* nonzero: ignore eps, run until k = max_rank (Sec. 4.1) */
    int32_t power;       /* P of randQB_pb (Fig. randQB_pb); 0 = randQB_b       */
    void* stream;        /* cudaStream_t                                        */
    int32_t flags;       /* bit set of RQB_FLAG_*; other bits must be 0         */
    int32_t reserved;
} rqb_config;

/* cfg.flags: record CUDA events around each step of the block loop and
 * report their durations in rqb_stats.phase_ms (costs a few microseconds of
 * host time per step; no extra synchronisation beyond the per-block one). */
#define RQB_FLAG_PHASE_TIMING 1
/* With power > 0: the Sec. 5.4 variant of the power scheme, which forms
 * Y = (A A^T)^power A Omega_i by plain products and orthonormalises once
 * (no orth between the products of Fig. randQB_pb).  Cheaper per block; the
 * unblocked scheme then stalls near sigma_1 eps_mach^(1/(2 power + 1))
 * (Sec. 5.4), the blocked one reaches full precision (Sec. 6.3).  The panel
 * is still orthonormalised by CholeskyQR2, so a Y whose condition number
 * exceeds about u^(-1/2) of the Gram's precision reports
 * RQB_ERR_BREAKDOWN. */
#define RQB_FLAG_SKIP_INNER_ORTH 2
/* BF16 handles (else RQB_ERR_UNSUPPORTED): the sketch draws Omega_i
 * (Fig. randQB_b line (2)) inside its kernel, per K-chunk and row tile,
 * straight into the shared-memory operand of the tensor-core MMA, instead of
 * writing Omega_i once per block to device memory and loading it from there.
 * Same values and results bit for bit.  Regenerating Omega_i for every row
 * tile costs more arithmetic than the loads it replaces, so the default
 * (buffered Omega_i) is the faster path on this part; the flag exists to
 * measure the alternative. */
#define RQB_FLAG_OMEGA_SMEM 4

/* Steps timed with RQB_FLAG_PHASE_TIMING (index into phase_ms/phase_calls). */
typedef enum {
    RQB_PHASE_SKETCH = 0,    /* line (3) first block: Omega_1 and A Omega_1, ||A||_F^2 */
    RQB_PHASE_ORTH = 1,      /* lines (3), (3'): CholeskyQR2 with re-projection        */
    RQB_PHASE_PROJECT = 2,   /* line (4): B_i = Q_i^T A, ||B_i||^2                     */
    RQB_PHASE_DOWNDATE = 3,  /* line (5) fused with line (3) of the next block         */
    RQB_PHASE_CONTROL = 4,   /* line (6): stop test and its host read-back             */
    RQB_NUM_PHASES = 8
} rqb_phase;

#define RQB_MAX_TRACKED_BLOCKS 512

typedef struct {
    int64_t k;            /* rank of the last factorization                    */
    int64_t blocks;       /* number of blocks s                                */
    int32_t status;       /* rqb_status of the last call                       */
    int32_t direct_tests; /* blocks whose stop decision used the direct norm   */
    double normA2;        /* ||A||_F^2 (FP64)                                  */
    double eps;           /* tolerance of the last call                        */
    /* per-block stopping quantities, first min(blocks, RQB_MAX_TRACKED_BLOCKS) */
    double E[RQB_MAX_TRACKED_BLOCKS];  /* ||A||^2 - sum_{j<=i} ||B_j||^2       */
    double D[RQB_MAX_TRACKED_BLOCKS];  /* direct ||A^(i)||_F^2 where computed,
                                          else -1                              */
    int32_t kernel_launches; /* kernels launched by the last call              */
    int32_t svd_sweeps;      /* Jacobi sweeps of the last rqb_svd              */
    double phase_ms[RQB_NUM_PHASES];     /* summed device time per step (ms)   */
    int32_t phase_calls[RQB_NUM_PHASES]; /* times each step ran                */
    int32_t gram_fallbacks; /* tensor-core handles: panels whose first Gram was
                               recomputed with exact products (section of
                               rqb_factor)                                     */
    int32_t tile_width;     /* rqb_factor_batched: columns of A per work item of
                               the projection, as picked by the autotuner      */
    int32_t near_identity;  /* panels whose second CholeskyQR factor came from
                               the near-identity expansion (||G - I||_F below
                               2^-28 for an FP64 factor, 1e-4 for an FP32 one)
                               instead of the elimination                      */
    int32_t fused_gram;     /* split-TF32 handles: panels whose second Gram was
                               formed as Y1^T Y1 - C^T C from the product that
                               gives C = Qbar^T Y1 (line (3'), ||C||_F^2 at most
                               0.05) instead of from the re-projected panel   */
    int32_t pass1_fp32;     /* tensor-core handles: panels whose first
                               CholeskyQR factor was the FP32 elimination of
                               the split-TF32 Gram (pivots spanning at most
                               1e3) rather than an FP64 one                   */
    int32_t reserved;
} rqb_stats;

typedef struct rqb_handle_s* rqb_handle;

/* Create a handle on the current CUDA device.  cfg is copied.
 * Errors: RQB_ERR_INVALID (null pointer, unknown dtype/prec, a flag bit other
 *         than the RQB_FLAG_* ones, max_rank < 0, power outside 0..8),
 *         RQB_ERR_UNSUPPORTED (dtype/prec pair not built: TF32X3 needs
 *         RQB_F32, RQB_PREC_BF16 needs RQB_BF16, and a BF16 handle needs
 *         power = 0), RQB_ERR_OOM. */
int rqb_create(rqb_handle* h, const rqb_config* cfg);

/* Release the handle and everything it owns (Q, B, workspace). */
int rqb_destroy(rqb_handle h);

/* randQB_b (Fig. randQB_b; with cfg.power > 0 randQB_pb, Fig. randQB_pb).
 *   A      device, m x n, leading dim lda >= m, read only (the residual is
 *          downdated in a handle-owned copy, eq. def3)
 *   eps    absolute Frobenius tolerance, >= 0 (Sec. 1.1 eq. (1))
 *   b      block size, 1 <= b <= 256
 *   seed   Omega seed
 * Outputs (handle-owned device buffers, valid until the next factor call on
 * this handle or rqb_destroy):
 *   *Q     m x k orthonormal, leading dim *ldq
 *   *B     k x n, leading dim *ldb
 *   *k     rank reached, a multiple of b except when capped by max_rank or
 *          min(m, n) (the last block is then shrunk to fit)
 * Stop rule: after B_i, E_i = ||A||_F^2 - sum_j ||B_j||_F^2 (FP64) is compared
 * with eps^2 (Sec. 4.2 with Prop. 4.1(b)); when E_i is within the rounding
 * band of the working precision around eps^2 the decision is taken on the
 * directly computed ||A^(i)||_F^2 instead, as in line (6).  BF16 handles
 * (A in BF16, Q and B returned in FP32) need m >= 128 and n >= 256
 * (RQB_ERR_UNSUPPORTED otherwise) and decide every block on the direct
 * ||A^(i)||_F^2 of the stored (rounded) residual, since the BF16 rounding of
 * each downdate moves the residual away from E_i; stats.E still reports E_i.
 * On split-TF32 and BF16 handles the first CholeskyQR pass of a panel takes
 * its Gram from split-TF32 tensor-core products (relative error ~1e-7); when
 * the FP64 Cholesky of it breaks down or its pivots put kappa(G) above 1e5,
 * the Gram is recomputed with exact products and FP64 sums
 * (stats.gram_fallbacks counts those panels).  The second pass always uses an
 * FP64-accumulated Gram.
 * Returns RQB_OK, RQB_NOT_CONVERGED, or an error. */
int rqb_factor(rqb_handle h, const void* A, int64_t m, int64_t n, int64_t lda,
               double eps, int64_t b, uint64_t seed,
               const void** Q, int64_t* ldq, const void** B, int64_t* ldb, int64_t* k);

/* As rqb_factor, with A, Q and B in HOST memory: A_host is copied to the
 * device, factored, and Q (m x k into Q_host, leading dim ldq_host >= m) and
 * B (k x n into B_host, leading dim ldb_host >= capacity) are copied back.
 * Q_host must hold cap columns and B_host cap rows, cap = max_rank (or
 * min(m, n)).  Pinned host buffers give the fastest copies. */
int rqb_factor_host(rqb_handle h, const void* A_host, int64_t m, int64_t n, int64_t lda,
                    double eps, int64_t b, uint64_t seed,
                    void* Q_host, int64_t ldq_host, void* B_host, int64_t ldb_host, int64_t* k);

/* randQB_b (Fig. randQB_b) for `count` independent FP32 matrices of any
 * sizes.  All matrices advance block by block together: block i of every
 * still-active matrix is one sequence of grouped launches covering the tiles
 * of all of them (largest matrices first), with each matrix's k, E_i and stop
 * decision kept on the device; blocks run in chunks of eight, each chunk one
 * captured CUDA graph.  Per matrix t (host arrays):
 *   A[t]   device pointer, m[t] x n[t], leading dim lda[t] >= m[t]
 *   eps[t] absolute tolerance
 * Shared: b (1 <= b <= 32), seed (each matrix uses the same Omega stream, its
 * own columns), the handle's max_rank (0 = min(m, n)).  Outputs (host arrays,
 * device pointers valid until the next batched call or rqb_destroy):
 *   Q[t], ldq[t], B[t], ldb[t], k[t], status[t] (RQB_OK, RQB_NOT_CONVERGED,
 *   RQB_ERR_BREAKDOWN or RQB_ERR_NONFINITE per matrix).
 * The handle must be FP32 with power = 0.  Workspace: a residual copy of
 * every matrix (sum of m[t] n[t] floats) besides the outputs.  Returns RQB_OK
 * when the launches ran (per-matrix results in status), else an error. */
int rqb_factor_batched(rqb_handle h, int64_t count, const void* const* A, const int64_t* m,
                       const int64_t* n, const int64_t* lda, const double* eps, int64_t b,
                       uint64_t seed, const void** Q, int64_t* ldq, const void** B, int64_t* ldb,
                       int64_t* k, int* status);

/* X (m x n, leading dim ldx, device) = Q B of the last factorization on this
 * handle, i.e. the approximation Q Q^T A (Prop. 4.1(b)). */
int rqb_reconstruct(rqb_handle h, void* X, int64_t ldx);

/* Adjoint of the last factorization on this handle, seen as the map
 * A -> X = Q Q^T A with Omega (the first k global columns) held fixed.  The
 * paper gives no derivatives; Q Q^T is the projector onto R(A Omega) (Sec. 4.1,
 * Prop. 4.1(c)), and differentiating it gives
 *   dL/dA = Q (Q^T G) + (I - Q Q^T)(G B^T + A (G^T Q)) R^{-T} Omega^T,
 *   R = B Omega (upper triangular by Prop. 4.1(c)),
 * computed from the stored Q, B and the regenerated Omega (no panel factors
 * are kept).  G = dL_dX (m x n, leading dim ldg), dL_dA (m x n, leading dim
 * ldda, caller-owned, overwritten).  The A passed to the factorization must
 * still be valid and unchanged.  Errors: RQB_ERR_INVALID (no factorization on
 * the handle, bad leading dimension), RQB_ERR_UNSUPPORTED (power > 0 or a
 * BF16 handle). */
int rqb_backward(rqb_handle h, const void* dL_dX, int64_t ldg, void* dL_dA, int64_t ldda);

/* Low-rank SVD from the last factorization on this handle (Sec. 2,
 * "Computing the low rank SVD"): with the full SVD of the k x n factor
 * B = U_hat D V_hat^T, the rank-r factors are U_r = Q U_hat(:, 1:r),
 * Sigma_r = D(1:r, 1:r) and V_r = V_hat(:, 1:r), so A ~ U_r Sigma_r V_r^T.
 * B's SVD is taken from G = B B^T (k x k; FP64 sums of exact products) by
 * cyclic Jacobi rotations in FP64 until a sweep rotates nothing (a rotation
 * is skipped when |g_pq| <= 1e-15 sqrt(g_pp g_qq)); sigma_i = sqrt(lambda_i),
 * U_hat = the eigenvectors, V_r^T = Sigma_r^-1 U_hat(:, 1:r)^T B.
 *   r      1 <= r <= k of the last factorization
 *   U      device, m x r, leading dim ldu >= m (handle's output type)
 *   S      HOST, r doubles, descending
 *   Vt     device, r x n = V_r^T, leading dim ldvt >= r (a row for a zero
 *          singular value is zero)
 * Cost: O(k^2 n) for G and O(k^3) per Jacobi sweep (typically 6-10 sweeps);
 * stats.svd_sweeps reports the sweeps.  Errors: RQB_ERR_INVALID (no
 * factorization, bad r or leading dimension), RQB_ERR_NONFINITE, RQB_ERR_OOM. */
int rqb_svd(rqb_handle h, int64_t r, void* U, int64_t ldu, double* S, void* Vt, int64_t ldvt);

/* Self-test of the failure path of the tensor-core kernels: every wait of
 * theirs on an mbarrier (a TMA copy, an MMA, a peer warp) is bounded (2 s of
 * %globaltimer or 2^28 polls); on expiry the kernel drains its copies and
 * MMAs, frees tensor memory and records RQB_ERR_TIMEOUT.  This call runs one
 * such wait on a barrier that nothing completes and returns its status
 * (RQB_ERR_TIMEOUT when the limit works), with the time waited in
 * *waited_ms (may be NULL).  The handle and the CUDA context stay usable. */
int rqb_wait_selftest(rqb_handle h, double* waited_ms);

/* Statistics of the last call on this handle. */
int rqb_get_stats(rqb_handle h, rqb_stats* out);

/* ------------------------------------------------------------------------
 * Step-level entry points: single steps of Fig. randQB_b on caller buffers,
 * for verification of each step against the oracle.  On a BF16 handle A and
 * W are BF16 and Y, Qi, Bi, Qbar FP32; sketch, project and downdate need
 * m >= 128 and n >= 256 there (RQB_ERR_UNSUPPORTED otherwise), and the
 * downdate stores W = rn_bf16(A - Qi Bi) (normW2 of the stored values).
 * ------------------------------------------------------------------------ */

/* Omega block (line (2)): Omega (n x ncols, leading dim ldo >= n) receives
 * global columns col0 .. col0 + ncols - 1 of the Omega defined above, in the
 * form the handle's products use (binary64, binary32, or for RQB_PREC_TF32X3
 * the binary32 value rounded to TF32; for BF16 handles rounded to BF16 and
 * written as floats). */
int rqb_omega(rqb_handle h, int64_t n, int64_t col0, int64_t ncols, uint64_t seed,
              void* Omega, int64_t ldo);

/* Sketch (line (3), product part): Y (m x ncols, leading dim ldy) = A Omega,
 * Omega = global columns col0 .. col0 + ncols - 1, 1 <= ncols <= 256.
 * If normA2 is non-NULL it receives ||A||_F^2 (FP64, host). */
int rqb_sketch(rqb_handle h, const void* A, int64_t m, int64_t n, int64_t lda,
               int64_t col0, int64_t ncols, uint64_t seed,
               void* Y, int64_t ldy, double* normA2);

/* Lines (3) and (3'): Qi (m x p, leading dim ldqi) = orth(Y) re-orthogonalised
 * against Qbar (m x kprev, leading dim ldqb; may be NULL when kprev = 0), by
 * CholeskyQR with FP64 Gram/Cholesky, the re-projection, and a second
 * CholeskyQR; diag(R) > 0.  Returns RQB_ERR_BREAKDOWN when a Gram matrix is
 * not numerically positive definite.  m >= p, 1 <= p <= 256. */
int rqb_orth(rqb_handle h, const void* Y, int64_t m, int64_t p, int64_t ldy,
             const void* Qbar, int64_t kprev, int64_t ldqb, void* Qi, int64_t ldqi);

/* Line (4): Bi (p x n, leading dim ldbi) = Qi^T A with Qi m x p (ldqi),
 * A m x n (lda).  If normB2 is non-NULL it receives ||Bi||_F^2 (FP64, host). */
int rqb_project(rqb_handle h, const void* Qi, int64_t m, int64_t p, int64_t ldqi,
                const void* A, int64_t n, int64_t lda, void* Bi, int64_t ldbi, double* normB2);

/* Line (5) fused with line (3) of the next block: W (m x n, leading dim ldw)
 * = A - Qi Bi (A may alias W exactly, for the in-place downdate), and
 * Y (m x ncols, leading dim ldy) = W Omega(:, col0 : col0 + ncols).
 * If normW2 is non-NULL it receives ||W||_F^2 (FP64, host). */
int rqb_downdate_sketch(rqb_handle h, const void* A, int64_t lda, const void* Qi, int64_t ldqi,
                        const void* Bi, int64_t ldbi, int64_t m, int64_t n, int64_t p,
                        void* W, int64_t ldw, int64_t col0, int64_t ncols, uint64_t seed,
                        void* Y, int64_t ldy, double* normW2);

/* ------------------------------------------------------------------------
 * Allocation-free sketch.  The paper has no counterpart: this entry point
 * exists for callers of this library that cannot allocate device memory --
 * code that runs where the allocator must not be touched (a real-time loop,
 * a host callback, a process whose memory pool owns the whole device) or
 * whose allocator is capped by someone else.
 *
 * rqb_sketch_noalloc computes the same Y = A Omega(:, col0 : col0 + ncols)
 * (and optionally ||A||_F^2) as rqb_sketch, without a handle and without
 * calling cudaMalloc, cudaFree or any allocating library routine.  Its
 * scratch -- the Omega block, the split-K partial sums and the FP64 norm
 * partials -- is one static device array of RQB_NOALLOC_SCRATCH_BYTES that
 * every GPU loading this library keeps until the process exits.
 *   dtype  RQB_F32 or RQB_F64 (element type of A and Y)
 *   A, Y   device, column-major; lda >= m, ldy >= m
 *   ncols  1..256 (FP32) or 1..128 (FP64)
 *   normA2 host pointer or NULL; when non-NULL the call synchronises stream
 *   stream cudaStream_t (NULL: legacy default stream)
 * Errors: RQB_ERR_INVALID (bad argument), RQB_ERR_SCRATCH_LIMIT when the
 * Omega block (n * ncols rounded up to 32/64/128/256 columns) does not fit
 * the fixed scratch, or when normA2 is asked for and the product has more
 * than 8192 row tiles (tiles of 128 rows for FP32 with ncols <= 128, else of
 * 64 rows: m > 1048576 or m > 524288) -- nothing is launched then;
 * RQB_ERR_CUDA on a runtime error.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  All calls share the one array and it keeps the
 * last call's contents: calls that overlap on the GPU (different streams, or
 * different host threads on one device) race on it and must be serialised by
 * the caller. */
#define RQB_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int rqb_sketch_noalloc(int32_t dtype, const void* A, int64_t m, int64_t n, int64_t lda,
                       int64_t col0, int64_t ncols, uint64_t seed, void* Y, int64_t ldy,
                       double* normA2, void* stream);

/* ------------------------------------------------------------------------
 * Self-test of the FP64 reciprocal and reciprocal square root of the
 * Cholesky pivots.  The paper has no counterpart: the library's Cholesky
 * tiles take 1/d and 1/sqrt(d) of their FP64 pivots as an FP32 estimate
 * refined by two Newton steps (published iteration, not CUDA's division or
 * square root), and this entry point applies those same device functions to
 * an array so that a test can hold them to their error bounds.
 *   x       device, count FP64 values > 0
 *   rcp     device, count outputs: 1 / x
 *   rsq     device, count outputs: 1 / sqrt(x)
 *   stream  cudaStream_t (NULL: legacy default stream); asynchronous
 * Errors: RQB_ERR_INVALID (null pointer, count < 1), RQB_ERR_CUDA. */
int rqb_fp64_recip_selftest(const double* x, int64_t count, double* rcp, double* rsq, void* stream);

/* ------------------------------------------------------------------------
 * Test hook: host-side failure injection for the out-of-memory path.  The
 * paper has no counterpart.  after >= 0: the library's next `after` device
 * allocations succeed and the one after them fails as if cudaMalloc had run
 * out of memory (the call that needed it returns RQB_ERR_OOM; nothing is
 * launched for the failed step and the handle stays usable); the injection
 * then switches itself off.  after = -1 switches it off.  Process-wide.
 * Errors: RQB_ERR_INVALID (after < -1). */
int rqb_inject_alloc_failure(int64_t after);

/* Human-readable name of a status code (static string). */
const char* rqb_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* RQB_H */
