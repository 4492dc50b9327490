// rqb_tc.h -- host launchers of the split-TF32 tensor-core kernels (internal).
//
// All matrices FP32 and column-major unless stated; np is the padded block
// width (32, 64, 128 or 256) and the MMA N.  Every pointer that feeds a
// tensor map must be 16-byte aligned with a leading dimension that is a
// multiple of 4; the launchers return cudaErrorInvalidValue otherwise.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "rqb_engine.h"

namespace rqb {
namespace tc {

// The tensor-core path needs m >= 128 and n >= 256 (one full TMA box).
bool shape_ok(long long m, long long n);

// Floats of partial-accumulator scratch the sketch and the projection need.
size_t partial_floats(long long m, long long n, int np, int sms);

// Omega_i (n x np, ld ldo): columns col0 .. col0+p-1 of the binary32
// Gaussian rounded to TF32; columns p .. np-1 zero.
cudaError_t omega(Ctx& cx, long long n, long long col0, int p, int np, uint64_t seed, float* out, long long ldo);

// Split copies of Q_i (m x p, ld ldq): Qhi / Qlo (ld ldql, np columns) and
// the row-major transpose pair Qt / Qtl (m x np).
cudaError_t split_q(Ctx& cx, const float* Qi, long long ldq, long long m, int p, int np, float* Qhi, float* Qlo,
                    long long ldql, float* Qt, float* Qtl);

// Bs / Bsl (np x n, ld np): B_i (p x n, ld ldbi) and its lo part, zero rows
// p .. np-1 (the staged form the update reads).
cudaError_t stage_b(Ctx& cx, const float* Bi, long long ldbi, int p, long long n, int np, float* Bs, float* Bsl);

// Y (m x np, ld ldy) = X (m x n, ld ldx) Omega (n x np, ld ldom).  With
// nrm_out, ||X||_F^2 too (FP64, from the converter warps' reads of X: one
// partial per CTA in nrm_part, at most nrm_cap of them), so that the first
// block needs no separate pass over A.
cudaError_t sketch(Ctx& cx, const float* X, long long ldx, long long m, long long n, const float* Om, long long ldom,
                   int np, float* Y, long long ldy, float* part, size_t part_cap, double* nrm_part = nullptr,
                   int nrm_cap = 0, double* nrm_out = nullptr);

// B (pcols x n, ld ldb) = Q_i^T X and the staged split copy Bs / Bsl
// (np x n, ld np); ||B||_F^2 into *sq_out.
cudaError_t project(Ctx& cx, const float* X, long long ldx, long long m, long long n, const float* Qhi,
                    const float* Qlo, long long ldql, int pcols, int np, float* B, long long ldb, float* Bs,
                    float* Bsl, float* part, size_t part_cap, double* sq_part, int sq_cap, double* sq_out);

// Wdst = Wsrc - Q_i B_i (m x n); Wdst may equal Wsrc.  With sq_out,
// ||Wdst||_F^2 (FP64, summed from one partial per CTA in sq_part) too.
cudaError_t update(Ctx& cx, const float* Wsrc, long long ldws, float* Wdst, long long ldwd, long long m,
                   long long n, const float* Qt, const float* Qtl, const float* Bs, const float* Bsl, int np,
                   double* sq_part, int sq_cap, double* sq_out);

// Workspace of reproject (FP32): Y's split (m x np, ld ldyl), C^T (np x kprev),
// C in Omega layout (kprev x np, ld ldom), staging Bs / Bsl (np x kprev),
// stream-K partials, FP64 norm partials.
struct ReprojScratch {
    float* Yhi;
    float* Ylo;
    long long ldyl;
    float* Ct;
    double* Ct64;     // C^T (np x kprev, ld np) summed across CTAs in FP64
    float* Yt;        // row-major split copies of Y (m x np): the K-major
    float* Ytl;       // operand of product()
    float* Om;
    long long ldom;
    float* Bs;
    float* Bsl;
    float* part;
    size_t part_cap;
    double* sq_part;
    int sq_cap;
    double* sq_out;
    double* trace_part;  // np / 32 parts of ||C||_F^2 (reproject_gram)
    int* fused;          // reproject_gram's decision (device)
};

// Line (3') on the tensor core: Y (m x np) <- Y - Qbar (Qbar^T Y), Qbar
// m x kprev (ld ldq), both products split-TF32; C = Qbar^T Y is summed
// across CTAs in FP64 (w.Ct64) and rounded to TF32 as the operand of the
// second product; needs reproject_ok(m, kprev).
bool reproject_ok(long long m, long long kprev);

// Out (m x np, ld ldo) = Y (m x np, ld ldy) C (np x np, ld ldc) with the
// split-TF32 update kernel (both operands split, three passes); uses
// w.Yhi / w.Ylo (m x np) and w.Bs / w.Bsl (np x np).  Out must be
// TMA-addressable and np >= 128 (product_ok).
bool product_ok(long long m, int np, long long ldo, const float* Out);

// G (np x np, FP64, ld np) = Y^T Y (m x np, ld ldy) with the split-TF32
// projection kernel: each CTA accumulates its stretch of rows in FP32 (TMEM
// and period drains, relative accuracy ~1e-7), and the CTAs' partials are
// summed in FP64; needs gram_ok.
// With keep_split, the same pass over Y also writes the row-major split
// copies w.Yt / w.Ytl, so that a following product() of the same Y can skip
// its own split (presplit).
bool gram_ok(long long m, int np, long long ldy, const float* Y);
// A nonzero *gate (device) makes the launches do nothing but the copies kept
// for product() (keep_split).
cudaError_t gram(Ctx& cx, const float* Y, long long ldy, long long m, int np, const ReprojScratch& w, double* G,
                 bool keep_split = false, const int* gate = nullptr);
cudaError_t product(Ctx& cx, const float* Y, long long ldy, long long m, const float* C, long long ldc, int np,
                    float* Out, long long ldo, const ReprojScratch& w, bool presplit = false);
cudaError_t reproject(Ctx& cx, const float* Qbar, long long ldq, long long m, long long kprev, float* Y,
                      long long ldy, int np, const ReprojScratch& w);

// Line (3') with the second CholeskyQR pass's Gram from the same product:
// one stream-K pass of Y^T [Qbar Y] gives C^T and S = Y^T Y; then
// Y <- Y - Qbar C~ (C~ = C rounded to TF32, the product's operand) and
// G (np x np, FP64) = S - C^T C.  For an orthonormal Qbar the Gram of the
// new Y is S - C^T C + d^T d with d = C~ - C (|d| <= 2^-11 |C|), so the two
// differ by d^T d plus C~^T (Qbar^T Qbar - I) C~, both of the order of
// ||C||^2 times 2^-22 or Qbar's loss of orthogonality.  *fused (device) is
// set to 1 when ||C||_F^2 <= 0.05, where S - C^T C has no cancellation,
// else 0: the caller then forms the Gram of the new Y directly with
// gram(..., fused), which makes only product()'s copies of the split when
// *fused is 1.
// trace_part: np / 32 doubles.  Needs reproject_gram_ok (which also checks
// that w.part holds the split-k parts of C^T C).
bool reproject_gram_ok(long long m, long long kprev, int np, long long ldy, const float* Y, const ReprojScratch& w);
cudaError_t reproject_gram(Ctx& cx, const float* Qbar, long long ldq, long long m, long long kprev, float* Y,
                           long long ldy, int np, const ReprojScratch& w, double* G, int* fused,
                           double* trace_part);

// ---------------------------------------------------------------------------
// BF16 storage path (A and the residual W in BF16; kind::f16 MMAs with FP32
// accumulation).  np is 64, 128 or 256; BF16 tensor-map sources need a
// 16-byte aligned base and a leading dimension that is a multiple of 8.

// Block width padded to the BF16 MMA chunk (64 values of K).
int pad_block16(int b);

// Floats of partial-accumulator scratch of sketch16 / project16.
size_t partial_floats16(long long m, long long n, int np, int sms);

// Omega_i (n x np, ld ldo): the binary32 Gaussian rounded to BF16; columns
// p .. np-1 zero.  omega16_f32 writes the same values as floats.
cudaError_t omega16(Ctx& cx, long long n, long long col0, int p, int np, uint64_t seed, __nv_bfloat16* out,
                    long long ldo);
cudaError_t omega16_f32(Ctx& cx, long long n, long long col0, int p, int np, uint64_t seed, float* out,
                        long long ldo);

// BF16 hi / lo splits of Q_i: column-major Qhi / Qlo (ld ldql) and the
// row-major transpose pair Qt / Qtl (m x np).
cudaError_t split_q16(Ctx& cx, const float* Qi, long long ldq, long long m, int p, int np, __nv_bfloat16* Qhi,
                      __nv_bfloat16* Qlo, long long ldql, __nv_bfloat16* Qt, __nv_bfloat16* Qtl);

// Bs / Bsl (np x n, ld np): BF16 hi / lo split of B_i, zero rows p .. np-1.
cudaError_t stage_b16(Ctx& cx, const float* Bi, long long ldbi, int p, long long n, int np, __nv_bfloat16* Bs,
                      __nv_bfloat16* Bsl);

// Omega_i drawn inside the BF16 sketch instead of read from a buffer: global
// columns col0 .. col0 + p - 1 of the Gaussian matrix of seed (BF16-rounded
// binary32 draws, the values omega16 writes).
struct OmegaGen {
    long long col0;
    int p;
    uint64_t seed;
};

// Y (m x np, FP32) = X (BF16) Omega (BF16): exact products, FP32 sums.  With
// gen, Omega is generated per K-chunk in shared memory by the kernel (Om and
// ldom are not read).  With nrm_out, ||X||_F^2 too (FP64; the epilogue warps
// square the W tiles in shared memory; one partial per CTA in nrm_part, at
// most nrm_cap), so that the first block needs no separate pass over A.
cudaError_t sketch16(Ctx& cx, const __nv_bfloat16* X, long long ldx, long long m, long long n,
                     const __nv_bfloat16* Om, long long ldom, int np, float* Y, long long ldy, float* part,
                     size_t part_cap, const OmegaGen* gen = nullptr, double* nrm_part = nullptr, int nrm_cap = 0,
                     double* nrm_out = nullptr);

// B (pcols x n, FP32) = Q_i^T X with Q_i as its BF16 split, the staged split
// copy Bs / Bsl of B, and ||B||_F^2 into *sq_out.
cudaError_t project16(Ctx& cx, const __nv_bfloat16* X, long long ldx, long long m, long long n,
                      const __nv_bfloat16* Qhi, const __nv_bfloat16* Qlo, long long ldql, int pcols, int np, float* B,
                      long long ldb, __nv_bfloat16* Bs, __nv_bfloat16* Bsl, float* part, size_t part_cap,
                      double* sq_part, int sq_cap, double* sq_out);

// Wdst = rn_bf16(Wsrc - Q_i B_i); Wdst may equal Wsrc (both TMA-addressable:
// 16-byte aligned, leading dimension a multiple of 8).  With sq_out,
// ||Wdst||_F^2 of the stored values.
cudaError_t update16(Ctx& cx, const __nv_bfloat16* Wsrc, long long ldws, __nv_bfloat16* Wdst, long long ldwd,
                     long long m, long long n, const __nv_bfloat16* Qt, const __nv_bfloat16* Qtl,
                     const __nv_bfloat16* Bs, const __nv_bfloat16* Bsl, int np, double* sq_part, int sq_cap,
                     double* sq_out);

// One bounded mbarrier wait that nothing completes (device pointer
// waited_ns receives the wait's duration); records RQB_ERR_TIMEOUT in cx.st.
cudaError_t wait_selftest(Ctx& cx, unsigned long long* waited_ns);

}  // namespace tc
}  // namespace rqb
