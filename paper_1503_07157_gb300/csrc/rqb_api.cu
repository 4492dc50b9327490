// rqb_api.cu -- C ABI of the randQB_b library: handle, workspace, and the
// block loop of Fig. randQB_b driving the SIMT kernels of rqb_kernels.cu and,
// for RQB_PREC_TF32X3, the split-TF32 tensor-core products of rqb_tc.cu.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "rqb_engine.h"
#include "rqb_tc.h"

using namespace rqb;

namespace rqb {

// Countdown of rqb_inject_alloc_failure: -1 off; k >= 0: k more device
// allocations succeed, the next one fails, then the injection is off again.
static std::atomic<long long> g_fail_countdown{-1};

bool alloc_should_fail() {
    long long c = g_fail_countdown.load();
    while (c >= 0)
        if (g_fail_countdown.compare_exchange_weak(c, c - 1)) return c == 0;
    return false;
}

bool pdl_enabled() {
    static const bool on = [] {
        const char* v = std::getenv("RQB_PDL");
        return !(v && v[0] == '0');
    }();
    return on;
}

namespace batched {
int factor_batched(cudaStream_t stream, int num_sms, int64_t count, const void* const* A, const int64_t* m,
                   const int64_t* n, const int64_t* lda, const double* eps, int64_t b, uint64_t seed, int64_t max_rank,
                   const void** Q, int64_t* ldq, const void** B, int64_t* ldb, int64_t* k, int* status, void** outbuf,
                   size_t* outbytes, void** workbuf, size_t* workbytes, void** cache, float* ms, int* launches,
                   int* proj_width);
void release_cache(void* cache);
}
}  // namespace rqb

namespace {

constexpr int kNrmCap = 8192;      // per-CTA FP64 partials
constexpr int kScalars = 16;       // FP64 scalars on the device

int round_up(int64_t v, int64_t q) { return (int)(((v + q - 1) / q) * q); }

int pad_block(int64_t b) { return b <= 32 ? 32 : b <= 64 ? 64 : b <= 128 ? 128 : 256; }
constexpr int kMaxPanel = 256;   // the widest padded panel pad_block gives
// pinned host block of a handle: its DevState mirror, the first CholeskyQR
// pass's scratch state and that pass's diag(R)
constexpr size_t kHostPinned = 2 * sizeof(DevState) + sizeof(double) * kMaxPanel;

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    int ensure(size_t need) {
        if (need <= bytes) return RQB_OK;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        if (rqb::alloc_should_fail()) return RQB_ERR_OOM;
        if (cudaMalloc(&p, need) != cudaSuccess) {
            cudaGetLastError();
            return RQB_ERR_OOM;
        }
        bytes = need;
        return RQB_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
};

// CUDA-event timing of the steps of the block loop (RQB_FLAG_PHASE_TIMING).
// Pairs of events are recorded on the handle's stream and read after the
// per-block synchronisation that the loop already performs.
struct PhaseTimer {
    static constexpr int kPairs = 16;
    bool on = false;
    bool pending = false;
    int n = 0;
    cudaEvent_t ev[2 * kPairs] = {};
    int phase[kPairs] = {};
    int create() {
        for (int i = 0; i < 2 * kPairs; ++i)
            if (cudaEventCreate(&ev[i]) != cudaSuccess) return RQB_ERR_CUDA;
        on = true;
        return RQB_OK;
    }
    void destroy() {
        for (int i = 0; i < 2 * kPairs; ++i)
            if (ev[i]) cudaEventDestroy(ev[i]);
        on = false;
    }
    // NVTX ranges named after the steps (host side, always on; a profiler
    // that records NVTX shows the block loop's structure); at most one open
    void begin(cudaStream_t s, int ph) {
        static const char* const kName[RQB_NUM_PHASES] = {"rqb sketch", "rqb orth", "rqb project", "rqb downdate",
                                                          "rqb control", "rqb phase 5", "rqb phase 6", "rqb phase 7"};
        close_range();
        nvtxRangePushA(kName[(ph >= 0 && ph < RQB_NUM_PHASES) ? ph : RQB_NUM_PHASES - 1]);
        range_open = true;
        if (!on || n >= kPairs) return;
        cudaEventRecord(ev[2 * n], s);
        phase[n] = ph;
        pending = true;
    }
    void end(cudaStream_t s) {
        close_range();
        if (!on || !pending) return;
        cudaEventRecord(ev[2 * n + 1], s);
        pending = false;
        ++n;
    }
    void close_range() {
        if (range_open) nvtxRangePop();
        range_open = false;
    }
    bool range_open = false;
    // after the stream has been synchronised
    void flush(rqb_stats* st) {
        for (int i = 0; i < n; ++i) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]) == cudaSuccess) {
                st->phase_ms[phase[i]] += ms;
                st->phase_calls[phase[i]] += 1;
            }
        }
        n = 0;
    }
};

}  // namespace

struct rqb_handle_s {
    rqb_config cfg{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 1;
    size_t esize = 4;          // bytes per element of A (Q and B: 8 for FP64, else 4)
    // device memory
    DevBuf state;              // DevState + FP64 scalars + FP64 partials
    DevBuf arena;              // Omega, Y, Y1, Gram, R, Rinv, C, partials
    DevBuf q, b, w, ahost;     // outputs, residual copy, staging for host input
    int64_t ldq = 0, ldb = 0, ldw = 0, kcap_alloc = 0;
    // host mirror
    DevState* hstate = nullptr;  // pinned, with the two below in the same allocation
    DevState* hstate2 = nullptr; // the first CholeskyQR pass's scratch state (tensor-core Gram check)
    double* hdiag = nullptr;     // diag(R) of that pass, up to kMaxPanel entries
    rqb_stats stats{};
    int last_status = RQB_OK;
    PhaseTimer timer;
    // the last factorization, for rqb_reconstruct / rqb_backward
    const void* last_A = nullptr;
    int64_t last_m = 0, last_n = 0, last_lda = 0, last_k = 0, last_b = 0;
    uint64_t last_seed = 0;
    bool have_factor = false;
    DevBuf adj;                // workspace of rqb_backward
    DevBuf tcbuf;              // operand copies and partials of the tensor-core products
    DevBuf svdbuf;             // workspace of rqb_svd
    DevBuf pcbuf;              // workspace of the tensor-core re-projection
    void* bat_out = nullptr;   // outputs of rqb_factor_batched
    size_t bat_out_bytes = 0;
    void* bat_work = nullptr;  // its descriptors and per-CTA scratch
    size_t bat_work_bytes = 0;
    void* bat_cache = nullptr; // its instantiated graph and autotuned tiles
};

namespace {

template <typename T>
struct Arena {
    T* Om;          // n x bp row-major
    T* Y;           // m x bp (ld m)
    T* Y1;          // max(m, n) x bp: panel scratch of orth_reproject
    T* Qt;          // m x bp (ld m): power-scheme panel
    T* Z;           // n x bp (ld n): A^T Q of the power scheme
    T* Zq;          // n x bp (ld n): orth(A^T Q)
    T* Rinv;        // bp x bp
    T* Cc;          // kprev x bp
    T* part;        // split partials
    size_t part_cap;
    double* G;      // bp x bp
    double* R;      // bp x bp
    double* Cd;     // kprev x bp
    double* dpart;  // FP64 split partials
    size_t dpart_cap;
    const tc::ReprojScratch* rp = nullptr;  // set: line (3') on the tensor core
};

struct Scal {
    DevState* st;
    double* s;       // kScalars
    double* nrm;     // kNrmCap
};

Scal scalars(rqb_handle h) {
    Scal r;
    r.st = reinterpret_cast<DevState*>(h->state.p);
    r.s = reinterpret_cast<double*>(reinterpret_cast<char*>(h->state.p) + 256);
    r.nrm = r.s + kScalars;
    return r;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

template <typename T>
int ensure_arena(rqb_handle h, int64_t m, int64_t n, int bp, int64_t kprev_max, Arena<T>* out) {
    const size_t part_cap = (size_t)16 * (size_t)std::max(m, n) * (size_t)bp;
    const int64_t kp = std::max<int64_t>(kprev_max, 1);
    const size_t dpart_cap = std::max<size_t>((size_t)128 * bp * bp, (size_t)8 * kp * bp);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    const size_t oOm = take(sizeof(T) * (size_t)n * bp);
    const size_t oY = take(sizeof(T) * (size_t)m * bp);
    const size_t oY1 = take(sizeof(T) * (size_t)std::max(m, n) * bp);
    const size_t oQt = take(sizeof(T) * (size_t)m * bp);
    const size_t oZ = take(sizeof(T) * (size_t)n * bp);
    const size_t oZq = take(sizeof(T) * (size_t)n * bp);
    const size_t oRinv = take(sizeof(T) * (size_t)bp * bp);
    const size_t oCc = take(sizeof(T) * (size_t)kp * bp);
    const size_t oPart = take(sizeof(T) * part_cap);
    const size_t oG = take(sizeof(double) * (size_t)bp * bp);
    const size_t oR = take(sizeof(double) * (size_t)bp * bp);
    const size_t oCd = take(sizeof(double) * (size_t)kp * bp);
    const size_t oDp = take(sizeof(double) * dpart_cap);
    int rc = h->arena.ensure(off);
    if (rc != RQB_OK) return rc;
    char* base = reinterpret_cast<char*>(h->arena.p);
    out->Om = reinterpret_cast<T*>(base + oOm);
    out->Y = reinterpret_cast<T*>(base + oY);
    out->Y1 = reinterpret_cast<T*>(base + oY1);
    out->Qt = reinterpret_cast<T*>(base + oQt);
    out->Z = reinterpret_cast<T*>(base + oZ);
    out->Zq = reinterpret_cast<T*>(base + oZq);
    out->Rinv = reinterpret_cast<T*>(base + oRinv);
    out->Cc = reinterpret_cast<T*>(base + oCc);
    out->part = reinterpret_cast<T*>(base + oPart);
    out->part_cap = part_cap;
    out->G = reinterpret_cast<double*>(base + oG);
    out->R = reinterpret_cast<double*>(base + oR);
    out->Cd = reinterpret_cast<double*>(base + oCd);
    out->dpart = reinterpret_cast<double*>(base + oDp);
    out->dpart_cap = std::max<size_t>(dpart_cap, 1);
    return RQB_OK;
}

// Workspace of the split-TF32 products: Omega_i in K-major order, the split
// copies of Q_i and B_i, and the stream-K partial accumulators.
struct TcArena {
    float* Om;       // n x bp, ld ldom
    int64_t ldom;
    float* Qhi;      // m x bp, ld ldql
    float* Qlo;
    int64_t ldql;
    float* Qt;       // m x bp row-major
    float* Qtl;
    float* Bs;       // bp x n, ld bp
    float* Bsl;
    float* part;
    size_t part_cap;
};

int ensure_tc(rqb_handle h, int64_t m, int64_t n, int bp, TcArena* out) {
    const int64_t ldom = round_up(n, 4), ldql = round_up(m, 4);
    const size_t part = tc::partial_floats(m, n, bp, h->num_sms);
    size_t off = 0;
    auto take = [&](size_t floats) { size_t o = off; off = align256(off + 4 * floats); return o; };
    const size_t oOm = take((size_t)ldom * bp);
    const size_t oQh = take((size_t)ldql * bp), oQl = take((size_t)ldql * bp);
    const size_t oQt = take((size_t)m * bp), oQtl = take((size_t)m * bp);
    const size_t oBs = take((size_t)n * bp), oBsl = take((size_t)n * bp);
    const size_t oP = take(part);
    int rc = h->tcbuf.ensure(off);
    if (rc != RQB_OK) return rc;
    char* base = reinterpret_cast<char*>(h->tcbuf.p);
    auto at = [&](size_t o) { return reinterpret_cast<float*>(base + o); };
    out->Om = at(oOm); out->ldom = ldom;
    out->Qhi = at(oQh); out->Qlo = at(oQl); out->ldql = ldql;
    out->Qt = at(oQt); out->Qtl = at(oQtl);
    out->Bs = at(oBs); out->Bsl = at(oBsl);
    out->part = at(oP); out->part_cap = part;
    return RQB_OK;
}

// Workspace of the split-TF32 re-projection (line (3')) for panels of bp
// columns against up to kcap earlier columns.
int ensure_reproj(rqb_handle h, int64_t m, int64_t kcap, int bp, tc::ReprojScratch* w) {
    const int64_t ldyl = round_up(m, 4), ldom = round_up(kcap, 4);
    // the fused re-projection's product has kcap + bp output rows at most
    const size_t part = tc::partial_floats(m, std::max<int64_t>(kcap, 256) + bp, bp, h->num_sms);
    size_t off = 0;
    auto take = [&](size_t floats) { size_t o = off; off = align256(off + 4 * floats); return o; };
    const size_t oYh = take((size_t)ldyl * bp), oYl = take((size_t)ldyl * bp);
    const size_t kb = (size_t)std::max<int64_t>(kcap, bp);
    const size_t oCt = take((size_t)bp * kb), oOm = take((size_t)ldom * bp);
    const size_t oBs = take((size_t)bp * kb), oBsl = take((size_t)bp * kb);
    const size_t oC64 = take(2 * (size_t)bp * (kb + bp));   // C^T and, after it, Y^T Y (reproject_gram)
    const size_t oTr = take(2 * 64 + 4);                    // trace parts (FP64) and the fused flag
    const size_t oYt = take((size_t)ldyl * bp), oYtl = take((size_t)ldyl * bp);
    const size_t oP = take(part);
    int rc = h->pcbuf.ensure(off);
    if (rc != RQB_OK) return rc;
    char* base = reinterpret_cast<char*>(h->pcbuf.p);
    auto at = [&](size_t o) { return reinterpret_cast<float*>(base + o); };
    Scal sc = scalars(h);
    w->Yhi = at(oYh); w->Ylo = at(oYl); w->ldyl = ldyl;
    w->Ct = at(oCt); w->Om = at(oOm); w->ldom = ldom;
    w->Bs = at(oBs); w->Bsl = at(oBsl);
    w->Ct64 = reinterpret_cast<double*>(base + oC64);
    w->trace_part = reinterpret_cast<double*>(base + oTr);
    w->fused = reinterpret_cast<int*>(base + oTr + sizeof(double) * 64);
    w->Yt = at(oYt); w->Ytl = at(oYtl);
    w->part = at(oP); w->part_cap = part;
    w->sq_part = sc.nrm; w->sq_cap = kNrmCap; w->sq_out = sc.s + 8;
    return RQB_OK;
}

bool tma_ok(const void* p, int64_t ld) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0 && ld % 4 == 0; }

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return RQB_OK;
    if (e == cudaErrorMemoryAllocation) return RQB_ERR_OOM;
    return RQB_ERR_CUDA;
}

#define RQB_CK(call)                                    \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_status(e_);  \
    } while (0)

// Rounding band of the downdated E relative to ||A||^2 in the working precision.
template <typename T> double band_rel();
template <> double band_rel<double>() { return 64.0 * 1.1102230246251565e-16; }
template <> double band_rel<float>() { return 32.0 * 5.9604644775390625e-08; }
// split-TF32 products keep about 21 bits per term: 4 * 2^-20
constexpr double kBandTf32x3 = 3.814697265625e-06;

// Read the device state (synchronises the stream).
int read_state(rqb_handle h, const Scal& sc) {
    RQB_CK(cudaMemcpyAsync(h->hstate, sc.st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
    RQB_CK(cudaStreamSynchronize(h->stream));
    h->timer.flush(&h->stats);
    h->stats.near_identity = h->hstate->near_id;
    h->stats.fused_gram = h->hstate->fused_gram;
    return h->hstate->err;
}

// Line (6) without line (5) for the tensor-core handles, whose stop test is
// the direct norm of the stored residual (the downdated E of line (6) would
// carry the rounding of the FP32 or BF16 storage and of the split products
// in every block).  With X the
// stored residual before block i (direct norm dprev) and B_i = Q_i^T X
// (norm nb), Pythagoras (Prop. 4.1) gives ||X - Q_i B_i||^2 = dprev - nb for
// an orthonormal Q_i.  The bound below adds 1e-4 dprev for Q_i's
// orthogonality and the computed B_i and nb (each ~1e-5 or less on these
// handles), 2e-5 ||B_i|| for the products of the update, and the rounding of
// the stored residual (rho = 2^-8 for BF16 storage, 2^-23 for FP32).  When it
// is below eps^2 the stored residual the update would produce passes the
// test, so the last block needs no update.
bool stops_without_update(double dprev, double nb, double eps2, double rho) {
    const double core = std::sqrt(std::max(dprev * (1.0 + 1e-4) - nb, 0.0)) + 2e-5 * std::sqrt(std::max(nb, 0.0));
    const double upper = (1.0 + rho) * (1.0 + rho) * core * core;
    return std::isfinite(upper) && upper <= eps2;
}

// Lines (3) and (3'): Qout (p columns, ld ldqo) from the panel Y (bp columns,
// ld ldy; columns >= p are zero) and Qbar (kprev columns, ld ldqb).
template <typename T>
int orth_reproject(rqb_handle h, Ctx& cx, const Arena<T>& ar, const T* Y, int64_t ldy, int64_t m, int p, int bp,
                   const T* Qbar, int64_t kprev, int64_t ldqb, T* Qout, int64_t ldqo) {
    // pass 1: CholeskyQR of Y, Y1 = Y R^{-1}.  On the tensor-core handles the
    // Gram is first taken from the split-TF32 products (relative error
    // ~1e-7): pass 1 only has to leave Y1 well conditioned for pass 2, which
    // it does while kappa(Y)^2 * 1e-7 << 1.  That Gram is factored on a
    // scratch state, first by the FP32 elimination (its rounding, about
    // sqrt(bp) u32 kappa(G) in Y1^T Y1 - I, is of the order of the Gram's
    // own): accepted when it does not break down and its pivots span at most
    // 1e3.  Otherwise the saved Gram is factored in FP64, accepted up to a
    // pivot span of 1e5; past that the Gram is recomputed with exact products
    // and FP64 sums and factored again.
    bool pass1 = false;
    bool split1 = false;   // w.Yt / w.Ytl hold Y's split for the product Y R^-1
    if constexpr (std::is_same<T, float>::value) {
        const size_t sq = (size_t)bp * bp;
        if (ar.rp && m <= ar.rp->ldyl && tc::gram_ok(m, bp, ldy, Y) && ar.dpart_cap >= 9 * sq) {
            if (bp > kMaxPanel) return RQB_ERR_INVALID;
            split1 = tc::product_ok(m, bp, m, ar.Y1);
            RQB_CK(tc::gram(cx, Y, ldy, m, bp, *ar.rp, ar.G, split1));
            // the elimination overwrites G: a copy past its scratch
            double* Gsave = ar.dpart + 8 * sq;
            RQB_CK(cudaMemcpyAsync(Gsave, ar.G, sizeof(double) * sq, cudaMemcpyDeviceToDevice, h->stream));
            DevState* st2 = reinterpret_cast<DevState*>(reinterpret_cast<char*>(h->state.p) + 128);
            Ctx cx2 = cx;
            cx2.st = st2;
            for (int attempt = 0; attempt < 2 && !pass1; ++attempt) {
                const bool fp64 = attempt == 1;
                if (fp64)
                    RQB_CK(cudaMemcpyAsync(ar.G, Gsave, sizeof(double) * sq, cudaMemcpyDeviceToDevice, h->stream));
                RQB_CK(cudaMemsetAsync(st2, 0, sizeof(DevState), h->stream));
                cx2.launches = cx.launches;
                RQB_CK(chol_inv<T>(cx2, ar.G, bp, p, ar.R, ar.Rinv, fp64, ar.dpart, 8 * sq));
                cx.launches = cx2.launches;
                // pinned host copies: the synchronisation inside the panel
                // waits for two small copies, not for staged pageable ones
                const DevState& hs = *h->hstate2;
                const double* diag = h->hdiag;
                RQB_CK(cudaMemcpyAsync(h->hstate2, st2, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
                RQB_CK(cudaMemcpy2DAsync(h->hdiag, sizeof(double), ar.R, sizeof(double) * (bp + 1), sizeof(double),
                                         bp, cudaMemcpyDeviceToHost, h->stream));
                RQB_CK(cudaStreamSynchronize(h->stream));
                double lo = HUGE_VAL, hi = 0.0;
                for (int i = 0; i < p; ++i) {
                    lo = std::min(lo, diag[i]);
                    hi = std::max(hi, diag[i]);
                }
                pass1 = hs.err == RQB_OK && lo > 0.0 && (hi / lo) * (hi / lo) <= (fp64 ? 1e5 : 1e3);
                h->stats.pass1_fp32 += (pass1 && !fp64) ? 1 : 0;
            }
            h->stats.gram_fallbacks += pass1 ? 0 : 1;
        }
    }
    if (!pass1) {
        RQB_CK(gemm_tn_f64acc<T>(cx, m, bp, bp, Y, ldy, Y, ldy, ar.G, bp, ar.dpart, ar.dpart_cap, true, true));
        RQB_CK(chol_inv<T>(cx, ar.G, bp, p, ar.R, ar.Rinv, true, ar.dpart, ar.dpart_cap));
    }
    bool tc1 = false;
    if constexpr (std::is_same<T, float>::value) {
        if (ar.rp && m <= ar.rp->ldyl && tc::product_ok(m, bp, m, ar.Y1)) {
            RQB_CK(tc::product(cx, Y, ldy, m, ar.Rinv, bp, bp, ar.Y1, m, *ar.rp, split1));
            tc1 = true;
        }
    }
    if (!tc1) {
        NNArgs<T> a;
        a.m = m; a.K = bp; a.nc = bp; a.nout = bp;
        a.X = Y; a.ldx = ldy;
        a.C = ar.Rinv; a.csk = 1; a.csj = bp; a.c_rowmajor = false;
        a.Out = ar.Y1; a.ldo = m;
        RQB_CK(gemm_nn<T>(cx, a));
    }
    // line (3'): Y1 -= Qbar (Qbar^T Y1).  On the tensor-core handles the same
    // product also gives Y1^T Y1, from which the second pass's Gram follows
    // (tc::reproject_gram); *fused is set on the device where that formula is
    // used, and the direct Gram below then does nothing
    bool done = false;
    const int* fused = nullptr;
    if constexpr (std::is_same<T, float>::value) {
        if (kprev > 0 && ar.rp && m <= ar.rp->ldyl && tc::reproject_ok(m, kprev) && tma_ok(Qbar, ldqb)) {
            if (tc::reproject_gram_ok(m, kprev, bp, m, ar.Y1, *ar.rp)) {
                RQB_CK(tc::reproject_gram(cx, Qbar, ldqb, m, kprev, ar.Y1, m, bp, *ar.rp, ar.G, ar.rp->fused,
                                          ar.rp->trace_part));
                fused = ar.rp->fused;
            } else {
                RQB_CK(tc::reproject(cx, Qbar, ldqb, m, kprev, ar.Y1, m, bp, *ar.rp));
            }
            done = true;
        }
    }
    if (kprev > 0 && !done) {
        RQB_CK(gemm_tn_f64acc<T>(cx, m, (int)kprev, bp, Qbar, ldqb, ar.Y1, m, ar.Cd, kprev, ar.dpart,
                                 ar.dpart_cap, false));
        RQB_CK((launch_reduce_split<double, T>(cx, kprev, bp, 1, ar.Cd, kprev, 0, ar.Cc, kprev, nullptr, 0,
                                               nullptr)));
        NNArgs<T> a;
        a.m = m; a.K = kprev; a.nc = bp; a.nout = bp;
        a.X = Qbar; a.ldx = ldqb;
        a.C = ar.Cc; a.csk = 1; a.csj = kprev; a.c_rowmajor = false;
        a.Out = ar.Y1; a.ldo = m;
        a.Yin = ar.Y1; a.ldyin = m; a.alpha = T(-1); a.beta = T(1);
        a.part = ar.part; a.part_cap = ar.part_cap; a.allow_split = 1;
        RQB_CK(gemm_nn<T>(cx, a));
    }
    // pass 2: CholeskyQR of Y1, Qout = Y1 R^{-1}.  Y1 is well conditioned
    // (kappa ~ 1 after pass 1), so on the tensor-core handles its Gram comes
    // from the split-TF32 products (relative error ~1e-7, about what FP32
    // products summed in FP32 over 128 rows and then in FP64 leave).
    bool tcg2 = false;
    bool split2 = false;   // w.Yt / w.Ytl hold Y1's split for the product Y1 R^-1
    if constexpr (std::is_same<T, float>::value) {
        if (ar.rp && m <= ar.rp->ldyl && tc::gram_ok(m, bp, m, ar.Y1)) {
            // after the fused re-projection only the product's copies of the split are made
            split2 = p == bp && tc::product_ok(m, bp, ldqo, Qout);
            RQB_CK(tc::gram(cx, ar.Y1, m, m, bp, *ar.rp, ar.G, split2, fused));
            tcg2 = true;
        }
    }
    if (!tcg2)
        RQB_CK(gemm_tn_f64acc<T>(cx, m, bp, bp, ar.Y1, m, ar.Y1, m, ar.G, bp, ar.dpart, ar.dpart_cap, false, true));
    RQB_CK(chol_inv<T>(cx, ar.G, bp, p, ar.R, ar.Rinv, sizeof(T) == 8, ar.dpart, ar.dpart_cap, true));
    bool tc2 = false;
    if constexpr (std::is_same<T, float>::value) {
        // full-width panels only: the product writes all bp columns
        if (ar.rp && m <= ar.rp->ldyl && p == bp && tc::product_ok(m, bp, ldqo, Qout)) {
            RQB_CK(tc::product(cx, ar.Y1, m, m, ar.Rinv, bp, bp, Qout, ldqo, *ar.rp, split2));
            tc2 = true;
        }
    }
    if (!tc2) {
        NNArgs<T> a;
        a.m = m; a.K = bp; a.nc = bp; a.nout = p;
        a.X = ar.Y1; a.ldx = m;
        a.C = ar.Rinv; a.csk = 1; a.csj = bp; a.c_rowmajor = false;
        a.Out = Qout; a.ldo = ldqo;
        RQB_CK(gemm_nn<T>(cx, a));
    }
    return RQB_OK;
}

// Fig. randQB_pb lines (3)-(8) for block i: Q_i = orth(A Omega_i); P times
// Q_i = orth(A^T Q_i), Q_i = orth(A Q_i), on the current (downdated) A; then
// line (8): Q_i = orth(Q_i - Qbar Qbar^T Q_i), written to Qi.  ar.Y holds
// A Omega_i on entry; its columns >= p are zero.
template <typename T>
int power_panel(rqb_handle h, Ctx& cx, const Arena<T>& ar, int64_t m, int64_t n, int p, int bp, const T* W,
                int64_t ldw, const T* Qbar, int64_t kprev, int64_t ldqb, T* Qi) {
    RQB_CK(cudaMemsetAsync(ar.Qt, 0, sizeof(T) * (size_t)m * bp, h->stream));
    RQB_CK(cudaMemsetAsync(ar.Z, 0, sizeof(T) * (size_t)n * bp, h->stream));
    RQB_CK(cudaMemsetAsync(ar.Zq, 0, sizeof(T) * (size_t)n * bp, h->stream));
    if (h->cfg.flags & RQB_FLAG_SKIP_INNER_ORTH) {
        // Sec. 5.4 variant: Y <- A (A^T Y), power times, then one orth with
        // the re-projection against the earlier blocks
        for (int j = 0; j < h->cfg.power; ++j) {
            RQB_CK(gemm_tn<T>(cx, m, (int)n, p, W, ldw, ar.Y, m, ar.Z, n, ar.part, ar.part_cap, nullptr, 0,
                              nullptr));
            NNArgs<T> a;
            a.m = m; a.K = n; a.nc = bp; a.nout = bp;
            a.X = W; a.ldx = ldw;
            a.C = ar.Z; a.csk = 1; a.csj = n; a.c_rowmajor = false;
            a.Out = ar.Y; a.ldo = m;
            a.part = ar.part; a.part_cap = ar.part_cap; a.allow_split = 1;
            RQB_CK(gemm_nn<T>(cx, a));
        }
        return orth_reproject<T>(h, cx, ar, ar.Y, m, m, p, bp, Qbar, kprev, ldqb, Qi, ldqb);
    }
    int rc = orth_reproject<T>(h, cx, ar, ar.Y, m, m, p, bp, nullptr, 0, m, ar.Qt, m);     // line (3)
    if (rc != RQB_OK) return rc;
    for (int j = 0; j < h->cfg.power; ++j) {
        // line (5): Z = A^T Q_i (n x p), Q_i' = orth(Z)
        RQB_CK(gemm_tn<T>(cx, m, (int)n, p, W, ldw, ar.Qt, m, ar.Z, n, ar.part, ar.part_cap, nullptr, 0, nullptr));
        rc = orth_reproject<T>(h, cx, ar, ar.Z, n, n, p, bp, nullptr, 0, n, ar.Zq, n);
        if (rc != RQB_OK) return rc;
        // line (6): Y = A Q_i', Q_i = orth(Y)
        NNArgs<T> a;
        a.m = m; a.K = n; a.nc = bp; a.nout = bp;
        a.X = W; a.ldx = ldw;
        a.C = ar.Zq; a.csk = 1; a.csj = n; a.c_rowmajor = false;
        a.Out = ar.Y; a.ldo = m;
        a.part = ar.part; a.part_cap = ar.part_cap; a.allow_split = 1;
        RQB_CK(gemm_nn<T>(cx, a));
        rc = orth_reproject<T>(h, cx, ar, ar.Y, m, m, p, bp, nullptr, 0, m, ar.Qt, m);
        if (rc != RQB_OK) return rc;
    }
    // line (8): re-projection against the earlier blocks and a final orth
    return orth_reproject<T>(h, cx, ar, ar.Qt, m, m, p, bp, Qbar, kprev, ldqb, Qi, ldqb);
}

// Fig. randQB_b with the split-TF32 products (RQB_PREC_TF32X3, FP32 data):
// line (3) sketch and line (4) projection stream-K on tcgen05, line (5) the
// tensor-core update W <- W - Q_i B_i, then the next sketch of the updated
// W; the panel of lines (3)/(3') and the stopping test as in factor_impl.
int factor_tc(rqb_handle h, const float* A, int64_t m, int64_t n, int64_t lda, double eps, int64_t b, uint64_t seed,
              int64_t* k_out) {
    const int64_t rmax = std::min(m, n);
    const int64_t kcap = (h->cfg.max_rank > 0 && h->cfg.max_rank < rmax) ? h->cfg.max_rank : rmax;
    const int bp = pad_block(b);
    const int fixed = h->cfg.fixed_rank ? 1 : 0;
    Arena<float> ar;
    int rc = ensure_arena<float>(h, m, n, bp, kcap, &ar);
    if (rc != RQB_OK) return rc;
    TcArena ta;
    rc = ensure_tc(h, m, n, bp, &ta);
    if (rc != RQB_OK) return rc;
    tc::ReprojScratch rp;
    if ((rc = ensure_reproj(h, h->cfg.power > 0 ? std::max(m, n) : m, kcap, bp, &rp)) != RQB_OK) return rc;
    ar.rp = &rp;
    const int64_t ldq = round_up(m, 4), ldb = round_up(kcap, 4), ldw = round_up(m, 4);
    if ((rc = h->q.ensure(sizeof(float) * (size_t)ldq * (size_t)kcap)) != RQB_OK) return rc;
    if ((rc = h->b.ensure(sizeof(float) * (size_t)ldb * (size_t)n)) != RQB_OK) return rc;
    if ((rc = h->w.ensure(sizeof(float) * (size_t)ldw * (size_t)n)) != RQB_OK) return rc;
    h->ldq = ldq;
    h->ldb = ldb;
    h->ldw = ldw;
    h->kcap_alloc = kcap;
    float* Q = reinterpret_cast<float*>(h->q.p);
    float* B = reinterpret_cast<float*>(h->b.p);
    float* W = reinterpret_cast<float*>(h->w.p);

    Scal sc = scalars(h);
    Ctx cx;
    cx.stream = h->stream;
    cx.num_sms = h->num_sms;
    cx.st = sc.st;
    RQB_CK(cudaMemsetAsync(sc.st, 0, sizeof(DevState), h->stream));

    const double eps2 = eps * eps;
    int64_t k = 0;
    int blocks = 0, direct = 0;
    int status = RQB_OK;
    bool converged = false;
    bool empty_exit = false;
    double dprev = 0.0;    // direct norm of the stored residual before the current block

    // A as the first W: read in place when TMA can address it, else copied
    const float* Wsrc = A;
    int64_t ldws = lda;
    h->timer.begin(h->stream, RQB_PHASE_SKETCH);
    if (!tma_ok(A, lda)) {
        RQB_CK(cudaMemcpy2DAsync(W, sizeof(float) * ldw, A, sizeof(float) * lda, sizeof(float) * m, n,
                                 cudaMemcpyDeviceToDevice, h->stream));
        Wsrc = W;
        ldws = ldw;
    }
    int p = (int)std::min<int64_t>(b, kcap);
    // ||A||_F^2 comes out of the first sketch's own reads of A (no pass of its own)
    RQB_CK(tc::omega(cx, n, 0, p, bp, seed, ta.Om, ta.ldom));
    RQB_CK(tc::sketch(cx, Wsrc, ldws, m, n, ta.Om, ta.ldom, bp, ar.Y, m, ta.part, ta.part_cap, sc.nrm, kNrmCap,
                      sc.s + 0));
    RQB_CK(launch_set_norm(cx, sc.s + 0));
    h->timer.end(h->stream);

    for (;;) {
        p = (int)std::min<int64_t>(b, kcap - k);
        float* Qi = Q + k * ldq;
        float* Bi = B + k;
        h->timer.begin(h->stream, RQB_PHASE_ORTH);
        rc = (h->cfg.power == 0) ? orth_reproject<float>(h, cx, ar, ar.Y, m, m, p, bp, Q, k, ldq, Qi, ldq)
                                 : power_panel<float>(h, cx, ar, m, n, p, bp, Wsrc, ldws, Q, k, ldq, Qi);
        if (rc != RQB_OK) return rc;
        RQB_CK(tc::split_q(cx, Qi, ldq, m, p, bp, ta.Qhi, ta.Qlo, ta.ldql, ta.Qt, ta.Qtl));
        h->timer.end(h->stream);
        h->timer.begin(h->stream, RQB_PHASE_PROJECT);
        RQB_CK(tc::project(cx, Wsrc, ldws, m, n, ta.Qhi, ta.Qlo, ta.ldql, p, bp, Bi, ldb, ta.Bs, ta.Bsl, ta.part,
                           ta.part_cap, sc.nrm, kNrmCap, sc.s + 1));
        h->timer.end(h->stream);
        h->timer.begin(h->stream, RQB_PHASE_CONTROL);
        RQB_CK(launch_stop_after_b(cx, sc.s + 1, eps2, kBandTf32x3, fixed));
        h->timer.end(h->stream);
        int err = read_state(h, sc);
        if (blocks == 0 && !fixed && h->hstate->normA2 <= eps2) {
            // ||A||_F <= eps already: the empty factorization meets the
            // tolerance (whatever the degenerate first panel did)
            empty_exit = true;
            converged = true;
            break;
        }
        if (err != RQB_OK) { status = err; break; }
        const int flag = h->hstate->flag;
        if (blocks < RQB_MAX_TRACKED_BLOCKS) {
            h->stats.E[blocks] = h->hstate->E;
            h->stats.D[blocks] = -1.0;
        }
        if (blocks == 0) dprev = h->hstate->normA2;
        k += p;
        blocks++;
        if (flag == kStop) { converged = true; break; }
        if (!fixed && stops_without_update(dprev, h->hstate->normB2, eps2, 0x1p-23)) {
            if (blocks - 1 < RQB_MAX_TRACKED_BLOCKS) h->stats.D[blocks - 1] = std::max(dprev - h->hstate->normB2, 0.0);
            converged = true;
            break;
        }
        if (flag == kContinue && k >= kcap) break;
        const int pn = (int)std::min<int64_t>(b, std::max<int64_t>(kcap - k, 0));
        // line (5) with ||A^(i)||_F^2 on the same pass; the split-TF32 products
        // carry a rounding of E far above eps^2 at small eps, so the stop is
        // decided on the direct norm (line (6))
        h->timer.begin(h->stream, RQB_PHASE_DOWNDATE);
        RQB_CK(tc::update(cx, Wsrc, ldws, W, ldw, m, n, ta.Qt, ta.Qtl, ta.Bs, ta.Bsl, bp, sc.nrm, kNrmCap, sc.s + 2));
        h->timer.end(h->stream);
        Wsrc = W;
        ldws = ldw;
        RQB_CK(launch_stop_direct(cx, sc.s + 2, eps2, true));
        err = read_state(h, sc);
        if (err != RQB_OK) { status = err; break; }
        if (flag == kAmbiguous) direct++;
        if (blocks - 1 < RQB_MAX_TRACKED_BLOCKS) h->stats.D[blocks - 1] = h->hstate->D;
        dprev = h->hstate->D;
        if (!fixed && h->hstate->flag == kStop) { converged = true; break; }
        if (k >= kcap) break;
        h->timer.begin(h->stream, RQB_PHASE_SKETCH);
        RQB_CK(tc::omega(cx, n, k, pn, bp, seed, ta.Om, ta.ldom));
        RQB_CK(tc::sketch(cx, W, ldw, m, n, ta.Om, ta.ldom, bp, ar.Y, m, ta.part, ta.part_cap));
        h->timer.end(h->stream);
    }
    if (status == RQB_OK && !empty_exit) {
        int err = read_state(h, sc);
        if (err != RQB_OK) status = err;
    }
    h->stats.k = k;
    h->stats.blocks = blocks;
    h->stats.direct_tests = direct;
    h->stats.normA2 = h->hstate->normA2;
    h->stats.eps = eps;
    h->stats.kernel_launches = cx.launches;
    *k_out = k;
    if (status != RQB_OK) return status;
    if (!fixed && !converged) return RQB_NOT_CONVERGED;
    return RQB_OK;
}

// Workspace of the BF16 products: Omega_i and the BF16 hi / lo splits of Q_i
// and B_i, and the stream-K partials (FP32).
struct TcArena16 {
    __nv_bfloat16* Om;     // n x bp, ld ldom
    int64_t ldom;
    __nv_bfloat16* Qhi;    // m x bp, ld ldql
    __nv_bfloat16* Qlo;
    int64_t ldql;
    __nv_bfloat16* Qt;     // m x bp row-major
    __nv_bfloat16* Qtl;
    __nv_bfloat16* Bs;     // bp x n, ld bp
    __nv_bfloat16* Bsl;
    float* part;
    size_t part_cap;
};

int ensure_tc16(rqb_handle h, int64_t m, int64_t n, int bp, TcArena16* out) {
    const int64_t ldom = round_up(n, 8), ldql = round_up(m, 8);
    const size_t part = tc::partial_floats16(m, n, bp, h->num_sms);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    const size_t oOm = take(2 * (size_t)ldom * bp);
    const size_t oQh = take(2 * (size_t)ldql * bp), oQl = take(2 * (size_t)ldql * bp);
    const size_t oQt = take(2 * (size_t)m * bp), oQtl = take(2 * (size_t)m * bp);
    const size_t oBs = take(2 * (size_t)n * bp), oBsl = take(2 * (size_t)n * bp);
    const size_t oP = take(4 * part);
    int rc = h->tcbuf.ensure(off);
    if (rc != RQB_OK) return rc;
    char* base = reinterpret_cast<char*>(h->tcbuf.p);
    auto at = [&](size_t o) { return reinterpret_cast<__nv_bfloat16*>(base + o); };
    out->Om = at(oOm); out->ldom = ldom;
    out->Qhi = at(oQh); out->Qlo = at(oQl); out->ldql = ldql;
    out->Qt = at(oQt); out->Qtl = at(oQtl);
    out->Bs = at(oBs); out->Bsl = at(oBsl);
    out->part = reinterpret_cast<float*>(base + oP); out->part_cap = part;
    return RQB_OK;
}

bool tma_ok16(const void* p, int64_t ld) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0 && ld % 8 == 0; }

// Fig. randQB_b with A and the residual stored in BF16 (RQB_BF16): the
// sketch, projection and update run on kind::f16 MMAs; Q_i and B_i are FP32
// (CholeskyQR2 panel on the FP32 SIMT kernels).  The update rounds the new
// residual to BF16, so E_i no longer tracks the stored residual: the stop
// test of line (6) is decided on the direct ||A^(i)||_F^2 of the stored
// values, summed by the update itself, every block.
// Lines (2), (3) on the BF16 path: Omega_i (global columns col0 ..) into its
// buffer and Y = X Omega_i, or with RQB_FLAG_OMEGA_SMEM Omega_i drawn inside
// the sketch kernel (the same values).
// With nrm_out, ||X||_F^2 out of the same pass over X (nrm_part: kNrmCap
// FP64 partials).
int sketch_block16(rqb_handle h, Ctx& cx, const TcArena16& ta, const __nv_bfloat16* X, int64_t ldx, int64_t m,
                   int64_t n, int64_t col0, int p, int bp, uint64_t seed, float* Y, double* nrm_part = nullptr,
                   double* nrm_out = nullptr) {
    if (h->cfg.flags & RQB_FLAG_OMEGA_SMEM) {
        const tc::OmegaGen gen{col0, p, seed};
        RQB_CK(tc::sketch16(cx, X, ldx, m, n, nullptr, 0, bp, Y, m, ta.part, ta.part_cap, &gen, nrm_part, kNrmCap,
                            nrm_out));
        return RQB_OK;
    }
    RQB_CK(tc::omega16(cx, n, col0, p, bp, seed, ta.Om, ta.ldom));
    RQB_CK(tc::sketch16(cx, X, ldx, m, n, ta.Om, ta.ldom, bp, Y, m, ta.part, ta.part_cap, nullptr, nrm_part, kNrmCap,
                        nrm_out));
    return RQB_OK;
}

int factor_bf16(rqb_handle h, const __nv_bfloat16* A, int64_t m, int64_t n, int64_t lda, double eps, int64_t b,
                uint64_t seed, int64_t* k_out) {
    const int64_t rmax = std::min(m, n);
    const int64_t kcap = (h->cfg.max_rank > 0 && h->cfg.max_rank < rmax) ? h->cfg.max_rank : rmax;
    const int bp = tc::pad_block16((int)b);
    const int fixed = h->cfg.fixed_rank ? 1 : 0;
    Arena<float> ar;
    int rc = ensure_arena<float>(h, m, n, bp, kcap, &ar);
    if (rc != RQB_OK) return rc;
    TcArena16 ta;
    rc = ensure_tc16(h, m, n, bp, &ta);
    if (rc != RQB_OK) return rc;
    tc::ReprojScratch rp;
    if ((rc = ensure_reproj(h, h->cfg.power > 0 ? std::max(m, n) : m, kcap, bp, &rp)) != RQB_OK) return rc;
    ar.rp = &rp;
    const int64_t ldq = round_up(m, 4), ldb = round_up(kcap, 4), ldw = round_up(m, 8);
    if ((rc = h->q.ensure(sizeof(float) * (size_t)ldq * (size_t)kcap)) != RQB_OK) return rc;
    if ((rc = h->b.ensure(sizeof(float) * (size_t)ldb * (size_t)n)) != RQB_OK) return rc;
    if ((rc = h->w.ensure(2 * (size_t)ldw * (size_t)n)) != RQB_OK) return rc;
    h->ldq = ldq;
    h->ldb = ldb;
    h->ldw = ldw;
    h->kcap_alloc = kcap;
    float* Q = reinterpret_cast<float*>(h->q.p);
    float* B = reinterpret_cast<float*>(h->b.p);
    __nv_bfloat16* W = reinterpret_cast<__nv_bfloat16*>(h->w.p);

    Scal sc = scalars(h);
    Ctx cx;
    cx.stream = h->stream;
    cx.num_sms = h->num_sms;
    cx.st = sc.st;
    RQB_CK(cudaMemsetAsync(sc.st, 0, sizeof(DevState), h->stream));

    const double eps2 = eps * eps;
    int64_t k = 0;
    int blocks = 0;
    int status = RQB_OK;
    bool converged = false;
    double dprev = 0.0;    // direct norm of the stored residual before the current block

    const __nv_bfloat16* Wsrc = A;
    int64_t ldws = lda;
    h->timer.begin(h->stream, RQB_PHASE_SKETCH);
    if (!tma_ok16(A, lda)) {
        RQB_CK(cudaMemcpy2DAsync(W, 2 * ldw, A, 2 * lda, 2 * m, n, cudaMemcpyDeviceToDevice, h->stream));
        Wsrc = W;
        ldws = ldw;
    }
    int p = (int)std::min<int64_t>(b, kcap);
    // ||A||_F^2 comes out of the first sketch's own reads of A (no pass of its own)
    if ((rc = sketch_block16(h, cx, ta, Wsrc, ldws, m, n, 0, p, bp, seed, ar.Y, sc.nrm, sc.s + 0)) != RQB_OK)
        return rc;
    RQB_CK(launch_set_norm(cx, sc.s + 0));
    h->timer.end(h->stream);

    for (;;) {
        p = (int)std::min<int64_t>(b, kcap - k);
        float* Qi = Q + k * ldq;
        float* Bi = B + k;
        h->timer.begin(h->stream, RQB_PHASE_ORTH);
        rc = orth_reproject<float>(h, cx, ar, ar.Y, m, m, p, bp, Q, k, ldq, Qi, ldq);
        if (rc != RQB_OK) return rc;
        RQB_CK(tc::split_q16(cx, Qi, ldq, m, p, bp, ta.Qhi, ta.Qlo, ta.ldql, ta.Qt, ta.Qtl));
        h->timer.end(h->stream);
        h->timer.begin(h->stream, RQB_PHASE_PROJECT);
        RQB_CK(tc::project16(cx, Wsrc, ldws, m, n, ta.Qhi, ta.Qlo, ta.ldql, p, bp, Bi, ldb, ta.Bs, ta.Bsl, ta.part,
                             ta.part_cap, sc.nrm, kNrmCap, sc.s + 1));
        // E_i bookkeeping only (reported in the statistics)
        RQB_CK(launch_stop_after_b(cx, sc.s + 1, eps2, 0.0, 1));
        h->timer.end(h->stream);
        if (!fixed) {
            // line (6) decided before line (5) when the bound on the stored
            // residual the update would leave is already below eps^2
            const int err0 = read_state(h, sc);
            if (blocks == 0) dprev = h->hstate->normA2;
            if (!(blocks == 0 && h->hstate->normA2 <= eps2) && err0 == RQB_OK &&
                stops_without_update(dprev, h->hstate->normB2, eps2, 0x1p-8)) {
                if (blocks < RQB_MAX_TRACKED_BLOCKS) {
                    h->stats.E[blocks] = h->hstate->E;
                    h->stats.D[blocks] = std::max(dprev - h->hstate->normB2, 0.0);
                }
                k += p;
                blocks++;
                converged = true;
                break;
            }
        }
        h->timer.begin(h->stream, RQB_PHASE_DOWNDATE);
        RQB_CK(tc::update16(cx, Wsrc, ldws, W, ldw, m, n, ta.Qt, ta.Qtl, ta.Bs, ta.Bsl, bp, sc.nrm, kNrmCap,
                            sc.s + 2));
        h->timer.end(h->stream);
        Wsrc = W;
        ldws = ldw;
        h->timer.begin(h->stream, RQB_PHASE_CONTROL);
        RQB_CK(launch_stop_direct(cx, sc.s + 2, eps2, true));
        h->timer.end(h->stream);
        const int err = read_state(h, sc);
        if (blocks == 0 && !fixed && h->hstate->normA2 <= eps2) {
            // ||A||_F <= eps already: the empty factorization meets the
            // tolerance (whatever the degenerate first panel did)
            converged = true;
            break;
        }
        if (err != RQB_OK) { status = err; break; }
        if (blocks < RQB_MAX_TRACKED_BLOCKS) {
            h->stats.E[blocks] = h->hstate->E;
            h->stats.D[blocks] = h->hstate->D;
        }
        dprev = h->hstate->D;
        k += p;
        blocks++;
        if (!fixed && h->hstate->flag == kStop) { converged = true; break; }
        if (k >= kcap) break;
        const int pn = (int)std::min<int64_t>(b, kcap - k);
        h->timer.begin(h->stream, RQB_PHASE_SKETCH);
        if ((rc = sketch_block16(h, cx, ta, W, ldw, m, n, k, pn, bp, seed, ar.Y)) != RQB_OK) return rc;
        h->timer.end(h->stream);
    }
    h->stats.k = k;
    h->stats.blocks = blocks;
    h->stats.direct_tests = blocks;
    h->stats.normA2 = h->hstate->normA2;
    h->stats.eps = eps;
    h->stats.kernel_launches = cx.launches;
    *k_out = k;
    if (status != RQB_OK) return status;
    if (!fixed && !converged) return RQB_NOT_CONVERGED;
    return RQB_OK;
}

template <typename T>
int factor_impl(rqb_handle h, const T* A, int64_t m, int64_t n, int64_t lda, double eps, int64_t b, uint64_t seed,
                int64_t* k_out) {
    if constexpr (std::is_same<T, float>::value) {
        if (h->cfg.prec == RQB_PREC_TF32X3 && tc::shape_ok(m, n))
            return factor_tc(h, A, m, n, lda, eps, b, seed, k_out);
    }
    const int64_t rmax = std::min(m, n);
    const int64_t kcap = (h->cfg.max_rank > 0 && h->cfg.max_rank < rmax) ? h->cfg.max_rank : rmax;
    const int bp = pad_block(b);
    const int fixed = h->cfg.fixed_rank ? 1 : 0;
    Arena<T> ar;
    int rc = ensure_arena<T>(h, m, n, bp, kcap, &ar);
    if (rc != RQB_OK) return rc;
    // outputs
    const int64_t ldq = round_up(m, 4), ldb = round_up(kcap, 4);
    rc = h->q.ensure(sizeof(T) * (size_t)ldq * (size_t)kcap);
    if (rc != RQB_OK) return rc;
    rc = h->b.ensure(sizeof(T) * (size_t)ldb * (size_t)n);
    if (rc != RQB_OK) return rc;
    h->ldq = ldq;
    h->ldb = ldb;
    h->kcap_alloc = kcap;
    T* Q = reinterpret_cast<T*>(h->q.p);
    T* B = reinterpret_cast<T*>(h->b.p);

    Scal sc = scalars(h);
    Ctx cx;
    cx.stream = h->stream;
    cx.num_sms = h->num_sms;
    cx.st = sc.st;
    RQB_CK(cudaMemsetAsync(sc.st, 0, sizeof(DevState), h->stream));

    const double eps2 = eps * eps;
    const double tau_rel = band_rel<T>();
    int64_t k = 0;
    int blocks = 0, direct = 0;
    int status = RQB_OK;
    bool converged = false;
    bool empty_exit = false;

    // block 1 sketch: Y = A Omega_1 with ||A||_F^2 on the same read
    int p = (int)std::min<int64_t>(b, kcap);
    h->timer.begin(h->stream, RQB_PHASE_SKETCH);
    RQB_CK(launch_omega<T>(cx, n, 0, p, bp, seed, ar.Om, bp, 1));
    {
        NNArgs<T> a;
        a.m = m; a.K = n; a.nc = bp; a.nout = bp;
        a.X = A; a.ldx = lda;
        a.C = ar.Om; a.csk = bp; a.csj = 1; a.c_rowmajor = true;
        a.Out = ar.Y; a.ldo = m;
        a.part = ar.part; a.part_cap = ar.part_cap; a.allow_split = 1;
        a.nrm_part = sc.nrm; a.nrm_cap = kNrmCap; a.nrm_out = sc.s + 0;
        RQB_CK(gemm_nn<T>(cx, a));
    }
    RQB_CK(launch_set_norm(cx, sc.s + 0));
    h->timer.end(h->stream);

    const T* Wsrc = A;
    int64_t ldws = lda;
    T* W = nullptr;
    int64_t ldw = 0;
    for (;;) {
        p = (int)std::min<int64_t>(b, kcap - k);
        T* Qi = Q + k * ldq;
        T* Bi = B + k;
        // lines (3), (3')
        h->timer.begin(h->stream, RQB_PHASE_ORTH);
        if (h->cfg.power == 0) {
            rc = orth_reproject<T>(h, cx, ar, ar.Y, m, m, p, bp, Q, k, ldq, Qi, ldq);
            if (rc != RQB_OK) return rc;
        } else {
            rc = power_panel<T>(h, cx, ar, m, n, p, bp, Wsrc, ldws, Q, k, ldq, Qi);
            if (rc != RQB_OK) return rc;
        }
        h->timer.end(h->stream);
        h->timer.begin(h->stream, RQB_PHASE_PROJECT);
        // line (4): B_i = Q_i^T A, ||B_i||^2
        RQB_CK(gemm_tn<T>(cx, m, p, n, Qi, ldq, Wsrc, ldws, Bi, ldb, ar.part, ar.part_cap, sc.nrm, kNrmCap,
                          sc.s + 1));
        h->timer.end(h->stream);
        // line (6), downdate form of the test
        h->timer.begin(h->stream, RQB_PHASE_CONTROL);
        RQB_CK(launch_stop_after_b(cx, sc.s + 1, eps2, tau_rel, fixed));
        h->timer.end(h->stream);
        int err = read_state(h, sc);
        if (blocks == 0 && !fixed && h->hstate->normA2 <= eps2) {
            // ||A||_F <= eps already: the empty factorization meets the
            // tolerance (whatever the degenerate first panel did)
            empty_exit = true;
            converged = true;
            break;
        }
        if (err != RQB_OK) { status = err; break; }
        const int flag = h->hstate->flag;
        if (blocks < RQB_MAX_TRACKED_BLOCKS) {
            h->stats.E[blocks] = h->hstate->E;
            h->stats.D[blocks] = -1.0;
        }
        k += p;
        blocks++;
        if (flag == kStop) { converged = true; break; }
        if (flag == kContinue && k >= kcap) break;
        // line (5) fused with line (3) of the next block (or only the direct
        // norm when the cap is reached with an ambiguous E)
        const int pn = (int)std::min<int64_t>(b, std::max<int64_t>(kcap - k, 0));
        if (!W) {
            ldw = round_up(m, 4);
            rc = h->w.ensure(sizeof(T) * (size_t)ldw * (size_t)n);
            if (rc != RQB_OK) return rc;
            W = reinterpret_cast<T*>(h->w.p);
            h->ldw = ldw;
        }
        h->timer.begin(h->stream, RQB_PHASE_DOWNDATE);
        RQB_CK(launch_omega<T>(cx, n, k, pn, bp, seed, ar.Om, bp, 1));
        RQB_CK(downdate_sketch<T>(cx, m, n, p, bp, Wsrc, ldws, Qi, ldq, Bi, ldb, ar.Om, W, ldw, ar.Y, m, ar.part,
                                  ar.part_cap, sc.nrm, kNrmCap, sc.s + 2));
        h->timer.end(h->stream);
        RQB_CK(launch_stop_direct(cx, sc.s + 2, eps2));
        Wsrc = W;
        ldws = ldw;
        if (flag == kAmbiguous) {
            err = read_state(h, sc);
            if (err != RQB_OK) { status = err; break; }
            direct++;
            if (blocks - 1 < RQB_MAX_TRACKED_BLOCKS) h->stats.D[blocks - 1] = h->hstate->D;
            if (h->hstate->flag == kStop) { converged = true; break; }
        }
        if (k >= kcap) break;
    }
    if (status == RQB_OK && !empty_exit) {
        int err = read_state(h, sc);
        if (err != RQB_OK) status = err;
    }
    h->stats.k = k;
    h->stats.blocks = blocks;
    h->stats.direct_tests = direct;
    h->stats.normA2 = h->hstate->normA2;
    h->stats.eps = eps;
    h->stats.kernel_launches = cx.launches;
    *k_out = k;
    if (status != RQB_OK) return status;
    if (!fixed && !converged) return RQB_NOT_CONVERGED;
    return RQB_OK;
}

int check_matrix(const void* p, int64_t m, int64_t n, int64_t ld) {
    if (!p || m <= 0 || n <= 0 || ld < m) return RQB_ERR_INVALID;
    return RQB_OK;
}

int max_block(const rqb_handle h) { return h->cfg.dtype == RQB_F64 ? 128 : 256; }

int set_device(rqb_handle h) { return cudaSetDevice(h->device) == cudaSuccess ? RQB_OK : RQB_ERR_CUDA; }

int finish(rqb_handle h, int rc) {
    h->timer.close_range();
    h->last_status = rc;
    h->stats.status = rc;
    return rc;
}

}  // namespace

extern "C" {

int rqb_inject_alloc_failure(int64_t after) {
    if (after < -1) return RQB_ERR_INVALID;
    rqb::g_fail_countdown.store(after);
    return RQB_OK;
}

const char* rqb_status_string(int status) {
    switch (status) {
        case RQB_OK: return "ok";
        case RQB_ERR_INVALID: return "invalid argument";
        case RQB_ERR_NONFINITE: return "non-finite value in A";
        case RQB_ERR_BREAKDOWN: return "Gram matrix of a panel is not positive definite";
        case RQB_ERR_OOM: return "out of memory";
        case RQB_ERR_TIMEOUT: return "bounded device wait expired";
        case RQB_ERR_CUDA: return "CUDA runtime error";
        case RQB_NOT_CONVERGED: return "rank cap reached before the tolerance";
        case RQB_ERR_UNSUPPORTED: return "unsupported configuration";
        case RQB_ERR_SCRATCH_LIMIT: return "request exceeds the fixed scratch of rqb_sketch_noalloc";
        default: return "unknown status";
    }
}

int rqb_create(rqb_handle* out, const rqb_config* cfg) {
    if (!out || !cfg) return RQB_ERR_INVALID;
    *out = nullptr;
    if ((cfg->flags & ~(RQB_FLAG_PHASE_TIMING | RQB_FLAG_SKIP_INNER_ORTH | RQB_FLAG_OMEGA_SMEM)) != 0 ||
        cfg->max_rank < 0 || cfg->power < 0)
        return RQB_ERR_INVALID;
    if ((cfg->flags & RQB_FLAG_OMEGA_SMEM) && cfg->dtype != RQB_BF16) return RQB_ERR_UNSUPPORTED;
    if (cfg->dtype != RQB_F64 && cfg->dtype != RQB_F32 && cfg->dtype != RQB_BF16) return RQB_ERR_INVALID;
    if (cfg->prec != RQB_PREC_NATIVE && cfg->prec != RQB_PREC_TF32X3 && cfg->prec != RQB_PREC_BF16)
        return RQB_ERR_INVALID;
    if ((cfg->prec == RQB_PREC_TF32X3 && cfg->dtype != RQB_F32) ||
        (cfg->prec == RQB_PREC_BF16 && cfg->dtype != RQB_BF16) || (cfg->dtype == RQB_BF16 && cfg->power != 0))
        return RQB_ERR_UNSUPPORTED;
    if (cfg->power > 8) return RQB_ERR_INVALID;
    rqb_handle h = new (std::nothrow) rqb_handle_s();
    if (!h) return RQB_ERR_OOM;
    h->cfg = *cfg;
    h->stream = reinterpret_cast<cudaStream_t>(cfg->stream);
    h->esize = (cfg->dtype == RQB_F64) ? 8 : (cfg->dtype == RQB_BF16) ? 2 : 4;
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return RQB_ERR_CUDA;
    }
    if (h->state.ensure(256 + sizeof(double) * (kScalars + kNrmCap)) != RQB_OK ||
        cudaMallocHost(reinterpret_cast<void**>(&h->hstate), kHostPinned) != cudaSuccess) {
        cudaGetLastError();
        h->state.release();
        delete h;
        return RQB_ERR_OOM;
    }
    std::memset(h->hstate, 0, kHostPinned);
    h->hstate2 = h->hstate + 1;
    h->hdiag = reinterpret_cast<double*>(h->hstate + 2);
    if ((cfg->flags & RQB_FLAG_PHASE_TIMING) && h->timer.create() != RQB_OK) {
        h->timer.destroy();
        cudaGetLastError();
        h->state.release();
        cudaFreeHost(h->hstate);
        delete h;
        return RQB_ERR_CUDA;
    }
    *out = h;
    return RQB_OK;
}

int rqb_destroy(rqb_handle h) {
    if (!h) return RQB_ERR_INVALID;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    h->state.release();
    h->arena.release();
    h->q.release();
    h->b.release();
    h->w.release();
    h->ahost.release();
    h->adj.release();
    h->tcbuf.release();
    h->svdbuf.release();
    h->pcbuf.release();
    rqb::batched::release_cache(h->bat_cache);
    if (h->bat_out) cudaFree(h->bat_out);
    if (h->bat_work) cudaFree(h->bat_work);
    if (h->hstate) cudaFreeHost(h->hstate);
    h->timer.destroy();
    delete h;
    return RQB_OK;
}

int rqb_factor(rqb_handle h, const void* A, int64_t m, int64_t n, int64_t lda, double eps, int64_t b,
               uint64_t seed, const void** Q, int64_t* ldq, const void** B, int64_t* ldb, int64_t* k) {
    if (!h) return RQB_ERR_INVALID;
    if (check_matrix(A, m, n, lda) != RQB_OK || !Q || !ldq || !B || !ldb || !k || b < 1 || b > max_block(h) ||
        !(eps >= 0.0) || !std::isfinite(eps))
        return finish(h, RQB_ERR_INVALID);
    if (set_device(h) != RQB_OK) return finish(h, RQB_ERR_CUDA);
    std::memset(&h->stats, 0, sizeof(h->stats));
    int64_t kk = 0;
    int rc;
    if (h->cfg.dtype == RQB_BF16)
        rc = tc::shape_ok(m, n) ? factor_bf16(h, static_cast<const __nv_bfloat16*>(A), m, n, lda, eps, b, seed, &kk)
                                : RQB_ERR_UNSUPPORTED;
    else if (h->cfg.dtype == RQB_F64)
        rc = factor_impl<double>(h, static_cast<const double*>(A), m, n, lda, eps, b, seed, &kk);
    else
        rc = factor_impl<float>(h, static_cast<const float*>(A), m, n, lda, eps, b, seed, &kk);
    *Q = h->q.p;
    *ldq = h->ldq;
    *B = h->b.p;
    *ldb = h->ldb;
    *k = kk;
    h->have_factor = (rc == RQB_OK || rc == RQB_NOT_CONVERGED) && kk > 0;
    h->last_A = A;
    h->last_m = m; h->last_n = n; h->last_lda = lda; h->last_k = kk; h->last_b = b; h->last_seed = seed;
    return finish(h, rc);
}

int rqb_factor_host(rqb_handle h, const void* A_host, int64_t m, int64_t n, int64_t lda, double eps, int64_t b,
                    uint64_t seed, void* Q_host, int64_t ldq_host, void* B_host, int64_t ldb_host, int64_t* k) {
    if (!h) return RQB_ERR_INVALID;
    const int64_t rmax = std::min(m, n);
    const int64_t kcap = (h->cfg.max_rank > 0 && h->cfg.max_rank < rmax) ? h->cfg.max_rank : rmax;
    if (check_matrix(A_host, m, n, lda) != RQB_OK || !Q_host || !B_host || !k || ldq_host < m ||
        ldb_host < kcap)
        return finish(h, RQB_ERR_INVALID);
    if (set_device(h) != RQB_OK) return finish(h, RQB_ERR_CUDA);
    const size_t es = h->esize, eo = (h->cfg.dtype == RQB_F64) ? 8 : 4;
    int rc = h->ahost.ensure(es * (size_t)m * (size_t)n);
    if (rc != RQB_OK) return finish(h, rc);
    if (cudaMemcpy2DAsync(h->ahost.p, es * m, A_host, es * lda, es * m, n, cudaMemcpyHostToDevice, h->stream) !=
        cudaSuccess) {
        cudaGetLastError();
        return finish(h, RQB_ERR_CUDA);
    }
    const void *Qd, *Bd;
    int64_t ldq, ldb, kk = 0;
    rc = rqb_factor(h, h->ahost.p, m, n, m, eps, b, seed, &Qd, &ldq, &Bd, &ldb, &kk);
    *k = kk;
    if (rc != RQB_OK && rc != RQB_NOT_CONVERGED) return finish(h, rc);
    if (kk > 0) {
        if (cudaMemcpy2DAsync(Q_host, eo * ldq_host, Qd, eo * ldq, eo * m, kk, cudaMemcpyDeviceToHost, h->stream) !=
                cudaSuccess ||
            cudaMemcpy2DAsync(B_host, eo * ldb_host, Bd, eo * ldb, eo * kk, n, cudaMemcpyDeviceToHost, h->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess) {
            cudaGetLastError();
            return finish(h, RQB_ERR_CUDA);
        }
    }
    return finish(h, rc);
}

int rqb_get_stats(rqb_handle h, rqb_stats* out) {
    if (!h || !out) return RQB_ERR_INVALID;
    *out = h->stats;
    out->status = h->last_status;
    return RQB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// step-level entry points
extern "C" int rqb_omega(rqb_handle h, int64_t n, int64_t col0, int64_t ncols, uint64_t seed, void* Omega, int64_t ldo) {
    if (!h) return RQB_ERR_INVALID;
    if (!Omega || n <= 0 || ncols <= 0 || col0 < 0 || ldo < n || ncols > (int64_t)1 << 30)
        return finish(h, RQB_ERR_INVALID);
    if (set_device(h) != RQB_OK) return finish(h, RQB_ERR_CUDA);
    Scal sc = scalars(h);
    Ctx cx;
    cx.stream = h->stream; cx.num_sms = h->num_sms; cx.st = sc.st;
    cudaError_t e;
    if (h->cfg.dtype == RQB_F64)
        e = launch_omega<double>(cx, n, col0, (int)ncols, (int)ncols, seed, static_cast<double*>(Omega), 1, ldo);
    else if (h->cfg.prec == RQB_PREC_TF32X3)
        e = tc::omega(cx, n, col0, (int)ncols, (int)ncols, seed, static_cast<float*>(Omega), ldo);
    else if (h->cfg.dtype == RQB_BF16)
        e = tc::omega16_f32(cx, n, col0, (int)ncols, (int)ncols, seed, static_cast<float*>(Omega), ldo);
    else
        e = launch_omega<float>(cx, n, col0, (int)ncols, (int)ncols, seed, static_cast<float*>(Omega), 1, ldo);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return finish(h, cuda_status(e));
}

namespace {
template <typename T>
int sketch_impl(rqb_handle h, const T* A, int64_t m, int64_t n, int64_t lda, int64_t col0, int p, uint64_t seed,
                T* Y, int64_t ldy, double* normA2) {
    const int bp = pad_block(p);
    Arena<T> ar;
    int rc = ensure_arena<T>(h, m, n, bp, 1, &ar);
    if (rc != RQB_OK) return rc;
    Scal sc = scalars(h);
    Ctx cx;
    cx.stream = h->stream; cx.num_sms = h->num_sms; cx.st = sc.st;
    RQB_CK(launch_omega<T>(cx, n, col0, p, bp, seed, ar.Om, bp, 1));
    NNArgs<T> a;
    a.m = m; a.K = n; a.nc = bp; a.nout = p;
    a.X = A; a.ldx = lda;
    a.C = ar.Om; a.csk = bp; a.csj = 1; a.c_rowmajor = true;
    a.Out = Y; a.ldo = ldy;
    a.part = ar.part; a.part_cap = ar.part_cap; a.allow_split = 1;
    if (normA2) { a.nrm_part = sc.nrm; a.nrm_cap = kNrmCap; a.nrm_out = sc.s + 0; }
    RQB_CK(gemm_nn<T>(cx, a));
    if (normA2) RQB_CK(cudaMemcpyAsync(normA2, sc.s + 0, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    RQB_CK(cudaStreamSynchronize(h->stream));
    return RQB_OK;
}

template <typename T>
int orth_impl(rqb_handle h, const T* Y, int64_t m, int p, int64_t ldy, const T* Qbar, int64_t kprev, int64_t ldqb,
              T* Qi, int64_t ldqi) {
    const int bp = pad_block(p);
    Arena<T> ar;
    int rc = ensure_arena<T>(h, m, 1, bp, kprev, &ar);
    if (rc != RQB_OK) return rc;
    tc::ReprojScratch rp;
    h->stats.gram_fallbacks = 0;
    h->stats.pass1_fp32 = 0;
    if (std::is_same<T, float>::value && (h->cfg.prec == RQB_PREC_TF32X3 || h->cfg.dtype == RQB_BF16) && m >= 128) {
        if ((rc = ensure_reproj(h, m, std::max<int64_t>(kprev, 1), bp, &rp)) != RQB_OK) return rc;
        ar.rp = &rp;
    }
    Scal sc = scalars(h);
    Ctx cx;
    cx.stream = h->stream; cx.num_sms = h->num_sms; cx.st = sc.st;
    RQB_CK(cudaMemsetAsync(sc.st, 0, sizeof(DevState), h->stream));
    // panel copy with zero padding to bp columns: Y_pad = Y * [I_p 0]
    RQB_CK(cudaMemsetAsync(ar.Y, 0, sizeof(T) * (size_t)m * bp, h->stream));
    RQB_CK(cudaMemcpy2DAsync(ar.Y, sizeof(T) * m, Y, sizeof(T) * ldy, sizeof(T) * m, p, cudaMemcpyDeviceToDevice,
                             h->stream));
    rc = orth_reproject<T>(h, cx, ar, ar.Y, m, m, p, bp, Qbar, kprev, ldqb, Qi, ldqi);
    if (rc != RQB_OK) return rc;
    return read_state(h, sc);
}

template <typename T>
int project_impl(rqb_handle h, const T* Qi, int64_t m, int p, int64_t ldqi, const T* A, int64_t n, int64_t lda,
                 T* Bi, int64_t ldbi, double* normB2) {
    const int bp = pad_block(p);
    Arena<T> ar;
    int rc = ensure_arena<T>(h, m, n, bp, 1, &ar);
    if (rc != RQB_OK) return rc;
    Scal sc = scalars(h);
    Ctx cx;
    cx.stream = h->stream; cx.num_sms = h->num_sms; cx.st = sc.st;
    RQB_CK(gemm_tn<T>(cx, m, p, n, Qi, ldqi, A, lda, Bi, ldbi, ar.part, ar.part_cap, sc.nrm, kNrmCap, sc.s + 1));
    if (normB2) RQB_CK(cudaMemcpyAsync(normB2, sc.s + 1, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    RQB_CK(cudaStreamSynchronize(h->stream));
    return RQB_OK;
}

template <typename T>
int dd_impl(rqb_handle h, const T* A, int64_t lda, const T* Qi, int64_t ldqi, const T* Bi, int64_t ldbi, int64_t m,
            int64_t n, int p, T* W, int64_t ldw, int64_t col0, int ncols, uint64_t seed, T* Y, int64_t ldy,
            double* normW2) {
    const int bp = pad_block(std::max(p, ncols));
    Arena<T> ar;
    int rc = ensure_arena<T>(h, m, n, bp, 1, &ar);
    if (rc != RQB_OK) return rc;
    Scal sc = scalars(h);
    Ctx cx;
    cx.stream = h->stream; cx.num_sms = h->num_sms; cx.st = sc.st;
    RQB_CK(launch_omega<T>(cx, n, col0, ncols, bp, seed, ar.Om, bp, 1));
    RQB_CK(downdate_sketch<T>(cx, m, n, p, bp, A, lda, Qi, ldqi, Bi, ldbi, ar.Om, W, ldw, ar.Y, m, ar.part,
                              ar.part_cap, sc.nrm, kNrmCap, sc.s + 2));
    RQB_CK(cudaMemcpy2DAsync(Y, sizeof(T) * ldy, ar.Y, sizeof(T) * m, sizeof(T) * m, ncols, cudaMemcpyDeviceToDevice,
                             h->stream));
    if (normW2) RQB_CK(cudaMemcpyAsync(normW2, sc.s + 2, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    RQB_CK(cudaStreamSynchronize(h->stream));
    return RQB_OK;
}
// Step entry points of a TF32X3 handle.
bool use_tc(const rqb_handle h, int64_t m, int64_t n) {
    return h->cfg.dtype == RQB_F32 && h->cfg.prec == RQB_PREC_TF32X3 && tc::shape_ok(m, n);
}

// X itself when TMA can address it, else a copy in the handle's W buffer.
int tma_source(rqb_handle h, const float* X, int64_t ldx, int64_t m, int64_t n, const float** out, int64_t* ldout) {
    if (tma_ok(X, ldx)) {
        *out = X;
        *ldout = ldx;
        return RQB_OK;
    }
    const int64_t ldw = round_up(m, 4);
    int rc = h->w.ensure(sizeof(float) * (size_t)ldw * (size_t)n);
    if (rc != RQB_OK) return rc;
    RQB_CK(cudaMemcpy2DAsync(h->w.p, sizeof(float) * ldw, X, sizeof(float) * ldx, sizeof(float) * m, n,
                             cudaMemcpyDeviceToDevice, h->stream));
    *out = reinterpret_cast<const float*>(h->w.p);
    *ldout = ldw;
    return RQB_OK;
}

int sketch_tc(rqb_handle h, const float* A, int64_t m, int64_t n, int64_t lda, int64_t col0, int p, uint64_t seed,
              float* Y, int64_t ldy, double* normA2) {
    const int bp = pad_block(p);
    Arena<float> ar;
    TcArena ta;
    int rc = ensure_arena<float>(h, m, n, bp, 1, &ar);
    if (rc == RQB_OK) rc = ensure_tc(h, m, n, bp, &ta);
    if (rc != RQB_OK) return rc;
    Scal sc = scalars(h);
    Ctx cx;
    cx.stream = h->stream; cx.num_sms = h->num_sms; cx.st = sc.st;
    RQB_CK(cudaMemsetAsync(sc.st, 0, sizeof(DevState), h->stream));
    const float* X;
    int64_t ldx;
    if ((rc = tma_source(h, A, lda, m, n, &X, &ldx)) != RQB_OK) return rc;
    RQB_CK(tc::omega(cx, n, col0, p, bp, seed, ta.Om, ta.ldom));
    RQB_CK(tc::sketch(cx, X, ldx, m, n, ta.Om, ta.ldom, bp, ar.Y, m, ta.part, ta.part_cap, sc.nrm, kNrmCap,
                      normA2 ? sc.s + 0 : nullptr));
    RQB_CK(cudaMemcpy2DAsync(Y, sizeof(float) * ldy, ar.Y, sizeof(float) * m, sizeof(float) * m, p,
                             cudaMemcpyDeviceToDevice, h->stream));
    if (normA2) RQB_CK(cudaMemcpyAsync(normA2, sc.s + 0, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return read_state(h, sc);
}

int project_tc(rqb_handle h, const float* Qi, int64_t m, int p, int64_t ldqi, const float* A, int64_t n, int64_t lda,
               float* Bi, int64_t ldbi, double* normB2) {
    const int bp = pad_block(p);
    TcArena ta;
    int rc = ensure_tc(h, m, n, bp, &ta);
    if (rc != RQB_OK) return rc;
    Scal sc = scalars(h);
    Ctx cx;
    cx.stream = h->stream; cx.num_sms = h->num_sms; cx.st = sc.st;
    RQB_CK(cudaMemsetAsync(sc.st, 0, sizeof(DevState), h->stream));
    const float* X;
    int64_t ldx;
    if ((rc = tma_source(h, A, lda, m, n, &X, &ldx)) != RQB_OK) return rc;
    RQB_CK(tc::split_q(cx, Qi, ldqi, m, p, bp, ta.Qhi, ta.Qlo, ta.ldql, ta.Qt, ta.Qtl));
    RQB_CK(tc::project(cx, X, ldx, m, n, ta.Qhi, ta.Qlo, ta.ldql, p, bp, Bi, ldbi, ta.Bs, ta.Bsl, ta.part,
                       ta.part_cap, sc.nrm, kNrmCap, sc.s + 1));
    if (normB2) RQB_CK(cudaMemcpyAsync(normB2, sc.s + 1, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return read_state(h, sc);
}

int dd_tc(rqb_handle h, const float* A, int64_t lda, const float* Qi, int64_t ldqi, const float* Bi, int64_t ldbi,
          int64_t m, int64_t n, int p, float* W, int64_t ldw, int64_t col0, int ncols, uint64_t seed, float* Y,
          int64_t ldy, double* normW2) {
    const int bpu = pad_block(p), bps = pad_block(ncols);
    Arena<float> ar;
    TcArena ta;
    int rc = ensure_arena<float>(h, m, n, bps, 1, &ar);
    if (rc == RQB_OK) rc = ensure_tc(h, m, n, std::max(bpu, bps), &ta);
    if (rc != RQB_OK) return rc;
    Scal sc = scalars(h);
    Ctx cx;
    cx.stream = h->stream; cx.num_sms = h->num_sms; cx.st = sc.st;
    RQB_CK(cudaMemsetAsync(sc.st, 0, sizeof(DevState), h->stream));
    RQB_CK(tc::split_q(cx, Qi, ldqi, m, p, bpu, ta.Qhi, ta.Qlo, ta.ldql, ta.Qt, ta.Qtl));
    RQB_CK(tc::stage_b(cx, Bi, ldbi, p, n, bpu, ta.Bs, ta.Bsl));
    // the update reads and writes W through TMA: unaligned operands go
    // through aligned copies (A into the handle's W buffer, the result into
    // the adjoint workspace, copied out afterwards)
    const float* Ax;
    int64_t ldax;
    if ((rc = tma_source(h, A, lda, m, n, &Ax, &ldax)) != RQB_OK) return rc;
    float* X = W;
    int64_t ldx = ldw;
    const bool copy_out = !tma_ok(W, ldw);
    if (copy_out) {
        ldx = round_up(m, 4);
        if ((rc = h->adj.ensure(sizeof(float) * (size_t)ldx * (size_t)n)) != RQB_OK) return rc;
        X = reinterpret_cast<float*>(h->adj.p);
    }
    RQB_CK(tc::update(cx, Ax, ldax, X, ldx, m, n, ta.Qt, ta.Qtl, ta.Bs, ta.Bsl, bpu, sc.nrm, kNrmCap,
                      normW2 ? sc.s + 2 : nullptr));
    if (copy_out)
        RQB_CK(cudaMemcpy2DAsync(W, sizeof(float) * ldw, X, sizeof(float) * ldx, sizeof(float) * m, n,
                                 cudaMemcpyDeviceToDevice, h->stream));
    RQB_CK(tc::omega(cx, n, col0, ncols, bps, seed, ta.Om, ta.ldom));
    RQB_CK(tc::sketch(cx, X, ldx, m, n, ta.Om, ta.ldom, bps, ar.Y, m, ta.part, ta.part_cap));
    RQB_CK(cudaMemcpy2DAsync(Y, sizeof(float) * ldy, ar.Y, sizeof(float) * m, sizeof(float) * m, ncols,
                             cudaMemcpyDeviceToDevice, h->stream));
    if (normW2) RQB_CK(cudaMemcpyAsync(normW2, sc.s + 2, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return read_state(h, sc);
}

// Step entry points of a BF16 handle (A and W in BF16; Q, B, Y in FP32).
int tma_source16(rqb_handle h, const __nv_bfloat16* X, int64_t ldx, int64_t m, int64_t n,
                 const __nv_bfloat16** out, int64_t* ldout) {
    if (tma_ok16(X, ldx)) {
        *out = X;
        *ldout = ldx;
        return RQB_OK;
    }
    const int64_t ldw = round_up(m, 8);
    int rc = h->w.ensure(2 * (size_t)ldw * (size_t)n);
    if (rc != RQB_OK) return rc;
    RQB_CK(cudaMemcpy2DAsync(h->w.p, 2 * ldw, X, 2 * ldx, 2 * m, n, cudaMemcpyDeviceToDevice, h->stream));
    *out = reinterpret_cast<const __nv_bfloat16*>(h->w.p);
    *ldout = ldw;
    return RQB_OK;
}

int sketch_bf16(rqb_handle h, const __nv_bfloat16* A, int64_t m, int64_t n, int64_t lda, int64_t col0, int p,
                uint64_t seed, float* Y, int64_t ldy, double* normA2) {
    const int bp = tc::pad_block16(p);
    Arena<float> ar;
    TcArena16 ta;
    int rc = ensure_arena<float>(h, m, n, bp, 1, &ar);
    if (rc == RQB_OK) rc = ensure_tc16(h, m, n, bp, &ta);
    if (rc != RQB_OK) return rc;
    Scal sc = scalars(h);
    Ctx cx;
    cx.stream = h->stream; cx.num_sms = h->num_sms; cx.st = sc.st;
    RQB_CK(cudaMemsetAsync(sc.st, 0, sizeof(DevState), h->stream));
    const __nv_bfloat16* X;
    int64_t ldx;
    if ((rc = tma_source16(h, A, lda, m, n, &X, &ldx)) != RQB_OK) return rc;
    if ((rc = sketch_block16(h, cx, ta, X, ldx, m, n, col0, p, bp, seed, ar.Y, sc.nrm,
                             normA2 ? sc.s + 0 : nullptr)) != RQB_OK)
        return rc;
    RQB_CK(cudaMemcpy2DAsync(Y, sizeof(float) * ldy, ar.Y, sizeof(float) * m, sizeof(float) * m, p,
                             cudaMemcpyDeviceToDevice, h->stream));
    if (normA2) RQB_CK(cudaMemcpyAsync(normA2, sc.s + 0, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return read_state(h, sc);
}

int project_bf16(rqb_handle h, const float* Qi, int64_t m, int p, int64_t ldqi, const __nv_bfloat16* A, int64_t n,
                 int64_t lda, float* Bi, int64_t ldbi, double* normB2) {
    const int bp = tc::pad_block16(p);
    TcArena16 ta;
    int rc = ensure_tc16(h, m, n, bp, &ta);
    if (rc != RQB_OK) return rc;
    Scal sc = scalars(h);
    Ctx cx;
    cx.stream = h->stream; cx.num_sms = h->num_sms; cx.st = sc.st;
    RQB_CK(cudaMemsetAsync(sc.st, 0, sizeof(DevState), h->stream));
    const __nv_bfloat16* X;
    int64_t ldx;
    if ((rc = tma_source16(h, A, lda, m, n, &X, &ldx)) != RQB_OK) return rc;
    RQB_CK(tc::split_q16(cx, Qi, ldqi, m, p, bp, ta.Qhi, ta.Qlo, ta.ldql, ta.Qt, ta.Qtl));
    RQB_CK(tc::project16(cx, X, ldx, m, n, ta.Qhi, ta.Qlo, ta.ldql, p, bp, Bi, ldbi, ta.Bs, ta.Bsl, ta.part,
                         ta.part_cap, sc.nrm, kNrmCap, sc.s + 1));
    if (normB2) RQB_CK(cudaMemcpyAsync(normB2, sc.s + 1, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return read_state(h, sc);
}

int dd_bf16(rqb_handle h, const __nv_bfloat16* A, int64_t lda, const float* Qi, int64_t ldqi, const float* Bi,
            int64_t ldbi, int64_t m, int64_t n, int p, __nv_bfloat16* W, int64_t ldw, int64_t col0, int ncols,
            uint64_t seed, float* Y, int64_t ldy, double* normW2) {
    const int bpu = tc::pad_block16(p), bps = tc::pad_block16(ncols);
    Arena<float> ar;
    TcArena16 ta;
    int rc = ensure_arena<float>(h, m, n, bps, 1, &ar);
    if (rc == RQB_OK) rc = ensure_tc16(h, m, n, std::max(bpu, bps), &ta);
    if (rc != RQB_OK) return rc;
    Scal sc = scalars(h);
    Ctx cx;
    cx.stream = h->stream; cx.num_sms = h->num_sms; cx.st = sc.st;
    RQB_CK(cudaMemsetAsync(sc.st, 0, sizeof(DevState), h->stream));
    RQB_CK(tc::split_q16(cx, Qi, ldqi, m, p, bpu, ta.Qhi, ta.Qlo, ta.ldql, ta.Qt, ta.Qtl));
    RQB_CK(tc::stage_b16(cx, Bi, ldbi, p, n, bpu, ta.Bs, ta.Bsl));
    // the update reads and writes W through TMA: unaligned operands go
    // through aligned copies (A into the handle's W buffer, the result into
    // the adjoint workspace, copied out afterwards)
    const __nv_bfloat16* Ax;
    int64_t ldax;
    if ((rc = tma_source16(h, A, lda, m, n, &Ax, &ldax)) != RQB_OK) return rc;
    __nv_bfloat16* X = W;
    int64_t ldx = ldw;
    const bool copy_out = !tma_ok16(W, ldw);
    if (copy_out) {
        ldx = round_up(m, 8);
        if ((rc = h->adj.ensure(2 * (size_t)ldx * (size_t)n)) != RQB_OK) return rc;
        X = reinterpret_cast<__nv_bfloat16*>(h->adj.p);
    }
    RQB_CK(tc::update16(cx, Ax, ldax, X, ldx, m, n, ta.Qt, ta.Qtl, ta.Bs, ta.Bsl, bpu, sc.nrm, kNrmCap,
                        normW2 ? sc.s + 2 : nullptr));
    if (copy_out)
        RQB_CK(cudaMemcpy2DAsync(W, 2 * ldw, X, 2 * ldx, 2 * m, n, cudaMemcpyDeviceToDevice, h->stream));
    if ((rc = sketch_block16(h, cx, ta, X, ldx, m, n, col0, (int)ncols, bps, seed, ar.Y)) != RQB_OK) return rc;
    RQB_CK(cudaMemcpy2DAsync(Y, sizeof(float) * ldy, ar.Y, sizeof(float) * m, sizeof(float) * m, ncols,
                             cudaMemcpyDeviceToDevice, h->stream));
    if (normW2) RQB_CK(cudaMemcpyAsync(normW2, sc.s + 2, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return read_state(h, sc);
}
}  // namespace

extern "C" {

int rqb_sketch(rqb_handle h, const void* A, int64_t m, int64_t n, int64_t lda, int64_t col0, int64_t ncols,
               uint64_t seed, void* Y, int64_t ldy, double* normA2) {
    if (!h) return RQB_ERR_INVALID;
    if (check_matrix(A, m, n, lda) != RQB_OK || !Y || ncols < 1 || ncols > 256 || ldy < m || col0 < 0 ||
        (h->cfg.dtype == RQB_F64 && ncols > 128))
        return finish(h, RQB_ERR_INVALID);
    if (set_device(h) != RQB_OK) return finish(h, RQB_ERR_CUDA);
    if (h->cfg.dtype == RQB_BF16)
        return finish(h, !tc::shape_ok(m, n) ? RQB_ERR_UNSUPPORTED
                                             : sketch_bf16(h, static_cast<const __nv_bfloat16*>(A), m, n, lda, col0,
                                                           (int)ncols, seed, static_cast<float*>(Y), ldy, normA2));
    if (use_tc(h, m, n))
        return finish(h, sketch_tc(h, static_cast<const float*>(A), m, n, lda, col0, (int)ncols, seed,
                                   static_cast<float*>(Y), ldy, normA2));
    int rc = (h->cfg.dtype == RQB_F64)
                 ? sketch_impl<double>(h, static_cast<const double*>(A), m, n, lda, col0, (int)ncols, seed,
                                       static_cast<double*>(Y), ldy, normA2)
                 : sketch_impl<float>(h, static_cast<const float*>(A), m, n, lda, col0, (int)ncols, seed,
                                      static_cast<float*>(Y), ldy, normA2);
    return finish(h, rc);
}

int rqb_orth(rqb_handle h, const void* Y, int64_t m, int64_t p, int64_t ldy, const void* Qbar, int64_t kprev,
             int64_t ldqb, void* Qi, int64_t ldqi) {
    if (!h) return RQB_ERR_INVALID;
    if (check_matrix(Y, m, p, ldy) != RQB_OK || !Qi || ldqi < m || p > m || p > max_block(h) || kprev < 0 ||
        (kprev > 0 && (!Qbar || ldqb < m)) || kprev + p > m)
        return finish(h, RQB_ERR_INVALID);
    if (set_device(h) != RQB_OK) return finish(h, RQB_ERR_CUDA);
    int rc = (h->cfg.dtype == RQB_F64)
                 ? orth_impl<double>(h, static_cast<const double*>(Y), m, (int)p, ldy,
                                     static_cast<const double*>(Qbar), kprev, ldqb, static_cast<double*>(Qi), ldqi)
                 : orth_impl<float>(h, static_cast<const float*>(Y), m, (int)p, ldy, static_cast<const float*>(Qbar),
                                    kprev, ldqb, static_cast<float*>(Qi), ldqi);
    return finish(h, rc);
}

int rqb_project(rqb_handle h, const void* Qi, int64_t m, int64_t p, int64_t ldqi, const void* A, int64_t n,
                int64_t lda, void* Bi, int64_t ldbi, double* normB2) {
    if (!h) return RQB_ERR_INVALID;
    if (check_matrix(Qi, m, p, ldqi) != RQB_OK || check_matrix(A, m, n, lda) != RQB_OK || !Bi || ldbi < p ||
        p > max_block(h))
        return finish(h, RQB_ERR_INVALID);
    if (set_device(h) != RQB_OK) return finish(h, RQB_ERR_CUDA);
    if (h->cfg.dtype == RQB_BF16)
        return finish(h, !tc::shape_ok(m, n)
                             ? RQB_ERR_UNSUPPORTED
                             : project_bf16(h, static_cast<const float*>(Qi), m, (int)p, ldqi,
                                            static_cast<const __nv_bfloat16*>(A), n, lda, static_cast<float*>(Bi),
                                            ldbi, normB2));
    if (use_tc(h, m, n))
        return finish(h, project_tc(h, static_cast<const float*>(Qi), m, (int)p, ldqi, static_cast<const float*>(A),
                                    n, lda, static_cast<float*>(Bi), ldbi, normB2));
    int rc = (h->cfg.dtype == RQB_F64)
                 ? project_impl<double>(h, static_cast<const double*>(Qi), m, (int)p, ldqi,
                                        static_cast<const double*>(A), n, lda, static_cast<double*>(Bi), ldbi, normB2)
                 : project_impl<float>(h, static_cast<const float*>(Qi), m, (int)p, ldqi,
                                       static_cast<const float*>(A), n, lda, static_cast<float*>(Bi), ldbi, normB2);
    return finish(h, rc);
}

int rqb_downdate_sketch(rqb_handle h, const void* A, int64_t lda, const void* Qi, int64_t ldqi, const void* Bi,
                        int64_t ldbi, int64_t m, int64_t n, int64_t p, void* W, int64_t ldw, int64_t col0,
                        int64_t ncols, uint64_t seed, void* Y, int64_t ldy, double* normW2) {
    if (!h) return RQB_ERR_INVALID;
    if (check_matrix(A, m, n, lda) != RQB_OK || check_matrix(Qi, m, p, ldqi) != RQB_OK ||
        check_matrix(Bi, p, n, ldbi) != RQB_OK || check_matrix(W, m, n, ldw) != RQB_OK || !Y || ldy < m ||
        ncols < 1 || ncols > max_block(h) || p > max_block(h) || col0 < 0 ||
        (A == W && lda != ldw))
        return finish(h, RQB_ERR_INVALID);
    if (set_device(h) != RQB_OK) return finish(h, RQB_ERR_CUDA);
    if (h->cfg.dtype == RQB_BF16)
        return finish(h, !tc::shape_ok(m, n)
                             ? RQB_ERR_UNSUPPORTED
                             : dd_bf16(h, static_cast<const __nv_bfloat16*>(A), lda, static_cast<const float*>(Qi),
                                       ldqi, static_cast<const float*>(Bi), ldbi, m, n, (int)p,
                                       static_cast<__nv_bfloat16*>(W), ldw, col0, (int)ncols, seed,
                                       static_cast<float*>(Y), ldy, normW2));
    if (use_tc(h, m, n))
        return finish(h, dd_tc(h, static_cast<const float*>(A), lda, static_cast<const float*>(Qi), ldqi,
                               static_cast<const float*>(Bi), ldbi, m, n, (int)p, static_cast<float*>(W), ldw, col0,
                               (int)ncols, seed, static_cast<float*>(Y), ldy, normW2));
    int rc = (h->cfg.dtype == RQB_F64)
                 ? dd_impl<double>(h, static_cast<const double*>(A), lda, static_cast<const double*>(Qi), ldqi,
                                   static_cast<const double*>(Bi), ldbi, m, n, (int)p, static_cast<double*>(W), ldw,
                                   col0, (int)ncols, seed, static_cast<double*>(Y), ldy, normW2)
                 : dd_impl<float>(h, static_cast<const float*>(A), lda, static_cast<const float*>(Qi), ldqi,
                                  static_cast<const float*>(Bi), ldbi, m, n, (int)p, static_cast<float*>(W), ldw, col0,
                                  (int)ncols, seed, static_cast<float*>(Y), ldy, normW2);
    return finish(h, rc);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// X = Q B, and the adjoint of A -> Q Q^T A (fixed Omega)
namespace {

template <typename T>
int reconstruct_impl(rqb_handle h, T* X, int64_t ldx) {
    Scal sc = scalars(h);
    Ctx cx;
    cx.stream = h->stream; cx.num_sms = h->num_sms; cx.st = sc.st;
    NNArgs<T> a;
    a.m = h->last_m; a.K = h->last_k; a.nc = (int)h->last_n; a.nout = (int)h->last_n;
    a.X = reinterpret_cast<const T*>(h->q.p); a.ldx = h->ldq;
    a.C = reinterpret_cast<const T*>(h->b.p); a.csk = 1; a.csj = h->ldb; a.c_rowmajor = false;
    a.Out = X; a.ldo = ldx;
    RQB_CK(gemm_nn<T>(cx, a));
    RQB_CK(cudaStreamSynchronize(h->stream));
    return RQB_OK;
}

// dA = Q (Q^T G) + (I - Q Q^T)(G B^T + A (G^T Q)) R^{-T} Omega^T,  R = B Omega
template <typename T>
int backward_impl(rqb_handle h, const T* G, int64_t ldg, T* dA, int64_t ldda) {
    const int64_t m = h->last_m, n = h->last_n, k = h->last_k;
    const T* A = reinterpret_cast<const T*>(h->last_A);
    const int64_t lda = h->last_lda;
    const T* Q = reinterpret_cast<const T*>(h->q.p);
    const T* B = reinterpret_cast<const T*>(h->b.p);
    const int64_t ldq = h->ldq, ldb = h->ldb;
    // workspace
    const size_t part_cap = std::max<size_t>((size_t)4 * k * std::max(m, n), (size_t)8 * m * 256);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    const size_t oOm = take(sizeof(T) * n * k), oR = take(sizeof(T) * k * k), oRd = take(sizeof(double) * k * k);
    const size_t oRi = take(sizeof(T) * k * k), oQtG = take(sizeof(T) * k * n), oM1 = take(sizeof(T) * m * k);
    const size_t oGtQ = take(sizeof(T) * n * k), oQtM = take(sizeof(T) * k * k), oN = take(sizeof(T) * m * k);
    const size_t oP = take(sizeof(T) * part_cap);
    int rc = h->adj.ensure(off);
    if (rc != RQB_OK) return rc;
    char* base = reinterpret_cast<char*>(h->adj.p);
    T* Om = reinterpret_cast<T*>(base + oOm);
    T* R = reinterpret_cast<T*>(base + oR);
    double* Rd = reinterpret_cast<double*>(base + oRd);
    T* Rinv = reinterpret_cast<T*>(base + oRi);
    T* QtG = reinterpret_cast<T*>(base + oQtG);
    T* M1 = reinterpret_cast<T*>(base + oM1);
    T* GtQ = reinterpret_cast<T*>(base + oGtQ);
    T* QtM = reinterpret_cast<T*>(base + oQtM);
    T* Nm = reinterpret_cast<T*>(base + oN);
    T* part = reinterpret_cast<T*>(base + oP);
    Scal sc = scalars(h);
    Ctx cx;
    cx.stream = h->stream; cx.num_sms = h->num_sms; cx.st = sc.st;

    // Omega (n x k, row-major) and R = B Omega, R^{-1}
    RQB_CK(launch_omega<T>(cx, n, 0, (int)k, (int)k, h->last_seed, Om, k, 1));
    {
        NNArgs<T> a;
        a.m = k; a.K = n; a.nc = (int)k; a.nout = (int)k;
        a.X = B; a.ldx = ldb;
        a.C = Om; a.csk = k; a.csj = 1; a.c_rowmajor = true;
        a.Out = R; a.ldo = k;
        a.part = part; a.part_cap = part_cap; a.allow_split = 1;
        RQB_CK(gemm_nn<T>(cx, a));
    }
    RQB_CK(launch_to_double<T>(cx, k, k, R, k, Rd, k));
    RQB_CK(tri_inverse<T>(cx, Rd, (int)k, Rinv));
    // dA = Q (Q^T G)
    RQB_CK(gemm_tn<T>(cx, m, (int)k, n, Q, ldq, G, ldg, QtG, k, part, part_cap, nullptr, 0, nullptr));
    {
        NNArgs<T> a;
        a.m = m; a.K = k; a.nc = (int)n; a.nout = (int)n;
        a.X = Q; a.ldx = ldq;
        a.C = QtG; a.csk = 1; a.csj = k; a.c_rowmajor = false;
        a.Out = dA; a.ldo = ldda;
        RQB_CK(gemm_nn<T>(cx, a));
    }
    // M1 = G B^T + A (G^T Q)
    {
        NNArgs<T> a;
        a.m = m; a.K = n; a.nc = (int)k; a.nout = (int)k;
        a.X = G; a.ldx = ldg;
        a.C = B; a.csk = ldb; a.csj = 1; a.c_rowmajor = true;   // C(c, j) = B(j, c)
        a.Out = M1; a.ldo = m;
        a.part = part; a.part_cap = part_cap; a.allow_split = 1;
        RQB_CK(gemm_nn<T>(cx, a));
    }
    RQB_CK(gemm_tn<T>(cx, m, (int)n, k, G, ldg, Q, ldq, GtQ, n, part, part_cap, nullptr, 0, nullptr));
    {
        NNArgs<T> a;
        a.m = m; a.K = n; a.nc = (int)k; a.nout = (int)k;
        a.X = A; a.ldx = lda;
        a.C = GtQ; a.csk = 1; a.csj = n; a.c_rowmajor = false;
        a.Out = M1; a.ldo = m;
        a.Yin = M1; a.ldyin = m; a.alpha = T(1); a.beta = T(1);
        a.part = part; a.part_cap = part_cap; a.allow_split = 1;
        RQB_CK(gemm_nn<T>(cx, a));
    }
    // M1 -= Q (Q^T M1)
    RQB_CK(gemm_tn<T>(cx, m, (int)k, k, Q, ldq, M1, m, QtM, k, part, part_cap, nullptr, 0, nullptr));
    {
        NNArgs<T> a;
        a.m = m; a.K = k; a.nc = (int)k; a.nout = (int)k;
        a.X = Q; a.ldx = ldq;
        a.C = QtM; a.csk = 1; a.csj = k; a.c_rowmajor = false;
        a.Out = M1; a.ldo = m;
        a.Yin = M1; a.ldyin = m; a.alpha = T(-1); a.beta = T(1);
        a.part = part; a.part_cap = part_cap; a.allow_split = 1;
        RQB_CK(gemm_nn<T>(cx, a));
    }
    // N = M1 R^{-T};  dA += N Omega^T
    {
        NNArgs<T> a;
        a.m = m; a.K = k; a.nc = (int)k; a.nout = (int)k;
        a.X = M1; a.ldx = m;
        a.C = Rinv; a.csk = k; a.csj = 1; a.c_rowmajor = true;  // C(c, j) = Rinv(j, c)
        a.Out = Nm; a.ldo = m;
        RQB_CK(gemm_nn<T>(cx, a));
    }
    {
        NNArgs<T> a;
        a.m = m; a.K = k; a.nc = (int)n; a.nout = (int)n;
        a.X = Nm; a.ldx = m;
        a.C = Om; a.csk = 1; a.csj = k; a.c_rowmajor = false;   // C(c, j) = Omega(j, c)
        a.Out = dA; a.ldo = ldda;
        a.Yin = dA; a.ldyin = ldda; a.alpha = T(1); a.beta = T(1);
        RQB_CK(gemm_nn<T>(cx, a));
    }
    int err = read_state(h, sc);
    return err;
}

}  // namespace

extern "C" int rqb_reconstruct(rqb_handle h, void* X, int64_t ldx) {
    if (!h) return RQB_ERR_INVALID;
    if (!h->have_factor || !X || ldx < h->last_m) return finish(h, RQB_ERR_INVALID);
    if (set_device(h) != RQB_OK) return finish(h, RQB_ERR_CUDA);
    int rc = (h->cfg.dtype == RQB_F64) ? reconstruct_impl<double>(h, static_cast<double*>(X), ldx)
                                       : reconstruct_impl<float>(h, static_cast<float*>(X), ldx);
    return finish(h, rc);
}

extern "C" int rqb_svd(rqb_handle h, int64_t r, void* U, int64_t ldu, double* S, void* Vt, int64_t ldvt) {
    if (!h) return RQB_ERR_INVALID;
    if (!h->have_factor || r < 1 || r > h->last_k || r > (int64_t)1 << 30 || !U || !S || !Vt || ldu < h->last_m ||
        ldvt < r)
        return finish(h, RQB_ERR_INVALID);
    if (set_device(h) != RQB_OK) return finish(h, RQB_ERR_CUDA);
    const int k = (int)h->last_k;
    int rc = h->svdbuf.ensure(svd_scratch_bytes(h->last_m, h->last_n, k, (int)r));
    if (rc != RQB_OK) return finish(h, rc);
    Scal sc = scalars(h);
    Ctx cx;
    cx.stream = h->stream; cx.num_sms = h->num_sms; cx.st = sc.st;
    int sweeps = 0;
    if (h->cfg.dtype == RQB_F64)
        rc = svd_lowrank<double>(cx, h->last_m, h->last_n, k, (int)r, static_cast<const double*>(h->q.p), h->ldq,
                                 static_cast<const double*>(h->b.p), h->ldb, static_cast<double*>(U), ldu, S,
                                 static_cast<double*>(Vt), ldvt, h->svdbuf.p, h->svdbuf.bytes, &sweeps);
    else
        rc = svd_lowrank<float>(cx, h->last_m, h->last_n, k, (int)r, static_cast<const float*>(h->q.p), h->ldq,
                                static_cast<const float*>(h->b.p), h->ldb, static_cast<float*>(U), ldu, S,
                                static_cast<float*>(Vt), ldvt, h->svdbuf.p, h->svdbuf.bytes, &sweeps);
    h->stats.kernel_launches = cx.launches;
    h->stats.svd_sweeps = sweeps;
    return finish(h, rc);
}

extern "C" int rqb_wait_selftest(rqb_handle h, double* waited_ms) {
    if (!h) return RQB_ERR_INVALID;
    if (set_device(h) != RQB_OK) return finish(h, RQB_ERR_CUDA);
    Scal sc = scalars(h);
    Ctx cx;
    cx.stream = h->stream; cx.num_sms = h->num_sms; cx.st = sc.st;
    unsigned long long* dns = reinterpret_cast<unsigned long long*>(sc.s + 15);
    RQB_CK(cudaMemsetAsync(sc.st, 0, sizeof(DevState), h->stream));
    RQB_CK(tc::wait_selftest(cx, dns));
    unsigned long long ns = 0;
    RQB_CK(cudaMemcpyAsync(&ns, dns, sizeof(ns), cudaMemcpyDeviceToHost, h->stream));
    const int err = read_state(h, sc);
    if (waited_ms) *waited_ms = (double)ns * 1e-6;
    return finish(h, err);
}

extern "C" int rqb_backward(rqb_handle h, const void* dL_dX, int64_t ldg, void* dL_dA, int64_t ldda) {
    if (!h) return RQB_ERR_INVALID;
    if (!h->have_factor || !dL_dX || !dL_dA || ldg < h->last_m || ldda < h->last_m) return finish(h, RQB_ERR_INVALID);
    if (h->cfg.power != 0 || h->cfg.dtype == RQB_BF16) return finish(h, RQB_ERR_UNSUPPORTED);
    if (set_device(h) != RQB_OK) return finish(h, RQB_ERR_CUDA);
    RQB_CK(cudaMemsetAsync(scalars(h).st, 0, sizeof(DevState), h->stream));
    int rc = (h->cfg.dtype == RQB_F64)
                 ? backward_impl<double>(h, static_cast<const double*>(dL_dX), ldg, static_cast<double*>(dL_dA), ldda)
                 : backward_impl<float>(h, static_cast<const float*>(dL_dX), ldg, static_cast<float*>(dL_dA), ldda);
    return finish(h, rc);
}

extern "C" int rqb_factor_batched(rqb_handle h, int64_t count, const void* const* A, const int64_t* m,
                                  const int64_t* n, const int64_t* lda, const double* eps, int64_t b, uint64_t seed,
                                  const void** Q, int64_t* ldq, const void** B, int64_t* ldb, int64_t* k,
                                  int* status) {
    if (!h) return RQB_ERR_INVALID;
    if (count < 1 || !A || !m || !n || !lda || !eps || !Q || !ldq || !B || !ldb || !k || !status || b < 1 || b > 32)
        return finish(h, RQB_ERR_INVALID);
    for (int64_t t = 0; t < count; ++t)
        if (check_matrix(A[t], m[t], n[t], lda[t]) != RQB_OK || !(eps[t] >= 0.0) || !std::isfinite(eps[t]))
            return finish(h, RQB_ERR_INVALID);
    if (h->cfg.dtype != RQB_F32 || h->cfg.power != 0) return finish(h, RQB_ERR_UNSUPPORTED);
    if (set_device(h) != RQB_OK) return finish(h, RQB_ERR_CUDA);
    std::memset(&h->stats, 0, sizeof(h->stats));
    float ms = 0.f;
    int launches = 0, width = 0;
    int rc = rqb::batched::factor_batched(h->stream, h->num_sms, count, A, m, n, lda, eps, b, seed, h->cfg.max_rank,
                                          Q, ldq, B, ldb, k, status, &h->bat_out, &h->bat_out_bytes, &h->bat_work,
                                          &h->bat_work_bytes, &h->bat_cache, &ms, &launches, &width);
    h->have_factor = false;
    h->stats.kernel_launches = launches;
    h->stats.tile_width = width;
    h->stats.phase_ms[RQB_PHASE_SKETCH] = ms;   // the whole batch
    h->stats.phase_calls[RQB_PHASE_SKETCH] = 1;
    return finish(h, rc);
}
