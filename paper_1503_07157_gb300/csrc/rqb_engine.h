// rqb_engine.h -- host-side launchers of the SIMT kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <utility>

#include "rqb_internal.cuh"

namespace rqb {

// Host-side allocation-failure injection for tests (rqb_inject_alloc_failure):
// true when the device allocation about to be made must fail as if
// cudaMalloc had returned an out-of-memory error.
bool alloc_should_fail();

// Raises `kernel`'s dynamic shared-memory limit to at least `bytes` on the
// current device.  The attribute is per device; the largest limit set for
// each (kernel, device) is remembered under a lock (several host threads and
// several devices may launch the same kernel) and never lowered, so calls
// with different sizes cannot undo one another.
inline cudaError_t smem_limit_once(const void* kernel, int bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> limit;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_pair(kernel, dev);
    const auto it = limit.find(key);
    if (it != limit.end() && it->second >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) limit[key] = bytes;
    return e;
}

template <typename K>
inline cudaError_t smem_limit(K kernel, int bytes) {
    return smem_limit_once(reinterpret_cast<const void*>(kernel), bytes);
}

// Programmatic dependent launches (pdl_wait / pdl_trigger in the kernels):
// on unless the environment sets RQB_PDL=0.
bool pdl_enabled();

// kernel<<<grid, block, smem, stream>>>(args...), with programmatic stream
// serialisation when pdl_enabled(): the launch may overlap the kernel before
// it in the stream up to the new kernel's pdl_wait().  Only kernels that call
// pdl_wait() before touching global memory are launched this way.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                              Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

struct Ctx {
    cudaStream_t stream = nullptr;
    int num_sms = 1;
    DevState* st = nullptr;
    int launches = 0;
};

// Arguments of Out = alpha * X C + beta * Yin (see k_gemm_nn).
template <typename T>
struct NNArgs {
    int64_t m = 0, K = 0;
    int nc = 0, nout = 0;
    const T* X = nullptr;
    int64_t ldx = 0;
    const T* C = nullptr;
    int64_t csk = 0, csj = 0;
    bool c_rowmajor = false;
    T* Out = nullptr;
    int64_t ldo = 0;
    T* part = nullptr;          // split partials (only when alpha = 1, beta = 0)
    size_t part_cap = 0;        // elements
    const T* Yin = nullptr;
    int64_t ldyin = 0;
    T alpha = T(1), beta = T(0);
    int allow_split = 0;
    double* nrm_part = nullptr; // non-NULL: also ||X||_F^2 into *nrm_out
    int nrm_cap = 0;
    double* nrm_out = nullptr;
};

template <typename T>
cudaError_t launch_omega(Ctx& cx, int64_t n, int64_t col0, int ncols, int ncols_pad, uint64_t seed, T* out,
                         int64_t rs, int64_t cs);
template <typename T>
cudaError_t launch_sumsq(Ctx& cx, int64_t m, int64_t n, const T* X, int64_t ldx, double* part, int part_cap,
                         double* out);
cudaError_t launch_sum_doubles(Ctx& cx, const double* part, int count, double* out);
template <typename TP, typename TO>
cudaError_t launch_reduce_split(Ctx& cx, int64_t rows, int64_t cols, int splits, const TP* part, int64_t ldp,
                                int64_t zstride, TO* out, int64_t ldo, double* sq_part, int sq_cap,
                                double* sq_out, double alpha = 1.0, double beta = 0.0, const TO* Yin = nullptr,
                                int64_t ldyin = 0, int sym = 0);
template <typename T>
cudaError_t gemm_nn(Ctx& cx, const NNArgs<T>& a);
template <typename T>
cudaError_t gemm_tn(Ctx& cx, int64_t m, int pn, int64_t qn, const T* X, int64_t ldx, const T* Y, int64_t ldy,
                    T* Out, int64_t ldo, T* part, size_t part_cap_elems, double* sq_part, int sq_cap,
                    double* sq_out);
template <typename T>
cudaError_t gemm_tn_f64acc(Ctx& cx, int64_t m, int pn, int64_t qn, const T* X, int64_t ldx, const T* Y,
                           int64_t ldy, double* Out, int64_t ldo, double* part, size_t part_cap_elems,
                           bool exact, bool sym = false);
// second_pass: G is the Gram of an already orthonormalised panel (the
// second CholeskyQR pass); the factor is first tried by the near-identity
// expansion (near_identity), the elimination running only when it does not
// apply.
template <typename T>
cudaError_t chol_inv(Ctx& cx, double* G, int bp, int p, double* R, T* Rinv, bool fp64_factor, double* scratch,
                     size_t scratch_doubles, bool second_pass = false);
template <typename T>
cudaError_t upper_inverse(Ctx& cx, const double* R, int bp, T* Rinv);
template <typename T>
cudaError_t chol_inv_blocked(Ctx& cx, double* G, int bp, int p, double* R, T* Rinv, double tol, double* scratch,
                             size_t scratch_doubles, bool fp64, const int* skip);
// Second CholeskyQR pass (rqb_chol.cu): R and Rinv by the near-identity
// expansion when ||G - I||_F <= tau, with *skip (device) set to 1 so that the
// elimination launched after it returns at once, else *skip = 0.  work holds
// kNearIdWork(bp) doubles (the norm's parts, the flags and, for FP32
// factors, the iterated route's five bp x bp FP32 matrices).
constexpr int kNearIdParts = 64;
inline size_t kNearIdWork(int bp) { return kNearIdParts + 2 + (5 * (size_t)bp * bp + 1) / 2; }
template <typename T>
cudaError_t near_identity(Ctx& cx, const double* G, int bp, int p, double* R, T* Rinv, double tau, double* work,
                          int* skip);
template <typename T>
cudaError_t downdate_sketch(Ctx& cx, int64_t m, int64_t n, int p, int bp, const T* Wsrc, int64_t ldws,
                            const T* Qi, int64_t ldq, const T* Bi, int64_t ldb, const T* Om, T* Wdst,
                            int64_t ldwd, T* Y, int64_t ldy, T* part, size_t part_cap_elems, double* nrm_part,
                            int nrm_cap, double* nrm_out);
template <typename T>
cudaError_t tri_inverse(Ctx& cx, const double* R, int kdim, T* Rinv);
template <typename T>
cudaError_t launch_to_double(Ctx& cx, int64_t rows, int64_t cols, const T* src, int64_t lds, double* dst,
                             int64_t ldd);
cudaError_t launch_set_norm(Ctx& cx, const double* nrm);
cudaError_t launch_stop_after_b(Ctx& cx, const double* nb2, double eps2, double tau_rel, int fixed);
cudaError_t launch_stop_direct(Ctx& cx, const double* d2, double eps2, bool always = false);

// Low-rank SVD of Q B (rqb_svd.cu): U (m x r), S_host (r, descending),
// Vt (r x n); returns an rqb_status.
size_t svd_scratch_bytes(int64_t m, int64_t n, int k, int r);
template <typename T>
int svd_lowrank(Ctx& cx, int64_t m, int64_t n, int k, int r, const T* Q, int64_t ldq, const T* B, int64_t ldb,
                T* U, int64_t ldu, double* S_host, T* Vt, int64_t ldvt, void* scratch, size_t scratch_bytes,
                int* sweeps_out);

}  // namespace rqb
