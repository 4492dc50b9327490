// rqb_noalloc.cu -- the sketch step (Y = A Omega) for callers that cannot
// allocate device memory.
//
// Some callers run where cudaMalloc is not available to them: inside code that
// must not touch the allocator (a real-time loop, a host callback, a memory
// pool that owns the whole device), or in a process whose allocator is
// instrumented or capped by someone else.  rqb_sketch_noalloc serves them: it
// needs no handle and allocates nothing.  Its scratch (the Omega block, the
// split-K partial sums of the sketch and the FP64 partials of ||A||_F^2) lives
// in one file-scope __device__ array of RQB_NOALLOC_SCRATCH_BYTES, which every
// GPU that loads this library holds until the process exits.
#include <cstring>
#include <mutex>

#include "rqb_engine.h"

namespace {

constexpr size_t kScratchBytes = RQB_NOALLOC_SCRATCH_BYTES;
constexpr int kNrmSlots = 8192;
constexpr int kMaxDevices = 64;

// The shared scratch.  In host code this name is only a stand-in for the
// symbol; the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per
// device, with that device current).
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return RQB_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return RQB_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return RQB_OK;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

template <typename T>
int sketch_noalloc(const T* A, int64_t m, int64_t n, int64_t lda, int64_t col0, int p, uint64_t seed, T* Y,
                   int64_t ldy, double* normA2, cudaStream_t stream) {
    const int bp = p <= 32 ? 32 : p <= 64 ? 64 : p <= 128 ? 128 : 256;
    // scratch layout: [FP64 scalar | FP64 norm partials | Omega n x bp | partials ...]
    const size_t off_nrm = 256;
    const size_t off_om = align256(off_nrm + sizeof(double) * kNrmSlots);
    const size_t om_bytes = sizeof(T) * (size_t)n * (size_t)bp;
    const size_t off_part = align256(off_om + om_bytes);
    if (off_part > kScratchBytes) return RQB_ERR_SCRATCH_LIMIT;
    // one FP64 norm partial per row tile of the product; the tile height is
    // gemm_nn's: 128 rows for FP32 up to 128 columns, 64 rows for FP32 at 256
    // columns and for every FP64 product
    const int64_t bm = (sizeof(T) == 4 && bp <= 128) ? 128 : 64;
    if (normA2 && (m + bm - 1) / bm > kNrmSlots) return RQB_ERR_SCRATCH_LIMIT;
    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != RQB_OK) return rc;
    char* s = static_cast<char*>(base);
    double* scal = reinterpret_cast<double*>(s);
    double* nrm = reinterpret_cast<double*>(s + off_nrm);
    T* Om = reinterpret_cast<T*>(s + off_om);
    T* part = reinterpret_cast<T*>(s + off_part);

    rqb::Ctx cx;
    cx.stream = stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&cx.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return RQB_ERR_CUDA;
    }
    // every scratch word the kernels read is written earlier in this call
    // (Omega including its zero padding, each split's partial, each norm slot)
    if (rqb::launch_omega<T>(cx, n, col0, p, bp, seed, Om, bp, 1) != cudaSuccess) return RQB_ERR_CUDA;
    rqb::NNArgs<T> a;
    a.m = m; a.K = n; a.nc = bp; a.nout = p;
    a.X = A; a.ldx = lda;
    a.C = Om; a.csk = bp; a.csj = 1; a.c_rowmajor = true;
    a.Out = Y; a.ldo = ldy;
    a.part = part; a.part_cap = (kScratchBytes - off_part) / sizeof(T); a.allow_split = 1;
    if (normA2) { a.nrm_part = nrm; a.nrm_cap = kNrmSlots; a.nrm_out = scal; }
    if (rqb::gemm_nn<T>(cx, a) != cudaSuccess) {
        cudaGetLastError();
        return RQB_ERR_CUDA;
    }
    if (normA2) {
        if (cudaMemcpyAsync(normA2, scal, sizeof(double), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess) {
            cudaGetLastError();
            return RQB_ERR_CUDA;
        }
    }
    return RQB_OK;
}

}  // namespace

extern "C" int rqb_sketch_noalloc(int32_t dtype, const void* A, int64_t m, int64_t n, int64_t lda, int64_t col0,
                                  int64_t ncols, uint64_t seed, void* Y, int64_t ldy, double* normA2,
                                  void* stream) {
    if (!A || !Y || m <= 0 || n <= 0 || lda < m || ldy < m || col0 < 0 || ncols < 1 ||
        (dtype != RQB_F32 && dtype != RQB_F64) || ncols > (dtype == RQB_F64 ? 128 : 256))
        return RQB_ERR_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return (dtype == RQB_F64)
               ? sketch_noalloc<double>(static_cast<const double*>(A), m, n, lda, col0, (int)ncols, seed,
                                        static_cast<double*>(Y), ldy, normA2, s)
               : sketch_noalloc<float>(static_cast<const float*>(A), m, n, lda, col0, (int)ncols, seed,
                                       static_cast<float*>(Y), ldy, normA2, s);
}
