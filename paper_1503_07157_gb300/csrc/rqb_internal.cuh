// rqb_internal.cuh -- shared device helpers of the GB300 randQB_b library.
//
// Everything here is internal to librqb.so: Philox4x32-10 and Box-Muller for
// the Gaussian test matrix (Fig. randQB_b line (2)), guarded global loads,
// and the launch-side bookkeeping used by every kernel file.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rqb.h"

namespace rqb {

// ---------------------------------------------------------------------------
// Device-side error word: kernels never trap; they record a status here and
// return, and the host reads it back after the launch sequence.
struct DevState {
    double normA2;     // ||A||_F^2
    double E;          // running downdate ||A||^2 - sum ||B_j||^2
    double normB2;     // ||B_i||^2 of the current block
    double D;          // direct ||A^(i)||_F^2 of the current block
    int32_t err;       // first error code recorded by a kernel (rqb_status)
    int32_t flag;      // stop decision of the current block (see StopFlag)
    int32_t near_id;   // second CholeskyQR passes factored by the near-identity expansion
    int32_t fused_gram;  // second Grams formed from the re-projection's product
};

enum StopFlag : int32_t { kContinue = 0, kStop = 1, kAmbiguous = 2 };

__device__ __forceinline__ void record_error(DevState* st, int code) {
    if (st) atomicCAS(&st->err, 0, code);
}

// Programmatic dependent launch (PTX griddepcontrol, sm_90 and later).  A
// kernel launched with the programmatic stream-serialisation attribute may
// start while the kernel before it in the stream is still running:
// pdl_wait() blocks until that kernel has completed and its memory is
// visible (for a normally launched kernel it returns at once), and
// pdl_trigger() lets the next such kernel launch before this one ends.
// Kernels that take part call pdl_trigger() first and pdl_wait() before
// their first global-memory access, read or write.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
//   (x0, x1, x2, x3) -> (hi(M1 x2) ^ x1 ^ k0, lo(M1 x2), hi(M0 x0) ^ x3 ^ k1, lo(M0 x0))
// with the key advanced by the Weyl constants between rounds.
struct Philox4 {
    uint32_t v[4];
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1) {
    const uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
    const uint32_t kWeylA = 0x9E3779B9u, kWeylB = 0xBB67AE85u;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t hiA = __umulhi(kMulA, c0), loA = kMulA * c0;
        const uint32_t hiB = __umulhi(kMulB, c2), loB = kMulB * c2;
        const uint32_t n0 = hiB ^ c1 ^ k0;
        const uint32_t n2 = hiA ^ c3 ^ k1;
        c0 = n0; c1 = loB; c2 = n2; c3 = loA;
        k0 += kWeylA;
        k1 += kWeylB;
    }
    Philox4 r;
    r.v[0] = c0; r.v[1] = c1; r.v[2] = c2; r.v[3] = c3;
    return r;
}

// Entry (r, c) of the Gaussian matrix Omega: the Philox block at counter
// (r, c/2, 0, 0) under key (seed low, seed high) gives u1, u2 in (0, 1);
// Box-Muller returns sqrt(-2 ln u1) cos(2 pi u2) for even c and
// sqrt(-2 ln u1) sin(2 pi u2) for odd c.
__device__ __forceinline__ double gaussian_f64(uint64_t seed, int64_t r, int64_t c) {
    const Philox4 x = philox4x32_10((uint32_t)r, (uint32_t)(c >> 1), 0u, 0u,
                                    (uint32_t)(seed & 0xffffffffull), (uint32_t)(seed >> 32));
    const double u1 = (__uint2double_rn(x.v[0] >> 5) * 67108864.0 + __uint2double_rn(x.v[1] >> 6) + 0.5) *
                      1.1102230246251565404e-16;  // 2^-53
    const double u2 = (__uint2double_rn(x.v[2] >> 5) * 67108864.0 + __uint2double_rn(x.v[3] >> 6) + 0.5) *
                      1.1102230246251565404e-16;
    const double rad = sqrt(-2.0 * log(u1));
    double s, co;
    sincospi(2.0 * u2, &s, &co);
    return (c & 1) ? rad * s : rad * co;
}

__device__ __forceinline__ float gaussian_f32(uint64_t seed, int64_t r, int64_t c) {
    const Philox4 x = philox4x32_10((uint32_t)r, (uint32_t)(c >> 1), 0u, 0u,
                                    (uint32_t)(seed & 0xffffffffull), (uint32_t)(seed >> 32));
    const float u1 = ((float)(x.v[0] >> 9) + 0.5f) * 1.1920928955078125e-7f;  // 2^-23
    const float u2 = ((float)(x.v[2] >> 9) + 0.5f) * 1.1920928955078125e-7f;
    const float rad = sqrtf(-2.0f * logf(u1));
    float s, co;
    sincospif(2.0f * u2, &s, &co);
    return (c & 1) ? rad * s : rad * co;
}

// Entries (r, 2 j) and (r, 2 j + 1) of Omega from their one Philox block:
// the values gaussian_f32 gives for those two columns, bit for bit.
__device__ __forceinline__ void gaussian_pair_f32(uint64_t seed, int64_t r, int64_t j, float* even, float* odd) {
    const Philox4 x = philox4x32_10((uint32_t)r, (uint32_t)j, 0u, 0u, (uint32_t)(seed & 0xffffffffull),
                                    (uint32_t)(seed >> 32));
    const float u1 = ((float)(x.v[0] >> 9) + 0.5f) * 1.1920928955078125e-7f;  // 2^-23
    const float u2 = ((float)(x.v[2] >> 9) + 0.5f) * 1.1920928955078125e-7f;
    const float rad = sqrtf(-2.0f * logf(u1));
    float s, co;
    sincospif(2.0f * u2, &s, &co);
    *even = rad * co;
    *odd = rad * s;
}

template <typename T>
__device__ __forceinline__ T gaussian(uint64_t seed, int64_t r, int64_t c);
template <>
__device__ __forceinline__ double gaussian<double>(uint64_t seed, int64_t r, int64_t c) {
    return gaussian_f64(seed, r, c);
}
template <>
__device__ __forceinline__ float gaussian<float>(uint64_t seed, int64_t r, int64_t c) {
    return gaussian_f32(seed, r, c);
}

// ---------------------------------------------------------------------------
// 16-byte vectors: 4 floats or 2 doubles.
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int N = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int N = 2; };

template <typename T>
__device__ __forceinline__ bool aligned16(const T* p) {
    return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

// Asynchronous 16-byte global -> shared copies (cp.async): both addresses
// 16-byte aligned; the bytes beyond src_bytes (0..16) are zero-filled.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------------------
// Host-side helpers shared by the .cu files.
struct LaunchCounter {
    int count = 0;
};

inline int ceil_div_i(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace rqb
