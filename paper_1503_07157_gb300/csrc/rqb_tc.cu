// rqb_tc.cu -- split-TF32 tensor-core kernels of randQB_b (RQB_PREC_TF32X3).
//
// The three products of a block of Fig. randQB_b that touch all of A run on
// tcgen05 with FP32 accumulators in TMEM, operands staged by TMA:
//   sketch   Y = W Omega_i        line (3), Omega_i rounded to TF32 (exact),
//                                 W split into hi + lo: 2 MMA passes
//   project  B_i^T = W^T Q_i      line (4), W and Q_i split: 3 passes
//   update   W <- W - Q_i B_i     line (5), Q_i and B_i split: 3 passes
// A split FP32 value x = hi + lo has hi = x (the MMA reads its TF32 part)
// and lo = rna_tf32(x - trunc_tf32(x)); the products hi*hi + hi*lo + lo*hi
// keep about 21 bits of each term.  The panel (Gram, Cholesky, re-projection) and the
// stopping test stay on the SIMT kernels with FP64 accumulation.
//
// Sketch and project reduce over a long K (n or m), so they run stream-K:
// one CTA per SM walks a contiguous range of (tile, K-chunk) units, writes
// one partial accumulator per tile segment it touches, and a second kernel
// sums the partials of each tile in CTA order (deterministic).  The update
// has K = b and walks whole output tiles.
//
// Warp roles in each CTA: warp 0 issues TMA loads, warp 1 owns TMEM and
// issues the MMAs (one thread), the remaining warps split operands into the
// MMA layout and drain accumulators.  Every wait is bounded (rqb_tc.cuh); on
// expiry the CTA drains its copies and MMAs, frees TMEM and records
// RQB_ERR_TIMEOUT.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "rqb_engine.h"
#include "rqb_internal.cuh"
#include "rqb_tc.cuh"
#include "rqb_tc.h"

namespace rqb {
namespace tc {
namespace {

enum Role { kSketch = 0, kProject = 1 };

struct StreamKParams {
    CUtensorMap mx;    // W: sketch box {128 rows, 32 cols}, no swizzle; project box {32 rows, 128 cols}, SW128
    CUtensorMap mw;    // Omega (sketch) or Q_i (project): box {32, np}, SW128
    CUtensorMap mwl;   // lo part of Q_i (project)
    float* part;       // P * G partial accumulators of 128 x np floats
    DevState* st;
    long long U;       // units = tiles * C
    int C;             // K chunks per tile
    int P;             // CTAs
    int G;             // partial slots per CTA
    int np;            // MMA N
    double* nrm_part = nullptr;  // sketch only, optional: ||X||_F^2, one FP64 partial per CTA
    // BF16 sketch generating Omega in shared memory (k_streamk16 with GEN):
    // rows om_n, global columns om_col0 .., om_p of them valid, seed
    long long om_n = 0, om_col0 = 0;
    int om_p = 0;
    unsigned long long om_seed = 0;
    // split-TF32 projection over two X matrices side by side: tiles >= tsplit
    // of X come from mx2 (its tile t - tsplit)
    CUtensorMap mx2;
    int tsplit = 0x7fffffff;
    // nonzero *gate: the launch does nothing (a product made unnecessary by
    // an earlier kernel's device-side decision)
    const int* gate = nullptr;
};

__host__ __device__ __forceinline__ long long unit_begin(long long U, int P, int p) { return U * p / P; }

constexpr int kMaxCover = 64;   // CTAs that may share one tile

// ---------------------------------------------------------------------------
// Stream-K sketch / project.
//
// The tensor core accumulates in FP32 with a one-sided rounding, so a long
// chain of MMAs into one accumulator drifts toward zero in proportion to its
// length (measured: about 2^-25.5 of the value per MMA, 2e-6 after 96
// MMAs).  The chain is therefore cut every kPeriod K-chunks (24 MMAs for the
// projection, 16 for the sketch): the MMA
// alternates between two TMEM accumulators, and the eight epilogue warps add
// each finished period into FP32 running sums in registers (round to
// nearest), which are written out at the end of a tile segment.
constexpr int kPeriod = 2;

template <int ROLE, int NP>
struct StreamKCfg {
    static constexpr int S = (ROLE == kProject && NP > 128) ? 2 : 3;   // TMA stages
    static constexpr uint32_t kW = (uint32_t)NP * 128u;                 // Omega / Q tile bytes
    static constexpr uint32_t kCv = ROLE == kSketch ? 2 * kTileBytes : kTileBytes;  // one conversion slot
    static constexpr size_t kSmem =
        (size_t)S * (kTileBytes + kW) + (ROLE == kProject ? (size_t)S * kW : 0) + 2 * (size_t)kCv + 1024;
};

template <int ROLE, int NP>
__global__ void __launch_bounds__(320, 1) k_streamk(const __grid_constant__ StreamKParams p) {
    pdl_wait();
    if (p.gate && *p.gate) return;   // before any barrier, shared memory or TMEM
    using Cfg = StreamKCfg<ROLE, NP>;
    constexpr int S = Cfg::S;
    constexpr uint32_t kW = Cfg::kW;
    constexpr int kHalf = NP / 2;          // accumulator columns per epilogue warp
    __shared__ __align__(8) uint64_t full[S], empty[S], cvfull[2], cvempty[2], accfull[2], accempty[2], drain;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ double nred[8];
    extern __shared__ uint8_t dsm[];
    uint8_t* base = dsm + (((smem_u32(dsm) + 1023u) & ~1023u) - smem_u32(dsm));
    uint8_t* sX = base;
    uint8_t* sW = sX + S * kTileBytes;
    uint8_t* sWl = sW + S * kW;
    uint8_t* sCv = (ROLE == kProject) ? sWl + S * kW : sWl;   // sketch: 2 x (hi, lo); project: 2 x lo
    constexpr uint32_t ncols = 2u * (uint32_t)NP;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int* ab = &abort_flag;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&cvfull[s], 8); mbar_init(&cvempty[s], 1);
            mbar_init(&accfull[s], 1); mbar_init(&accempty[s], 8);
        }
        mbar_init(&drain, 1);
        abort_flag = 0;
        fence_mbar_init();
        prefetch_map(&p.mx);
        prefetch_map(&p.mw);
        if (ROLE == kProject) prefetch_map(&p.mwl);
        if (ROLE == kProject && p.tsplit != 0x7fffffff) prefetch_map(&p.mx2);
    }
    if (warp == 1) tmem_alloc(&tmem_base, ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const long long u0 = unit_begin(p.U, p.P, blockIdx.x), u1 = unit_begin(p.U, p.P, blockIdx.x + 1);
    // unit u is chunk kc = u % C of tile u / C; a period ends at every kPeriod-th
    // chunk of a tile, at the tile's last chunk and at the end of the CTA's range
    auto seg_end = [&](long long u) { return u + 1 == u1 || (u + 1) % p.C == 0; };
    auto period_end = [&](long long u) { return seg_end(u) || ((u % p.C) + 1) % kPeriod == 0; };

    if (warp == 0) {
        if (lane == 0) {
            long long q = 0;
            for (long long u = u0; u < u1; ++u, ++q) {
                const int s = (int)(q % S);
                const uint32_t r = (uint32_t)(q / S);
                if (r > 0 && !mbar_wait(&empty[s], (r - 1) & 1u, ab)) break;
                const int t = (int)(u / p.C), kc = (int)(u % p.C);
                if (ROLE == kSketch) {
                    mbar_arrive_expect_tx(&full[s], kTileBytes + kW);
                    tma_load_2d(sX + s * kTileBytes, &p.mx, t * kBM, kc * kKC, &full[s]);
                    tma_load_2d(sW + s * kW, &p.mw, kc * kKC, 0, &full[s]);
                } else {
                    mbar_arrive_expect_tx(&full[s], kTileBytes + 2u * kW);
                    const bool second = t >= p.tsplit;
                    tma_load_2d(sX + s * kTileBytes, second ? &p.mx2 : &p.mx, kc * kKC,
                                (second ? t - p.tsplit : t) * kBM, &full[s]);
                    tma_load_2d(sW + s * kW, &p.mw, kc * kKC, 0, &full[s]);
                    tma_load_2d(sWl + s * kW, &p.mwl, kc * kKC, 0, &full[s]);
                }
            }
            // the last loads issued must land before the CTA's shared memory is released
            for (long long qq = (q > S ? q - S : 0); qq < q; ++qq)
                mbar_wait(&full[qq % S], (uint32_t)(qq / S) & 1u, ab, false);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_tf32(NP);
            int g = 0;             // periods issued
            bool first = true;     // next chunk starts a period
            long long q = 0;
            for (long long u = u0; u < u1; ++u, ++q) {
                const int s = (int)(q % S), cs = (int)(q & 1);
                const uint32_t r = (uint32_t)(q / S), cr = (uint32_t)(q >> 1);
                if (!mbar_wait(&full[s], r & 1u, ab)) break;
                if (!mbar_wait(&cvfull[cs], cr & 1u, ab)) break;
                const int abuf = g & 1, use = g >> 1;
                if (first && use > 0 && !mbar_wait(&accempty[abuf], (uint32_t)(use - 1) & 1u, ab)) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(abuf * NP);
                if (ROLE == kSketch) {
                    const uint32_t a0 = smem_u32(sCv + cs * Cfg::kCv), a1 = a0 + kTileBytes;
                    const uint32_t b0 = smem_u32(sW + s * kW);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_tf32(d, desc_k_sw128(a0 + kk * 32), desc_k_sw128(b0 + kk * 32), idesc,
                                 (first && kk == 0) ? 0u : 1u);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_tf32(d, desc_k_sw128(a1 + kk * 32), desc_k_sw128(b0 + kk * 32), idesc, 1u);
                } else {
                    const uint32_t a0 = smem_u32(sX + s * kTileBytes), a1 = smem_u32(sCv + cs * Cfg::kCv);
                    const uint32_t b0 = smem_u32(sW + s * kW), b1 = smem_u32(sWl + s * kW);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_tf32(d, desc_k_sw128(a0 + kk * 32), desc_k_sw128(b0 + kk * 32), idesc,
                                 (first && kk == 0) ? 0u : 1u);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_tf32(d, desc_k_sw128(a0 + kk * 32), desc_k_sw128(b1 + kk * 32), idesc, 1u);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_tf32(d, desc_k_sw128(a1 + kk * 32), desc_k_sw128(b0 + kk * 32), idesc, 1u);
                }
                mma_commit(&empty[s]);
                mma_commit(&cvempty[cs]);
                if (period_end(u)) {
                    mma_commit(&accfull[abuf]);
                    ++g;
                    first = true;
                } else {
                    first = false;
                }
            }
            // every MMA issued has completed before TMEM is released
            mma_commit(&drain);
            mbar_wait(&drain, 0, ab, false);
        }
    } else {
        const int ct = threadIdx.x - 64;          // 0..255
        const int e = warp - 2;                   // 0..7
        const int quarter = warp & 3;             // TMEM lanes this warp may read
        const int half = e >> 2;                  // accumulator columns [half NP/2, (half+1) NP/2)
        const int row = quarter * 32 + lane;      // accumulator row held by this thread
        float acc[kHalf];
#pragma unroll
        for (int i = 0; i < kHalf; ++i) acc[i] = 0.f;
        double nrm = 0.0;   // ||X||_F^2 of the tiles this thread converts
        int g = 0;
        long long q = 0;
        for (long long u = u0; u < u1; ++u, ++q) {
            const int s = (int)(q % S), cs = (int)(q & 1);
            const uint32_t r = (uint32_t)(q / S), cr = (uint32_t)(q >> 1);
            bool ok = mbar_wait(&full[s], r & 1u, ab);
            if (ok && cr > 0) ok = mbar_wait(&cvempty[cs], (cr - 1) & 1u, ab);
            if (!__all_sync(0xffffffffu, ok)) break;
            if (ROLE == kSketch) {
                // raw tile [32 cols][128 rows] -> K-major rows (hi, lo): thread ct
                // converts columns [16 h, 16 h + 16) of row ct % 128, h = ct / 128
                const int rr = ct & (kBM - 1), h = ct >> 7;
                const float* raw = reinterpret_cast<const float*>(sX + s * kTileBytes);
                float x[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) x[j] = raw[(16 * h + j) * kBM + rr];
                if (p.nrm_part) {
                    // the stream-K units partition the matrix, and the TMA box
                    // fills zeros past its edges: every entry is squared once.
                    // Each square is split exactly (e = fma(x, x, -x*x)) and the
                    // 16 of a unit are summed with TwoSum in FP32 pairs, then
                    // added in FP64
                    float hi = 0.f, lo = 0.f;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float p2 = __fmul_rn(x[j], x[j]);
                        const float e2 = fmaf(x[j], x[j], -p2);
                        const float t = __fadd_rn(hi, p2);
                        const float z = __fsub_rn(t, hi);
                        lo += __fadd_rn(__fsub_rn(hi, __fsub_rn(t, z)), __fsub_rn(p2, z)) + e2;
                        hi = t;
                    }
                    nrm += (double)hi + (double)lo;
                }
                uint8_t* hi = sCv + cs * Cfg::kCv;
                uint8_t* lo = hi + kTileBytes;
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4) {
                    const int c = 4 * h + c4;
                    const uint32_t off = (uint32_t)rr * 128u + ((uint32_t)(c ^ (rr & 7)) << 4);
                    *reinterpret_cast<float4*>(hi + off) =
                        make_float4(x[4 * c4], x[4 * c4 + 1], x[4 * c4 + 2], x[4 * c4 + 3]);
                    *reinterpret_cast<float4*>(lo + off) =
                        make_float4(tf32_lo(x[4 * c4]), tf32_lo(x[4 * c4 + 1]), tf32_lo(x[4 * c4 + 2]),
                                    tf32_lo(x[4 * c4 + 3]));
                }
            } else {
                const float4* src = reinterpret_cast<const float4*>(sX + s * kTileBytes);
                float4* dst = reinterpret_cast<float4*>(sCv + cs * Cfg::kCv);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float4 v = src[ct + 256 * i];
                    dst[ct + 256 * i] = make_float4(tf32_lo(v.x), tf32_lo(v.y), tf32_lo(v.z), tf32_lo(v.w));
                }
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&cvfull[cs]);
            if (period_end(u)) {
                const int abuf = g & 1, use = g >> 1;
                const bool okw = mbar_wait(&accfull[abuf], (uint32_t)use & 1u, ab);
                if (!__all_sync(0xffffffffu, okw)) break;
                tc_fence_after();
                const uint32_t tl =
                    tmem + (uint32_t)(abuf * NP + half * kHalf) + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
                for (int c0 = 0; c0 < kHalf; c0 += 16) {
                    float v[16];
                    tmem_ld16(tl + (uint32_t)c0, v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) acc[c0 + i] += v[i];
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&accempty[abuf]);
                ++g;
                if (seg_end(u)) {
                    const int seg = (int)(u / p.C - u0 / p.C);
                    float* slot = p.part + ((size_t)blockIdx.x * p.G + seg) * (size_t)kBM * NP;
                    if (ROLE == kSketch) {
#pragma unroll
                        for (int i = 0; i < kHalf; ++i) slot[(size_t)(half * kHalf + i) * kBM + row] = acc[i];
                    } else {
                        float4* d4 = reinterpret_cast<float4*>(slot + (size_t)row * NP + half * kHalf);
#pragma unroll
                        for (int i = 0; i < kHalf / 4; ++i)
                            d4[i] = make_float4(acc[4 * i], acc[4 * i + 1], acc[4 * i + 2], acc[4 * i + 3]);
                    }
#pragma unroll
                    for (int i = 0; i < kHalf; ++i) acc[i] = 0.f;
                }
            }
        }
        if (ROLE == kSketch && p.nrm_part) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
            if (lane == 0) nred[e] = nrm;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, ncols);
    if (threadIdx.x == 0 && abort_flag) record_error(p.st, RQB_ERR_TIMEOUT);
    if (ROLE == kSketch && p.nrm_part && threadIdx.x == 64) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < 8; ++w) t += nred[w];
        p.nrm_part[blockIdx.x] = t;
    }
}

// ---------------------------------------------------------------------------
// BF16 storage path (A and its residual in BF16, products on kind::f16 with
// FP32 accumulation).  A 128-row x 128-byte tile holds 64 BF16 of K and an MMA
// step covers K = 16, so a chunk is four MMAs as in the TF32 kernels.
//   sketch   Y = W Omega_i: W read MN-major straight from TMA (two 64-row
//            boxes), Omega_i in BF16 (exact), one pass
//   project  B_i^T = W^T Q_i: W K-major, Q_i split into BF16 hi + lo, two passes
constexpr int kKC16 = 64;    // K per chunk of the BF16 kernels

template <int ROLE, int NP>
struct StreamK16Cfg {
    static constexpr int S = (ROLE == kProject && NP > 128) ? 2 : 4;    // TMA stages
    static constexpr uint32_t kW = (uint32_t)NP * 128u;                  // Omega / Q tile bytes
    static constexpr uint32_t kStage = kTileBytes + (ROLE == kProject ? 2u : 1u) * kW;
    static constexpr size_t kSmem = (size_t)S * kStage + 1024;
};

// Omega's K-chunk kc of the BF16 sketch written by 256 threads (ct) into the
// operand stage dst in the layout a TMA load with the 128-byte swizzle gives:
// one 128-byte row of 64 K values per column c, 16-byte group j of row c at
// group j ^ (c % 8).  Entry (kk, c) is the binary32 Gaussian at row
// 64 kc + kk and global column om_col0 + c rounded to BF16 (nearest even),
// zero past row om_n or column om_p: the values k_omega_bf16 writes.
template <int NP>
__device__ __forceinline__ void gen_omega_chunk(uint8_t* dst, int kc, const StreamKParams& p, int ct) {
    constexpr int kPairs = NP / 2;
    constexpr int kRowStep = 256 / kPairs;
    const int c0 = 2 * (ct % kPairs);
    const long long g0 = p.om_col0 + c0;
    for (int kk = ct / kPairs; kk < kKC16; kk += kRowStep) {
        const long long r = (long long)kc * kKC16 + kk;
        float v0 = 0.f, v1 = 0.f;
        if (r < p.om_n && c0 < p.om_p) {
            if ((g0 & 1) == 0) {
                float a, b;
                gaussian_pair_f32(p.om_seed, r, g0 >> 1, &a, &b);
                v0 = a;
                v1 = (c0 + 1 < p.om_p) ? b : 0.f;
            } else {
                v0 = gaussian_f32(p.om_seed, r, g0);
                if (c0 + 1 < p.om_p) v1 = gaussian_f32(p.om_seed, r, g0 + 1);
            }
        }
        const uint32_t grp = (uint32_t)(kk >> 3), inr = (uint32_t)(kk & 7) * 2u;
        *reinterpret_cast<__nv_bfloat16*>(dst + (uint32_t)c0 * 128u + ((grp ^ (uint32_t)(c0 & 7)) << 4) + inr) =
            __float2bfloat16_rn(v0);
        *reinterpret_cast<__nv_bfloat16*>(dst + (uint32_t)(c0 + 1) * 128u + ((grp ^ (uint32_t)((c0 + 1) & 7)) << 4) +
                                          inr) = __float2bfloat16_rn(v1);
    }
}

// GEN (sketch only): Omega is not loaded by TMA but generated per unit by the
// eight epilogue warps into the stage (gen_omega_chunk), which they may
// overwrite once the MMAs of the stage's previous use have completed.
template <int ROLE, int NP, bool GEN = false>
__global__ void __launch_bounds__(320, 1) k_streamk16(const __grid_constant__ StreamKParams p) {
    pdl_wait();
    using Cfg = StreamK16Cfg<ROLE, NP>;
    constexpr int S = Cfg::S;
    constexpr uint32_t kW = Cfg::kW, kStage = Cfg::kStage;
    constexpr int kHalf = NP / 2;
    static_assert(!GEN || ROLE == kSketch, "Omega is generated only by the sketch");
    __shared__ __align__(8) uint64_t full[S], empty[S], omfull[S], accfull[2], accempty[2], drain;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ double nred16[8];
    // sketch with nrm_part: the epilogue warps also square every W tile, so a
    // stage is free once the MMAs and those eight warps are done with it
    const bool nrm = (ROLE == kSketch) && (p.nrm_part != nullptr);
    extern __shared__ uint8_t dsm[];
    uint8_t* base = dsm + (((smem_u32(dsm) + 1023u) & ~1023u) - smem_u32(dsm));
    constexpr uint32_t ncols = 2u * (uint32_t)NP;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int* ab = &abort_flag;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], nrm ? 9 : 1);
            if (GEN) mbar_init(&omfull[s], 8);
        }
        for (int s = 0; s < 2; ++s) { mbar_init(&accfull[s], 1); mbar_init(&accempty[s], 8); }
        mbar_init(&drain, 1);
        abort_flag = 0;
        fence_mbar_init();
        prefetch_map(&p.mx);
        if (!GEN) prefetch_map(&p.mw);
        if (ROLE == kProject) prefetch_map(&p.mwl);
    }
    if (warp == 1) tmem_alloc(&tmem_base, ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const long long u0 = unit_begin(p.U, p.P, blockIdx.x), u1 = unit_begin(p.U, p.P, blockIdx.x + 1);
    auto seg_end = [&](long long u) { return u + 1 == u1 || (u + 1) % p.C == 0; };
    // the one-pass sketch accumulates four K-chunks (16 MMAs, as the
    // split-TF32 sketch) per period, the two-pass projection two (16 MMAs)
    constexpr int kPer16 = (ROLE == kSketch) ? 2 * kPeriod : kPeriod;
    auto period_end = [&](long long u) { return seg_end(u) || ((u % p.C) + 1) % kPer16 == 0; };

    if (warp == 0) {
        if (lane == 0) {
            long long q = 0;
            for (long long u = u0; u < u1; ++u, ++q) {
                const int s = (int)(q % S);
                const uint32_t r = (uint32_t)(q / S);
                if (r > 0 && !mbar_wait(&empty[s], (r - 1) & 1u, ab)) break;
                const int t = (int)(u / p.C), kc = (int)(u % p.C);
                uint8_t* st = base + s * kStage;
                if (ROLE == kSketch) {
                    mbar_arrive_expect_tx(&full[s], GEN ? kTileBytes : kTileBytes + kW);
                    tma_load_2d(st, &p.mx, t * kBM, kc * kKC16, &full[s]);
                    tma_load_2d(st + kTileBytes / 2, &p.mx, t * kBM + 64, kc * kKC16, &full[s]);
                    if (!GEN) tma_load_2d(st + kTileBytes, &p.mw, kc * kKC16, 0, &full[s]);
                } else {
                    mbar_arrive_expect_tx(&full[s], kTileBytes + 2u * kW);
                    tma_load_2d(st, &p.mx, kc * kKC16, t * kBM, &full[s]);
                    tma_load_2d(st + kTileBytes, &p.mw, kc * kKC16, 0, &full[s]);
                    tma_load_2d(st + kTileBytes + kW, &p.mwl, kc * kKC16, 0, &full[s]);
                }
            }
            for (long long qq = (q > S ? q - S : 0); qq < q; ++qq)
                mbar_wait(&full[qq % S], (uint32_t)(qq / S) & 1u, ab, false);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(NP, ROLE == kSketch ? 1 : 0);
            int g = 0;
            bool first = true;
            long long q = 0;
            for (long long u = u0; u < u1; ++u, ++q) {
                const int s = (int)(q % S);
                const uint32_t r = (uint32_t)(q / S);
                if (!mbar_wait(&full[s], r & 1u, ab)) break;
                if (GEN && !mbar_wait(&omfull[s], r & 1u, ab)) break;
                const int abuf = g & 1, use = g >> 1;
                if (first && use > 0 && !mbar_wait(&accempty[abuf], (uint32_t)(use - 1) & 1u, ab)) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(abuf * NP);
                const uint32_t a0 = smem_u32(base + s * kStage), b0 = a0 + kTileBytes;
                if (ROLE == kSketch) {
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_bf16(d, desc_mn_sw128(a0 + kk * 2048, kTileBytes / 2), desc_k_sw128(b0 + kk * 32), idesc,
                                 (first && kk == 0) ? 0u : 1u);
                } else {
                    const uint32_t b1 = b0 + kW;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_bf16(d, desc_k_sw128(a0 + kk * 32), desc_k_sw128(b0 + kk * 32), idesc,
                                 (first && kk == 0) ? 0u : 1u);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_bf16(d, desc_k_sw128(a0 + kk * 32), desc_k_sw128(b1 + kk * 32), idesc, 1u);
                }
                mma_commit(&empty[s]);
                if (period_end(u)) {
                    mma_commit(&accfull[abuf]);
                    ++g;
                    first = true;
                } else {
                    first = false;
                }
            }
            mma_commit(&drain);
            mbar_wait(&drain, 0, ab, false);
        }
    } else {
        const int e = warp - 2;
        const int quarter = warp & 3;
        const int half = e >> 2;
        const int row = quarter * 32 + lane;
        float acc[kHalf];
#pragma unroll
        for (int i = 0; i < kHalf; ++i) acc[i] = 0.f;
        double sq = 0.0;     // ||W||_F^2 of the tile parts this thread squares (nrm)
        int g = 0;
        long long q = 0;
        for (long long u = u0; u < u1; ++u, ++q) {
            if (nrm) {
                // the stream-K units partition W and the TMA boxes zero-fill
                // past its edges: every entry is squared once.  A BF16 square
                // is exact in FP32; the 32 of a thread are summed with TwoSum
                // in FP32 pairs, then added in FP64
                const int s = (int)(q % S);
                const uint32_t r = (uint32_t)(q / S);
                const bool okn = mbar_wait(&full[s], r & 1u, ab);
                if (!__all_sync(0xffffffffu, okn)) break;
                const uint4* tile = reinterpret_cast<const uint4*>(base + s * kStage);
                float hi = 0.f, lo = 0.f;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint4 w4 = tile[((int)threadIdx.x - 64) + 256 * i];
                    const uint32_t w[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float v = __uint_as_float((j & 1) ? (w[j >> 1] & 0xffff0000u) : (w[j >> 1] << 16));
                        const float p2 = __fmul_rn(v, v);
                        const float t = __fadd_rn(hi, p2);
                        const float z = __fsub_rn(t, hi);
                        lo += __fadd_rn(__fsub_rn(hi, __fsub_rn(t, z)), __fsub_rn(p2, z));
                        hi = t;
                    }
                }
                sq += (double)hi + (double)lo;
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
            }
            if constexpr (GEN) {
                const int s = (int)(q % S);
                const uint32_t r = (uint32_t)(q / S);
                const bool okg = (r == 0) || mbar_wait(&empty[s], (r - 1) & 1u, ab);
                if (!__all_sync(0xffffffffu, okg)) break;
                gen_omega_chunk<NP>(base + s * kStage + kTileBytes, (int)(u % p.C), p, (int)threadIdx.x - 64);
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&omfull[s]);
            }
            if (!period_end(u)) continue;
            const int abuf = g & 1, use = g >> 1;
            const bool okw = mbar_wait(&accfull[abuf], (uint32_t)use & 1u, ab);
            if (!__all_sync(0xffffffffu, okw)) break;
            tc_fence_after();
            const uint32_t tl = tmem + (uint32_t)(abuf * NP + half * kHalf) + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
            for (int c0 = 0; c0 < kHalf; c0 += 16) {
                float v[16];
                tmem_ld16(tl + (uint32_t)c0, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) acc[c0 + i] += v[i];
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&accempty[abuf]);
            ++g;
            if (seg_end(u)) {
                const int seg = (int)(u / p.C - u0 / p.C);
                float* slot = p.part + ((size_t)blockIdx.x * p.G + seg) * (size_t)kBM * NP;
                if (ROLE == kSketch) {
#pragma unroll
                    for (int i = 0; i < kHalf; ++i) slot[(size_t)(half * kHalf + i) * kBM + row] = acc[i];
                } else {
                    float4* d4 = reinterpret_cast<float4*>(slot + (size_t)row * NP + half * kHalf);
#pragma unroll
                    for (int i = 0; i < kHalf / 4; ++i)
                        d4[i] = make_float4(acc[4 * i], acc[4 * i + 1], acc[4 * i + 2], acc[4 * i + 3]);
                }
#pragma unroll
                for (int i = 0; i < kHalf; ++i) acc[i] = 0.f;
            }
        }
        if (nrm) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
            if (lane == 0) nred16[e] = sq;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, ncols);
    if (threadIdx.x == 0 && abort_flag) record_error(p.st, RQB_ERR_TIMEOUT);
    if (nrm && threadIdx.x == 64) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < 8; ++w) t += nred16[w];
        p.nrm_part[blockIdx.x] = t;
    }
}

// ---------------------------------------------------------------------------
// Update W_dst = W_src - Q_i B_i on 128 x NJ output tiles, K = bp in chunks of
// 32: D = Q_i^T-tile (M = rows) x B_i-tile (N = columns), three passes.
// Warps 2..9 drain the accumulator: thread (quarter, lane) owns row
// 32 quarter + lane, and the two warps of a quarter split the NJ columns
// into halves.  W travels by TMA in both directions, one half tile
// (128 x NJ/2 FP32) at a time through a ring of three buffers: warp 10 loads
// half tile h = 2 g + half of the CTA's g-th tile into buffer h mod 3, the
// four warps of that half replace it by the difference in shared memory and
// one of them stores it (TMA store) and hands the buffer back once the store
// has read it.  ||W_dst||_F^2 per CTA on the same pass.
struct UpdateParams {
    CUtensorMap mqt, mqtl;  // Q_i^T row-major (bp x m as {bp, m}), box {32, 128}
    CUtensorMap mbs, mbsl;  // B_i staged column-major (bp x n), box {32, NJ}
    CUtensorMap mws, mwd;   // W_src / W_dst, m x n column-major, box {128 rows, NJ / 2 columns}
    DevState* st;
    double* sq_part;        // per-CTA ||W_dst||_F^2 partials (FP64), or null
    long long m, n;
    int RT, CT, C;
    int sub;                // 1: W_dst = W_src - Q_i B_i; 0: W_dst = Q_i B_i (W_src unused)
};

constexpr int kUpdThreads = 352;   // warps 0 (operand TMA), 1 (MMA), 2..9 (epilogue), 10 (W loads)
constexpr int kWRing = 3;          // half-tile W buffers

template <int NJ, int S>
__global__ void __launch_bounds__(kUpdThreads, 1) k_update(const __grid_constant__ UpdateParams p) {
    pdl_wait();
    __shared__ __align__(8) uint64_t full[S], empty[S], accfull[2], accempty[2], wfull[kWRing], wempty[kWRing],
        drain;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ double red[8];
    extern __shared__ uint8_t dsm[];
    uint8_t* base = dsm + (((smem_u32(dsm) + 1023u) & ~1023u) - smem_u32(dsm));
    constexpr uint32_t kB = (uint32_t)NJ * 128u;           // one B tile (NJ rows x 128 B)
    constexpr uint32_t kStage = 2u * kTileBytes + 2u * kB;
    constexpr int kHalf = NJ / 2;
    constexpr uint32_t kWHalf = (uint32_t)kBM * kHalf * 4u;  // one FP32 half tile
    uint8_t* wbuf = base + S * kStage;
    constexpr uint32_t kCols = 2u * NJ;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int* ab = &abort_flag;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int s = 0; s < 2; ++s) { mbar_init(&accfull[s], 1); mbar_init(&accempty[s], 8); }
        for (int s = 0; s < kWRing; ++s) { mbar_init(&wfull[s], 1); mbar_init(&wempty[s], 1); }
        mbar_init(&drain, 1);
        abort_flag = 0;
        fence_mbar_init();
        prefetch_map(&p.mqt);
        prefetch_map(&p.mqtl);
        prefetch_map(&p.mbs);
        prefetch_map(&p.mbsl);
        prefetch_map(&p.mws);
        prefetch_map(&p.mwd);
    }
    if (warp == 1) tmem_alloc(&tmem_base, kCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const int T = p.RT * p.CT;

    if (warp == 0) {
        if (lane == 0) {
            long long q = 0;
            bool stop = false;
            for (int t = blockIdx.x; t < T && !stop; t += gridDim.x) {
                const int rt = t / p.CT, ctile = t % p.CT;
                for (int kc = 0; kc < p.C; ++kc, ++q) {
                    const int s = (int)(q % S);
                    const uint32_t r = (uint32_t)(q / S);
                    if (r > 0 && !mbar_wait(&empty[s], (r - 1) & 1u, ab)) { stop = true; break; }
                    uint8_t* st = base + s * kStage;
                    mbar_arrive_expect_tx(&full[s], kStage);
                    tma_load_2d(st, &p.mqt, kc * kKC, rt * kBM, &full[s]);
                    tma_load_2d(st + kTileBytes, &p.mqtl, kc * kKC, rt * kBM, &full[s]);
                    tma_load_2d(st + 2 * kTileBytes, &p.mbs, kc * kKC, ctile * NJ, &full[s]);
                    tma_load_2d(st + 2 * kTileBytes + kB, &p.mbsl, kc * kKC, ctile * NJ, &full[s]);
                }
            }
            for (long long qq = (q > S ? q - S : 0); qq < q; ++qq)
                mbar_wait(&full[qq % S], (uint32_t)(qq / S) & 1u, ab, false);
        }
    } else if (warp == 10) {
        if (lane == 0) {
            long long h = 0;
            bool stop = false;
            for (int t = blockIdx.x; t < T && !stop; t += gridDim.x) {
                for (int hf = 0; hf < 2; ++hf, ++h) {
                    const int b = (int)(h % kWRing);
                    const uint32_t use = (uint32_t)(h / kWRing);
                    if (use > 0 && !mbar_wait(&wempty[b], (use - 1) & 1u, ab)) { stop = true; break; }
                    if (p.sub) {
                        mbar_arrive_expect_tx(&wfull[b], kWHalf);
                        tma_load_2d(wbuf + b * kWHalf, &p.mws, (t / p.CT) * kBM, (t % p.CT) * NJ + hf * kHalf,
                                    &wfull[b]);
                    } else {
                        mbar_arrive(&wfull[b]);     // the buffer is free; nothing to load
                    }
                }
            }
            if (p.sub)
                for (long long hh = (h > kWRing ? h - kWRing : 0); hh < h; ++hh)
                    mbar_wait(&wfull[hh % kWRing], (uint32_t)(hh / kWRing) & 1u, ab, false);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_tf32(NJ);
            long long q = 0;
            int g = 0;
            bool stop = false;
            for (int t = blockIdx.x; t < T && !stop; t += gridDim.x, ++g) {
                const int abuf = g & 1, use = g >> 1;
                if (use > 0 && !mbar_wait(&accempty[abuf], (uint32_t)(use - 1) & 1u, ab)) break;
                const uint32_t d = tmem + (uint32_t)(abuf * NJ);
                for (int kc = 0; kc < p.C; ++kc, ++q) {
                    const int s = (int)(q % S);
                    const uint32_t r = (uint32_t)(q / S);
                    if (!mbar_wait(&full[s], r & 1u, ab)) { stop = true; break; }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(base + s * kStage), a1 = a0 + kTileBytes;
                    const uint32_t b0 = a0 + 2 * kTileBytes, b1 = b0 + kB;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_tf32(d, desc_k_sw128(a0 + kk * 32), desc_k_sw128(b0 + kk * 32), idesc,
                                 (kc == 0 && kk == 0) ? 0u : 1u);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_tf32(d, desc_k_sw128(a0 + kk * 32), desc_k_sw128(b1 + kk * 32), idesc, 1u);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_tf32(d, desc_k_sw128(a1 + kk * 32), desc_k_sw128(b0 + kk * 32), idesc, 1u);
                    mma_commit(&empty[s]);
                }
                if (stop) break;
                mma_commit(&accfull[abuf]);
            }
            mma_commit(&drain);
            mbar_wait(&drain, 0, ab, false);
        }
    } else {
        const int e = warp - 2;               // 0..7
        const int quarter = warp & 3;
        const int half = e >> 2;
        const bool issuer = (lane == 0 && (e & 3) == 0);
        const int row = quarter * 32 + lane;
        double sq = 0.0;
        int g = 0;
        for (int t = blockIdx.x; t < T; t += gridDim.x, ++g) {
            const int abuf = g & 1, use = g >> 1;
            const long long h = 2LL * g + half;
            const int b = (int)(h % kWRing);
            bool okw = mbar_wait(&accfull[abuf], (uint32_t)use & 1u, ab);
            if (okw) okw = mbar_wait(&wfull[b], (uint32_t)(h / kWRing) & 1u, ab);
            // the four warps of this half leave together (the barrier counts them)
            named_barrier(1 + half, 128);
            if (*ab || !okw) break;
            tc_fence_after();
            const int rt = t / p.CT, ctile = t % p.CT;
            const long long r = (long long)rt * kBM + row;
            const long long j0 = (long long)ctile * NJ + half * kHalf;
            const bool rok = r < p.m;
            // half tile column-major: element (row, col) at col * 512 + row * 4
            float* wt = reinterpret_cast<float*>(wbuf + b * kWHalf) + row;
            const uint32_t tl = tmem + (uint32_t)(abuf * NJ + half * kHalf) + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
            for (int c0 = 0; c0 < kHalf; c0 += 16) {
                float v[16];
                tmem_ld16(tl + (uint32_t)c0, v);
                float sq16 = 0.f;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float d = p.sub ? wt[(c0 + i) * kBM] - v[i] : v[i];
                    wt[(c0 + i) * kBM] = d;
                    if (rok && j0 + c0 + i < p.n) sq16 = fmaf(d, d, sq16);
                }
                sq += (double)sq16;
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&accempty[abuf]);
            fence_async_smem();
            named_barrier(1 + half, 128);
            if (issuer) {
                tma_store_2d(&p.mwd, rt * kBM, ctile * NJ + half * kHalf, wbuf + b * kWHalf);
                bulk_commit();
                bulk_wait_read<0>();
                mbar_arrive(&wempty[b]);
            }
        }
        if (issuer) bulk_wait<0>();
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        if (lane == 0) red[e] = sq;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, kCols);
    if (threadIdx.x == 0) {
        if (abort_flag) record_error(p.st, RQB_ERR_TIMEOUT);
        if (p.sq_part) {
            double t = 0.0;
            for (int i = 0; i < 8; ++i) t += red[i];
            p.sq_part[blockIdx.x] = t;
        }
    }
}

// Wide split-TF32 update / product: the same as k_update on 128 x 256 tiles
// (N = 256 MMAs: a quarter fewer operand bytes per multiply-add), K in chunks
// of 16 (64-byte swizzle rows, 48 KB per stage) through three stages, and W
// in 128 x 32 eighths of the tile through a ring of four 16 KB buffers
// (warp 10 loads eighth w into slot w % 4 in update mode; one epilogue thread
// stores it and hands the previous slot back once that store has read it).
// TMEM: two 256-column accumulators.
constexpr int kKCt = 16;                            // K per chunk (one 64-byte swizzle row of FP32)
constexpr int kNJt = 256;                           // tile columns
constexpr int kStt = 3;                             // operand stages
constexpr int kWRt = 4;                             // W eighth buffers
constexpr uint32_t kQt = kBM * kKCt * 4;            // Q_i^T hi or lo chunk: 8 KB
constexpr uint32_t kBt = kNJt * kKCt * 4;           // B hi or lo chunk: 16 KB
constexpr uint32_t kStageT = 2 * kQt + 2 * kBt;     // 48 KB
constexpr uint32_t kWEt = kBM * 32 * 4;             // W eighth: 16 KB
constexpr size_t kUpdwSmem = (size_t)kStt * kStageT + (size_t)kWRt * kWEt + 1024;

__global__ void __launch_bounds__(kUpdThreads, 1) k_updatew(const __grid_constant__ UpdateParams p) {
    pdl_wait();
    __shared__ __align__(8) uint64_t full[kStt], empty[kStt], accfull[2], accempty[2], wfull[kWRt], wempty[kWRt],
        drain;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ double red[8];
    extern __shared__ uint8_t dsm[];
    uint8_t* base = dsm + (((smem_u32(dsm) + 1023u) & ~1023u) - smem_u32(dsm));
    uint8_t* wbuf = base + kStt * kStageT;
    constexpr uint32_t kCols = 2u * kNJt;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int* ab = &abort_flag;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStt; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int s = 0; s < 2; ++s) { mbar_init(&accfull[s], 1); mbar_init(&accempty[s], 8); }
        for (int s = 0; s < kWRt; ++s) { mbar_init(&wfull[s], 1); mbar_init(&wempty[s], 1); }
        mbar_init(&drain, 1);
        abort_flag = 0;
        fence_mbar_init();
        prefetch_map(&p.mqt);
        prefetch_map(&p.mqtl);
        prefetch_map(&p.mbs);
        prefetch_map(&p.mbsl);
        prefetch_map(&p.mws);
        prefetch_map(&p.mwd);
    }
    if (warp == 1) tmem_alloc(&tmem_base, kCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const int T = p.RT * p.CT;

    if (warp == 0) {
        if (lane == 0) {
            long long q = 0;
            bool stop = false;
            for (int t = blockIdx.x; t < T && !stop; t += gridDim.x) {
                const int rt = t / p.CT, ctile = t % p.CT;
                for (int kc = 0; kc < p.C; ++kc, ++q) {
                    const int s = (int)(q % kStt);
                    const uint32_t r = (uint32_t)(q / kStt);
                    if (r > 0 && !mbar_wait(&empty[s], (r - 1) & 1u, ab)) { stop = true; break; }
                    uint8_t* st = base + s * kStageT;
                    mbar_arrive_expect_tx(&full[s], kStageT);
                    tma_load_2d(st, &p.mqt, kc * kKCt, rt * kBM, &full[s]);
                    tma_load_2d(st + kQt, &p.mqtl, kc * kKCt, rt * kBM, &full[s]);
                    tma_load_2d(st + 2 * kQt, &p.mbs, kc * kKCt, ctile * kNJt, &full[s]);
                    tma_load_2d(st + 2 * kQt + kBt, &p.mbsl, kc * kKCt, ctile * kNJt, &full[s]);
                }
            }
            for (long long qq = (q > kStt ? q - kStt : 0); qq < q; ++qq)
                mbar_wait(&full[qq % kStt], (uint32_t)(qq / kStt) & 1u, ab, false);
        }
    } else if (warp == 10) {
        if (lane == 0) {
            long long w = 0;   // eighths issued
            bool stop = false;
            for (int t = blockIdx.x; t < T && !stop; t += gridDim.x) {
                for (int qq = 0; qq < 8; ++qq, ++w) {
                    const int slot = (int)(w % kWRt);
                    const long long use = w / kWRt;
                    if (use > 0 && !mbar_wait(&wempty[slot], (uint32_t)(use - 1) & 1u, ab)) { stop = true; break; }
                    if (p.sub) {
                        mbar_arrive_expect_tx(&wfull[slot], kWEt);
                        tma_load_2d(wbuf + slot * kWEt, &p.mws, (t / p.CT) * kBM, (t % p.CT) * kNJt + qq * 32,
                                    &wfull[slot]);
                    } else {
                        mbar_arrive(&wfull[slot]);   // the buffer is free; nothing to load
                    }
                }
            }
            if (p.sub)
                for (long long ww = (w > kWRt ? w - kWRt : 0); ww < w; ++ww)
                    mbar_wait(&wfull[ww % kWRt], (uint32_t)(ww / kWRt) & 1u, ab, false);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_tf32(kNJt);
            long long q = 0;
            int g = 0;
            bool stop = false;
            for (int t = blockIdx.x; t < T && !stop; t += gridDim.x, ++g) {
                const int abuf = g & 1, use = g >> 1;
                if (use > 0 && !mbar_wait(&accempty[abuf], (uint32_t)(use - 1) & 1u, ab)) break;
                const uint32_t d = tmem + (uint32_t)(abuf * kNJt);
                for (int kc = 0; kc < p.C; ++kc, ++q) {
                    const int s = (int)(q % kStt);
                    const uint32_t r = (uint32_t)(q / kStt);
                    if (!mbar_wait(&full[s], r & 1u, ab)) { stop = true; break; }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(base + s * kStageT), a1 = a0 + kQt;
                    const uint32_t b0 = a0 + 2 * kQt, b1 = b0 + kBt;
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk)
                        mma_tf32(d, desc_k_sw64(a0 + kk * 32), desc_k_sw64(b0 + kk * 32), idesc,
                                 (kc == 0 && kk == 0) ? 0u : 1u);
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk)
                        mma_tf32(d, desc_k_sw64(a0 + kk * 32), desc_k_sw64(b1 + kk * 32), idesc, 1u);
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk)
                        mma_tf32(d, desc_k_sw64(a1 + kk * 32), desc_k_sw64(b0 + kk * 32), idesc, 1u);
                    mma_commit(&empty[s]);
                }
                if (stop) break;
                mma_commit(&accfull[abuf]);
            }
            mma_commit(&drain);
            mbar_wait(&drain, 0, ab, false);
        }
    } else {
        const int e = warp - 2;
        const int quarter = warp & 3;                 // TMEM lanes this warp may read
        const int half = e >> 2;                      // columns [16 half, 16 half + 16) of each W eighth
        const bool issuer = (warp == 2 && lane == 0);
        const int row = quarter * 32 + lane;          // tile row of this thread
        double sq = 0.0;
        int g = 0;
        long long w = 0;                              // eighths consumed
        bool stop = false;
        for (int t = blockIdx.x; t < T && !stop; t += gridDim.x, ++g) {
            const int abuf = g & 1, use = g >> 1;
            const bool oka = mbar_wait(&accfull[abuf], (uint32_t)use & 1u, ab);
            const int rt = t / p.CT, ctile = t % p.CT;
            const long long r = (long long)rt * kBM + row;
            const bool rok = r < p.m;
            for (int qq = 0; qq < 8; ++qq, ++w) {
                const int slot = (int)(w % kWRt);
                bool okw = oka && mbar_wait(&wfull[slot], (uint32_t)(w / kWRt) & 1u, ab);
                // all eight warps leave together (the named barrier below counts them)
                named_barrier(1, 256);
                if (*ab || !okw) { stop = true; break; }
                tc_fence_after();
                const long long j0 = (long long)ctile * kNJt + qq * 32 + half * 16;
                // W eighth column-major: element (row, col) at col * 512 + row * 4
                float* wt = reinterpret_cast<float*>(wbuf + slot * kWEt) + row;
                const uint32_t tl =
                    tmem + (uint32_t)(abuf * kNJt + qq * 32 + half * 16) + ((uint32_t)(quarter * 32) << 16);
                float v[16];
                tmem_ld16(tl, v);
                float sq16 = 0.f;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int cl = half * 16 + i;
                    const float d = p.sub ? wt[cl * kBM] - v[i] : v[i];
                    wt[cl * kBM] = d;
                    if (rok && j0 + i < p.n) sq16 = fmaf(d, d, sq16);
                }
                sq += (double)sq16;
                if (qq == 7) {   // the accumulator is read: hand it back
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&accempty[abuf]);
                }
                fence_async_smem();
                named_barrier(1, 256);
                if (issuer) {
                    tma_store_2d(&p.mwd, rt * kBM, ctile * kNJt + qq * 32, wbuf + slot * kWEt);
                    bulk_commit();
                    // the previous eighth's store has read its buffer: hand it back
                    bulk_wait_read<1>();
                    if (w > 0) mbar_arrive(&wempty[(w - 1) % kWRt]);
                }
            }
        }
        if (issuer) bulk_wait<0>();
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        if (lane == 0) red[e] = sq;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, kCols);
    if (threadIdx.x == 0) {
        if (abort_flag) record_error(p.st, RQB_ERR_TIMEOUT);
        if (p.sq_part) {
            double t = 0.0;
            for (int i = 0; i < 8; ++i) t += red[i];
            p.sq_part[blockIdx.x] = t;
        }
    }
}

// ---------------------------------------------------------------------------
// Small kernels around the products.

// Omega_i in the K-major layout of the sketch: out[j + c ldo] = rna_tf32 of the
// binary32 Gaussian (j, col0 + c) for c < p, zero for p <= c < bp.
__global__ void k_omega_tf32(long long n, long long col0, int p, int bp, uint64_t seed, float* __restrict__ out,
                             long long ldo) {
    pdl_trigger();
    pdl_wait();
    const long long total = n * bp;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long j = e % n;
        const int c = (int)(e / n);
        out[j + c * ldo] = c < p ? tf32_rna(gaussian_f32(seed, j, col0 + c)) : 0.f;
    }
}

// From Q_i (m x p, column-major, ld ldq): Qhi = Q_i and its lo part Qlo
// (column-major, ld ldql, bp columns), Qt = Q_i^T as row-major m x bp and
// its lo part Qtl; columns p..bp-1 are zero.  32 x 32 tiles transposed
// through shared memory.  A nonzero *gate drops the column-major copies (the
// kernel then returns at once when Qt is NULL).
__global__ void k_split_q(const float* __restrict__ Qi, long long ldq, long long m, int p, int bp,
                          float* __restrict__ Qhi, float* __restrict__ Qlo, long long ldql, float* __restrict__ Qt,
                          float* __restrict__ Qtl, const int* __restrict__ gate) {
    pdl_trigger();
    pdl_wait();
    if (gate && *gate) {
        if (Qt == nullptr) return;
        Qhi = nullptr;
    }
    __shared__ float tile[32][33];
    const long long r0 = (long long)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
    for (int i = ty; i < 32; i += 8) {
        const long long r = r0 + tx;
        const int c = c0 + i;
        float v = 0.f;
        if (r < m && c < p) v = Qi[r + c * ldq];
        if (r < m && Qhi) {
            Qhi[r + c * ldql] = v;
            Qlo[r + c * ldql] = tf32_lo(v);
        }
        tile[i][tx] = v;
    }
    if (Qt == nullptr) return;     // column-major copies only
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        const long long r = r0 + i;
        const int c = c0 + tx;
        if (r < m) {
            const float v = tile[tx][i];
            Qt[r * bp + c] = v;
            Qtl[r * bp + c] = tf32_lo(v);
        }
    }
}

// Omega-layout copy of the re-projection coefficients: Om[j + c ldo] =
// rna_tf32(Ct[c + j ldc]) for j < kprev, c < np (Ct is C^T, np x kprev);
// with C32, also C32[j + c ldc32] = Ct[c + j ldc] rounded to FP32.
// Split-k parts of C^T C for the fused second-pass Gram.  C is kprev x np
// (FP32, ld ldc, k contiguous).  CTA (t, s) takes the 32 x 32 upper tile
// t = (I, J), I <= J (t = J (J + 1) / 2 + I), over k in [128 s, 128 s + 128),
// and writes its 1024 sums to part[(t KS + s) 1024 + i + 32 j] (KS =
// gridDim.y), in FP64.  Products are summed in FP32 over 32 k, and the four
// 32-k sums pairwise.
__global__ void __launch_bounds__(256) k_gram_part(const float* __restrict__ C, long long ldc, long long kprev,
                                                   double* __restrict__ part) {
    pdl_trigger();
    pdl_wait();
    __shared__ float As[32][129], Bs[32][129];   // [column of the tile][k]: conflict-free along k and along columns
    int J = 0;
    while ((J + 1) * (J + 2) / 2 <= (int)blockIdx.x) ++J;
    const int I = (int)blockIdx.x - J * (J + 1) / 2;
    const long long k0 = (long long)blockIdx.y * 128;
    const int tid = threadIdx.x;
    float va[16], vb[16];   // all 32 loads of a thread in flight at once
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int e = tid + 256 * r, kk = e & 127, c = e >> 7;
        const bool in = k0 + kk < kprev;
        va[r] = in ? C[(k0 + kk) + (long long)(I * 32 + c) * ldc] : 0.f;
        vb[r] = in ? C[(k0 + kk) + (long long)(J * 32 + c) * ldc] : 0.f;
    }
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int e = tid + 256 * r, kk = e & 127, c = e >> 7;
        As[c][kk] = va[r];
        Bs[c][kk] = vb[r];
    }
    __syncthreads();
    const int lr = tid & 31, lc = (tid >> 5) * 4;
    float cs[4][4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
        for (int kk = 32 * h; kk < 32 * h + 32; ++kk) {
            const float x = As[lr][kk];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fmaf(x, Bs[lc + q][kk], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) cs[h][q] = acc[q];
    }
    double* out = part + ((size_t)blockIdx.x * gridDim.y + blockIdx.y) * 1024;
#pragma unroll
    for (int q = 0; q < 4; ++q) out[lr + 32 * (lc + q)] = (double)((cs[0][q] + cs[1][q]) + (cs[2][q] + cs[3][q]));
}

// G (np x np, FP64, ld np) = S - C^T C on the 32 x 32 upper tiles, one per
// CTA (numbered as in k_gram_part), the KS parts of each entry summed in the
// order s = 0, 1, ...: S[i + j lds] = (Y^T Y)(i, j), upper triangle read.
// Each entry of G is written once, the lower triangle as the mirror of the
// upper.  Diagonal tiles also write trace_part[I], the sum of their
// (C^T C)_ii.
__global__ void __launch_bounds__(256) k_gram_fin(const double* __restrict__ S, long long lds,
                                                  const double* __restrict__ part, int KS, int np,
                                                  double* __restrict__ G, double* __restrict__ trace_part) {
    pdl_trigger();
    pdl_wait();
    __shared__ double dsum[32];
    int J = 0;
    while ((J + 1) * (J + 2) / 2 <= (int)blockIdx.x) ++J;
    const int I = (int)blockIdx.x - J * (J + 1) / 2;
    const double* pp = part + (size_t)blockIdx.x * KS * 1024;
    double vs[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 4
    for (int s = 0; s < KS; ++s) {
#pragma unroll
        for (int r = 0; r < 4; ++r) vs[r] += pp[(size_t)s * 1024 + threadIdx.x + 256 * r];
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int e = threadIdx.x + 256 * r;
        const double v = vs[r];
        const int li = e & 31, lj = e >> 5;
        const int i = I * 32 + li, j = J * 32 + lj;
        if (i <= j) {
            const double g = S[i + (long long)j * lds] - v;
            G[i + (long long)j * np] = g;
            if (i < j) G[j + (long long)i * np] = g;
        }
        if (I == J && li == lj) dsum[li] = v;
    }
    if (I == J) {
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int d = 0; d < 32; ++d) t += dsum[d];
            trace_part[I] = t;
        }
    }
}

// *fused = 1 when ||C||_F^2, the sum of the nparts trace parts, is <= thr
// (counted in st->fused_gram), else 0.
__global__ void k_gram_gate(const double* __restrict__ trace_part, int nparts, double thr, int* __restrict__ fused,
                            DevState* st) {
    pdl_trigger();
    pdl_wait();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < nparts; ++b) t += trace_part[b];
        const int f = (t <= thr) ? 1 : 0;   // 0 for a NaN
        *fused = f;
        if (f && st) atomicAdd(&st->fused_gram, 1);
    }
}

template <typename TC>
__global__ void k_ct_to_omega(const TC* __restrict__ Ct, long long ldc, long long kprev, int np,
                              float* __restrict__ Om, long long ldo, float* __restrict__ C32, long long ldc32) {
    pdl_trigger();
    pdl_wait();
    __shared__ TC tile[32][33];
    const long long j0 = (long long)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int i = ty; i < 32; i += 8) {
        const long long j = j0 + i;
        if (j < kprev) tile[i][tx] = Ct[(c0 + tx) + j * ldc];
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        const long long j = j0 + tx;
        if (j < kprev) {
            const float v = (float)tile[tx][i];
            Om[j + (long long)(c0 + i) * ldo] = tf32_rna(v);
            if (C32) C32[j + (long long)(c0 + i) * ldc32] = v;
        }
    }
}

// Bs / Bsl (np x n, ld np) from B_i (p x n, ld ldbi); rows p..np-1 zero.
__global__ void k_stage_b(const float* __restrict__ Bi, long long ldbi, int p, long long n, int np,
                          float* __restrict__ Bs, float* __restrict__ Bsl) {
    pdl_trigger();
    pdl_wait();
    const long long total = n * np;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % np);
        const long long j = e / np;
        const float v = c < p ? Bi[c + j * ldbi] : 0.f;
        Bs[e] = v;
        Bsl[e] = tf32_lo(v);
    }
}

__device__ __forceinline__ int first_cta(long long x, long long U, int P) {
    int p = (int)((x * P) / U);
    while (p + 1 < P && unit_begin(U, P, p + 1) <= x) ++p;
    while (p > 0 && unit_begin(U, P, p) > x) --p;
    return p;
}

// Offsets (in floats) of the partial slots that hold tile t, in CTA order,
// into off[0 .. count), returned as count.  Called by every thread of a CTA
// of at least kMaxCover threads (it synchronises): thread i takes the i-th
// CTA from the first one covering tile t, so the divisions of unit_begin run
// in parallel; the covering CTAs are the prefix of those whose range starts
// before the tile ends.  The host plan keeps the number of CTAs covering one
// tile at most kMaxCover.  q0: a shared int for the first CTA.
__device__ __forceinline__ int tile_slots(long long U, int C, int P, int G, int np, int t, size_t* off, int* q0) {
    const long long x0 = (long long)t * C, x1 = x0 + C;
    if (threadIdx.x == 0) *q0 = first_cta(x0, U, P);
    __syncthreads();
    const int q = *q0 + (int)threadIdx.x;
    bool covers = false;
    if (threadIdx.x < kMaxCover && q < P) {
        const long long ub = unit_begin(U, P, q);
        if (ub < x1) {
            covers = true;
            off[threadIdx.x] = ((size_t)q * G + (int)(t - ub / C)) * (size_t)kBM * np;
        }
    }
    return __syncthreads_count(covers);
}

// Y[r + c ldy] (r < m, c < np) = sum over the CTAs covering tile r / 128 of
// their partials, in CTA order (FP32, at most a few terms, round to nearest);
// with sub, Y = sub - that sum (sub may alias Y).  One CTA per tile and
// slice; each thread sums four consecutive rows of a column with 16-byte
// loads of the partials (and a 16-byte store where Y allows it).
constexpr int kReduceSlices = 8;   // least CTAs per tile in the reductions (gridDim.y)

__device__ __forceinline__ float4 add4(float4 a, float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

// The nc partials of one float4 of a tile, summed in CTA order (FP32, round
// to nearest), with four loads in flight.
__device__ __forceinline__ float4 sum_partials(const float* __restrict__ part, const size_t* off, int nc, int idx) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    int q = 0;
    for (; q + 4 <= nc; q += 4) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = *reinterpret_cast<const float4*>(part + off[q + u] + idx);
#pragma unroll
        for (int u = 0; u < 4; ++u) acc = add4(acc, v[u]);
    }
    for (; q < nc; ++q) acc = add4(acc, *reinterpret_cast<const float4*>(part + off[q] + idx));
    return acc;
}

__global__ void k_reduce_sketch(const float* __restrict__ part, long long U, int C, int P, int G, int np, long long m,
                                float* Y, long long ldy, const float* sub) {
    pdl_trigger();
    pdl_wait();
    __shared__ size_t off[kMaxCover];
    __shared__ int count;
    const int t = blockIdx.x;
    const int nc = tile_slots(U, C, P, G, np, t, off, &count);
    const int span = np * kBM / (int)gridDim.y;
    const int i0 = blockIdx.y * span;
    const bool vec = (ldy % 4 == 0) && ((reinterpret_cast<uintptr_t>(Y) & 15u) == 0) &&
                     ((reinterpret_cast<uintptr_t>(sub) & 15u) == 0);
    for (int idx = i0 + 4 * (int)threadIdx.x; idx < i0 + span; idx += 4 * (int)blockDim.x) {   // c * 128 + row
        const int c = idx / kBM, rl = idx % kBM;
        const long long r = (long long)t * kBM + rl;
        if (r >= m) continue;
        float4 acc = sum_partials(part, off, nc, idx);
        float* y = Y + r + c * ldy;
        const float* sv = sub ? sub + r + c * ldy : nullptr;
        if (vec && r + 4 <= m) {
            if (sv) {
                const float4 s4 = *reinterpret_cast<const float4*>(sv);
                acc = make_float4(s4.x - acc.x, s4.y - acc.y, s4.z - acc.z, s4.w - acc.w);
            }
            *reinterpret_cast<float4*>(y) = acc;
        } else {
            const float a4[4] = {acc.x, acc.y, acc.z, acc.w};
            for (int i = 0; i < 4 && r + i < m; ++i) y[i] = sv ? sv[i] - a4[i] : a4[i];
        }
    }
}

// B_i: B[c + j ldb] (c < pcols) and the staged split copy Bs / Bsl (np x n,
// column-major, ld np) from the partials of the projection; ||B_i||_F^2 of
// the tile into sq_part[tile * slices + slice] (FP64).  Each thread sums four
// consecutive rows c of a column j (16-byte loads and staged stores).
__global__ void k_reduce_project(const float* __restrict__ part, long long U, int C, int P, int G, int np, int pcols,
                                 long long n, float* __restrict__ B, long long ldb, float* __restrict__ Bs,
                                 float* __restrict__ Bsl, double* __restrict__ sq_part) {
    pdl_trigger();
    pdl_wait();
    __shared__ size_t off[kMaxCover];
    __shared__ int count;
    __shared__ double red[32];
    const int t = blockIdx.x;
    const int nc = tile_slots(U, C, P, G, np, t, off, &count);
    double sq = 0.0;
    const int span = np * kBM / (int)gridDim.y;
    const int i0 = blockIdx.y * span;
    for (int idx = i0 + 4 * (int)threadIdx.x; idx < i0 + span; idx += 4 * (int)blockDim.x) {   // jl * np + c
        const int jl = idx / np, c = idx % np;
        const long long j = (long long)t * kBM + jl;
        if (j >= n) continue;
        const float4 v = sum_partials(part, off, nc, idx);
        *reinterpret_cast<float4*>(Bs + c + j * np) = v;
        *reinterpret_cast<float4*>(Bsl + c + j * np) = make_float4(tf32_lo(v.x), tf32_lo(v.y), tf32_lo(v.z), tf32_lo(v.w));
        const float v4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (c + i < pcols) {
                B[c + i + j * ldb] = v4[i];
                sq += (double)v4[i] * (double)v4[i];
            }
    }
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        sq_part[(size_t)t * gridDim.y + blockIdx.y] = s;
    }
}

// Sum2 step (Ogita, Rump and Oishi, "Accurate sum and dot product", 2005):
// s collects the FP32 sum and e the FP32 sum of the exact rounding errors of
// its additions (TwoSum), so that s + e carries the sum of n terms to within
// about (n u)^2 of the sum of their magnitudes (u = 2^-24), on the FP32 pipe.
__device__ __forceinline__ void sum2_add(float& s, float& e, float x) {
    const float t = s + x;
    const float z = t - s;
    e += (s - (t - z)) + (x - z);
    s = t;
}

// The panel's coefficient products (the Grams Y^T Y and C^T = Y^T Qbar of
// lines (3), (3')): out[c + j ldo] (c < pcols, j < n) = the sum of the FP32
// partials of the CTAs covering tile j / 128, stored in FP64.  Each partial
// is one CTA's stretch of the reduction over m, accumulated in FP32 by the
// tensor core and the period drains.  The partials of an entry are cut into
// four runs of consecutive CTAs; a quarter of the threads sums each run in
// CTA order by Sum2 (sum2_add: about 10^-10 of the magnitudes for the ~100
// partials of an entry, far below the partials' own FP32 rounding, and on
// the FP32 pipe, where this part's FP64 pipe does two operations per clock
// per SM), and the four run sums are added in FP64 in run order (a fixed
// order, independent of the launch).  sym (a Gram, X = Q): the entries
// above the diagonal mirror those below it, which are summed once and stored
// at both positions.
__global__ void k_reduce_project64(const float* __restrict__ part, long long U, int C, int P, int G, int np,
                                   int pcols, long long n, double* __restrict__ out, long long ldo, int sym,
                                   const int* __restrict__ gate) {
    pdl_trigger();
    pdl_wait();
    if (gate && *gate) return;
    __shared__ size_t off[kMaxCover];
    __shared__ int count;
    __shared__ double runs[3][256];   // run sums 1..3 of the 256 entries in flight
    const int t = blockIdx.x;
    const int nc = tile_slots(U, C, P, G, np, t, off, &count);
    const int g = (int)threadIdx.x >> 6, lt = (int)threadIdx.x & 63;
    const int q0 = nc * g / 4, q1 = nc * (g + 1) / 4;
    const int span = np * kBM / (int)gridDim.y;
    const int i0 = blockIdx.y * span;
    for (int base = i0; base < i0 + span; base += 256) {   // 64 threads x 4 consecutive entries (jl * np + c)
        const int idx = base + 4 * lt;
        const int jl = idx / np, c = idx % np;
        const long long j = (long long)t * kBM + jl;
        const bool live = idx < i0 + span && j < n && !(sym && c + 3 < j);
        float as[4] = {0.f, 0.f, 0.f, 0.f}, ae[4] = {0.f, 0.f, 0.f, 0.f};
        if (live) {
            int q = q0;
            for (; q + 4 <= q1; q += 4) {   // four partial loads in flight
                float4 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = *reinterpret_cast<const float4*>(part + off[q + u] + idx);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    sum2_add(as[0], ae[0], v[u].x);
                    sum2_add(as[1], ae[1], v[u].y);
                    sum2_add(as[2], ae[2], v[u].z);
                    sum2_add(as[3], ae[3], v[u].w);
                }
            }
            for (; q < q1; ++q) {
                const float4 v = *reinterpret_cast<const float4*>(part + off[q] + idx);
                sum2_add(as[0], ae[0], v.x);
                sum2_add(as[1], ae[1], v.y);
                sum2_add(as[2], ae[2], v.z);
                sum2_add(as[3], ae[3], v.w);
            }
        }
        double a[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = (double)as[i] + (double)ae[i];
        if (g > 0) {
#pragma unroll
            for (int i = 0; i < 4; ++i) runs[g - 1][4 * lt + i] = a[i];
        }
        __syncthreads();
        if (g == 0 && live) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const double v = ((a[i] + runs[0][4 * lt + i]) + runs[1][4 * lt + i]) + runs[2][4 * lt + i];
                // sym: every entry written once, from the lower triangle
                if (c + i < pcols && (!sym || c + i >= j)) out[c + i + j * ldo] = v;
                if (sym && c + i > j) out[j + (long long)(c + i) * ldo] = v;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// BF16 update: Wdst = round_bf16(Wsrc - Q_i B_i) on 128 x NJ tiles, K = bp in
// chunks of 64; Q_i^T and B_i split into BF16 hi + lo, three passes (the
// lo x lo term is below 2^-17 of the product).  The W tile travels by TMA in
// both directions: warp 10 loads tile g of Wsrc into one of two W buffers,
// the eight epilogue warps replace it in shared memory by the rounded
// difference, and one thread stores it with a TMA store.  ||Wdst||_F^2 of
// the rounded values (exact FP32 squares) per CTA.
struct UpdateParams16 {
    CUtensorMap mqt, mqtl;  // Q_i^T hi / lo, row-major m x bp (as {bp, m}), box {64, 128}
    CUtensorMap mbs, mbsl;  // B_i hi / lo, bp x n column-major, box {64, NJ}
    CUtensorMap mws, mwd;   // Wsrc / Wdst, m x n column-major, box {128 rows, NJ columns}, no swizzle
    DevState* st;
    double* sq_part;
    long long m, n;
    int RT, CT, C;
};

constexpr int kUpd16Threads = 352;   // warps 0 (operand TMA), 1 (MMA), 2..9 (epilogue), 10 (W loads)

template <int NJ, int S>
__global__ void __launch_bounds__(kUpd16Threads, 1) k_update16(const __grid_constant__ UpdateParams16 p) {
    pdl_wait();
    __shared__ __align__(8) uint64_t full[S], empty[S], accfull[2], accempty[2], wfull[2], wempty[2], drain;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ double red[8];
    extern __shared__ uint8_t dsm[];
    uint8_t* base = dsm + (((smem_u32(dsm) + 1023u) & ~1023u) - smem_u32(dsm));
    constexpr uint32_t kB = (uint32_t)NJ * 128u;
    constexpr uint32_t kStage = 2u * kTileBytes + 2u * kB;
    constexpr uint32_t kWTile = (uint32_t)kBM * NJ * 2u;   // one BF16 W tile
    uint8_t* wbuf = base + S * kStage;
    constexpr uint32_t kCols = 2u * NJ;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int* ab = &abort_flag;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&accfull[s], 1); mbar_init(&accempty[s], 8);
            mbar_init(&wfull[s], 1); mbar_init(&wempty[s], 1);
        }
        mbar_init(&drain, 1);
        abort_flag = 0;
        fence_mbar_init();
        prefetch_map(&p.mqt);
        prefetch_map(&p.mqtl);
        prefetch_map(&p.mbs);
        prefetch_map(&p.mbsl);
        prefetch_map(&p.mws);
        prefetch_map(&p.mwd);
    }
    if (warp == 1) tmem_alloc(&tmem_base, kCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const int T = p.RT * p.CT;

    if (warp == 0) {
        if (lane == 0) {
            long long q = 0;
            bool stop = false;
            for (int t = blockIdx.x; t < T && !stop; t += gridDim.x) {
                const int rt = t / p.CT, ctile = t % p.CT;
                for (int kc = 0; kc < p.C; ++kc, ++q) {
                    const int s = (int)(q % S);
                    const uint32_t r = (uint32_t)(q / S);
                    if (r > 0 && !mbar_wait(&empty[s], (r - 1) & 1u, ab)) { stop = true; break; }
                    uint8_t* st = base + s * kStage;
                    mbar_arrive_expect_tx(&full[s], kStage);
                    tma_load_2d(st, &p.mqt, kc * kKC16, rt * kBM, &full[s]);
                    tma_load_2d(st + kTileBytes, &p.mqtl, kc * kKC16, rt * kBM, &full[s]);
                    tma_load_2d(st + 2 * kTileBytes, &p.mbs, kc * kKC16, ctile * NJ, &full[s]);
                    tma_load_2d(st + 2 * kTileBytes + kB, &p.mbsl, kc * kKC16, ctile * NJ, &full[s]);
                }
            }
            for (long long qq = (q > S ? q - S : 0); qq < q; ++qq)
                mbar_wait(&full[qq % S], (uint32_t)(qq / S) & 1u, ab, false);
        }
    } else if (warp == 10) {
        if (lane == 0) {
            int g = 0;
            for (int t = blockIdx.x; t < T; t += gridDim.x, ++g) {
                const int b = g & 1, use = g >> 1;
                if (use > 0 && !mbar_wait(&wempty[b], (uint32_t)(use - 1) & 1u, ab)) break;
                mbar_arrive_expect_tx(&wfull[b], kWTile);
                tma_load_2d(wbuf + b * kWTile, &p.mws, (t / p.CT) * kBM, (t % p.CT) * NJ, &wfull[b]);
            }
            for (int gg = (g > 2 ? g - 2 : 0); gg < g; ++gg)
                mbar_wait(&wfull[gg & 1], (uint32_t)(gg >> 1) & 1u, ab, false);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(NJ, 0);
            long long q = 0;
            int g = 0;
            bool stop = false;
            for (int t = blockIdx.x; t < T && !stop; t += gridDim.x, ++g) {
                const int abuf = g & 1, use = g >> 1;
                if (use > 0 && !mbar_wait(&accempty[abuf], (uint32_t)(use - 1) & 1u, ab)) break;
                const uint32_t d = tmem + (uint32_t)(abuf * NJ);
                for (int kc = 0; kc < p.C; ++kc, ++q) {
                    const int s = (int)(q % S);
                    const uint32_t r = (uint32_t)(q / S);
                    if (!mbar_wait(&full[s], r & 1u, ab)) { stop = true; break; }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(base + s * kStage), a1 = a0 + kTileBytes;
                    const uint32_t b0 = a0 + 2 * kTileBytes, b1 = b0 + kB;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_bf16(d, desc_k_sw128(a0 + kk * 32), desc_k_sw128(b0 + kk * 32), idesc,
                                 (kc == 0 && kk == 0) ? 0u : 1u);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_bf16(d, desc_k_sw128(a0 + kk * 32), desc_k_sw128(b1 + kk * 32), idesc, 1u);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_bf16(d, desc_k_sw128(a1 + kk * 32), desc_k_sw128(b0 + kk * 32), idesc, 1u);
                    mma_commit(&empty[s]);
                }
                if (stop) break;
                mma_commit(&accfull[abuf]);
            }
            mma_commit(&drain);
            mbar_wait(&drain, 0, ab, false);
        }
    } else {
        const int e = warp - 2;
        const int quarter = warp & 3;
        const int half = e >> 2;
        constexpr int kHalf = NJ / 2;
        const bool issuer = (warp == 2 && lane == 0);
        const int row = quarter * 32 + lane;          // tile row of this thread
        double sq = 0.0;
        int g = 0;
        for (int t = blockIdx.x; t < T; t += gridDim.x, ++g) {
            const int abuf = g & 1, use = g >> 1;
            bool okw = mbar_wait(&accfull[abuf], (uint32_t)use & 1u, ab);
            if (okw) okw = mbar_wait(&wfull[abuf], (uint32_t)use & 1u, ab);
            // all eight warps leave together (the named barrier below counts them)
            named_barrier(1, 256);
            if (*ab || !okw) break;
            tc_fence_after();
            const int rt = t / p.CT, ctile = t % p.CT;
            const long long r = (long long)rt * kBM + row;
            const long long j0 = (long long)ctile * NJ + half * kHalf;
            const bool rok = r < p.m;
            // W tile column-major: element (row, col) at col * 256 + row * 2
            unsigned short* wt = reinterpret_cast<unsigned short*>(wbuf + abuf * kWTile) + row;
            const uint32_t tl = tmem + (uint32_t)(abuf * NJ + half * kHalf) + ((uint32_t)(quarter * 32) << 16);
            float sq32 = 0.f;
#pragma unroll 1
            for (int c0 = 0; c0 < kHalf; c0 += 16) {
                float v[16];
                tmem_ld16(tl + (uint32_t)c0, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int cl = half * kHalf + c0 + i;
                    const float w = __bfloat162float(__ushort_as_bfloat16(wt[cl * kBM]));
                    const __nv_bfloat16 o = __float2bfloat16_rn(w - v[i]);
                    wt[cl * kBM] = __bfloat16_as_ushort(o);
                    if (rok && j0 + c0 + i < p.n) {
                        const float of = __bfloat162float(o);
                        sq32 = fmaf(of, of, sq32);
                    }
                }
                if ((c0 & 31) == 16) {
                    sq += (double)sq32;
                    sq32 = 0.f;
                }
            }
            sq += (double)sq32;
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&accempty[abuf]);
            fence_async_smem();
            named_barrier(1, 256);
            if (issuer) {
                tma_store_2d(&p.mwd, rt * kBM, ctile * NJ, wbuf + abuf * kWTile);
                bulk_commit();
                // the previous tile's store has read its buffer: hand it back
                bulk_wait_read<1>();
                if (g > 0) mbar_arrive(&wempty[abuf ^ 1]);
            }
        }
        if (issuer) bulk_wait<0>();
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        if (lane == 0) red[e] = sq;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, kCols);
    if (threadIdx.x == 0) {
        if (abort_flag) record_error(p.st, RQB_ERR_TIMEOUT);
        if (p.sq_part) {
            double t = 0.0;
            for (int i = 0; i < 8; ++i) t += red[i];
            p.sq_part[blockIdx.x] = t;
        }
    }
}

// Wide BF16 update: the same product on 128 x 256 tiles (N = 256 MMAs read a
// quarter fewer operand bytes per multiply-add than N = 128 ones), K in
// chunks of 32 (64-byte swizzle rows, 48 KB per stage) through three stages,
// and the W tile in 128 x 64 quarters through a ring of four 16 KB buffers
// (warp 10 loads quarter w into slot w % 4; the epilogue warps replace it by
// the rounded difference; one thread stores it and hands the previous slot
// back once that store has read it).  TMEM: two 256-column accumulators.
constexpr int kKCw = 32;                            // K per chunk
constexpr int kNJw = 256;                           // tile columns
constexpr int kStw = 3;                             // operand stages
constexpr int kWRw = 4;                             // W quarter buffers
constexpr uint32_t kQw = kBM * kKCw * 2;            // Q_i^T hi or lo chunk: 8 KB
constexpr uint32_t kBw = kNJw * kKCw * 2;           // B_i hi or lo chunk: 16 KB
constexpr uint32_t kStageW = 2 * kQw + 2 * kBw;     // 48 KB
constexpr uint32_t kWQw = kBM * 64 * 2;             // W quarter: 16 KB
constexpr size_t kUpd16wSmem = (size_t)kStw * kStageW + (size_t)kWRw * kWQw + 1024;

__global__ void __launch_bounds__(kUpd16Threads, 1) k_update16w(const __grid_constant__ UpdateParams16 p) {
    pdl_wait();
    __shared__ __align__(8) uint64_t full[kStw], empty[kStw], accfull[2], accempty[2], wfull[kWRw], wempty[kWRw],
        drain;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ double red[8];
    extern __shared__ uint8_t dsm[];
    uint8_t* base = dsm + (((smem_u32(dsm) + 1023u) & ~1023u) - smem_u32(dsm));
    uint8_t* wbuf = base + kStw * kStageW;
    constexpr uint32_t kCols = 2u * kNJw;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int* ab = &abort_flag;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStw; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int s = 0; s < 2; ++s) { mbar_init(&accfull[s], 1); mbar_init(&accempty[s], 8); }
        for (int s = 0; s < kWRw; ++s) { mbar_init(&wfull[s], 1); mbar_init(&wempty[s], 1); }
        mbar_init(&drain, 1);
        abort_flag = 0;
        fence_mbar_init();
        prefetch_map(&p.mqt);
        prefetch_map(&p.mqtl);
        prefetch_map(&p.mbs);
        prefetch_map(&p.mbsl);
        prefetch_map(&p.mws);
        prefetch_map(&p.mwd);
    }
    if (warp == 1) tmem_alloc(&tmem_base, kCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const int T = p.RT * p.CT;

    if (warp == 0) {
        if (lane == 0) {
            long long q = 0;
            bool stop = false;
            for (int t = blockIdx.x; t < T && !stop; t += gridDim.x) {
                const int rt = t / p.CT, ctile = t % p.CT;
                for (int kc = 0; kc < p.C; ++kc, ++q) {
                    const int s = (int)(q % kStw);
                    const uint32_t r = (uint32_t)(q / kStw);
                    if (r > 0 && !mbar_wait(&empty[s], (r - 1) & 1u, ab)) { stop = true; break; }
                    uint8_t* st = base + s * kStageW;
                    mbar_arrive_expect_tx(&full[s], kStageW);
                    tma_load_2d(st, &p.mqt, kc * kKCw, rt * kBM, &full[s]);
                    tma_load_2d(st + kQw, &p.mqtl, kc * kKCw, rt * kBM, &full[s]);
                    tma_load_2d(st + 2 * kQw, &p.mbs, kc * kKCw, ctile * kNJw, &full[s]);
                    tma_load_2d(st + 2 * kQw + kBw, &p.mbsl, kc * kKCw, ctile * kNJw, &full[s]);
                }
            }
            for (long long qq = (q > kStw ? q - kStw : 0); qq < q; ++qq)
                mbar_wait(&full[qq % kStw], (uint32_t)(qq / kStw) & 1u, ab, false);
        }
    } else if (warp == 10) {
        if (lane == 0) {
            long long w = 0;   // quarters issued
            bool stop = false;
            for (int t = blockIdx.x; t < T && !stop; t += gridDim.x) {
                for (int qq = 0; qq < 4; ++qq, ++w) {
                    const int slot = (int)(w % kWRw);
                    const long long use = w / kWRw;
                    if (use > 0 && !mbar_wait(&wempty[slot], (uint32_t)(use - 1) & 1u, ab)) { stop = true; break; }
                    mbar_arrive_expect_tx(&wfull[slot], kWQw);
                    tma_load_2d(wbuf + slot * kWQw, &p.mws, (t / p.CT) * kBM, (t % p.CT) * kNJw + qq * 64,
                                &wfull[slot]);
                }
            }
            for (long long ww = (w > kWRw ? w - kWRw : 0); ww < w; ++ww)
                mbar_wait(&wfull[ww % kWRw], (uint32_t)(ww / kWRw) & 1u, ab, false);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(kNJw, 0);
            long long q = 0;
            int g = 0;
            bool stop = false;
            for (int t = blockIdx.x; t < T && !stop; t += gridDim.x, ++g) {
                const int abuf = g & 1, use = g >> 1;
                if (use > 0 && !mbar_wait(&accempty[abuf], (uint32_t)(use - 1) & 1u, ab)) break;
                const uint32_t d = tmem + (uint32_t)(abuf * kNJw);
                for (int kc = 0; kc < p.C; ++kc, ++q) {
                    const int s = (int)(q % kStw);
                    const uint32_t r = (uint32_t)(q / kStw);
                    if (!mbar_wait(&full[s], r & 1u, ab)) { stop = true; break; }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(base + s * kStageW), a1 = a0 + kQw;
                    const uint32_t b0 = a0 + 2 * kQw, b1 = b0 + kBw;
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk)
                        mma_bf16(d, desc_k_sw64(a0 + kk * 32), desc_k_sw64(b0 + kk * 32), idesc,
                                 (kc == 0 && kk == 0) ? 0u : 1u);
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk)
                        mma_bf16(d, desc_k_sw64(a0 + kk * 32), desc_k_sw64(b1 + kk * 32), idesc, 1u);
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk)
                        mma_bf16(d, desc_k_sw64(a1 + kk * 32), desc_k_sw64(b0 + kk * 32), idesc, 1u);
                    mma_commit(&empty[s]);
                }
                if (stop) break;
                mma_commit(&accfull[abuf]);
            }
            mma_commit(&drain);
            mbar_wait(&drain, 0, ab, false);
        }
    } else {
        const int e = warp - 2;
        const int quarter = warp & 3;                 // TMEM lanes this warp may read
        const int half = e >> 2;                      // columns [32 half, 32 half + 32) of each W quarter
        const bool issuer = (warp == 2 && lane == 0);
        const int row = quarter * 32 + lane;          // tile row of this thread
        double sq = 0.0;
        int g = 0;
        long long w = 0;                              // quarters consumed
        bool stop = false;
        for (int t = blockIdx.x; t < T && !stop; t += gridDim.x, ++g) {
            const int abuf = g & 1, use = g >> 1;
            const bool oka = mbar_wait(&accfull[abuf], (uint32_t)use & 1u, ab);
            const int rt = t / p.CT, ctile = t % p.CT;
            const long long r = (long long)rt * kBM + row;
            const bool rok = r < p.m;
            for (int qq = 0; qq < 4; ++qq, ++w) {
                const int slot = (int)(w % kWRw);
                bool okw = oka && mbar_wait(&wfull[slot], (uint32_t)(w / kWRw) & 1u, ab);
                // all eight warps leave together (the named barrier below counts them)
                named_barrier(1, 256);
                if (*ab || !okw) { stop = true; break; }
                tc_fence_after();
                const long long j0 = (long long)ctile * kNJw + qq * 64 + half * 32;
                // W quarter column-major: element (row, col) at col * 256 + row * 2
                unsigned short* wt = reinterpret_cast<unsigned short*>(wbuf + slot * kWQw) + row;
                const uint32_t tl =
                    tmem + (uint32_t)(abuf * kNJw + qq * 64 + half * 32) + ((uint32_t)(quarter * 32) << 16);
                float sq32 = 0.f;
#pragma unroll 1
                for (int c0 = 0; c0 < 32; c0 += 16) {
                    float v[16];
                    tmem_ld16(tl + (uint32_t)c0, v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int cl = half * 32 + c0 + i;
                        const float wv = __bfloat162float(__ushort_as_bfloat16(wt[cl * kBM]));
                        const __nv_bfloat16 o = __float2bfloat16_rn(wv - v[i]);
                        wt[cl * kBM] = __bfloat16_as_ushort(o);
                        if (rok && j0 + c0 + i < p.n) {
                            const float of = __bfloat162float(o);
                            sq32 = fmaf(of, of, sq32);
                        }
                    }
                }
                sq += (double)sq32;
                if (qq == 3) {   // the accumulator is read: hand it back
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&accempty[abuf]);
                }
                fence_async_smem();
                named_barrier(1, 256);
                if (issuer) {
                    tma_store_2d(&p.mwd, rt * kBM, ctile * kNJw + qq * 64, wbuf + slot * kWQw);
                    bulk_commit();
                    // the previous quarter's store has read its buffer: hand it back
                    bulk_wait_read<1>();
                    if (w > 0) mbar_arrive(&wempty[(w - 1) % kWRw]);
                }
            }
        }
        if (issuer) bulk_wait<0>();
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        if (lane == 0) red[e] = sq;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, kCols);
    if (threadIdx.x == 0) {
        if (abort_flag) record_error(p.st, RQB_ERR_TIMEOUT);
        if (p.sq_part) {
            double t = 0.0;
            for (int i = 0; i < 8; ++i) t += red[i];
            p.sq_part[blockIdx.x] = t;
        }
    }
}

// x = hi + lo with hi = rn_bf16(x) and lo = rn_bf16(x - hi) (x - hi is exact
// in FP32): the pair holds x to 2^-18 relative.
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Omega_i for the BF16 products: the binary32 Gaussian (j, col0 + c) rounded
// to BF16 (nearest even), out[j + c ldo] for c < p, zero for p <= c < bp.
// OutT = __nv_bfloat16 (the MMA operand) or float (the same values widened).
template <typename OutT>
__global__ void k_omega_bf16(long long n, long long col0, int p, int bp, uint64_t seed, OutT* __restrict__ out,
                             long long ldo) {
    pdl_trigger();
    pdl_wait();
    const long long total = n * bp;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long j = e % n;
        const int c = (int)(e / n);
        const __nv_bfloat16 v = __float2bfloat16_rn(c < p ? gaussian_f32(seed, j, col0 + c) : 0.f);
        if constexpr (sizeof(OutT) == 2) out[j + c * ldo] = v;
        else out[j + c * ldo] = __bfloat162float(v);
    }
}

// BF16 splits of Q_i (m x p, ld ldq): Qhi / Qlo column-major (ld ldql, bp
// columns) and the row-major transpose pair Qt / Qtl (m x bp).
__global__ void k_split_q16(const float* __restrict__ Qi, long long ldq, long long m, int p, int bp,
                            __nv_bfloat16* __restrict__ Qhi, __nv_bfloat16* __restrict__ Qlo, long long ldql,
                            __nv_bfloat16* __restrict__ Qt, __nv_bfloat16* __restrict__ Qtl) {
    pdl_trigger();
    pdl_wait();
    __shared__ float tile[32][33];
    const long long r0 = (long long)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int i = ty; i < 32; i += 8) {
        const long long r = r0 + tx;
        const int c = c0 + i;
        float v = 0.f;
        if (r < m && c < p) v = Qi[r + c * ldq];
        if (r < m) split_bf16(v, Qhi[r + c * ldql], Qlo[r + c * ldql]);
        tile[i][tx] = v;
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        const long long r = r0 + i;
        const int c = c0 + tx;
        if (r < m) split_bf16(tile[tx][i], Qt[r * bp + c], Qtl[r * bp + c]);
    }
}

// Bs / Bsl (bp x n, ld bp, BF16 hi / lo) from B_i (p x n, ld ldbi).
__global__ void k_stage_b16(const float* __restrict__ Bi, long long ldbi, int p, long long n, int bp,
                            __nv_bfloat16* __restrict__ Bs, __nv_bfloat16* __restrict__ Bsl) {
    pdl_trigger();
    pdl_wait();
    const long long total = n * bp;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % bp);
        const long long j = e / bp;
        split_bf16(c < p ? Bi[c + j * ldbi] : 0.f, Bs[e], Bsl[e]);
    }
}

// As k_reduce_project, with the staged copy of B_i split into BF16 hi / lo.
__global__ void k_reduce_project16(const float* __restrict__ part, long long U, int C, int P, int G, int np,
                                   int pcols, long long n, float* __restrict__ B, long long ldb,
                                   __nv_bfloat16* __restrict__ Bs, __nv_bfloat16* __restrict__ Bsl,
                                   double* __restrict__ sq_part) {
    pdl_trigger();
    pdl_wait();
    __shared__ size_t off[kMaxCover];
    __shared__ int count;
    __shared__ double red[32];
    const int t = blockIdx.x;
    const int nc = tile_slots(U, C, P, G, np, t, off, &count);
    double sq = 0.0;
    const int span = np * kBM / (int)gridDim.y;
    const int i0 = blockIdx.y * span;
#pragma unroll 4
    for (int idx = i0 + 4 * (int)threadIdx.x; idx < i0 + span; idx += 4 * (int)blockDim.x) {
        const int jl = idx / np, c = idx % np;
        const long long j = (long long)t * kBM + jl;
        if (j >= n) continue;
        const float4 v = sum_partials(part, off, nc, idx);
        const float v4[4] = {v.x, v.y, v.z, v.w};
        __align__(8) __nv_bfloat16 hi[4], lo[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) split_bf16(v4[i], hi[i], lo[i]);
        *reinterpret_cast<uint2*>(Bs + c + j * np) = *reinterpret_cast<const uint2*>(hi);
        *reinterpret_cast<uint2*>(Bsl + c + j * np) = *reinterpret_cast<const uint2*>(lo);
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (c + i < pcols) {
                B[c + i + j * ldb] = v4[i];
                sq += (double)v4[i] * (double)v4[i];
            }
    }
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        sq_part[(size_t)t * gridDim.y + blockIdx.y] = s;
    }
}

// Self-test of the bounded wait: one thread waits on an mbarrier that no
// thread or copy ever completes; the wait gives up after its limit and the
// kernel records RQB_ERR_TIMEOUT and the time it waited.
__global__ void k_wait_selftest(DevState* st, unsigned long long* waited_ns) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long t0 = globaltimer_ns();
        const bool ok = mbar_wait(&bar, 0, &abort_flag);
        *waited_ns = globaltimer_ns() - t0;
        if (!ok) record_error(st, RQB_ERR_TIMEOUT);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side.
namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
    });
    return fn;
}

// 2-D map of esize-byte elements: `inner` contiguous elements per line,
// `outer` lines `ld` elements apart; boxes of box_inner x box_outer, zero
// fill out of bounds.  The base must be 16-byte aligned and the line pitch a
// multiple of 16 bytes.
cudaError_t make_map_t(CUtensorMap* map, const void* base, CUtensorMapDataType dt, int esize, long long inner,
                       long long outer, long long ld, int box_inner, int box_outer, bool swizzle128,
                       bool swizzle64 = false) {
    EncodeTiledFn enc = encoder();
    if (!enc) return cudaErrorNotSupported;
    if ((reinterpret_cast<uintptr_t>(base) & 15u) != 0 || ((ld * esize) & 15) != 0 || inner < box_inner ||
        outer < box_outer)
        return cudaErrorInvalidValue;
    const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    const cuuint64_t strides[1] = {(cuuint64_t)(ld * esize)};
    const cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = enc(map, dt, 2, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           swizzle128  ? CU_TENSOR_MAP_SWIZZLE_128B
                           : swizzle64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                       : CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t make_map(CUtensorMap* map, const float* base, long long inner, long long outer, long long ld,
                     int box_inner, int box_outer, bool swizzle128) {
    return make_map_t(map, base, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, inner, outer, ld, box_inner, box_outer,
                      swizzle128);
}

cudaError_t make_map(CUtensorMap* map, const __nv_bfloat16* base, long long inner, long long outer, long long ld,
                     int box_inner, int box_outer, bool swizzle128) {
    return make_map_t(map, base, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, inner, outer, ld, box_inner, box_outer,
                      swizzle128);
}

// FP32 map with the 64-byte swizzle (boxes of 16 elements along `inner`).
cudaError_t make_map_sw64(CUtensorMap* map, const float* base, long long inner, long long outer, long long ld,
                          int box_outer) {
    return make_map_t(map, base, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, inner, outer, ld, 16, box_outer, false, true);
}

// BF16 map with the 64-byte swizzle (boxes of 32 elements along `inner`).
cudaError_t make_map_sw64(CUtensorMap* map, const __nv_bfloat16* base, long long inner, long long outer,
                          long long ld, int box_outer) {
    return make_map_t(map, base, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, inner, outer, ld, 32, box_outer, false, true);
}

constexpr int kUpdNJ = 128, kUpdStages = 2;
constexpr size_t kUpdSmem =
    (size_t)kUpdStages * (2 * kTileBytes + 2 * kUpdNJ * 128) + (size_t)kWRing * kBM * (kUpdNJ / 2) * 4 + 1024;

template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int ROLE, int NP>
cudaError_t launch_streamk_np(Ctx& cx, const StreamKParams& p) {
    constexpr size_t smem = StreamKCfg<ROLE, NP>::kSmem;
    cudaError_t e = allow_smem(k_streamk<ROLE, NP>, smem);
    if (e != cudaSuccess) return e;
    {
        const cudaError_t le_ = launch_pdl(k_streamk<ROLE, NP>, dim3(p.P), dim3(320), smem, cx.stream, p);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    return cudaGetLastError();
}

template <int ROLE>
cudaError_t launch_streamk(Ctx& cx, const StreamKParams& p, int np) {
    switch (np) {
        case 32: return launch_streamk_np<ROLE, 32>(cx, p);
        case 64: return launch_streamk_np<ROLE, 64>(cx, p);
        case 128: return launch_streamk_np<ROLE, 128>(cx, p);
        case 256: return launch_streamk_np<ROLE, 256>(cx, p);
        default: return cudaErrorInvalidValue;
    }
}

template <int ROLE, int NP, bool GEN = false>
cudaError_t launch_streamk16_np(Ctx& cx, const StreamKParams& p) {
    constexpr size_t smem = StreamK16Cfg<ROLE, NP>::kSmem;
    cudaError_t e = allow_smem(k_streamk16<ROLE, NP, GEN>, smem);
    if (e != cudaSuccess) return e;
    {
        const cudaError_t le_ = launch_pdl(k_streamk16<ROLE, NP, GEN>, dim3(p.P), dim3(320), smem, cx.stream, p);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    return cudaGetLastError();
}

template <int ROLE, bool GEN = false>
cudaError_t launch_streamk16(Ctx& cx, const StreamKParams& p, int np) {
    switch (np) {
        case 64: return launch_streamk16_np<ROLE, 64, GEN>(cx, p);
        case 128: return launch_streamk16_np<ROLE, 128, GEN>(cx, p);
        case 256: return launch_streamk16_np<ROLE, 256, GEN>(cx, p);
        default: return cudaErrorInvalidValue;
    }
}

constexpr int kUpd16Stages = 2;
constexpr size_t kUpd16Smem =
    (size_t)kUpd16Stages * (2 * kTileBytes + 2 * kUpdNJ * 128) + 2 * (size_t)kBM * kUpdNJ * 2 + 1024;

struct Plan {
    long long U;
    int tiles, C, P, G;
};

Plan plan(long long tiles, long long C, int sms) {
    Plan pl;
    pl.tiles = (int)tiles;
    pl.C = (int)C;
    pl.U = tiles * C;
    // every CTA covers at least minlen = floor(U / P) units, so a tile of C
    // units meets at most ceil(C / minlen) + 1 CTAs: keep that <= kMaxCover
    const long long minlen = (C + kMaxCover - 2) / (kMaxCover - 1);
    pl.P = (int)std::max<long long>(1, std::min<long long>({(long long)sms, pl.U, pl.U / minlen}));
    const long long maxlen = (pl.U + pl.P - 1) / pl.P;
    pl.G = (int)((maxlen - 1) / C + 2);
    return pl;
}

// CTAs per tile of the reductions: at least kReduceSlices, more (up to 64)
// when there are few tiles, so that the reduction still fills the GPU.
int reduce_slices(int tiles, int sms) {
    int sl = kReduceSlices;
    while (sl < 64 && (long long)tiles * sl < 4LL * sms) sl *= 2;
    return sl;
}

}  // namespace

bool shape_ok(long long m, long long n) { return m >= 128 && n >= 256; }

size_t partial_floats(long long m, long long n, int np, int sms) {
    const Plan a = plan((m + kBM - 1) / kBM, (n + kKC - 1) / kKC, sms);   // sketch
    const Plan b = plan((n + kBM - 1) / kBM, (m + kKC - 1) / kKC, sms);
    return (size_t)std::max(a.P * a.G, b.P * b.G) * kBM * np;
}

cudaError_t omega(Ctx& cx, long long n, long long col0, int p, int np, uint64_t seed, float* out, long long ldo) {
    const long long total = n * np;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 8LL * cx.num_sms);
    {
        const cudaError_t le_ = launch_pdl(k_omega_tf32, dim3(blocks), dim3(256), 0, cx.stream, n, col0, p, np, seed,
                                           out, ldo);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    return cudaGetLastError();
}

cudaError_t split_q(Ctx& cx, const float* Qi, long long ldq, long long m, int p, int np, float* Qhi, float* Qlo,
                    long long ldql, float* Qt, float* Qtl) {
    dim3 grid((unsigned)((m + 31) / 32), (unsigned)(np / 32));
    {
        const cudaError_t le_ = launch_pdl(k_split_q, dim3(grid), dim3(256), 0, cx.stream, Qi, ldq, m, p, np, Qhi, Qlo,
                                           ldql, Qt, Qtl, static_cast<const int*>(nullptr));
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    return cudaGetLastError();
}

cudaError_t stage_b(Ctx& cx, const float* Bi, long long ldbi, int p, long long n, int np, float* Bs, float* Bsl) {
    const long long total = n * np;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 8LL * cx.num_sms);
    {
        const cudaError_t le_ = launch_pdl(k_stage_b, dim3(blocks), dim3(256), 0, cx.stream, Bi, ldbi, p, n, np, Bs,
                                           Bsl);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    return cudaGetLastError();
}

cudaError_t sketch(Ctx& cx, const float* X, long long ldx, long long m, long long n, const float* Om, long long ldom,
                   int np, float* Y, long long ldy, float* part, size_t part_cap, double* nrm_part, int nrm_cap,
                   double* nrm_out) {
    StreamKParams p;
    cudaError_t e;
    if ((e = make_map(&p.mx, X, m, n, ldx, kBM, kKC, false)) != cudaSuccess) return e;
    if ((e = make_map(&p.mw, Om, n, np, ldom, kKC, np, true)) != cudaSuccess) return e;
    p.mwl = p.mw;
    const Plan pl = plan((m + kBM - 1) / kBM, (n + kKC - 1) / kKC, cx.num_sms);
    if ((size_t)pl.P * pl.G * kBM * np > part_cap) return cudaErrorInvalidValue;
    if (nrm_out && pl.P > nrm_cap) return cudaErrorInvalidValue;
    p.part = part;
    p.st = cx.st;
    p.U = pl.U; p.C = pl.C; p.P = pl.P; p.G = pl.G; p.np = np;
    p.nrm_part = nrm_out ? nrm_part : nullptr;
    if ((e = launch_streamk<kSketch>(cx, p, np)) != cudaSuccess) return e;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const dim3 rgrid(pl.tiles, reduce_slices(pl.tiles, cx.num_sms));
    {
        const cudaError_t le_ = launch_pdl(k_reduce_sketch, dim3(rgrid), dim3(256), 0, cx.stream, part, pl.U, pl.C,
                                           pl.P, pl.G, np, m, Y, ldy, nullptr);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return nrm_out ? launch_sum_doubles(cx, nrm_part, pl.P, nrm_out) : cudaSuccess;
}

// Y = sub - X Omega (sub may alias Y), otherwise as sketch().
cudaError_t sketch_sub(Ctx& cx, const float* X, long long ldx, long long m, long long n, const float* Om,
                       long long ldom, int np, float* Y, long long ldy, const float* sub, float* part,
                       size_t part_cap) {
    StreamKParams p;
    cudaError_t e;
    if ((e = make_map(&p.mx, X, m, n, ldx, kBM, kKC, false)) != cudaSuccess) return e;
    if ((e = make_map(&p.mw, Om, n, np, ldom, kKC, np, true)) != cudaSuccess) return e;
    p.mwl = p.mw;
    const Plan pl = plan((m + kBM - 1) / kBM, (n + kKC - 1) / kKC, cx.num_sms);
    if ((size_t)pl.P * pl.G * kBM * np > part_cap) return cudaErrorInvalidValue;
    p.part = part;
    p.st = cx.st;
    p.U = pl.U; p.C = pl.C; p.P = pl.P; p.G = pl.G; p.np = np;
    if ((e = launch_streamk<kSketch>(cx, p, np)) != cudaSuccess) return e;
    const dim3 rgrid(pl.tiles, reduce_slices(pl.tiles, cx.num_sms));
    {
        const cudaError_t le_ = launch_pdl(k_reduce_sketch, dim3(rgrid), dim3(256), 0, cx.stream, part, pl.U, pl.C,
                                           pl.P, pl.G, np, m, Y, ldy, sub);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    return cudaGetLastError();
}

cudaError_t project(Ctx& cx, const float* X, long long ldx, long long m, long long n, const float* Qhi,
                    const float* Qlo, long long ldql, int pcols, int np, float* B, long long ldb, float* Bs,
                    float* Bsl, float* part, size_t part_cap, double* sq_part, int sq_cap, double* sq_out) {
    StreamKParams p;
    cudaError_t e;
    if ((e = make_map(&p.mx, X, m, n, ldx, kKC, kBM, true)) != cudaSuccess) return e;
    if ((e = make_map(&p.mw, Qhi, m, np, ldql, kKC, np, true)) != cudaSuccess) return e;
    if ((e = make_map(&p.mwl, Qlo, m, np, ldql, kKC, np, true)) != cudaSuccess) return e;
    const Plan pl = plan((n + kBM - 1) / kBM, (m + kKC - 1) / kKC, cx.num_sms);
    const int sl = reduce_slices(pl.tiles, cx.num_sms);
    if ((size_t)pl.P * pl.G * kBM * np > part_cap || pl.tiles * sl > sq_cap) return cudaErrorInvalidValue;
    p.part = part;
    p.st = cx.st;
    p.U = pl.U; p.C = pl.C; p.P = pl.P; p.G = pl.G; p.np = np;
    if ((e = launch_streamk<kProject>(cx, p, np)) != cudaSuccess) return e;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    {
        const cudaError_t le_ = launch_pdl(k_reduce_project, dim3(pl.tiles, sl), dim3(256), 0, cx.stream, part, pl.U,
                                           pl.C, pl.P, pl.G, np, pcols, n, B, ldb, Bs, Bsl, sq_part);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_sum_doubles(cx, sq_part, pl.tiles * sl, sq_out);
}

// out (pcols x n, FP64, ld ldo) = Q^T X as project(), the CTAs' FP32
// partials summed in FP64 (k_reduce_project64); no staged copies, no norm.
// With X2, X is [X X2] side by side: n columns of X (a multiple of 128) then
// n2 of X2 (ld ldx2), out pcols x (n + n2).  A nonzero *gate makes both
// launches do nothing.
cudaError_t project64(Ctx& cx, const float* X, long long ldx, long long m, long long n, const float* Qhi,
                      const float* Qlo, long long ldql, int pcols, int np, double* out, long long ldo, float* part,
                      size_t part_cap, bool sym = false, const float* X2 = nullptr, long long ldx2 = 0,
                      long long n2 = 0, const int* gate = nullptr) {
    StreamKParams p;
    cudaError_t e;
    if ((e = make_map(&p.mx, X, m, n, ldx, kKC, kBM, true)) != cudaSuccess) return e;
    if ((e = make_map(&p.mw, Qhi, m, np, ldql, kKC, np, true)) != cudaSuccess) return e;
    if ((e = make_map(&p.mwl, Qlo, m, np, ldql, kKC, np, true)) != cudaSuccess) return e;
    if (X2) {
        if (n % kBM != 0) return cudaErrorInvalidValue;
        if ((e = make_map(&p.mx2, X2, m, n2, ldx2, kKC, kBM, true)) != cudaSuccess) return e;
        p.tsplit = (int)(n / kBM);
        n += n2;
    }
    p.gate = gate;
    const Plan pl = plan((n + kBM - 1) / kBM, (m + kKC - 1) / kKC, cx.num_sms);
    const int sl = reduce_slices(pl.tiles, cx.num_sms);
    if ((size_t)pl.P * pl.G * kBM * np > part_cap) return cudaErrorInvalidValue;
    p.part = part;
    p.st = cx.st;
    p.U = pl.U; p.C = pl.C; p.P = pl.P; p.G = pl.G; p.np = np;
    if ((e = launch_streamk<kProject>(cx, p, np)) != cudaSuccess) return e;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    {
        const cudaError_t le_ = launch_pdl(k_reduce_project64, dim3(pl.tiles, sl), dim3(256), 0, cx.stream, part, pl.U,
                                           pl.C, pl.P, pl.G, np, pcols, n, out, ldo, sym ? 1 : 0, gate);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    return cudaGetLastError();
}

cudaError_t update_impl(Ctx& cx, const float* Wsrc, long long ldws, float* Wdst, long long ldwd, long long m,
                        long long n, const float* Qt, const float* Qtl, const float* Bs, const float* Bsl, int np,
                        double* sq_part, int sq_cap, double* sq_out, int sub) {
    UpdateParams p;
    cudaError_t e;
    p.sub = sub;
    if (!sub) {
        Wsrc = Wdst;     // the source map is not read
        ldws = ldwd;
    }
    if (n >= kNJt && m >= kBM && np % kKCt == 0) {
        // 128 x 256 tiles (k_updatew)
        if ((e = make_map_sw64(&p.mqt, Qt, np, m, np, kBM)) != cudaSuccess) return e;
        if ((e = make_map_sw64(&p.mqtl, Qtl, np, m, np, kBM)) != cudaSuccess) return e;
        if ((e = make_map_sw64(&p.mbs, Bs, np, n, np, kNJt)) != cudaSuccess) return e;
        if ((e = make_map_sw64(&p.mbsl, Bsl, np, n, np, kNJt)) != cudaSuccess) return e;
        if ((e = make_map(&p.mws, Wsrc, m, n, ldws, kBM, 32, false)) != cudaSuccess) return e;
        if ((e = make_map(&p.mwd, Wdst, m, n, ldwd, kBM, 32, false)) != cudaSuccess) return e;
        p.st = cx.st;
        p.sq_part = sq_out ? sq_part : nullptr;
        p.m = m; p.n = n;
        p.RT = (int)((m + kBM - 1) / kBM);
        p.CT = (int)((n + kNJt - 1) / kNJt);
        p.C = np / kKCt;
        const long long T = (long long)p.RT * p.CT;
        const int grid = (int)std::min<long long>(cx.num_sms, T);
        if (sq_out && grid > sq_cap) return cudaErrorInvalidValue;
        if ((e = allow_smem(k_updatew, kUpdwSmem)) != cudaSuccess) return e;
        {
            const cudaError_t le_ = launch_pdl(k_updatew, dim3(grid), dim3(kUpdThreads), kUpdwSmem, cx.stream, p);
            if (le_ != cudaSuccess) return le_;
        }
        cx.launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        return sq_out ? launch_sum_doubles(cx, sq_part, grid, sq_out) : cudaSuccess;
    }
    if ((e = make_map(&p.mqt, Qt, np, m, np, kKC, kBM, true)) != cudaSuccess) return e;
    if ((e = make_map(&p.mqtl, Qtl, np, m, np, kKC, kBM, true)) != cudaSuccess) return e;
    if ((e = make_map(&p.mbs, Bs, np, n, np, kKC, kUpdNJ, true)) != cudaSuccess) return e;
    if ((e = make_map(&p.mbsl, Bsl, np, n, np, kKC, kUpdNJ, true)) != cudaSuccess) return e;
    if ((e = make_map(&p.mws, Wsrc, m, n, ldws, kBM, kUpdNJ / 2, false)) != cudaSuccess) return e;
    if ((e = make_map(&p.mwd, Wdst, m, n, ldwd, kBM, kUpdNJ / 2, false)) != cudaSuccess) return e;
    p.st = cx.st;
    p.sq_part = sq_out ? sq_part : nullptr;
    p.m = m; p.n = n;
    p.RT = (int)((m + kBM - 1) / kBM);
    p.CT = (int)((n + kUpdNJ - 1) / kUpdNJ);
    p.C = np / kKC;
    const long long T = (long long)p.RT * p.CT;
    const int grid = (int)std::min<long long>(cx.num_sms, T);
    if (sq_out && grid > sq_cap) return cudaErrorInvalidValue;
    if ((e = allow_smem(k_update<kUpdNJ, kUpdStages>, kUpdSmem)) != cudaSuccess) return e;
    {
        const cudaError_t le_ = launch_pdl(k_update<kUpdNJ, kUpdStages>, dim3(grid), dim3(kUpdThreads), kUpdSmem,
                                           cx.stream, p);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return sq_out ? launch_sum_doubles(cx, sq_part, grid, sq_out) : cudaSuccess;
}

cudaError_t update(Ctx& cx, const float* Wsrc, long long ldws, float* Wdst, long long ldwd, long long m,
                   long long n, const float* Qt, const float* Qtl, const float* Bs, const float* Bsl, int np,
                   double* sq_part, int sq_cap, double* sq_out) {
    return update_impl(cx, Wsrc, ldws, Wdst, ldwd, m, n, Qt, Qtl, Bs, Bsl, np, sq_part, sq_cap, sq_out, 1);
}

// G (np x np, FP32, ld np, in w.Ct) = Y^T Y by the stream-K projection with
// Y split into hi / lo (three passes, FP32 accumulation with period drains).
bool gram_ok(long long m, int np, long long ldy, const float* Y) {
    return m >= 128 && np >= kBM && (ldy % 4) == 0 && (reinterpret_cast<uintptr_t>(Y) & 15u) == 0;
}

cudaError_t gram(Ctx& cx, const float* Y, long long ldy, long long m, int np, const ReprojScratch& w, double* G,
                 bool keep_split, const int* gate) {
    cudaError_t e;
    dim3 g1((unsigned)((m + 31) / 32), (unsigned)(np / 32));
    {
        const cudaError_t le_ = launch_pdl(k_split_q, dim3(g1), dim3(256), 0, cx.stream, Y, ldy, m, np, np, w.Yhi,
                                           w.Ylo, w.ldyl, keep_split ? w.Yt : nullptr, keep_split ? w.Ytl : nullptr,
                                           gate);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return project64(cx, Y, ldy, m, np, w.Yhi, w.Ylo, w.ldyl, np, np, G, np, w.part, w.part_cap, true, nullptr, 0, 0,
                     gate);
}

// Out (m x np, ld ldo) = Y (m x np, ld ldy) C (np x np, ld ldc), split-TF32.
bool product_ok(long long m, int np, long long ldo, const float* Out) {
    return m >= 128 && np >= kUpdNJ && (ldo % 4) == 0 && (reinterpret_cast<uintptr_t>(Out) & 15u) == 0;
}

cudaError_t product(Ctx& cx, const float* Y, long long ldy, long long m, const float* C, long long ldc, int np,
                    float* Out, long long ldo, const ReprojScratch& w, bool presplit) {
    cudaError_t e;
    if (!presplit) {
        dim3 g1((unsigned)((m + 31) / 32), (unsigned)(np / 32));
        {
            const cudaError_t le_ = launch_pdl(k_split_q, dim3(g1), dim3(256), 0, cx.stream, Y, ldy, m, np, np,
                                               nullptr, nullptr, 0, w.Yt, w.Ytl, static_cast<const int*>(nullptr));
            if (le_ != cudaSuccess) return le_;
        }
        cx.launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const long long total = (long long)np * np;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 8LL * cx.num_sms);
    {
        const cudaError_t le_ = launch_pdl(k_stage_b, dim3(blocks), dim3(256), 0, cx.stream, C, ldc, np, np, np, w.Bs,
                                           w.Bsl);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return update_impl(cx, nullptr, 0, Out, ldo, m, np, w.Yt, w.Ytl, w.Bs, w.Bsl, np, nullptr, 0, nullptr, 0);
}

// ---------------------------------------------------------------------------
// BF16 storage path.
int pad_block16(int b) { return b <= 64 ? 64 : b <= 128 ? 128 : 256; }

size_t partial_floats16(long long m, long long n, int np, int sms) {
    const Plan a = plan((m + kBM - 1) / kBM, (n + kKC16 - 1) / kKC16, sms);
    const Plan b = plan((n + kBM - 1) / kBM, (m + kKC16 - 1) / kKC16, sms);
    return (size_t)std::max(a.P * a.G, b.P * b.G) * kBM * np;
}

cudaError_t omega16(Ctx& cx, long long n, long long col0, int p, int np, uint64_t seed, __nv_bfloat16* out,
                    long long ldo) {
    const long long total = n * np;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 8LL * cx.num_sms);
    {
        const cudaError_t le_ = launch_pdl(k_omega_bf16<__nv_bfloat16>, dim3(blocks), dim3(256), 0, cx.stream, n, col0,
                                           p, np, seed, out, ldo);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    return cudaGetLastError();
}

cudaError_t omega16_f32(Ctx& cx, long long n, long long col0, int p, int np, uint64_t seed, float* out,
                        long long ldo) {
    const long long total = n * np;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 8LL * cx.num_sms);
    {
        const cudaError_t le_ = launch_pdl(k_omega_bf16<float>, dim3(blocks), dim3(256), 0, cx.stream, n, col0, p, np,
                                           seed, out, ldo);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    return cudaGetLastError();
}

cudaError_t split_q16(Ctx& cx, const float* Qi, long long ldq, long long m, int p, int np, __nv_bfloat16* Qhi,
                      __nv_bfloat16* Qlo, long long ldql, __nv_bfloat16* Qt, __nv_bfloat16* Qtl) {
    dim3 grid((unsigned)((m + 31) / 32), (unsigned)(np / 32));
    {
        const cudaError_t le_ = launch_pdl(k_split_q16, dim3(grid), dim3(256), 0, cx.stream, Qi, ldq, m, p, np, Qhi,
                                           Qlo, ldql, Qt, Qtl);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    return cudaGetLastError();
}

cudaError_t stage_b16(Ctx& cx, const float* Bi, long long ldbi, int p, long long n, int np, __nv_bfloat16* Bs,
                      __nv_bfloat16* Bsl) {
    const long long total = n * np;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 8LL * cx.num_sms);
    {
        const cudaError_t le_ = launch_pdl(k_stage_b16, dim3(blocks), dim3(256), 0, cx.stream, Bi, ldbi, p, n, np, Bs,
                                           Bsl);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    return cudaGetLastError();
}

cudaError_t sketch16(Ctx& cx, const __nv_bfloat16* X, long long ldx, long long m, long long n,
                     const __nv_bfloat16* Om, long long ldom, int np, float* Y, long long ldy, float* part,
                     size_t part_cap, const OmegaGen* gen, double* nrm_part, int nrm_cap, double* nrm_out) {
    StreamKParams p;
    cudaError_t e;
    if ((e = make_map(&p.mx, X, m, n, ldx, 64, kKC16, true)) != cudaSuccess) return e;
    if (gen) {
        if (gen->p < 1 || gen->p > np) return cudaErrorInvalidValue;
        p.om_n = n;
        p.om_col0 = gen->col0;
        p.om_p = gen->p;
        p.om_seed = gen->seed;
        p.mw = p.mx;   // not read
    } else if ((e = make_map(&p.mw, Om, n, np, ldom, kKC16, np, true)) != cudaSuccess) {
        return e;
    }
    p.mwl = p.mw;
    const Plan pl = plan((m + kBM - 1) / kBM, (n + kKC16 - 1) / kKC16, cx.num_sms);
    if ((size_t)pl.P * pl.G * kBM * np > part_cap) return cudaErrorInvalidValue;
    if (nrm_out && pl.P > nrm_cap) return cudaErrorInvalidValue;
    p.part = part;
    p.st = cx.st;
    p.U = pl.U; p.C = pl.C; p.P = pl.P; p.G = pl.G; p.np = np;
    p.nrm_part = nrm_out ? nrm_part : nullptr;
    e = gen ? launch_streamk16<kSketch, true>(cx, p, np) : launch_streamk16<kSketch>(cx, p, np);
    if (e != cudaSuccess) return e;
    const dim3 rgrid(pl.tiles, reduce_slices(pl.tiles, cx.num_sms));
    {
        const cudaError_t le_ = launch_pdl(k_reduce_sketch, dim3(rgrid), dim3(256), 0, cx.stream, part, pl.U, pl.C,
                                           pl.P, pl.G, np, m, Y, ldy, nullptr);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return nrm_out ? launch_sum_doubles(cx, nrm_part, pl.P, nrm_out) : cudaSuccess;
}

cudaError_t project16(Ctx& cx, const __nv_bfloat16* X, long long ldx, long long m, long long n,
                      const __nv_bfloat16* Qhi, const __nv_bfloat16* Qlo, long long ldql, int pcols, int np, float* B,
                      long long ldb, __nv_bfloat16* Bs, __nv_bfloat16* Bsl, float* part, size_t part_cap,
                      double* sq_part, int sq_cap, double* sq_out) {
    StreamKParams p;
    cudaError_t e;
    if ((e = make_map(&p.mx, X, m, n, ldx, kKC16, kBM, true)) != cudaSuccess) return e;
    if ((e = make_map(&p.mw, Qhi, m, np, ldql, kKC16, np, true)) != cudaSuccess) return e;
    if ((e = make_map(&p.mwl, Qlo, m, np, ldql, kKC16, np, true)) != cudaSuccess) return e;
    const Plan pl = plan((n + kBM - 1) / kBM, (m + kKC16 - 1) / kKC16, cx.num_sms);
    const int sl = reduce_slices(pl.tiles, cx.num_sms);
    if ((size_t)pl.P * pl.G * kBM * np > part_cap || pl.tiles * sl > sq_cap) return cudaErrorInvalidValue;
    p.part = part;
    p.st = cx.st;
    p.U = pl.U; p.C = pl.C; p.P = pl.P; p.G = pl.G; p.np = np;
    if ((e = launch_streamk16<kProject>(cx, p, np)) != cudaSuccess) return e;
    {
        const cudaError_t le_ = launch_pdl(k_reduce_project16, dim3(pl.tiles, sl), dim3(256), 0, cx.stream, part, pl.U,
                                           pl.C, pl.P, pl.G, np, pcols, n, B, ldb, Bs, Bsl, sq_part);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_sum_doubles(cx, sq_part, pl.tiles * sl, sq_out);
}

cudaError_t update16(Ctx& cx, const __nv_bfloat16* Wsrc, long long ldws, __nv_bfloat16* Wdst, long long ldwd,
                     long long m, long long n, const __nv_bfloat16* Qt, const __nv_bfloat16* Qtl,
                     const __nv_bfloat16* Bs, const __nv_bfloat16* Bsl, int np, double* sq_part, int sq_cap,
                     double* sq_out) {
    UpdateParams16 p;
    cudaError_t e;
    if (n >= kNJw && m >= kBM && np % kKCw == 0) {
        // 128 x 256 tiles (k_update16w)
        if ((e = make_map_sw64(&p.mqt, Qt, np, m, np, kBM)) != cudaSuccess) return e;
        if ((e = make_map_sw64(&p.mqtl, Qtl, np, m, np, kBM)) != cudaSuccess) return e;
        if ((e = make_map_sw64(&p.mbs, Bs, np, n, np, kNJw)) != cudaSuccess) return e;
        if ((e = make_map_sw64(&p.mbsl, Bsl, np, n, np, kNJw)) != cudaSuccess) return e;
        if ((e = make_map(&p.mws, Wsrc, m, n, ldws, kBM, 64, false)) != cudaSuccess) return e;
        if ((e = make_map(&p.mwd, Wdst, m, n, ldwd, kBM, 64, false)) != cudaSuccess) return e;
        p.st = cx.st;
        p.sq_part = sq_out ? sq_part : nullptr;
        p.m = m; p.n = n;
        p.RT = (int)((m + kBM - 1) / kBM);
        p.CT = (int)((n + kNJw - 1) / kNJw);
        p.C = np / kKCw;
        const long long T = (long long)p.RT * p.CT;
        const int grid = (int)std::min<long long>(cx.num_sms, T);
        if (sq_out && grid > sq_cap) return cudaErrorInvalidValue;
        if ((e = allow_smem(k_update16w, kUpd16wSmem)) != cudaSuccess) return e;
        {
            const cudaError_t le_ = launch_pdl(k_update16w, dim3(grid), dim3(kUpd16Threads), kUpd16wSmem, cx.stream,
                                               p);
            if (le_ != cudaSuccess) return le_;
        }
        cx.launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        return sq_out ? launch_sum_doubles(cx, sq_part, grid, sq_out) : cudaSuccess;
    }
    if ((e = make_map(&p.mqt, Qt, np, m, np, kKC16, kBM, true)) != cudaSuccess) return e;
    if ((e = make_map(&p.mqtl, Qtl, np, m, np, kKC16, kBM, true)) != cudaSuccess) return e;
    if ((e = make_map(&p.mbs, Bs, np, n, np, kKC16, kUpdNJ, true)) != cudaSuccess) return e;
    if ((e = make_map(&p.mbsl, Bsl, np, n, np, kKC16, kUpdNJ, true)) != cudaSuccess) return e;
    if ((e = make_map(&p.mws, Wsrc, m, n, ldws, kBM, kUpdNJ, false)) != cudaSuccess) return e;
    if ((e = make_map(&p.mwd, Wdst, m, n, ldwd, kBM, kUpdNJ, false)) != cudaSuccess) return e;
    p.st = cx.st;
    p.sq_part = sq_out ? sq_part : nullptr;
    p.m = m; p.n = n;
    p.RT = (int)((m + kBM - 1) / kBM);
    p.CT = (int)((n + kUpdNJ - 1) / kUpdNJ);
    p.C = np / kKC16;
    const long long T = (long long)p.RT * p.CT;
    const int grid = (int)std::min<long long>(cx.num_sms, T);
    if (sq_out && grid > sq_cap) return cudaErrorInvalidValue;
    if ((e = allow_smem(k_update16<kUpdNJ, kUpd16Stages>, kUpd16Smem)) != cudaSuccess) return e;
    {
        const cudaError_t le_ = launch_pdl(k_update16<kUpdNJ, kUpd16Stages>, dim3(grid), dim3(kUpd16Threads),
                                           kUpd16Smem, cx.stream, p);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return sq_out ? launch_sum_doubles(cx, sq_part, grid, sq_out) : cudaSuccess;
}

// ---------------------------------------------------------------------------
// Line (3'): Y <- Y - Qbar (Qbar^T Y) with the split-TF32 products.
bool reproject_ok(long long m, long long kprev) { return m >= 128 && kprev >= 128; }

cudaError_t reproject(Ctx& cx, const float* Qbar, long long ldq, long long m, long long kprev, float* Y,
                      long long ldy, int np, const ReprojScratch& w) {
    cudaError_t e;
    // C^T = Y^T Qbar (np x kprev): the projection kernel with X = Qbar and Y in
    // the place of Q_i
    dim3 g1((unsigned)((m + 31) / 32), (unsigned)(np / 32));
    {
        const cudaError_t le_ = launch_pdl(k_split_q, dim3(g1), dim3(256), 0, cx.stream, Y, ldy, m, np, np, w.Yhi,
                                           w.Ylo, w.ldyl, nullptr, nullptr, static_cast<const int*>(nullptr));
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = project64(cx, Qbar, ldq, m, kprev, w.Yhi, w.Ylo, w.ldyl, np, np, w.Ct64, np, w.part,
                       w.part_cap)) != cudaSuccess)
        return e;
    // C in the sketch's Omega layout (rounded to TF32), then Y -= Qbar C
    dim3 g2((unsigned)((kprev + 31) / 32), (unsigned)(np / 32));
    {
        const cudaError_t le_ = launch_pdl(k_ct_to_omega<double>, dim3(g2), dim3(256), 0, cx.stream, w.Ct64, np, kprev,
                                           np, w.Om, w.ldom, static_cast<float*>(nullptr), 0LL);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return sketch_sub(cx, Qbar, ldq, m, kprev, w.Om, w.ldom, np, Y, ldy, Y, w.part, w.part_cap);
}

bool reproject_gram_ok(long long m, long long kprev, int np, long long ldy, const float* Y, const ReprojScratch& w) {
    if (!(reproject_ok(m, kprev) && kprev % kBM == 0 && np % 32 == 0 && np <= 64 * 32 && gram_ok(m, np, ldy, Y)))
        return false;
    const size_t tiles = (size_t)(np / 32) * (np / 32 + 1) / 2;
    return 2 * tiles * (size_t)(kprev / 128) * 1024 <= w.part_cap;
}

cudaError_t reproject_gram(Ctx& cx, const float* Qbar, long long ldq, long long m, long long kprev, float* Y,
                           long long ldy, int np, const ReprojScratch& w, double* G, int* fused,
                           double* trace_part) {
    cudaError_t e;
    dim3 g1((unsigned)((m + 31) / 32), (unsigned)(np / 32));
    {
        const cudaError_t le_ = launch_pdl(k_split_q, dim3(g1), dim3(256), 0, cx.stream, Y, ldy, m, np, np, w.Yhi,
                                           w.Ylo, w.ldyl, nullptr, nullptr, static_cast<const int*>(nullptr));
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // Y^T [Qbar Y]: C^T in columns 0 .. kprev - 1 of w.Ct64 (ld np), S = Y^T Y after them
    if ((e = project64(cx, Qbar, ldq, m, kprev, w.Yhi, w.Ylo, w.ldyl, np, np, w.Ct64, np, w.part, w.part_cap,
                       false, Y, ldy, np)) != cudaSuccess)
        return e;
    dim3 g2((unsigned)((kprev + 31) / 32), (unsigned)(np / 32));
    {
        const cudaError_t le_ = launch_pdl(k_ct_to_omega<double>, dim3(g2), dim3(256), 0, cx.stream, w.Ct64, np, kprev,
                                           np, w.Om, w.ldom, w.Ct, kprev);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = sketch_sub(cx, Qbar, ldq, m, kprev, w.Om, w.ldom, np, Y, ldy, Y, w.part, w.part_cap)) != cudaSuccess)
        return e;
    // the sketch's partials are consumed: its buffer holds the parts of C^T C,
    // formed from the FP32 copy of C (w.Ct, kprev x np) made beside Om
    const int nb = np / 32, tiles = nb * (nb + 1) / 2, KS = (int)(kprev / 128);
    double* parts = reinterpret_cast<double*>(w.part);
    {
        const cudaError_t le_ = launch_pdl(k_gram_part, dim3(tiles, KS), dim3(256), 0, cx.stream,
                                           static_cast<const float*>(w.Ct), kprev, kprev, parts);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    {
        const cudaError_t le_ = launch_pdl(k_gram_fin, dim3(tiles), dim3(256), 0, cx.stream,
                                           static_cast<const double*>(w.Ct64 + (size_t)kprev * np), (long long)np,
                                           static_cast<const double*>(parts), KS, np, G, trace_part);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    {
        const cudaError_t le_ = launch_pdl(k_gram_gate, dim3(1), dim3(32), 0, cx.stream,
                                           static_cast<const double*>(trace_part), nb, 0.05, fused, cx.st);
        if (le_ != cudaSuccess) return le_;
    }
    cx.launches++;
    return cudaGetLastError();
}

cudaError_t wait_selftest(Ctx& cx, unsigned long long* waited_ns) {
    k_wait_selftest<<<1, 32, 0, cx.stream>>>(cx.st, waited_ns);
    cx.launches++;
    return cudaGetLastError();
}

}  // namespace tc
}  // namespace rqb
