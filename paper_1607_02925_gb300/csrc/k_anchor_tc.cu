// Anchor-pass products on the 5th-generation tensor cores (tcgen05), for X
// stored in BF16:
//   xtw_tc_kernel: Y = X^T W  — M = 128 data points per CTA, N = PP, K = d.
//   xy_tc_kernel:  G = X Y    — M = 128 rows of X per CTA, N = PP, K = a chunk
//                               of columns (split-K; fixed-order reduction after).
// X tiles and the small operand stream through shared memory by TMA
// (128-byte swizzle) in a multi-stage mbarrier pipeline; one thread issues the
// MMAs into a TMEM accumulator; four warps read it back with tcgen05.ld.  The
// FP32 small operand is split into BF16 hi + lo, both multiplied into the same
// accumulator, so its rounding error is ~2^-17 instead of 2^-9.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "kernels.cuh"
#include "tc_common.cuh"

namespace lra {

namespace {

using namespace tc;

constexpr int kBM = 128;                // rows of the MMA tile
constexpr int kBK = 64;                 // K elements per pipeline stage (128 B of BF16)
constexpr int kATile = kBM * kBK * 2;   // 16 KB
constexpr int kAccCols1 = 128;          // TMEM columns per accumulator (PP <= 112)

__device__ __forceinline__ uint8_t *align1024(uint8_t *p) {
    return reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

// NA = 1: X stored in BF16.  NA = 2: X stored in FP32 and streamed as its
// BF16 hi + lo pair (x = hi + lo + r, |r| <= 2^-17 |x|).
// MT = number of 128-row M tiles per work tile sharing each small-operand tile
// (MT accumulators): halves the small operand's L2 traffic and doubles the X
// bytes in flight per stage.
//
// The kernels are persistent: one CTA per SM walks the work tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...  Warp 0 (one lane) streams the
// stages by TMA through a ring that runs on across tiles, warp 1 (one lane)
// issues the MMAs, and warps 2-5 drain the accumulators.  TMEM holds two
// accumulator sets, so the drain of tile t overlaps the MMAs of tile t + 1.
template <int PP, int NA, int MT>
struct Tile {
    static constexpr int kA1 = NA * kATile;         // one M tile: hi [+ lo]
    static constexpr int kA = MT * kA1;
    static constexpr int kB = PP * 128;             // one of hi / lo: PP rows x 128 B
    static constexpr int kStage = kA + 2 * kB;      // multiple of 1024
    static constexpr int kFit = (216 * 1024) / kStage;
    static constexpr int kStages = kFit > 6 ? 6 : kFit;
    static constexpr int kSmem = kStages * kStage + 1024 + 512;
    static constexpr uint32_t kAccCols = MT * kAccCols1;  // one accumulator set
    static constexpr uint32_t kTmemCols = 2 * kAccCols;   // two sets (<= 512)
    static_assert(kStages >= 2, "pipeline needs two stages");
};

constexpr int kThreads = 192;  // producer warp, MMA warp, four epilogue warps

// Control block after the stages: ring barriers, accumulator barriers, the
// MMA issuer's unwinding barrier, TMEM address.
struct Ctl {
    uint64_t full[6], empty[6], accf[2], acce[2], mmadone;
    uint32_t tmem;
};

// K blocks accumulated into one TMEM accumulator before the epilogue reads it
// out and adds it in FP32 registers (round to nearest).  The tensor core's
// FP32 accumulation does not round to nearest: every MMA shortens the running
// sum slightly toward zero, a bias that grows with the number of MMAs into one
// accumulator (about 1.3e-5 relative after the 768 MMAs of a 4096-long FP32
// pair product).  Restarting the accumulator every 4 K blocks (48 MMAs) keeps
// that bias near 1e-6 for the FP32 pair; BF16 X (relative tolerance 1e-2)
// keeps one accumulator per tile.
template <int NA>
__host__ __device__ constexpr int seg_kb() { return NA == 2 ? 4 : (1 << 30); }

template <int PP, int NA, int MT>
__device__ __forceinline__ void init_ctl(Ctl *ctl) {
    using T = Tile<PP, NA, MT>;
    for (int s = 0; s < T::kStages; ++s) {
        mbar_init(&ctl->full[s], 1);
        mbar_init(&ctl->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
        mbar_init(&ctl->accf[b], 1);
        mbar_init(&ctl->acce[b], 4);  // one arrival per epilogue warp
    }
    mbar_init(&ctl->mmadone, 1);
    fence_barrier_init();
}

// After an error the producer waits (bounded) for the stages it still has in
// flight, so that no TMA write lands after the CTA has exited.
template <int S>
__device__ __forceinline__ void drain_issued(Ctl *ctl, int issued) {
    for (int g = (issued > S ? issued - S : 0); g < issued; ++g)
        mbar_wait(&ctl->full[g % S], (uint32_t)(g / S) & 1u);
}

// After an error the MMA issuer waits (bounded) until every MMA it issued has
// completed, so that none writes TMEM once the CTA frees it.
__device__ __forceinline__ void drain_mmas(Ctl *ctl) {
    mma_commit(&ctl->mmadone);
    mbar_wait(&ctl->mmadone, 0u);
}

// ---------------------------------------------------------------------------
// Y = X^T W: work tile = MT x 128 data points (rows of X^T), K = d
// ---------------------------------------------------------------------------
// FMT = 1: BF16 operands.  FMT = 0: FP16 operands (FP16 storage): X holds
// fp16(xscale x), the small operand fp16 hi / lo of w sw, and tcs holds the
// scales: tcs[0] = sw, tcs[1] = 1 / (xscale sw), tcs[2 + c] = sy_c (the
// multiplier of column c of Y in its FP16 hi / lo copy), tcs[2 + PP + c] =
// 1 / (xscale sy_c).  All are powers of two, so the scaling is exact.
template <int PP, int NA, int MT, int FMT>
__global__ void __launch_bounds__(kThreads, 1) xtw_tc_kernel(const __grid_constant__ CUtensorMap tmX,
                                                             const __grid_constant__ CUtensorMap tmXl,
                                                             const __grid_constant__ CUtensorMap tmW,
                                                             int nkb, int64_t n, float *__restrict__ Y32,
                                                             uint16_t *__restrict__ Yb, int64_t ldy,
                                                             int *__restrict__ err, long long lim,
                                                             const float *__restrict__ tcs) {
    using T = Tile<PP, NA, MT>;
    constexpr int S = T::kStages;
    constexpr int KS = seg_kb<NA>();
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = align1024(smem_raw);
    Ctl *ctl = reinterpret_cast<Ctl *>(smem + S * T::kStage);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles = (int)((n + kBM * MT - 1) / (kBM * MT));

    if (threadIdx.x == 0) {
        init_ctl<PP, NA, MT>(ctl);
        prefetch_tmap(&tmX);
        if (NA == 2) prefetch_tmap(&tmXl);
        prefetch_tmap(&tmW);
    }
    if (warp == 1) {
        tmem_alloc(&ctl->tmem, T::kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl->tmem;

    if (warp == 0 && lane == 0) {
        // TMA producer: one ring position per (tile, k-block)
        int g = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const int64_t i0 = (int64_t)tile * kBM * MT;
            for (int kb = 0; kb < nkb; ++kb, ++g) {
                const int st = g % S;
                if (g >= S && !mbar_wait(&ctl->empty[st], ((uint32_t)(g / S) & 1u) ^ 1u, lim)) {
                    atomicOr(err, kErrTimeout);
                    ok = false;
                    break;
                }
                uint8_t *a = smem + st * T::kStage;
                mbar_expect_tx(&ctl->full[st], T::kStage);
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) {
                    const int row = (int)i0 + mt * kBM;
                    tma_load_2d(a + mt * T::kA1, &tmX, kb * kBK, row, &ctl->full[st]);
                    if (NA == 2) tma_load_2d(a + mt * T::kA1 + kATile, &tmXl, kb * kBK, row, &ctl->full[st]);
                }
                tma_load_2d(a + T::kA, &tmW, kb * kBK, 0, &ctl->full[st]);
                tma_load_2d(a + T::kA + T::kB, &tmW, kb * kBK, PP, &ctl->full[st]);
            }
        }
        if (!ok) drain_issued<S>(ctl, g);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: the K blocks of a tile form segments of KS; segment sc
        // (counted over the CTA's whole walk) accumulates into set sc & 1
        constexpr uint32_t idesc = instr_desc(FMT, 0, 0, PP, kBM);
        int g = 0, sc = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            for (int s0 = 0; s0 < nkb && ok; s0 += KS, ++sc) {
                const int buf = sc & 1;
                if (sc >= 2 && !mbar_wait(&ctl->acce[buf], (uint32_t)((sc >> 1) - 1) & 1u, lim)) {
                    atomicOr(err, kErrTimeout);
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t accb = tmem + buf * T::kAccCols;
                const int s1 = (nkb - s0 < KS) ? nkb : s0 + KS;
                for (int kb = s0; kb < s1; ++kb, ++g) {
                    const int st = g % S;
                    if (!mbar_wait(&ctl->full[st], (uint32_t)(g / S) & 1u, lim)) {
                        atomicOr(err, kErrTimeout);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a = smem_u32(smem + st * T::kStage);
                    const uint32_t bh = a + T::kA, bl = bh + T::kB;
#pragma unroll
                    for (int ks = 0; ks < kBK / 16; ++ks) {
                        const uint64_t bhd = sw128_desc(bh + ks * 32, 16, 1024);
                        const uint64_t bld = sw128_desc(bl + ks * 32, 16, 1024);
#pragma unroll
                        for (int mt = 0; mt < MT; ++mt) {
                            const uint32_t am = a + mt * T::kA1;
                            const uint32_t acc = accb + mt * kAccCols1;
                            const uint64_t ad = sw128_desc(am + ks * 32, 16, 1024);
                            mma_f16(acc, ad, bhd, idesc, ((kb - s0) | ks) != 0);
                            mma_f16(acc, ad, bld, idesc, 1u);
                            if (NA == 2) mma_f16(acc, sw128_desc(am + kATile + ks * 32, 16, 1024), bhd, idesc, 1u);
                        }
                    }
                    mma_commit(&ctl->empty[st]);
                }
                if (ok) mma_commit(&ctl->accf[buf]);
            }
        }
        if (!ok) drain_mmas(ctl);
    } else if (warp >= 2) {
        // epilogue: warp w drains TMEM lanes 32 (w % 4) .. + 31 of every M tile
        const int q = warp & 3;
        int sc = 0;
        bool ok = true;
        const float ysc = FMT == 0 ? tcs[1] : 1.0f;
        auto store = [&](int64_t i, int c, const float *v0) {
            if (i >= n) return;
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = FMT == 0 ? v0[j] * ysc : v0[j];
            if (Y32) {
                float4 *dst = reinterpret_cast<float4 *>(Y32 + i * PP + c);
#pragma unroll
                for (int u = 0; u < 4; ++u) dst[u] = make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
            }
            if (Yb) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    uint16_t hi, lo;
                    if constexpr (FMT == 0) {
                        const float y = v[j] * tcs[2 + c + j];
                        const __half h = __float2half_rn(y);
                        hi = __half_as_ushort(h);
                        lo = __half_as_ushort(__float2half_rn(y - __half2float(h)));
                    } else {
                        const __nv_bfloat16 h = __float2bfloat16_rn(v[j]);
                        hi = __bfloat16_as_ushort(h);
                        lo = __bfloat16_as_ushort(__float2bfloat16_rn(v[j] - __bfloat162float(h)));
                    }
                    Yb[(int64_t)(c + j) * ldy + i] = hi;
                    Yb[(int64_t)(PP + c + j) * ldy + i] = lo;
                }
            }
        };
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const int64_t i0 = (int64_t)tile * kBM * MT;
            if constexpr (NA == 2) {
                // MT = 1: the segments' partial sums are added in registers
                float accv[PP];
                for (int s0 = 0; s0 < nkb; s0 += KS, ++sc) {
                    const int buf = sc & 1;
                    if (!mbar_wait(&ctl->accf[buf], (uint32_t)(sc >> 1) & 1u, lim)) {
                        if (lane == 0) atomicOr(err, kErrTimeout);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + buf * T::kAccCols;
#pragma unroll
                    for (int c = 0; c < PP; c += 16) {
                        float v[16];
                        tmem_ld16(tl + c, v);
#pragma unroll
                        for (int j = 0; j < 16; ++j) accv[c + j] = (s0 == 0) ? v[j] : accv[c + j] + v[j];
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&ctl->acce[buf]);
                }
                if (!ok) break;
                const int64_t i = i0 + q * 32 + lane;
#pragma unroll
                for (int c = 0; c < PP; c += 16) store(i, c, accv + c);
            } else {
                // one segment per tile
                const int buf = sc & 1;
                if (!mbar_wait(&ctl->accf[buf], (uint32_t)(sc >> 1) & 1u, lim)) {
                    if (lane == 0) atomicOr(err, kErrTimeout);
                    break;
                }
                tc_fence_after();
#pragma unroll 1
                for (int mt = 0; mt < MT; ++mt) {
                    const int64_t i = i0 + mt * kBM + q * 32 + lane;
                    const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + buf * T::kAccCols + mt * kAccCols1;
#pragma unroll
                    for (int c = 0; c < PP; c += 16) {
                        float v[16];
                        tmem_ld16(tl + c, v);
                        store(i, c, v);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&ctl->acce[buf]);
                ++sc;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, T::kTmemCols);
    }
}

// ---------------------------------------------------------------------------
// Partial G = X[rows, chunk] Y[chunk, :] (X is the MN-major operand here).
// Work tile = (MT x 128 rows of X, one column chunk); row tiles vary fastest,
// so the CTAs in flight share the chunk's Y tiles in L2.
// ---------------------------------------------------------------------------
template <int PP, int NA, int MT, int FMT>
__global__ void __launch_bounds__(kThreads, 1) xy_tc_kernel(const __grid_constant__ CUtensorMap tmX,
                                                            const __grid_constant__ CUtensorMap tmXl,
                                                            const __grid_constant__ CUtensorMap tmY,
                                                            int64_t cols_per_chunk, int nchunks, int64_t n,
                                                            int64_t dpad, float *__restrict__ Gp,
                                                            int *__restrict__ err, long long lim) {
    using T = Tile<PP, NA, MT>;
    constexpr int S = T::kStages;
    constexpr int KS = seg_kb<NA>();
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = align1024(smem_raw);
    Ctl *ctl = reinterpret_cast<Ctl *>(smem + S * T::kStage);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rtiles = (int)((dpad + kBM * MT - 1) / (kBM * MT));
    const int ntiles = rtiles * nchunks;
    // K blocks of a chunk (0 for an empty chunk)
    auto chunk_kb = [&](int ch, int64_t &c0) {
        c0 = (int64_t)ch * cols_per_chunk;
        const int64_t c1 = (c0 + cols_per_chunk < n) ? c0 + cols_per_chunk : n;
        return c1 > c0 ? (int)((c1 - c0 + kBK - 1) / kBK) : 0;
    };

    if (threadIdx.x == 0) {
        init_ctl<PP, NA, MT>(ctl);
        prefetch_tmap(&tmX);
        if (NA == 2) prefetch_tmap(&tmXl);
        prefetch_tmap(&tmY);
    }
    if (warp == 1) {
        tmem_alloc(&ctl->tmem, T::kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl->tmem;

    if (warp == 0 && lane == 0) {
        int g = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const int rt = tile % rtiles, ch = tile / rtiles;
            const int64_t r0 = (int64_t)rt * kBM * MT;
            int64_t c0;
            const int nkb = chunk_kb(ch, c0);
            for (int kb = 0; kb < nkb; ++kb, ++g) {
                const int st = g % S;
                if (g >= S && !mbar_wait(&ctl->empty[st], ((uint32_t)(g / S) & 1u) ^ 1u, lim)) {
                    atomicOr(err, kErrTimeout);
                    ok = false;
                    break;
                }
                uint8_t *a = smem + st * T::kStage;
                const int col = (int)(c0 + (int64_t)kb * kBK);
                mbar_expect_tx(&ctl->full[st], T::kStage);
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) {
                    // rows past dpad (an odd number of 128-row tiles) read as zeros
                    const int row = (int)r0 + mt * kBM;
                    uint8_t *am = a + mt * T::kA1;
                    tma_load_2d(am, &tmX, row, col, &ctl->full[st]);
                    tma_load_2d(am + kATile / 2, &tmX, row + 64, col, &ctl->full[st]);
                    if (NA == 2) {
                        tma_load_2d(am + kATile, &tmXl, row, col, &ctl->full[st]);
                        tma_load_2d(am + kATile + kATile / 2, &tmXl, row + 64, col, &ctl->full[st]);
                    }
                }
                tma_load_2d(a + T::kA, &tmY, col, 0, &ctl->full[st]);
                tma_load_2d(a + T::kA + T::kB, &tmY, col, PP, &ctl->full[st]);
            }
        }
        if (!ok) drain_issued<S>(ctl, g);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: segments of KS K blocks; segment sc accumulates into set
        // sc & 1 (an empty chunk is one empty segment, drained as zeros)
        constexpr uint32_t idesc = instr_desc(FMT, 1, 0, PP, kBM);
        int g = 0, sc = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            int64_t c0;
            const int nkb = chunk_kb(tile / rtiles, c0);
            const int nseg = nkb > 0 ? (nkb + KS - 1) / KS : 1;
            for (int sg = 0; sg < nseg && ok; ++sg, ++sc) {
                const int buf = sc & 1;
                if (sc >= 2 && !mbar_wait(&ctl->acce[buf], (uint32_t)((sc >> 1) - 1) & 1u, lim)) {
                    atomicOr(err, kErrTimeout);
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t accb = tmem + buf * T::kAccCols;
                const int s0 = sg * KS;
                const int s1 = (nkb - s0 < KS) ? nkb : s0 + KS;
                for (int kb = s0; kb < s1; ++kb, ++g) {
                    const int st = g % S;
                    if (!mbar_wait(&ctl->full[st], (uint32_t)(g / S) & 1u, lim)) {
                        atomicOr(err, kErrTimeout);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a = smem_u32(smem + st * T::kStage);
                    const uint32_t bh = a + T::kA, bl = bh + T::kB;
#pragma unroll
                    for (int ks = 0; ks < kBK / 16; ++ks) {
                        const uint64_t bhd = sw128_desc(bh + ks * 32, 16, 1024);
                        const uint64_t bld = sw128_desc(bl + ks * 32, 16, 1024);
#pragma unroll
                        for (int mt = 0; mt < MT; ++mt) {
                            // A: 64-row MN blocks 8 KB apart, 8-column K groups 1 KB apart
                            const uint32_t am = a + mt * T::kA1;
                            const uint32_t acc = accb + mt * kAccCols1;
                            const uint64_t ad = sw128_desc(am + ks * 2048, kATile / 2, 1024);
                            mma_f16(acc, ad, bhd, idesc, ((kb - s0) | ks) != 0);
                            mma_f16(acc, ad, bld, idesc, 1u);
                            if (NA == 2)
                                mma_f16(acc, sw128_desc(am + kATile + ks * 2048, kATile / 2, 1024), bhd, idesc, 1u);
                        }
                    }
                    mma_commit(&ctl->empty[st]);
                }
                if (ok) mma_commit(&ctl->accf[buf]);
            }
        }
        if (!ok) drain_mmas(ctl);
    } else if (warp >= 2) {
        const int q = warp & 3;
        int sc = 0;
        bool ok = true;
        auto store = [&](float *out, int64_t r, int c, const float *v) {
            if (r < dpad) {
                float4 *dst = reinterpret_cast<float4 *>(out + c);
#pragma unroll
                for (int u = 0; u < 4; ++u) dst[u] = make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
            }
        };
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const int rt = tile % rtiles, ch = tile / rtiles;
            int64_t c0;
            const int nkb = chunk_kb(ch, c0);
            const int nseg = nkb > 0 ? (nkb + KS - 1) / KS : 1;
            const int64_t r0 = (int64_t)rt * kBM * MT;
            if constexpr (NA == 2) {
                // MT = 1: the segments' partial sums are added in registers
                float accv[PP];
                for (int sg = 0; sg < nseg; ++sg, ++sc) {
                    const int buf = sc & 1;
                    if (!mbar_wait(&ctl->accf[buf], (uint32_t)(sc >> 1) & 1u, lim)) {
                        if (lane == 0) atomicOr(err, kErrTimeout);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + buf * T::kAccCols;
#pragma unroll
                    for (int c = 0; c < PP; c += 16) {
                        float v[16];
                        if (nkb > 0) {
                            tmem_ld16(tl + c, v);
                        } else {
#pragma unroll
                            for (int u = 0; u < 16; ++u) v[u] = 0.0f;
                        }
#pragma unroll
                        for (int j = 0; j < 16; ++j) accv[c + j] = (sg == 0) ? v[j] : accv[c + j] + v[j];
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&ctl->acce[buf]);
                }
                if (!ok) break;
                const int64_t r = r0 + q * 32 + lane;
                float *out = Gp + (int64_t)ch * dpad * PP + r * PP;
#pragma unroll
                for (int c = 0; c < PP; c += 16) store(out, r, c, accv + c);
            } else {
                const int buf = sc & 1;
                if (!mbar_wait(&ctl->accf[buf], (uint32_t)(sc >> 1) & 1u, lim)) {
                    if (lane == 0) atomicOr(err, kErrTimeout);
                    break;
                }
                tc_fence_after();
#pragma unroll 1
                for (int mt = 0; mt < MT; ++mt) {
                    const int64_t r = r0 + mt * kBM + q * 32 + lane;
                    float *out = Gp + (int64_t)ch * dpad * PP + r * PP;
                    const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + buf * T::kAccCols + mt * kAccCols1;
#pragma unroll
                    for (int c = 0; c < PP; c += 16) {
                        float v[16];
                        if (nkb > 0) {
                            tmem_ld16(tl + c, v);
                        } else {
#pragma unroll
                            for (int u = 0; u < 16; ++u) v[u] = 0.0f;
                        }
                        store(out, r, c, v);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&ctl->acce[buf]);
                ++sc;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, T::kTmemCols);
    }
}

// ---------------------------------------------------------------------------
// operand preparation
// ---------------------------------------------------------------------------
// Wb[j][r] = hi / Wb[PP + j][r] = lo of W[r + j ld] (zero for j >= p)
__global__ void pack_hilo_kernel(const float *__restrict__ W, int64_t ld, int64_t rows, int p, int PP,
                                 __nv_bfloat16 *__restrict__ Wb) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * PP) return;
    const int j = (int)(e / rows);
    const int64_t r = e % rows;
    const float w = j < p ? W[r + (int64_t)j * ld] : 0.0f;
    const __nv_bfloat16 hi = __float2bfloat16_rn(w);
    Wb[e] = hi;
    Wb[(int64_t)PP * rows + e] = __float2bfloat16_rn(w - __bfloat162float(hi));
}

// X (FP32, dpad x ncols) -> BF16 hi + lo with x = hi + lo + r, |r| <= 2^-17 |x|
__global__ void split_hilo_kernel(const float *__restrict__ X, int64_t count, __nv_bfloat16 *__restrict__ Xh,
                                  __nv_bfloat16 *__restrict__ Xl) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        const float x = X[e];
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        Xh[e] = hi;
        Xl[e] = __float2bfloat16_rn(x - __bfloat162float(hi));
    }
}

// Yb (hi/lo, column-major, leading dim ldy) from Y (n x PP row-major FP32)
// FP16 operands (FP16 storage): scales from the block W.  sw puts
// max |w| in [2^13, 2^14); sy_c bounds column c of Y = X^T W through
// |y_ic| <= ||x_i|| ||w_c|| <= sqrt(max_i ||x_i||^2) ||w_c|| and puts the bound
// in [2^13, 2^14), so the FP16 hi / lo copy of Y never overflows and its
// typical entries stay in FP16's normal range.
__device__ __forceinline__ float pow2_below(float target, float v) {
    // the largest power of two s with s v < target (1 for v = 0 or non-finite v)
    if (!(v > 0.0f) || !isfinite(v)) return 1.0f;
    int e = 0;
    frexpf(target / v, &e);  // target / v in [2^(e-1), 2^e)
    return ldexpf(1.0f, e - 1);
}

// Per column c (one CTA each): ||w_c|| gives sy_c; max |w_c| goes to
// tcs[2 + 2 PP + c] for the block maximum taken by tc_sw_kernel.
__global__ void __launch_bounds__(256) tc_colstats_kernel(const float *__restrict__ W, int64_t ld, int64_t rows,
                                                          int p, int PP, float xscale, float xmaxnorm,
                                                          float *__restrict__ tcs) {
    __shared__ float smax[256];
    __shared__ double snorm[256];
    const int c = blockIdx.x;
    float mx = 0.0f;
    double a = 0.0;
    if (c < p)
        for (int64_t r = threadIdx.x; r < rows; r += 256) {
            const float w = W[r + (int64_t)c * ld];
            mx = fmaxf(mx, fabsf(w));
            a += (double)w * (double)w;
        }
    smax[threadIdx.x] = mx;
    snorm[threadIdx.x] = a;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            smax[threadIdx.x] = fmaxf(smax[threadIdx.x], smax[threadIdx.x + w]);
            snorm[threadIdx.x] += snorm[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const float sy = pow2_below(16384.0f, xmaxnorm * (float)sqrt(snorm[0]));
        tcs[2 + c] = sy;
        tcs[2 + PP + c] = 1.0f / (xscale * sy);
        tcs[2 + 2 * PP + c] = smax[0];
    }
}

// sw from the column maxima (one warp, fixed order)
__global__ void tc_sw_kernel(int PP, float xscale, float *__restrict__ tcs) {
    float mx = 0.0f;
    for (int c = threadIdx.x; c < PP; c += 32) mx = fmaxf(mx, tcs[2 + 2 * PP + c]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (threadIdx.x == 0) {
        const float sw = pow2_below(16384.0f, mx);
        tcs[0] = sw;
        tcs[1] = 1.0f / (xscale * sw);
    }
}

// Wb[j][r] = hi / Wb[PP + j][r] = lo of sw W[r + j ld] in FP16 (zero for j >= p)
__global__ void pack_hilo_f16_kernel(const float *__restrict__ W, int64_t ld, int64_t rows, int p, int PP,
                                     const float *__restrict__ tcs, __half *__restrict__ Wb) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * PP) return;
    const int j = (int)(e / rows);
    const int64_t r = e % rows;
    const float w = j < p ? W[r + (int64_t)j * ld] * tcs[0] : 0.0f;
    const __half hi = __float2half_rn(w);
    Wb[e] = hi;
    Wb[(int64_t)PP * rows + e] = __float2half_rn(w - __half2float(hi));
}

// FP16 copy of a given FP32 Y: sy_c from the column maxima of Y (one CTA per column)
__global__ void __launch_bounds__(256) y_scales_kernel(const float *__restrict__ Y, int64_t n, int PP, int p,
                                                       float xscale, float *__restrict__ tcs) {
    __shared__ float smax[256];
    const int c = blockIdx.x;
    float mx = 0.0f;
    if (c < p)
        for (int64_t i = threadIdx.x; i < n; i += 256) mx = fmaxf(mx, fabsf(Y[i * PP + c]));
    smax[threadIdx.x] = mx;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) smax[threadIdx.x] = fmaxf(smax[threadIdx.x], smax[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const float sy = pow2_below(16384.0f, smax[0]);
        tcs[2 + c] = sy;
        tcs[2 + PP + c] = 1.0f / (xscale * sy);
    }
}

__global__ void y_hilo_f16_kernel(const float *__restrict__ Y, int64_t n, int PP, const float *__restrict__ tcs,
                                  __half *__restrict__ Yb, int64_t ldy) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * PP) return;
    const int j = (int)(e / n);
    const int64_t i = e % n;
    const float y = Y[i * PP + j] * tcs[2 + j];
    const __half hi = __float2half_rn(y);
    Yb[(int64_t)j * ldy + i] = hi;
    Yb[(int64_t)(PP + j) * ldy + i] = __float2half_rn(y - __half2float(hi));
}

__global__ void y_hilo_kernel(const float *__restrict__ Y, int64_t n, int PP, __nv_bfloat16 *__restrict__ Yb,
                              int64_t ldy) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * PP) return;
    const int j = (int)(e / n);
    const int64_t i = e % n;
    const float y = Y[i * PP + j];
    const __nv_bfloat16 hi = __float2bfloat16_rn(y);
    Yb[(int64_t)j * ldy + i] = hi;
    Yb[(int64_t)(PP + j) * ldy + i] = __float2bfloat16_rn(y - __bfloat162float(hi));
}

// ---------------------------------------------------------------------------
// host: tensor maps
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::mutex mu;
    std::lock_guard<std::mutex> g(mu);
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        LRA_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !p) {
            set_error("cuTensorMapEncodeTiled not available");
            throw Error{LRA_ECUDA};
        }
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D BF16 tensor: dim0 (contiguous) = e0 elements, dim1 = e1, row pitch ld0
// elements; box = b0 x b1; 128-byte swizzle; out-of-range reads return 0.
CUtensorMap make_map(const void *base, uint64_t e0, uint64_t e1, uint64_t ld0, uint32_t b0, uint32_t b1,
                     bool f16 = false) {
    CUtensorMap m;
    const cuuint64_t dims[2] = {e0, e1};
    const cuuint64_t strides[1] = {ld0 * 2};
    const cuuint32_t box[2] = {b0, b1};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = encode_fn()(&m, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                                   const_cast<void *>(base), dims, strides,
                                   box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
        throw Error{LRA_ECUDA};
    }
    return m;
}

// Streaming multiprocessors of the current device (one persistent CTA each).
int sm_count() {
    int dev = 0, v = 0;
    LRA_CUDA(cudaGetDevice(&dev));
    LRA_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
    return v > 0 ? v : 1;
}

template <typename F>
void dispatch_tc_pp(int PP, F &&f) {
    switch (PP) {
        case 16: f(std::integral_constant<int, 16>{}); break;
        case 32: f(std::integral_constant<int, 32>{}); break;
        case 48: f(std::integral_constant<int, 48>{}); break;
        case 64: f(std::integral_constant<int, 64>{}); break;
        case 80: f(std::integral_constant<int, 80>{}); break;
        case 96: f(std::integral_constant<int, 96>{}); break;
        case 112: f(std::integral_constant<int, 112>{}); break;
        default:
            set_error("unsupported padded p " + std::to_string(PP));
            throw Error{LRA_EUNSUPPORTED};
    }
}

}  // namespace

int64_t tc_ldy(int64_t n) { return round_up(n, 64); }

void pack_hilo(cudaStream_t s, const float *W, int64_t ld, int64_t rows, int p, int PP, __nv_bfloat16 *Wb) {
    pack_hilo_kernel<<<(unsigned)ceil_div(rows * PP, 256), 256, 0, s>>>(W, ld, rows, p, PP, Wb);
    LRA_LAUNCHED();
}

void y_hilo(cudaStream_t s, const float *Y, int64_t n, int PP, __nv_bfloat16 *Yb, int64_t ldy) {
    y_hilo_kernel<<<(unsigned)ceil_div(n * PP, 256), 256, 0, s>>>(Y, n, PP, Yb, ldy);
    LRA_LAUNCHED();
}

void pack_hilo_f16(cudaStream_t s, const float *W, int64_t ld, int64_t rows, int p, int PP, float xscale,
                   double xmaxnorm, float *tcs, __half *Wb) {
    tc_colstats_kernel<<<(unsigned)PP, 256, 0, s>>>(W, ld, rows, p, PP, xscale, (float)xmaxnorm, tcs);
    LRA_LAUNCHED();
    tc_sw_kernel<<<1, 32, 0, s>>>(PP, xscale, tcs);
    LRA_LAUNCHED();
    pack_hilo_f16_kernel<<<(unsigned)ceil_div(rows * PP, 256), 256, 0, s>>>(W, ld, rows, p, PP, tcs, Wb);
    LRA_LAUNCHED();
}

void y_hilo_f16(cudaStream_t s, const float *Y, int64_t n, int PP, int p, float xscale, float *tcs, __half *Yb,
                int64_t ldy) {
    y_scales_kernel<<<(unsigned)PP, 256, 0, s>>>(Y, n, PP, p, xscale, tcs);
    LRA_LAUNCHED();
    y_hilo_f16_kernel<<<(unsigned)ceil_div(n * PP, 256), 256, 0, s>>>(Y, n, PP, tcs, Yb, ldy);
    LRA_LAUNCHED();
}

void split_hilo(cudaStream_t s, const float *X, int64_t count, __nv_bfloat16 *Xh, __nv_bfloat16 *Xl) {
    const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(count, 256), 152 * 64);
    split_hilo_kernel<<<blocks, 256, 0, s>>>(X, count, Xh, Xl);
    LRA_LAUNCHED();
}

int tc_rows_per_cta(int PP, bool pair) { return (!pair && PP >= 64) ? 2 * kBM : kBM; }

void xtw_tc(cudaStream_t s, const void *X, const void *Xl, int64_t dpad, int64_t n, const void *Wb, int PP,
            float *Y32, void *Yb, int64_t ldy, int *err, long long wait_cycles, bool f16, const float *tcs) {
    const long long lim = wait_cycles > 0 ? wait_cycles : kWaitCycles;
    const CUtensorMap mx = make_map(X, dpad, n, dpad, kBK, kBM, f16);
    const CUtensorMap mxl = make_map(Xl ? Xl : X, dpad, n, dpad, kBK, kBM, f16);
    const CUtensorMap mw = make_map(Wb, dpad, 2 * PP, dpad, kBK, PP, f16);
    const int nkb = (int)(dpad / kBK);
    const int rows = tc_rows_per_cta(PP, Xl != nullptr);
    uint16_t *yb = static_cast<uint16_t *>(Yb);
    dispatch_tc_pp(PP, [&](auto ppc) {
        constexpr int P = decltype(ppc)::value;
        const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(n, rows), sm_count());
        auto launch = [&](auto kern, int smem) {
            ensure_smem(kern, (int)smem);
            kern<<<grid, kThreads, smem, s>>>(mx, mxl, mw, nkb, n, Y32, yb, ldy, err, lim, tcs);
            LRA_LAUNCHED();
        };
        if (Xl)
            launch(xtw_tc_kernel<P, 2, 1, 1>, Tile<P, 2, 1>::kSmem);
        else if (f16)
            rows == kBM ? launch(xtw_tc_kernel<P, 1, 1, 0>, Tile<P, 1, 1>::kSmem)
                        : launch(xtw_tc_kernel<P, 1, 2, 0>, Tile<P, 1, 2>::kSmem);
        else if (rows == kBM)
            launch(xtw_tc_kernel<P, 1, 1, 1>, Tile<P, 1, 1>::kSmem);
        else
            launch(xtw_tc_kernel<P, 1, 2, 1>, Tile<P, 1, 2>::kSmem);
    });
}

void xy_tc(cudaStream_t s, const void *X, const void *Xl, int64_t dpad, int64_t n, const void *Yb, int64_t ldy,
           int PP, float *Gp, int nchunks, int *err, long long wait_cycles, bool f16) {
    const long long lim = wait_cycles > 0 ? wait_cycles : kWaitCycles;
    const CUtensorMap mx = make_map(X, dpad, n, dpad, 64, kBK, f16);
    const CUtensorMap mxl = make_map(Xl ? Xl : X, dpad, n, dpad, 64, kBK, f16);
    const CUtensorMap my = make_map(Yb, n, 2 * PP, ldy, kBK, PP, f16);
    const int64_t cpc = round_up(ceil_div(n, nchunks), kBK);
    const int rows = tc_rows_per_cta(PP, Xl != nullptr);
    dispatch_tc_pp(PP, [&](auto ppc) {
        constexpr int P = decltype(ppc)::value;
        const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(dpad, rows) * nchunks, sm_count());
        auto launch = [&](auto kern, int smem) {
            ensure_smem(kern, (int)smem);
            kern<<<grid, kThreads, smem, s>>>(mx, mxl, my, cpc, nchunks, n, dpad, Gp, err, lim);
            LRA_LAUNCHED();
        };
        if (Xl)
            launch(xy_tc_kernel<P, 2, 1, 1>, Tile<P, 2, 1>::kSmem);
        else if (f16)
            rows == kBM ? launch(xy_tc_kernel<P, 1, 1, 0>, Tile<P, 1, 1>::kSmem)
                        : launch(xy_tc_kernel<P, 1, 2, 0>, Tile<P, 1, 2>::kSmem);
        else if (rows == kBM)
            launch(xy_tc_kernel<P, 1, 1, 1>, Tile<P, 1, 1>::kSmem);
        else
            launch(xy_tc_kernel<P, 1, 2, 1>, Tile<P, 1, 2>::kSmem);
    });
}

}  // namespace lra
