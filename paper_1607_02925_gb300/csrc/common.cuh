// Shared definitions of the CUDA path: error plumbing, launch accounting,
// counter-based random numbers (SplitMix64), and warp helpers.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "lra.h"

namespace lra {

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);

struct Error {
    lra_status st;
};

#define LRA_CUDA(call)                                                                   \
    do {                                                                                 \
        cudaError_t e__ = (call);                                                        \
        if (e__ != cudaSuccess) {                                                        \
            ::lra::set_error(std::string(#call) + ": " + cudaGetErrorString(e__) + " @" + \
                             __FILE__ + ":" + std::to_string(__LINE__));                  \
            throw ::lra::Error{LRA_ECUDA};                                               \
        }                                                                                \
    } while (0)

#define LRA_LAUNCHED()                                                                   \
    do {                                                                                 \
        ::lra::count_launch();                                                           \
        cudaError_t e__ = cudaGetLastError();                                            \
        if (e__ != cudaSuccess) {                                                        \
            ::lra::set_error(std::string("kernel launch: ") + cudaGetErrorString(e__) +  \
                             " @" + __FILE__ + ":" + std::to_string(__LINE__));           \
            throw ::lra::Error{LRA_ECUDA};                                               \
        }                                                                                \
    } while (0)

// Kernel launches of the calling thread (reported per lra_solve).
void count_launch();
int64_t launches_of_thread();

// Raise a kernel's dynamic shared-memory limit to at least `bytes`.  The
// attribute is per function and shared by all threads, so it is only ever
// raised: a concurrent launch needing less is still covered.
void ensure_smem(const void *kernel, int bytes);
template <typename K>
inline void ensure_smem(K *kernel, int bytes) {
    ensure_smem(reinterpret_cast<const void *>(kernel), bytes);
}

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea, Flood 2014): state += gamma; out = mix64(state).
// The t-th word of the stream with key K is mix64(K + gamma (t + 1)).
// ---------------------------------------------------------------------------
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t stream_key(uint64_t seed, uint64_t stream, uint64_t a,
                                                        uint64_t b) {
    uint64_t h = mix64(seed + kGamma * (stream + 1));
    h = mix64(h + kGamma * (a + 1));
    h = mix64(h + kGamma * (b + 1));
    return h;
}

__host__ __device__ __forceinline__ uint64_t stream_word(uint64_t key, uint64_t t) {
    return mix64(key + kGamma * (t + 1));
}

// ---------------------------------------------------------------------------
// Element conversion
// ---------------------------------------------------------------------------
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f32(__half v) { return __half2float(v); }

// Four consecutive elements (16-byte aligned for float, 8-byte for the 16-bit
// types) widened to FP32.
template <typename TX>
__device__ __forceinline__ void load4_f32(const TX *p, float (&x)[4]) {
    if constexpr (sizeof(TX) == 4) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        x[0] = q.x; x[1] = q.y; x[2] = q.z; x[3] = q.w;
    } else {
        const uint2 q = *reinterpret_cast<const uint2 *>(p);
        const TX *e = reinterpret_cast<const TX *>(&q);
#pragma unroll
        for (int v = 0; v < 4; ++v) x[v] = to_f32(e[v]);
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__host__ __device__ __forceinline__ int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// Row padding of every d-long vector the library stores (X columns, d x p
// blocks): rows d..dpad-1 hold zeros, so tiles need no row bounds checks.
constexpr int kRowPad = 128;

// Column padding of packed row-major d x PP / n x PP blocks.
inline int pad_p(int p) {
    if (p <= 16) return 16;
    return (int)round_up(p, 16);
}

}  // namespace lra
