// Setup kernels: column norms and ||X||_F^2, the integer sampling distribution
// q_i ~ ||x_i||^2 with its prefix sums, the sampler, the Gaussian start block,
// and storage conversions.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "kernels.cuh"

namespace lra {

// ---------------------------------------------------------------------------
// ||x_i||^2, FP64 accumulation (x^2 of an FP32 value is exact in FP64).
// One warp per column; columns are contiguous (ldx = dpad, multiple of 128).
// ---------------------------------------------------------------------------
template <typename TX>
__global__ void __launch_bounds__(256) colnorms_kernel(const TX *__restrict__ X, int64_t ldx,
                                                       int64_t rows, int64_t n, double inv2,
                                                       double *__restrict__ norm2) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (i >= n) return;
    const TX *col = X + i * ldx;
    double acc = 0.0;
    constexpr int V = 16 / sizeof(TX);  // elements per 16-byte load
    for (int64_t r = (int64_t)lane * V; r < rows; r += 32 * V) {
        const uint4 raw = *reinterpret_cast<const uint4 *>(col + r);
        const TX *e = reinterpret_cast<const TX *>(&raw);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const double x = (double)to_f32(e[v]);
            acc = fma(x, x, acc);
        }
    }
    acc = warp_sum(acc);
    if (lane == 0) norm2[i] = acc * inv2;
}

void colnorms(cudaStream_t s, const void *X, lra_dtype dt, int64_t ldx, int64_t d, int64_t n,
              double *norm2, double xscale) {
    (void)d;
    const int64_t rows = ldx;  // padding rows are zero
    dim3 grid((unsigned)ceil_div(n, 8));
    const double inv2 = 1.0 / (xscale * xscale);  // a power of two: exact
    if (dt == LRA_BF16)
        colnorms_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>((const __nv_bfloat16 *)X, ldx, rows, n, inv2, norm2);
    else if (dt == LRA_F16)
        colnorms_kernel<__half><<<grid, 256, 0, s>>>((const __half *)X, ldx, rows, n, inv2, norm2);
    else
        colnorms_kernel<float><<<grid, 256, 0, s>>>((const float *)X, ldx, rows, n, inv2, norm2);
    LRA_LAUNCHED();
}

// ---------------------------------------------------------------------------
// FP16 storage: max |x| over the FP32 copy (non-negative floats compare as
// their bit patterns, so an atomicMax on the bits is exact and order-free),
// then fp16(xscale x) with xscale = 2^(14 - floor(log2 max)).
// ---------------------------------------------------------------------------
__global__ void maxabs_kernel(const float *__restrict__ X, int64_t count, unsigned *__restrict__ out) {
    float mx = 0.0f;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        mx = fmaxf(mx, fabsf(X[e]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(mx));
}

__global__ void to_f16_kernel(const float *__restrict__ X, int64_t count, float xscale, __half *__restrict__ Xs) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        Xs[e] = __float2half_rn(X[e] * xscale);
}

float f16_storage_scale(cudaStream_t s, const float *X32, int64_t count, unsigned *scratch) {
    LRA_CUDA(cudaMemsetAsync(scratch, 0, sizeof(unsigned), s));
    const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(count, 256), 152 * 16);
    maxabs_kernel<<<blocks, 256, 0, s>>>(X32, count, scratch);
    LRA_LAUNCHED();
    unsigned bits = 0;
    LRA_CUDA(cudaMemcpyAsync(&bits, scratch, sizeof(bits), cudaMemcpyDeviceToHost, s));
    LRA_CUDA(cudaStreamSynchronize(s));
    float mx;
    std::memcpy(&mx, &bits, sizeof(mx));
    if (!(mx > 0.0f) || !std::isfinite(mx)) return 1.0f;
    int e = 0;
    std::frexp(mx, &e);  // mx in [2^(e-1), 2^e)
    return std::ldexp(1.0f, 15 - e);
}

void to_f16(cudaStream_t s, const float *X32, int64_t count, float xscale, __half *Xs) {
    const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(count, 256), 152 * 64);
    to_f16_kernel<<<blocks, 256, 0, s>>>(X32, count, xscale, Xs);
    LRA_LAUNCHED();
}

// ---------------------------------------------------------------------------
// Fixed-order sum and max of n doubles in one block (deterministic).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) sum_max_kernel(const double *__restrict__ v, int64_t n,
                                                       double *__restrict__ out) {
    __shared__ double ss[1024], sm[1024];
    double acc = 0.0, mx = -INFINITY;
    for (int64_t i = threadIdx.x; i < n; i += 1024) {
        const double x = v[i];
        acc += x;
        mx = fmax(mx, x);
    }
    ss[threadIdx.x] = acc;
    sm[threadIdx.x] = mx;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            ss[threadIdx.x] += ss[threadIdx.x + w];
            sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = ss[0];
        out[1] = sm[0];
    }
}

void sum_max(cudaStream_t s, const double *v, int64_t n, double *out, double *scratch) {
    (void)scratch;
    sum_max_kernel<<<1, 1024, 0, s>>>(v, n, out);
    LRA_LAUNCHED();
}

// ---------------------------------------------------------------------------
// Sampling distribution.  w_i = max(1, floor(norm2_i * (2^32 / max))) for
// norm2_i > 0, else 0 (uniform: 1).  Inclusive scan in uint64 (exact).
// ---------------------------------------------------------------------------
__global__ void weights_kernel(const double *__restrict__ norm2, int64_t n, int mode,
                               const double *__restrict__ maxn, uint64_t *__restrict__ w) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (mode == LRA_SAMPLE_UNIFORM) {
        w[i] = 1ull;
        return;
    }
    const double mx = *maxn;
    const double v = norm2[i];
    uint64_t wi = 0;
    // a non-finite norm (or maximum) gets no weight; the callers reject such
    // input from the FP64 sum of the norms
    if (v > 0.0 && mx > 0.0 && isfinite(v) && isfinite(mx)) {
        const double scale = __ddiv_rn(4294967296.0, mx);
        const double f = floor(__dmul_rn(v, scale));
        wi = (uint64_t)f;
        if (wi == 0) wi = 1;
    }
    w[i] = wi;
}

// Tile scan: 256 threads x 4 elements; writes inclusive prefix within the tile
// and the tile total.
__global__ void __launch_bounds__(256) scan_tiles_kernel(uint64_t *__restrict__ a, int64_t n,
                                                         uint64_t *__restrict__ tile_sums) {
    __shared__ uint64_t warp_tot[8];
    const int64_t base = (int64_t)blockIdx.x * 1024 + threadIdx.x * 4;
    uint64_t v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = (base + j < n) ? a[base + j] : 0ull;
    v[1] += v[0];
    v[2] += v[1];
    v[3] += v[2];
    uint64_t t = v[3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
    }
    if (lane == 31) warp_tot[warp] = t;
    __syncthreads();
    uint64_t off = 0;
    for (int w2 = 0; w2 < warp; ++w2) off += warp_tot[w2];
    const uint64_t excl = off + t - v[3];
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (base + j < n) a[base + j] = v[j] + excl;
    if (threadIdx.x == 255) tile_sums[blockIdx.x] = off + t;
}

// Exclusive scan of the tile totals in one block (sequential chunks of 1024).
__global__ void __launch_bounds__(1024) scan_sums_kernel(uint64_t *__restrict__ sums, int64_t nt) {
    __shared__ uint64_t buf[1024];
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < nt; b += 1024) {
        const int64_t i = b + threadIdx.x;
        const uint64_t x = i < nt ? sums[i] : 0ull;
        buf[threadIdx.x] = x;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            uint64_t y = (int)threadIdx.x >= o ? buf[threadIdx.x - o] : 0ull;
            __syncthreads();
            buf[threadIdx.x] += y;
            __syncthreads();
        }
        const uint64_t incl = buf[threadIdx.x];
        const uint64_t c0 = carry;
        if (i < nt) sums[i] = c0 + incl - x;
        __syncthreads();
        if (threadIdx.x == 1023) carry = c0 + incl;
        __syncthreads();
    }
}

__global__ void add_offsets_kernel(uint64_t *__restrict__ a, int64_t n,
                                   const uint64_t *__restrict__ offs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] += offs[i >> 10];
}

// c_i = total / w_i (FP32 of the FP64 quotient), block maxima of
// (total / w_i) norm2_i.
__global__ void __launch_bounds__(256) cvec_kernel(const uint64_t *__restrict__ cum, int64_t n,
                                                   const double *__restrict__ norm2,
                                                   float *__restrict__ c,
                                                   double *__restrict__ blockmax) {
    __shared__ double sm[256];
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const double total = (double)cum[n - 1];
    double k = 0.0;
    if (i < n) {
        const uint64_t w = cum[i] - (i > 0 ? cum[i - 1] : 0ull);
        float ci = 0.0f;
        if (w > 0) {
            const double q = __ddiv_rn(total, (double)w);
            ci = (float)q;
            k = __dmul_rn(q, norm2[i]);
        }
        c[i] = ci;
    }
    sm[threadIdx.x] = k;
    __syncthreads();
    for (int w2 = 128; w2 > 0; w2 >>= 1) {
        if ((int)threadIdx.x < w2) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + w2]);
        __syncthreads();
    }
    if (threadIdx.x == 0) blockmax[blockIdx.x] = sm[0];
}

__global__ void __launch_bounds__(1024) max_kernel(const double *__restrict__ v, int64_t n,
                                                   double *__restrict__ out) {
    __shared__ double sm[1024];
    double mx = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 1024) mx = fmax(mx, v[i]);
    sm[threadIdx.x] = mx;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sm[0];
}

void sampling_table(cudaStream_t s, const double *norm2, int64_t n, int mode, const double *maxn,
                    uint64_t *cum, float *c, double *kappa_out, uint64_t *scratch) {
    const int64_t nb256 = ceil_div(n, 256);
    weights_kernel<<<(unsigned)nb256, 256, 0, s>>>(norm2, n, mode, maxn, cum);
    LRA_LAUNCHED();
    const int64_t nt = ceil_div(n, 1024);
    scan_tiles_kernel<<<(unsigned)nt, 256, 0, s>>>(cum, n, scratch);
    LRA_LAUNCHED();
    scan_sums_kernel<<<1, 1024, 0, s>>>(scratch, nt);
    LRA_LAUNCHED();
    add_offsets_kernel<<<(unsigned)nb256, 256, 0, s>>>(cum, n, scratch);
    LRA_LAUNCHED();
    double *bm = reinterpret_cast<double *>(scratch);  // reuse: nb256 doubles
    cvec_kernel<<<(unsigned)nb256, 256, 0, s>>>(cum, n, norm2, c, bm);
    LRA_LAUNCHED();
    max_kernel<<<1, 1024, 0, s>>>(bm, nb256, kappa_out);
    LRA_LAUNCHED();
}

// ---------------------------------------------------------------------------
// Sampler: r_t = floor(u_t total / 2^64), idx_t = first i with cum[i] > r_t.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) sample_kernel(const uint64_t *__restrict__ cum, int64_t n,
                                                     uint64_t key, int64_t m,
                                                     int32_t *__restrict__ idx,
                                                     const float *__restrict__ c,
                                                     float *__restrict__ cval) {
    const int64_t t = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (t >= m) return;
    const uint64_t total = cum[n - 1];
    const uint64_t r = __umul64hi(stream_word(key, (uint64_t)t), total);
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (cum[mid] > r)
            hi = mid;
        else
            lo = mid + 1;
    }
    idx[t] = (int32_t)lo;
    if (cval) cval[t] = c[lo];
}

void sample(cudaStream_t s, const uint64_t *cum, int64_t n, uint64_t key, int64_t m, int32_t *idx,
            const float *c, float *cval) {
    if (m <= 0) return;
    sample_kernel<<<(unsigned)ceil_div(m, 256), 256, 0, s>>>(cum, n, key, m, idx, c, cval);
    LRA_LAUNCHED();
}

__global__ void gather_c_kernel(const int32_t *__restrict__ idx, const float *__restrict__ c, int64_t m,
                                int64_t n, float *__restrict__ cval, int *__restrict__ bad) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    const int32_t i = idx[t];
    if (i < 0 || i >= n) {
        *bad = 1;
        cval[t] = 0.0f;
    } else {
        cval[t] = c[i];
    }
}

void gather_c(cudaStream_t s, const int32_t *idx, const float *c, int64_t m, int64_t n, float *cval,
              int *bad) {
    LRA_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    if (m <= 0) return;
    gather_c_kernel<<<(unsigned)ceil_div(m, 256), 256, 0, s>>>(idx, c, m, n, cval, bad);
    LRA_LAUNCHED();
}

// ---------------------------------------------------------------------------
// Gaussian start block by Box-Muller on counter words (FP64, then FP32).
// ---------------------------------------------------------------------------
__global__ void gaussian_kernel(uint64_t key, int64_t d, int64_t dpad, int p, float *__restrict__ out) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t count = d * (int64_t)p;
    if (2 * q >= count) return;
    const uint64_t u1 = stream_word(key, 2 * (uint64_t)q);
    const uint64_t u2 = stream_word(key, 2 * (uint64_t)q + 1);
    const double U1 = ((double)(u1 >> 11) + 1.0) * 0x1.0p-53;
    const double U2 = (double)(u2 >> 11) * 0x1.0p-53;
    const double rad = sqrt(-2.0 * log(U1));
    double sn, cs;
    sincospi(2.0 * U2, &sn, &cs);
    const int64_t e0 = 2 * q, e1 = 2 * q + 1;
    out[(e0 % d) + (e0 / d) * dpad] = (float)(rad * cs);
    if (e1 < count) out[(e1 % d) + (e1 / d) * dpad] = (float)(rad * sn);
}

void gaussian(cudaStream_t s, uint64_t key, int64_t d, int64_t dpad, int p, float *out) {
    LRA_CUDA(cudaMemsetAsync(out, 0, sizeof(float) * dpad * p, s));
    const int64_t pairs = ceil_div(d * (int64_t)p, 2);
    gaussian_kernel<<<(unsigned)ceil_div(pairs, 256), 256, 0, s>>>(key, d, dpad, p, out);
    LRA_LAUNCHED();
}

// ---------------------------------------------------------------------------
// Storage conversions: column-major src (leading dim ld) -> dst (leading dim
// dpad), rows d..dpad-1 set to zero.  BF16 conversion rounds to nearest even.
// ---------------------------------------------------------------------------
template <typename TS>
__device__ __forceinline__ float load_f32(const TS *p) { return to_f32(*p); }
template <>
__device__ __forceinline__ float load_f32<double>(const double *p) { return __double2float_rn(*p); }

// Column-major conversion: CTA per column (grid-stride over columns), threads
// along the rows, no per-element division; rows d..dpad-1 are written as zeros.
// An FP32 source with 16-byte aligned columns (ld a multiple of 4) moves as float4.
template <typename TS, typename TD>
__global__ void __launch_bounds__(256) convert_kernel(const TS *__restrict__ src, int64_t ld, int64_t d,
                                                      int64_t ncols, TD *__restrict__ dst, int64_t dpad,
                                                      bool vec4) {
    for (int64_t col = blockIdx.x; col < ncols; col += gridDim.x) {
        const TS *sc = src + col * ld;
        TD *dc = dst + col * dpad;
        if constexpr (sizeof(TS) == 4 && sizeof(TD) == 4) {
            if (vec4) {
                const int64_t d4 = d >> 2;
                for (int64_t q = threadIdx.x; q < (dpad >> 2); q += blockDim.x) {
                    float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    if (q < d4) {
                        v = reinterpret_cast<const float4 *>(sc)[q];
                    } else if (4 * q < d) {
                        const int64_t r = 4 * q;
                        v.x = sc[r];
                        if (r + 1 < d) v.y = sc[r + 1];
                        if (r + 2 < d) v.z = sc[r + 2];
                    }
                    reinterpret_cast<float4 *>(dc)[q] = v;
                }
                continue;
            }
        }
        for (int64_t r = threadIdx.x; r < dpad; r += blockDim.x) {
            TD out;
            if constexpr (sizeof(TS) == 8 && sizeof(TD) == 2) {
                out = r < d ? __double2bfloat16(sc[r]) : __float2bfloat16_rn(0.0f);
            } else {
                const float v = r < d ? load_f32(sc + r) : 0.0f;
                if constexpr (sizeof(TD) == 2)
                    out = __float2bfloat16_rn(v);
                else
                    out = v;
            }
            dc[r] = out;
        }
    }
}

template <typename TD>
static void convert_dispatch(cudaStream_t s, const void *src, lra_dtype sdt, int64_t ld, int64_t d,
                             int64_t ncols, TD *dst, int64_t dpad) {
    if (ncols <= 0) return;
    const unsigned blocks = (unsigned)std::min<int64_t>(ncols, 152 * 16);
    const bool vec4 = sdt == LRA_F32 && (ld % 4) == 0 && (reinterpret_cast<uintptr_t>(src) % 16) == 0;
    switch (sdt) {
        case LRA_F32:
            convert_kernel<float, TD><<<blocks, 256, 0, s>>>((const float *)src, ld, d, ncols, dst, dpad, vec4);
            break;
        case LRA_BF16:
            convert_kernel<__nv_bfloat16, TD><<<blocks, 256, 0, s>>>((const __nv_bfloat16 *)src, ld, d,
                                                                    ncols, dst, dpad, false);
            break;
        case LRA_F64:
            convert_kernel<double, TD><<<blocks, 256, 0, s>>>((const double *)src, ld, d, ncols, dst, dpad, false);
            break;
        default:
            set_error("unsupported source dtype");
            throw Error{LRA_EUNSUPPORTED};
    }
    LRA_LAUNCHED();
}

void convert_to_f32(cudaStream_t s, const void *src, lra_dtype sdt, int64_t ld, int64_t d,
                    int64_t ncols, float *dst, int64_t dpad) {
    convert_dispatch<float>(s, src, sdt, ld, d, ncols, dst, dpad);
}

void convert_to_bf16(cudaStream_t s, const void *src, lra_dtype sdt, int64_t ld, int64_t d,
                     int64_t ncols, __nv_bfloat16 *dst, int64_t dpad) {
    convert_dispatch<__nv_bfloat16>(s, src, sdt, ld, d, ncols, dst, dpad);
}

}  // namespace lra
