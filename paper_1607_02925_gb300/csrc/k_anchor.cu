// Anchor pass of SVRGsolve (Sec. 2.3): M = lambda Wt - X (X^T Wt) - B, as two
// streaming passes over X (Y = X^T Wt, then G = X Y split over column chunks
// with a fixed-order reduction) and an epilogue.  CUDA-core FP32 FMA kernels,
// register-tiled, X staged through shared memory in 128-byte column segments.
#include <cuda_bf16.h>

#include <algorithm>

#include "kernels.cuh"

namespace lra {

namespace {

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    const int sz = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(sz));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

__device__ __forceinline__ float comp(const float4 &v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

// --- X^T W: tile of TI = 128 columns of X, K chunk of 32 rows ---------------
constexpr int kTI = 128;
constexpr int kKC = 32;
constexpr int kXS = kKC + 4;  // shared row stride (floats) of a staged column segment

template <typename TX>
struct XtwLoader {
    // FP32: 32 rows = 8 x 16B per column -> 1024 loads, 4 per thread.
    // BF16: 32 rows = 4 x 16B per column -> 512 loads, 2 per thread.
    static constexpr int V = 16 / sizeof(TX);     // elements per 16 B
    static constexpr int PER_COL = kKC / V;       // 16 B loads per column segment
    static constexpr int N = kTI * PER_COL / 256;  // loads per thread
    uint4 r[N];
    __device__ __forceinline__ void load(const TX *X, int64_t ldx, int64_t i0, int64_t n, int64_t k0) {
#pragma unroll
        for (int s = 0; s < N; ++s) {
            const int v = threadIdx.x + 256 * s;
            const int col = v / PER_COL, part = v % PER_COL;
            const int64_t i = i0 + col;
            if (i < n)
                r[s] = __ldg(reinterpret_cast<const uint4 *>(X + i * ldx + k0 + part * V));
            else
                r[s] = make_uint4(0, 0, 0, 0);
        }
    }
    __device__ __forceinline__ void store(float *xs) const {
#pragma unroll
        for (int s = 0; s < N; ++s) {
            const int v = threadIdx.x + 256 * s;
            const int col = v / PER_COL, part = v % PER_COL;
            float *dst = xs + col * kXS + part * V;
            if constexpr (V == 4) {
                *reinterpret_cast<uint4 *>(dst) = r[s];
            } else {
                const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&r[s]);
                float4 a = make_float4(__bfloat162float(e[0]), __bfloat162float(e[1]),
                                       __bfloat162float(e[2]), __bfloat162float(e[3]));
                float4 b = make_float4(__bfloat162float(e[4]), __bfloat162float(e[5]),
                                       __bfloat162float(e[6]), __bfloat162float(e[7]));
                *reinterpret_cast<float4 *>(dst) = a;
                *reinterpret_cast<float4 *>(dst + 4) = b;
            }
        }
    }
};

template <typename TX, int PP>
__global__ void __launch_bounds__(256) xtw_kernel(const TX *__restrict__ X, int64_t ldx, int64_t dpad,
                                                  int64_t n, const float *__restrict__ Wr,
                                                  float *__restrict__ Y) {
    constexpr int JG = PP / 4;
    extern __shared__ __align__(16) float smem[];
    float *Xs = smem;                    // [2][kTI][kXS]
    float *Ws = smem + 2 * kTI * kXS;    // [2][kKC][PP]
    const int tid = threadIdx.x;
    const int tj = tid >> 6;
    const int ti = tid & 63;
    const int64_t i0 = (int64_t)blockIdx.x * kTI;
    const int nchunks = (int)(dpad / kKC);

    float acc[2][JG];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int j = 0; j < JG; ++j) acc[a][j] = 0.0f;

    XtwLoader<TX> ld;
    auto load_w = [&](int c, int buf) {
        const float *src = Wr + (int64_t)c * kKC * PP;
        float *dst = Ws + buf * kKC * PP;
        for (int e = tid; e < kKC * PP / 4; e += 256) cp_async16(dst + 4 * e, src + 4 * e, true);
        cp_async_commit();
    };

    ld.load(X, ldx, i0, n, 0);
    load_w(0, 0);
    ld.store(Xs);
    cp_async_wait_all();
    __syncthreads();

    for (int c = 0; c < nchunks; ++c) {
        const int buf = c & 1;
        if (c + 1 < nchunks) {
            ld.load(X, ldx, i0, n, (int64_t)(c + 1) * kKC);
            load_w(c + 1, buf ^ 1);
        }
        const float *xs = Xs + buf * kTI * kXS;
        const float *ws = Ws + buf * kKC * PP + tj * JG;
#pragma unroll
        for (int k = 0; k < kKC; k += 4) {
            const float4 xa = *reinterpret_cast<const float4 *>(xs + ti * kXS + k);
            const float4 xb = *reinterpret_cast<const float4 *>(xs + (ti + 64) * kXS + k);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const float a = comp(xa, kk), b = comp(xb, kk);
                const float *wrow = ws + (k + kk) * PP;
#pragma unroll
                for (int j = 0; j < JG; j += 4) {
                    const float4 w = *reinterpret_cast<const float4 *>(wrow + j);
                    acc[0][j + 0] = fmaf(a, w.x, acc[0][j + 0]);
                    acc[0][j + 1] = fmaf(a, w.y, acc[0][j + 1]);
                    acc[0][j + 2] = fmaf(a, w.z, acc[0][j + 2]);
                    acc[0][j + 3] = fmaf(a, w.w, acc[0][j + 3]);
                    acc[1][j + 0] = fmaf(b, w.x, acc[1][j + 0]);
                    acc[1][j + 1] = fmaf(b, w.y, acc[1][j + 1]);
                    acc[1][j + 2] = fmaf(b, w.z, acc[1][j + 2]);
                    acc[1][j + 3] = fmaf(b, w.w, acc[1][j + 3]);
                }
            }
        }
        if (c + 1 < nchunks) {
            ld.store(Xs + (buf ^ 1) * kTI * kXS);
            cp_async_wait_all();
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const int64_t i = i0 + ti + 64 * a;
        if (i < n) {
            float *dst = Y + i * PP + tj * JG;
#pragma unroll
            for (int j = 0; j < JG; j += 4)
                *reinterpret_cast<float4 *>(dst + j) =
                    make_float4(acc[a][j], acc[a][j + 1], acc[a][j + 2], acc[a][j + 3]);
        }
    }
}

// --- X Y: tile of TR = 128 rows, K chunk of 32 columns ------------------------
constexpr int kTR = 128;
constexpr int kXS2 = kTR + 4;

template <typename TX>
struct XyLoader {
    // FP32: 128 rows = 32 x 16B per column -> 1024 loads, 4 per thread.
    // BF16: 128 rows = 16 x 16B per column -> 512 loads, 2 per thread.
    static constexpr int V = 16 / sizeof(TX);
    static constexpr int PER_COL = kTR / V;
    static constexpr int N = kKC * PER_COL / 256;
    uint4 r[N];
    __device__ __forceinline__ void load(const TX *X, int64_t ldx, int64_t r0, int64_t c0, int64_t c1) {
#pragma unroll
        for (int s = 0; s < N; ++s) {
            const int v = threadIdx.x + 256 * s;
            const int col = v / PER_COL, part = v % PER_COL;
            const int64_t i = c0 + col;
            if (i < c1)
                r[s] = __ldg(reinterpret_cast<const uint4 *>(X + i * ldx + r0 + part * V));
            else
                r[s] = make_uint4(0, 0, 0, 0);
        }
    }
    __device__ __forceinline__ void store(float *xs) const {
#pragma unroll
        for (int s = 0; s < N; ++s) {
            const int v = threadIdx.x + 256 * s;
            const int col = v / PER_COL, part = v % PER_COL;
            float *dst = xs + col * kXS2 + part * V;
            if constexpr (V == 4) {
                *reinterpret_cast<uint4 *>(dst) = r[s];
            } else {
                const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&r[s]);
                float4 a = make_float4(__bfloat162float(e[0]), __bfloat162float(e[1]),
                                       __bfloat162float(e[2]), __bfloat162float(e[3]));
                float4 b = make_float4(__bfloat162float(e[4]), __bfloat162float(e[5]),
                                       __bfloat162float(e[6]), __bfloat162float(e[7]));
                *reinterpret_cast<float4 *>(dst) = a;
                *reinterpret_cast<float4 *>(dst + 4) = b;
            }
        }
    }
};

template <typename TX, int PP>
__global__ void __launch_bounds__(256) xy_kernel(const TX *__restrict__ X, int64_t ldx, int64_t dpad,
                                                 int64_t n, const float *__restrict__ Y,
                                                 float *__restrict__ Gp, int64_t cols_per_chunk) {
    constexpr int JG = PP / 4;
    extern __shared__ __align__(16) float smem[];
    float *Xs = smem;                   // [2][kKC][kXS2]
    float *Ys = smem + 2 * kKC * kXS2;  // [2][kKC][PP]
    const int tid = threadIdx.x;
    const int tj = tid >> 6;
    const int tr = tid & 63;
    const int64_t r0 = (int64_t)blockIdx.x * kTR;
    const int64_t c0 = (int64_t)blockIdx.y * cols_per_chunk;
    const int64_t c1 = (c0 + cols_per_chunk < n) ? c0 + cols_per_chunk : n;
    const int nsteps = (int)ceil_div(c1 - c0, kKC);

    float acc[2][JG];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int j = 0; j < JG; ++j) acc[a][j] = 0.0f;

    XyLoader<TX> ld;
    auto load_y = [&](int st, int buf) {
        const int64_t cs = c0 + (int64_t)st * kKC;
        float *dst = Ys + buf * kKC * PP;
        for (int e = tid; e < kKC * PP / 4; e += 256) {
            const int row = (4 * e) / PP;
            const bool valid = cs + row < c1;
            const float *src = valid ? (Y + (cs + row) * PP + (4 * e) % PP) : Y;
            cp_async16(dst + 4 * e, src, valid);
        }
        cp_async_commit();
    };

    if (nsteps > 0) {
        ld.load(X, ldx, r0, c0, c1);
        load_y(0, 0);
        ld.store(Xs);
        cp_async_wait_all();
    }
    __syncthreads();

    for (int st = 0; st < nsteps; ++st) {
        const int buf = st & 1;
        if (st + 1 < nsteps) {
            ld.load(X, ldx, r0, c0 + (int64_t)(st + 1) * kKC, c1);
            load_y(st + 1, buf ^ 1);
        }
        const float *xs = Xs + buf * kKC * kXS2;
        const float *ys = Ys + buf * kKC * PP + tj * JG;
#pragma unroll 4
        for (int ii = 0; ii < kKC; ++ii) {
            const float a = xs[ii * kXS2 + tr];
            const float b = xs[ii * kXS2 + tr + 64];
            const float *yrow = ys + ii * PP;
#pragma unroll
            for (int j = 0; j < JG; j += 4) {
                const float4 w = *reinterpret_cast<const float4 *>(yrow + j);
                acc[0][j + 0] = fmaf(a, w.x, acc[0][j + 0]);
                acc[0][j + 1] = fmaf(a, w.y, acc[0][j + 1]);
                acc[0][j + 2] = fmaf(a, w.z, acc[0][j + 2]);
                acc[0][j + 3] = fmaf(a, w.w, acc[0][j + 3]);
                acc[1][j + 0] = fmaf(b, w.x, acc[1][j + 0]);
                acc[1][j + 1] = fmaf(b, w.y, acc[1][j + 1]);
                acc[1][j + 2] = fmaf(b, w.z, acc[1][j + 2]);
                acc[1][j + 3] = fmaf(b, w.w, acc[1][j + 3]);
            }
        }
        if (st + 1 < nsteps) {
            ld.store(Xs + (buf ^ 1) * kKC * kXS2);
            cp_async_wait_all();
        }
        __syncthreads();
    }
    float *out = Gp + (int64_t)blockIdx.y * dpad * PP;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const int64_t r = r0 + tr + 64 * a;
        float *dst = out + r * PP + tj * JG;
#pragma unroll
        for (int j = 0; j < JG; j += 4)
            *reinterpret_cast<float4 *>(dst + j) =
                make_float4(acc[a][j], acc[a][j + 1], acc[a][j + 2], acc[a][j + 3]);
    }
}

// --- epilogue: M = lambda Wt - sum_c Gp[c] - B (or G only) -------------------
// CTA = 16 rows x PP; four independent chunk accumulators per element, combined
// in a fixed order (deterministic).  With Z (a subproblem of the accelerated
// solve, lambda = lambda_0 + gamma): M = lambda Wt - G - (B + gamma Z), and the
// original residual r = lambda_0 Wt - G - B is summed as a third norm; both
// are formed in FP64 from the FP32 inputs, so neither B + gamma Z nor the
// cancellation M - gamma (Wt - Z) is rounded.  With Z (a subproblem of the accelerated
// solve, lambda = lambda_0 + gamma): M = lambda Wt - G - (B + gamma Z), and the
// original residual r = lambda_0 Wt - G - B is summed as a third norm; both
// are formed in FP64 from the FP32 inputs, so neither B + gamma Z nor the
// cancellation M - gamma (Wt - Z) is rounded.
constexpr int kER = 16;

__global__ void __launch_bounds__(256) epilogue_kernel(const float *__restrict__ Gp, int nchunks,
                                                       int64_t dpad, int PP, int p, double lam,
                                                       const float *__restrict__ Wt,
                                                       const float *__restrict__ B,
                                                       const float *__restrict__ Z, double gamma,
                                                       float *__restrict__ out, int mode,
                                                       double *__restrict__ partial,
                                                       const float *__restrict__ colscale) {
    extern __shared__ __align__(16) float tile[];  // [kER][PP + 1]
    __shared__ double red[3][8];
    const int tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * kER;
    const int ts = PP + 1;
    const int64_t stride = dpad * PP;
    for (int e = tid; e < kER * PP; e += 256) {
        const int64_t off = r0 * PP + e;
        float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
        int c = 0;
        for (; c + 3 < nchunks; c += 4) {
            a0 += Gp[(c + 0) * stride + off];
            a1 += Gp[(c + 1) * stride + off];
            a2 += Gp[(c + 2) * stride + off];
            a3 += Gp[(c + 3) * stride + off];
        }
        for (; c < nchunks; ++c) a0 += Gp[c * stride + off];
        float g = (a0 + a1) + (a2 + a3);
        if (colscale) g *= colscale[e % PP];  // a power of two: exact
        tile[(e / PP) * ts + (e % PP)] = g;
    }
    __syncthreads();
    double m2 = 0.0, b2 = 0.0, r2 = 0.0;
    for (int e = tid; e < kER * p; e += 256) {
        const int r = e % kER, j = e / kER;
        const int64_t gi = (r0 + r) + (int64_t)j * dpad;
        const float g = tile[r * ts + j];
        if (mode == 0) {
            const float b = B[gi];
            if (Z) {
                const double w = Wt[gi], z = Z[gi];
                const double rr = (lam - gamma) * w - (double)g - (double)b;
                const float m = (float)(rr + gamma * (w - z));
                const double bb = (double)b + gamma * z;
                out[gi] = m;
                m2 += (double)m * (double)m;
                b2 += bb * bb;
                r2 += rr * rr;
            } else {
                const float m = (float)((double)lam * (double)Wt[gi] - (double)g - (double)b);
                out[gi] = m;
                m2 += (double)m * (double)m;
                b2 += (double)b * (double)b;
            }
        } else {
            out[gi] = g;
        }
    }
    if (mode == 0) {
        const int ns = Z ? 3 : 2;
        m2 = warp_sum(m2);
        b2 = warp_sum(b2);
        r2 = warp_sum(r2);
        if ((tid & 31) == 0) {
            red[0][tid >> 5] = m2;
            red[1][tid >> 5] = b2;
            red[2][tid >> 5] = r2;
        }
        __syncthreads();
        if (tid == 0) {
            double a[3] = {0.0, 0.0, 0.0};
            for (int w = 0; w < 8; ++w)
                for (int q = 0; q < ns; ++q) a[q] += red[q][w];
            for (int q = 0; q < ns; ++q) partial[ns * blockIdx.x + q] = a[q];
        }
    }
}

// one warp: strided partial sums, then a fixed shuffle tree (deterministic)
__global__ void norms_final_kernel(const double *__restrict__ partial, int nb, int ns,
                                   double *__restrict__ norms) {
    double a[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nb; b += 32)
        for (int q = 0; q < ns; ++q) a[q] += partial[ns * b + q];
    for (int q = 0; q < 3; ++q) a[q] = warp_sum(a[q]);
    if (threadIdx.x == 0)
        for (int q = 0; q < ns; ++q) norms[q] = a[q];
}

__global__ void pack_rm_kernel(const float *__restrict__ W, int64_t ldw, int64_t rows, int p, int PP,
                               float *__restrict__ Wr) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * PP) return;
    const int64_t r = e / PP;
    const int j = (int)(e % PP);
    Wr[e] = j < p ? W[r + (int64_t)j * ldw] : 0.0f;
}

template <typename F>
void dispatch_pp(int PP, F &&f) {
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

void pack_rm(cudaStream_t s, const float *W, int64_t ldw, int64_t rows, int p, int PP, float *Wr) {
    const int64_t total = rows * PP;
    pack_rm_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, s>>>(W, ldw, rows, p, PP, Wr);
    LRA_LAUNCHED();
}

void xtw(cudaStream_t s, const void *X, lra_dtype dt, int64_t ldx, int64_t dpad, int64_t n,
         const float *Wr, int PP, float *Y) {
    dispatch_pp(PP, [&](auto ppc) {
        constexpr int P = decltype(ppc)::value;
        const size_t smem = sizeof(float) * (2 * kTI * kXS + 2 * kKC * P);
        const dim3 grid((unsigned)ceil_div(n, kTI));
        if (dt == LRA_BF16) {
            auto k = xtw_kernel<__nv_bfloat16, P>;
            ensure_smem(k, (int)smem);
            k<<<grid, 256, smem, s>>>((const __nv_bfloat16 *)X, ldx, dpad, n, Wr, Y);
        } else {
            auto k = xtw_kernel<float, P>;
            ensure_smem(k, (int)smem);
            k<<<grid, 256, smem, s>>>((const float *)X, ldx, dpad, n, Wr, Y);
        }
        LRA_LAUNCHED();
    });
}

// Split of the n columns for the X Y passes: the grid is (row tiles) x
// chunks with one resident CTA per SM, so the chunk count is chosen to fill
// whole waves of 152 SMs: the smallest count giving at least two waves at >= 97%
// occupancy of the last one, else the best-filled count up to 64 chunks.
int xy_chunks(int64_t dpad, int64_t n, int rows_per_cta) {
    const int64_t row_tiles = ceil_div(dpad, rows_per_cta);
    const int64_t maxc = std::max<int64_t>(1, std::min<int64_t>(64, ceil_div(n, 4 * kKC)));
    int64_t best = 1;
    double best_eff = -1.0;
    for (int64_t c = 1; c <= maxc; ++c) {
        const int64_t units = row_tiles * c;
        const int64_t waves = ceil_div(units, 152);
        const double eff = (double)units / (double)(waves * 152);
        if (units >= 2 * 152 && eff >= 0.97) return (int)c;
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = c;
        }
    }
    return (int)best;
}

void xy(cudaStream_t s, const void *X, lra_dtype dt, int64_t ldx, int64_t dpad, int64_t n,
        const float *Y, int PP, float *Gp, int nchunks) {
    const int64_t cpc = round_up(ceil_div(n, nchunks), kKC);
    dispatch_pp(PP, [&](auto ppc) {
        constexpr int P = decltype(ppc)::value;
        const size_t smem = sizeof(float) * (2 * kKC * kXS2 + 2 * kKC * P);
        const dim3 grid((unsigned)(dpad / kTR), (unsigned)nchunks);
        if (dt == LRA_BF16) {
            auto k = xy_kernel<__nv_bfloat16, P>;
            ensure_smem(k, (int)smem);
            k<<<grid, 256, smem, s>>>((const __nv_bfloat16 *)X, ldx, dpad, n, Y, Gp, cpc);
        } else {
            auto k = xy_kernel<float, P>;
            ensure_smem(k, (int)smem);
            k<<<grid, 256, smem, s>>>((const float *)X, ldx, dpad, n, Y, Gp, cpc);
        }
        LRA_LAUNCHED();
    });
}

void anchor_epilogue(cudaStream_t s, const float *Gp, int nchunks, int64_t dpad, int PP, int p,
                     double lam, const float *Wt, const float *B, float *M, double *norms,
                     double *scratch, const float *Z, double gamma, const float *colscale) {
    const int nb = (int)(dpad / kER);
    const size_t smem = sizeof(float) * kER * (PP + 1);
    const int mode = (Wt != nullptr) ? 0 : 1;
    epilogue_kernel<<<nb, 256, smem, s>>>(Gp, nchunks, dpad, PP, p, lam, Wt, B, Z, gamma, M, mode, scratch,
                                          colscale);
    LRA_LAUNCHED();
    if (mode == 0 && norms) {
        norms_final_kernel<<<1, 32, 0, s>>>(scratch, nb, Z ? 3 : 2, norms);
        LRA_LAUNCHED();
    }
}

}  // namespace lra
