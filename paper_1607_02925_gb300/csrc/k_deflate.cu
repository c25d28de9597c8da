// Deflation applied on the fly (Algorithm 6, Sec. 3).  A stage that starts at
// index s works on X' = (I - U U^T) X, U the dpad x c orthonormal columns found
// by the earlier stages (c = s - 1).  X' is never formed: its products, column
// norms and sampled columns come from X and Gt = X^T U (n x PPc row-major, row
// i holding g_i = U^T x_i):
//   X'^T W = X^T (W - U (U^T W))          the small operand projected first;
//   X' Y   = (I - U U^T) (X Y)            the d x p product projected after;
//   ||x'_i||^2 = ||x_i||^2 - ||g_i||^2    (U orthonormal);
//   x'_i   = x_i - U g_i                  a sampled column of the inner loop.
#include <algorithm>

#include "kernels.cuh"

namespace lra {

namespace {

constexpr int kCoefA = 8;  // coefficients (rows of C) per CTA of defl_coef_kernel

// C[a ldc + j] = sum_r U[r + a ldu] V[r rs + j cs] for a in [a0, a0 + 8), one
// column j per CTA; FP32 products summed in FP64, rows in a fixed order.
__global__ void __launch_bounds__(256) defl_coef_kernel(const float *__restrict__ U, int64_t ldu, int c,
                                                        const float *__restrict__ V, int64_t rs, int64_t cs,
                                                        int64_t rows, float *__restrict__ C, int ldc) {
    __shared__ double red[kCoefA][8];
    const int j = blockIdx.y, a0 = blockIdx.x * kCoefA;
    const int na = min(kCoefA, c - a0);
    double acc[kCoefA];
#pragma unroll
    for (int q = 0; q < kCoefA; ++q) acc[q] = 0.0;
    for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) {
        const float v = V[r * rs + (int64_t)j * cs];
#pragma unroll
        for (int q = 0; q < kCoefA; ++q)
            if (q < na) acc[q] = fma((double)U[r + (int64_t)(a0 + q) * ldu], (double)v, acc[q]);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kCoefA; ++q) {
        const double t = warp_sum(acc[q]);
        if (lane == 0) red[q][w] = t;
    }
    __syncthreads();
    if (threadIdx.x < na) {
        double t = 0.0;
        for (int u = 0; u < (int)(blockDim.x >> 5); ++u) t += red[threadIdx.x][u];
        C[(int64_t)(a0 + threadIdx.x) * ldc + j] = (float)t;
    }
}

// V[r + j ldv] -= sum_a U[r + a ldu] C[a ldc + j] (V rows x p column-major)
__global__ void defl_sub_kernel(const float *__restrict__ U, int64_t ldu, int c, const float *__restrict__ C,
                                int ldc, float *__restrict__ V, int64_t ldv, int64_t rows, int p) {
    const int64_t total = rows * p;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / rows, r = e - j * rows;
        float acc = 0.0f;
        for (int a = 0; a < c; ++a) acc = fmaf(U[r + (int64_t)a * ldu], C[(int64_t)a * ldc + j], acc);
        V[r + j * ldv] -= acc;
    }
}

__global__ void defl_norms_kernel(const double *__restrict__ norm2, const float *__restrict__ Gt, int PPc, int c,
                                  int64_t n, double *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double g2 = 0.0;
        for (int a = 0; a < c; ++a) {
            const double g = Gt[i * PPc + a];
            g2 = fma(g, g, g2);
        }
        out[i] = fmax(0.0, norm2[i] - g2);
    }
}

// out[:, t] = x_{idx[t]} - U g_{idx[t]} for t < m (FP32, dpad x m column-major):
// CTA (row block of 256, column block of kGatherT) with the block's g vectors
// in shared memory, so that each row of U is read once per kGatherT columns.
constexpr int kGatherT = 16;

__global__ void __launch_bounds__(256) defl_gather_kernel(const float *__restrict__ X, int64_t ldx, int64_t dpad,
                                                          const int32_t *__restrict__ idx, int64_t m,
                                                          const float *__restrict__ U, int c,
                                                          const float *__restrict__ Gt, int PPc,
                                                          float *__restrict__ out) {
    extern __shared__ float gs[];  // [kGatherT][c]
    const int64_t t0 = (int64_t)blockIdx.y * kGatherT;
    const int nt = m - t0 < kGatherT ? (int)(m - t0) : kGatherT;
    for (int e = threadIdx.x; e < kGatherT * c; e += blockDim.x) {
        const int tt = e / c, a = e - tt * c;
        gs[e] = tt < nt ? Gt[(int64_t)idx[t0 + tt] * PPc + a] : 0.0f;
    }
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= dpad) return;
    float acc[kGatherT];
#pragma unroll
    for (int tt = 0; tt < kGatherT; ++tt) acc[tt] = (X && tt < nt) ? X[r + (int64_t)idx[t0 + tt] * ldx] : 0.0f;
    for (int a = 0; a < c; ++a) {
        const float u = U[r + (int64_t)a * dpad];
#pragma unroll
        for (int tt = 0; tt < kGatherT; ++tt) acc[tt] = fmaf(-u, gs[tt * c + a], acc[tt]);
    }
#pragma unroll
    for (int tt = 0; tt < kGatherT; ++tt)
        if (tt < nt) out[r + (t0 + tt) * dpad] = acc[tt];
}

// out[rowidx[e] + t dpad] += cval[e] over the entries e of compressed column
// idx[t] (rows are distinct within a column): warp per sampled column
__global__ void defl_scatter_csc_kernel(const int64_t *__restrict__ colptr, const int32_t *__restrict__ rowidx,
                                        const float *__restrict__ cval, const int32_t *__restrict__ idx, int64_t m,
                                        int64_t dpad, float *__restrict__ out) {
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= m) return;
    const int64_t i = idx[t];
    for (int64_t e = colptr[i] + (threadIdx.x & 31); e < colptr[i + 1]; e += 32) out[rowidx[e] + t * dpad] += cval[e];
}

unsigned grid_of(int64_t items) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(items, 256), 152 * 8));
}

}  // namespace

void defl_coef(cudaStream_t s, const float *U, int64_t ldu, int c, const float *V, int64_t rs, int64_t cs,
               int64_t rows, int p, float *C, int ldc) {
    if (c <= 0 || p <= 0) return;
    const dim3 grid((unsigned)ceil_div(c, kCoefA), (unsigned)p);
    defl_coef_kernel<<<grid, 256, 0, s>>>(U, ldu, c, V, rs, cs, rows, C, ldc);
    LRA_LAUNCHED();
}

void defl_project(cudaStream_t s, const float *U, int64_t ldu, int c, float *V, int64_t ldv, int64_t rows, int p,
                  float *C) {
    if (c <= 0 || p <= 0) return;
    defl_coef(s, U, ldu, c, V, 1, ldv, rows, p, C, p);
    defl_sub_kernel<<<grid_of(rows * p), 256, 0, s>>>(U, ldu, c, C, p, V, ldv, rows, p);
    LRA_LAUNCHED();
}

void defl_norms(cudaStream_t s, const double *norm2, const float *Gt, int PPc, int c, int64_t n, double *out) {
    defl_norms_kernel<<<grid_of(n), 256, 0, s>>>(norm2, Gt, PPc, c, n, out);
    LRA_LAUNCHED();
}

void defl_gather(cudaStream_t s, const float *X, int64_t ldx, int64_t dpad, const int32_t *idx, int64_t m,
                 const float *U, int c, const float *Gt, int PPc, float *out) {
    if (m <= 0) return;
    const dim3 grid((unsigned)ceil_div(dpad, 256), (unsigned)ceil_div(m, kGatherT));
    const size_t smem = sizeof(float) * kGatherT * std::max(c, 1);
    ensure_smem(defl_gather_kernel, (int)smem);
    defl_gather_kernel<<<grid, 256, smem, s>>>(X, ldx, dpad, idx, m, U, c, Gt, PPc, out);
    LRA_LAUNCHED();
}

void defl_gather_csc(cudaStream_t s, const int64_t *colptr, const int32_t *rowidx, const float *cval, int64_t dpad,
                     const int32_t *idx, int64_t m, const float *U, int c, const float *Gt, int PPc, float *out) {
    if (m <= 0) return;
    defl_gather(s, nullptr, 0, dpad, idx, m, U, c, Gt, PPc, out);
    defl_scatter_csc_kernel<<<(unsigned)ceil_div(m, 8), 256, 0, s>>>(colptr, rowidx, cval, idx, m, dpad, out);
    LRA_LAUNCHED();
}

}  // namespace lra
