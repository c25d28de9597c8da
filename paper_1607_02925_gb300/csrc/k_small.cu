// p x p and d x p kernels of the outer loop: Gram matrices (FP64 accumulation),
// Cholesky and triangular solve (FP64 / FP32, CholeskyQR2 of Algorithm 1's QR
// step), right-multiplication of tall blocks by small matrices, the symmetric
// eigenproblem of Algorithm 2 (cyclic Jacobi in one CTA, Rayleigh quotients in
// FP64), and small vector helpers.
#include <algorithm>
#include <type_traits>

#include "kernels.cuh"

namespace lra {

namespace {

// ---------------------------------------------------------------------------
// Gram G = A^T A.  Each CTA takes row tiles of 64 rows; thread owns 4x4 blocks
// of (a, b) pairs with a-block <= b-block; partials reduced in fixed order.
// kF64 = false: FP32 products summed over a tile, then added to FP64
// accumulators (tall n x p blocks).  kF64 = true: every product accumulated in
// FP64 (d x p bases, whose Gram must resolve deviations from I near FP32
// rounding).  With Ah != nullptr, A is read as the BF16 pair Ah + Al
// (column-major, leading dimension rows), a sum that FP32 holds exactly.
// ---------------------------------------------------------------------------
constexpr int kGR = 64;        // rows per tile
constexpr int kGMaxBlk = 2;    // 4x4 blocks per thread (406 blocks at p = 112 -> 2 per thread)

template <bool kF64>
__global__ void __launch_bounds__(256) gram_kernel(const float *__restrict__ A, const __nv_bfloat16 *__restrict__ Ah,
                                                   const __nv_bfloat16 *__restrict__ Al, int split, int64_t rows,
                                                   int64_t rs, int64_t cs, int p, int p4,
                                                   double *__restrict__ part) {
    using T = typename std::conditional<kF64, double, float>::type;
    extern __shared__ __align__(16) float As[];  // [kGR][p4]
    const int tid = threadIdx.x;
    const int nb = p4 / 4;
    const int npairs = nb * (nb + 1) / 2;
    int ba[kGMaxBlk], bb[kGMaxBlk];
    int nown = 0;
#pragma unroll
    for (int u = 0; u < kGMaxBlk; ++u) {
        const int q = tid + 256 * u;
        ba[u] = bb[u] = 0;
        if (q < npairs) {
            // q -> (a <= b) in row-major upper-triangle order
            int a = 0, rem = q;
            while (rem >= nb - a) {
                rem -= nb - a;
                ++a;
            }
            ba[u] = a;
            bb[u] = a + rem;
            nown = u + 1;
        }
    }
    double acc[kGMaxBlk][16];
#pragma unroll
    for (int u = 0; u < kGMaxBlk; ++u)
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[u][e] = 0.0;

    for (int64_t t0 = (int64_t)blockIdx.x * kGR; t0 < rows; t0 += (int64_t)gridDim.x * kGR) {
        __syncthreads();
        for (int e = tid; e < kGR * p4; e += 256) {
            int r, j;
            if (rs == 1) {
                r = e % kGR;
                j = e / kGR;
            } else {
                j = e % p4;
                r = e / p4;
            }
            const int64_t row = t0 + r;
            float v = 0.0f;
            if (row < rows && j < p) {
                const int64_t o = row * rs + (int64_t)j * cs;
                if (Ah) {
                    v = __bfloat162float(Ah[o]) + __bfloat162float(Al[o]);
                } else {
                    v = A[o];
                    if (split) {  // the BF16 pair hi + lo of v, as the tensor-core passes see it
                        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
                        v = __bfloat162float(hi) + __bfloat162float(__float2bfloat16_rn(v - __bfloat162float(hi)));
                    }
                }
            }
            As[r * p4 + j] = v;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kGMaxBlk; ++u) {
            if (u < nown) {
                T f[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) f[e] = kF64 ? acc[u][e] : 0.0f;
                const float *pa = As + 4 * ba[u];
                const float *pb = As + 4 * bb[u];
                for (int r = 0; r < kGR; ++r) {
                    const float4 x = *reinterpret_cast<const float4 *>(pa + r * p4);
                    const float4 y = *reinterpret_cast<const float4 *>(pb + r * p4);
                    const T xa[4] = {x.x, x.y, x.z, x.w};
                    const T ya[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) f[4 * i + j] = fma(xa[i], ya[j], f[4 * i + j]);
                }
#pragma unroll
                for (int e = 0; e < 16; ++e) acc[u][e] = kF64 ? (double)f[e] : acc[u][e] + (double)f[e];
            }
        }
    }
    double *out = part + (int64_t)blockIdx.x * p4 * p4;
#pragma unroll
    for (int u = 0; u < kGMaxBlk; ++u) {
        if (u < nown) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) out[(4 * ba[u] + i) * p4 + 4 * bb[u] + j] = acc[u][4 * i + j];
        }
    }
}

__global__ void gram_reduce_kernel(const double *__restrict__ part, int nparts, int p, int p4,
                                   double *__restrict__ G) {
    // thread per entry (a, b) of the partials' row-major p4 x p4 layout (coalesced
    // reads); only the stored blocks (a-block <= b-block) are summed, each into
    // both G[a + b p] and G[b + a p]
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= p4 * p4) return;
    const int a = e / p4, b = e % p4;
    if (a >= p || b >= p || a / 4 > b / 4) return;
    // four independent partial sums over interleaved parts, combined in a fixed order
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    const int64_t stride = (int64_t)p4 * p4;
    int c = 0;
    for (; c + 3 < nparts; c += 4) {
        s0 += part[(c + 0) * stride + e];
        s1 += part[(c + 1) * stride + e];
        s2 += part[(c + 2) * stride + e];
        s3 += part[(c + 3) * stride + e];
    }
    for (; c < nparts; ++c) s0 += part[c * stride + e];
    const double v = (s0 + s1) + (s2 + s3);
    G[a + (int64_t)b * p] = v;
    if (a / 4 < b / 4) G[b + (int64_t)a * p] = v;
}

// ---------------------------------------------------------------------------
// Cross Gram H = (A^T B + B^T A)/2 for A, B dpad x p column-major (A optionally
// the BF16 pair Ah + Al): with B = X (X^T A) this is the Rayleigh-Ritz matrix
// A^T X X^T A from a d-long contraction.  64-row tiles, thread owns 4x4 blocks
// over all (a, b) block pairs; FP32 sums over a tile added into FP64; partials
// reduced (and symmetrised) in fixed order.
// ---------------------------------------------------------------------------
constexpr int kCMaxBlk = 4;    // 784 block pairs at p = 112 -> up to 4 per thread

__global__ void __launch_bounds__(256) cross_gram_kernel(const float *__restrict__ A,
                                                         const __nv_bfloat16 *__restrict__ Ah,
                                                         const __nv_bfloat16 *__restrict__ Al,
                                                         const float *__restrict__ B, int64_t rows, int64_t ld,
                                                         int p, int p4, double *__restrict__ part) {
    extern __shared__ __align__(16) float cs_[];
    float *As = cs_, *Bs = cs_ + kGR * p4;  // [kGR][p4] each
    const int tid = threadIdx.x;
    const int nb = p4 / 4;
    const int npairs = nb * nb;
    int ba[kCMaxBlk], bb[kCMaxBlk];
    int nown = 0;
#pragma unroll
    for (int u = 0; u < kCMaxBlk; ++u) {
        const int q = tid + 256 * u;
        ba[u] = bb[u] = 0;
        if (q < npairs) {
            ba[u] = q / nb;
            bb[u] = q % nb;
            nown = u + 1;
        }
    }
    double acc[kCMaxBlk][16];
#pragma unroll
    for (int u = 0; u < kCMaxBlk; ++u)
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[u][e] = 0.0;
    for (int64_t t0 = (int64_t)blockIdx.x * kGR; t0 < rows; t0 += (int64_t)gridDim.x * kGR) {
        __syncthreads();
        for (int e = tid; e < kGR * p4; e += 256) {
            const int r = e % kGR, j = e / kGR;
            const int64_t row = t0 + r;
            float va = 0.0f, vb = 0.0f;
            if (row < rows && j < p) {
                const int64_t o = row + (int64_t)j * ld;
                va = Ah ? __bfloat162float(Ah[o]) + __bfloat162float(Al[o]) : A[o];
                vb = B[o];
            }
            As[r * p4 + j] = va;
            Bs[r * p4 + j] = vb;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kCMaxBlk; ++u) {
            if (u < nown) {
                float f[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) f[e] = 0.0f;
                const float *pa = As + 4 * ba[u];
                const float *pb = Bs + 4 * bb[u];
                for (int r = 0; r < kGR; ++r) {
                    const float4 x = *reinterpret_cast<const float4 *>(pa + r * p4);
                    const float4 y = *reinterpret_cast<const float4 *>(pb + r * p4);
                    const float xa[4] = {x.x, x.y, x.z, x.w};
                    const float ya[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) f[4 * i + j] = fmaf(xa[i], ya[j], f[4 * i + j]);
                }
#pragma unroll
                for (int e = 0; e < 16; ++e) acc[u][e] += (double)f[e];
            }
        }
    }
    double *out = part + (int64_t)blockIdx.x * p4 * p4;
#pragma unroll
    for (int u = 0; u < kCMaxBlk; ++u) {
        if (u < nown) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) out[(4 * ba[u] + i) * p4 + 4 * bb[u] + j] = acc[u][4 * i + j];
        }
    }
}

// C[a][b] = sum_c part[c][a][b] (chunks in order, coalesced), then
// H[a + b p] = (C[a][b] + C[b][a]) / 2
__global__ void cross_reduce_kernel(const double *__restrict__ part, int nparts, int p4,
                                    double *__restrict__ C) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= p4 * p4) return;
    const int64_t stride = (int64_t)p4 * p4;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int c = 0;
    for (; c + 3 < nparts; c += 4) {
        s0 += part[(c + 0) * stride + e];
        s1 += part[(c + 1) * stride + e];
        s2 += part[(c + 2) * stride + e];
        s3 += part[(c + 3) * stride + e];
    }
    for (; c < nparts; ++c) s0 += part[c * stride + e];
    C[e] = (s0 + s1) + (s2 + s3);
}

__global__ void symmetrise_kernel(const double *__restrict__ C, int p, int p4, double *__restrict__ H) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= p * p) return;
    const int a = e % p, b = e / p;
    H[e] = 0.5 * (C[a * p4 + b] + C[b * p4 + a]);
}

// Rayleigh-Ritz on a basis S that is orthonormal only to rounding: with
// G = S^T S = I + F and H = S^T A S, the Ritz values of the orthonormalised
// basis S G^(-1/2) are those of G^(-1/2) H G^(-1/2) = H - (F H + H F)/2 + O(F^2)
// = 2H - (G H + H G)/2 + O(F^2).  One CTA per column j, thread = row i; G and
// H symmetric and column-major.
__global__ void ortho_correct_kernel(const double *__restrict__ H, const double *__restrict__ G, int p,
                                     double *__restrict__ Hc) {
    __shared__ double hj[LRA_MAX_P], gj[LRA_MAX_P];
    const int j = blockIdx.x, i = threadIdx.x;
    if (i < p) {
        hj[i] = H[i + (int64_t)j * p];
        gj[i] = G[i + (int64_t)j * p];
    }
    __syncthreads();
    if (i >= p) return;
    double a0 = 0.0, a1 = 0.0;
    for (int l = 0; l < p; ++l) {
        a0 = fma(G[i + (int64_t)l * p], hj[l], a0);  // (G H)_ij, G_il = G_li
        a1 = fma(H[i + (int64_t)l * p], gj[l], a1);  // (H G)_ij
    }
    Hc[i + (int64_t)j * p] = 2.0 * hj[i] - 0.5 * (a0 + a1);
}

int gram_blocks(int64_t rows) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(rows, kGR), 152)); }

// ---------------------------------------------------------------------------
// Cholesky G = L L^T in FP64, one CTA, one barrier per column: step c reads
// column c (not yet scaled) and updates the trailing lower triangle; the
// scaling of column c by its pivot is applied when R is written out.
// R = L^T (upper, FP32 row-major); status = 1 if a pivot is not positive.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) chol_kernel(const double *__restrict__ G, int p,
                                                   float *__restrict__ R, int *__restrict__ status,
                                                   double near_id) {
    extern __shared__ __align__(16) double sl[];
    const int ld = p + 1;
    double *L = sl;               // [p][ld]
    double *piv = sl + p * ld;    // [p]
    double *g0 = piv + p;         // [p] original diagonal
    __shared__ int bad;
    __shared__ double wsum[8];
    const int tid = threadIdx.x, nt = blockDim.x;
    if (near_id > 0.0) {
        // G = I + E with ||E||_F <= near_id: R = I + F, F upper with F + F^T = E
        // to first order (F = triu(E, 1) + diag(E) / 2); the dropped F^T F is
        // below near_id^2 in norm
        double e2 = 0.0;
        for (int e = tid; e < p * p; e += nt) {
            const double v = G[e] - ((e % p) == (e / p) ? 1.0 : 0.0);
            e2 = fma(v, v, e2);
        }
        e2 = warp_sum(e2);
        if ((tid & 31) == 0) wsum[tid >> 5] = e2;
        __syncthreads();
        double tot = 0.0;
        for (int w = 0; w < (nt >> 5); ++w) tot += wsum[w];
        if (sqrt(tot) <= near_id) {
            for (int e = tid; e < p * p; e += nt) {
                const int a = e / p, b = e % p;  // R[a][b], G column-major
                R[e] = b > a ? (float)G[a + (int64_t)b * p] : (b == a ? (float)(0.5 * (1.0 + G[e])) : 0.0f);
            }
            if (tid == 0) *status = 0;
            return;
        }
    }
    if (tid == 0) bad = 0;
    for (int e = tid; e < p * p; e += nt) L[(e % p) * ld + e / p] = G[e];
    for (int c = tid; c < p; c += nt) g0[c] = G[c + (int64_t)c * p];
    __syncthreads();
    for (int c = 0; c < p; ++c) {
        double dd = L[c * ld + c];
        // a pivot at the rounding level of its original diagonal means the
        // columns are linearly dependent to working precision
        if (!(dd > 1e-14 * g0[c]) || !isfinite(dd)) {
            if (tid == 0) bad = 1;
            dd = 1.0;
        }
        if (tid == 0) piv[c] = sqrt(dd);
        const double inv = 1.0 / dd;  // (l_rc / sqrt dd)(l_sc / sqrt dd) = l_rc l_sc / dd
        // trailing update of the lower triangle: warp per row, lanes along the
        // row; column c is only read in this step
        const int lane = tid & 31, nw = nt >> 5;
        for (int rr = c + 1 + (tid >> 5); rr < p; rr += nw) {
            const double lr = L[rr * ld + c] * inv;
            for (int ss = c + 1 + lane; ss <= rr; ss += 32) L[rr * ld + ss] -= lr * L[ss * ld + c];
        }
        __syncthreads();
    }
    for (int e = tid; e < p * p; e += nt) {
        const int a = e / p, b = e % p;  // R[a][b] = L[b][a] / piv[a] for b > a
        float v = 0.0f;
        if (b == a)
            v = (float)piv[a];
        else if (b > a)
            v = (float)(L[b * ld + a] / piv[a]);
        R[e] = v;
    }
    if (tid == 0) *status = bad;
}

// Q = W R^-1 row by row (forward substitution q_j = (w_j - sum_{l<j} q_l R_lj) / R_jj),
// one thread per row; R in shared memory, the row's q in shared memory.
constexpr int kTrsmRows = 64;  // rows (threads) per CTA

__global__ void __launch_bounds__(kTrsmRows) trsm_rows_kernel(const float *__restrict__ W, int64_t rows,
                                                              int64_t ld, int p, const float *__restrict__ R,
                                                              float *__restrict__ Q) {
    extern __shared__ __align__(16) float sr[];
    float *Rs = sr;               // [p][p]
    float *qs = sr + p * p;       // [p][kTrsmRows]
    const int tid = threadIdx.x;
    for (int e = tid; e < p * p; e += kTrsmRows) Rs[e] = R[e];
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * kTrsmRows + tid;
    if (r >= rows) return;
    for (int j = 0; j < p; ++j) {
        // four interleaved partial sums shorten the dependent chain
        float s0 = W[r + (int64_t)j * ld], s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
        int l = 0;
        for (; l + 3 < j; l += 4) {
            s0 = fmaf(-qs[(l + 0) * kTrsmRows + tid], Rs[(l + 0) * p + j], s0);
            s1 = fmaf(-qs[(l + 1) * kTrsmRows + tid], Rs[(l + 1) * p + j], s1);
            s2 = fmaf(-qs[(l + 2) * kTrsmRows + tid], Rs[(l + 2) * p + j], s2);
            s3 = fmaf(-qs[(l + 3) * kTrsmRows + tid], Rs[(l + 3) * p + j], s3);
        }
        for (; l < j; ++l) s0 = fmaf(-qs[l * kTrsmRows + tid], Rs[l * p + j], s0);
        const float q = ((s0 + s1) + (s2 + s3)) / Rs[j * p + j];
        qs[j * kTrsmRows + tid] = q;
        Q[r + (int64_t)j * ld] = q;
    }
}

// ---------------------------------------------------------------------------
// Out (rows x q) = A (rows x p) T (p x q, FP32 row-major).  CTA = 128 rows x
// 16 output columns; thread = one row x 8 columns.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) apply_right_kernel(const float *__restrict__ A, int64_t rows,
                                                          int64_t ars, int64_t acs, int p,
                                                          const float *__restrict__ T, int q,
                                                          float *__restrict__ Out, int64_t ors,
                                                          int64_t ocs) {
    extern __shared__ __align__(16) float Ts[];  // [p][16]
    const int tid = threadIdx.x;
    const int c0 = blockIdx.y * 16;
    for (int e = tid; e < p * 16; e += 256) {
        const int l = e / 16, j = e % 16;
        Ts[e] = (c0 + j < q) ? T[l * q + c0 + j] : 0.0f;
    }
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * 128 + (tid & 127);
    const int half = tid >> 7;
    if (r >= rows) return;
    float acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = 0.0f;
    for (int l = 0; l < p; ++l) {
        const float a = A[r * ars + (int64_t)l * acs];
        const float4 t0 = *reinterpret_cast<const float4 *>(Ts + l * 16 + half * 8);
        const float4 t1 = *reinterpret_cast<const float4 *>(Ts + l * 16 + half * 8 + 4);
        acc[0] = fmaf(a, t0.x, acc[0]);
        acc[1] = fmaf(a, t0.y, acc[1]);
        acc[2] = fmaf(a, t0.z, acc[2]);
        acc[3] = fmaf(a, t0.w, acc[3]);
        acc[4] = fmaf(a, t1.x, acc[4]);
        acc[5] = fmaf(a, t1.y, acc[5]);
        acc[6] = fmaf(a, t1.z, acc[6]);
        acc[7] = fmaf(a, t1.w, acc[7]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int c = c0 + half * 8 + j;
        if (c < q) Out[r * ors + (int64_t)c * ocs] = acc[j];
    }
}

// ---------------------------------------------------------------------------
// Cyclic Jacobi in FP32, one CTA, round-robin ordering (p2 = p rounded up to
// even; index m = p2 - 1 is the fixed player): in round r index a is paired
// with a' = r if a = m, m if a = r, else (2r - a) mod m.  Classical rotation
// (Golub & Van Loan, sym.schur2) for pair (i < j): tau = (a_jj - a_ii)/(2 a_ij),
// t = sign(tau)/(|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2), s = t c.  The
// two-sided update A' = J^T A J and V' = V J of all disjoint pairs of a round is
// computed elementwise into a second buffer:
//   A'[a][b] = al_a (al_b A[a][b] + be_b A[a][b']) + be_a (al_b A[a'][b] + be_b A[a'][b'])
// with (al, be) = (c, -s) for the smaller index of a pair, (c, +s) for the
// larger; two barriers per round.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int rr_partner(int a, int r, int m) {
    if (a == m) return r;
    if (a == r) return m;
    int q = (2 * r - a) % m;
    return q < 0 ? q + m : q;
}

__global__ void __launch_bounds__(512) jacobi_kernel(const double *__restrict__ H, int p,
                                                     double *__restrict__ Vout, int max_sweeps, double tol) {
    extern __shared__ __align__(16) float jb[];
    const int p2 = p + (p & 1);
    const int ld = p2 + 1;
    const int sz = p2 * ld;
    float *A0 = jb, *A1 = jb + sz, *V0 = jb + 2 * sz, *V1 = jb + 3 * sz;
    float *al = jb + 4 * sz;        // [p2] alpha of each index this round
    float *be = al + p2;            // [p2] beta (-s for the smaller index, +s for the larger)
    int *part = reinterpret_cast<int *>(be + p2);  // [p2] partner this round
    __shared__ double red_off[16], red_tot[16];
    __shared__ int stop, rotated;
    const int tid = threadIdx.x, nt = blockDim.x;
    const float eps = 1e-7f;
    if (tid == 0) rotated = 0;
    for (int e = tid; e < p2 * p2; e += nt) {
        const int a = e / p2, b = e % p2;
        A0[a * ld + b] = (a < p && b < p) ? (float)H[a + (int64_t)b * p] : 0.0f;
        V0[a * ld + b] = (a == b) ? 1.0f : 0.0f;
    }
    __syncthreads();
    const int m = p2 - 1;
    const int tpr = nt / p2;          // threads per row in the update phase (>= 4)
    const int row = tid / tpr, q = tid - (tid / tpr) * tpr;
    float *A = A0, *An = A1, *V = V0, *Vn = V1;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int e = tid; e < p2 * p2; e += nt) {
            const int a = e / p2, b = e % p2;
            const double v = (double)A[a * ld + b];
            tot += v * v;
            if (a != b) off += v * v;
        }
        off = warp_sum(off);
        tot = warp_sum(tot);
        if ((tid & 31) == 0) {
            red_off[tid >> 5] = off;
            red_tot[tid >> 5] = tot;
        }
        __syncthreads();
        if (tid == 0) {
            double o = 0.0, t = 0.0;
            for (int w = 0; w < (nt >> 5); ++w) {
                o += red_off[w];
                t += red_tot[w];
            }
            // squared relative off-diagonal mass below tol: the FP64 refinement
            // that follows squares the remaining rotation angles
            stop = (o <= tol * t || (sweep > 0 && !rotated)) ? 1 : 0;
            rotated = 0;
        }
        __syncthreads();
        if (stop) break;
        for (int r = 0; r < m; ++r) {
            // phase 1: partner, and the (alpha, beta) of each index for this round
            for (int i = tid; i < p2; i += nt) {
                const int j = rr_partner(i, r, m);
                part[i] = j;
                if (i < j) {
                    const float aij = A[i * ld + j], aii = A[i * ld + i], ajj = A[j * ld + j];
                    float c = 1.0f, s = 0.0f;
                    if (aij != 0.0f && fabsf(aij) > eps * sqrtf(fabsf(aii * ajj))) {
                        const float tau = (ajj - aii) / (2.0f * aij);
                        const float t = fabsf(tau) > 1e15f ? 1.0f / (2.0f * tau)
                                                             : copysignf(1.0f, tau) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
                        c = 1.0f / sqrtf(1.0f + t * t);
                        s = t * c;
                        rotated = 1;
                    }
                    al[i] = c;
                    al[j] = c;
                    be[i] = -s;
                    be[j] = s;
                }
            }
            __syncthreads();
            // phase 2: A' = J^T A J and V' = V J elementwise into the other buffers
            // thread = (row a, column offset q): columns q, q + tpr, ... of row a
            if (row < p2) {
                const int a = row, ap = part[a];
                const float ala = al[a], bea = be[a];
                const float *Aa = A + a * ld, *Aap = A + ap * ld, *Va = V + a * ld;
                float *Ana = An + a * ld, *Vna = Vn + a * ld;
                for (int b = q; b < p2; b += tpr) {
                    const int bp = part[b];
                    const float alb = al[b], beb = be[b];
                    const float x = alb * Aa[b] + beb * Aa[bp];
                    const float y = alb * Aap[b] + beb * Aap[bp];
                    Ana[b] = (bp == a && beb != 0.0f) ? 0.0f : ala * x + bea * y;
                    Vna[b] = alb * Va[b] + beb * Va[bp];
                }
            }
            __syncthreads();
            float *t = A; A = An; An = t;
            t = V; V = Vn; Vn = t;
        }
    }
    for (int e = tid; e < p * p; e += nt) {
        const int a = e % p, b = e / p;
        Vout[e] = (double)V[a * ld + b];
    }
}

// C = op(A) B for p x p FP64 column-major matrices (op = transpose if ta),
// optionally C = alpha C + beta I afterwards; one CTA per column of C.
__global__ void __launch_bounds__(128) gemm_pp_kernel(const double *__restrict__ A,
                                                      const double *__restrict__ B, int p, int ta,
                                                      double alpha, double beta,
                                                      double *__restrict__ C) {
    __shared__ double bj[LRA_MAX_P + 16];
    const int j = blockIdx.x;
    for (int l = threadIdx.x; l < p; l += blockDim.x) bj[l] = B[l + (int64_t)j * p];
    __syncthreads();
    for (int i = threadIdx.x; i < p; i += blockDim.x) {
        double s = 0.0;
        if (ta)
            for (int l = 0; l < p; ++l) s += A[l + (int64_t)i * p] * bj[l];
        else
            for (int l = 0; l < p; ++l) s += A[i + (int64_t)l * p] * bj[l];
        C[i + (int64_t)j * p] = alpha * s + (i == j ? beta : 0.0);
    }
}

// First-order rotation of nearly diagonal B = V^T H V: F = I + E with
// E_ij = B_ij / (B_jj - B_ii) (i != j), skipped where |B_ij| > 0.1 |B_jj - B_ii|
// (near-degenerate pairs, whose rotation does not change the spanned space).
__global__ void correction_kernel(const double *__restrict__ B, int p, double *__restrict__ F) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= p * p) return;
    const int i = e % p, j = e / p;
    double v = 0.0;
    if (i == j) {
        v = 1.0;
    } else {
        const double gap = B[j + (int64_t)j * p] - B[i + (int64_t)i * p];
        const double bij = B[e];
        if (fabs(bij) <= 0.1 * fabs(gap) && gap != 0.0) v = bij / gap;
    }
    F[e] = v;
}

// rho_j = v_j^T H v_j / v_j^T v_j in FP64, one CTA per eigenvector.
__global__ void __launch_bounds__(128) rayleigh_kernel(const double *__restrict__ H,
                                                       const double *__restrict__ V, int p,
                                                       double *__restrict__ rho) {
    __shared__ double v[LRA_MAX_P + 16];
    __shared__ double red[2][4];
    const int j = blockIdx.x, tid = threadIdx.x;
    for (int a = tid; a < p; a += 128) v[a] = V[a + (int64_t)j * p];
    __syncthreads();
    double num = 0.0, den = 0.0;
    for (int a = tid; a < p; a += 128) {
        double hv = 0.0;
        for (int b = 0; b < p; ++b) hv += H[a + (int64_t)b * p] * v[b];
        num += v[a] * hv;
        den += v[a] * v[a];
    }
    num = warp_sum(num);
    den = warp_sum(den);
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = num;
        red[1][tid >> 5] = den;
    }
    __syncthreads();
    if (tid == 0) {
        const double nn = red[0][0] + red[0][1] + red[0][2] + red[0][3];
        const double dd = red[1][0] + red[1][1] + red[1][2] + red[1][3];
        rho[j] = nn / dd;
    }
}

// Sort descending (ties by index), normalise each vector, sign: largest |entry| > 0.
__global__ void __launch_bounds__(128) sort_sign_kernel(const double *__restrict__ rho_in,
                                                        const double *__restrict__ V, int p,
                                                        double *__restrict__ evals,
                                                        double *__restrict__ evecs) {
    const int j = blockIdx.x, tid = threadIdx.x;
    __shared__ int rank;
    __shared__ double nrm;
    __shared__ int amax;
    if (tid == 0) {
        const double rj = rho_in[j];
        int r = 0;
        for (int i = 0; i < p; ++i) {
            const double ri = rho_in[i];
            if (ri > rj || (ri == rj && i < j)) ++r;
        }
        rank = r;
        double s = 0.0, best = -1.0;
        int bi = 0;
        for (int a = 0; a < p; ++a) {
            const double v = V[a + (int64_t)j * p];
            s += v * v;
            if (fabs(v) > best) {
                best = fabs(v);
                bi = a;
            }
        }
        nrm = sqrt(s);
        amax = bi;
        evals[r] = rj;
    }
    __syncthreads();
    const double sg = V[amax + (int64_t)j * p] < 0.0 ? -1.0 : 1.0;
    for (int a = tid; a < p; a += 128) evecs[a + (int64_t)rank * p] = sg * V[a + (int64_t)j * p] / nrm;
}

// P = V diag(1/(lam - rho)) V^T (FP64 -> FP32 row-major), one CTA per row.
__global__ void ritz_inverse_kernel(const double *__restrict__ V, const double *__restrict__ rho,
                                    int p, double lam, float *__restrict__ P) {
    const int a = blockIdx.x;
    for (int b = threadIdx.x; b < p; b += blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < p; ++j) s += V[a + (int64_t)j * p] * V[b + (int64_t)j * p] / (lam - rho[j]);
        P[a * p + b] = (float)s;
    }
}

// P (p x p FP32 row-major) = V diag(1/(lam - rho)): the Galerkin inverse
// (lam I - H)^-1 expressed from the Ritz basis S V
__global__ void ritz_scaled_kernel(const double *__restrict__ V, const double *__restrict__ rho, int p,
                                   double lam, float *__restrict__ P) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= p * p) return;
    const int a = e / p, j = e % p;
    P[e] = (float)(V[a + (int64_t)j * p] / (lam - rho[j]));
}

// dst[:, j] = src[:, j] / (lam - rho[j])
__global__ void shift_scale_cols_kernel(const float *__restrict__ src, float *__restrict__ dst, int64_t rows,
                                        int64_t ld, int p, const double *__restrict__ rho, double lam) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * p;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / rows, r = e - j * rows;
        dst[r + j * ld] = (float)((double)src[r + j * ld] / (lam - rho[j]));
    }
}

__global__ void evecs_to_rm_kernel(const double *__restrict__ V, int p, int k, float *__restrict__ T) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= p * k) return;
    const int a = e / k, j = e % k;
    T[e] = (float)V[a + (int64_t)j * p];
}

__global__ void __launch_bounds__(256) col_dots_kernel(const float *__restrict__ A,
                                                       const float *__restrict__ B, int64_t rows,
                                                       int64_t ld, double *__restrict__ out) {
    __shared__ double red[8];
    const int j = blockIdx.x;
    double s = 0.0;
    for (int64_t r = threadIdx.x; r < rows; r += 256)
        s += (double)A[r + (int64_t)j * ld] * (double)B[r + (int64_t)j * ld];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        out[j] = t;
    }
}

__global__ void scale_cols_rsqrt_kernel(float *__restrict__ A, int64_t rows, int64_t ld, int p,
                                        const double *__restrict__ n2) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * p) return;
    const int j = (int)(e / rows);
    const int64_t r = e % rows;
    A[r + j * ld] = (float)((double)A[r + j * ld] / sqrt(n2[j]));
}

__global__ void scale_block_kernel(float *__restrict__ A, int64_t rows, int64_t ld, int p, float alpha) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * p) return;
    const int j = (int)(e / rows);
    const int64_t r = e % rows;
    A[r + j * ld] *= alpha;
}

// Z = W + beta (W - Wold), Wold = W (first: Z = W, Wold not read).
__global__ void acc_extrapolate_kernel(const float *__restrict__ W, float *__restrict__ Wold,
                                       float *__restrict__ Z, int64_t rows, int64_t ld, int p, float beta,
                                       int first) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * p) return;
    const int j = (int)(e / rows);
    const int64_t i = e % rows + (int64_t)j * ld;
    const float w = W[i];
    Z[i] = first ? w : w + beta * (w - Wold[i]);
    Wold[i] = w;
}

}  // namespace

void acc_extrapolate(cudaStream_t s, const float *W, float *Wold, float *Z, int64_t rows, int64_t ld, int p,
                     float beta, bool first) {
    acc_extrapolate_kernel<<<(unsigned)ceil_div(rows * p, 256), 256, 0, s>>>(W, Wold, Z, rows, ld, p, beta,
                                                                              first ? 1 : 0);
    LRA_LAUNCHED();
}

int64_t gram_scratch(int p) {
    const int p4 = (int)round_up(p, 4);
    return (int64_t)2 * 152 * p4 * p4;
}

void gram(cudaStream_t s, const float *A, int64_t rows, int64_t rs, int64_t cs, int p, double *G,
          double *scratch) {
    const int p4 = (int)round_up(p, 4);
    const int nb = gram_blocks(rows);
    const size_t smem = sizeof(float) * kGR * p4;
    LRA_CUDA(cudaMemsetAsync(scratch, 0, sizeof(double) * nb * p4 * p4, s));
    gram_kernel<false><<<nb, 256, smem, s>>>(A, nullptr, nullptr, 0, rows, rs, cs, p, p4, scratch);
    LRA_LAUNCHED();
    gram_reduce_kernel<<<(unsigned)ceil_div(p4 * p4, 256), 256, 0, s>>>(scratch, nb, p, p4, G);
    LRA_LAUNCHED();
}

void gram64(cudaStream_t s, const float *A, const __nv_bfloat16 *Ah, const __nv_bfloat16 *Al, int64_t rows,
            int64_t ld, int p, double *G, double *scratch, bool split) {
    const int p4 = (int)round_up(p, 4);
    const int nb = gram_blocks(rows);
    const size_t smem = sizeof(float) * kGR * p4;
    LRA_CUDA(cudaMemsetAsync(scratch, 0, sizeof(double) * nb * p4 * p4, s));
    gram_kernel<true><<<nb, 256, smem, s>>>(A, Ah, Al, split ? 1 : 0, rows, 1, ld, p, p4, scratch);
    LRA_LAUNCHED();
    gram_reduce_kernel<<<(unsigned)ceil_div(p4 * p4, 256), 256, 0, s>>>(scratch, nb, p, p4, G);
    LRA_LAUNCHED();
}

void cross_gram(cudaStream_t s, const float *A, const __nv_bfloat16 *Ah, const __nv_bfloat16 *Al, const float *B,
                int64_t rows, int64_t ld, int p, double *H, double *scratch) {
    const int p4 = (int)round_up(p, 4);
    const int nb = gram_blocks(rows);
    const size_t smem = sizeof(float) * 2 * kGR * p4;
    ensure_smem(cross_gram_kernel, (int)smem);
    cross_gram_kernel<<<nb, 256, smem, s>>>(A, Ah, Al, B, rows, ld, p, p4, scratch);
    LRA_LAUNCHED();
    double *C = scratch + (int64_t)nb * p4 * p4;  // gram_scratch holds 2 x 152 partials
    cross_reduce_kernel<<<(unsigned)ceil_div(p4 * p4, 256), 256, 0, s>>>(scratch, nb, p4, C);
    LRA_LAUNCHED();
    symmetrise_kernel<<<(unsigned)ceil_div(p * p, 256), 256, 0, s>>>(C, p, p4, H);
    LRA_LAUNCHED();
}

namespace {
__global__ void copy_full_kernel(const double *__restrict__ C, int p, int p4, double *__restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= p * p) return;
    const int a = e % p, b = e / p;
    out[e] = C[a * p4 + b];
}
}  // namespace

void cross_full(cudaStream_t s, const float *A, const float *B, int64_t rows, int64_t ld, int p, double *out,
                double *scratch) {
    const int p4 = (int)round_up(p, 4);
    const int nb = gram_blocks(rows);
    const size_t smem = sizeof(float) * 2 * kGR * p4;
    ensure_smem(cross_gram_kernel, (int)smem);
    cross_gram_kernel<<<nb, 256, smem, s>>>(A, nullptr, nullptr, B, rows, ld, p, p4, scratch);
    LRA_LAUNCHED();
    double *C = scratch + (int64_t)nb * p4 * p4;
    cross_reduce_kernel<<<(unsigned)ceil_div(p4 * p4, 256), 256, 0, s>>>(scratch, nb, p4, C);
    LRA_LAUNCHED();
    copy_full_kernel<<<(unsigned)ceil_div(p * p, 256), 256, 0, s>>>(C, p, p4, out);
    LRA_LAUNCHED();
}

void ortho_correct(cudaStream_t s, const double *H, const double *G, int p, double *Hc) {
    ortho_correct_kernel<<<p, (unsigned)round_up(p, 32), 0, s>>>(H, G, p, Hc);
    LRA_LAUNCHED();
}

void chol(cudaStream_t s, const double *G, int p, float *R, int *status, double near_id) {
    const size_t smem = sizeof(double) * ((size_t)p * (p + 1) + 2 * p);
    ensure_smem(chol_kernel, (int)smem);
    const int nt = p <= 48 ? 128 : 256;
    chol_kernel<<<1, nt, smem, s>>>(G, p, R, status, near_id);
    LRA_LAUNCHED();
}

void trsm_rows(cudaStream_t s, const float *W, int64_t rows, int64_t ld, int p, const float *R, float *Q) {
    const size_t smem = sizeof(float) * ((size_t)p * p + (size_t)p * kTrsmRows);
    ensure_smem(trsm_rows_kernel, (int)smem);
    trsm_rows_kernel<<<(unsigned)ceil_div(rows, kTrsmRows), kTrsmRows, smem, s>>>(W, rows, ld, p, R, Q);
    LRA_LAUNCHED();
}


void apply_right(cudaStream_t s, const float *A, int64_t rows, int64_t ars, int64_t acs, int p,
                 const float *T, int q, float *Out, int64_t ors, int64_t ocs) {
    const dim3 grid((unsigned)ceil_div(rows, 128), (unsigned)ceil_div(q, 16));
    const size_t smem = sizeof(float) * p * 16;
    apply_right_kernel<<<grid, 256, smem, s>>>(A, rows, ars, acs, p, T, q, Out, ors, ocs);
    LRA_LAUNCHED();
}

// Eigenvectors: cyclic Jacobi in FP32 (one CTA; FP32 runs at 64x the FP64 rate
// of this GPU), then an FP64 refinement spread over p CTAs per step:
// Newton-Schulz orthonormalisation V <- V (3 I - V^T V) / 2, B = V^T H V, the
// first-order rotation V <- V (I + E) that annihilates B's off-diagonal to
// second order, a second orthonormalisation, and FP64 Rayleigh quotients.
void sym_eig(cudaStream_t s, const double *H, int p, double *evals, double *evecs, double *work, int passes,
             double jacobi_tol) {
    const int p2 = p + (p & 1);
    const size_t pp = (size_t)p * p;
    double *V = work;           // p*p
    double *rho = work + pp;    // p
    double *T1 = evecs;         // scratch until the final sort (p*p)
    double *T2 = work + pp + p;  // p*p
    double *V2 = T2 + pp;       // p*p
    const size_t smem = sizeof(float) * (4 * p2 * (p2 + 1) + 3 * p2);
    ensure_smem(jacobi_kernel, (int)smem);
    const int nt = p2 <= 16 ? 128 : 512;
    jacobi_kernel<<<1, nt, smem, s>>>(H, p, V, 40, jacobi_tol);
    LRA_LAUNCHED();
    auto gemm = [&](const double *A, const double *B, int ta, double alpha, double beta, double *C) {
        gemm_pp_kernel<<<p, 128, 0, s>>>(A, B, p, ta, alpha, beta, C);
        LRA_LAUNCHED();
    };
    auto orthonormalise = [&](double *Vin, double *Vout) {
        gemm(Vin, Vin, 1, -0.5, 1.5, T1);   // T1 = 1.5 I - 0.5 V^T V
        gemm(Vin, T1, 0, 1.0, 0.0, Vout);   // Vout = V T1
    };
    for (int pass = 0; pass < passes; ++pass) {  // each pass squares the off-diagonal
        orthonormalise(V, V2);
        gemm(H, V2, 0, 1.0, 0.0, T1);       // T1 = H V
        gemm(V2, T1, 1, 1.0, 0.0, T2);      // T2 = V^T H V
        correction_kernel<<<(unsigned)ceil_div((int64_t)pp, 256), 256, 0, s>>>(T2, p, T1);
        LRA_LAUNCHED();
        gemm(V2, T1, 0, 1.0, 0.0, V);       // V = V2 (I + E)
    }
    orthonormalise(V, V2);
    rayleigh_kernel<<<p, 128, 0, s>>>(H, V2, p, rho);
    LRA_LAUNCHED();
    sort_sign_kernel<<<p, 128, 0, s>>>(rho, V2, p, evals, evecs);
    LRA_LAUNCHED();
}

int64_t sym_eig_work(int p) { return (int64_t)3 * p * p + p; }

void ritz_inverse(cudaStream_t s, const double *evecs, const double *evals, int p, double lam, float *P) {
    ritz_inverse_kernel<<<p, 128, 0, s>>>(evecs, evals, p, lam, P);
    LRA_LAUNCHED();
}

void ritz_scaled(cudaStream_t s, const double *evecs, const double *evals, int p, double lam, float *P) {
    ritz_scaled_kernel<<<(unsigned)ceil_div(p * p, 256), 256, 0, s>>>(evecs, evals, p, lam, P);
    LRA_LAUNCHED();
}

void shift_scale_cols(cudaStream_t s, const float *src, float *dst, int64_t rows, int64_t ld, int p,
                      const double *evals, double lam) {
    const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(rows * p, 256), 152 * 16);
    shift_scale_cols_kernel<<<blocks, 256, 0, s>>>(src, dst, rows, ld, p, evals, lam);
    LRA_LAUNCHED();
}

void evecs_to_rm(cudaStream_t s, const double *evecs, int p, int k, float *T) {
    evecs_to_rm_kernel<<<(unsigned)ceil_div(p * k, 256), 256, 0, s>>>(evecs, p, k, T);
    LRA_LAUNCHED();
}

void col_dots(cudaStream_t s, const float *A, const float *B, int64_t rows, int64_t ld, int p, double *out) {
    col_dots_kernel<<<p, 256, 0, s>>>(A, B, rows, ld, out);
    LRA_LAUNCHED();
}

void scale_cols_rsqrt(cudaStream_t s, float *A, int64_t rows, int64_t ld, int p, const double *n2) {
    scale_cols_rsqrt_kernel<<<(unsigned)ceil_div(rows * p, 256), 256, 0, s>>>(A, rows, ld, p, n2);
    LRA_LAUNCHED();
}

void scale_block(cudaStream_t s, float *A, int64_t rows, int64_t ld, int p, float alpha) {
    scale_block_kernel<<<(unsigned)ceil_div(rows * p, 256), 256, 0, s>>>(A, rows, ld, p, alpha);
    LRA_LAUNCHED();
}

}  // namespace lra
