// p x p and d x p kernels of the outer loop: Gram matrices (FP64 accumulation),
// Cholesky and triangular inverse (FP64, CholeskyQR2 of Algorithm 1's QR
// step), right-multiplication of tall blocks by small matrices, the symmetric
// eigenproblem of Algorithm 2 (cyclic Jacobi in one CTA, Rayleigh quotients in
// FP64), and small vector helpers.
#include <algorithm>

#include "kernels.cuh"

namespace lra {

namespace {

// ---------------------------------------------------------------------------
// Gram G = A^T A.  Each CTA takes row tiles of 64 rows; thread owns 4x4 blocks
// of (a, b) pairs with a-block <= b-block; FP32 products summed over a tile,
// then added to FP64 accumulators; partials reduced in fixed order.
// ---------------------------------------------------------------------------
constexpr int kGR = 64;        // rows per tile
constexpr int kGMaxBlk = 2;    // 4x4 blocks per thread (406 blocks at p = 112 -> 2 per thread)

__global__ void __launch_bounds__(256) gram_kernel(const float *__restrict__ A, int64_t rows,
                                                   int64_t rs, int64_t cs, int p, int p4,
                                                   double *__restrict__ part) {
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
            As[r * p4 + j] = (row < rows && j < p) ? A[row * rs + (int64_t)j * cs] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kGMaxBlk; ++u) {
            if (u < nown) {
                float f[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) f[e] = 0.0f;
                const float *pa = As + 4 * ba[u];
                const float *pb = As + 4 * bb[u];
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
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= p * p) return;
    int a = e % p, b = e / p;  // G column-major: G[a + b p]
    if (a / 4 > b / 4) {
        const int t = a;
        a = b;
        b = t;
    }
    double s = 0.0;
    for (int c = 0; c < nparts; ++c) s += part[(int64_t)c * p4 * p4 + a * p4 + b];
    G[e] = s;
}

int gram_blocks(int64_t rows) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(rows, kGR), 2 * 152)); }

// ---------------------------------------------------------------------------
// Cholesky G = L L^T (L = R^T) and L^-1, FP64, one CTA.  Rinv = (L^-1)^T as
// FP32 row-major.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) chol_inv_kernel(const double *__restrict__ G, int p,
                                                       float *__restrict__ Rinv, int *__restrict__ status) {
    extern __shared__ __align__(16) double sm[];
    const int ld = p + 1;
    double *L = sm;            // [p][ld]
    double *Li = sm + p * ld;  // [p][ld]
    __shared__ int bad;
    const int tid = threadIdx.x;
    if (tid == 0) bad = 0;
    for (int e = tid; e < p * p; e += 256) {
        const int a = e % p, b = e / p;
        L[a * ld + b] = G[e];
        Li[a * ld + b] = 0.0;
    }
    __syncthreads();
    for (int c = 0; c < p; ++c) {
        if (tid == 0) {
            const double piv = L[c * ld + c];
            if (!(piv > 0.0) || !isfinite(piv)) {
                bad = 1;
                L[c * ld + c] = 1.0;
            } else {
                L[c * ld + c] = sqrt(piv);
            }
        }
        __syncthreads();
        const double dcc = L[c * ld + c];
        for (int r = c + 1 + tid; r < p; r += 256) L[r * ld + c] /= dcc;
        __syncthreads();
        const int m = p - c - 1;
        for (int e = tid; e < m * m; e += 256) {
            const int r = c + 1 + e / m, s = c + 1 + e % m;
            if (s <= r) L[r * ld + s] -= L[r * ld + c] * L[s * ld + c];
        }
        __syncthreads();
    }
    // column j of L^-1 by forward substitution (one thread per column)
    for (int j = tid; j < p; j += 256) {
        for (int i = j; i < p; ++i) {
            double s = (i == j) ? 1.0 : 0.0;
            for (int k = j; k < i; ++k) s -= L[i * ld + k] * Li[k * ld + j];
            Li[i * ld + j] = s / L[i * ld + i];
        }
    }
    __syncthreads();
    for (int e = tid; e < p * p; e += 256) {
        const int a = e / p, b = e % p;  // Rinv[a][b] = Li[b][a] (upper triangular)
        Rinv[e] = (float)Li[b * ld + a];
    }
    if (tid == 0) *status = bad;
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
// Cyclic Jacobi (round-robin parallel ordering) in one CTA.  T = float: the
// eigenvectors are FP32-accurate; eigenvalues are recomputed afterwards as FP64
// Rayleigh quotients of the FP64 matrix.  Classical rotation (Golub & Van Loan,
// sym.schur2): tau = (a_jj - a_ii) / (2 a_ij), t = sign(tau)/(|tau| + sqrt(1 +
// tau^2)), c = 1/sqrt(1 + t^2), s = t c; A <- J^T A J, V <- V J.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(512) jacobi_kernel(const double *__restrict__ H, int p,
                                                     double *__restrict__ Vout, int max_sweeps) {
    extern __shared__ __align__(16) unsigned char raw[];
    const int p2 = p + (p & 1);
    const int ld = p2 + 1;
    T *A = reinterpret_cast<T *>(raw);  // [p2][ld]
    T *V = A + p2 * ld;                 // [p2][ld]
    T *cs = V + p2 * ld;                // [p2/2]
    T *sn = cs + p2 / 2;                // [p2/2]
    int *pi = reinterpret_cast<int *>(sn + p2 / 2);  // [p2/2]
    int *pj = pi + p2 / 2;
    __shared__ double red_off[16], red_tot[16];
    __shared__ int stop, rotated;
    const int tid = threadIdx.x, nt = blockDim.x;
    const T eps = sizeof(T) == 4 ? (T)1e-7 : (T)1e-15;
    if (tid == 0) rotated = 0;
    for (int e = tid; e < p2 * p2; e += nt) {
        const int a = e / p2, b = e % p2;
        A[a * ld + b] = (a < p && b < p) ? (T)H[a + (int64_t)b * p] : (T)0;
        V[a * ld + b] = (a == b) ? (T)1 : (T)0;
    }
    __syncthreads();
    const int mrounds = p2 - 1;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        // convergence: off-diagonal mass vs total
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
            // squared relative off-diagonal mass: FP32 sweeps stop at 1e-5 (the
            // FP64 refinement that follows squares it twice); FP64 at 1e-14
            const double tol = sizeof(T) == 4 ? 1e-10 : 1e-28;
            stop = (o <= tol * t || (sweep > 0 && !rotated)) ? 1 : 0;
            rotated = 0;
        }
        __syncthreads();
        if (stop) break;
        for (int rnd = 0; rnd < mrounds; ++rnd) {
            for (int k = tid; k < p2 / 2; k += nt) {
                int i, j;
                if (k == 0) {
                    i = rnd;
                    j = mrounds;
                } else {
                    i = (rnd + k) % mrounds;
                    j = (rnd - k + mrounds) % mrounds;
                }
                if (i > j) {
                    const int t = i;
                    i = j;
                    j = t;
                }
                pi[k] = i;
                pj[k] = j;
                const T aij = A[i * ld + j];
                const T aii = A[i * ld + i], ajj = A[j * ld + j];
                T c = (T)1, s = (T)0;
                if (aij != (T)0 && fabs(aij) > eps * sqrt(fabs(aii * ajj))) {
                    const T tau = (ajj - aii) / ((T)2 * aij);
                    T t;
                    if (fabs(tau) > (T)1e15)
                        t = (T)1 / ((T)2 * tau);
                    else
                        t = (tau >= (T)0 ? (T)1 : (T)-1) / (fabs(tau) + sqrt((T)1 + tau * tau));
                    c = (T)1 / sqrt((T)1 + t * t);
                    s = t * c;
                    rotated = 1;
                }
                cs[k] = c;
                sn[k] = s;
            }
            __syncthreads();
            // columns: A <- A J, V <- V J
            for (int e = tid; e < (p2 / 2) * p2; e += nt) {
                const int k = e / p2, l = e % p2;
                const T c = cs[k], s = sn[k];
                if (s == (T)0) continue;
                const int i = pi[k], j = pj[k];
                const T ai = A[l * ld + i], aj = A[l * ld + j];
                A[l * ld + i] = c * ai - s * aj;
                A[l * ld + j] = s * ai + c * aj;
                const T vi = V[l * ld + i], vj = V[l * ld + j];
                V[l * ld + i] = c * vi - s * vj;
                V[l * ld + j] = s * vi + c * vj;
            }
            __syncthreads();
            // rows: A <- J^T A
            for (int e = tid; e < (p2 / 2) * p2; e += nt) {
                const int k = e / p2, l = e % p2;
                const T c = cs[k], s = sn[k];
                if (s == (T)0) continue;
                const int i = pi[k], j = pj[k];
                const T ai = A[i * ld + l], aj = A[j * ld + l];
                A[i * ld + l] = c * ai - s * aj;
                A[j * ld + l] = s * ai + c * aj;
            }
            __syncthreads();
            for (int k = tid; k < p2 / 2; k += nt) {
                if (sn[k] != (T)0) {
                    A[pi[k] * ld + pj[k]] = (T)0;
                    A[pj[k] * ld + pi[k]] = (T)0;
                }
            }
            __syncthreads();
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

}  // namespace

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
    gram_kernel<<<nb, 256, smem, s>>>(A, rows, rs, cs, p, p4, scratch);
    LRA_LAUNCHED();
    gram_reduce_kernel<<<(unsigned)ceil_div(p * p, 256), 256, 0, s>>>(scratch, nb, p, p4, G);
    LRA_LAUNCHED();
}

void chol_inv(cudaStream_t s, const double *G, int p, float *Rinv, int *status) {
    const size_t smem = sizeof(double) * 2 * p * (p + 1);
    LRA_CUDA(cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    chol_inv_kernel<<<1, 256, smem, s>>>(G, p, Rinv, status);
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
void sym_eig(cudaStream_t s, const double *H, int p, double *evals, double *evecs, double *work) {
    const int p2 = p + (p & 1);
    const size_t pp = (size_t)p * p;
    double *V = work;           // p*p
    double *rho = work + pp;    // p
    double *T1 = evecs;         // scratch until the final sort (p*p)
    double *T2 = work + pp + p;  // p*p
    double *V2 = T2 + pp;       // p*p
    const size_t smem = sizeof(float) * (2 * p2 * (p2 + 1) + p2) + sizeof(int) * p2;
    LRA_CUDA(cudaFuncSetAttribute(jacobi_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    jacobi_kernel<float><<<1, 512, smem, s>>>(H, p, V, 40);
    LRA_LAUNCHED();
    auto gemm = [&](const double *A, const double *B, int ta, double alpha, double beta, double *C) {
        gemm_pp_kernel<<<p, 128, 0, s>>>(A, B, p, ta, alpha, beta, C);
        LRA_LAUNCHED();
    };
    auto orthonormalise = [&](double *Vin, double *Vout) {
        gemm(Vin, Vin, 1, -0.5, 1.5, T1);   // T1 = 1.5 I - 0.5 V^T V
        gemm(Vin, T1, 0, 1.0, 0.0, Vout);   // Vout = V T1
    };
    for (int pass = 0; pass < 2; ++pass) {  // each pass squares the off-diagonal
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
