/*
 * FP64 oracle: the SVRG inner loop, written as plain loops.
 *
 * TEST INFRASTRUCTURE ONLY.  Called (through ctypes) by oracle/lra_oracle.py,
 * which is itself used only by the tests, the smoke check and the CPU baseline
 * of the benchmark.  The library never links or calls this file.
 *
 * What it computes (Sec. 2.3 of the paper, SVRGsolve after Theorem 3): the
 * linear system (lambda I - X X^T) W = B is the minimiser of
 *     F(W) = 1/2 tr(W^T (lambda I - X X^T) W) - tr(B^T W)
 *          = sum_i q_i f_i(W),  f_i(W) = 1/2 tr(W^T (lambda I - c_i x_i x_i^T) W) - tr(B^T W),
 * with sampling probabilities q_i and c_i = 1/q_i.  Given the anchor Wt and the
 * anchor gradient M = grad F(Wt) = lambda Wt - X X^T Wt - B, one variance-reduced
 * step with sampled column i is
 *     r = x_i^T (W - Wt)                                   (1 x p)
 *     W <- W - eta [ lambda (W - Wt) - c_i x_i r + M ]
 * i.e. grad f_i(W) - grad f_i(Wt) + grad F(Wt).  With a batch of b samples per
 * step (b = 1 above) the stochastic term is the average of the b terms, each
 * r taken at the same W.  The p columns of W are independent chains that share
 * the sampled index sequence.
 *
 * X is read exactly as stored (FP64, or FP32 widened element by element).
 * Matrices are column-major: X is d x n with leading dimension ldx, W/Wt/M are
 * d x p with leading dimension d.
 */
#include <stdint.h>
#include <stdlib.h>

static void inner_loop(int64_t d, int64_t p, const double *Xd, const float *Xf, int64_t ldx,
                       const int64_t *idx, int64_t m, int64_t batch, const double *c, double eta,
                       double lam, const double *Wt, const double *M, double *W)
{
    /* step t uses the batch idx[t b], ..., idx[t b + b - 1]; every r_u is taken
       at the same W, and the stochastic term is their average */
    double *r = (double *)malloc(sizeof(double) * (size_t)(p * batch > 0 ? p * batch : 1));
    const double invb = 1.0 / (double)batch;
    for (int64_t t = 0; t < m; ++t) {
        /* r_{u,j} = x_{i_u}^T (W_j - Wt_j) */
        for (int64_t u = 0; u < batch; ++u) {
            const int64_t i = idx[t * batch + u];
            for (int64_t j = 0; j < p; ++j) {
                double acc = 0.0;
                for (int64_t row = 0; row < d; ++row) {
                    const double x = Xd ? Xd[i * ldx + row] : (double)Xf[i * ldx + row];
                    acc += x * (W[j * d + row] - Wt[j * d + row]);
                }
                r[u * p + j] = acc;
            }
        }
        /* W_j <- W_j - eta [ lambda (W_j - Wt_j) - (1/b) sum_u c_{i_u} x_{i_u} r_{u,j} + M_j ] */
        for (int64_t j = 0; j < p; ++j) {
            for (int64_t row = 0; row < d; ++row) {
                double sg = 0.0;
                for (int64_t u = 0; u < batch; ++u) {
                    const int64_t i = idx[t * batch + u];
                    const double x = Xd ? Xd[i * ldx + row] : (double)Xf[i * ldx + row];
                    sg += c[i] * x * r[u * p + j];
                }
                const double diff = W[j * d + row] - Wt[j * d + row];
                const double g = lam * diff - invb * sg + M[j * d + row];
                W[j * d + row] -= eta * g;
            }
        }
    }
    free(r);
}

void oracle_svrg_inner_f64(int64_t d, int64_t p, const double *X, int64_t ldx,
                           const int64_t *idx, int64_t m, int64_t batch, const double *c, double eta,
                           double lam, const double *Wt, const double *M, double *W)
{
    inner_loop(d, p, X, NULL, ldx, idx, m, batch, c, eta, lam, Wt, M, W);
}

void oracle_svrg_inner_f32(int64_t d, int64_t p, const float *X, int64_t ldx,
                           const int64_t *idx, int64_t m, int64_t batch, const double *c, double eta,
                           double lam, const double *Wt, const double *M, double *W)
{
    inner_loop(d, p, NULL, X, ldx, idx, m, batch, c, eta, lam, Wt, M, W);
}

/*
 * The same epoch (batch b as above) for a sparse X given by its columns x_i in compressed form
 * (colptr[n+1], rowidx[nnz], val[nnz] FP32: column i holds val[k] at row
 * rowidx[k] for colptr[i] <= k < colptr[i+1]).
 *
 * A step touches only the rows of x_i once W - Wt is kept in the factored form
 *     W - Wt = a Z + b M,
 * which the dense step maps to itself (with g = 1 - eta lambda):
 *     W' - Wt = g (a Z + b M) + eta c_i x_i r - eta M
 *             = a' (Z + (eta c_i / a') x_i r) + b' M,   a' = g a,  b' = g b - eta,
 * and r = x_i^T (W - Wt) = a (x_i^T Z) + b (x_i^T M).  Start: Z = W - Wt, a = 1,
 * b = 0.  When a falls below 2^-30 the factor is folded into Z (Z <- a Z,
 * a <- 1).  End: W = Wt + a Z + b M.
 */
void oracle_svrg_inner_csc(int64_t d, int64_t p, const int64_t *colptr, const int32_t *rowidx,
                           const float *val, const int64_t *idx, int64_t m, int64_t batch, const double *c,
                           double eta, double lam, const double *Wt, const double *M, double *W)
{
    double *Z = (double *)malloc(sizeof(double) * (size_t)(d * p > 0 ? d * p : 1));
    double *r = (double *)malloc(sizeof(double) * (size_t)(p * batch > 0 ? p * batch : 1));
    const double g = 1.0 - eta * lam;
    double a = 1.0, b = 0.0;
    for (int64_t e = 0; e < d * p; ++e) Z[e] = W[e] - Wt[e];
    for (int64_t t = 0; t < m; ++t) {
        for (int64_t u = 0; u < batch; ++u) {
            const int64_t i = idx[t * batch + u];
            const int64_t k0 = colptr[i], k1 = colptr[i + 1];
            for (int64_t j = 0; j < p; ++j) {
                double sz = 0.0, sm = 0.0;
                for (int64_t k = k0; k < k1; ++k) {
                    const int64_t row = rowidx[k];
                    sz += (double)val[k] * Z[j * d + row];
                    sm += (double)val[k] * M[j * d + row];
                }
                r[u * p + j] = a * sz + b * sm;
            }
        }
        const double a1 = g * a;
        b = g * b - eta;
        for (int64_t u = 0; u < batch; ++u) {
            const int64_t i = idx[t * batch + u];
            const int64_t k0 = colptr[i], k1 = colptr[i + 1];
            const double s = eta * c[i] / (a1 * (double)batch);
            for (int64_t j = 0; j < p; ++j)
                for (int64_t k = k0; k < k1; ++k) Z[j * d + rowidx[k]] += s * (double)val[k] * r[u * p + j];
        }
        a = a1;
        if (a < 0x1p-30) {
            for (int64_t e = 0; e < d * p; ++e) Z[e] *= a;
            a = 1.0;
        }
    }
    for (int64_t e = 0; e < d * p; ++e) W[e] = Wt[e] + a * Z[e] + b * M[e];
    free(Z);
    free(r);
}
