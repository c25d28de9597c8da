// Launch wrappers of the CUDA kernels (one translation unit per family).
// All matrices follow the library's internal layouts:
//   X            : storage dtype, column-major, leading dimension ldx = dpad
//                  (rows d..dpad-1 are zero), n columns.
//   d x p blocks : FP32 column-major, leading dimension dpad, rows >= d zero.
//   packed (rm)  : FP32 row-major with PP = pad_p(p) columns, zero padded.
#pragma once

#include "common.cuh"

namespace lra {

// ---- setup (k_setup.cu) ---------------------------------------------------
void colnorms(cudaStream_t s, const void *X, lra_dtype dt, int64_t ldx, int64_t d, int64_t n,
              double *norm2, double xscale = 1.0);
// FP16 storage: the power of two that puts max |x| of X32 (count entries) in
// [2^14, 2^15) (scratch: one device word; synchronises s), and X16 = fp16(xscale X32)
float f16_storage_scale(cudaStream_t s, const float *X32, int64_t count, unsigned *scratch);
void to_f16(cudaStream_t s, const float *X32, int64_t count, float xscale, __half *Xs);
// out[0] = sum_i v_i (fixed-order), out[1] = max_i v_i; scratch >= 2 * 1024 doubles
void sum_max(cudaStream_t s, const double *v, int64_t n, double *out, double *scratch);
// Integer weights, their inclusive prefix sums (cum), c_i = total / w_i and
// kappa = max_i (total / w_i) norm2_i.  scratch: >= ceil(n/1024) + 2048 uint64.
void sampling_table(cudaStream_t s, const double *norm2, int64_t n, int mode, const double *maxn,
                    uint64_t *cum, float *c, double *kappa_out, uint64_t *scratch);
// idx[t] = first i with cum[i] > mulhi(u_t, total); cval[t] = c[idx[t]] if cval
void sample(cudaStream_t s, const uint64_t *cum, int64_t n, uint64_t key, int64_t m, int32_t *idx,
            const float *c, float *cval);
// cval[t] = c[idx[t]]; bad[0] = 1 if an index is outside [0, n)
void gather_c(cudaStream_t s, const int32_t *idx, const float *c, int64_t m, int64_t n, float *cval,
              int *bad);
// Box-Muller N(0,1) block (dpad x p, rows >= d left zero)
void gaussian(cudaStream_t s, uint64_t key, int64_t d, int64_t dpad, int p, float *out);
// storage conversions (column-major, any ld -> dpad)
void convert_to_f32(cudaStream_t s, const void *src, lra_dtype sdt, int64_t ld, int64_t d,
                    int64_t ncols, float *dst, int64_t dpad);
void convert_to_bf16(cudaStream_t s, const void *src, lra_dtype sdt, int64_t ld, int64_t d,
                     int64_t ncols, __nv_bfloat16 *dst, int64_t dpad);

// ---- anchor pass (k_anchor.cu) --------------------------------------------
// Wr (dpad x PP row-major) <- W (dpad x p column-major, leading dim ldw)
void pack_rm(cudaStream_t s, const float *W, int64_t ldw, int64_t rows, int p, int PP, float *Wr);
// Y (n x PP row-major) = X^T Wr
void xtw(cudaStream_t s, const void *X, lra_dtype dt, int64_t ldx, int64_t dpad, int64_t n,
         const float *Wr, int PP, float *Y);
// partial G over column chunks: Gp[c] (dpad x PP row-major) = X[:, chunk c] Y[chunk c, :]
int xy_chunks(int64_t dpad, int64_t n, int rows_per_cta = 128);
void xy(cudaStream_t s, const void *X, lra_dtype dt, int64_t ldx, int64_t dpad, int64_t n,
        const float *Y, int PP, float *Gp, int nchunks);
// M = lambda Wt - sum_c Gp[c] - B (dpad x p column-major); if norms: norms[0] =
// ||M||_F^2, norms[1] = ||B||_F^2 (FP64).  If M == nullptr: G = sum_c Gp[c] is
// written to G (dpad x p) instead.  scratch >= 2 * (dpad/32) doubles.
// (Z != nullptr: M = lam Wt - G - (B + gamma Z) and norms[2] = ||(lam - gamma) Wt - G - B||^2;
// scratch then holds 3 doubles per 16 rows)
void anchor_epilogue(cudaStream_t s, const float *Gp, int nchunks, int64_t dpad, int PP, int p,
                     double lam, const float *Wt, const float *B, float *M, double *norms,
                     double *scratch, const float *Z = nullptr, double gamma = 0.0,
                     const float *colscale = nullptr);

// ---- anchor pass on tensor cores, BF16 X (k_anchor_tc.cu) ---------------
// leading dimension of the hi/lo BF16 copy of Y (n rounded up to 64)
int64_t tc_ldy(int64_t n);
// rows of X per CTA of the tensor-core passes (256 = two M tiles sharing the
// small operand: BF16 X with PP >= 64; else 128)
int tc_rows_per_cta(int PP, bool pair);
// Wb = [hi; lo] BF16 split of W (rows x p column-major, leading dim ld), each
// PP x rows column-major (zero for columns >= p)
void pack_hilo(cudaStream_t s, const float *W, int64_t ld, int64_t rows, int p, int PP, __nv_bfloat16 *Wb);
// Yb = [hi; lo] BF16 split of Y (n x PP row-major), each PP x ldy column-major
void y_hilo(cudaStream_t s, const float *Y, int64_t n, int PP, __nv_bfloat16 *Yb, int64_t ldy);
// FP32 X -> BF16 pair (x = hi + lo + r, |r| <= 2^-17 |x|), count elements
void split_hilo(cudaStream_t s, const float *X, int64_t count, __nv_bfloat16 *Xh, __nv_bfloat16 *Xl);
// Y = X^T W on tcgen05: writes Y32 (n x PP row-major) and/or Yb (hi/lo) when
// non-null.  X is BF16 (Xl == nullptr) or the BF16 pair (X, Xl) of an FP32 X.
void xtw_tc(cudaStream_t s, const void *X, const void *Xl, int64_t dpad, int64_t n, const void *Wb, int PP,
            float *Y32, void *Yb, int64_t ldy, int *err, long long wait_cycles = 0, bool f16 = false,
            const float *tcs = nullptr);
// partial G = X Y per column chunk on tcgen05 (same Gp layout as xy); with
// FP16 operands column c of each partial carries the factor xscale sy_c
void xy_tc(cudaStream_t s, const void *X, const void *Xl, int64_t dpad, int64_t n, const void *Yb, int64_t ldy,
           int PP, float *Gp, int nchunks, int *err, long long wait_cycles = 0, bool f16 = false);
// FP16 operands (FP16 storage): scales into tcs (2 + 2 PP floats: see the
// tensor-core kernels) and the FP16 hi / lo small operand
void pack_hilo_f16(cudaStream_t s, const float *W, int64_t ld, int64_t rows, int p, int PP, float xscale,
                   double xmaxnorm, float *tcs, __half *Wb);
void y_hilo_f16(cudaStream_t s, const float *Y, int64_t n, int PP, int p, float xscale, float *tcs, __half *Yb,
                int64_t ldy);

// ---- SVRG inner loop (k_inner.cu) -----------------------------------------
// m steps of `batch` samples each (idx, cval: m * batch entries); batch a power of two <= 16
void svrg_inner(cudaStream_t s, const void *X, lra_dtype dt, int64_t ldx, int64_t dpad, int p,
                float *W, const float *Wt, const float *M, const int32_t *idx, const float *cval,
                int64_t m, float eta, float lam, int batch = 1, float cscale = 1.0f);

// ---- p x p and d x p helpers (k_small.cu) -------------------------------
// G (p x p FP64, column-major) = A^T A, A rows x p with strides (rs, cs).
// scratch >= gram_scratch(p) doubles
int64_t gram_scratch(int p);
void gram(cudaStream_t s, const float *A, int64_t rows, int64_t rs, int64_t cs, int p, double *G,
          double *scratch);
// G = A^T A with every product accumulated in FP64; A column-major rows x p
// (leading dimension ld), read as FP32 A, as the BF16 pair Ah + Al when
// Ah != nullptr, or as the BF16 pair of A (round-to-nearest hi, then lo of the
// remainder) when split.  scratch >= gram_scratch(p) doubles
void gram64(cudaStream_t s, const float *A, const __nv_bfloat16 *Ah, const __nv_bfloat16 *Al, int64_t rows,
            int64_t ld, int p, double *G, double *scratch, bool split = false);
// H = (A^T B + B^T A)/2 (FP64, p x p column-major) for A, B rows x p column-major
// (leading dim ld; A read as the BF16 pair Ah + Al when Ah != nullptr).
// scratch >= gram_scratch(p) doubles
void cross_gram(cudaStream_t s, const float *A, const __nv_bfloat16 *Ah, const __nv_bfloat16 *Al, const float *B,
                int64_t rows, int64_t ld, int p, double *H, double *scratch);
// out (p x p FP64 column-major) = A^T B for A, B rows x p column-major (leading dim ld)
void cross_full(cudaStream_t s, const float *A, const float *B, int64_t rows, int64_t ld, int p, double *out,
                double *scratch);
// Hc = 2H - (G H + H G)/2: Rayleigh-Ritz matrix of the orthonormalised basis
// to first order in G - I (all p x p FP64 column-major, symmetric)
void ortho_correct(cudaStream_t s, const double *H, const double *G, int p, double *Hc);
// Cholesky G = R^T R in FP64 (one barrier per column); R upper FP32 row-major
// near_id > 0: when ||G - I||_F <= near_id, R is the first-order factor
// I + triu(G - I, 1) + diag(G - I) / 2 (error below near_id^2) instead
void chol(cudaStream_t s, const double *G, int p, float *R, int *status, double near_id = 0.0);
// Q = W R^-1 by row-wise forward substitution (W, Q rows x p column-major)
void trsm_rows(cudaStream_t s, const float *W, int64_t rows, int64_t ld, int p, const float *R, float *Q);
// Out (rows x q) = A (rows x p) T (p x q, FP32 row-major); strides for A and Out
void apply_right(cudaStream_t s, const float *A, int64_t rows, int64_t ars, int64_t acs, int p,
                 const float *T, int q, float *Out, int64_t ors, int64_t ocs);
// Symmetric eigendecomposition of H (p x p FP64 column-major); evals desc,
// evecs column-major FP64 (largest |entry| positive).  work >= sym_eig_work(p) doubles.
int64_t sym_eig_work(int p);
// passes: FP64 refinement passes after the FP32 sweeps (each squares the residual rotation)
// jacobi_tol: the FP32 sweeps stop once the squared off-diagonal mass is below
// jacobi_tol times the total (1e-10 by default; the refinement squares what is left)
void sym_eig(cudaStream_t s, const double *H, int p, double *evals, double *evecs, double *work, int passes = 2,
             double jacobi_tol = 1e-10);
// P (p x p FP32 row-major) = V_k diag(f(rho)) V_k^T with f = 1/(lam - rho):
// the Galerkin inverse (lam I - H)^-1 on the Ritz basis.  kcols = p.
void ritz_inverse(cudaStream_t s, const double *evecs, const double *evals, int p, double lam,
                  float *P);
// P (p x p FP32 row-major) = V diag(1/(lam - rho))
void ritz_scaled(cudaStream_t s, const double *evecs, const double *evals, int p, double lam, float *P);
// dst[:, j] = src[:, j] / (lam - rho[j]) (rows x p column-major, leading dim ld)
void shift_scale_cols(cudaStream_t s, const float *src, float *dst, int64_t rows, int64_t ld, int p,
                      const double *evals, double lam);
// T (p x k FP32 row-major) = first k columns of evecs
void evecs_to_rm(cudaStream_t s, const double *evecs, int p, int k, float *T);
// out[j] = sum_r A[r, j] B[r, j] (FP64) for j < p (column-major, leading dim ld)
void col_dots(cudaStream_t s, const float *A, const float *B, int64_t rows, int64_t ld, int p,
              double *out);
// A[:, j] *= 1/sqrt(n2[j])  (n2 device FP64)
void scale_cols_rsqrt(cudaStream_t s, float *A, int64_t rows, int64_t ld, int p, const double *n2);
// A = alpha * A (all rows x p)
void scale_block(cudaStream_t s, float *A, int64_t rows, int64_t ld, int p, float alpha);
void acc_extrapolate(cudaStream_t s, const float *W, float *Wold, float *Z, int64_t rows, int64_t ld, int p,
                     float beta, bool first);

// ---- sparse X (k_sparse.cu) -----------------------------------------------
// Segment length of the row work list of X Y (rows longer than this are split).
constexpr int kSparseSeg = 1024;
// bad[0] |= 1 rowptr out of order/range, 2 column out of [0, n), 4 columns not
// strictly increasing in a row, 8 value not finite, 16 rowptr[0]/rowptr[d] wrong
void csr_check(cudaStream_t s, const int64_t *rowptr, const int32_t *colidx, const float *val, int64_t d,
               int64_t n, int64_t nnz, int *bad);
// int64 scratch of an exclusive scan over N entries
int64_t sparse_scan_scratch(int64_t N);
// compressed columns (colptr[n+1], rowidx, cval) of a valid CSR, rows sorted
// within each column; cnt: n int64, cursor: n int scratch
void csr_transpose(cudaStream_t s, const int64_t *rowptr, const int32_t *colidx, const float *val, int64_t d,
                   int64_t n, int64_t nnz, int64_t *colptr, int32_t *rowidx, float *cval, int64_t *cnt,
                   int *cursor, int64_t *scan_scratch);
// item_off[dpad+1]: exclusive scan of the segment counts (nseg: dpad int64 scratch)
void sparse_row_items(cudaStream_t s, const int64_t *rowptr, int64_t d, int64_t dpad, int seg, int64_t *nseg,
                      int64_t *item_off, int64_t *scan_scratch);
void sparse_fill_items(cudaStream_t s, const int64_t *item_off, int64_t dpad, int2 *items);
void sparse_colnorms(cudaStream_t s, const int64_t *colptr, const float *cval, int64_t n, double *norm2);
// Y (n x PP row-major) = X^T Wr (Wr dpad x PP row-major, columns >= p zero)
void spmm_xt(cudaStream_t s, const int64_t *colptr, const int32_t *rowidx, const float *cval, int64_t n,
             int64_t d, const float *Wr, int PP, int p, float *Y);
// G (dpad x PP row-major) = X Y (Y columns >= p zero); partial >= nitems x PP floats
void spmm_x(cudaStream_t s, const int64_t *rowptr, const int32_t *colidx, const float *val, int64_t d,
            int64_t dpad, const int64_t *item_off, const int2 *items, int64_t nitems, int seg, const float *Y,
            int PP, int p, float *G, float *partial);
// Deflated columns x'_i = x_i - U g_i of the sparse inner loop: U dpad x c
// column-major (orthonormal), Gt n x PPc row-major with g_i in row i, scratch
// >= 3 c PP floats.
struct InnerDefl {
    const float *U = nullptr;
    int c = 0;
    const float *Gt = nullptr;
    int PPc = 0;
    float *scratch = nullptr;
};
// m inner steps in factored form: W (dpad x p col-major) from W = Wt + (W - Wt);
// Mr = M packed dpad x PP row-major; Z: dpad x PP scratch; ab: 2 doubles.
// defl != nullptr: the steps of the deflated matrix (I - U U^T) X
void svrg_inner_csc(cudaStream_t s, const int64_t *colptr, const int32_t *rowidx, const float *cval, int64_t dpad,
                    int p, int PP, float *W, const float *Wt, const float *Mr, float *Z, double *ab,
                    const int32_t *idx, const float *cvals, int64_t m, double eta, double lam, int batch = 1,
                    const InnerDefl *defl = nullptr);

// ---- deflation applied on the fly (k_deflate.cu) -------------------------
// C (c x p; row a at C + a ldc) = U^T V for U rows x c column-major (leading
// dim ldu) and V[r rs + j cs]; FP32 products summed in FP64
void defl_coef(cudaStream_t s, const float *U, int64_t ldu, int c, const float *V, int64_t rs, int64_t cs,
               int64_t rows, int p, float *C, int ldc);
// V <- V - U (U^T V) for V rows x p column-major (leading dim ldv); C: c x p scratch
void defl_project(cudaStream_t s, const float *U, int64_t ldu, int c, float *V, int64_t ldv, int64_t rows, int p,
                  float *C);
// out[i] = max(0, norm2[i] - sum_{a < c} Gt[i PPc + a]^2)
void defl_norms(cudaStream_t s, const double *norm2, const float *Gt, int PPc, int c, int64_t n, double *out);
// out[:, t] = X[:, idx[t]] - U g_{idx[t]} for t < m (X FP32 dpad x n column-major
// with leading dim ldx, U dpad x c, out FP32 dpad x m column-major)
void defl_gather(cudaStream_t s, const float *X, int64_t ldx, int64_t dpad, const int32_t *idx, int64_t m,
                 const float *U, int c, const float *Gt, int PPc, float *out);
// the same for a sparse X given by its compressed columns
void defl_gather_csc(cudaStream_t s, const int64_t *colptr, const int32_t *rowidx, const float *cval, int64_t dpad,
                     const int32_t *idx, int64_t m, const float *U, int c, const float *Gt, int PPc, float *out);

}  // namespace lra
