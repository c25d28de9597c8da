// Algorithm 6 with adaptive partitioning of {1..k} and deflation (Sec. 3:
// Algorithms 3, 4, 5, 6, 7).  Stage t, starting at index s with the columns
// u_1..u_{s-1} found so far, works on the deflated matrix
// X_{-(s-1)} = (I - U U^T) X (Sec. 3 assumes the projection applied to X's
// columns).  It is applied on the fly: the stage's Engine projects the small
// operand before each X^T pass and the d x p result after each X pass, draws
// samples by the deflated column norms ||x_i||^2 - ||U^T x_i||^2, and steps on
// the deflated columns x_i - U (U^T x_i); no d x n copy is made.  Each stage
// runs the same kernels as the q = k path:
//   Algorithm 3 on A_{-(s-1)} (k - s + 1 vectors, eps' = 1/(9 p^2));
//   Algorithm 4: the first multiplicative gap -> Algorithm 1 on A_{-(s-1)}
//   with q - s + 1 columns; otherwise Algorithm 7 (the shift), Algorithm 3 on
//   D_{-(s-1)} = (lam I - A_{-(s-1)})^{-1} (eps' = 1/(9p)), Algorithm 5 (the
//   first additive gap >= 5 Delta / 9, else k) and Algorithm 1 on D_{-(s-1)}
//   with p' = q - s + 1 columns (q < k) or p - (s - 1) (q = k, oversampled);
//   s = q + 1.
// The columns are orthonormalised together (CholeskyQR2) and Algorithm 2 with
// X X^T on the exact FP32 values returns U.
#include <chrono>
#include <cstring>
#include <memory>
#include <vector>

#include "engine.h"

namespace lra {

namespace {

// Algorithm 4: offset j of the first q = s + j in I \ {k} with
// lam_hat[j + 1] <= lam_hat[j] (1 - p^-2), or -1
int alg4(const double *lam_hat, int kk, int p) {
    for (int j = 0; j + 1 < kk; ++j)
        if (lam_hat[j + 1] <= lam_hat[j] * (1.0 - 1.0 / ((double)p * p))) return j;
    return -1;
}

// Algorithm 5: offset of the first q in I \ {k} with inv[j + 1] - inv[j] >=
// 5 Delta / 9 (inv = estimates of lam - lambda_i), else kk - 1 (q = k)
int alg5(const double *inv, int kk, double delta) {
    for (int j = 0; j + 1 < kk; ++j)
        if (inv[j + 1] - inv[j] >= 5.0 * delta / 9.0) return j;
    return kk - 1;
}

}  // namespace

lra_status solve_partitioned(lra_mat *mat, int k, int p, double eps, uint64_t seed, const Opts &o, float *U_out,
                             double *ritz_out, lra_report *rep) {
    const auto t_all = std::chrono::steady_clock::now();
    const int64_t launches0 = launches_of_thread();
    lra_ctx *ctx = mat->ctx;
    cudaStream_t s = ctx->stream;
    const int64_t d = mat->d, dpad = mat->dpad, n = mat->n;
    lra_report R;
    std::memset(&R, 0, sizeof(R));
    R.struct_size = sizeof(R);

    // the original matrix's workspace: Delta, the columns found, the deflation
    // products and the final Rayleigh-Ritz step
    Workspace ws0(ctx, dpad, n, p + 1, nullptr, ws_items(mat));
    Engine e0(mat, ws0, s);
    std::unique_ptr<KernelTimer> timer;
    if (o.profile) {
        timer.reset(new KernelTimer(s));
        e0.timer = timer.get();
    }
    e0.ensure_table(o.sampling);
    R.fro2 = mat->fro2;
    double delta = o.delta;
    if (!(delta > 0)) {
        const lra_status st = e0.delta_estimate(k, p, seed, delta);
        if (st != LRA_OK) return st;
    }
    R.delta = delta;
    struct Buf {  // device buffer released on every exit path
        lra_ctx *c;
        size_t b;
        void *p;
        Buf(lra_ctx *c_, size_t b_) : c(c_), b(b_), p(dev_alloc(c_, b_)) {}
        ~Buf() { dev_free(c, p, b); }
    };
    Buf ubuf(ctx, sizeof(float) * dpad * p);
    float *Ucols = static_cast<float *>(ubuf.p);
    LRA_CUDA(cudaMemsetAsync(Ucols, 0, sizeof(float) * dpad * p, s));

    // the deflation view of the stages after the first: U^T x_i (in ws0.Y, n x
    // pad_p(c)), the deflated norms and sampling tables, projection scratch,
    // and the inner loop's deflated columns in chunks of up to 256 MB (dense X,
    // and CSR X up to d = 8192, where the dense steps are faster than the
    // factored ones; larger CSR X steps in factored form)
    const int PPp = pad_p(p);
    const int64_t mcap =
        (mat->sp && dpad > 8192)
            ? 0
            : std::max<int64_t>(64, std::min<int64_t>(65536, (int64_t)((256ull << 20) / (sizeof(float) * dpad))));
    Buf bn(ctx, sizeof(double) * n), bsm(ctx, sizeof(double) * 4), bV(ctx, sizeof(float) * dpad * p),
        bC(ctx, sizeof(float) * (size_t)p * p), bG0(ctx, sizeof(float) * dpad * PPp),
        bcum0(ctx, sizeof(uint64_t) * n), bc0(ctx, sizeof(float) * n), bcum1(ctx, sizeof(uint64_t) * n),
        bc1(ctx, sizeof(float) * n), bcols(ctx, sizeof(float) * dpad * std::max<int64_t>(mcap, 1)),
        biota(ctx, sizeof(int32_t) * std::max<int64_t>(mcap, 1)), blk(ctx, sizeof(float) * 3 * (size_t)p * PPp);
    Deflation D;
    D.U = Ucols;
    D.Gt = ws0.Y;
    D.norm2 = static_cast<double *>(bn.p);
    D.sm = static_cast<double *>(bsm.p);
    D.V = static_cast<float *>(bV.p);
    D.C = static_cast<float *>(bC.p);
    D.G0 = static_cast<float *>(bG0.p);
    D.table[0].cum = static_cast<uint64_t *>(bcum0.p);
    D.table[0].c = static_cast<float *>(bc0.p);
    D.table[1].cum = static_cast<uint64_t *>(bcum1.p);
    D.table[1].c = static_cast<float *>(bc1.p);
    D.cols = static_cast<float *>(bcols.p);
    D.mcap = mcap;
    D.iota = static_cast<int32_t *>(biota.p);
    D.lk = static_cast<float *>(blk.p);
    if (mcap > 0) {
        std::vector<int32_t> iota((size_t)mcap);
        for (int64_t i = 0; i < mcap; ++i) iota[(size_t)i] = (int32_t)i;
        LRA_CUDA(cudaMemcpyAsync(D.iota, iota.data(), sizeof(int32_t) * mcap, cudaMemcpyHostToDevice, s));
        LRA_CUDA(cudaStreamSynchronize(s));
    }

    lra_status status = LRA_OK;
    int s_idx = 1, t = 0, ncols = 0;
    std::vector<double> lam_hat(k + 1), theta(k + 1), inv(k + 1);
    while (s_idx <= k) {
        ++t;
        const uint64_t seed_t = stream_key(seed, LRA_STREAM_PART, (uint64_t)t, 0);
        const int kk = k - s_idx + 1;
        if (s_idx > 1) {
            // g_i = U^T x_i from the exact FP32 values, then the deflated norms
            D.c = ncols;
            D.PPc = pad_p(ncols);
            e0.xt_mul(Ucols, ncols, ws0.Y, true);
            defl_norms(s, mat->norm2, D.Gt, D.PPc, D.c, n, D.norm2);
            sum_max(s, D.norm2, n, D.sm, nullptr);
            double h[2];
            LRA_CUDA(cudaMemcpyAsync(h, D.sm, sizeof(h), cudaMemcpyDeviceToHost, s));
            LRA_CUDA(cudaStreamSynchronize(s));
            D.fro2 = h[0];
            D.maxn = h[1];
            D.table[0].ok = D.table[1].ok = false;
        }
        Workspace ws(ctx, dpad, n, p, nullptr, ws_items(mat));
        Engine e(mat, ws, s);
        e.timer = timer.get();
        if (s_idx > 1) e.defl = &D;
        e.ensure_table(o.sampling);
        int it3 = 0;
        lra_status st = e.alg3_a(kk, 1.0 / (9.0 * p * p), o.part_max_iters, seed_t, lam_hat.data(), it3);
        if (st != LRA_OK) return st;
        const int j = alg4(lam_hat.data(), kk, p);
        int q, keep, iters = 0, kind;
        lra_status bst = LRA_OK;
        const float *cols = nullptr;
        if (j >= 0) {
            kind = 1;
            q = s_idx + j;
            keep = j + 1;
            const double rf = (lam_hat[j + 1] / lam_hat[j]) * (lam_hat[j + 1] / lam_hat[j]);
            st = e.power_block(keep, eps, rf, seed_t, o, iters, bst);
            if (st != LRA_OK) return st;
            cols = ws.U;
        } else {
            kind = 2;
            int64_t solve_count = 0;
            const double l1hat = e.lambda1_estimate(seed_t);
            const double l1up = l1hat / (1.0 - 0.25);
            double lam = 0, inv1 = 0, mu = 0;
            int rounds = 0;
            st = e.shift_tune(seed_t, l1hat, delta, o, solve_count, lam, inv1, mu, rounds, nullptr);
            if (st == LRA_EDIVERGED) return st;
            int itd = 0;
            st = e.alg3_d(kk, 1.0 / (9.0 * p), o.part_max_iters, seed_t, lam, mu, l1up, l1hat, o, solve_count,
                          theta.data(), itd);
            if (st != LRA_OK) return st;
            for (int i = 0; i < kk; ++i) inv[i] = 1.0 / theta[i];
            const int jj = alg5(inv.data(), kk, delta);
            q = s_idx + jj;
            const int pp = q == k ? p - (s_idx - 1) : q - s_idx + 1;
            keep = q == k ? pp : q - s_idx + 1;
            // rate floor of a block without oversampling, from Algorithm 3 on D
            const double rf = q == k ? -1.0 : (inv[jj] / inv[jj + 1]) * (inv[jj] / inv[jj + 1]);
            float *S = nullptr;
            std::vector<double> E;
            st = e.loop_d(q - s_idx + 1, pp, eps, seed_t, lam, mu, l1up, o, solve_count, rf, S, iters, E, bst, R,
                          nullptr);
            if (st != LRA_OK) return st;
            // Ritz vectors S V[:, :keep] into ws.U
            evecs_to_rm(s, ws.evecs, pp, keep, ws.P);
            apply_right(s, S, dpad, 1, dpad, pp, ws.P, keep, ws.U, 1, dpad);
            cols = ws.U;
            R.shift_rounds += rounds;
            R.lambda = lam;
            R.mu_lb = mu;
        }
        if (bst != LRA_OK) status = bst;
        R.outer_iters += iters;
        R.solves += e.stats.solves;
        R.epochs += e.stats.epochs;
        R.inner_steps += e.stats.inner_steps;
        R.x_passes += e.stats.x_passes;
        if (t <= LRA_MAX_P) {
            R.part_q[t - 1] = q;
            R.part_kind[t - 1] = kind;
        }
        R.part_stages = t;
        // append and orthonormalise all columns found so far
        LRA_CUDA(cudaMemcpyAsync(Ucols + (size_t)ncols * dpad, cols, sizeof(float) * dpad * keep,
                                 cudaMemcpyDeviceToDevice, s));
        ncols += keep;
        st = e0.cholqr2(Ucols, ncols);
        if (st != LRA_OK) return st;
        s_idx = q + 1;
    }
    // Algorithm 2 with X X^T on the p columns (exact FP32 values of X)
    e0.ritz(Ucols, p, true);
    evecs_to_rm(s, ws0.evecs, p, k, ws0.P);
    apply_right(s, Ucols, dpad, 1, dpad, p, ws0.P, k, ws0.U, 1, dpad);
    LRA_CUDA(cudaMemcpy2DAsync(U_out, sizeof(float) * d, ws0.U, sizeof(float) * dpad, sizeof(float) * d, k,
                               cudaMemcpyDefault, s));
    LRA_CUDA(cudaMemcpyAsync(ritz_out, ws0.evals, sizeof(double) * k, cudaMemcpyDefault, s));
    LRA_CUDA(cudaMemcpyAsync(ws0.host, ws0.evals, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
    LRA_CUDA(cudaStreamSynchronize(s));
    double sk = 0.0;
    for (int j = 0; j < k; ++j) sk += ws0.host[j];
    R.err_est = mat->fro2 - sk;
    R.solves += e0.stats.solves;
    R.x_passes += e0.stats.x_passes;
    R.status = status;
    R.kernel_launches = launches_of_thread() - launches0;
    if (timer) {
        double ms[KernelTimer::NKIND];
        int64_t cnt[KernelTimer::NKIND], cols[KernelTimer::NKIND];
        timer->collect(ms, cnt, cols);
        for (int i = 0; i < KernelTimer::NKIND; ++i) R.phase_ms[i] = ms[i];
        R.xtw_ms = ms[0];
        R.xy_ms = ms[1];
        R.inner_ms = ms[2];
        R.xtw_launches = cnt[0];
        R.xy_launches = cnt[1];
        R.inner_launches = cnt[2];
        R.xtw_cols = cols[0];
        R.xy_cols = cols[1];
    }
    R.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_all).count();
    if (rep) {
        const size_t sz = std::min(rep->struct_size ? rep->struct_size : sizeof(R), sizeof(R));
        std::memcpy(rep, &R, sz);
        rep->struct_size = sz;
    }
    return status;
}

}  // namespace lra
