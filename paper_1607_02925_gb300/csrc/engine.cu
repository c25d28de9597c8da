// The method's steps on the device (q = k branch of Algorithm 6):
//   lambda_1 estimate (Algorithm 3, C = X X^T, k = 1), shift tuning
//   (Algorithm 7), subspace iteration (Algorithm 1) on (lambda I - X X^T)^-1
//   with SVRG solves (Sec. 2.3), CholeskyQR2, and Rayleigh-Ritz (Algorithm 2).
// Host code only sequences kernels and reads back the few scalars that drive
// control flow (residual norms, Ritz values).
#include <chrono>
#include <cstring>

#include "engine.h"

namespace lra {

void *dev_alloc(lra_ctx *ctx, size_t bytes, cudaStream_t s) {
    if (ctx->budget) {
        const size_t now = ctx->used.fetch_add(bytes) + bytes;
        if (now > ctx->budget) {
            ctx->used.fetch_sub(bytes);
            set_error("device memory budget exceeded");
            throw Error{LRA_ENOMEM};
        }
    } else {
        ctx->used.fetch_add(bytes);
    }
    void *p = nullptr;
    const cudaError_t e = s ? cudaMallocAsync(&p, bytes, s) : cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        ctx->used.fetch_sub(bytes);
        cudaGetLastError();
        set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
        throw Error{LRA_ENOMEM};
    }
    return p;
}

void dev_free(lra_ctx *ctx, void *p, size_t bytes, cudaStream_t s) {
    if (!p) return;
    if (s)
        cudaFreeAsync(p, s);
    else
        cudaFree(p);
    ctx->used.fetch_sub(bytes);
}

Opts read_opts(const lra_options *o, lra_dtype storage) {
    Opts r;
    if (o) {
        if (o->struct_size < sizeof(lra_options)) {
            set_error("lra_options.struct_size too small");
            throw Error{LRA_EINVAL};
        }
        r.shift_policy = o->shift_policy;
        r.lambda = o->lambda;
        r.delta = o->delta;
        r.theta_eta = o->theta_eta;
        r.theta_m = o->theta_m;
        r.tau = o->tau;
        r.max_epochs = o->max_epochs;
        r.m_max = o->m_max;
        r.min_outer = o->min_outer;
        r.max_outer = o->max_outer;
        r.fixed_epochs = o->fixed_epochs;
        r.sampling = o->sampling;
        r.warm_start = o->warm_start;
        r.max_shift_rounds = o->max_shift_rounds;
        r.lambda1_hat = o->lambda1_hat;
        r.trace_E = o->trace_E;
        r.trace_cap = o->trace_cap;
        r.profile = o->profile;
        r.batch = o->batch;
        r.acc = o->acc;
        r.acc_theta = o->acc_theta;
        r.acc_max_outer = o->acc_max_outer;
        r.acc_target = o->acc_target;
        r.partition = o->partition;
        r.part_max_iters = o->part_max_iters;
        r.wait_cycles = o->wait_cycles;
    }
    if (r.tau <= 0.0) r.tau = (storage == LRA_BF16) ? 1e-3 : (storage == LRA_F16 ? 1e-4 : 1e-5);
    if (r.shift_policy < 0 || r.shift_policy > 2 || r.theta_eta <= 0 || r.theta_m <= 0 ||
        r.max_epochs < 1 || r.max_outer < 0 || r.sampling < 0 || r.sampling > 1 || r.fixed_epochs < 0 ||
        r.max_shift_rounds < 1 || r.m_max < 0 || !(r.delta >= 0.0) || r.batch < 1 || r.batch > 16 ||
        (r.batch & (r.batch - 1)) != 0 || r.acc < 0 || r.acc > 1 || !(r.acc_theta > 0.0 && r.acc_theta <= 1.0) ||
        r.acc_max_outer < 1 || r.acc_target < 0 || r.partition < 0 || r.partition > 1 || r.part_max_iters < 1 ||
        r.wait_cycles < 0) {
        set_error("invalid lra_options field");
        throw Error{LRA_EINVAL};
    }
    return r;
}

// ---------------------------------------------------------------------------
// Workspace
// ---------------------------------------------------------------------------
size_t workspace_bytes(int64_t dpad, int64_t n, int pmax, int64_t sp_items) {
    const int PP = pad_p(pmax);
    const int nch = sp_items >= 0 ? 1 : std::max(xy_chunks(dpad, n, 128), xy_chunks(dpad, n, 256));
    size_t b = 0;
    b += 8 * sizeof(float) * dpad * pmax;       // S W Wt M T1 U, accelerated solve: Za Wo
    b += sizeof(float) * dpad * PP;             // Wr
    b += 2 * sizeof(float) * n * PP;            // Q Y
    b += sizeof(float) * (size_t)nch * dpad * PP;  // Gp
    b += sizeof(double) * (9 * pmax * pmax + gram_scratch(pmax) + dpad);
    b += sizeof(float) * (2 + 3 * (size_t)PP);  // scales of FP16 tensor-core operands
    if (sp_items >= 0)
        b += sizeof(float) * (size_t)sp_items * PP;                 // partial
    else
        b += 2 * sizeof(__nv_bfloat16) * PP * (dpad + tc_ldy(n));  // Wb Yb
    b += sizeof(double) * gram_scratch(pmax);  // side-stream Gram scratch
    return b;
}

Workspace::Workspace(lra_ctx *c, int64_t dpad_, int64_t n_, int pmax_, cudaStream_t alloc_stream,
                     int64_t sp_items_)
    : ctx(c), dpad(dpad_), n(n_), pmax(pmax_), PPmax(pad_p(pmax_)), sp_items(sp_items_), astream(alloc_stream) {
    auto zero = [&](void *p, size_t bytes) {
        if (astream)
            LRA_CUDA(cudaMemsetAsync(p, 0, bytes, astream));
        else
            LRA_CUDA(cudaMemset(p, 0, bytes));
    };
    try {
        const size_t blk = (size_t)dpad * pmax;
        S = alloc<float>(blk);
        W = alloc<float>(blk);
        Wt = alloc<float>(blk);
        M = alloc<float>(blk);
        T1 = alloc<float>(blk);
        U = alloc<float>(blk);
        Za = alloc<float>(blk);
        Wo = alloc<float>(blk);
        Wr = alloc<float>((size_t)dpad * PPmax);
        Q = alloc<float>((size_t)n * PPmax);
        Y = alloc<float>((size_t)n * PPmax);
        zero(Q, sizeof(float) * n * PPmax);
        zero(Y, sizeof(float) * n * PPmax);
        nchunks = sp_items >= 0 ? 1 : std::max(xy_chunks(dpad, n, 128), xy_chunks(dpad, n, 256));
        Gp = alloc<float>((size_t)nchunks * dpad * PPmax);
        const size_t pp = (size_t)pmax * pmax;
        H = alloc<double>(pp);
        Hc = alloc<double>(pp);
        evals = alloc<double>(pmax);
        evecs = alloc<double>(pp);
        eigwork = alloc<double>(sym_eig_work(pmax));
        gscr = alloc<double>(gram_scratch(pmax));
        gscr2 = alloc<double>(gram_scratch(pmax));
        LRA_CUDA(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
        LRA_CUDA(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
        LRA_CUDA(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
        Gm = alloc<double>(pp);
        norms = alloc<double>(4);
        epi = alloc<double>(3 * (dpad / 16) + 8);
        dots = alloc<double>(pmax + 4);
        Rinv = alloc<float>(pp);
        P = alloc<float>(pp);
        status = alloc<int>(4);
        tcerr = alloc<int>(4);
        zero(tcerr, sizeof(int) * 4);
        tcs = alloc<float>(2 + 3 * (size_t)PPmax);
        if (sp_items >= 0) {
            partial = alloc<float>((size_t)std::max<int64_t>(sp_items, 1) * PPmax);
        } else {
            ldy = tc_ldy(n);
            Wb = alloc<__nv_bfloat16>((size_t)2 * PPmax * dpad);
            Yb = alloc<__nv_bfloat16>((size_t)2 * PPmax * ldy);
        }
        LRA_CUDA(cudaMallocHost(&host, sizeof(double) * (2 * pmax + 16)));
        LRA_CUDA(cudaMallocHost(&hstat, sizeof(int) * 4));
        hstat[0] = hstat[1] = 0;
    } catch (...) {
        for (auto &a : allocs) dev_free(ctx, a.first, a.second, astream);
        allocs.clear();
        if (side) cudaStreamDestroy(side);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        throw;
    }
}

Workspace::~Workspace() {
    if (side) cudaStreamSynchronize(side);
    if (astream) cudaStreamSynchronize(astream);
    for (auto &a : allocs) dev_free(ctx, a.first, a.second, astream);
    if (idx) dev_free(ctx, idx, sizeof(int32_t) * idx_cap, astream);
    if (cval) dev_free(ctx, cval, sizeof(float) * idx_cap, astream);
    if (astream) cudaStreamSynchronize(astream);
    if (host) cudaFreeHost(host);
    if (hstat) cudaFreeHost(hstat);
    if (side) cudaStreamDestroy(side);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
}

void Workspace::ensure_idx(int64_t m) {
    if (m <= idx_cap) return;
    const int64_t cap = std::max<int64_t>(m, 2 * idx_cap);
    // stream-ordered frees wait for the stream's earlier work; plain frees need
    // the device idle first
    if (!astream) cudaDeviceSynchronize();
    if (idx) dev_free(ctx, idx, sizeof(int32_t) * idx_cap, astream);
    if (cval) dev_free(ctx, cval, sizeof(float) * idx_cap, astream);
    idx = nullptr;
    cval = nullptr;
    idx_cap = 0;
    idx = static_cast<int32_t *>(dev_alloc(ctx, sizeof(int32_t) * cap, astream));
    cval = static_cast<float *>(dev_alloc(ctx, sizeof(float) * cap, astream));
    idx_cap = cap;
}

// ---------------------------------------------------------------------------
// Kernel timer
// ---------------------------------------------------------------------------
KernelTimer::~KernelTimer() {
    for (auto e : pool_) cudaEventDestroy(e);
}

size_t KernelTimer::event() {
    if (used_ == pool_.size()) {
        cudaEvent_t e;
        LRA_CUDA(cudaEventCreate(&e));
        pool_.push_back(e);
    }
    return used_++;
}

void KernelTimer::begin(Kind k, int cols) {
    const size_t a = event();
    LRA_CUDA(cudaEventRecord(pool_[a], s_));
    recs_.push_back({(int)k, cols, a, a});
}

void KernelTimer::end() {
    const size_t b = event();
    LRA_CUDA(cudaEventRecord(pool_[b], s_));
    recs_.back().e1 = b;
}

void KernelTimer::collect(double ms[NKIND], int64_t launches[NKIND], int64_t cols[NKIND]) {
    LRA_CUDA(cudaStreamSynchronize(s_));
    for (int i = 0; i < NKIND; ++i) {
        ms[i] = 0.0;
        launches[i] = 0;
        cols[i] = 0;
    }
    for (const auto &r : recs_) {
        float t = 0.0f;
        LRA_CUDA(cudaEventElapsedTime(&t, pool_[r.e0], pool_[r.e1]));
        ms[r.kind] += t;
        launches[r.kind] += 1;
        cols[r.kind] += r.cols;
    }
}

// ---------------------------------------------------------------------------
// Engine
// ---------------------------------------------------------------------------
void Engine::sync() { LRA_CUDA(cudaStreamSynchronize(s_)); }

void Engine::ensure_norms() {
    std::lock_guard<std::mutex> g(mat_->setup_mu);
    if (mat_->have_norms) return;
    if (!mat_->norm2) {
        mat_->norm2 = static_cast<double *>(dev_alloc(mat_->ctx, sizeof(double) * mat_->n));
        mat_->dev_sm = static_cast<double *>(dev_alloc(mat_->ctx, sizeof(double) * 4));
    }
    if (mat_->sp)
        sparse_colnorms(s_, mat_->sp->colptr, mat_->sp->cval, mat_->n, mat_->norm2);
    else
        colnorms(s_, mat_->X, mat_->storage, mat_->dpad, mat_->d, mat_->n, mat_->norm2, mat_->xscale);
    sum_max(s_, mat_->norm2, mat_->n, mat_->dev_sm, nullptr);
    double h[2];
    LRA_CUDA(cudaMemcpyAsync(h, mat_->dev_sm, sizeof(h), cudaMemcpyDeviceToHost, s_));
    sync();
    if (!std::isfinite(h[0])) {
        set_error("X has a non-finite entry (||X||_F^2 is not finite)");
        throw Error{LRA_EINVAL};
    }
    mat_->fro2 = h[0];
    mat_->maxn = h[1];
    mat_->have_norms = true;
}

const lra_mat::Table &Engine::defl_table(int mode) {
    auto &t = defl->table[mode];
    if (t.ok) return t;
    const int64_t n = mat_->n;
    const int64_t scr = std::max<int64_t>(ceil_div(n, 1024) + 16, ceil_div(n, 256) + 16);
    uint64_t *scratch = static_cast<uint64_t *>(dev_alloc(mat_->ctx, sizeof(uint64_t) * scr, s_));
    try {
        sampling_table(s_, defl->norm2, n, mode, defl->sm + 1, t.cum, t.c, defl->sm + 2, scratch);
        uint64_t tot = 0;
        double kp = 0;
        LRA_CUDA(cudaMemcpyAsync(&tot, t.cum + n - 1, sizeof(tot), cudaMemcpyDeviceToHost, s_));
        LRA_CUDA(cudaMemcpyAsync(&kp, defl->sm + 2, sizeof(kp), cudaMemcpyDeviceToHost, s_));
        sync();
        t.total = tot;
        t.kappa = kp;
        t.ok = true;
    } catch (...) {
        cudaStreamSynchronize(s_);
        dev_free(mat_->ctx, scratch, sizeof(uint64_t) * scr, s_);
        throw;
    }
    dev_free(mat_->ctx, scratch, sizeof(uint64_t) * scr, s_);
    if (t.total == 0) {
        set_error("the deflated X has no non-zero column");
        throw Error{LRA_EINVAL};
    }
    return t;
}

void Engine::project(float *V, int p) {
    if (defl && defl->c > 0) defl_project(s_, defl->U, mat_->dpad, defl->c, V, mat_->dpad, mat_->dpad, p, defl->C);
}

const lra_mat::Table &Engine::ensure_table(int mode) {
    if (defl) return defl_table(mode);
    ensure_norms();
    std::lock_guard<std::mutex> g(mat_->setup_mu);
    auto &t = mat_->table[mode];
    if (t.ok) return t;
    const int64_t n = mat_->n;
    if (!t.cum) {
        t.cum = static_cast<uint64_t *>(dev_alloc(mat_->ctx, sizeof(uint64_t) * n));
        t.c = static_cast<float *>(dev_alloc(mat_->ctx, sizeof(float) * n));
    }
    const int64_t scr = std::max<int64_t>(ceil_div(n, 1024) + 16, ceil_div(n, 256) + 16);
    uint64_t *scratch = static_cast<uint64_t *>(dev_alloc(mat_->ctx, sizeof(uint64_t) * scr, s_));
    double *kap = reinterpret_cast<double *>(mat_->dev_sm) + 2;
    try {
        sampling_table(s_, mat_->norm2, n, mode, mat_->dev_sm + 1, t.cum, t.c, kap, scratch);
        uint64_t tot = 0;
        double kp = 0;
        LRA_CUDA(cudaMemcpyAsync(&tot, t.cum + n - 1, sizeof(tot), cudaMemcpyDeviceToHost, s_));
        LRA_CUDA(cudaMemcpyAsync(&kp, kap, sizeof(kp), cudaMemcpyDeviceToHost, s_));
        sync();
        t.total = tot;
        t.kappa = kp;
        t.ok = true;
    } catch (...) {
        cudaStreamSynchronize(s_);
        dev_free(mat_->ctx, scratch, sizeof(uint64_t) * scr, s_);
        throw;
    }
    dev_free(mat_->ctx, scratch, sizeof(uint64_t) * scr, s_);
    if (t.total == 0) {
        set_error("X has no non-zero column");
        throw Error{LRA_EINVAL};
    }
    return t;
}

void Engine::check_tc() {
    int e = 0;
    LRA_CUDA(cudaMemcpyAsync(&e, ws_.tcerr, sizeof(int), cudaMemcpyDeviceToHost, s_));
    sync();
    if (e) {
        set_error("a tensor-core pipeline wait timed out");
        throw Error{LRA_ETIMEOUT};
    }
}

void Engine::xt_mul(const float *W, int p, float *Y, bool use32, bool keep_hilo) {
    const int PP = pad_p(p);
    if (defl && defl->c > 0) {
        // X'^T W = X^T (I - U U^T) W
        LRA_CUDA(cudaMemcpyAsync(defl->V, W, sizeof(float) * mat_->dpad * p, cudaMemcpyDeviceToDevice, s_));
        project(defl->V, p);
        W = defl->V;
    }
    if (mat_->sp) {
        pack_rm(s_, W, mat_->dpad, mat_->dpad, p, PP, ws_.Wr);
        if (timer) timer->begin(KernelTimer::XTW, p);
        spmm_xt(s_, mat_->sp->colptr, mat_->sp->rowidx, mat_->sp->cval, mat_->n, mat_->d, ws_.Wr, PP, p, Y);
        if (timer) timer->end();
    } else if (tc(use32)) {
        const bool f16 = mat_->storage == LRA_F16;
        if (f16) {
            ensure_norms();  // the bound max_i ||x_i|| behind the scales of Y's FP16 copy
            pack_hilo_f16(s_, W, mat_->dpad, mat_->dpad, p, PP, mat_->xscale, std::sqrt(mat_->maxn), ws_.tcs,
                          reinterpret_cast<__half *>(ws_.Wb));
        } else {
            pack_hilo(s_, W, mat_->dpad, mat_->dpad, p, PP, ws_.Wb);
        }
        if (timer) timer->begin(KernelTimer::XTW, p);
        // the 16-bit hi/lo copy of Y feeds a following X Y pass; an FP32 result
        // (Rayleigh-Ritz, the power steps) is used alone unless keep_hilo
        xtw_tc(s_, tcx(), mat_->Xl, mat_->dpad, mat_->n, ws_.Wb, PP, Y, (Y && !keep_hilo) ? nullptr : ws_.Yb,
               ws_.ldy, ws_.tcerr, tc_wait_, f16, ws_.tcs);
        if (timer) timer->end();
    } else {
        pack_rm(s_, W, mat_->dpad, mat_->dpad, p, PP, ws_.Wr);
        if (timer) timer->begin(KernelTimer::XTW, p);
        xtw(s_, xptr(use32), xdt(use32), mat_->dpad, mat_->dpad, mat_->n, ws_.Wr, PP, Y);
        if (timer) timer->end();
    }
    stats.x_passes += 1;
}

void Engine::xy_pass(const float *Y32, int p, bool use32) {
    const int PP = pad_p(p);
    if (mat_->sp) {
        const auto &sp = *mat_->sp;
        ws_.nch = 1;
        if (timer) timer->begin(KernelTimer::XY, p);
        gscale_ = nullptr;
        spmm_x(s_, sp.rowptr, sp.colidx, sp.val, mat_->d, mat_->dpad, sp.item_off, sp.items, sp.nitems, kSparseSeg,
               Y32, PP, p, ws_.Gp, ws_.partial);
        if (timer) timer->end();
    } else if (tc(use32)) {
        const bool f16 = mat_->storage == LRA_F16;
        if (Y32) {
            if (f16)
                y_hilo_f16(s_, Y32, mat_->n, PP, p, mat_->xscale, ws_.tcs, reinterpret_cast<__half *>(ws_.Yb),
                           ws_.ldy);
            else
                y_hilo(s_, Y32, mat_->n, PP, ws_.Yb, ws_.ldy);
        }
        ws_.nch = xy_chunks(mat_->dpad, mat_->n, tc_rows_per_cta(PP, mat_->Xl != nullptr));
        if (timer) timer->begin(KernelTimer::XY, p);
        xy_tc(s_, tcx(), mat_->Xl, mat_->dpad, mat_->n, ws_.Yb, ws_.ldy, PP, ws_.Gp, ws_.nch, ws_.tcerr, tc_wait_,
              f16);
        if (timer) timer->end();
        // FP16 operands: column c of the partials carries xscale sy_c
        gscale_ = f16 ? ws_.tcs + 2 + PP : nullptr;
    } else {
        gscale_ = nullptr;
        ws_.nch = xy_chunks(mat_->dpad, mat_->n, 128);
        if (timer) timer->begin(KernelTimer::XY, p);
        xy(s_, xptr(use32), xdt(use32), mat_->dpad, mat_->dpad, mat_->n, Y32, PP, ws_.Gp, ws_.nch);
        if (timer) timer->end();
    }
    stats.x_passes += 1;
}

void Engine::x_mul(const float *Y, int p, float *G, bool use32) {
    xy_pass(Y, p, use32);
    anchor_epilogue(s_, ws_.Gp, ws_.nch, mat_->dpad, pad_p(p), p, 0.0, nullptr, nullptr, G, nullptr,
                    ws_.epi, nullptr, 0.0, gscale_);
    project(G, p);  // X' Y = (I - U U^T) X Y
}

void Engine::a_apply(const float *W, int p, float *G) {
    if (tc(false)) {
        xt_mul(W, p, nullptr, false);
        xy_pass(nullptr, p, false);
    } else {
        xt_mul(W, p, ws_.Y, false);
        xy_pass(ws_.Y, p, false);
    }
    anchor_epilogue(s_, ws_.Gp, ws_.nch, mat_->dpad, pad_p(p), p, 0.0, nullptr, nullptr, G, nullptr,
                    ws_.epi, nullptr, 0.0, gscale_);
    project(G, p);
}

void Engine::anchor(const float *Wt, const float *B, int p, double lam, float *M, const float *G0,
                    double *nM2, double *nB2, const AccHook *acc, double *nR2) {
    const int PP = pad_p(p);
    const float *Gsrc = ws_.Gp;
    int nch = 0;
    if (G0) {
        Gsrc = G0;  // X X^T Wt supplied by the caller (one dpad x PP chunk)
        nch = 1;
    } else if (tc(false)) {
        xt_mul(Wt, p, nullptr, false);
        xy_pass(nullptr, p, false);
    } else {
        xt_mul(Wt, p, ws_.Y, false);
        xy_pass(ws_.Y, p, false);
    }
    const float *colscale = G0 ? nullptr : gscale_;
    if (!G0) nch = ws_.nch;
    if (!G0 && defl && defl->c > 0) {
        // X' X'^T Wt = (I - U U^T) X X^T (I - U U^T) Wt: the partials summed,
        // projected and handed to the epilogue as one chunk
        anchor_epilogue(s_, Gsrc, nch, mat_->dpad, PP, p, 0.0, nullptr, nullptr, defl->V, nullptr, ws_.epi, nullptr,
                        0.0, colscale);
        project(defl->V, p);
        pack_rm(s_, defl->V, mat_->dpad, mat_->dpad, p, PP, defl->G0);
        Gsrc = defl->G0;
        nch = 1;
        colscale = nullptr;
    }
    if (timer) timer->begin(KernelTimer::EPI, p);
    anchor_epilogue(s_, Gsrc, nch, mat_->dpad, PP, p, lam, Wt, B, M, ws_.norms, ws_.epi, acc ? acc->Z : nullptr,
                    acc ? acc->gamma : 0.0, colscale);
    if (timer) timer->end();
    if (nM2 || nB2) {
        LRA_CUDA(cudaMemcpyAsync(ws_.host, ws_.norms, (acc ? 3 : 2) * sizeof(double), cudaMemcpyDeviceToHost, s_));
        if (tc(false)) check_tc();
        sync();
        if (nM2) *nM2 = ws_.host[0];
        if (nB2) *nB2 = ws_.host[1];
        if (acc && nR2) *nR2 = ws_.host[2];
    }
}

void Engine::inner(float *W, const float *Wt, const float *M, int p, const int32_t *idx,
                   const float *cval, int64_t m, double eta, double lam, int batch) {
    const bool deflated = defl && defl->c > 0;
    if (mat_->sp && !(deflated && defl->mcap > 0)) {
        // factored form: Mr = M row-major in Wr, Z in the G buffer (both free
        // between the anchor's epilogue and the next X pass)
        const int PP = pad_p(p);
        pack_rm(s_, M, mat_->dpad, mat_->dpad, p, PP, ws_.Wr);
        InnerDefl id;
        if (deflated) {
            id.U = defl->U;
            id.c = defl->c;
            id.Gt = defl->Gt;
            id.PPc = defl->PPc;
            id.scratch = defl->lk;
        }
        if (timer) timer->begin(KernelTimer::INNER, p);
        svrg_inner_csc(s_, mat_->sp->colptr, mat_->sp->rowidx, mat_->sp->cval, mat_->dpad, p, PP, W, Wt, ws_.Wr,
                       ws_.Gp, ws_.dots, idx, cval, m, eta, lam, batch, deflated ? &id : nullptr);
        if (timer) timer->end();
        return;
    }
    if (deflated) {
        // the sampled columns of X' = (I - U U^T) X, formed chunk by chunk from the
        // exact FP32 values (dense X, or a CSR X with d small enough for the dense
        // steps), then the same steps on them in sampling order
        const int64_t per = std::max<int64_t>(1, defl->mcap / batch);
        if (timer) timer->begin(KernelTimer::INNER, p);
        for (int64_t t0 = 0; t0 < m; t0 += per) {
            const int64_t mt = std::min(per, m - t0);
            if (mat_->sp)
                defl_gather_csc(s_, mat_->sp->colptr, mat_->sp->rowidx, mat_->sp->cval, mat_->dpad, idx + t0 * batch,
                                mt * batch, defl->U, defl->c, defl->Gt, defl->PPc, defl->cols);
            else
                defl_gather(s_, mat_->X32, mat_->dpad, mat_->dpad, idx + t0 * batch, mt * batch, defl->U, defl->c,
                            defl->Gt, defl->PPc, defl->cols);
            svrg_inner(s_, defl->cols, LRA_F32, mat_->dpad, mat_->dpad, p, W, Wt, M, defl->iota, cval + t0 * batch,
                       mt, (float)eta, (float)lam, batch, 1.0f);
        }
        if (timer) timer->end();
        return;
    }
    if (timer) timer->begin(KernelTimer::INNER, p);
    svrg_inner(s_, mat_->X, mat_->storage, mat_->dpad, mat_->dpad, p, W, Wt, M, idx, cval, m,
               (float)eta, (float)lam, batch, 1.0f / (mat_->xscale * mat_->xscale));
    if (timer) timer->end();
}

lra_status Engine::cholqr2(float *W, int p, bool deferred) {
    const int64_t dpad = mat_->dpad;
    if (timer) timer->begin(KernelTimer::QR, p);
    LRA_CUDA(cudaMemsetAsync(ws_.status, 0, sizeof(int) * 2, s_));
    for (int pass = 0; pass < 2; ++pass) {
        gram(s_, W, dpad, 1, dpad, p, ws_.Gm, ws_.gscr);
        // the second pass's Gram is I + E with E at the first pass's rounding
        // level for a well-conditioned block: its Cholesky factor to first order
        // (error below 1e-9) replaces the FP64 factorisation there
        chol(s_, ws_.Gm, p, ws_.Rinv, ws_.status + pass, pass == 1 ? 3e-5 : 0.0);
        trsm_rows(s_, W, dpad, dpad, p, ws_.Rinv, ws_.T1);
        LRA_CUDA(cudaMemcpyAsync(W, ws_.T1, sizeof(float) * dpad * p, cudaMemcpyDeviceToDevice, s_));
    }
    if (timer) timer->end();
    LRA_CUDA(cudaMemcpyAsync(ws_.hstat, ws_.status, sizeof(int) * 2, cudaMemcpyDeviceToHost, s_));
    if (deferred) return LRA_OK;  // the caller reads the flags after its next synchronisation
    sync();
    return qr_status();
}

lra_status Engine::qr_status() const {
    if (ws_.hstat[0] || ws_.hstat[1]) {
        set_error("CholeskyQR2: Gram matrix not positive definite");
        return LRA_ENUMERIC;
    }
    return LRA_OK;
}

void Engine::ritz(const float *S, int p, bool use32, int passes, bool with_xq) {
    const int PP = pad_p(p);
    // The FP64 Gram of the basis (for the orthogonality correction below)
    // depends on S alone: it runs on the side stream, on the FP64 units, while
    // the X passes stream X through the tensor cores.
    LRA_CUDA(cudaEventRecord(ws_.ev_fork, s_));
    LRA_CUDA(cudaStreamWaitEvent(ws_.side, ws_.ev_fork, 0));
    // the basis as the tensor-core pass used it: its BF16 pair for FP32 and BF16
    // storage; FP16 storage splits it into FP16 hi/lo of a power-of-two multiple,
    // whose sum is S to about 2^-22, so S itself is used there
    const bool bf16_pair = tc(use32) && mat_->storage != LRA_F16 && !(defl && defl->c > 0);
    gram64(ws_.side, S, nullptr, nullptr, mat_->dpad, mat_->dpad, p, ws_.Gm, ws_.gscr2, bf16_pair);
    LRA_CUDA(cudaEventRecord(ws_.ev_join, ws_.side));
    xt_mul(S, p, ws_.Q, use32, with_xq);
    if (with_xq) {
        // X Q (kept in T1 for the warm start) and H = S^T (X Q): the Ritz
        // matrix from a d-long contraction instead of the n-long Q^T Q
        x_mul(tc(use32) ? nullptr : ws_.Q, p, ws_.T1, use32);
        if (timer) timer->begin(KernelTimer::RITZ, p);
        if (bf16_pair)
            cross_gram(s_, nullptr, ws_.Wb, ws_.Wb + (size_t)PP * mat_->dpad, ws_.T1, mat_->dpad, mat_->dpad, p,
                       ws_.H, ws_.gscr);
        else
            cross_gram(s_, S, nullptr, nullptr, ws_.T1, mat_->dpad, mat_->dpad, p, ws_.H, ws_.gscr);
    } else {
        if (timer) timer->begin(KernelTimer::RITZ, p);
        gram(s_, ws_.Q, mat_->n, PP, 1, p, ws_.H, ws_.gscr);
    }
    // S is orthonormal to FP32 rounding only; correct H to first order in
    // S^T S - I, with the Gram of the basis the X pass actually used (its BF16
    // pair on the tensor-core path).
    LRA_CUDA(cudaStreamWaitEvent(s_, ws_.ev_join, 0));
    ortho_correct(s_, ws_.H, ws_.Gm, p, ws_.Hc);
    if (timer) timer->end();
    if (timer) timer->begin(KernelTimer::EIG, p);
    // inside the outer loop (with_xq) the basis is already close to the Ritz
    // vectors and one refinement pass follows: looser sweeps suffice there
    sym_eig(s_, ws_.Hc, p, ws_.evals, ws_.evecs, ws_.eigwork, passes, with_xq ? 1e-8 : 1e-10);
    if (timer) timer->end();
}

void Engine::normalize(float *z) {
    col_dots(s_, z, z, mat_->dpad, mat_->dpad, 1, ws_.dots);
    scale_cols_rsqrt(s_, z, mat_->dpad, mat_->dpad, 1, ws_.dots);
}

double Engine::dot1(const float *a, const float *b) {
    col_dots(s_, a, b, mat_->dpad, mat_->dpad, 1, ws_.dots);
    LRA_CUDA(cudaMemcpyAsync(ws_.host, ws_.dots, sizeof(double), cudaMemcpyDeviceToHost, s_));
    sync();
    return ws_.host[0];
}

void Engine::step_params(double lam, double mu, double l1up, double kappa, const Opts &o,
                         double &eta, int64_t &m) const {
    // a batch of b samples divides the variance term kappa lambda1_up by b
    const int b = o.batch;
    eta = o.theta_eta * mu / (lam * lam + kappa * l1up / b);
    const double mm = std::ceil(o.theta_m / (eta * mu));
    const int64_t m_max = std::max<int64_t>(1, (o.m_max > 0 ? o.m_max : 50 * mat_->n) / b);
    m = (mm > (double)m_max) ? m_max : (int64_t)mm;
}

lra_status Engine::svrg_solve(const float *B, float *W, int p, double lam, double mu, double l1up,
                              uint64_t seed, int64_t solve_id, const Opts &o, const float *G0,
                              SolveInfo &info, const AccHook *acc) {
    const auto &tab = ensure_table(o.sampling);
    double eta;
    int64_t m;
    step_params(lam, mu, l1up, tab.kappa, o, eta, m);
    info = SolveInfo();
    info.m = m;
    info.eta = eta;
    stats.solves += 1;
    const size_t blk = sizeof(float) * mat_->dpad * p;
    const int max_e = o.fixed_epochs > 0 ? o.fixed_epochs : o.max_epochs;
    double best = INFINITY, prev = INFINITY, res0 = INFINITY;
    for (int e = 0; e < max_e; ++e) {
        LRA_CUDA(cudaMemcpyAsync(ws_.Wt, W, blk, cudaMemcpyDeviceToDevice, s_));
        double nM2, nB2, nR2 = 0.0;
        anchor(ws_.Wt, B, p, lam, ws_.M, (e == 0) ? G0 : nullptr, &nM2, &nB2, acc, &nR2);
        stats.epochs += 1;
        const double res = nB2 > 0 ? std::sqrt(nM2 / nB2) : 0.0;
        info.epochs = e + 1;
        info.residual = res;
        if (e == 0) res0 = res;
        // divergence: above 10x the best, above the start and above 1e-3 (a
        // rebound at the rounding floor is left to the stall rule)
        if (!std::isfinite(res) || (res > 10.0 * best && res > std::max(res0, 1e-3))) {
            set_error("SVRG: residual " + std::to_string(res) + " after a best of " + std::to_string(best) +
                      " at epoch " + std::to_string(e) + " (lambda " + std::to_string(lam) + ", mu " +
                      std::to_string(mu) + ", p " + std::to_string(p) + ")");
            info.status = LRA_EDIVERGED;
            return LRA_EDIVERGED;
        }
        double tol = o.tau;
        if (acc) {
            if (e == 0) {
                // the original system's residual at W, (lam - gamma) W - X X^T W - B,
                // summed by the anchor's epilogue
                info.outer_res = std::sqrt(nR2);
                if (o.fixed_epochs <= 0 && info.outer_res <= o.tau * acc->nB) {
                    info.outer_done = true;
                    return LRA_OK;
                }
            }
            tol = nB2 > 0 ? std::max(o.tau * acc->nB, o.acc_theta * acc->sq * info.outer_res) / std::sqrt(nB2)
                          : 0.0;
        }
        if (o.fixed_epochs <= 0) {
            if (res <= tol) return LRA_OK;
            if (e >= 3 && res > 0.9 * prev) return LRA_OK;
        }
        if (e == max_e - 1) {
            if (o.fixed_epochs <= 0) info.status = LRA_ENOTCONV;
            return LRA_OK;
        }
        best = std::min(best, res);
        prev = res;
        const int64_t ns = m * o.batch;  // samples of the epoch
        ws_.ensure_idx(ns);
        const uint64_t key = stream_key(seed, LRA_STREAM_SVRG, (uint64_t)solve_id, (uint64_t)e);
        sample(s_, tab.cum, mat_->n, key, ns, ws_.idx, tab.c, ws_.cval);
        inner(W, ws_.Wt, ws_.M, p, ws_.idx, ws_.cval, m, eta, lam, o.batch);
        info.inner_steps += m;
        stats.inner_steps += m;
    }
    return LRA_OK;
}

double Engine::acc_gamma(double lam, double mu, double l1up, double kappa, const Opts &o) const {
    // Smallest gamma >= 0 at which an SVRG epoch of the subproblem
    // ((lam + g) I - A) draws at most T samples: with K = kappa l1up / b and
    // c = theta_m / theta_eta the uncapped epoch is b c ((lam + g)^2 + K) /
    // (mu + g)^2 samples; equal to T at the positive root of
    // (1 - a) g^2 + 2 (lam - a mu) g + lam^2 + K - a mu^2 = 0, a = T / (b c),
    // raised by 1e-9 relative so that ceil() of the epoch length is not decided
    // by the last bit of a value sitting exactly on the integer T / b.
    const int b = std::max(1, o.batch);
    const double T = (double)(o.acc_target > 0 ? o.acc_target : mat_->n);
    const double K = kappa * l1up / b;
    const double a = T * o.theta_eta / (b * o.theta_m);
    const double C = lam * lam + K - a * mu * mu;
    if (C <= 0.0 || a <= 1.0) return 0.0;
    const double h = lam - a * mu;
    return (h + std::sqrt(h * h + (a - 1.0) * C)) / (a - 1.0) * (1.0 + 1e-9);
}

lra_status Engine::acc_solve(const float *B, float *W, int p, double lam, double mu, double l1up,
                             uint64_t seed, int64_t &solve_count, const Opts &o, const float *G0,
                             SolveInfo &info) {
    // AccSVRGsolve (Sec. 1, Cor. mainCond; the acceleration of Frostig et al.,
    // which the paper does not print): accelerated proximal point on
    // F(W) = 1/2 tr W^T (lam I - A) W - tr B^T W.  Subproblem s is the
    // shifted system ((lam + gamma) I - A) W = B + gamma Z_s, solved by SVRG
    // from W_s; then Z_{s+1} = W_{s+1} + beta (W_{s+1} - W_s) with
    // beta = (1 - sqrt q) / (1 + sqrt q), q = mu / (mu + gamma).  The loop ends
    // when the original residual, read off a subproblem's first anchor, is
    // below tau ||B||; no X pass is added.
    const auto &tab = ensure_table(o.sampling);
    const double gamma = acc_gamma(lam, mu, l1up, tab.kappa, o);
    if (!(gamma > 0.0)) return svrg_solve(B, W, p, lam, mu, l1up, seed, solve_count++, o, G0, info);
    const double q = mu / (mu + gamma), sq = std::sqrt(q), beta = (1.0 - sq) / (1.0 + sq);
    const int64_t dpad = mat_->dpad;
    col_dots(s_, B, B, dpad, dpad, p, ws_.dots);
    acc_extrapolate(s_, W, ws_.Wo, ws_.Za, dpad, dpad, p, 0.0f, true);
    LRA_CUDA(cudaMemcpyAsync(ws_.host, ws_.dots, sizeof(double) * p, cudaMemcpyDeviceToHost, s_));
    sync();
    double b2 = 0.0;
    for (int j = 0; j < p; ++j) b2 += ws_.host[j];
    const AccHook hook{gamma, std::sqrt(b2), sq, ws_.Za};
    info = SolveInfo();
    info.gamma = gamma;
    info.status = o.fixed_epochs > 0 ? LRA_OK : LRA_ENOTCONV;
    // stall: after w subproblems (an expected contraction of e^-2) a residual
    // above half the one w before, the rounding floor of the path
    const int w = std::max(3, (int)std::ceil(2.0 / sq));
    std::vector<double> hist;
    for (int s = 0; s < o.acc_max_outer; ++s) {
        SolveInfo sub;
        // the subproblem's right-hand side B + gamma Z is formed inside the anchor's
        // epilogue (FP64), from B and Z
        const lra_status st = svrg_solve(B, W, p, lam + gamma, mu + gamma, l1up, seed, solve_count++, o,
                                         s == 0 ? G0 : nullptr, sub, &hook);
        info.epochs += sub.epochs;
        info.inner_steps += sub.inner_steps;
        info.m = sub.m;
        info.eta = sub.eta;
        info.outer = s + 1;
        info.outer_res = sub.outer_res;
        info.residual = hook.nB > 0 ? sub.outer_res / hook.nB : 0.0;
        if (st != LRA_OK || sub.status == LRA_EDIVERGED) {
            info.status = LRA_EDIVERGED;
            return LRA_EDIVERGED;
        }
        if (sub.outer_done) {
            info.status = LRA_OK;
            info.outer_done = true;
            return LRA_OK;
        }
        hist.push_back(sub.outer_res);
        if (o.fixed_epochs <= 0 && (int)hist.size() > w && hist.back() > 0.5 * hist[hist.size() - 1 - w]) {
            info.status = LRA_OK;
            return LRA_OK;
        }
        acc_extrapolate(s_, W, ws_.Wo, ws_.Za, dpad, dpad, p, (float)beta, false);
    }
    return LRA_OK;
}

lra_status Engine::solve_linear(const float *B, float *W, int p, double lam, double mu, double l1up,
                                uint64_t seed, int64_t &solve_count, const Opts &o, const float *G0,
                                SolveInfo &info) {
    if (o.acc) return acc_solve(B, W, p, lam, mu, l1up, seed, solve_count, o, G0, info);
    return svrg_solve(B, W, p, lam, mu, l1up, seed, solve_count++, o, G0, info);
}

double Engine::lambda1_estimate(uint64_t seed) {
    const int64_t d = mat_->d;
    const int L = (int)std::ceil(4.0 * std::log(4.0 * (double)d));
    float *z = ws_.S;
    gaussian(s_, stream_key(seed, LRA_STREAM_POWER_A, 0, 0), d, mat_->dpad, 1, z);
    normalize(z);
    for (int l = 0; l < L; ++l) {
        a_apply(z, 1, ws_.W);
        LRA_CUDA(cudaMemcpyAsync(z, ws_.W, sizeof(float) * mat_->dpad, cudaMemcpyDeviceToDevice, s_));
        normalize(z);
    }
    xt_mul(z, 1, ws_.Y, false);
    gram(s_, ws_.Y, mat_->n, pad_p(1), 1, 1, ws_.Gm, ws_.gscr);
    LRA_CUDA(cudaMemcpyAsync(ws_.host, ws_.Gm, sizeof(double), cudaMemcpyDeviceToHost, s_));
    sync();
    if (tc(false)) check_tc();
    return ws_.host[0];
}

lra_status Engine::d_top_inverse(uint64_t seed, int rnd, double lam, double mu, double l1up,
                                 const Opts &o, int64_t &solve_count, double &inv) {
    const int64_t d = mat_->d, dpad = mat_->dpad;
    const int L = (int)std::ceil(9.0 * std::log(9.0 * (double)d));
    float *z = ws_.S;
    float *w = ws_.U;  // solve output (one column)
    gaussian(s_, stream_key(seed, LRA_STREAM_POWER_D, (uint64_t)rnd, 0), d, dpad, 1, z);
    normalize(z);
    double scale = 1.0 / lam;
    SolveInfo info;
    for (int l = 0; l <= L; ++l) {
        LRA_CUDA(cudaMemcpyAsync(w, z, sizeof(float) * dpad, cudaMemcpyDeviceToDevice, s_));
        scale_block(s_, w, dpad, dpad, 1, (float)scale);
        const lra_status st = solve_linear(z, w, 1, lam, mu, l1up, seed, solve_count, o, nullptr, info);
        if (st != LRA_OK || info.status == LRA_EDIVERGED) return LRA_EDIVERGED;
        if (l == L) {
            const double lt = dot1(z, w);
            if (!(lt > 0.0) || !std::isfinite(lt)) {
                set_error("Algorithm 3 on D: z^T D z = " + std::to_string(lt) + " at lambda " + std::to_string(lam));
                return LRA_EDIVERGED;
            }
            inv = 1.0 / lt;
            return LRA_OK;
        }
        const double nw = std::sqrt(dot1(w, w));
        if (!(nw > 0.0) || !std::isfinite(nw)) {
            set_error("Algorithm 3 on D: ||D z|| = " + std::to_string(nw) + " at lambda " + std::to_string(lam));
            return LRA_EDIVERGED;
        }
        scale = nw;
        LRA_CUDA(cudaMemcpyAsync(z, w, sizeof(float) * dpad, cudaMemcpyDeviceToDevice, s_));
        normalize(z);
    }
    return LRA_OK;
}

lra_status Engine::shift_tune(uint64_t seed, double l1hat, double delta, const Opts &o,
                              int64_t &solve_count, double &lam, double &inv, double &mu,
                              int &rounds, std::vector<double> *history) {
    const double eps = 1.0 / 9.0;
    const double l1up = l1hat / (1.0 - 0.25);
    lam = 1.5 * l1hat;
    mu = lam - l1up;
    inv = INFINITY;
    rounds = 0;
    for (int rnd = 0; rnd < o.max_shift_rounds; ++rnd) {
        double est = 0.0;
        const lra_status st = d_top_inverse(seed, rnd, lam, mu, l1up, o, solve_count, est);
        rounds = rnd + 1;
        if (history) {
            history->push_back(lam);
            history->push_back(est);
        }
        if (st != LRA_OK) return st;
        inv = est;
        if (delta / 27.0 <= est && est <= delta / 5.0) {
            mu = (1.0 - eps) * est;
            return LRA_OK;
        }
        lam = lam - 0.5 * (1.0 - eps) * est;
        mu = 0.5 * (1.0 - eps) * est;
    }
    return LRA_ENOTCONV;
}

lra_status Engine::delta_estimate(int k, int p, uint64_t seed, double &delta) {
    const int q = p + 1;
    const int64_t d = mat_->d;
    const double eps = 1.0 / (9.0 * p * p);
    const int L = (int)std::min(200.0, std::ceil((1.0 / eps) * std::log((double)d / eps)));
    float *S = ws_.S;
    gaussian(s_, stream_key(seed, LRA_STREAM_DELTA, 0, 0), d, mat_->dpad, q, S);
    lra_status st = cholqr2(S, q);
    if (st != LRA_OK) return st;
    for (int l = 0; l < L; ++l) {
        a_apply(S, q, ws_.W);
        LRA_CUDA(cudaMemcpyAsync(S, ws_.W, sizeof(float) * mat_->dpad * q, cudaMemcpyDeviceToDevice, s_));
        st = cholqr2(S, q);
        if (st != LRA_OK) return st;
    }
    ritz(S, q, false);
    LRA_CUDA(cudaMemcpyAsync(ws_.host, ws_.evals, sizeof(double) * q, cudaMemcpyDeviceToHost, s_));
    sync();
    delta = (ws_.host[k - 1] - ws_.host[p]) / 1.5;
    return LRA_OK;
}

static double ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// Stop rule of the outer loop: the predicted remaining decrease of E_l is at
// most (eps/4) E_l, remaining = max(D_l, 0) r / (1 - r) with D_j = E_{j-1} - E_j
// and r the geometric-mean rate of the last w <= 4 differences (the upper clamp
// when D_{l-w} <= 0), at least r_floor, clamped to [0, 1 - 1e-6].
constexpr double kRateMax = 1.0 - 1e-6;

// Theorem 2's per-iteration factor of E's excess, ((lambda - rho_k)/(lambda - rho_p))^2,
// from the current Ritz values (a floor for the observed rate).
static double theory_rate(double lam, const double *rho, int k, int p) {
    const double den = lam - rho[p - 1];
    if (den <= 0.0) return kRateMax;
    const double f = std::min(std::max((lam - rho[k - 1]) / den, 0.0), 1.0);
    return f * f;
}

static bool outer_stop(const std::vector<double> &E, double eps, int ell, int min_outer, double r_floor) {
    if (ell + 1 < std::max(3, min_outer)) return false;
    const size_t n = E.size();
    const size_t w = std::min<size_t>(4, n - 2);
    const double d1 = E[n - 2] - E[n - 1];
    const double d0 = E[n - 2 - w] - E[n - 1 - w];
    double r;
    if (d0 > 0 && d1 > 0)
        r = std::pow(d1 / d0, 1.0 / (double)w);
    else if (d0 > 0)
        r = 0.0;
    else
        r = kRateMax;
    r = std::min(std::max(std::max(r, r_floor), 0.0), kRateMax);
    const double remaining = std::max(d1, 0.0) * r / (1.0 - r);
    return remaining <= 0.25 * eps * E[n - 1];
}

static int alg3_iters(double eps, int64_t d, int cap) {
    const double L = std::ceil((1.0 / eps) * std::log((double)d / eps));
    return (int)std::max(1.0, std::min(L, (double)cap));
}

lra_status Engine::alg3_a(int kk, double eps, int cap, uint64_t seed, double *vals, int &iters) {
    // Algorithm 3 with C = A: Algorithm 1 with kk columns for L steps, then the
    // Ritz values of the final basis (Algorithm 2 with C = A)
    const int64_t d = mat_->d, dpad = mat_->dpad;
    const int L = alg3_iters(eps, d, cap);
    float *S = ws_.S, *W = ws_.W;
    gaussian(s_, stream_key(seed, LRA_STREAM_BLOCK, 0, 0), d, dpad, kk, S);
    lra_status st = cholqr2(S, kk);
    if (st != LRA_OK) return st;
    for (int l = 0; l < L; ++l) {
        a_apply(S, kk, W);
        std::swap(S, W);
        cholqr2(S, kk, true);
        if ((l & 63) == 63) {
            sync();
            if ((st = qr_status()) != LRA_OK) return st;
        }
    }
    a_apply(S, kk, W);
    cross_gram(s_, S, nullptr, nullptr, W, dpad, dpad, kk, ws_.H, ws_.gscr);
    sym_eig(s_, ws_.H, kk, ws_.evals, ws_.evecs, ws_.eigwork);
    LRA_CUDA(cudaMemcpyAsync(ws_.host, ws_.evals, sizeof(double) * kk, cudaMemcpyDeviceToHost, s_));
    sync();
    if ((st = qr_status()) != LRA_OK) return st;
    if (tc(false)) check_tc();
    for (int j = 0; j < kk; ++j) {
        vals[j] = ws_.host[j];
        if (!std::isfinite(vals[j])) {
            set_error("Algorithm 3: non-finite Ritz value");
            return LRA_ENUMERIC;
        }
    }
    iters = L;
    return LRA_OK;
}

lra_status Engine::alg3_d(int kk, double eps, int cap, uint64_t seed, double lam, double mu, double l1up,
                          double l1hat, const Opts &o, int64_t &solve_count, double *vals, int &iters) {
    // Algorithm 3 with C = D = (lam I - A)^{-1}: every product D S a solve.  The
    // solve of step l starts from the previous step's Galerkin projection of D,
    // W0 = S C H C^T with H = sym(S_prev^T D S_prev) and C = S^T S_prev (kk x kk,
    // on the host); the first from S / (lam - lambda_hat).
    const int64_t d = mat_->d, dpad = mat_->dpad;
    const int L = alg3_iters(eps, d, cap);
    float *S = ws_.S, *W = ws_.W, *Sp = ws_.T1;
    gaussian(s_, stream_key(seed, LRA_STREAM_BLOCK, 2, 0), d, dpad, kk, S);
    lra_status st = cholqr2(S, kk);
    if (st != LRA_OK) return st;
    std::vector<double> Hh((size_t)kk * kk), Ch((size_t)kk * kk), T((size_t)kk * kk);
    std::vector<float> Tf((size_t)kk * kk);
    double *h = ws_.host;
    for (int l = 0; l <= L; ++l) {
        if (l == 0) {
            LRA_CUDA(cudaMemcpyAsync(W, S, sizeof(float) * dpad * kk, cudaMemcpyDeviceToDevice, s_));
            scale_block(s_, W, dpad, dpad, kk, (float)(1.0 / (lam - l1hat)));
        } else {
            cross_full(s_, S, Sp, dpad, dpad, kk, ws_.Gm, ws_.gscr);
            LRA_CUDA(cudaMemcpyAsync(Ch.data(), ws_.Gm, sizeof(double) * kk * kk, cudaMemcpyDeviceToHost, s_));
            sync();
            // T = C H C^T (all column-major), then row-major FP32 for apply_right
            for (int a = 0; a < kk; ++a)
                for (int b = 0; b < kk; ++b) {
                    double acc = 0.0;
                    for (int i = 0; i < kk; ++i)
                        for (int j = 0; j < kk; ++j)
                            acc += Ch[a + (size_t)i * kk] * Hh[i + (size_t)j * kk] * Ch[b + (size_t)j * kk];
                    T[a + (size_t)b * kk] = acc;
                }
            for (int a = 0; a < kk; ++a)
                for (int b = 0; b < kk; ++b) Tf[(size_t)a * kk + b] = (float)T[a + (size_t)b * kk];
            LRA_CUDA(cudaMemcpyAsync(ws_.P, Tf.data(), sizeof(float) * kk * kk, cudaMemcpyHostToDevice, s_));
            apply_right(s_, S, dpad, 1, dpad, kk, ws_.P, kk, W, 1, dpad);
        }
        SolveInfo info;
        st = solve_linear(S, W, kk, lam, mu, l1up, seed, solve_count, o, nullptr, info);
        if (st != LRA_OK || info.status == LRA_EDIVERGED) return LRA_EDIVERGED;
        cross_gram(s_, S, nullptr, nullptr, W, dpad, dpad, kk, ws_.H, ws_.gscr);
        if (l == L) {
            sym_eig(s_, ws_.H, kk, ws_.evals, ws_.evecs, ws_.eigwork);
            LRA_CUDA(cudaMemcpyAsync(h, ws_.evals, sizeof(double) * kk, cudaMemcpyDeviceToHost, s_));
            sync();
            if ((st = qr_status()) != LRA_OK) return st;
            for (int j = 0; j < kk; ++j) {
                vals[j] = h[j];
                if (!(vals[j] > 0.0) || !std::isfinite(vals[j])) {
                    set_error("Algorithm 3 on D: non-positive Ritz value");
                    return LRA_EDIVERGED;
                }
            }
            break;
        }
        LRA_CUDA(cudaMemcpyAsync(Hh.data(), ws_.H, sizeof(double) * kk * kk, cudaMemcpyDeviceToHost, s_));
        LRA_CUDA(cudaMemcpyAsync(Sp, S, sizeof(float) * dpad * kk, cudaMemcpyDeviceToDevice, s_));
        sync();
        if (l > 0 && (st = qr_status()) != LRA_OK) return st;
        std::swap(S, W);
        st = cholqr2(S, kk, true);
    }
    if (tc(false)) check_tc();
    iters = L;
    return LRA_OK;
}

lra_status Engine::power_block(int b, double eps, double r_floor, uint64_t seed, const Opts &o, int &iters,
                               lra_status &status) {
    // Algorithm 1 on A with b columns and no oversampling (a block found by
    // Algorithm 4); Rayleigh-Ritz with A each iteration and the outer loop's
    // stop rule on E = ||X||_F^2 - sum of the b Ritz values
    const int64_t d = mat_->d, dpad = mat_->dpad;
    float *S = ws_.S, *W = ws_.W;
    gaussian(s_, stream_key(seed, LRA_STREAM_BLOCK, 1, 0), d, dpad, b, S);
    lra_status st = cholqr2(S, b);
    if (st != LRA_OK) return st;
    std::vector<double> E;
    int ell = 0;
    status = LRA_OK;
    double *h = ws_.host;
    while (true) {
        ritz(S, b, false, 2, false);
        LRA_CUDA(cudaMemcpyAsync(h, ws_.evals, sizeof(double) * b, cudaMemcpyDeviceToHost, s_));
        sync();
        if (ell > 0 && (st = qr_status()) != LRA_OK) return st;
        double sb = 0.0;
        for (int j = 0; j < b; ++j) sb += h[j];
        E.push_back(fro2() - sb);
        if (outer_stop(E, eps, ell, o.min_outer, r_floor)) break;
        if (ell >= o.max_outer) {
            status = LRA_ENOTCONV;
            break;
        }
        a_apply(S, b, W);
        std::swap(S, W);
        cholqr2(S, b, true);
        ++ell;
    }
    // Ritz vectors S V into ws.U
    evecs_to_rm(s_, ws_.evecs, b, b, ws_.P);
    apply_right(s_, S, dpad, 1, dpad, b, ws_.P, b, ws_.U, 1, dpad);
    if (tc(false)) check_tc();
    iters = ell;
    return LRA_OK;
}

lra_status Engine::loop_d(int k, int p, double eps, uint64_t seed, double lam, double mu, double l1up,
                          const Opts &o, int64_t &solve_count, double r_floor, float *&S_out, int &ell,
                          std::vector<double> &E, lra_status &status, lra_report &R,
                          const std::atomic<int> *cancel) {
    const int64_t d = mat_->d, dpad = mat_->dpad;
    status = LRA_OK;
    float *S = ws_.S, *W = ws_.W;
    gaussian(s_, stream_key(seed, LRA_STREAM_INIT, 0, 0), d, dpad, p, S);
    lra_status st = cholqr2(S, p);
    if (st != LRA_OK) return st;
    E.clear();
    ell = 0;
    const int PP = pad_p(p);
    double *h = ws_.host;
    while (true) {
        ritz(S, p, false, 1, o.warm_start != 0);
        LRA_CUDA(cudaMemcpyAsync(h, ws_.evals, sizeof(double) * p, cudaMemcpyDeviceToHost, s_));
        sync();
        if (ell > 0 && (st = qr_status()) != LRA_OK) return st;  // the previous step's CholeskyQR2
        double sk = 0.0;
        for (int j = 0; j < k; ++j) sk += h[j];
        E.push_back(fro2() - sk);
        if (o.trace_E && (int)E.size() <= o.trace_cap) o.trace_E[E.size() - 1] = E.back();
        const double rf = r_floor >= 0.0 ? r_floor : theory_rate(lam, h, k, p);
        if (outer_stop(E, eps, ell, o.min_outer, rf)) break;
        if (ell >= o.max_outer) {
            status = LRA_ENOTCONV;
            break;
        }
        if (cancel && cancel->load()) return LRA_ECANCELLED;
        const float *G0 = nullptr;
        if (o.warm_start) {
            // Move the basis onto the Ritz vectors, S <- S V (same span, so the
            // same Algorithm 1 step; the next Rayleigh-Ritz matrix is then
            // nearly diagonal and the eigensolver's sweeps stop early).  Warm
            // start in that basis: W0 = S V diag(1/(lam - rho)); the first
            // anchor's X X^T W0 = (X Q) V diag(1/(lam - rho)) with X Q from the
            // Rayleigh-Ritz step: a d x p product.
            if (timer) timer->begin(KernelTimer::WARM, p);
            evecs_to_rm(s_, ws_.evecs, p, p, ws_.P);
            apply_right(s_, S, dpad, 1, dpad, p, ws_.P, p, W, 1, dpad);
            LRA_CUDA(cudaMemcpyAsync(S, W, sizeof(float) * dpad * p, cudaMemcpyDeviceToDevice, s_));
            shift_scale_cols(s_, S, W, dpad, dpad, p, ws_.evals, lam);
            ritz_scaled(s_, ws_.evecs, ws_.evals, p, lam, ws_.P);
            apply_right(s_, ws_.T1, dpad, 1, dpad, p, ws_.P, p, ws_.Gp, PP, 1);
            if (timer) timer->end();
            G0 = ws_.Gp;
        } else {
            LRA_CUDA(cudaMemsetAsync(W, 0, sizeof(float) * dpad * p, s_));
        }
        SolveInfo info;
        st = solve_linear(S, W, p, lam, mu, l1up, seed, solve_count, o, G0, info);
        if (st != LRA_OK) return st;
        R.eta = info.eta;
        R.m = info.m;
        R.last_residual = info.residual;
        std::swap(S, W);
        cholqr2(S, p, true);
        ++ell;
    }
    S_out = S;
    return LRA_OK;
}

lra_status Engine::solve(int k, int p, double eps, uint64_t seed, const Opts &o, float *U,
                         double *ritz_out, lra_report *rep, const std::atomic<int> *cancel) {
    const auto t_all = std::chrono::steady_clock::now();
    const int64_t launches0 = launches_of_thread();
    const int64_t d = mat_->d, dpad = mat_->dpad;
    tc_wait_ = o.wait_cycles;
    std::unique_ptr<KernelTimer> own_timer;
    if (o.profile) {
        own_timer.reset(new KernelTimer(s_));
        timer = own_timer.get();
    }
    lra_report R;
    std::memset(&R, 0, sizeof(R));
    R.struct_size = sizeof(R);
    auto t0 = std::chrono::steady_clock::now();
    const auto &tab = ensure_table(o.sampling);
    (void)tab;
    R.fro2 = mat_->fro2;
    const double l1hat = o.lambda1_hat > 0 ? o.lambda1_hat : lambda1_estimate(seed);
    const double l1up = l1hat / (1.0 - 0.25);
    R.lambda1_hat = l1hat;
    R.ms_setup = ms_since(t0);

    t0 = std::chrono::steady_clock::now();
    int64_t solve_count = 0;
    double lam = 0, mu = 0, delta = o.delta;
    lra_status status = LRA_OK;
    if (o.shift_policy == LRA_SHIFT_PAPER) {
        if (!(delta > 0)) {
            status = delta_estimate(k, p, seed, delta);
            if (status != LRA_OK) return status;
        }
        double inv = 0;
        int rounds = 0;
        status = shift_tune(seed, l1hat, delta, o, solve_count, lam, inv, mu, rounds, nullptr);
        R.shift_rounds = rounds;
        if (status == LRA_EDIVERGED) return status;
        status = LRA_OK;  // a capped tuning still yields a valid shift > lambda_1
    } else if (o.shift_policy == LRA_SHIFT_FAR) {
        lam = 2.0 * l1up;
        mu = lam - l1up;
    } else {
        lam = o.lambda;
        mu = lam - l1up;
        if (!(mu > 0)) {
            set_error("FIXED shift must exceed lambda_hat_1 / (1 - 1/4)");
            return LRA_EINVAL;
        }
    }
    R.lambda = lam;
    R.delta = delta;
    R.mu_lb = mu;
    R.ms_shift = ms_since(t0);

    t0 = std::chrono::steady_clock::now();
    float *S = nullptr;
    std::vector<double> E;
    int ell = 0;
    lra_status lst = LRA_OK;
    lra_status st = loop_d(k, p, eps, seed, lam, mu, l1up, o, solve_count, -1.0, S, ell, E, lst, R, cancel);
    if (st != LRA_OK) return st;
    if (lst != LRA_OK) status = lst;
    double *h = ws_.host;
    R.outer_iters = ell;
    R.ms_outer = ms_since(t0);

    t0 = std::chrono::steady_clock::now();
    if (tc(false)) {
        // Algorithm 2 on the exact FP32 values of X (the iteration streamed X as
        // BF16 or as a BF16 pair): the answer is measured there
        ritz(S, p, true);
    }
    if (tc(false)) check_tc();
    evecs_to_rm(s_, ws_.evecs, p, k, ws_.P);
    apply_right(s_, S, dpad, 1, dpad, p, ws_.P, k, ws_.U, 1, dpad);
    LRA_CUDA(cudaMemcpy2DAsync(U, sizeof(float) * d, ws_.U, sizeof(float) * dpad, sizeof(float) * d, k,
                               cudaMemcpyDefault, s_));
    LRA_CUDA(cudaMemcpyAsync(ritz_out, ws_.evals, sizeof(double) * k, cudaMemcpyDefault, s_));
    LRA_CUDA(cudaMemcpyAsync(h, ws_.evals, sizeof(double) * k, cudaMemcpyDeviceToHost, s_));
    sync();
    {
        double sk = 0.0;
        for (int j = 0; j < k; ++j) sk += h[j];
        R.err_est = mat_->fro2 - sk;
    }
    R.ms_final = ms_since(t0);
    R.solves = stats.solves;
    R.epochs = stats.epochs;
    R.inner_steps = stats.inner_steps;
    R.x_passes = stats.x_passes;
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
        timer = nullptr;
    }
    R.ms_total = ms_since(t_all);
    if (rep) {
        const size_t sz = std::min(rep->struct_size ? rep->struct_size : sizeof(R), sizeof(R));
        std::memcpy(rep, &R, sz);
        rep->struct_size = sz;
    }
    return status;
}

}  // namespace lra
