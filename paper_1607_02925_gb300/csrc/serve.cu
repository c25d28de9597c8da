// Request loop entry points (lra_submit / lra_poll / lra_cancel) and the
// worker pool behind them.
#include <chrono>
#include <cstring>

#include "serve.h"

namespace lra {

namespace {

// Device bytes a job needs while it runs: its workspace, the epoch index
// buffers at their cap, and the result buffers.
size_t job_footprint(const lra_mat *m, int k, int p, const Opts &o) {
    const int pmax = (o.shift_policy == LRA_SHIFT_PAPER && !(o.delta > 0)) ? p + 1 : p;
    const int64_t mcap = o.m_max > 0 ? o.m_max : 50 * m->n;
    const size_t idx = sizeof(int32_t) * 2 * (size_t)std::min<int64_t>(mcap, 4 * m->n + 4096);
    return workspace_bytes(m->dpad, m->n, pmax, ws_items(m)) + idx + sizeof(float) * m->d * k + 64 * 1024;
}

int env_int(const char *name, int dflt) {
    const char *v = getenv(name);
    return v ? atoi(v) : dflt;
}

}  // namespace

Server::Server(lra_ctx *ctx, int slots) : ctx_(ctx) {
    size_t free_b = 0, total_b = 0;
    LRA_CUDA(cudaMemGetInfo(&free_b, &total_b));
    // the most the context may hold: its budget if set, else what it holds now
    // plus 90% of what is free now
    limit_ = ctx->budget ? ctx->budget : ctx->used.load() + (size_t)(0.9 * (double)free_b);
    streams_.resize(slots);
    for (int i = 0; i < slots; ++i) LRA_CUDA(cudaStreamCreateWithFlags(&streams_[i], cudaStreamNonBlocking));
    for (int i = 0; i < slots; ++i) threads_.emplace_back(&Server::worker, this, i);
}

Server::~Server() {
    {
        std::lock_guard<std::mutex> g(mu_);
        stop_ = true;
        for (auto &kv : jobs_) kv.second->cancel.store(1);
    }
    cv_work_.notify_all();
    for (auto &t : threads_) t.join();
    for (auto &kv : jobs_) {
        auto &j = kv.second;
        if (j->U) dev_free(ctx_, j->U, j->U_bytes, j->stream);
        if (j->ritz) dev_free(ctx_, j->ritz, j->ritz_bytes, j->stream);
        if (j->state == Job::QUEUED) j->mat->busy.fetch_sub(1);  // never started
    }
    cudaDeviceSynchronize();
    for (auto s : streams_) cudaStreamDestroy(s);
}

// What the loop could hand out with no job running: the limit minus the
// context's memory outside the running jobs (matrices, their sampling tables,
// unpolled results), read at the time of the call, so that matrices created
// after the loop started are accounted for.
size_t Server::idle_capacity_locked() const {
    const size_t used = ctx_->used.load();
    const size_t outside = used > job_bytes_ ? used - job_bytes_ : 0;
    return limit_ > outside ? limit_ - outside : 0;
}

size_t Server::capacity_locked() const {
    const size_t idle = idle_capacity_locked();
    return idle > reserved_ ? idle - reserved_ : 0;
}

// First queued job (in arrival order) whose footprint fits; nullptr if none.
// With no job running, a queued job larger than the idle capacity (matrices
// created after it was queued took the memory) can never start: it ends with
// LRA_ENOMEM instead of waiting forever.
std::shared_ptr<Job> Server::admit_locked() {
    const size_t cap = capacity_locked();
    for (auto it = queue_.begin(); it != queue_.end(); ++it) {
        if ((*it)->footprint <= cap) {
            auto j = *it;
            queue_.erase(it);
            reserved_ += j->footprint;
            j->state = Job::RUNNING;
            return j;
        }
    }
    if (reserved_ == 0) {
        const size_t idle = idle_capacity_locked();
        bool failed = false;
        for (auto it = queue_.begin(); it != queue_.end();) {
            if ((*it)->footprint > idle) {
                auto j = *it;
                it = queue_.erase(it);
                j->state = Job::DONE;
                j->status = LRA_ENOMEM;
                j->error = "job footprint exceeds the device memory left to the request loop";
                j->mat->busy.fetch_sub(1);
                failed = true;
            } else {
                ++it;
            }
        }
        if (failed) cv_done_.notify_all();
    }
    return nullptr;
}

void Server::worker(int slot) {
    cudaSetDevice(ctx_->device);
    const cudaStream_t s = streams_[slot];
    while (true) {
        std::shared_ptr<Job> j;
        {
            std::unique_lock<std::mutex> lk(mu_);
            cv_work_.wait(lk, [&] { return stop_ || (!queue_.empty() && (j = admit_locked()) != nullptr); });
            if (stop_ && !j) return;
        }
        lra_status st = LRA_OK;
        if (j->cancel.load()) {
            st = LRA_ECANCELLED;
        } else {
            try {
                Workspace ws(ctx_, j->mat->dpad, j->mat->n,
                             (j->opts.shift_policy == LRA_SHIFT_PAPER && !(j->opts.delta > 0)) ? j->p + 1 : j->p, s,
                             ws_items(j->mat));
                j->U_bytes = sizeof(float) * j->mat->d * j->k;
                j->ritz_bytes = sizeof(double) * j->k;
                j->stream = s;
                j->U = static_cast<float *>(dev_alloc(ctx_, j->U_bytes, s));
                j->ritz = static_cast<double *>(dev_alloc(ctx_, j->ritz_bytes, s));
                {
                    size_t held = j->U_bytes + j->ritz_bytes;
                    for (const auto &a : ws.allocs) held += a.second;
                    std::lock_guard<std::mutex> g(mu_);
                    j->held = held;
                    job_bytes_ += held;
                }
                Engine e(j->mat, ws, s);
                std::memset(&j->rep, 0, sizeof(j->rep));
                j->rep.struct_size = sizeof(j->rep);
                st = e.solve(j->k, j->p, j->eps, j->seed, j->opts, j->U, j->ritz, &j->rep, &j->cancel);
                cudaStreamSynchronize(s);
            } catch (const Error &err) {
                st = err.st;
                j->error = lra_last_error();
                cudaStreamSynchronize(s);
            } catch (...) {
                st = LRA_ECUDA;
                cudaStreamSynchronize(s);
            }
        }
        {
            std::lock_guard<std::mutex> g(mu_);
            j->status = st;
            j->rep.status = st;
            j->state = Job::DONE;
            reserved_ -= j->footprint;
            job_bytes_ -= j->held;  // the workspace is freed; unpolled results count as outside memory
            j->held = 0;
            j->mat->busy.fetch_sub(1);
        }
        cv_done_.notify_all();
        cv_work_.notify_all();
    }
}

lra_status Server::submit(lra_mat *mat, int k, int p, double eps, uint64_t seed, const Opts &o,
                          lra_job *out) {
    auto j = std::make_shared<Job>();
    j->mat = mat;
    j->k = k;
    j->p = p;
    j->eps = eps;
    j->seed = seed;
    j->opts = o;
    j->opts.trace_E = nullptr;  // the caller's trace buffer is not kept across calls
    j->opts.trace_cap = 0;
    j->footprint = job_footprint(mat, k, p, o);
    {
        std::lock_guard<std::mutex> g(mu_);
        if (j->footprint > idle_capacity_locked()) {
            set_error("job footprint exceeds the device memory available to the request loop");
            return LRA_ENOMEM;
        }
        j->id = next_id_++;
        mat->busy.fetch_add(1);
        jobs_[j->id] = j;
        queue_.push_back(j);
    }
    cv_work_.notify_one();
    *out = j->id;
    return LRA_OK;
}

lra_status Server::poll(lra_job id, int timeout_ms, float *U, double *ritz, lra_report *rep) {
    std::shared_ptr<Job> j;
    {
        std::unique_lock<std::mutex> lk(mu_);
        auto it = jobs_.find(id);
        if (it == jobs_.end()) {
            set_error("unknown job");
            return LRA_EINVAL;
        }
        j = it->second;
        auto done = [&] { return j->state == Job::DONE; };
        if (!done()) {
            if (timeout_ms == 0) return LRA_EAGAIN;
            if (timeout_ms < 0)
                cv_done_.wait(lk, done);
            else if (!cv_done_.wait_for(lk, std::chrono::milliseconds(timeout_ms), done))
                return LRA_ETIMEOUT;
        }
        jobs_.erase(id);
    }
    lra_status st = j->status;
    try {
        if (j->U && U && (st == LRA_OK || st == LRA_ENOTCONV))
            LRA_CUDA(cudaMemcpy(U, j->U, j->U_bytes, cudaMemcpyDefault));
        if (j->ritz && ritz && (st == LRA_OK || st == LRA_ENOTCONV))
            LRA_CUDA(cudaMemcpy(ritz, j->ritz, j->ritz_bytes, cudaMemcpyDefault));
    } catch (const Error &e) {
        st = e.st;
    }
    if (rep) {
        const size_t sz = std::min(rep->struct_size ? rep->struct_size : sizeof(j->rep), sizeof(j->rep));
        std::memcpy(rep, &j->rep, sz);
        rep->struct_size = sz;
    }
    if (j->U) dev_free(ctx_, j->U, j->U_bytes, j->stream);
    if (j->ritz) dev_free(ctx_, j->ritz, j->ritz_bytes, j->stream);
    j->U = nullptr;
    j->ritz = nullptr;
    if (!j->error.empty()) set_error(j->error);
    return st;
}

lra_status Server::cancel(lra_job id) {
    std::lock_guard<std::mutex> g(mu_);
    auto it = jobs_.find(id);
    if (it == jobs_.end()) {
        set_error("unknown job");
        return LRA_EINVAL;
    }
    auto j = it->second;
    j->cancel.store(1);
    if (j->state == Job::QUEUED) {
        for (auto q = queue_.begin(); q != queue_.end(); ++q) {
            if (*q == j) {
                queue_.erase(q);
                break;
            }
        }
        j->state = Job::DONE;
        j->status = LRA_ECANCELLED;
        j->mat->busy.fetch_sub(1);
        cv_done_.notify_all();
    }
    return LRA_OK;
}

}  // namespace lra

using namespace lra;

extern "C" {

lra_status lra_submit(lra_ctx *ctx, lra_mat *mat, int k, int p, double eps, uint64_t seed,
                      const lra_options *opt, lra_job *out) {
    if (!ctx || !mat || !out || mat->ctx != ctx) {
        set_error("null argument or matrix of another context");
        return LRA_EINVAL;
    }
    if (!(k >= 1 && k < p && p < mat->d) || p > mat->n || !(eps > 0.0 && eps < 1.0)) {
        set_error("need 1 <= k < p < d, p <= n, 0 < eps < 1");
        return LRA_EINVAL;
    }
    if (p > LRA_MAX_P) {
        set_error("p > LRA_MAX_P");
        return LRA_EUNSUPPORTED;
    }
    try {
        const Opts o = read_opts(opt, mat->storage);
        if (o.partition) {
            // Algorithm 6's stages allocate their deflation buffers (U^T X, the
            // deflated sampling tables, the inner loop's deflated columns) as they
            // go, which admission by a fixed footprint does not account for
            set_error("the request loop runs the q = k path; partition = 1 needs lra_solve");
            return LRA_EUNSUPPORTED;
        }
        {
            std::lock_guard<std::recursive_mutex> lk(ctx->mu);
            if (!ctx->server) {
                int prev = -1;
                cudaGetDevice(&prev);
                if (prev != ctx->device) LRA_CUDA(cudaSetDevice(ctx->device));
                ctx->server.reset(new Server(ctx, env_int("LRA_SERVE_SLOTS", 8)));
                if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
            }
        }
        return ctx->server->submit(mat, k, p, eps, seed, o, out);
    } catch (const Error &e) {
        return e.st;
    } catch (...) {
        set_error("unexpected exception");
        return LRA_ECUDA;
    }
}

lra_status lra_poll(lra_ctx *ctx, lra_job job, int timeout_ms, float *U, double *ritz, lra_report *rep) {
    if (!ctx || !ctx->server) {
        set_error("no request loop on this context");
        return LRA_EINVAL;
    }
    return ctx->server->poll(job, timeout_ms, U, ritz, rep);
}

lra_status lra_cancel(lra_ctx *ctx, lra_job job) {
    if (!ctx || !ctx->server) {
        set_error("no request loop on this context");
        return LRA_EINVAL;
    }
    return ctx->server->cancel(job);
}

}  // extern "C"
