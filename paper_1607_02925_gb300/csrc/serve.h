// Request loop: continuous batching of many rank-k solves on one GPU.
//
// Jobs enter a FIFO queue.  A fixed pool of worker threads, each owning a CUDA
// stream, admits the first queued job whose device-memory footprint fits what
// the context has left, runs it with the same engine as lra_solve (its own
// workspace from the stream-ordered allocator), and publishes the result.
// Jobs admitted while others run overlap on the GPU; since no reduction order
// depends on co-running work, a job's result is the same alone and in the mix.
#pragma once

#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "engine.h"

namespace lra {

struct Job {
    lra_job id = 0;
    lra_mat *mat = nullptr;
    int k = 0, p = 0;
    double eps = 0.0;
    uint64_t seed = 0;
    Opts opts;
    size_t footprint = 0;
    enum State { QUEUED, RUNNING, DONE } state = QUEUED;
    lra_status status = LRA_OK;
    std::atomic<int> cancel{0};
    cudaStream_t stream = nullptr;  // the worker stream that ran the job
    float *U = nullptr;      // device, d x k (column-major, leading dim d)
    double *ritz = nullptr;  // device, k
    size_t U_bytes = 0, ritz_bytes = 0;
    size_t held = 0;          // bytes counted in Server::job_bytes_ while the job runs
    lra_report rep{};
    std::string error;
};

class Server {
   public:
    explicit Server(lra_ctx *ctx, int slots);
    ~Server();
    lra_status submit(lra_mat *mat, int k, int p, double eps, uint64_t seed, const Opts &o, lra_job *out);
    lra_status poll(lra_job job, int timeout_ms, float *U, double *ritz, lra_report *rep);
    lra_status cancel(lra_job job);

   private:
    void worker(int slot);
    std::shared_ptr<Job> admit_locked();
    size_t idle_capacity_locked() const;
    size_t capacity_locked() const;

    lra_ctx *ctx_;
    std::mutex mu_;
    std::condition_variable cv_work_, cv_done_;
    std::deque<std::shared_ptr<Job>> queue_;
    std::map<lra_job, std::shared_ptr<Job>> jobs_;
    size_t reserved_ = 0;    // footprints of running jobs
    size_t limit_ = 0;       // device bytes the context may reach (budget, or used + 90% of free at start)
    size_t job_bytes_ = 0;   // bytes the running jobs hold (workspace and result buffers)
    lra_job next_id_ = 1;
    bool stop_ = false;
    std::vector<std::thread> threads_;
    std::vector<cudaStream_t> streams_;
};

}  // namespace lra
