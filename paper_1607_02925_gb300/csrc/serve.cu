// Request loop entry points (lra_submit / lra_poll / lra_cancel).
#include "serve.h"

namespace lra {
Server::Server(lra_ctx *ctx) { (void)ctx; }
Server::~Server() {}
}  // namespace lra

extern "C" {

lra_status lra_submit(lra_ctx *ctx, lra_mat *mat, int k, int p, double eps, uint64_t seed,
                      const lra_options *opt, lra_job *out) {
    (void)ctx; (void)mat; (void)k; (void)p; (void)eps; (void)seed; (void)opt; (void)out;
    lra::set_error("request loop not built yet");
    return LRA_EUNSUPPORTED;
}

lra_status lra_poll(lra_ctx *ctx, lra_job job, int timeout_ms, float *U, double *ritz, lra_report *rep) {
    (void)ctx; (void)job; (void)timeout_ms; (void)U; (void)ritz; (void)rep;
    lra::set_error("request loop not built yet");
    return LRA_EUNSUPPORTED;
}

lra_status lra_cancel(lra_ctx *ctx, lra_job job) {
    (void)ctx; (void)job;
    lra::set_error("request loop not built yet");
    return LRA_EUNSUPPORTED;
}

}  // extern "C"
