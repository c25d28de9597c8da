// Host-side objects of the library: contexts, matrices, per-solve workspaces
// and the Engine that chains the kernels into the method's steps.
#pragma once

#include <atomic>
#include <condition_variable>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "kernels.cuh"

namespace lra {
class Server;
}

struct lra_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    size_t budget = 0;               // 0 = unlimited
    std::atomic<size_t> used{0};     // device bytes allocated through this context
    std::recursive_mutex mu;         // serialises step entry points and lra_solve
    std::atomic<int> nmats{0};
    std::unique_ptr<lra::Server> server;
};

struct lra_mat {
    lra_ctx *ctx = nullptr;
    int64_t d = 0, n = 0, dpad = 0;
    lra_dtype storage = LRA_F32;
    void *X = nullptr;     // storage dtype, dpad x n column-major
    float *X32 = nullptr;  // FP32 copy (== X when storage is FP32)
    // FP32 storage: BF16 pair (x = hi + lo + r, |r| <= 2^-17 |x|) streamed by the
    // tensor-core X passes; null for BF16 storage
    __nv_bfloat16 *Xh = nullptr, *Xl = nullptr;
    // FP16 storage: X holds fp16(xscale x) with xscale a power of two that puts
    // max |x| in [2^14, 2^15) (FP16's normal range starts at 2^-14); every pass
    // over X divides it out again (the X passes, column norms, inner steps)
    float xscale = 1.0f;
    // sparse X (X == nullptr): CSR of the d rows, compressed columns x_i, and
    // the row work list of X Y (item = (row, segment of kSparseSeg entries))
    struct Sparse {
        int64_t nnz = 0, nitems = 0;
        int64_t *rowptr = nullptr, *colptr = nullptr, *item_off = nullptr;
        int32_t *colidx = nullptr, *rowidx = nullptr;
        float *val = nullptr, *cval = nullptr;
        int2 *items = nullptr;
    };
    Sparse *sp = nullptr;
    // setup cache (a0)
    std::mutex setup_mu;
    bool have_norms = false;
    double *norm2 = nullptr;  // device, n
    double fro2 = 0.0, maxn = 0.0;
    double *dev_sm = nullptr;  // device [sum, max]
    struct Table {
        bool ok = false;
        uint64_t *cum = nullptr;
        float *c = nullptr;
        uint64_t total = 0;
        double kappa = 0.0;
    } table[2];
    std::atomic<int> busy{0};
};

namespace lra {

// Device allocation charged to a context's budget (stream-ordered when s != nullptr).
void *dev_alloc(lra_ctx *ctx, size_t bytes, cudaStream_t s = nullptr);
void dev_free(lra_ctx *ctx, void *p, size_t bytes, cudaStream_t s = nullptr);

struct Opts {
    int shift_policy = LRA_SHIFT_PAPER;
    double lambda = 0.0, delta = 0.0;
    double theta_eta = 0.25, theta_m = 2.0, tau = 0.0;
    int max_epochs = 60;
    int64_t m_max = 0;
    int min_outer = 3, max_outer = 2000, fixed_epochs = 0;
    int sampling = LRA_SAMPLE_IMPORTANCE, warm_start = 1, max_shift_rounds = 30;
    double lambda1_hat = 0.0;
    double *trace_E = nullptr;
    int trace_cap = 0;
    int profile = 0;
    int batch = 1;
    int acc = 0;               // accelerated solves (proximal-point loop around SVRG)
    double acc_theta = 0.5;
    int acc_max_outer = 200;
    int64_t acc_target = 0;    // samples per epoch the proximal weight aims for; 0 = n
    int partition = 0;         // 1: Algorithm 6 with adaptive partitioning and deflation
    int part_max_iters = 2000; // cap on Algorithm 3's iteration count
    int64_t wait_cycles = 0;   // tensor-core pipeline wait limit (0 = the kernels' default)
};

// CUDA-event timing of individual kernel launches on the engine's stream.
class KernelTimer {
   public:
    enum Kind { XTW = 0, XY = 1, INNER = 2, RITZ = 3, EIG = 4, QR = 5, WARM = 6, EPI = 7, NKIND = 8 };
    explicit KernelTimer(cudaStream_t s) : s_(s) {}
    ~KernelTimer();
    void begin(Kind k, int cols);
    void end();
    // summed milliseconds, launch counts and processed columns per kind
    void collect(double ms[NKIND], int64_t launches[NKIND], int64_t cols[NKIND]);

   private:
    size_t event();
    struct Rec {
        int kind, cols;
        size_t e0, e1;
    };
    cudaStream_t s_;
    std::vector<cudaEvent_t> pool_;
    size_t used_ = 0;
    std::vector<Rec> recs_;
};
Opts read_opts(const lra_options *o, lra_dtype storage);

struct SolveInfo {
    int epochs = 0;
    int64_t inner_steps = 0;
    int64_t m = 0;
    double eta = 0.0;
    double residual = NAN;
    lra_status status = LRA_OK;
    // accelerated solves: subproblems solved, proximal weight, and the residual
    // ||(lambda I - A) W - B||_F read at the last subproblem's first anchor
    int outer = 0;
    double gamma = 0.0;
    double outer_res = NAN;
    bool outer_done = false;
};

// One subproblem of an accelerated solve: the system solved is
// ((lambda + gamma) I - A) W = B + gamma Z; nB = ||B||_F of the original system.
struct AccHook {
    double gamma, nB, sq;
    const float *Z;
};

struct Stats {
    int64_t solves = 0, epochs = 0, inner_steps = 0, x_passes = 0;
};

// Per-solve buffers on the device, sized for up to pmax columns.
struct Workspace {
    lra_ctx *ctx = nullptr;
    int64_t dpad = 0, n = 0;
    int pmax = 0, PPmax = 0;
    float *S = nullptr, *W = nullptr, *Wt = nullptr, *M = nullptr, *T1 = nullptr, *U = nullptr;
    float *Wr = nullptr, *Q = nullptr, *Y = nullptr, *Gp = nullptr;
    int nchunks = 0;  // capacity of Gp in dpad x PP chunks
    int nch = 1;      // chunks written by the last X Y pass
    double *gscr2 = nullptr;  // Gram scratch of the side stream
    cudaStream_t side = nullptr;          // second stream for work independent of the X passes
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    double *H = nullptr, *Hc = nullptr, *evals = nullptr, *evecs = nullptr, *eigwork = nullptr, *gscr = nullptr;
    double *Gm = nullptr, *norms = nullptr, *epi = nullptr, *dots = nullptr;
    float *Rinv = nullptr, *P = nullptr;
    float *Za = nullptr, *Wo = nullptr;  // accelerated solve: extrapolated point Z, previous W
    __nv_bfloat16 *Wb = nullptr, *Yb = nullptr;  // BF16 hi/lo operands of the tensor-core passes
    int64_t ldy = 0;
    int *status = nullptr;
    int *tcerr = nullptr;  // error word of the tensor-core kernels
    float *tcs = nullptr;  // scales of the FP16 tensor-core operands (2 + 3 PPmax)
    int32_t *idx = nullptr;
    float *cval = nullptr;
    int64_t idx_cap = 0;
    double *host = nullptr;  // pinned readback area
    int *hstat = nullptr;    // pinned CholeskyQR2 status flags
    std::vector<std::pair<void *, size_t>> allocs;

    // astream != nullptr: buffers come from the stream-ordered allocator on that
    // stream (no device-wide synchronisation on free; used by the request loop)
    cudaStream_t astream = nullptr;

    float *partial = nullptr;  // sparse X: per-segment rows of X Y (nitems x PP)
    int64_t sp_items = -1;

    // sp_items >= 0: buffers of a sparse X with that many row items (one G
    // chunk, no BF16 operands); -1: dense X
    Workspace(lra_ctx *c, int64_t dpad_, int64_t n_, int pmax_, cudaStream_t alloc_stream = nullptr,
              int64_t sp_items_ = -1);
    ~Workspace();
    void ensure_idx(int64_t m);
    template <typename T>
    T *alloc(size_t count) {
        const size_t bytes = std::max<size_t>(16, sizeof(T) * count);
        void *p = dev_alloc(ctx, bytes, astream);
        allocs.emplace_back(p, bytes);
        return static_cast<T *>(p);
    }
};

size_t workspace_bytes(int64_t dpad, int64_t n, int pmax, int64_t sp_items = -1);

// Deflation applied on the fly (Algorithm 6, Sec. 3): a stage's matrix is
// X' = (I - U U^T) X for the orthonormal columns U (dpad x c) of the earlier
// stages.  The Engine of such a stage projects the small operand before each
// X^T pass and the d x p result after each X pass, samples by the deflated
// column norms, and feeds its inner loop the deflated columns x_i - U g_i.
struct Deflation {
    const float *U = nullptr;
    int c = 0, PPc = 0;
    const float *Gt = nullptr;  // n x PPc row-major: row i = g_i = U^T x_i
    double *norm2 = nullptr;    // n: ||x_i||^2 - ||g_i||^2
    double *sm = nullptr;       // device [sum, max, kappa]
    double fro2 = 0.0, maxn = 0.0;
    lra_mat::Table table[2];
    float *V = nullptr;         // dpad x pmax: a projected block
    float *C = nullptr;         // c x pmax coefficients U^T V
    float *G0 = nullptr;        // dpad x PPmax row-major: projected X X^T W of an anchor
    float *cols = nullptr;      // dense X: deflated sampled columns, dpad x mcap
    int64_t mcap = 0;
    int32_t *iota = nullptr;    // 0, 1, ..., mcap - 1
    float *lk = nullptr;        // sparse X: 3 c PPmax floats of the inner loop
};

// Algorithm 6 with adaptive partitioning and deflation (partition.cu)
lra_status solve_partitioned(lra_mat *mat, int k, int p, double eps, uint64_t seed, const Opts &o, float *U,
                             double *ritz, lra_report *rep);
// the sp_items argument of a workspace for X products on `m`
inline int64_t ws_items(const lra_mat *m) { return m->sp ? m->sp->nitems : -1; }

class Engine {
   public:
    Engine(lra_mat *mat, Workspace &ws, cudaStream_t s) : mat_(mat), ws_(ws), s_(s) {}

    // a0 setup
    void ensure_norms();
    const lra_mat::Table &ensure_table(int mode);

    // X products on p columns (internal padded layouts)
    // Y n x PP rm; keep_hilo: also leave Y's BF16 hi/lo copy for a following X Y pass
    void xt_mul(const float *W, int p, float *Y, bool use32, bool keep_hilo = false);
    void x_mul(const float *Y, int p, float *G, bool use32);             // G dpad x p
    void a_apply(const float *W, int p, float *G);                       // G = X X^T W
    // G0 != nullptr: X X^T Wt precomputed (dpad x PP row-major), no X pass
    // acc != nullptr: the subproblem anchor of an accelerated solve (B is the
    // original right-hand side; M uses B + gamma Z; *nR2 = the original residual)
    void anchor(const float *Wt, const float *B, int p, double lam, float *M, const float *G0,
                double *nM2, double *nB2, const struct AccHook *acc = nullptr, double *nR2 = nullptr);
    // m steps of `batch` samples (idx / cval hold m * batch entries)
    void inner(float *W, const float *Wt, const float *M, int p, const int32_t *idx,
               const float *cval, int64_t m, double eta, double lam, int batch = 1);
    // deferred: enqueue the status read-back without waiting (check with qr_status()
    // after the next synchronisation of the stream)
    lra_status cholqr2(float *W, int p, bool deferred = false);
    lra_status qr_status() const;
    // -> ws.Q, ws.H, ws.evals, ws.evecs; passes = FP64 refinement passes of the eigensolver
    // with_xq: also leave X Q in ws.T1 and take H = S^T (X Q)
    void ritz(const float *S, int p, bool use32, int passes = 2, bool with_xq = false);
    void normalize(float *z);                      // one column, in place
    double dot1(const float *a, const float *b);   // host read

    void step_params(double lam, double mu, double l1up, double kappa, const Opts &o, double &eta,
                     int64_t &m) const;
    lra_status svrg_solve(const float *B, float *W, int p, double lam, double mu, double l1up,
                          uint64_t seed, int64_t solve_id, const Opts &o, const float *G0,
                          SolveInfo &info, const AccHook *acc = nullptr);
    // proximal weight of the accelerated solve (0: plain SVRG already balanced)
    double acc_gamma(double lam, double mu, double l1up, double kappa, const Opts &o) const;
    // accelerated solve; one solve id per subproblem (solve_count advances by info.outer)
    lra_status acc_solve(const float *B, float *W, int p, double lam, double mu, double l1up,
                         uint64_t seed, int64_t &solve_count, const Opts &o, const float *G0,
                         SolveInfo &info);
    // (lambda I - A)^{-1} B: acc_solve when o.acc is set, else svrg_solve
    lra_status solve_linear(const float *B, float *W, int p, double lam, double mu, double l1up,
                            uint64_t seed, int64_t &solve_count, const Opts &o, const float *G0,
                            SolveInfo &info);
    double lambda1_estimate(uint64_t seed);
    lra_status d_top_inverse(uint64_t seed, int rnd, double lam, double mu, double l1up,
                             const Opts &o, int64_t &solve_count, double &inv);
    lra_status shift_tune(uint64_t seed, double l1hat, double delta, const Opts &o,
                          int64_t &solve_count, double &lam, double &inv, double &mu, int &rounds,
                          std::vector<double> *history);
    lra_status delta_estimate(int k, int p, uint64_t seed, double &delta);
    lra_status solve(int k, int p, double eps, uint64_t seed, const Opts &o, float *U,
                     double *ritz, lra_report *rep, const std::atomic<int> *cancel);
    // Algorithm 1 on D = (lam I - A)^{-1} with p columns from the Gaussian start
    // (seed, INIT) and Rayleigh-Ritz with A every iteration, stopped on E_l with
    // k target columns and the rate floor r_floor (< 0: from the Ritz values).
    // Hard errors are returned; `status` is LRA_OK or LRA_ENOTCONV.  On return
    // S points at the final basis (ws.S or ws.W) and ws.evals / ws.evecs hold
    // its Ritz pairs with A.
    lra_status loop_d(int k, int p, double eps, uint64_t seed, double lam, double mu, double l1up,
                      const Opts &o, int64_t &solve_count, double r_floor, float *&S, int &ell,
                      std::vector<double> &E, lra_status &status, lra_report &R,
                      const std::atomic<int> *cancel);
    // Algorithm 3 on A with kk vectors: L = min(ceil(eps^-1 ln(d/eps)), cap) block
    // power steps from the start (seed, BLOCK, 0), then the Ritz values (host, desc)
    lra_status alg3_a(int kk, double eps, int cap, uint64_t seed, double *vals, int &iters);
    // Algorithm 3 on D = (lam I - A)^{-1} with kk vectors from (seed, BLOCK, 2),
    // every product a solve warm-started by the previous iteration's Galerkin
    // projection; values are eigenvalue estimates of D (host, desc)
    lra_status alg3_d(int kk, double eps, int cap, uint64_t seed, double lam, double mu, double l1up,
                      double l1hat, const Opts &o, int64_t &solve_count, double *vals, int &iters);
    // Algorithm 1 on A with b columns (no oversampling) from (seed, BLOCK, 1),
    // Rayleigh-Ritz with A every iteration, stopped on E with rate floor r_floor;
    // the Ritz vectors are left in ws.U (b columns), values in ws.host[0..b)
    lra_status power_block(int b, double eps, double r_floor, uint64_t seed, const Opts &o, int &iters,
                           lra_status &status);

    void sync();
    void check_tc();  // raise if a tensor-core kernel reported a timed-out wait
    // ||X||_F^2 of the matrix the engine works on (the deflated one under defl)
    double fro2() const { return defl ? defl->fro2 : mat_->fro2; }
    Stats stats;
    KernelTimer *timer = nullptr;
    Deflation *defl = nullptr;  // non-null: the engine works on (I - U U^T) X
    long long tc_wait_ = 0;  // pipeline wait limit of the tensor-core passes (0 = default)
    const float *gscale_ = nullptr;  // per-column factor of the last X Y pass's partials (FP16 storage)

   private:
    // tensor-core passes: BF16 X, or the BF16 pair of an FP32 X; the exact FP32
    // values (use32) go through the CUDA-core kernels
    bool tc(bool use32) const {
        return !use32 && !mat_->sp && (mat_->storage == LRA_BF16 || mat_->storage == LRA_F16 || mat_->Xh != nullptr);
    }
    const void *tcx() const { return mat_->Xh ? static_cast<const void *>(mat_->Xh) : mat_->X; }
    // G-partials of one X Y pass into ws.Gp; Y32 == nullptr means ws.Yb already holds Y
    void xy_pass(const float *Y32, int p, bool use32);
    const void *xptr(bool use32) const { return use32 ? (const void *)mat_->X32 : mat_->X; }
    // V <- (I - U U^T) V for a dpad x p column-major block (no-op without defl)
    void project(float *V, int p);
    const lra_mat::Table &defl_table(int mode);
    lra_dtype xdt(bool use32) const { return use32 ? LRA_F32 : mat_->storage; }
    lra_mat *mat_;
    Workspace &ws_;
    cudaStream_t s_;
};

}  // namespace lra
