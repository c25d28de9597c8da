// C ABI entry points (include/lra.h): argument validation, object lifetime,
// conversion between the caller's layouts (leading dimension d) and the
// library's padded device layouts, and error-status translation.
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "engine.h"
#include "serve.h"

namespace lra {

static thread_local std::string g_last_error;
static thread_local int64_t g_launches = 0;

void set_error(const std::string &msg) { g_last_error = msg; }
void count_launch() { ++g_launches; }
int64_t launches_of_thread() { return g_launches; }

void ensure_smem(const void *kernel, int bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, int> limit;  // (device, kernel) -> bytes set
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(mu);
    int &cur = limit[{dev, kernel}];
    if (bytes > cur) {
        LRA_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        cur = bytes;
    }
}

}  // namespace lra

using namespace lra;

#define LRA_TRY(...)                                         \
    try {                                                    \
        __VA_ARGS__                                          \
    } catch (const lra::Error &e__) {                        \
        return e__.st;                                       \
    } catch (const std::bad_alloc &) {                       \
        lra::set_error("host allocation failed");            \
        return LRA_ENOMEM;                                   \
    } catch (...) {                                          \
        lra::set_error("unexpected exception");              \
        return LRA_ECUDA;                                    \
    }

static lra_status einval(const char *msg) {
    set_error(msg);
    return LRA_EINVAL;
}

namespace {

// Scoped device selection.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) LRA_CUDA(cudaSetDevice(dev));
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

size_t dtype_size(lra_dtype t) {
    switch (t) {
        case LRA_F32: return 4;
        case LRA_BF16: return 2;
        case LRA_F16: return 2;
        case LRA_F64: return 8;
    }
    return 0;
}

// Caller d x p block (leading dimension d) <-> padded device block (dpad).
struct Padded {
    lra_ctx *ctx;
    float *p = nullptr;
    size_t bytes = 0;
    Padded(lra_ctx *c, int64_t dpad, int cols) : ctx(c) {
        bytes = sizeof(float) * dpad * std::max(cols, 1);
        p = static_cast<float *>(dev_alloc(ctx, bytes));
        LRA_CUDA(cudaMemsetAsync(p, 0, bytes, ctx->stream));
    }
    ~Padded() {
        if (p) {
            cudaStreamSynchronize(ctx->stream);
            dev_free(ctx, p, bytes);
        }
    }
    void upload(const float *src, int64_t d, int64_t dpad, int cols) {
        LRA_CUDA(cudaMemcpy2DAsync(p, sizeof(float) * dpad, src, sizeof(float) * d, sizeof(float) * d,
                                   cols, cudaMemcpyDefault, ctx->stream));
    }
    void download(float *dst, int64_t d, int64_t dpad, int cols) {
        LRA_CUDA(cudaMemcpy2DAsync(dst, sizeof(float) * d, p, sizeof(float) * dpad, sizeof(float) * d,
                                   cols, cudaMemcpyDefault, ctx->stream));
    }
};

lra_status check_mat(const lra_mat *m) {
    if (!m || !m->ctx || (!m->X && !m->sp)) return einval("null matrix");
    return LRA_OK;
}

}  // namespace

extern "C" {

void lra_options_default(lra_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->struct_size = sizeof(*opt);
    opt->shift_policy = LRA_SHIFT_PAPER;
    opt->theta_eta = 0.25;
    opt->theta_m = 2.0;
    opt->tau = 0.0;
    opt->max_epochs = 60;
    opt->m_max = 0;
    opt->min_outer = 3;
    opt->max_outer = 2000;
    opt->fixed_epochs = 0;
    opt->sampling = LRA_SAMPLE_IMPORTANCE;
    opt->warm_start = 1;
    opt->max_shift_rounds = 30;
    opt->batch = 1;
    opt->acc = 0;
    opt->acc_theta = 0.5;
    opt->acc_max_outer = 200;
    opt->acc_target = 0;
    opt->partition = 0;
    opt->part_max_iters = 2000;
    opt->wait_cycles = 0;
}

const char *lra_status_str(lra_status s) {
    switch (s) {
        case LRA_OK: return "LRA_OK";
        case LRA_EINVAL: return "LRA_EINVAL";
        case LRA_ENOMEM: return "LRA_ENOMEM";
        case LRA_ECUDA: return "LRA_ECUDA";
        case LRA_ENOTCONV: return "LRA_ENOTCONV";
        case LRA_EDIVERGED: return "LRA_EDIVERGED";
        case LRA_ENUMERIC: return "LRA_ENUMERIC";
        case LRA_ETIMEOUT: return "LRA_ETIMEOUT";
        case LRA_EAGAIN: return "LRA_EAGAIN";
        case LRA_EBUSY: return "LRA_EBUSY";
        case LRA_ECANCELLED: return "LRA_ECANCELLED";
        case LRA_EUNSUPPORTED: return "LRA_EUNSUPPORTED";
    }
    return "LRA_UNKNOWN";
}

const char *lra_last_error(void) { return g_last_error.c_str(); }

uint64_t lra_stream_key(uint64_t seed, uint64_t stream, uint64_t a, uint64_t b) {
    return stream_key(seed, stream, a, b);
}

lra_status lra_init(int device, size_t hbm_budget_bytes, lra_ctx **out) {
    if (!out) return einval("out is NULL");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        set_error("no CUDA device");
        return LRA_ECUDA;
    }
    if (device < 0 || device >= ndev) return einval("device out of range");
    LRA_TRY({
        DeviceGuard g(device);
        auto *ctx = new lra_ctx();
        ctx->device = device;
        ctx->budget = hbm_budget_bytes;
        const cudaError_t e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete ctx;
            set_error(std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
            return LRA_ECUDA;
        }
        *out = ctx;
        return LRA_OK;
    })
}

void *lra_ctx_stream(lra_ctx *ctx) { return ctx ? (void *)ctx->stream : nullptr; }

lra_status lra_finalize(lra_ctx *ctx) {
    if (!ctx) return einval("null context");
    if (ctx->nmats.load() > 0) {
        set_error("matrices still alive");
        return LRA_EBUSY;
    }
    LRA_TRY({
        DeviceGuard g(ctx->device);
        ctx->server.reset();
        cudaStreamSynchronize(ctx->stream);
        cudaStreamDestroy(ctx->stream);
        delete ctx;
        return LRA_OK;
    })
}

lra_status lra_create_dense(lra_ctx *ctx, int64_t d, int64_t n, lra_dtype src, const void *X,
                            int64_t ld, int src_on_device, lra_dtype storage, lra_mat **out) {
    if (!ctx || !out || !X) return einval("null argument");
    if (d < 1 || n < 2 || ld < d) return einval("need d >= 1, n >= 2, ld >= d");
    if (n > (int64_t)INT32_MAX) return einval("n must fit in int32");
    if (src != LRA_F32 && src != LRA_BF16 && src != LRA_F64) {
        set_error("source dtype must be F32, BF16 or F64");
        return LRA_EUNSUPPORTED;
    }
    if (storage != LRA_F32 && storage != LRA_BF16 && storage != LRA_F16) {
        set_error("storage dtype must be F32, BF16 or F16");
        return LRA_EUNSUPPORTED;
    }
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    lra_mat *m = nullptr;
    void *stage = nullptr;
    size_t stage_bytes = 0;
    LRA_TRY({
        DeviceGuard g(ctx->device);
        m = new lra_mat();
        m->ctx = ctx;
        m->d = d;
        m->n = n;
        m->dpad = round_up(d, kRowPad);
        m->storage = storage;
        const size_t ncell = (size_t)m->dpad * n;
        try {
            m->X32 = static_cast<float *>(dev_alloc(ctx, sizeof(float) * ncell));
            if (storage == LRA_BF16 || storage == LRA_F16) m->X = dev_alloc(ctx, sizeof(__nv_bfloat16) * ncell);
            else m->X = m->X32;
            const size_t es = dtype_size(src);
            const cudaStream_t s = ctx->stream;
            const bool dev = src_on_device != 0;
            // columns per chunk: about 256 MB of source
            const int64_t cols = std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)((256ull << 20) / (es * ld))));
            if (!dev) {
                stage_bytes = es * ld * cols;
                stage = dev_alloc(ctx, stage_bytes);
            }
            for (int64_t c0 = 0; c0 < n; c0 += cols) {
                const int64_t nc = std::min(cols, n - c0);
                const unsigned char *srcp = static_cast<const unsigned char *>(X) + es * ld * c0;
                const void *from = srcp;
                if (!dev) {
                    LRA_CUDA(cudaMemcpyAsync(stage, srcp, es * ld * nc, cudaMemcpyHostToDevice, s));
                    from = stage;
                }
                convert_to_f32(s, from, src, ld, d, nc, m->X32 + (size_t)c0 * m->dpad, m->dpad);
                if (storage == LRA_BF16) {
                    // BF16 storage = round-to-nearest-even of the FP32 copy
                    convert_to_bf16(s, m->X32 + (size_t)c0 * m->dpad, LRA_F32, m->dpad, m->dpad, nc,
                                    static_cast<__nv_bfloat16 *>(m->X) + (size_t)c0 * m->dpad, m->dpad);
                }
                if (!dev) LRA_CUDA(cudaStreamSynchronize(s));
            }
            if (storage == LRA_F16) {
                // FP16 storage: fp16(xscale x), xscale a power of two that puts
                // max |x| in [2^14, 2^15) (the FP32 copy keeps the exact values)
                unsigned *word = static_cast<unsigned *>(dev_alloc(ctx, sizeof(unsigned)));
                try {
                    m->xscale = f16_storage_scale(s, m->X32, (int64_t)ncell, word);
                } catch (...) {
                    dev_free(ctx, word, sizeof(unsigned));
                    throw;
                }
                dev_free(ctx, word, sizeof(unsigned));
                to_f16(s, m->X32, (int64_t)ncell, m->xscale, static_cast<__half *>(m->X));
            }
            if (storage == LRA_F32) {
                // the tensor-core passes stream the FP32 values as a BF16 pair
                m->Xh = static_cast<__nv_bfloat16 *>(dev_alloc(ctx, sizeof(__nv_bfloat16) * ncell));
                m->Xl = static_cast<__nv_bfloat16 *>(dev_alloc(ctx, sizeof(__nv_bfloat16) * ncell));
                split_hilo(s, m->X32, (int64_t)ncell, m->Xh, m->Xl);
            }
            LRA_CUDA(cudaStreamSynchronize(s));
        } catch (...) {
            if (m->Xh) dev_free(ctx, m->Xh, sizeof(__nv_bfloat16) * ncell);
            if (m->Xl) dev_free(ctx, m->Xl, sizeof(__nv_bfloat16) * ncell);
            cudaStreamSynchronize(ctx->stream);
            if (stage) dev_free(ctx, stage, stage_bytes);
            if (m->X && m->X != m->X32) dev_free(ctx, m->X, sizeof(__nv_bfloat16) * ncell);
            if (m->X32) dev_free(ctx, m->X32, sizeof(float) * ncell);
            delete m;
            throw;
        }
        if (stage) dev_free(ctx, stage, stage_bytes);
        ctx->nmats.fetch_add(1);
        *out = m;
        return LRA_OK;
    })
}

namespace {

// Free every buffer of a sparse matrix record (null entries are skipped).
void free_sparse(lra_ctx *ctx, lra_mat *m) {
    auto *sp = m->sp;
    if (!sp) return;
    const int64_t d = m->d, n = m->n, dpad = m->dpad, nnz = sp->nnz;
    if (sp->rowptr) dev_free(ctx, sp->rowptr, sizeof(int64_t) * (d + 1));
    if (sp->colidx) dev_free(ctx, sp->colidx, sizeof(int32_t) * std::max<int64_t>(nnz, 1));
    if (sp->val) dev_free(ctx, sp->val, sizeof(float) * std::max<int64_t>(nnz, 1));
    if (sp->colptr) dev_free(ctx, sp->colptr, sizeof(int64_t) * (n + 1));
    if (sp->rowidx) dev_free(ctx, sp->rowidx, sizeof(int32_t) * std::max<int64_t>(nnz, 1));
    if (sp->cval) dev_free(ctx, sp->cval, sizeof(float) * std::max<int64_t>(nnz, 1));
    if (sp->item_off) dev_free(ctx, sp->item_off, sizeof(int64_t) * (dpad + 1));
    if (sp->items) dev_free(ctx, sp->items, sizeof(int2) * std::max<int64_t>(sp->nitems, 1));
    delete sp;
    m->sp = nullptr;
}

}  // namespace

lra_status lra_create_csr(lra_ctx *ctx, int64_t d, int64_t n, int64_t nnz, const int64_t *rowptr,
                          const int32_t *colidx, const float *val, int src_on_device, lra_mat **out) {
    if (!ctx || !out || !rowptr || (nnz > 0 && (!colidx || !val))) return einval("null argument");
    if (d < 1 || n < 2 || nnz < 0) return einval("bad shape");
    if (n > (int64_t)INT32_MAX || d > (int64_t)INT32_MAX) return einval("d and n must fit in int32");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    lra_mat *m = nullptr;
    LRA_TRY({
        DeviceGuard g(ctx->device);
        m = new lra_mat();
        m->ctx = ctx;
        m->d = d;
        m->n = n;
        m->dpad = round_up(d, kRowPad);
        m->storage = LRA_F32;
        m->sp = new lra_mat::Sparse();
        auto &sp = *m->sp;
        sp.nnz = nnz;
        const cudaStream_t s = ctx->stream;
        const cudaMemcpyKind kind = src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        const int64_t nz1 = std::max<int64_t>(nnz, 1);
        int64_t *cnt = nullptr, *scr = nullptr;
        int *cursor = nullptr, *bad = nullptr;
        const int64_t scr_len = sparse_scan_scratch(std::max(n, m->dpad));
        auto free_tmp = [&]() {
            cudaStreamSynchronize(s);
            if (cnt) dev_free(ctx, cnt, sizeof(int64_t) * std::max(n, m->dpad));
            if (scr) dev_free(ctx, scr, sizeof(int64_t) * scr_len);
            if (cursor) dev_free(ctx, cursor, sizeof(int) * n);
            if (bad) dev_free(ctx, bad, sizeof(int) * 4);
            cnt = scr = nullptr;
            cursor = bad = nullptr;
        };
        try {
            sp.rowptr = static_cast<int64_t *>(dev_alloc(ctx, sizeof(int64_t) * (d + 1)));
            sp.colidx = static_cast<int32_t *>(dev_alloc(ctx, sizeof(int32_t) * nz1));
            sp.val = static_cast<float *>(dev_alloc(ctx, sizeof(float) * nz1));
            LRA_CUDA(cudaMemcpyAsync(sp.rowptr, rowptr, sizeof(int64_t) * (d + 1), kind, s));
            if (nnz > 0) {
                LRA_CUDA(cudaMemcpyAsync(sp.colidx, colidx, sizeof(int32_t) * nnz, kind, s));
                LRA_CUDA(cudaMemcpyAsync(sp.val, val, sizeof(float) * nnz, kind, s));
            }
            bad = static_cast<int *>(dev_alloc(ctx, sizeof(int) * 4));
            csr_check(s, sp.rowptr, sp.colidx, sp.val, d, n, nnz, bad);
            int hb = 0;
            LRA_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
            LRA_CUDA(cudaStreamSynchronize(s));
            if (hb) {
                std::string why = "invalid CSR:";
                if (hb & 16) why += " rowptr[0] != 0 or rowptr[d] != nnz;";
                if (hb & 1) why += " row pointers decreasing or out of [0, nnz];";
                if (hb & 2) why += " column index out of [0, n);";
                if (hb & 4) why += " column indices not strictly increasing within a row;";
                if (hb & 8) why += " value not finite;";
                set_error(why);
                throw Error{LRA_EINVAL};
            }
            // compressed columns (the x_i of the inner loop and of X^T W)
            sp.colptr = static_cast<int64_t *>(dev_alloc(ctx, sizeof(int64_t) * (n + 1)));
            sp.rowidx = static_cast<int32_t *>(dev_alloc(ctx, sizeof(int32_t) * nz1));
            sp.cval = static_cast<float *>(dev_alloc(ctx, sizeof(float) * nz1));
            cnt = static_cast<int64_t *>(dev_alloc(ctx, sizeof(int64_t) * std::max(n, m->dpad)));
            scr = static_cast<int64_t *>(dev_alloc(ctx, sizeof(int64_t) * scr_len));
            cursor = static_cast<int *>(dev_alloc(ctx, sizeof(int) * n));
            csr_transpose(s, sp.rowptr, sp.colidx, sp.val, d, n, nnz, sp.colptr, sp.rowidx, sp.cval, cnt, cursor,
                          scr);
            // row work list of X Y
            sp.item_off = static_cast<int64_t *>(dev_alloc(ctx, sizeof(int64_t) * (m->dpad + 1)));
            sparse_row_items(s, sp.rowptr, d, m->dpad, kSparseSeg, cnt, sp.item_off, scr);
            LRA_CUDA(cudaMemcpyAsync(&sp.nitems, sp.item_off + m->dpad, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            LRA_CUDA(cudaStreamSynchronize(s));
            sp.items = static_cast<int2 *>(dev_alloc(ctx, sizeof(int2) * std::max<int64_t>(sp.nitems, 1)));
            sparse_fill_items(s, sp.item_off, m->dpad, sp.items);
            free_tmp();
        } catch (...) {
            free_tmp();
            free_sparse(ctx, m);
            delete m;
            throw;
        }
        ctx->nmats.fetch_add(1);
        *out = m;
        return LRA_OK;
    })
}

lra_status lra_mat_destroy(lra_mat *m) {
    if (!m) return einval("null matrix");
    if (m->busy.load() > 0) {
        set_error("matrix in use by a running job");
        return LRA_EBUSY;
    }
    lra_ctx *ctx = m->ctx;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    LRA_TRY({
        DeviceGuard g(ctx->device);
        cudaStreamSynchronize(ctx->stream);
        const size_t ncell = (size_t)m->dpad * m->n;
        free_sparse(ctx, m);
        if (m->X && m->X != m->X32) dev_free(ctx, m->X, sizeof(__nv_bfloat16) * ncell);
        if (m->X32) dev_free(ctx, m->X32, sizeof(float) * ncell);
        if (m->Xh) dev_free(ctx, m->Xh, sizeof(__nv_bfloat16) * ncell);
        if (m->Xl) dev_free(ctx, m->Xl, sizeof(__nv_bfloat16) * ncell);
        if (m->norm2) dev_free(ctx, m->norm2, sizeof(double) * m->n);
        if (m->dev_sm) dev_free(ctx, m->dev_sm, sizeof(double) * 4);
        for (auto &t : m->table) {
            if (t.cum) dev_free(ctx, t.cum, sizeof(uint64_t) * m->n);
            if (t.c) dev_free(ctx, t.c, sizeof(float) * m->n);
        }
        ctx->nmats.fetch_sub(1);
        delete m;
        return LRA_OK;
    })
}

lra_status lra_mat_info(const lra_mat *m, int64_t *d, int64_t *n, lra_dtype *storage, double *fro2) {
    if (check_mat(m) != LRA_OK) return LRA_EINVAL;
    if (d) *d = m->d;
    if (n) *n = m->n;
    if (storage) *storage = m->storage;
    if (fro2) {
        lra_mat *mm = const_cast<lra_mat *>(m);
        std::lock_guard<std::recursive_mutex> lk(mm->ctx->mu);
        LRA_TRY({
            DeviceGuard g(mm->ctx->device);
            Workspace ws(mm->ctx, mm->dpad, 1, 1);
            Engine e(mm, ws, mm->ctx->stream);
            e.ensure_norms();
            *fro2 = mm->fro2;
        })
    }
    return LRA_OK;
}

lra_status lra_solve(lra_mat *mat, int k, int p, double eps, uint64_t seed, const lra_options *opt,
                     float *U, double *ritz, lra_report *rep) {
    if (check_mat(mat) != LRA_OK) return LRA_EINVAL;
    if (!U || !ritz) return einval("U and ritz are required");
    if (!(k >= 1 && k < p && p < mat->d)) return einval("need 1 <= k < p < d");
    if (p > mat->n) return einval("need p <= n");
    if (p > LRA_MAX_P) {
        set_error("p > LRA_MAX_P");
        return LRA_EUNSUPPORTED;
    }
    if (!(eps > 0.0 && eps < 1.0)) return einval("need 0 < eps < 1");
    lra_ctx *ctx = mat->ctx;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    LRA_TRY({
        DeviceGuard g(ctx->device);
        const Opts o = read_opts(opt, mat->storage);
        if (o.shift_policy == LRA_SHIFT_PAPER && !(o.delta > 0) && p + 1 > LRA_MAX_P) {
            set_error("estimating Delta needs p + 1 <= LRA_MAX_P");
            return LRA_EUNSUPPORTED;
        }
        const int pmax = (o.shift_policy == LRA_SHIFT_PAPER && !(o.delta > 0)) ? p + 1 : p;
        mat->busy.fetch_add(1);
        struct Release {
            lra_mat *m;
            ~Release() { m->busy.fetch_sub(1); }
        } rel{mat};
        if (o.partition) {
            if (!(o.delta > 0) && p + 1 > LRA_MAX_P) {
                set_error("estimating Delta needs p + 1 <= LRA_MAX_P");
                return LRA_EUNSUPPORTED;
            }
            const lra_status st = solve_partitioned(mat, k, p, eps, seed, o, U, ritz, rep);
            if (st != LRA_OK && st != LRA_ENOTCONV && rep) rep->status = st;
            return st;
        }
        Workspace ws(ctx, mat->dpad, mat->n, pmax, nullptr, ws_items(mat));
        Engine e(mat, ws, ctx->stream);
        const lra_status st = e.solve(k, p, eps, seed, o, U, ritz, rep, nullptr);
        if (st != LRA_OK && st != LRA_ENOTCONV && rep) rep->status = st;
        return st;
    })
}

// ---------------------------------------------------------------------------
// Step entry points
// ---------------------------------------------------------------------------

lra_status lra_colnorms(lra_mat *mat, double *norm2, double *fro2) {
    if (check_mat(mat) != LRA_OK || !norm2) return einval("null argument");
    std::lock_guard<std::recursive_mutex> lk(mat->ctx->mu);
    LRA_TRY({
        DeviceGuard g(mat->ctx->device);
        Workspace ws(mat->ctx, mat->dpad, 1, 1);
        Engine e(mat, ws, mat->ctx->stream);
        e.ensure_norms();
        LRA_CUDA(cudaMemcpyAsync(norm2, mat->norm2, sizeof(double) * mat->n, cudaMemcpyDefault, mat->ctx->stream));
        LRA_CUDA(cudaStreamSynchronize(mat->ctx->stream));
        if (fro2) *fro2 = mat->fro2;
        return LRA_OK;
    })
}

lra_status lra_sampling_table(lra_ctx *ctx, int64_t n, const double *norm2, int mode, uint64_t *cum,
                              float *c, uint64_t *total, double *kappa) {
    if (!ctx || !norm2 || !cum || !c || n < 1) return einval("null argument");
    if (mode != LRA_SAMPLE_IMPORTANCE && mode != LRA_SAMPLE_UNIFORM) return einval("bad mode");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    void *scr = nullptr;
    size_t scr_bytes = 0;
    LRA_TRY({
        DeviceGuard g(ctx->device);
        const cudaStream_t s = ctx->stream;
        const int64_t nscr = std::max<int64_t>(ceil_div(n, 1024) + 16, ceil_div(n, 256) + 16);
        scr_bytes = sizeof(uint64_t) * nscr + sizeof(double) * 4;
        scr = dev_alloc(ctx, scr_bytes);
        double *sm = reinterpret_cast<double *>(static_cast<uint64_t *>(scr) + nscr);
        try {
            sum_max(s, norm2, n, sm, nullptr);
            sampling_table(s, norm2, n, mode, sm + 1, cum, c, sm + 2, static_cast<uint64_t *>(scr));
            uint64_t tot = 0;
            double kp = 0, sum = 0;
            LRA_CUDA(cudaMemcpyAsync(&tot, cum + n - 1, sizeof(tot), cudaMemcpyDeviceToHost, s));
            LRA_CUDA(cudaMemcpyAsync(&kp, sm + 2, sizeof(kp), cudaMemcpyDeviceToHost, s));
            LRA_CUDA(cudaMemcpyAsync(&sum, sm, sizeof(sum), cudaMemcpyDeviceToHost, s));
            LRA_CUDA(cudaStreamSynchronize(s));
            if (!std::isfinite(sum)) {
                dev_free(ctx, scr, scr_bytes);
                return einval("a column norm is not finite");
            }
            if (total) *total = tot;
            if (kappa) *kappa = kp;
        } catch (...) {
            cudaStreamSynchronize(s);
            dev_free(ctx, scr, scr_bytes);
            throw;
        }
        dev_free(ctx, scr, scr_bytes);
        return LRA_OK;
    })
}

lra_status lra_sample(lra_ctx *ctx, int64_t n, const uint64_t *cum, uint64_t total, uint64_t key,
                      int64_t m, int32_t *idx) {
    (void)total;
    if (!ctx || !cum || (m > 0 && !idx) || n < 1 || m < 0) return einval("bad argument");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    LRA_TRY({
        DeviceGuard g(ctx->device);
        sample(ctx->stream, cum, n, key, m, idx, nullptr, nullptr);
        LRA_CUDA(cudaStreamSynchronize(ctx->stream));
        return LRA_OK;
    })
}

lra_status lra_gaussian_block(lra_ctx *ctx, uint64_t seed, uint64_t stream, uint64_t a, int64_t d, int p,
                              float *out) {
    if (!ctx || !out || d < 1 || p < 1) return einval("bad argument");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    LRA_TRY({
        DeviceGuard g(ctx->device);
        gaussian(ctx->stream, stream_key(seed, stream, a, 0), d, d, p, out);
        LRA_CUDA(cudaStreamSynchronize(ctx->stream));
        return LRA_OK;
    })
}

lra_status lra_anchor(lra_mat *mat, int p, const float *Wt, const float *B, double lambda, float *M,
                      double *normM2, double *normB2) {
    if (check_mat(mat) != LRA_OK || !Wt || !B || !M) return einval("null argument");
    if (p < 1 || p > LRA_MAX_P) return einval("bad p");
    lra_ctx *ctx = mat->ctx;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    LRA_TRY({
        DeviceGuard g(ctx->device);
        Workspace ws(ctx, mat->dpad, mat->n, p, nullptr, ws_items(mat));
        Engine e(mat, ws, ctx->stream);
        Padded pw(ctx, mat->dpad, p), pb(ctx, mat->dpad, p), pm(ctx, mat->dpad, p);
        pw.upload(Wt, mat->d, mat->dpad, p);
        pb.upload(B, mat->d, mat->dpad, p);
        double a = 0, b = 0;
        e.anchor(pw.p, pb.p, p, lambda, pm.p, nullptr, &a, &b);
        pm.download(M, mat->d, mat->dpad, p);
        LRA_CUDA(cudaStreamSynchronize(ctx->stream));
        if (normM2) *normM2 = a;
        if (normB2) *normB2 = b;
        return LRA_OK;
    })
}

lra_status lra_xt_mul(lra_mat *mat, int p, const float *W, float *Y, int use_f32_copy) {
    if (check_mat(mat) != LRA_OK || !W || !Y) return einval("null argument");
    if (p < 1 || p > LRA_MAX_P) return einval("bad p");
    lra_ctx *ctx = mat->ctx;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    LRA_TRY({
        DeviceGuard g(ctx->device);
        Workspace ws(ctx, mat->dpad, mat->n, p, nullptr, ws_items(mat));
        Engine e(mat, ws, ctx->stream);
        Padded pw(ctx, mat->dpad, p);
        pw.upload(W, mat->d, mat->dpad, p);
        e.xt_mul(pw.p, p, ws.Q, use_f32_copy != 0);
        // row-major n x PP -> column-major n x p
        LRA_CUDA(cudaMemcpy2DAsync(Y, sizeof(float), ws.Q, sizeof(float) * pad_p(p), sizeof(float), mat->n,
                                   cudaMemcpyDefault, ctx->stream));
        for (int j = 1; j < p; ++j)
            LRA_CUDA(cudaMemcpy2DAsync(Y + (size_t)j * mat->n, sizeof(float), ws.Q + j, sizeof(float) * pad_p(p),
                                       sizeof(float), mat->n, cudaMemcpyDefault, ctx->stream));
        LRA_CUDA(cudaStreamSynchronize(ctx->stream));
        return LRA_OK;
    })
}

lra_status lra_x_mul(lra_mat *mat, int p, const float *Y, float *G, int use_f32_copy) {
    if (check_mat(mat) != LRA_OK || !Y || !G) return einval("null argument");
    if (p < 1 || p > LRA_MAX_P) return einval("bad p");
    lra_ctx *ctx = mat->ctx;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    LRA_TRY({
        DeviceGuard g(ctx->device);
        Workspace ws(ctx, mat->dpad, mat->n, p, nullptr, ws_items(mat));
        Engine e(mat, ws, ctx->stream);
        const int PP = pad_p(p);
        LRA_CUDA(cudaMemsetAsync(ws.Y, 0, sizeof(float) * mat->n * PP, ctx->stream));
        for (int j = 0; j < p; ++j)
            LRA_CUDA(cudaMemcpy2DAsync(ws.Y + j, sizeof(float) * PP, Y + (size_t)j * mat->n, sizeof(float),
                                       sizeof(float), mat->n, cudaMemcpyDefault, ctx->stream));
        Padded pg(ctx, mat->dpad, p);
        e.x_mul(ws.Y, p, pg.p, use_f32_copy != 0);
        pg.download(G, mat->d, mat->dpad, p);
        LRA_CUDA(cudaStreamSynchronize(ctx->stream));
        return LRA_OK;
    })
}

lra_status lra_svrg_inner(lra_mat *mat, int p, float *W, const float *Wt, const float *M,
                          const int32_t *idx, int64_t m, const float *c, double eta, double lambda) {
    return lra_svrg_inner_batched(mat, p, W, Wt, M, idx, m, 1, c, eta, lambda);
}

lra_status lra_svrg_inner_batched(lra_mat *mat, int p, float *W, const float *Wt, const float *M,
                                  const int32_t *idx, int64_t m, int batch, const float *c, double eta,
                                  double lambda) {
    if (check_mat(mat) != LRA_OK || !W || !Wt || !M || (m > 0 && (!idx || !c))) return einval("null argument");
    if (p < 1 || p > LRA_MAX_P || m < 0) return einval("bad p or m");
    if (batch < 1 || batch > 16 || (batch & (batch - 1)) != 0) return einval("batch must be a power of two <= 16");
    const int64_t ns = m * batch;
    lra_ctx *ctx = mat->ctx;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    LRA_TRY({
        DeviceGuard g(ctx->device);
        Workspace ws(ctx, mat->dpad, 1, p);
        Engine e(mat, ws, ctx->stream);
        Padded pw(ctx, mat->dpad, p), pt(ctx, mat->dpad, p), pm(ctx, mat->dpad, p);
        pw.upload(W, mat->d, mat->dpad, p);
        pt.upload(Wt, mat->d, mat->dpad, p);
        pm.upload(M, mat->d, mat->dpad, p);
        // cval[t] = c[idx[t]], the sampler's output convention
        size_t cb = sizeof(float) * std::max<int64_t>(ns, 1);
        float *cval = static_cast<float *>(dev_alloc(ctx, cb));
        try {
            gather_c(ctx->stream, idx, c, ns, mat->n, cval, ws.status);
            int bad = 0;
            LRA_CUDA(cudaMemcpyAsync(&bad, ws.status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
            LRA_CUDA(cudaStreamSynchronize(ctx->stream));
            if (bad) {
                set_error("index out of range");
                throw Error{LRA_EINVAL};
            }
            e.inner(pw.p, pt.p, pm.p, p, idx, cval, m, eta, lambda, batch);
            pw.download(W, mat->d, mat->dpad, p);
            LRA_CUDA(cudaStreamSynchronize(ctx->stream));
        } catch (...) {
            cudaStreamSynchronize(ctx->stream);
            dev_free(ctx, cval, cb);
            throw;
        }
        dev_free(ctx, cval, cb);
        return LRA_OK;
    })
}

lra_status lra_svrg_solve(lra_mat *mat, int p, const float *B, float *W, double lambda, double mu,
                          double lambda1_up, uint64_t seed, int64_t solve_id, const lra_options *opt,
                          lra_solve_info *info) {
    if (check_mat(mat) != LRA_OK || !B || !W) return einval("null argument");
    if (p < 1 || p > LRA_MAX_P) return einval("bad p");
    if (!(mu > 0) || !(lambda > 0) || !(lambda1_up > 0)) return einval("need lambda, mu, lambda1_up > 0");
    lra_ctx *ctx = mat->ctx;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    LRA_TRY({
        DeviceGuard g(ctx->device);
        const Opts o = read_opts(opt, mat->storage);
        Workspace ws(ctx, mat->dpad, mat->n, p, nullptr, ws_items(mat));
        Engine e(mat, ws, ctx->stream);
        Padded pb(ctx, mat->dpad, p), pw(ctx, mat->dpad, p);
        pb.upload(B, mat->d, mat->dpad, p);
        pw.upload(W, mat->d, mat->dpad, p);
        SolveInfo si;
        int64_t sc = solve_id;
        const lra_status st = e.solve_linear(pb.p, pw.p, p, lambda, mu, lambda1_up, seed, sc, o, nullptr, si);
        pw.download(W, mat->d, mat->dpad, p);
        LRA_CUDA(cudaStreamSynchronize(ctx->stream));
        if (info) {
            info->epochs = si.epochs;
            info->inner_steps = si.inner_steps;
            info->m = si.m;
            info->eta = si.eta;
            info->residual = si.residual;
            info->status = si.status;
            info->outer = si.outer;
            info->gamma = si.gamma;
        }
        return st;
    })
}

lra_status lra_gram(lra_ctx *ctx, int64_t rows, int p, const float *A, int64_t lda, double *G) {
    if (!ctx || !A || !G || rows < 1 || p < 1 || p > LRA_MAX_P + 1 || lda < rows) return einval("bad argument");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    LRA_TRY({
        DeviceGuard g(ctx->device);
        const size_t sb = sizeof(double) * gram_scratch(p);
        double *scr = static_cast<double *>(dev_alloc(ctx, sb));
        try {
            gram(ctx->stream, A, rows, 1, lda, p, G, scr);
            LRA_CUDA(cudaStreamSynchronize(ctx->stream));
        } catch (...) {
            cudaStreamSynchronize(ctx->stream);
            dev_free(ctx, scr, sb);
            throw;
        }
        dev_free(ctx, scr, sb);
        return LRA_OK;
    })
}

lra_status lra_cholqr2(lra_ctx *ctx, int64_t d, int p, float *W) {
    if (!ctx || !W || d < 1 || p < 1 || p > LRA_MAX_P + 1 || p > d) return einval("bad argument");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    LRA_TRY({
        DeviceGuard g(ctx->device);
        // a throwaway matrix record gives the engine its row padding
        lra_mat fake;
        fake.ctx = ctx;
        fake.d = d;
        fake.n = 1;
        fake.dpad = round_up(d, kRowPad);
        Workspace ws(ctx, fake.dpad, 1, p);
        Engine e(&fake, ws, ctx->stream);
        Padded pw(ctx, fake.dpad, p);
        pw.upload(W, d, fake.dpad, p);
        const lra_status st = e.cholqr2(pw.p, p);
        pw.download(W, d, fake.dpad, p);
        LRA_CUDA(cudaStreamSynchronize(ctx->stream));
        return st;
    })
}

lra_status lra_sym_eig(lra_ctx *ctx, int p, const double *H, double *evals, double *evecs) {
    if (!ctx || !H || !evals || !evecs || p < 1 || p > LRA_MAX_P + 1) return einval("bad argument");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    LRA_TRY({
        DeviceGuard g(ctx->device);
        const size_t wb = sizeof(double) * sym_eig_work(p);
        double *work = static_cast<double *>(dev_alloc(ctx, wb));
        try {
            sym_eig(ctx->stream, H, p, evals, evecs, work);
            LRA_CUDA(cudaStreamSynchronize(ctx->stream));
        } catch (...) {
            cudaStreamSynchronize(ctx->stream);
            dev_free(ctx, work, wb);
            throw;
        }
        dev_free(ctx, work, wb);
        return LRA_OK;
    })
}

lra_status lra_ritz(lra_mat *mat, int p, const float *S, int use_f32_copy, double *H, double *evals,
                    double *evecs) {
    if (check_mat(mat) != LRA_OK || !S || !evals || !evecs) return einval("null argument");
    if (p < 1 || p > LRA_MAX_P) return einval("bad p");
    lra_ctx *ctx = mat->ctx;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    LRA_TRY({
        DeviceGuard g(ctx->device);
        Workspace ws(ctx, mat->dpad, mat->n, p, nullptr, ws_items(mat));
        Engine e(mat, ws, ctx->stream);
        Padded ps(ctx, mat->dpad, p);
        ps.upload(S, mat->d, mat->dpad, p);
        e.ritz(ps.p, p, use_f32_copy != 0);
        if (H) LRA_CUDA(cudaMemcpyAsync(H, ws.H, sizeof(double) * p * p, cudaMemcpyDefault, ctx->stream));
        LRA_CUDA(cudaMemcpyAsync(evals, ws.evals, sizeof(double) * p, cudaMemcpyDefault, ctx->stream));
        LRA_CUDA(cudaMemcpyAsync(evecs, ws.evecs, sizeof(double) * p * p, cudaMemcpyDefault, ctx->stream));
        LRA_CUDA(cudaStreamSynchronize(ctx->stream));
        return LRA_OK;
    })
}

lra_status lra_lambda1_estimate(lra_mat *mat, uint64_t seed, double *lambda1_hat) {
    if (check_mat(mat) != LRA_OK || !lambda1_hat) return einval("null argument");
    lra_ctx *ctx = mat->ctx;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    LRA_TRY({
        DeviceGuard g(ctx->device);
        Workspace ws(ctx, mat->dpad, mat->n, 1, nullptr, ws_items(mat));
        Engine e(mat, ws, ctx->stream);
        *lambda1_hat = e.lambda1_estimate(seed);
        return LRA_OK;
    })
}

lra_status lra_shift_tune(lra_mat *mat, uint64_t seed, double lambda1_hat, double delta,
                          const lra_options *opt, int64_t *solve_count, double *lambda, double *inv_est,
                          double *mu_lb, int *rounds, double *history) {
    if (check_mat(mat) != LRA_OK || !lambda || !(lambda1_hat > 0) || !(delta > 0)) return einval("bad argument");
    lra_ctx *ctx = mat->ctx;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    LRA_TRY({
        DeviceGuard g(ctx->device);
        const Opts o = read_opts(opt, mat->storage);
        Workspace ws(ctx, mat->dpad, mat->n, 1, nullptr, ws_items(mat));
        Engine e(mat, ws, ctx->stream);
        int64_t sc = solve_count ? *solve_count : 0;
        double lam = 0, inv = 0, mu = 0;
        int r = 0;
        std::vector<double> hist;
        const lra_status st = e.shift_tune(seed, lambda1_hat, delta, o, sc, lam, inv, mu, r, &hist);
        *lambda = lam;
        if (inv_est) *inv_est = inv;
        if (mu_lb) *mu_lb = mu;
        if (rounds) *rounds = r;
        if (solve_count) *solve_count = sc;
        if (history) std::memcpy(history, hist.data(), sizeof(double) * std::min<size_t>(hist.size(), 2 * (size_t)o.max_shift_rounds));
        return st;
    })
}

lra_status lra_delta_estimate(lra_mat *mat, int k, int p, uint64_t seed, double *delta) {
    if (check_mat(mat) != LRA_OK || !delta) return einval("null argument");
    if (!(k >= 1 && k < p && p < mat->d) || p + 1 > LRA_MAX_P) return einval("bad k or p");
    lra_ctx *ctx = mat->ctx;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    LRA_TRY({
        DeviceGuard g(ctx->device);
        Workspace ws(ctx, mat->dpad, mat->n, p + 1, nullptr, ws_items(mat));
        Engine e(mat, ws, ctx->stream);
        return e.delta_estimate(k, p, seed, *delta);
    })
}

}  // extern "C"
