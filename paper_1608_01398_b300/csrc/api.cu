// C ABI of libiht: contexts, datasets, and the entry points of include/iht.h.
// Argument checking and marshalling only; every step of the method runs in
// the kernels of geno.cu, grad_*.cu, select.cu and solver.cu.
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <new>
#include <vector>

#include "common.cuh"

namespace iht {

static thread_local char g_last_cuda[256] = "";
static std::atomic<uint64_t> g_launches{0};

void note_launch(int n) { g_launches.fetch_add((uint64_t)(int64_t)n, std::memory_order_relaxed); }
uint64_t launches_noted() { return g_launches.load(std::memory_order_relaxed); }

static std::atomic<int> g_fault[3];         // pending injected faults by kind

bool fault_take(int kind)
{
    if (kind <= 0 || kind >= 3) return false;
    int n = g_fault[kind].load(std::memory_order_relaxed);
    while (n > 0)
        if (g_fault[kind].compare_exchange_weak(n, n - 1, std::memory_order_relaxed)) return true;
    return false;
}

cudaError_t dev_malloc_raw(void **ptr, size_t bytes)
{
    if (fault_take(IHT_FAULT_ALLOC)) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(ptr, bytes);
}

cudaError_t dev_malloc_async_raw(void **ptr, size_t bytes, cudaStream_t s)
{
    if (fault_take(IHT_FAULT_ALLOC)) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocAsync(ptr, bytes, s);
}

void set_cuda_error(cudaError_t e, const char *where)
{
    snprintf(g_last_cuda, sizeof(g_last_cuda), "%s (%s) at %s", cudaGetErrorName(e),
             cudaGetErrorString(e), where);
}

void free_workspace(Workspace *ws)
{
    if (!ws) return;
    void *ptrs[] = {ws->used, ws->rowmask, ws->counts, ws->u64, ws->v64, ws->u32, ws->v32,
                    ws->y64, ws->r64, ws->zv, ws->rc64, ws->r32, ws->g, ws->Mj, ws->partials, ws->rows_dev,
                    ws->ybuf, ws->fbuf, ws->cand, ws->S, ws->Sp, ws->bS, ws->bSp, ws->coef,
                    ws->cols, ws->sc, ws->cu64, ws->cv64, ws->zc, ws->gam, ws->zs, ws->gram,
                    ws->chol, ws->hvec};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (ws->sc_host) cudaFreeHost(ws->sc_host);
    free_batchwork(ws->bw);
    for (cudaEvent_t e : ws->prof_ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : ws->gev)
        if (e) cudaEventDestroy(e);
    if (ws->iter_exec) cudaGraphExecDestroy(ws->iter_exec);
    free_fused(ws);
    if (ws->cap_stream) cudaStreamDestroy(ws->cap_stream);
    delete ws;
}

int ensure_workspace(iht_dataset *ds, int)
{
    if (ds->ws) return IHT_OK;
    Workspace *ws = new (std::nothrow) Workspace();
    if (!ws) return IHT_ENOMEM;
    ds->ws = ws;
    const int64_t p = ds->p, np = ds->n_pad;
    ws->p = p;
    ws->n_pad = np;
    auto A = [](void **ptr, size_t bytes) { return dev_malloc(ptr, bytes ? bytes : 16); };
    cudaError_t e = cudaSuccess;
#define ALLOC(field, bytes)                                        \
    if (e == cudaSuccess) e = A((void **)&ws->field, (size_t)(bytes));
    ALLOC(used, sizeof(int32_t) * np);
    ALLOC(rowmask, sizeof(uint32_t) * (ds->stride / 4));
    ALLOC(counts, sizeof(int32_t) * 4 * p);
    ALLOC(u64, sizeof(double) * p);
    ALLOC(v64, sizeof(double) * p);
    ALLOC(u32, sizeof(float) * p);
    ALLOC(v32, sizeof(float) * p);
    ALLOC(y64, sizeof(double) * np);
    ALLOC(r64, sizeof(double) * np);
    ALLOC(zv, sizeof(double) * np);
    ALLOC(rc64, sizeof(double) * np);
    ALLOC(r32, sizeof(float) * np);
    ALLOC(g, sizeof(float) * (p + kMaxCov));
    ALLOC(Mj, sizeof(float) * p);
    ALLOC(partials, sizeof(double) * 3 * kPartials);
    ALLOC(rows_dev, sizeof(int32_t) * np);
    ALLOC(ybuf, sizeof(double) * np);
    ALLOC(fbuf, sizeof(float) * np);
    ALLOC(cand, sizeof(int32_t) * kMaxCand);
    ALLOC(S, sizeof(int32_t) * kMaxK);
    ALLOC(Sp, sizeof(int32_t) * kMaxK);
    ALLOC(bS, sizeof(double) * kMaxK);
    ALLOC(bSp, sizeof(double) * kMaxK);
    ALLOC(coef, sizeof(double) * kMaxCand);
    ALLOC(cols, sizeof(int32_t) * kMaxCand);
    ALLOC(sc, sizeof(Scalars));
#undef ALLOC
    if (e == cudaSuccess) e = cudaMallocHost((void **)&ws->sc_host, sizeof(Scalars));
    if (e == cudaSuccess) e = cudaMemsetAsync(ws->sc, 0, sizeof(Scalars), ds->ctx->stream);
    if (e != cudaSuccess) {
        set_cuda_error(e, "workspace allocation");
        free_workspace(ws);
        ds->ws = nullptr;
        return e == cudaErrorMemoryAllocation ? IHT_ENOMEM : IHT_ECUDA;
    }
    int rc = ensure_selwork(ds->ctx, p);
    if (rc) return rc;
    if (zmul_blocks(ds) > kPartials) return IHT_EINVAL;   // n above 262k samples
    return IHT_OK;
}

static int reset_err(iht_dataset *ds)
{
    IHT_CUDA(cudaMemsetAsync(&ds->ws->sc->err, 0, sizeof(int32_t), ds->ctx->stream));
    return IHT_OK;
}

static int read_err(iht_dataset *ds, int32_t *err)
{
    cudaStream_t s = ds->ctx->stream;
    IHT_CUDA(cudaMemcpyAsync(&ds->ws->sc_host->err, &ds->ws->sc->err, sizeof(int32_t),
                             cudaMemcpyDeviceToHost, s));
    IHT_CUDA(cudaStreamSynchronize(s));
    *err = ds->ws->sc_host->err;
    return IHT_OK;
}

// Rows to the device (copied into the workspace when they live on the host).
static int stage_rows(iht_dataset *ds, const int32_t *rows, int64_t n_rows, int mem,
                      const int32_t **rows_dev)
{
    *rows_dev = nullptr;
    if (!rows) return IHT_OK;
    if (n_rows > ds->n) return IHT_EINVAL;
    if (mem == IHT_DEVICE) {
        *rows_dev = rows;
        return IHT_OK;
    }
    if (n_rows > 0)
        IHT_CUDA(cudaMemcpyAsync(ds->ws->rows_dev, rows, sizeof(int32_t) * n_rows,
                                 cudaMemcpyHostToDevice, ds->ctx->stream));
    *rows_dev = ds->ws->rows_dev;
    return IHT_OK;
}

// Row set + statistics of a call; EINVAL for bad or duplicate rows.  The
// all-rows statistics are cached: a call without a row list reuses them when
// the workspace still holds them (u, v are computed once and kept, Sec. 2.3.2).
static int prepare_rows(iht_dataset *ds, const int32_t *rows, int64_t n_rows, int mem,
                        const int32_t **rows_dev)
{
    int rc;
    if ((rc = reset_err(ds))) return rc;
    if (!rows && ds->ws->rowset_all) {
        *rows_dev = nullptr;
        return IHT_OK;
    }
    ds->ws->rowset_all = false;
    if ((rc = stage_rows(ds, rows, n_rows, mem, rows_dev))) return rc;
    if ((rc = setup_rows(ds, *rows_dev, n_rows))) return rc;
    if (rows) {
        int32_t err = 0;
        if ((rc = read_err(ds, &err))) return rc;
        if (err & 2) return IHT_EINVAL;
    }
    if ((rc = launch_counts(ds, n_rows))) return rc;
    ds->ws->rowset_all = rows == nullptr;
    return IHT_OK;
}

}  // namespace iht

using namespace iht;

extern "C" {

void iht_default_options(iht_options *o)
{
    if (!o) return;
    o->max_iter = 100;
    o->max_backtrack = 50;
    o->tol = 1e-4;
    o->c = 0.01;
    o->kappa = 2.0;
    o->in_mem = IHT_HOST;
    o->out_mem = IHT_HOST;
    o->grad_impl = 0;
    o->profile = 0;
    o->variant = IHT_VARIANT_IHT;
    o->flags = 0;
}

const char *iht_strerror(int s)
{
    switch (s) {
    case IHT_OK: return "ok";
    case IHT_EINVAL: return "invalid argument";
    case IHT_ENOMEM: return "out of memory";
    case IHT_ENOTCONV: return "not converged within max_iter (results valid)";
    case IHT_ENUMERIC: return "non-finite input or zero step-size denominator";
    case IHT_ETIMEOUT: return "bounded device wait timed out";
    case IHT_ECUDA: return "CUDA runtime error";
    case IHT_EAGAIN: return "result not ready";
    default: return "unknown status";
    }
}

const char *iht_last_cuda_error(void) { return g_last_cuda; }

uint64_t iht_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int iht_fault_inject(int kind, int32_t count)
{
    if (kind == IHT_FAULT_NONE) {
        g_fault[IHT_FAULT_ALLOC].store(0);
        g_fault[IHT_FAULT_TIMEOUT].store(0);
        return IHT_OK;
    }
    if ((kind != IHT_FAULT_ALLOC && kind != IHT_FAULT_TIMEOUT) || count < 0) return IHT_EINVAL;
    g_fault[kind].store(count);
    return IHT_OK;
}

int iht_create(iht_ctx **out, int device, void *stream)
{
    if (!out) return IHT_EINVAL;
    *out = nullptr;
    int count = 0;
    IHT_CUDA(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count) return IHT_EINVAL;
    DeviceGuard g(device);
    if (!g.ok) return IHT_ECUDA;
    iht_ctx *c = new (std::nothrow) iht_ctx();
    if (!c) return IHT_ENOMEM;
    c->device = device;
    c->stream = (cudaStream_t)stream;
    cudaError_t e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        set_cuda_error(e, "cudaDeviceGetAttribute");
        delete c;
        return IHT_ECUDA;
    }
    *out = c;
    return IHT_OK;
}

int iht_destroy(iht_ctx *ctx)
{
    if (!ctx) return IHT_EINVAL;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->sel.hist) cudaFree(ctx->sel.hist);
    if (ctx->sel.st) cudaFree(ctx->sel.st);
    if (ctx->sel.cand) cudaFree(ctx->sel.cand);
    delete ctx;
    return IHT_OK;
}

int iht_load_bed(iht_ctx *ctx, const uint8_t *bed, size_t bed_bytes, int mem, int64_t n,
                 int64_t p, iht_dataset **out)
{
    if (!ctx || !bed || !out || n < 1 || p < 1 || (mem != IHT_HOST && mem != IHT_DEVICE))
        return IHT_EINVAL;
    if (p > 0x7fffffffLL || n > 0x7fffffffLL) return IHT_EINVAL;
    *out = nullptr;
    const int64_t nbytes = (n + 3) / 4;
    if ((int64_t)bed_bytes != 3 + p * nbytes) return IHT_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return IHT_ECUDA;
    uint8_t magic[3];
    if (mem == IHT_HOST) {
        memcpy(magic, bed, 3);
    } else {
        IHT_CUDA(cudaMemcpy(magic, bed, 3, cudaMemcpyDeviceToHost));
    }
    if (magic[0] != 0x6C || magic[1] != 0x1B || magic[2] != 0x01) return IHT_EINVAL;
    iht_dataset *ds = new (std::nothrow) iht_dataset();
    if (!ds) return IHT_ENOMEM;
    ds->ctx = ctx;
    ds->n = n;
    ds->p = p;
    ds->stride = (nbytes + 127) / 128 * 128;
    ds->rowb = (nbytes + 15) / 16 * 16;
    ds->n_pad = 4 * ds->stride;
    ds->ws = nullptr;
    ds->miss_off = nullptr;
    ds->miss_idx = nullptr;
    ds->miss_total = 0;
    ds->miss_idx16 = n <= 65536;
    cudaError_t e = dev_malloc(&ds->G, (size_t)(p * ds->stride));
    if (e != cudaSuccess) {
        set_cuda_error(e, "cudaMalloc(genotypes)");
        delete ds;
        return e == cudaErrorMemoryAllocation ? IHT_ENOMEM : IHT_ECUDA;
    }
    e = cudaMemcpy2DAsync(ds->G, ds->stride, bed + 3, nbytes, nbytes, p, cudaMemcpyDefault,
                          ctx->stream);
    int rc = IHT_OK;
    if (e != cudaSuccess) {
        set_cuda_error(e, "cudaMemcpy2DAsync(genotypes)");
        rc = IHT_ECUDA;
    }
    if (rc == IHT_OK) rc = launch_fix_padding(ds);
    if (rc == IHT_OK) rc = build_missing_lists(ds);
    if (rc == IHT_OK) {
        e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) {
            set_cuda_error(e, "iht_load_bed");
            rc = IHT_ECUDA;
        }
    }
    if (rc != IHT_OK) {
        cudaFree(ds->G);
        if (ds->miss_off) cudaFree(ds->miss_off);
        if (ds->miss_idx) cudaFree(ds->miss_idx);
        if (ds->miss_goff) cudaFree(ds->miss_goff);
        if (ds->miss_gidx) cudaFree(ds->miss_gidx);
        if (ds->miss_ioff) cudaFree(ds->miss_ioff);
        if (ds->miss_iidx) cudaFree(ds->miss_iidx);
        delete ds;
        return rc;
    }
    *out = ds;
    return IHT_OK;
}

int iht_dataset_free(iht_dataset *ds)
{
    if (!ds) return IHT_EINVAL;
    DeviceGuard g(ds->ctx->device);
    cudaStreamSynchronize(ds->ctx->stream);
    free_workspace(ds->ws);
    cudaFree(ds->G);
    if (ds->cov) cudaFree(ds->cov);
    if (ds->miss_off) cudaFree(ds->miss_off);
    if (ds->miss_idx) cudaFree(ds->miss_idx);
    if (ds->miss_goff) cudaFree(ds->miss_goff);
    if (ds->miss_gidx) cudaFree(ds->miss_gidx);
    if (ds->miss_ioff) cudaFree(ds->miss_ioff);
    if (ds->miss_iidx) cudaFree(ds->miss_iidx);
    delete ds;
    return IHT_OK;
}

int iht_set_covariates(iht_dataset *ds, const double *cov, int32_t q, int mem)
{
    if (!ds || q < 0 || q > kMaxCov || (q > 0 && !cov) || (mem != IHT_HOST && mem != IHT_DEVICE))
        return IHT_EINVAL;
    DeviceGuard g(ds->ctx->device);
    if (!g.ok) return IHT_ECUDA;
    cudaStream_t s = ds->ctx->stream;
    IHT_CUDA(cudaStreamSynchronize(s));
    if (ds->cov) cudaFree(ds->cov);
    ds->cov = nullptr;
    ds->q = 0;
    if (q == 0) return IHT_OK;
    double *d = nullptr;
    IHT_CUDA(dev_malloc(&d, sizeof(double) * (size_t)q * ds->n_pad));
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(double) * (size_t)q * ds->n_pad, s);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(d, sizeof(double) * ds->n_pad, cov, sizeof(double) * ds->n,
                              sizeof(double) * ds->n, q, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(d);
        set_cuda_error(e, "iht_set_covariates");
        return IHT_ECUDA;
    }
    ds->cov = d;
    ds->q = q;
    return IHT_OK;
}

int iht_dataset_shape(const iht_dataset *ds, int64_t *n, int64_t *p, int64_t *stride)
{
    if (!ds) return IHT_EINVAL;
    if (n) *n = ds->n;
    if (p) *p = ds->p;
    if (stride) *stride = ds->stride;
    return IHT_OK;
}

int iht_counts(iht_dataset *ds, const int32_t *rows, int64_t n_rows, int mem, int32_t *counts_out,
               double *u_out, double *v_out)
{
    if (!ds || (mem != IHT_HOST && mem != IHT_DEVICE)) return IHT_EINVAL;
    if (!rows) n_rows = ds->n;
    if (n_rows < 0 || n_rows > ds->n) return IHT_EINVAL;
    DeviceGuard g(ds->ctx->device);
    if (!g.ok) return IHT_ECUDA;
    int rc = ensure_workspace(ds, 0);
    if (rc) return rc;
    const int32_t *rows_dev = nullptr;
    if ((rc = prepare_rows(ds, rows, n_rows, mem, &rows_dev))) return rc;
    cudaStream_t s = ds->ctx->stream;
    const cudaMemcpyKind kind = mem == IHT_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (counts_out)
        IHT_CUDA(cudaMemcpyAsync(counts_out, ds->ws->counts, sizeof(int32_t) * 4 * ds->p, kind, s));
    if (u_out) IHT_CUDA(cudaMemcpyAsync(u_out, ds->ws->u64, sizeof(double) * ds->p, kind, s));
    if (v_out) IHT_CUDA(cudaMemcpyAsync(v_out, ds->ws->v64, sizeof(double) * ds->p, kind, s));
    IHT_CUDA(cudaStreamSynchronize(s));
    return IHT_OK;
}

int iht_gradient(iht_dataset *ds, const int32_t *rows, int64_t n_rows, const float *r,
                 float *g_out, int impl)
{
    if (!ds || !r || !g_out || impl < 0 || impl > 2) return IHT_EINVAL;
    if (!rows) n_rows = ds->n;
    if (n_rows < 1 || n_rows > ds->n) return IHT_EINVAL;
    DeviceGuard g(ds->ctx->device);
    if (!g.ok) return IHT_ECUDA;
    int rc = ensure_workspace(ds, 0);
    if (rc) return rc;
    const int32_t *rows_dev = nullptr;
    if ((rc = prepare_rows(ds, rows, n_rows, IHT_DEVICE, &rows_dev))) return rc;
    if ((rc = scatter_rows_f32(ds, rows_dev, n_rows, r, ds->ws->r32))) return rc;
    if ((rc = grad_tc_reset_status(ds))) return rc;
    if ((rc = launch_grad_impl(ds, impl, ds->ws->r32, g_out, nullptr))) return rc;
    int timed_out = 0;
    if ((rc = grad_tc_status(ds, &timed_out))) return rc;      // synchronises
    return timed_out ? IHT_ETIMEOUT : IHT_OK;
}

int iht_topk(iht_ctx *ctx, const float *w, int64_t p, int32_t k, int32_t *idx_out)
{
    if (!ctx || !w || !idx_out || p < 1 || k < 1 || k > p || k > kMaxCand) return IHT_EINVAL;
    if (p > 0x7fffffffLL) return IHT_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return IHT_ECUDA;
    int rc = ensure_selwork(ctx, p);
    if (rc) return rc;
    IHT_CUDA(cudaMemsetAsync(&ctx->sel.st->err, 0, sizeof(uint32_t), ctx->stream));
    if ((rc = select_topk(ctx, w, p, k, idx_out, nullptr))) return rc;
    uint32_t err = 0;
    IHT_CUDA(cudaMemcpyAsync(&err, &ctx->sel.st->err, sizeof(err), cudaMemcpyDeviceToHost, ctx->stream));
    IHT_CUDA(cudaStreamSynchronize(ctx->stream));
    return (err & 1u) ? IHT_ENUMERIC : IHT_OK;
}

int iht_zmul(iht_dataset *ds, const int32_t *rows, int64_t n_rows, const double *u,
             const double *v, const int32_t *cols, int32_t m, const double *coef, double *out)
{
    if (!ds || !out || m < 0 || (m > 0 && (!cols || !coef)) || ((u == nullptr) != (v == nullptr)))
        return IHT_EINVAL;
    if (!rows) n_rows = ds->n;
    if (n_rows < 0 || n_rows > ds->n) return IHT_EINVAL;
    DeviceGuard g(ds->ctx->device);
    if (!g.ok) return IHT_ECUDA;
    int rc = ensure_workspace(ds, 0);
    if (rc) return rc;
    const int32_t *rows_dev = nullptr;
    if ((rc = prepare_rows(ds, rows, n_rows, IHT_DEVICE, &rows_dev))) return rc;
    Workspace *ws = ds->ws;
    if ((rc = launch_zmul(ds, cols, m, coef, u ? u : ws->u64, v ? v : ws->v64, ws->used, nullptr,
                          ws->zv, nullptr)))
        return rc;
    if ((rc = gather_rows_f64(ds, rows_dev, n_rows, ws->zv, out))) return rc;
    IHT_CUDA(cudaStreamSynchronize(ds->ctx->stream));
    return IHT_OK;
}

static int fit_impl(iht_dataset *ds, const int32_t *rows, int64_t n_rows, const double *y,
                    int32_t k, const iht_options *opt_in, double *beta_out, int32_t *support_out,
                    iht_result *info, iht_trace *trace, const SolveInit *init = nullptr)
{
    iht_options opt;
    if (opt_in)
        opt = *opt_in;
    else
        iht_default_options(&opt);
    if (!ds || !y || !beta_out || !support_out) return IHT_EINVAL;
    if (!rows) n_rows = ds->n;
    const int64_t P = ds->p + ds->q;
    if (n_rows < 2 || n_rows > ds->n || k < 1 || k > P || k > kMaxK) return IHT_EINVAL;
    if ((opt.in_mem != IHT_HOST && opt.in_mem != IHT_DEVICE) ||
        (opt.out_mem != IHT_HOST && opt.out_mem != IHT_DEVICE) || opt.max_iter < 0 ||
        opt.max_backtrack < 0 || !(opt.kappa > 1.0) || !(opt.c >= 0.0 && opt.c < 1.0) ||
        !(opt.tol >= 0.0) || opt.grad_impl < 0 || opt.grad_impl > 2 ||
        (opt.variant != IHT_VARIANT_IHT && opt.variant != IHT_VARIANT_HTP) ||
        (opt.flags & ~IHT_FIT_BETA_ZEROED))
        return IHT_EINVAL;
    if (init && (ds->q > 0 || opt.variant != IHT_VARIANT_IHT)) return IHT_EINVAL;
    DeviceGuard g(ds->ctx->device);
    if (!g.ok) return IHT_ECUDA;
    int rc = ensure_workspace(ds, k);
    if (rc) return rc;
    Workspace *ws = ds->ws;
    cudaStream_t s = ds->ctx->stream;
    const int32_t *rows_dev = nullptr;
    if ((rc = prepare_rows(ds, rows, n_rows, opt.in_mem, &rows_dev))) return rc;
    const double *y_dev = y;
    if (opt.in_mem == IHT_HOST) {
        IHT_CUDA(cudaMemcpyAsync(ws->ybuf, y, sizeof(double) * n_rows, cudaMemcpyHostToDevice, s));
        y_dev = ws->ybuf;
    }
    if ((rc = check_finite_y(ds, n_rows, y_dev))) return rc;
    if ((rc = scatter_rows_f64(ds, rows_dev, n_rows, y_dev, ws->y64))) return rc;
    if ((rc = cov_setup(ds, n_rows))) return rc;
    ws->out_want = opt.out_mem == IHT_HOST && !trace ? 1 : 0;
    ws->out_ready = 0;
    rc = run_solve_host(ds, k, &opt, (int)n_rows, trace, opt.max_iter, init);
    ws->out_want = 0;
    if (rc) return rc;
    const Scalars &h = *ws->sc_host;
    if (opt.out_mem == IHT_DEVICE) {
        if ((rc = write_beta_device(ds, k, beta_out))) return rc;
        IHT_CUDA(cudaMemcpyAsync(support_out, ws->S, sizeof(int32_t) * k, cudaMemcpyDeviceToDevice, s));
        IHT_CUDA(cudaStreamSynchronize(s));
    } else if (ws->out_ready) {                  // copied with the solve's final scalars
        ws->out_ready = 0;
        const int32_t *hS = static_cast<const int32_t *>(ws->out_host);
        const double *hb = reinterpret_cast<const double *>(hS + kMaxK);
        memcpy(support_out, hS, sizeof(int32_t) * k);
        if (!(opt.flags & IHT_FIT_BETA_ZEROED)) memset(beta_out, 0, sizeof(double) * P);
        for (int c = 0; c < k; ++c) beta_out[hS[c]] = hb[c];
    } else {
        double *bS = (double *)malloc(sizeof(double) * k);
        if (!bS) return IHT_ENOMEM;
        cudaError_t e = cudaMemcpyAsync(support_out, ws->S, sizeof(int32_t) * k,
                                        cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(bS, ws->bS, sizeof(double) * k, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            free(bS);
            set_cuda_error(e, "iht_fit outputs");
            return IHT_ECUDA;
        }
        if (!(opt.flags & IHT_FIT_BETA_ZEROED)) memset(beta_out, 0, sizeof(double) * P);
        for (int c = 0; c < k; ++c) beta_out[support_out[c]] = bS[c];
        free(bS);
    }
    if (info) {
        info->iterations = h.iter;
        info->status = h.status;
        info->backtracks = h.bt_total;
        info->reserved = 0;
        info->objective = h.f;
        info->mu = h.mu;
        info->grad_ms = opt.profile ? ws->prof_ms : 0.0;
        info->grad_launches = opt.profile ? ws->nprof : 0;
        info->graph_replays = ws->graph_replays;
    }
    return h.status;
}

int iht_fit(iht_dataset *ds, const int32_t *rows, int64_t n_rows, const double *y, int32_t k,
            const iht_options *opt, double *beta_out, int32_t *support_out, iht_result *info)
{
    return fit_impl(ds, rows, n_rows, y, k, opt, beta_out, support_out, info, nullptr);
}

int iht_fit_trace(iht_dataset *ds, const int32_t *rows, int64_t n_rows, const double *y,
                  int32_t k, const iht_options *opt, double *beta_out, int32_t *support_out,
                  iht_result *info, iht_trace *trace)
{
    return fit_impl(ds, rows, n_rows, y, k, opt, beta_out, support_out, info, trace);
}

int iht_fit_resume(iht_dataset *ds, const int32_t *rows, int64_t n_rows, const double *y,
                   const void *state, size_t state_bytes, const iht_options *opt,
                   double *beta_out, int32_t *support_out, iht_result *info)
{
    if (!ds || !state) return IHT_EINVAL;
    int64_t n = 0, p = 0, nr = 0;
    int32_t k = 0;
    int rc = iht_state_load(state, state_bytes, kMaxK, &n, &p, &nr, &k, nullptr, nullptr, nullptr);
    if (rc) return rc;
    if (!rows) n_rows = ds->n;
    if (n != ds->n || p != ds->p || nr != n_rows) return IHT_EINVAL;
    std::vector<int32_t> S((size_t)k);
    std::vector<double> b((size_t)k);
    iht_result st{};
    if ((rc = iht_state_load(state, state_bytes, kMaxK, &n, &p, &nr, &k, S.data(), b.data(), &st)))
        return rc;
    SolveInit init{S.data(), b.data(), st.iterations, st.backtracks};
    if (init.iter < 0 || init.backtracks < 0) return IHT_EINVAL;
    return fit_impl(ds, rows, n_rows, y, k, opt, beta_out, support_out, info, nullptr, &init);
}

}  // extern "C"
