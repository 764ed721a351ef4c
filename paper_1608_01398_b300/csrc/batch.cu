// a7: b IHT solves on one dataset that share every pass over the genotypes.
//
// Each solve follows the single-solve path step for step (same readings,
// statistics over its own rows, same tails), but an iteration of the batch
// is one multi-column gradient pass (grad_mrhs.cu) for all solves still
// running, then every O(nk) step as one launch over the batch
// (solver.cu / select.cu batched kernels, blockIdx = solve).  Solves retire
// independently: a finished solve drops out of the gradient columns and its
// blocks of the tail kernels return at once.  Row sets shared by several
// solves (a cross-validation fold used along a path of model sizes) have
// their per-SNP statistics computed once (Sec. 2.3.2).
//
// An iteration is one replay of a CUDA graph (the gradient pass, candidates,
// g_S, Z_S g_S and two attempts; the second attempt's kernels return at once
// for every solve whose first step was accepted), with one host
// synchronisation, once its number of active columns has been seen: a new
// count runs once as direct launches and is captured when it comes again, in
// the same call or a later one.
#include <stdlib.h>
#include <string.h>

#include <new>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "common.cuh"

namespace iht {

constexpr int kBatchGraphPairs = 32;       // gradient passes timed per replay (1408 columns)
constexpr size_t kBatchGraphs = 64;        // cached iteration graphs per workspace

struct BatchWork {
    int nb = 0, kcap = 0, nsets = 0;       // capacities
    int64_t rows_cap = 0, y_cap = 0;
    Scalars *sc = nullptr, *sc_host = nullptr;
    double *y64 = nullptr, *r64 = nullptr, *rc64 = nullptr, *zv = nullptr;
    float *r32 = nullptr, *g = nullptr;
    int32_t *S = nullptr, *Sp = nullptr, *cand = nullptr;
    double *bS = nullptr, *bSp = nullptr, *coef = nullptr, *partials = nullptr;
    SelState *st = nullptr;
    uint32_t *hist = nullptr;
    unsigned long long *selcand = nullptr;
    BSolve *bs = nullptr, *bs_host = nullptr;
    SelJob *jobs = nullptr, *jobs_host = nullptr;     // 2 nb: top-k then candidates
    MrCol *cols = nullptr, *cols_host = nullptr;
    // row sets
    int32_t *set_used = nullptr, *set_err = nullptr, *set_err_host = nullptr;
    uint32_t *set_rowmask = nullptr;
    double *set_u64 = nullptr, *set_v64 = nullptr;
    float *set_u32 = nullptr, *set_v32 = nullptr;
    int32_t *rows_dev = nullptr;           // staged host row lists
    double *ybuf = nullptr;                // staged host phenotypes
    cudaEvent_t ev[2 * kProfEvents] = {};
    // iteration graphs, keyed by sizes, scratch identities and the active set
    struct Graph {
        cudaGraphExec_t exec = nullptr;
        int launches = 0;                  // kernels per replay
        int pairs = 0;                     // gradient event pairs per replay
        uint64_t used = 0;                 // last use (least recently used is replaced)
    };
    std::unordered_map<std::string, Graph> graphs;
    std::unordered_set<std::string> graph_seen;   // keys run once as direct launches
    uint64_t graph_clock = 0;
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t gev[2 * kBatchGraphPairs] = {};
};

void free_batchwork(BatchWork *w)
{
    if (!w) return;
    void *dev[] = {w->sc, w->y64, w->r64, w->rc64, w->zv, w->r32, w->g, w->S, w->Sp, w->cand,
                   w->bS, w->bSp, w->coef, w->partials, w->st, w->hist, w->selcand,
                   w->bs, w->jobs, w->cols, w->set_used, w->set_err, w->set_rowmask, w->set_u64,
                   w->set_v64, w->set_u32, w->set_v32, w->rows_dev, w->ybuf};
    for (void *p : dev)
        if (p) cudaFree(p);
    void *host[] = {w->sc_host, w->bs_host, w->jobs_host, w->cols_host, w->set_err_host};
    for (void *p : host)
        if (p) cudaFreeHost(p);
    for (cudaEvent_t e : w->ev)
        if (e) cudaEventDestroy(e);
    for (auto &kv : w->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    for (cudaEvent_t e : w->gev)
        if (e) cudaEventDestroy(e);
    if (w->cap_stream) cudaStreamDestroy(w->cap_stream);
    delete w;
}

// Capacity for nb solves of sparsity <= kcap over nsets row sets, rows_total
// staged row indices and y_total staged phenotype values.
static int ensure_batchwork(iht_dataset *ds, int nb, int kcap, int nsets, int64_t rows_total,
                            int64_t y_total)
{
    BatchWork *&w = ds->ws->bw;
    if (w && w->nb >= nb && w->kcap >= kcap && w->nsets >= nsets && w->rows_cap >= rows_total &&
        w->y_cap >= y_total)
        return IHT_OK;
    if (w) {
        nb = std::max(nb, w->nb);
        kcap = std::max(kcap, w->kcap);
        nsets = std::max(nsets, w->nsets);
        rows_total = std::max(rows_total, w->rows_cap);
        y_total = std::max(y_total, w->y_cap);
        cudaStreamSynchronize(ds->ctx->stream);
        free_batchwork(w);
        w = nullptr;
    }
    BatchWork *x = new (std::nothrow) BatchWork();
    if (!x) return IHT_ENOMEM;
    const size_t np = (size_t)ds->n_pad, p = (size_t)ds->p, B = (size_t)nb, K = (size_t)kcap;
    cudaError_t e = cudaSuccess;
#define BALLOC(field, bytes) \
    if (e == cudaSuccess) e = dev_malloc((void **)&x->field, std::max<size_t>(16, (size_t)(bytes)));
    BALLOC(sc, sizeof(Scalars) * B);
    BALLOC(y64, sizeof(double) * B * np);
    BALLOC(r64, sizeof(double) * B * np);
    BALLOC(rc64, sizeof(double) * B * np);
    BALLOC(zv, sizeof(double) * B * np);
    BALLOC(r32, sizeof(float) * B * np);
    BALLOC(g, sizeof(float) * B * p);
    BALLOC(S, sizeof(int32_t) * B * K);
    BALLOC(Sp, sizeof(int32_t) * B * K);
    BALLOC(cand, sizeof(int32_t) * B * 2 * K);
    BALLOC(bS, sizeof(double) * B * K);
    BALLOC(bSp, sizeof(double) * B * K);
    BALLOC(coef, sizeof(double) * B * K);
    BALLOC(partials, sizeof(double) * B * 3 * kPartials);
    BALLOC(st, sizeof(SelState) * 2 * B);
    BALLOC(hist, sizeof(uint32_t) * 2 * B * kSelBins);
    BALLOC(selcand, sizeof(unsigned long long) * 2 * B * kSelCap);
    BALLOC(bs, sizeof(BSolve) * B);
    BALLOC(jobs, sizeof(SelJob) * 2 * B);
    BALLOC(cols, sizeof(MrCol) * B);
    BALLOC(set_used, sizeof(int32_t) * nsets * np);
    BALLOC(set_err, sizeof(int32_t) * nsets);
    BALLOC(set_rowmask, sizeof(uint32_t) * nsets * (ds->stride / 4));
    BALLOC(set_u64, sizeof(double) * nsets * p);
    BALLOC(set_v64, sizeof(double) * nsets * p);
    BALLOC(set_u32, sizeof(float) * nsets * p);
    BALLOC(set_v32, sizeof(float) * nsets * p);
    BALLOC(rows_dev, sizeof(int32_t) * rows_total);
    BALLOC(ybuf, sizeof(double) * y_total);
#undef BALLOC
    if (e == cudaSuccess) e = cudaMallocHost((void **)&x->sc_host, sizeof(Scalars) * B);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&x->bs_host, sizeof(BSolve) * B);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&x->jobs_host, sizeof(SelJob) * 2 * B);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&x->cols_host, sizeof(MrCol) * B);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&x->set_err_host, sizeof(int32_t) * nsets);
    // selection scratch starts zeroed; every selection leaves it so
    if (e == cudaSuccess) e = cudaMemsetAsync(x->st, 0, sizeof(SelState) * 2 * B, ds->ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(x->hist, 0, sizeof(uint32_t) * 2 * B * kSelBins, ds->ctx->stream);
    if (e != cudaSuccess) {
        set_cuda_error(e, "batch workspace allocation");
        free_batchwork(x);
        return e == cudaErrorMemoryAllocation ? IHT_ENOMEM : IHT_ECUDA;
    }
    x->nb = nb;
    x->kcap = kcap;
    x->nsets = nsets;
    x->rows_cap = rows_total;
    x->y_cap = y_total;
    w = x;
    return IHT_OK;
}

static RowSet batch_rowset(iht_dataset *ds, BatchWork *w, int q)
{
    const size_t np = (size_t)ds->n_pad, p = (size_t)ds->p;
    RowSet rs;
    rs.used = w->set_used + q * np;
    rs.rowmask = w->set_rowmask + q * (size_t)(ds->stride / 4);
    rs.counts = nullptr;
    rs.u64 = w->set_u64 + q * p;
    rs.v64 = w->set_v64 + q * p;
    rs.u32 = w->set_u32 + q * p;
    rs.v32 = w->set_v32 + q * p;
    return rs;
}

struct SetKey {
    const int32_t *rows;
    int64_t n_rows;
};

// Distinct row sets of the solves (same rows pointer and length = same set).
static void dedupe_sets(int b, const int32_t *const *rows, const int64_t *n_rows, int64_t n,
                        std::vector<SetKey> &sets, std::vector<int> &set_of)
{
    sets.clear();
    set_of.assign(b, -1);
    for (int c = 0; c < b; ++c) {
        const int64_t nr = rows[c] ? n_rows[c] : n;
        int q = -1;
        for (size_t t = 0; t < sets.size(); ++t)
            if (sets[t].rows == rows[c] && sets[t].n_rows == nr) {
                q = (int)t;
                break;
            }
        if (q < 0) {
            sets.push_back(SetKey{rows[c], nr});
            q = (int)sets.size() - 1;
        }
        set_of[c] = q;
    }
}

// Row marks and statistics of every set; EINVAL when a set has bad or
// duplicate rows.  Host row lists are staged (rows_mem).
static int build_sets(iht_dataset *ds, BatchWork *w, const std::vector<SetKey> &sets, int rows_mem,
                      std::vector<const int32_t *> &rows_dev)
{
    cudaStream_t s = ds->ctx->stream;
    const int nsets = (int)sets.size();
    rows_dev.assign(nsets, nullptr);
    IHT_CUDA(cudaMemsetAsync(w->set_err, 0, sizeof(int32_t) * nsets, s));
    int64_t off = 0;
    for (int q = 0; q < nsets; ++q) {
        const SetKey &k = sets[q];
        if (k.rows) {
            if (rows_mem == IHT_HOST) {
                if (k.n_rows > 0)
                    IHT_CUDA(cudaMemcpyAsync(w->rows_dev + off, k.rows, sizeof(int32_t) * k.n_rows,
                                             cudaMemcpyHostToDevice, s));
                rows_dev[q] = w->rows_dev + off;
                off += k.n_rows;
            } else {
                rows_dev[q] = k.rows;
            }
        }
        int rc = setup_rowset(ds, rows_dev[q], k.n_rows, batch_rowset(ds, w, q), w->set_err + q);
        if (rc) return rc;
    }
    {   // statistics of all sets, several per pass over the genotypes
        std::vector<RowSet> rs(nsets);
        std::vector<int64_t> nr(nsets);
        for (int q = 0; q < nsets; ++q) {
            rs[q] = batch_rowset(ds, w, q);
            nr[q] = sets[q].n_rows;
        }
        int rc = launch_counts_sets(ds, rs.data(), nr.data(), nsets);
        if (rc) return rc;
    }
    IHT_CUDA(cudaMemcpyAsync(w->set_err_host, w->set_err, sizeof(int32_t) * nsets,
                             cudaMemcpyDeviceToHost, s));
    IHT_CUDA(cudaStreamSynchronize(s));
    for (int q = 0; q < nsets; ++q)
        if (w->set_err_host[q] & 2) return IHT_EINVAL;
    return IHT_OK;
}

// Column descriptors of the listed solves, uploaded for the multi-column pass.
static int batch_cols(iht_dataset *ds, BatchWork *w, const std::vector<int> &act,
                      const std::vector<int> &set_of)
{
    const size_t np = (size_t)ds->n_pad, p = (size_t)ds->p;
    for (size_t a = 0; a < act.size(); ++a) {
        const int c = act[a];
        const RowSet rs = batch_rowset(ds, w, set_of[c]);
        MrCol &C = w->cols_host[a];
        C.r32 = w->r32 + c * np;
        C.u32 = rs.u32;
        C.v32 = rs.v32;
        C.g = w->g + c * p;
        C.scale = 0.0f;
        C.R = 0.0f;
    }
    IHT_CUDA(cudaMemcpyAsync(w->cols, w->cols_host, sizeof(MrCol) * act.size(), cudaMemcpyHostToDevice,
                             ds->ctx->stream));
    return IHT_OK;
}

// Gradient of the listed solves (impl 0/2: one multi-column pass; 1: one
// CUDA-core pass per solve).
static int batch_grad(iht_dataset *ds, BatchWork *w, const std::vector<int> &act,
                      const std::vector<int> &set_of, int impl, ProfEvents *prof = nullptr)
{
    cudaStream_t s = ds->ctx->stream;
    const size_t np = (size_t)ds->n_pad, p = (size_t)ds->p;
    if (act.empty()) return IHT_OK;
    if (impl == 1) {
        for (int c : act) {
            const RowSet rs = batch_rowset(ds, w, set_of[c]);
            prof_begin(prof, s);
            int rc = launch_grad_simt_stats(ds, w->r32 + c * np, rs.u32, rs.v32, w->g + c * p);
            prof_end(prof, s);
            if (rc) return rc;
        }
        return IHT_OK;
    }
    int rc = batch_cols(ds, w, act, set_of);
    if (rc) return rc;
    return launch_grad_mrhs(ds, w->cols, (int)act.size(), prof, impl == 2 ? nullptr : w->cols_host);
}

// One backtracking attempt of every solve that takes part (first: the
// iteration's first attempt; else only solves whose last candidate was
// rejected): projection, candidate residual, decision, centring.
static int batch_attempt(iht_dataset *ds, BatchWork *w, int b, int kmax, bool first)
{
    int rc;
    if ((rc = launch_merge_batch(ds, w->bs, b, first))) return rc;
    if ((rc = launch_zmul_batch(ds, w->bs, b, kmax, kZmulResidual))) return rc;
    if ((rc = launch_decide_batch(ds, w->bs, b))) return rc;
    return launch_center_batch(ds, w->bs, b, false);
}

// Candidates, g_S and Z_S g_S after the gradient.
static int batch_step(iht_dataset *ds, BatchWork *w, int b, int kmax)
{
    int rc;
    if ((rc = select_topk_batch(ds->ctx, w->jobs + b, b, ds->p))) return rc;
    if ((rc = launch_gather_gS_batch(ds, w->bs, b))) return rc;
    return launch_zmul_batch(ds, w->bs, b, kmax, kZmulStep);
}

// Key of the iteration graph over ncols active columns (w->cols_host filled).
// Only the column count shapes the captured launches: the column descriptors
// live in w->cols, uploaded before every replay, and every other kernel runs
// over all b solves, each block gated by its solve's flags on the device; a
// single column with impl 0 runs the single-column pass, whose pointers come
// from the host and join the key.
static std::string batch_graph_key(BatchWork *w, int b, int kmax, int impl, bool prof, int ncols)
{
    std::vector<uint64_t> key = {(uint64_t)b, (uint64_t)kmax, (uint64_t)impl, (uint64_t)prof,
                                 grad_mrhs_scratch_id(), grad_tc_scratch_id(), (uint64_t)ncols};
    if (ncols == 1 && impl != 2) {
        const MrCol &C = w->cols_host[0];
        key.insert(key.end(), {(uint64_t)(uintptr_t)C.r32, (uint64_t)(uintptr_t)C.u32, (uint64_t)(uintptr_t)C.v32,
                               (uint64_t)(uintptr_t)C.g});
    }
    return std::string(reinterpret_cast<const char *>(key.data()), key.size() * sizeof(uint64_t));
}

// The cached graph under key k, or null.
static BatchWork::Graph *batch_graph_find(BatchWork *w, const std::string &k)
{
    auto it = w->graphs.find(k);
    if (it == w->graphs.end()) return nullptr;
    it->second.used = ++w->graph_clock;
    return &it->second;
}

// The graph of one iteration over the active solves act (multi-column
// gradient; w->cols uploaded by the caller before every replay), captured on
// the workspace's private stream (the caller's may be the legacy default
// stream) and cached under k (batch_graph_key).
static int batch_graph(iht_dataset *ds, BatchWork *w, int b, int kmax, int impl, bool prof,
                       const std::vector<int> &act, const std::string &k, BatchWork::Graph **out)
{
    if ((*out = batch_graph_find(w, k))) return IHT_OK;
    if (w->graphs.size() >= kBatchGraphs) {        // replace the least recently used
        auto lru = w->graphs.begin();
        for (auto g = w->graphs.begin(); g != w->graphs.end(); ++g)
            if (g->second.used < lru->second.used) lru = g;
        cudaGraphExecDestroy(lru->second.exec);
        w->graphs.erase(lru);
    }
    if (!w->cap_stream) IHT_CUDA(cudaStreamCreateWithFlags(&w->cap_stream, cudaStreamNonBlocking));
    if (prof && !w->gev[0])
        for (cudaEvent_t &e : w->gev) IHT_CUDA(cudaEventCreate(&e));
    ProfEvents pe;
    pe.ev = w->gev;
    pe.cap = prof ? kBatchGraphPairs : 0;
    cudaStream_t user = ds->ctx->stream;
    ds->ctx->stream = w->cap_stream;
    const uint64_t before = launches_noted();
    cudaError_t e = cudaStreamBeginCapture(w->cap_stream, cudaStreamCaptureModeThreadLocal);
    int rc = IHT_OK;
    if (e == cudaSuccess) {
        rc = launch_grad_mrhs(ds, w->cols, (int)act.size(), prof ? &pe : nullptr,
                              impl == 2 ? nullptr : w->cols_host);
        if (!rc) rc = batch_step(ds, w, b, kmax);
        for (int attempt = 0; !rc && attempt < 2; ++attempt) rc = batch_attempt(ds, w, b, kmax, attempt == 0);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(w->cap_stream, &graph) : e;
    ds->ctx->stream = user;
    const int n = (int)(launches_noted() - before);
    note_launch(-n);                                  // captured, not run
    if (rc == IHT_OK && e2 != cudaSuccess) {
        set_cuda_error(e2, "batch iteration capture");
        rc = IHT_ECUDA;
    }
    BatchWork::Graph g;
    if (rc == IHT_OK) {
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        if (e != cudaSuccess) {
            set_cuda_error(e, "batch iteration graph instantiate");
            rc = IHT_ECUDA;
        }
    }
    if (graph) cudaGraphDestroy(graph);
    if (rc) return rc;
    g.launches = n;
    g.pairs = pe.n;
    g.used = ++w->graph_clock;
    *out = &(w->graphs[k] = g);
    return IHT_OK;
}

// Device scratch of one cross-validation call, freed with the object.
struct CvScratch {
    std::vector<void *> p;
    ~CvScratch()
    {
        for (void *x : p)
            if (x) cudaFree(x);
    }
    template <typename T>
    cudaError_t alloc(T **out, size_t count)
    {
        void *x = nullptr;
        const cudaError_t e = dev_malloc(&x, std::max<size_t>(16, sizeof(T) * count));
        if (e == cudaSuccess) p.push_back(x);
        *out = static_cast<T *>(x);
        return e;
    }
};

}  // namespace iht

using namespace iht;

extern "C" {

int iht_fit_batch(iht_dataset *ds, int32_t b, const iht_solve_desc *solves,
                  const iht_options *opt_in, double *betas, int32_t *supports, double *beta_s,
                  iht_result *infos)
{
    iht_options opt;
    if (opt_in)
        opt = *opt_in;
    else
        iht_default_options(&opt);
    if (!ds || b < 1 || !solves || !supports) return IHT_EINVAL;
    if ((opt.in_mem != IHT_HOST && opt.in_mem != IHT_DEVICE) ||
        (opt.out_mem != IHT_HOST && opt.out_mem != IHT_DEVICE) || opt.max_iter < 0 ||
        opt.max_backtrack < 0 || !(opt.kappa > 1.0) || !(opt.c >= 0.0 && opt.c < 1.0) ||
        !(opt.tol >= 0.0) || opt.grad_impl < 0 || opt.grad_impl > 2 ||
        opt.variant != IHT_VARIANT_IHT || ds->q > 0)
        return IHT_EINVAL;
    int kmax = 0;
    int64_t ytot = 0;
    for (int c = 0; c < b; ++c) {
        const iht_solve_desc &d = solves[c];
        const int64_t nr = d.rows ? d.n_rows : ds->n;
        if (!d.y || nr < 2 || nr > ds->n || d.k < 1 || d.k > ds->p || d.k > kMaxK) return IHT_EINVAL;
        kmax = std::max(kmax, (int)d.k);
        ytot += nr;
    }
    if (opt.grad_impl != 1 && !grad_mrhs_supported(ds)) return IHT_EINVAL;
    DeviceGuard g(ds->ctx->device);
    if (!g.ok) return IHT_ECUDA;
    int rc = ensure_workspace(ds, kmax);
    if (rc) return rc;
    cudaStream_t s = ds->ctx->stream;
    std::vector<const int32_t *> rows(b);
    std::vector<int64_t> nrows(b);
    for (int c = 0; c < b; ++c) {
        rows[c] = solves[c].rows;
        nrows[c] = solves[c].n_rows;
    }
    std::vector<SetKey> sets;
    std::vector<int> set_of;
    dedupe_sets(b, rows.data(), nrows.data(), ds->n, sets, set_of);
    int64_t rtot = 0;
    for (const SetKey &k : sets)
        if (k.rows) rtot += k.n_rows;
    if ((rc = ensure_batchwork(ds, b, kmax, (int)sets.size(), opt.in_mem == IHT_HOST ? rtot : 0,
                               opt.in_mem == IHT_HOST ? ytot : 0)))
        return rc;
    BatchWork *w = ds->ws->bw;
    std::vector<const int32_t *> set_rows;
    if ((rc = build_sets(ds, w, sets, opt.in_mem, set_rows))) return rc;

    const size_t np = (size_t)ds->n_pad, p = (size_t)ds->p, K = (size_t)w->kcap;
    const int npart = zmul_blocks(ds);

    // phenotypes, finite check, per-solve state
    if ((rc = grad_mrhs_reset_status(ds)) || (rc = grad_tc_reset_status(ds))) return rc;
    IHT_CUDA(cudaMemsetAsync(w->sc, 0, sizeof(Scalars) * b, s));
    int64_t yoff = 0, koff = 0;
    for (int c = 0; c < b; ++c) {
        const iht_solve_desc &d = solves[c];
        const int64_t nr = d.rows ? d.n_rows : ds->n;
        const double *ydev = d.y;
        if (opt.in_mem == IHT_HOST) {
            IHT_CUDA(cudaMemcpyAsync(w->ybuf + yoff, d.y, sizeof(double) * nr, cudaMemcpyHostToDevice, s));
            ydev = w->ybuf + yoff;
            yoff += nr;
        }
        if ((rc = check_finite_y_sc(ds, nr, ydev, w->sc + c))) return rc;
        if ((rc = scatter_rows_f64(ds, set_rows[set_of[c]], nr, ydev, w->y64 + c * np))) return rc;
    }
    IHT_CUDA(cudaMemcpyAsync(w->sc_host, w->sc, sizeof(Scalars) * b, cudaMemcpyDeviceToHost, s));
    IHT_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < b; ++c) {
        const int32_t err = w->sc_host[c].err;
        Scalars h{};
        h.c = opt.c;
        h.kappa = opt.kappa;
        h.tol = opt.tol;
        h.max_iter = opt.max_iter;
        h.max_backtrack = opt.max_backtrack;
        h.k = solves[c].k;
        h.n_rows = (int32_t)(solves[c].rows ? solves[c].n_rows : ds->n);
        h.status = (err & 1) ? IHT_ENUMERIC : IHT_ENOTCONV;
        h.done = (err & 1) || opt.max_iter <= 0 ? 1 : 0;
        h.err = err;
        h.fresh = 1;
        w->sc_host[c] = h;
        const RowSet rs = batch_rowset(ds, w, set_of[c]);
        BSolve &B = w->bs_host[c];
        B.sc = w->sc + c;
        B.used = rs.used;
        B.u64 = rs.u64;
        B.v64 = rs.v64;
        B.y64 = w->y64 + c * np;
        B.r64 = w->r64 + c * np;
        B.rc64 = w->rc64 + c * np;
        B.zv = w->zv + c * np;
        B.r32 = w->r32 + c * np;
        B.g = w->g + c * p;
        B.S = w->S + c * K;
        B.Sp = w->Sp + c * K;
        B.cand = w->cand + c * 2 * K;
        B.bS = w->bS + c * K;
        B.bSp = w->bSp + c * K;
        B.coef = w->coef + c * K;
        B.partials = w->partials + (size_t)c * 3 * kPartials;
        B.k = solves[c].k;
        B.K = (int32_t)std::min<int64_t>(2 * (int64_t)solves[c].k, ds->p);
        B.out_off = koff;
        koff += B.k;
        for (int t = 0; t < 2; ++t) {            // t = 0: S^0 = top-k; t = 1: candidates
            SelJob &J = w->jobs_host[t * b + c];
            J.keys = B.g;
            J.out = t == 0 ? B.S : B.cand;
            J.st = w->st + t * b + c;
            J.hist = w->hist + (size_t)(t * b + c) * kSelBins;
            J.cand = w->selcand + (size_t)(t * b + c) * kSelCap;
            J.done = &w->sc[c].done;
            J.K = (uint32_t)(t == 0 ? B.k : B.K);
        }
    }
    IHT_CUDA(cudaMemcpyAsync(w->sc, w->sc_host, sizeof(Scalars) * b, cudaMemcpyHostToDevice, s));
    IHT_CUDA(cudaMemcpyAsync(w->bs, w->bs_host, sizeof(BSolve) * b, cudaMemcpyHostToDevice, s));
    IHT_CUDA(cudaMemcpyAsync(w->jobs, w->jobs_host, sizeof(SelJob) * 2 * b, cudaMemcpyHostToDevice, s));

    const bool prof = opt.profile != 0;
    if (prof && !w->ev[0])
        for (int e = 0; e < 2 * kProfEvents; ++e) IHT_CUDA(cudaEventCreate(&w->ev[e]));
    ProfEvents pe;
    pe.ev = w->ev;
    pe.cap = prof ? kProfEvents : 0;
    auto grad = [&](const std::vector<int> &act) -> int {
        return batch_grad(ds, w, act, set_of, opt.grad_impl, prof ? &pe : nullptr);
    };

    std::vector<int> act;
    auto active = [&]() {
        act.clear();
        for (int c = 0; c < b; ++c)
            if (!w->sc_host[c].done) act.push_back(c);
    };
    // beta = 0: r = y, objective, centred residual, g^0, S^0 = top-k |g^0|
    if ((rc = launch_zmul_batch(ds, w->bs, b, kmax, kZmulInit))) return rc;
    if ((rc = launch_init_objective_batch(ds, w->bs, b))) return rc;
    if ((rc = launch_center_batch(ds, w->bs, b, true))) return rc;
    active();
    if ((rc = grad(act))) return rc;
    // solves stopped before S^0 (non-finite y, max_iter = 0) report support -1
    IHT_CUDA(cudaMemsetAsync(w->S, 0xFF, sizeof(int32_t) * b * K, s));
    if ((rc = select_topk_batch(ds->ctx, w->jobs, b, ds->p))) return rc;
    IHT_CUDA(cudaMemsetAsync(w->bS, 0, sizeof(double) * b * K, s));

    double graph_ms = 0.0;
    int graph_pairs = 0, replays = 0;
    std::vector<int> prev;
    for (int it = 0; it < opt.max_iter && !act.empty(); ++it) {
        BatchWork::Graph *gr = nullptr;
        bool replay = false;
        std::string key;
        if (it > 0 && opt.grad_impl != 1) {
            // a graph for this many active columns exists, or the count ran
            // before (in this call or an earlier one: capture it now); a new
            // count runs once as direct launches first (the tuner may time a
            // new width)
            if ((rc = batch_cols(ds, w, act, set_of))) return rc;
            key = batch_graph_key(w, b, kmax, opt.grad_impl, prof, (int)act.size());
            replay = batch_graph_find(w, key) != nullptr || act == prev || w->graph_seen.count(key);
            if (!replay && w->graph_seen.size() < 64 * kBatchGraphs) w->graph_seen.insert(key);
        }
        if (replay) {
            if ((rc = batch_graph(ds, w, b, kmax, opt.grad_impl, prof, act, key, &gr))) return rc;
            IHT_CUDA(cudaGraphLaunch(gr->exec, s));
            note_launch(gr->launches);
            ++replays;
        } else {
            if (it > 0 && (rc = grad(act))) return rc;
            if ((rc = batch_step(ds, w, b, kmax))) return rc;
            if ((rc = batch_attempt(ds, w, b, kmax, true))) return rc;
        }
        for (;;) {
            IHT_CUDA(cudaMemcpyAsync(w->sc_host, w->sc, sizeof(Scalars) * b, cudaMemcpyDeviceToHost, s));
            IHT_CUDA(cudaStreamSynchronize(s));
            bool again = false;
            for (int c : act) again |= !w->sc_host[c].done && w->sc_host[c].live && w->sc_host[c].retry;
            if (!again) break;
            if ((rc = batch_attempt(ds, w, b, kmax, false))) return rc;
        }
        for (int e = 0; gr && prof && e < gr->pairs; ++e) {     // the replay's gradient passes
            float ms = 0.0f;
            IHT_CUDA(cudaEventElapsedTime(&ms, w->gev[2 * e], w->gev[2 * e + 1]));
            graph_ms += ms;
            ++graph_pairs;
        }
        prev = act;
        active();
    }
    int timed_out = 0, tc_timed_out = 0;
    if (opt.grad_impl != 1 && (rc = grad_mrhs_status(ds, &timed_out))) return rc;
    if (opt.grad_impl == 0 && (rc = grad_tc_status(ds, &tc_timed_out))) return rc;
    if (timed_out || tc_timed_out) return IHT_ETIMEOUT;
    double grad_ms = graph_ms;
    const int nprof = pe.n + graph_pairs;
    for (int e = 0; prof && e < pe.n; ++e) {
        float ms = 0.0f;
        IHT_CUDA(cudaEventElapsedTime(&ms, w->ev[2 * e], w->ev[2 * e + 1]));
        grad_ms += ms;
    }

    // outputs: supports / beta_S concatenated in solve order (koff entries), dense betas
    if (opt.out_mem == IHT_DEVICE) {
        if (betas) {
            IHT_CUDA(cudaMemsetAsync(betas, 0, sizeof(double) * b * p, s));
            if ((rc = launch_scatter_beta_batch(ds, w->bs, b, kmax, betas))) return rc;
        }
        if ((rc = launch_compact_support_batch(ds, w->bs, b, kmax, supports, beta_s))) return rc;
        IHT_CUDA(cudaStreamSynchronize(s));
    } else {
        // compacted on the device (into the candidate scratch), then one copy each
        int32_t *sup_dev = w->cand;                               // >= sum of k entries
        double *bs_dev = w->coef;
        if ((rc = launch_compact_support_batch(ds, w->bs, b, kmax, sup_dev, bs_dev))) return rc;
        std::vector<double> bsh(beta_s ? 0 : (size_t)koff);
        double *bdst = beta_s ? beta_s : bsh.data();
        IHT_CUDA(cudaMemcpyAsync(supports, sup_dev, sizeof(int32_t) * koff, cudaMemcpyDeviceToHost, s));
        IHT_CUDA(cudaMemcpyAsync(bdst, bs_dev, sizeof(double) * koff, cudaMemcpyDeviceToHost, s));
        IHT_CUDA(cudaStreamSynchronize(s));
        if (betas) {
            memset(betas, 0, sizeof(double) * b * p);
            int64_t o = 0;
            for (int c = 0; c < b; ++c) {
                for (int t = 0; t < solves[c].k; ++t) {
                    const int32_t j = supports[o + t];
                    if (j >= 0 && (size_t)j < p) betas[(size_t)c * p + j] = bdst[o + t];
                }
                o += solves[c].k;
            }
        }
    }
    if (infos) {
        for (int c = 0; c < b; ++c) {
            const Scalars &h = w->sc_host[c];
            iht_result &r = infos[c];
            r.iterations = h.iter;
            r.status = h.status;
            r.backtracks = h.bt_total;
            r.reserved = 0;
            r.objective = h.f;
            r.mu = h.mu;
            r.grad_ms = prof ? grad_ms : 0.0;
            r.grad_launches = prof ? nprof : 0;
            r.graph_replays = replays;
        }
    }
    return IHT_OK;
}

int iht_cv(iht_dataset *ds, const double *y, const int32_t *fold, int32_t q, const int32_t *ks, int32_t nk,
           const iht_options *opt_in, double *mse, double *mse_fold, int32_t *k_best, double *beta_out,
           int32_t *support_out, iht_result *info)
{
    if (!ds || !y || !fold || !ks || q < 2 || q > 64 || nk < 1) return IHT_EINVAL;
    iht_options opt;
    if (opt_in)
        opt = *opt_in;
    else
        iht_default_options(&opt);
    const int64_t n = ds->n, p = ds->p;
    if (opt.variant != IHT_VARIANT_IHT || ds->q > 0) return IHT_EINVAL;
    for (int t = 0; t < nk; ++t)
        if (ks[t] < 1 || ks[t] > p || ks[t] > kMaxK) return IHT_EINVAL;
    // partitions: test rows of f, training rows = the other partitions' (label
    // -1: a subject outside the selection and the refit)
    std::vector<std::vector<int32_t>> train(q), test(q);
    std::vector<int32_t> inside;
    for (int64_t i = 0; i < n; ++i) {
        const int32_t f = fold[i];
        if (f < -1 || f >= q) return IHT_EINVAL;
        if (f < 0) continue;
        test[f].push_back((int32_t)i);
        inside.push_back((int32_t)i);
    }
    const int64_t n_in = (int64_t)inside.size();
    for (int f = 0; f < q; ++f) {
        if (test[f].empty() || n_in - (int64_t)test[f].size() < 2) return IHT_EINVAL;
        train[f].reserve(n_in - test[f].size());
        for (int32_t i : inside)
            if (fold[i] != f) train[f].push_back(i);
    }
    std::vector<std::vector<double>> ytr(q);
    for (int f = 0; f < q; ++f) {
        ytr[f].resize(train[f].size());
        for (size_t a = 0; a < train[f].size(); ++a) ytr[f][a] = y[train[f][a]];
    }
    const int nb = q * nk;
    std::vector<iht_solve_desc> solves(nb);
    int64_t ktot = 0;
    std::vector<int64_t> koff(nb);
    for (int f = 0; f < q; ++f)
        for (int t = 0; t < nk; ++t) {
            iht_solve_desc &d = solves[f * nk + t];
            memset(&d, 0, sizeof(d));
            d.rows = train[f].data();
            d.n_rows = (int64_t)train[f].size();
            d.y = ytr[f].data();
            d.k = ks[t];
            koff[f * nk + t] = ktot;
            ktot += ks[t];
        }
    DeviceGuard g(ds->ctx->device);
    if (!g.ok) return IHT_ECUDA;
    cudaStream_t s = ds->ctx->stream;
    CvScratch sc;
    int32_t *sup_d = nullptr, *used_d = nullptr;
    double *bs_d = nullptr, *y64_d = nullptr, *out_d = nullptr, *part_d = nullptr;
    CvJob *jobs_d = nullptr;
    const size_t np = (size_t)ds->n_pad;
    const int nblk = zmul_blocks(ds);
    IHT_CUDA(sc.alloc(&sup_d, ktot));
    IHT_CUDA(sc.alloc(&bs_d, ktot));
    IHT_CUDA(sc.alloc(&used_d, (size_t)q * np));
    IHT_CUDA(sc.alloc(&y64_d, np));
    IHT_CUDA(sc.alloc(&out_d, (size_t)nb * np));
    IHT_CUDA(sc.alloc(&part_d, (size_t)nb * 3 * nblk));
    IHT_CUDA(sc.alloc(&jobs_d, (size_t)nb));

    // every (partition, size) fit as one batch, host inputs, device outputs
    iht_options o = opt;
    o.in_mem = IHT_HOST;
    o.out_mem = IHT_DEVICE;
    std::vector<iht_result> fits(nb);
    int rc = iht_fit_batch(ds, nb, solves.data(), &o, nullptr, sup_d, bs_d, fits.data());
    if (rc) return rc;
    for (const iht_result &r : fits)
        if (r.status == IHT_ENUMERIC) return IHT_ENUMERIC;

    // out-of-fold residuals with the training rows' statistics (row set f of
    // the batch: the solves list partition f's training rows first at f * nk)
    BatchWork *w = ds->ws->bw;
    std::vector<SetKey> sets;
    std::vector<int> set_of;
    {
        std::vector<const int32_t *> rows(nb);
        std::vector<int64_t> nrows(nb);
        for (int c = 0; c < nb; ++c) {
            rows[c] = solves[c].rows;
            nrows[c] = solves[c].n_rows;
        }
        dedupe_sets(nb, rows.data(), nrows.data(), n, sets, set_of);
    }
    std::vector<int32_t> used_h((size_t)q * np, 0);
    std::vector<double> y64_h(np, 0.0);
    for (int f = 0; f < q; ++f)
        for (int32_t i : test[f]) used_h[(size_t)f * np + i] = 1;
    for (int64_t i = 0; i < n; ++i) y64_h[i] = y[i];
    std::vector<CvJob> jobs(nb);
    for (int f = 0; f < q; ++f)
        for (int t = 0; t < nk; ++t) {
            const int c = f * nk + t;
            const RowSet rs = batch_rowset(ds, w, set_of[c]);
            CvJob &J = jobs[c];
            J.S = sup_d + koff[c];
            J.bS = bs_d + koff[c];
            J.k = ks[t];
            J.used = used_d + (size_t)f * np;
            J.u64 = rs.u64;
            J.v64 = rs.v64;
            J.y64 = y64_d;
            J.out = out_d + (size_t)c * np;
            J.partials = part_d + (size_t)c * 3 * nblk;
        }
    IHT_CUDA(cudaMemcpyAsync(used_d, used_h.data(), sizeof(int32_t) * used_h.size(), cudaMemcpyHostToDevice, s));
    IHT_CUDA(cudaMemcpyAsync(y64_d, y64_h.data(), sizeof(double) * np, cudaMemcpyHostToDevice, s));
    IHT_CUDA(cudaMemcpyAsync(jobs_d, jobs.data(), sizeof(CvJob) * nb, cudaMemcpyHostToDevice, s));
    if ((rc = launch_cv_resid(ds, jobs_d, nb))) return rc;
    std::vector<double> part_h((size_t)nb * 3 * nblk);
    IHT_CUDA(cudaMemcpyAsync(part_h.data(), part_d, sizeof(double) * part_h.size(), cudaMemcpyDeviceToHost, s));
    IHT_CUDA(cudaStreamSynchronize(s));

    // MSE per partition and size (block sums in order), averaged over partitions
    std::vector<double> mf((size_t)q * nk), mm(nk, 0.0);
    for (int c = 0; c < nb; ++c) {
        double ss = 0.0;
        for (int b = 0; b < nblk; ++b) ss += part_h[(size_t)c * 3 * nblk + 3 * b + 1];
        mf[c] = ss / (double)test[c / nk].size();
    }
    for (int t = 0; t < nk; ++t) {
        double a = 0.0;
        for (int f = 0; f < q; ++f) a += mf[f * nk + t];
        mm[t] = a / q;
    }
    int best = 0;
    for (int t = 1; t < nk; ++t)
        if (mm[t] < mm[best]) best = t;
    if (mse) memcpy(mse, mm.data(), sizeof(double) * nk);
    if (mse_fold) memcpy(mse_fold, mf.data(), sizeof(double) * mf.size());
    if (k_best) *k_best = ks[best];

    // the refit on all rows of the partitions at the chosen size
    std::vector<double> bfull(beta_out ? 0 : (size_t)p);
    std::vector<int32_t> sfull(support_out ? 0 : (size_t)ks[best]);
    iht_options ro = opt;
    ro.in_mem = IHT_HOST;
    ro.out_mem = IHT_HOST;
    const bool all = n_in == n;
    std::vector<double> yin(all ? 0 : (size_t)n_in);
    for (int64_t a = 0; !all && a < n_in; ++a) yin[a] = y[inside[a]];
    return iht_fit(ds, all ? nullptr : inside.data(), n_in, all ? y : yin.data(), ks[best], &ro,
                   beta_out ? beta_out : bfull.data(), support_out ? support_out : sfull.data(), info);
}

int iht_gradient_batch(iht_dataset *ds, int32_t b, const int32_t *const *rows_list,
                       const int64_t *n_rows, const float *R, float *G_out, int impl)
{
    if (!ds || b < 1 || !rows_list || !n_rows || !R || !G_out || impl < 0 || impl > 2)
        return IHT_EINVAL;
    for (int c = 0; c < b; ++c) {
        const int64_t nr = rows_list[c] ? n_rows[c] : ds->n;
        if (nr < 1 || nr > ds->n) return IHT_EINVAL;
    }
    if (impl != 1 && !grad_mrhs_supported(ds)) return IHT_EINVAL;
    DeviceGuard g(ds->ctx->device);
    if (!g.ok) return IHT_ECUDA;
    int rc = ensure_workspace(ds, 0);
    if (rc) return rc;
    std::vector<SetKey> sets;
    std::vector<int> set_of;
    dedupe_sets(b, rows_list, n_rows, ds->n, sets, set_of);
    if ((rc = ensure_batchwork(ds, b, 1, (int)sets.size(), 0, 0))) return rc;
    BatchWork *w = ds->ws->bw;
    std::vector<const int32_t *> set_rows;
    if ((rc = build_sets(ds, w, sets, IHT_DEVICE, set_rows))) return rc;
    const size_t np = (size_t)ds->n_pad, p = (size_t)ds->p;
    std::vector<int> act(b);
    for (int c = 0; c < b; ++c) {
        act[c] = c;
        if ((rc = scatter_rows_f32(ds, set_rows[set_of[c]], sets[set_of[c]].n_rows,
                                   R + (size_t)c * ds->n, w->r32 + c * np)))
            return rc;
    }
    if ((rc = grad_mrhs_reset_status(ds)) || (rc = grad_tc_reset_status(ds))) return rc;
    if ((rc = batch_grad(ds, w, act, set_of, impl))) return rc;
    cudaStream_t s = ds->ctx->stream;
    IHT_CUDA(cudaMemcpyAsync(G_out, w->g, sizeof(float) * b * p, cudaMemcpyDeviceToDevice, s));
    IHT_CUDA(cudaStreamSynchronize(s));
    int timed_out = 0, tc_timed_out = 0;
    if (impl != 1 && (rc = grad_mrhs_status(ds, &timed_out))) return rc;
    if (impl == 0 && (rc = grad_tc_status(ds, &tc_timed_out))) return rc;
    return timed_out || tc_timed_out ? IHT_ETIMEOUT : IHT_OK;
}

}  // extern "C"
