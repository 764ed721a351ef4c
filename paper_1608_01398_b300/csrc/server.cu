// a8: continuous-batching IHT server.
//
// A worker thread owns a stream on the dataset's device and runs ticks.  At
// the start of a tick it admits queued requests (first come, first served)
// while a slot is free and the request's device footprint fits the budget;
// a newly admitted solve gets its row marks, phenotype and the beta = 0
// set-up, and the per-SNP statistics of all requests admitted in the same
// tick come from one pass over the genotypes.  The tick then runs one IHT
// iteration for every active solve: one multi-column gradient pass (each
// solve is a column; the newly admitted ones take g^0 from it and select
// S^0 = top-k |g^0| first), then the candidate selection, step size and
// backtracking attempts as batched launches over the slots (blockIdx = slot,
// empty and finished slots return at once).  Solves that stopped are copied
// out, their memory is released on the stream and their slot is free for the
// next tick.  Every per-solve computation reads only that solve's data, so a
// solve's result does not depend on the solves that shared its ticks.
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "common.cuh"

namespace iht {

using Clock = std::chrono::steady_clock;

struct SrvRequest {
    uint64_t ticket = 0;
    bool all_rows = true;
    std::vector<int32_t> rows;
    std::vector<double> y;
    int32_t k = 0;
    int64_t n_rows = 0;
    size_t bytes = 0;
    Clock::time_point t_submit;
};

struct SrvResult {
    std::vector<int32_t> S;
    std::vector<double> bS;
    iht_result info{};
    double latency = 0.0;
};

// Device pieces of one admitted solve, carved from one stream-ordered block.
struct SlotMem {
    RowSet rs;
    double *y64, *r64, *rc64, *zv;
    float *r32, *g;
    int32_t *S, *Sp, *cand;
    double *bS, *bSp, *coef, *partials;
    SelState *st;
    uint32_t *hist;
    unsigned long long *selcand;
    int32_t *rows;
    double *ystage;
};

struct Slot {
    bool busy = false;
    bool fresh = false;
    uint64_t ticket = 0;
    int32_t k = 0, K = 0;
    int64_t n_rows = 0;
    void *block = nullptr;
    size_t bytes = 0;
    Clock::time_point t_submit;
    SlotMem m{};
};

static size_t al256(size_t b) { return (b + 255) / 256 * 256; }

// Carves (or, with base == nullptr, only sizes) the pieces of one solve.
static size_t slot_layout(const iht_dataset *ds, int k, int64_t n_rows, char *base, SlotMem *m)
{
    const size_t np = (size_t)ds->n_pad, p = (size_t)ds->p;
    const size_t K = (size_t)std::min<int64_t>(2 * (int64_t)k, ds->p);
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *q = base ? base + off : nullptr;
        off += al256(std::max<size_t>(bytes, 16));
        return q;
    };
    SlotMem t{};
    t.rs.used = (int32_t *)take(sizeof(int32_t) * np);
    t.rs.rowmask = (uint32_t *)take(sizeof(uint32_t) * (size_t)(ds->stride / 4));
    t.rs.counts = nullptr;
    t.rs.u64 = (double *)take(sizeof(double) * p);
    t.rs.v64 = (double *)take(sizeof(double) * p);
    t.rs.u32 = (float *)take(sizeof(float) * p);
    t.rs.v32 = (float *)take(sizeof(float) * p);
    t.y64 = (double *)take(sizeof(double) * np);
    t.r64 = (double *)take(sizeof(double) * np);
    t.rc64 = (double *)take(sizeof(double) * np);
    t.zv = (double *)take(sizeof(double) * np);
    t.r32 = (float *)take(sizeof(float) * np);
    t.g = (float *)take(sizeof(float) * p);
    t.S = (int32_t *)take(sizeof(int32_t) * k);
    t.Sp = (int32_t *)take(sizeof(int32_t) * k);
    t.cand = (int32_t *)take(sizeof(int32_t) * K);
    t.bS = (double *)take(sizeof(double) * k);
    t.bSp = (double *)take(sizeof(double) * k);
    t.coef = (double *)take(sizeof(double) * k);
    t.partials = (double *)take(sizeof(double) * 3 * kPartials);
    t.st = (SelState *)take(sizeof(SelState) * 2);
    t.hist = (uint32_t *)take(sizeof(uint32_t) * 2 * kSelBins);
    t.selcand = (unsigned long long *)take(sizeof(unsigned long long) * 2 * kSelCap);
    t.rows = (int32_t *)take(sizeof(int32_t) * (size_t)n_rows);
    t.ystage = (double *)take(sizeof(double) * (size_t)n_rows);
    if (m) *m = t;
    return off;
}

}  // namespace iht

using namespace iht;

struct iht_server {
    iht_ctx ctx{};              // own stream on the dataset's device
    iht_dataset view{};         // shares the caller's genotypes and missing-call lists
    iht_options opt{};
    int max_slots = 0;
    uint64_t budget = 0;
    // fixed device arrays, one entry per slot (+ pinned mirrors)
    Scalars *sc = nullptr, *sc_host = nullptr;
    BSolve *bs = nullptr, *bs_host = nullptr;
    SelJob *jobs_c = nullptr, *jobs_c_host = nullptr;   // candidate selection, per slot
    SelJob *jobs_s = nullptr, *jobs_s_host = nullptr;   // S^0 of the newly admitted slots
    MrCol *cols = nullptr, *cols_host = nullptr;
    int32_t *outS_host = nullptr;                        // retirement staging, k <= kMaxK per slot
    double *outB_host = nullptr;
    std::vector<Slot> slots;
    // host side, guarded by mu
    std::mutex mu;
    std::condition_variable cv;
    std::deque<SrvRequest> pending;
    std::unordered_set<uint64_t> live;                   // queued or running tickets
    std::unordered_map<uint64_t, SrvResult> results;
    uint64_t next_ticket = 1;
    iht_server_stats st{};
    int failed = 0;                                      // worker status once it failed
    bool stop = false;
    std::thread worker;
};

namespace iht {

static int srv_admit_setup(iht_server *S, const std::vector<int> &fresh, std::vector<SrvRequest> &reqs)
{
    iht_dataset *ds = &S->view;
    cudaStream_t s = ds->ctx->stream;
    const int64_t np = ds->n_pad;
    std::vector<RowSet> rsets;
    std::vector<int64_t> nrows;
    for (size_t a = 0; a < fresh.size(); ++a) {
        Slot &sl = S->slots[fresh[a]];
        const SrvRequest &q = reqs[a];
        IHT_CUDA(dev_malloc_async(&sl.block, q.bytes, s));
        slot_layout(ds, q.k, q.n_rows, (char *)sl.block, &sl.m);
        SlotMem &m = sl.m;
        sl.busy = true;
        sl.fresh = true;
        sl.ticket = q.ticket;
        sl.k = q.k;
        sl.K = (int32_t)std::min<int64_t>(2 * (int64_t)q.k, ds->p);
        sl.n_rows = q.n_rows;
        sl.bytes = q.bytes;
        sl.t_submit = q.t_submit;
        const int c = fresh[a];
        Scalars h{};
        h.c = S->opt.c;
        h.kappa = S->opt.kappa;
        h.tol = S->opt.tol;
        h.max_iter = S->opt.max_iter;
        h.max_backtrack = S->opt.max_backtrack;
        h.k = q.k;
        h.n_rows = (int32_t)q.n_rows;
        h.status = IHT_ENOTCONV;
        h.done = S->opt.max_iter <= 0 ? 1 : 0;
        h.fresh = 1;
        S->sc_host[c] = h;
        IHT_CUDA(cudaMemcpyAsync(S->sc + c, S->sc_host + c, sizeof(Scalars), cudaMemcpyHostToDevice, s));
        if (!q.all_rows)
            IHT_CUDA(cudaMemcpyAsync(m.rows, q.rows.data(), sizeof(int32_t) * q.n_rows,
                                     cudaMemcpyHostToDevice, s));
        IHT_CUDA(cudaMemcpyAsync(m.ystage, q.y.data(), sizeof(double) * q.n_rows,
                                 cudaMemcpyHostToDevice, s));
        IHT_CUDA(cudaMemsetAsync(m.S, 0xFF, sizeof(int32_t) * q.k, s));
        IHT_CUDA(cudaMemsetAsync(m.bS, 0, sizeof(double) * q.k, s));
        // selection scratch starts zeroed; every selection leaves it so
        IHT_CUDA(cudaMemsetAsync(m.st, 0, sizeof(SelState) * 2, s));
        IHT_CUDA(cudaMemsetAsync(m.hist, 0, sizeof(uint32_t) * 2 * kSelBins, s));
        const int32_t *rows_dev = q.all_rows ? nullptr : m.rows;
        int rc;
        if ((rc = setup_rowset(ds, rows_dev, q.n_rows, m.rs, &S->sc[c].err))) return rc;
        if ((rc = check_finite_y_sc(ds, q.n_rows, m.ystage, S->sc + c))) return rc;
        if ((rc = scatter_rows_f64(ds, rows_dev, q.n_rows, m.ystage, m.y64))) return rc;
        rsets.push_back(m.rs);
        nrows.push_back(q.n_rows);
        BSolve &B = S->bs_host[c];
        B.sc = S->sc + c;
        B.used = m.rs.used;
        B.u64 = m.rs.u64;
        B.v64 = m.rs.v64;
        B.y64 = m.y64;
        B.r64 = m.r64;
        B.rc64 = m.rc64;
        B.zv = m.zv;
        B.r32 = m.r32;
        B.g = m.g;
        B.S = m.S;
        B.Sp = m.Sp;
        B.cand = m.cand;
        B.bS = m.bS;
        B.bSp = m.bSp;
        B.coef = m.coef;
        B.partials = m.partials;
        B.k = q.k;
        B.K = sl.K;
        B.out_off = 0;
        IHT_CUDA(cudaMemcpyAsync(S->bs + c, &B, sizeof(BSolve), cudaMemcpyHostToDevice, s));
        SelJob &J = S->jobs_c_host[c];
        J.keys = m.g;
        J.out = m.cand;
        J.st = m.st + 1;
        J.hist = m.hist + kSelBins;
        J.cand = m.selcand + kSelCap;
        J.done = &S->sc[c].done;
        J.K = (uint32_t)sl.K;
        IHT_CUDA(cudaMemcpyAsync(S->jobs_c + c, &J, sizeof(SelJob), cudaMemcpyHostToDevice, s));
    }
    int rc = launch_counts_sets(ds, rsets.data(), nrows.data(), (int)rsets.size());
    if (rc) return rc;
    // input errors of the new solves (bad rows, non-finite y) end them before the first step
    for (int c : fresh)
        IHT_CUDA(cudaMemcpyAsync(&S->sc_host[c].err, &S->sc[c].err, sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, s));
    IHT_CUDA(cudaStreamSynchronize(s));
    for (int c : fresh) {
        Scalars &h = S->sc_host[c];
        if (h.err) {
            h.done = 1;
            h.status = (h.err & 2) ? IHT_EINVAL : IHT_ENUMERIC;
            IHT_CUDA(cudaMemcpyAsync(S->sc + c, &h, sizeof(Scalars), cudaMemcpyHostToDevice, s));
        }
    }
    (void)np;
    return IHT_OK;
}

// One IHT iteration for every active slot; fresh slots get their set-up first.
static int srv_tick(iht_server *S, const std::vector<int> &fresh)
{
    iht_dataset *ds = &S->view;
    cudaStream_t s = ds->ctx->stream;
    const int nb = S->max_slots;
    int kmax = 1;
    std::vector<int> act;
    for (int c = 0; c < nb; ++c) {
        const Slot &sl = S->slots[c];
        if (!sl.busy) continue;
        kmax = std::max(kmax, (int)sl.k);
        if (!S->sc_host[c].done) act.push_back(c);
    }
    int rc;
    if (!fresh.empty()) {
        if ((rc = launch_zmul_batch(ds, S->bs, nb, kmax, kZmulInit))) return rc;
        if ((rc = launch_init_objective_batch(ds, S->bs, nb))) return rc;
        if ((rc = launch_center_batch(ds, S->bs, nb, true))) return rc;
    }
    if (!act.empty()) {
        for (size_t a = 0; a < act.size(); ++a) {
            const SlotMem &m = S->slots[act[a]].m;
            MrCol &C = S->cols_host[a];
            C.r32 = m.r32;
            C.u32 = m.rs.u32;
            C.v32 = m.rs.v32;
            C.g = m.g;
            C.scale = 0.0f;
            C.R = 0.0f;
        }
        IHT_CUDA(cudaMemcpyAsync(S->cols, S->cols_host, sizeof(MrCol) * act.size(),
                                 cudaMemcpyHostToDevice, s));
        if ((rc = launch_grad_mrhs(ds, S->cols, (int)act.size(), nullptr, S->cols_host))) return rc;
    }
    if (!fresh.empty()) {
        int nf = 0;
        for (int c : fresh) {
            const SlotMem &m = S->slots[c].m;
            SelJob &J = S->jobs_s_host[nf++];
            J.keys = m.g;
            J.out = m.S;
            J.st = m.st;
            J.hist = m.hist;
            J.cand = m.selcand;
            J.done = &S->sc[c].done;
            J.K = (uint32_t)S->slots[c].k;
        }
        IHT_CUDA(cudaMemcpyAsync(S->jobs_s, S->jobs_s_host, sizeof(SelJob) * nf, cudaMemcpyHostToDevice, s));
        if ((rc = select_topk_batch(&S->ctx, S->jobs_s, nf, ds->p))) return rc;
        if ((rc = launch_finish_fresh_batch(ds, S->bs, nb, kmax))) return rc;
        for (int c : fresh) S->slots[c].fresh = false;
    }
    if (act.empty()) return IHT_OK;
    if ((rc = select_topk_batch(&S->ctx, S->jobs_c, nb, ds->p))) return rc;
    if ((rc = launch_gather_gS_batch(ds, S->bs, nb))) return rc;
    if ((rc = launch_zmul_batch(ds, S->bs, nb, kmax, kZmulStep))) return rc;
    for (int attempt = 0;; ++attempt) {
        if ((rc = launch_merge_batch(ds, S->bs, nb, attempt == 0))) return rc;
        if ((rc = launch_zmul_batch(ds, S->bs, nb, kmax, kZmulResidual))) return rc;
        if ((rc = launch_decide_batch(ds, S->bs, nb))) return rc;
        if ((rc = launch_center_batch(ds, S->bs, nb, false))) return rc;
        IHT_CUDA(cudaMemcpyAsync(S->sc_host, S->sc, sizeof(Scalars) * nb, cudaMemcpyDeviceToHost, s));
        IHT_CUDA(cudaStreamSynchronize(s));
        bool again = false;
        for (int c : act) again |= !S->sc_host[c].done && S->sc_host[c].live && S->sc_host[c].retry;
        if (!again) break;
    }
    return IHT_OK;
}

// Copies out the solves that stopped and frees their slots.
static int srv_retire(iht_server *S)
{
    iht_dataset *ds = &S->view;
    cudaStream_t s = ds->ctx->stream;
    std::vector<int> out;
    for (int c = 0; c < S->max_slots; ++c)
        if (S->slots[c].busy && S->sc_host[c].done) out.push_back(c);
    if (out.empty()) return IHT_OK;
    for (int c : out) {
        const Slot &sl = S->slots[c];
        IHT_CUDA(cudaMemcpyAsync(S->outS_host + (size_t)c * kMaxK, sl.m.S, sizeof(int32_t) * sl.k,
                                 cudaMemcpyDeviceToHost, s));
        IHT_CUDA(cudaMemcpyAsync(S->outB_host + (size_t)c * kMaxK, sl.m.bS, sizeof(double) * sl.k,
                                 cudaMemcpyDeviceToHost, s));
    }
    IHT_CUDA(cudaStreamSynchronize(s));
    const Clock::time_point now = Clock::now();
    std::vector<std::pair<uint64_t, SrvResult>> done;
    for (int c : out) {
        Slot &sl = S->slots[c];
        const Scalars &h = S->sc_host[c];
        SrvResult r;
        r.S.assign(S->outS_host + (size_t)c * kMaxK, S->outS_host + (size_t)c * kMaxK + sl.k);
        r.bS.assign(S->outB_host + (size_t)c * kMaxK, S->outB_host + (size_t)c * kMaxK + sl.k);
        r.info.iterations = h.iter;
        r.info.status = h.status;
        r.info.backtracks = h.bt_total;
        r.info.objective = h.f;
        r.info.mu = h.mu;
        r.latency = std::chrono::duration<double>(now - sl.t_submit).count();
        done.emplace_back(sl.ticket, std::move(r));
        IHT_CUDA(cudaFreeAsync(sl.block, s));
        sl.block = nullptr;
        sl.busy = false;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    for (auto &d : done) {
        S->results.emplace(d.first, std::move(d.second));
        S->live.erase(d.first);
    }
    for (int c : out) {
        S->st.bytes_in_use -= S->slots[c].bytes;
        S->st.completed += 1;
        S->st.active -= 1;
    }
    return IHT_OK;
}

static void srv_run(iht_server *S)
{
    cudaSetDevice(S->ctx.device);
    int rc = IHT_OK;
    for (;;) {
        std::vector<int> fresh;
        std::vector<SrvRequest> reqs;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] { return S->stop || !S->pending.empty() || S->st.active > 0; });
            if (S->stop) break;
            // admission: first come, first served, while a slot is free and the footprint fits
            int free_slot = 0;
            while (!S->pending.empty()) {
                const SrvRequest &q = S->pending.front();
                while (free_slot < S->max_slots && S->slots[free_slot].busy) ++free_slot;
                if (free_slot >= S->max_slots) break;
                if (S->budget && S->st.bytes_in_use + q.bytes > S->budget) break;
                S->slots[free_slot].busy = true;            // reserved; filled below
                fresh.push_back(free_slot);
                S->st.bytes_in_use += q.bytes;
                S->st.max_bytes_in_use = std::max(S->st.max_bytes_in_use, S->st.bytes_in_use);
                S->st.admitted += 1;
                S->st.active += 1;
                S->st.max_active = std::max(S->st.max_active, S->st.active);
                reqs.push_back(std::move(S->pending.front()));
                S->pending.pop_front();
            }
            S->st.ticks += 1;
        }
        if (!fresh.empty() && (rc = srv_admit_setup(S, fresh, reqs))) break;
        if ((rc = srv_tick(S, fresh))) break;
        if ((rc = srv_retire(S))) break;
        if ((S->st.ticks & 15) == 0) {             // bounded waits of the gradient passes
            int timed_out = 0, tc_timed_out = 0;
            if ((rc = grad_mrhs_status(&S->view, &timed_out))) break;
            if ((rc = grad_tc_status(&S->view, &tc_timed_out))) break;
            if (timed_out || tc_timed_out) {
                rc = IHT_ETIMEOUT;
                break;
            }
        }
    }
    if (rc != IHT_OK) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->failed = rc;
    }
    cudaStreamSynchronize(S->ctx.stream);
    grad_mrhs_release_thread();
    grad_tc_release_thread();
}

static size_t srv_footprint(const iht_dataset *ds, int k, int64_t n_rows)
{
    return slot_layout(ds, k, n_rows, nullptr, nullptr);
}

static void srv_free(iht_server *S)
{
    DeviceGuard g(S->ctx.device);
    if (S->ctx.stream) cudaStreamSynchronize(S->ctx.stream);
    for (Slot &sl : S->slots)
        if (sl.block) cudaFree(sl.block);
    void *dev[] = {S->sc, S->bs, S->jobs_c, S->jobs_s, S->cols};
    for (void *p : dev)
        if (p) cudaFree(p);
    void *host[] = {S->sc_host, S->bs_host, S->jobs_c_host, S->jobs_s_host, S->cols_host,
                    S->outS_host, S->outB_host};
    for (void *p : host)
        if (p) cudaFreeHost(p);
    if (S->ctx.sel.hist) cudaFree(S->ctx.sel.hist);
    if (S->ctx.sel.st) cudaFree(S->ctx.sel.st);
    if (S->ctx.sel.cand) cudaFree(S->ctx.sel.cand);
    if (S->ctx.stream) cudaStreamDestroy(S->ctx.stream);
    delete S;
}

}  // namespace iht

extern "C" {

void iht_server_default_options(iht_server_options *o)
{
    if (!o) return;
    o->max_slots = 64;
    o->reserved = 0;
    o->hbm_budget = 0;
    iht_default_options(&o->solve);
}

int iht_server_create(iht_dataset *ds, const iht_server_options *opt_in, iht_server **out)
{
    if (!ds || !out) return IHT_EINVAL;
    *out = nullptr;
    iht_server_options opt;
    if (opt_in)
        opt = *opt_in;
    else
        iht_server_default_options(&opt);
    const iht_options &so = opt.solve;
    if (opt.max_slots < 1 || opt.max_slots > 1024 || so.max_iter < 0 || so.max_backtrack < 0 ||
        !(so.kappa > 1.0) || !(so.c >= 0.0 && so.c < 1.0) || !(so.tol >= 0.0) ||
        so.variant != IHT_VARIANT_IHT || ds->q > 0)
        return IHT_EINVAL;
    if (!grad_mrhs_supported(ds) || zmul_blocks(ds) > kPartials) return IHT_EINVAL;
    DeviceGuard g(ds->ctx->device);
    if (!g.ok) return IHT_ECUDA;
    iht_server *S = new (std::nothrow) iht_server();
    if (!S) return IHT_ENOMEM;
    S->ctx.device = ds->ctx->device;
    S->ctx.num_sms = ds->ctx->num_sms;
    S->opt = so;
    S->max_slots = opt.max_slots;
    S->budget = opt.hbm_budget;
    cudaError_t e = cudaStreamCreateWithFlags(&S->ctx.stream, cudaStreamNonBlocking);
    S->view = *ds;
    S->view.ctx = &S->ctx;
    S->view.ws = nullptr;
    const size_t B = (size_t)opt.max_slots;
    if (e == cudaSuccess) e = dev_malloc(&S->sc, sizeof(Scalars) * B);
    if (e == cudaSuccess) e = dev_malloc(&S->bs, sizeof(BSolve) * B);
    if (e == cudaSuccess) e = dev_malloc(&S->jobs_c, sizeof(SelJob) * B);
    if (e == cudaSuccess) e = dev_malloc(&S->jobs_s, sizeof(SelJob) * B);
    if (e == cudaSuccess) e = dev_malloc(&S->cols, sizeof(MrCol) * B);
    if (e == cudaSuccess) e = cudaMallocHost(&S->sc_host, sizeof(Scalars) * B);
    if (e == cudaSuccess) e = cudaMallocHost(&S->bs_host, sizeof(BSolve) * B);
    if (e == cudaSuccess) e = cudaMallocHost(&S->jobs_c_host, sizeof(SelJob) * B);
    if (e == cudaSuccess) e = cudaMallocHost(&S->jobs_s_host, sizeof(SelJob) * B);
    if (e == cudaSuccess) e = cudaMallocHost(&S->cols_host, sizeof(MrCol) * B);
    if (e == cudaSuccess) e = cudaMallocHost(&S->outS_host, sizeof(int32_t) * B * kMaxK);
    if (e == cudaSuccess) e = cudaMallocHost(&S->outB_host, sizeof(double) * B * kMaxK);
    if (e != cudaSuccess) {
        set_cuda_error(e, "iht_server_create");
        srv_free(S);
        return e == cudaErrorMemoryAllocation ? IHT_ENOMEM : IHT_ECUDA;
    }
    // empty slots: finished solves whose blocks return at once
    memset(S->sc_host, 0, sizeof(Scalars) * B);
    memset(S->bs_host, 0, sizeof(BSolve) * B);
    memset(S->jobs_c_host, 0, sizeof(SelJob) * B);
    for (size_t c = 0; c < B; ++c) {
        S->sc_host[c].done = 1;
        S->bs_host[c].sc = S->sc + c;
        S->jobs_c_host[c].done = &S->sc[c].done;
        S->jobs_c_host[c].K = 1;
    }
    e = cudaMemcpyAsync(S->sc, S->sc_host, sizeof(Scalars) * B, cudaMemcpyHostToDevice, S->ctx.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S->bs, S->bs_host, sizeof(BSolve) * B, cudaMemcpyHostToDevice, S->ctx.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S->jobs_c, S->jobs_c_host, sizeof(SelJob) * B, cudaMemcpyHostToDevice,
                            S->ctx.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->ctx.stream);
    if (e != cudaSuccess) {
        set_cuda_error(e, "iht_server_create");
        srv_free(S);
        return IHT_ECUDA;
    }
    int rc = ensure_selwork(&S->ctx, ds->p);
    if (rc) {
        srv_free(S);
        return rc;
    }
    S->slots.resize(B);
    try {
        S->worker = std::thread(srv_run, S);
    } catch (...) {
        srv_free(S);
        return IHT_ENOMEM;
    }
    *out = S;
    return IHT_OK;
}

int iht_server_submit(iht_server *S, const iht_solve_desc *req, uint64_t *ticket)
{
    if (!S || !req || !ticket || !req->y) return IHT_EINVAL;
    const iht_dataset *ds = &S->view;
    const int64_t nr = req->rows ? req->n_rows : ds->n;
    if (nr < 2 || nr > ds->n || req->k < 1 || req->k > ds->p || req->k > kMaxK) return IHT_EINVAL;
    SrvRequest q;
    q.all_rows = req->rows == nullptr;
    if (!q.all_rows) q.rows.assign(req->rows, req->rows + nr);
    q.y.assign(req->y, req->y + nr);
    q.k = req->k;
    q.n_rows = nr;
    q.bytes = srv_footprint(ds, req->k, nr);
    if (S->budget && q.bytes > S->budget) return IHT_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->failed) return S->failed;
    q.ticket = S->next_ticket++;
    q.t_submit = Clock::now();
    *ticket = q.ticket;
    S->live.insert(q.ticket);
    S->pending.push_back(std::move(q));
    S->st.submitted += 1;
    S->cv.notify_one();
    return IHT_OK;
}

int iht_server_poll(iht_server *S, uint64_t ticket, int32_t *support, double *beta_s,
                    iht_result *info, double *latency_s)
{
    if (!S) return IHT_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->results.find(ticket);
    if (it == S->results.end()) {
        if (S->failed) return S->failed;
        return S->live.count(ticket) ? IHT_EAGAIN : IHT_EINVAL;
    }
    const SrvResult &r = it->second;
    if (support) memcpy(support, r.S.data(), sizeof(int32_t) * r.S.size());
    if (beta_s) memcpy(beta_s, r.bS.data(), sizeof(double) * r.bS.size());
    if (info) *info = r.info;
    if (latency_s) *latency_s = r.latency;
    S->results.erase(it);
    return IHT_OK;
}

int iht_server_get_stats(iht_server *S, iht_server_stats *out)
{
    if (!S || !out) return IHT_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->st;
    return S->failed ? S->failed : IHT_OK;
}

int iht_server_destroy(iht_server *S)
{
    if (!S) return IHT_EINVAL;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    srv_free(S);
    return IHT_OK;
}

}  // extern "C"
