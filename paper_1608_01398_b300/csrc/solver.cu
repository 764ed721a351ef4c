// a3-a6: the O(nk) part of one IHT iteration, on the device.
//
//   k_gather_gS   coef = g_S, num = ||g_S||^2                     (Sec. 2.3.1)
//   k_zmul_*      out = base + sign * Z[:, cols] coef, per-block partial sums
//                 of out, out^2 and (out - prev)^2 (sparse product X_k beta_k,
//                 Sec. 2.3.2-2.3.3)
//   k_merge       mu = num / den on the first attempt; w = beta + mu g on S u C;
//                 S+ = top-k |w|, beta+ = w on S+ (Eq. ihta)
//   k_decide      backtracking test (Sec. 2.3.1): with d = beta+ - beta,
//                 Z d = r - r+, so ||Z d||^2 is the (out - prev)^2 sum of the
//                 residual pass; mu >= omega -> mu / kappa and another attempt,
//                 else accept: objective, convergence test, state copy, trace
//   k_center      r32 = r - mean(r) on the used rows (exact: every column of Z
//                 sums to zero over the used rows)
// Every kernel returns at once when the solve is done, so a fixed launch
// sequence can run past convergence without changing the result.
//
// C is the candidate list: the top min(2k, p) of |g| over all SNPs.  Off the
// support w_j = mu g_j, so the order of |w| there is the order of |g|; at most
// k candidates lie on S, hence the top-k of |w| over all p lies in S u C.
#include <math.h>

#include "bodies.cuh"

namespace iht {




__global__ void __launch_bounds__(1024) k_gather_gS(const float *__restrict__ g,
                                                    const int32_t *__restrict__ S, int k,
                                                    double *__restrict__ coef, Scalars *sc)
{
    if (sc->done) return;
    gather_gS_body(g, S, k, coef, sc);
}


__global__ void __launch_bounds__(kZmulThreads) k_zmul(const uint8_t *__restrict__ G, int64_t stride,
                                              int64_t rowb, const int32_t *__restrict__ cols, int m,
                                              const double *__restrict__ coef, double sign,
                                              const double *__restrict__ u64,
                                              const double *__restrict__ v64,
                                              const int32_t *__restrict__ used,
                                              const double *__restrict__ base,
                                              const double *__restrict__ prev,
                                              double *__restrict__ out, double *__restrict__ partials,
                                              int64_t n_pad, const int32_t *__restrict__ done,
                                              int64_t psnp, const double *__restrict__ zc)
{
    if (done && *done) return;
    zmul_body(G, stride, rowb, cols, m, coef, sign, u64, v64, used, base, prev, out, partials, n_pad,
              psnp, zc, (int)blockIdx.x);
}

static int zmul_threads(const iht_dataset *) { return kZmulThreads; }

int zmul_blocks(const iht_dataset *ds) { return ceil_div(ds->n_pad, zmul_threads(ds)); }

// out = base + sign * Z[:, cols] coef (device, stream-ordered); partials get
// zmul_blocks() triples (sum, sum of squares, sum of (out - prev)^2) when not
// null.
// cov: the columns may include covariates (indices p .. p+q-1, after the SNPs
// of an ascending list), standardised over the solve's rows (workspace zc).
int zmul_run(iht_dataset *ds, const int32_t *cols, int m, const double *coef, double sign,
             const double *u, const double *v, const int32_t *used, const double *base,
             double *out, double *partials, const int32_t *done, const double *prev = nullptr,
             bool cov = true)
{
    const double *zc = cov && ds->q > 0 ? ds->ws->zc : nullptr;
    k_zmul<<<zmul_blocks(ds), zmul_threads(ds), 0, ds->ctx->stream>>>(ds->G, ds->stride, ds->rowb, cols, m, coef,
                                                         sign, u, v, used, base, prev, out, partials,
                                                         ds->n_pad, done, ds->p, zc);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

int launch_zmul(iht_dataset *ds, const int32_t *cols, int32_t m, const double *coef,
                const double *u, const double *v, const int32_t *used, const double *base,
                double *out, double *partials)
{
    return zmul_run(ds, cols, m, coef, 1.0, u, v, used, base, out, partials, nullptr, nullptr, false);
}

// ---------------------------------------------------------------------------
// Projection for one step size: one block of 1024 threads.


__global__ void __launch_bounds__(kMergeThreads) k_merge(MergeArgs A)
{
    const int d = A.sc->done || (A.skip && *A.skip);
    __syncthreads();   // every thread has read the flag before thread 0 may set it
    if (d) return;
    merge_body(A);
}

// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_decide(Scalars *sc, const double *partials, int npart,
                                                int32_t *S, double *bS, const int32_t *Sp,
                                                const double *bSp, TraceDev tr, const int32_t *skip)
{
    if (sc->done || (skip && *skip)) return;
    decide_body(sc, partials, npart, S, bS, Sp, bSp, tr);
}

// HTP: after the refit beta+ on S+ (bSp) and its residual (partials: sum r+,
// sum r+^2): objective, the stopping test against beta on S, state copy, trace.
// One block; thread 0 walks S and S+ (both ascending) in order.
__global__ void __launch_bounds__(256) k_htp_finish(Scalars *sc, const double *partials, int npart,
                                                    int32_t *S, double *bS, const int32_t *Sp,
                                                    const double *bSp, TraceDev tr)
{
    if (sc->done) return;
    const int k = sc->k;
    double s = 0.0, s2 = 0.0, d2 = 0.0;
    if (threadIdx.x < 32) warp_partials(partials, npart, s, s2, d2);
    if (threadIdx.x == 0) {
        double dd = 0.0, bb = 0.0;
        int a = 0, b = 0;
        while (a < k || b < k) {
            const int32_t ja = a < k ? S[a] : 0x7fffffff, jb = b < k ? Sp[b] : 0x7fffffff;
            double d;
            if (ja == jb) {
                d = bSp[b] - bS[a];
                bb += bS[a] * bS[a];
                ++a;
                ++b;
            } else if (ja < jb) {
                d = -bS[a];
                bb += bS[a] * bS[a];
                ++a;
            } else {
                d = bSp[b];
                ++b;
            }
            dd += d * d;
        }
        sc->sum_r = s;
        sc->sumsq_r = s2;
        sc->f = 0.5 * s2;
        sc->dd = dd;
        sc->bb = bb;
        sc->step = sqrt(dd) / (sqrt(bb) + 1.0);
        if (tr.objective) tr.objective[sc->iter] = sc->f;
    }
    __syncthreads();
    const int it = sc->iter;
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        S[c] = Sp[c];
        bS[c] = bSp[c];
        if (tr.supp) tr.supp[(size_t)it * k + c] = Sp[c];
        if (tr.beta) tr.beta[(size_t)it * k + c] = bSp[c];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        sc->iter = it + 1;
        if (sc->step < sc->tol) {
            sc->status = IHT_OK;
            sc->done = 1;
        } else if (sc->iter >= sc->max_iter) {
            sc->status = IHT_ENOTCONV;
            sc->done = 1;
        }
    }
}


__global__ void k_init_objective(Scalars *sc, const double *partials, int npart)
{
    if (sc->done) return;
    init_objective_body(sc, partials, npart);
}

// The start of a solve captured in a graph (one warp): the solve's scalars
// from init, keeping the flags the set-up kernels raised (bit 0: non-finite
// input, bit 1: bad rows), which stop the solve at once with ENUMERIC /
// EINVAL; then the objective of beta = 0 as k_init_objective forms it.
__global__ void k_init_solve(Scalars *sc, const Scalars *init, const double *partials, int npart)
{
    constexpr int kWords = (int)(sizeof(Scalars) / sizeof(unsigned long long));
    const int lane = threadIdx.x & 31;
    int32_t err = lane == 0 ? sc->err : 0;
    err = __shfl_sync(0xffffffffu, err, 0);
    for (int w = lane; w < kWords; w += 32)
        reinterpret_cast<unsigned long long *>(sc)[w] = reinterpret_cast<const unsigned long long *>(init)[w];
    __syncwarp();
    if (lane == 0) {
        sc->err = err;
        if (err) {
            sc->status = (err & 1) ? IHT_ENUMERIC : IHT_EINVAL;
            sc->done = 1;
            sc->skip1 = sc->skip2 = 1;
        }
    }
    __syncwarp();
    if (sc->done) return;
    init_objective_body(sc, partials, npart);
}



__global__ void k_center(const double *__restrict__ src, double *__restrict__ r64,
                         const int32_t *__restrict__ used, int64_t n_pad, const Scalars *sc,
                         float *__restrict__ r32)
{
    if (sc->done || sc->retry) return;
    center_body(src, r64, used, n_pad, sc, r32);
}

__global__ void k_check_finite(const double *__restrict__ y, int64_t n, Scalars *sc)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !isfinite(y[i])) atomicOr(&sc->err, 1);
}

// ---------------------------------------------------------------------------
// Host orchestration of one solve.

static void configure_merge(iht_dataset *ds)
{
    static thread_local int configured_dev = -1;
    if (configured_dev != ds->ctx->device) {
        cudaFuncSetAttribute(k_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MergeShared));
        configured_dev = ds->ctx->device;
    }
}

int launch_merge(iht_dataset *ds, int K, int first, const int32_t *skip = nullptr)
{
    static thread_local int configured_dev = -1;
    const int smem = (int)sizeof(MergeShared);
    if (configured_dev != ds->ctx->device) {
        IHT_CUDA(cudaFuncSetAttribute(k_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        configured_dev = ds->ctx->device;
    }
    Workspace *ws = ds->ws;
    MergeArgs A;
    A.g = ws->g;
    A.S = ws->S;
    A.bS = ws->bS;
    A.cand = ws->cand;
    A.K = K;
    A.partials = ws->partials;
    A.npart = zmul_blocks(ds);
    A.first = first;
    A.skip = skip;
    A.Sp = ws->Sp;
    A.bSp = ws->bSp;
    A.sc = ws->sc;
    k_merge<<<1, kMergeThreads, smem, ds->ctx->stream>>>(A);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

// The gradient pass; e0/e1 (optional) are recorded around its main kernel.
static int launch_grad_ev(iht_dataset *ds, int impl, const int32_t *done, cudaEvent_t e0, cudaEvent_t e1,
                          uint32_t *hist = nullptr, uint32_t *hflag = nullptr)
{
    Workspace *ws = ds->ws;
    cudaStream_t s = ds->ctx->stream;
    const bool tc = impl == 2 || (impl == 0 && grad_tc_supported(ds));
    int rc;
    if (tc && (rc = prepare_grad_tc(ds, ws->r32, done))) return rc;
    // inside a stream capture the records must be external to become event nodes of the graph
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (e0 || e1) IHT_CUDA(cudaStreamIsCapturing(s, &cap));
    const unsigned flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (e0) IHT_CUDA(cudaEventRecordWithFlags(e0, s, flags));
    if (hist && !tc) return IHT_EINVAL;                      // (only the tensor-core pass counts keys)
    rc = tc ? launch_grad_tc_main(ds, ws->r32, ws->g, done, hist, hflag)
            : launch_grad_simt(ds, ws->r32, ws->g, done);
    if (rc) return rc;
    if (e1) IHT_CUDA(cudaEventRecordWithFlags(e1, s, flags));
    return launch_cov_grad(ds, ws->r32, ws->g, done, hist, hflag);   // covariate entries p .. p+q-1
}

int launch_grad(iht_dataset *ds, int impl, const int32_t *done, bool profile, uint32_t *hist = nullptr,
                uint32_t *hflag = nullptr)
{
    Workspace *ws = ds->ws;
    const bool rec = profile && ws->nprof < kProfEvents;
    const int rc = launch_grad_ev(ds, impl, done, rec ? ws->prof_ev[2 * ws->nprof] : nullptr,
                                  rec ? ws->prof_ev[2 * ws->nprof + 1] : nullptr, hist, hflag);
    if (rc) return rc;
    if (rec) ++ws->nprof;
    return IHT_OK;
}

// One backtracking attempt: projection, candidate residual, decision, centring.
// skip (not null): every kernel returns at once when *skip (an attempt
// enqueued before it was known to be needed).
static int enqueue_attempt(iht_dataset *ds, int k, int K, int first, const int32_t *skip,
                           const TraceDev &tr)
{
    Workspace *ws = ds->ws;
    cudaStream_t s = ds->ctx->stream;
    int rc;
    if ((rc = launch_merge(ds, K, first, skip))) return rc;
    if ((rc = zmul_run(ds, ws->Sp, k, ws->bSp, -1.0, ws->u64, ws->v64, ws->used, ws->y64, ws->rc64,
                       ws->partials, skip ? skip : &ws->sc->done, ws->r64)))
        return rc;
    k_decide<<<1, 256, 0, s>>>(ws->sc, ws->partials, zmul_blocks(ds), ws->S, ws->bS, ws->Sp, ws->bSp, tr,
                               skip);
    k_center<<<ceil_div(ds->n_pad, 256), 256, 0, s>>>(ws->rc64, ws->r64, ws->used, ds->n_pad, ws->sc,
                                                      ws->r32);
    note_launch(2);
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

// One iteration from the current gradient: candidates, step size, two
// attempts (the second returns at once unless the first was rejected), and the
// next gradient (returns at once if the solve stopped or the second attempt
// was rejected too).
static int enqueue_iteration(iht_dataset *ds, int k, int K, int impl, cudaEvent_t e0, cudaEvent_t e1)
{
    Workspace *ws = ds->ws;
    cudaStream_t s = ds->ctx->stream;
    const int32_t *done = &ws->sc->done;
    int rc;
    // candidates, and g_S with ||g_S||^2 in the same launch's last block
    if ((rc = select_topk(ds->ctx, ws->g, ds->p + ds->q, K, ws->cand, done, ws->S, k, ws->coef, ws->sc)))
        return rc;
    if ((rc = zmul_run(ds, ws->S, k, ws->coef, 1.0, ws->u64, ws->v64, ws->used, nullptr, ws->zv,
                       ws->partials, done)))
        return rc;
    if ((rc = enqueue_attempt(ds, k, K, 1, nullptr, TraceDev{}))) return rc;
    if ((rc = enqueue_attempt(ds, k, K, 0, &ws->sc->skip1, TraceDev{}))) return rc;
    return launch_grad_ev(ds, impl, &ws->sc->skip2, e0, e1);
}

// The iteration as a CUDA graph (captured on a private stream: the caller's
// stream may be the legacy default stream), cached in the workspace while the
// key (sizes, gradient kernel, profiling, and every scratch address the
// kernels were captured with) is unchanged.
static int iteration_graph(iht_dataset *ds, int k, int K, int impl, bool prof, cudaGraphExec_t *exec)
{
    Workspace *ws = ds->ws;
    const uint64_t key[8] = {(uint64_t)k | ((uint64_t)ds->q << 32), (uint64_t)K, (uint64_t)impl,
                             (uint64_t)prof, (uint64_t)(uintptr_t)ws->S, (uint64_t)(uintptr_t)ws->cand,
                             grad_tc_scratch_id(), (uint64_t)(uintptr_t)ds->ctx->sel.cand};
    if (ws->iter_exec && std::equal(key, key + 8, ws->iter_key)) {
        *exec = ws->iter_exec;
        return IHT_OK;
    }
    if (ws->iter_exec) {
        cudaGraphExecDestroy(ws->iter_exec);
        ws->iter_exec = nullptr;
    }
    if (!ws->cap_stream) IHT_CUDA(cudaStreamCreateWithFlags(&ws->cap_stream, cudaStreamNonBlocking));
    if (prof && !ws->gev[0])
        for (cudaEvent_t &e : ws->gev) IHT_CUDA(cudaEventCreate(&e));
    configure_merge(ds);
    cudaStream_t user = ds->ctx->stream;
    ds->ctx->stream = ws->cap_stream;
    const uint64_t before = launches_noted();
    cudaError_t e = cudaStreamBeginCapture(ws->cap_stream, cudaStreamCaptureModeThreadLocal);
    int rc = IHT_OK;
    if (e == cudaSuccess)
        rc = enqueue_iteration(ds, k, K, impl, prof ? ws->gev[0] : nullptr, prof ? ws->gev[1] : nullptr);
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(ws->cap_stream, &graph) : e;
    ds->ctx->stream = user;
    const int n = (int)(launches_noted() - before);
    note_launch(-n);                                   // captured, not run
    if (rc == IHT_OK && e2 != cudaSuccess) {
        set_cuda_error(e2, "iteration capture");
        rc = IHT_ECUDA;
    }
    if (rc == IHT_OK) {
        e = cudaGraphInstantiate(&ws->iter_exec, graph, 0);
        if (e != cudaSuccess) {
            set_cuda_error(e, "iteration graph instantiate");
            ws->iter_exec = nullptr;
            rc = IHT_ECUDA;
        }
    }
    if (graph) cudaGraphDestroy(graph);
    if (rc) return rc;
    std::copy(key, key + 8, ws->iter_key);
    ws->iter_launches = n;
    *exec = ws->iter_exec;
    return IHT_OK;
}

// y64 and the row set are in place; runs the solve, leaves S/bS and scalars.
// A solve's first steps from beta = 0 (r = y, objective, centred residual, g^0,
// S^0 = top-k |g^0|, beta_S = 0), enqueued on the context's stream (the fused
// solve captures them ahead of its loop); the scalars come from ws->sc_init.
int enqueue_solve_setup(iht_dataset *ds, int k, int impl, uint32_t *hist, uint32_t *hflag)
{
    Workspace *ws = ds->ws;
    cudaStream_t s = ds->ctx->stream;
    const int npart = zmul_blocks(ds);
    const int64_t P = ds->p + ds->q;
    int rc;
    if ((rc = zmul_run(ds, ws->cols, 0, ws->coef, -1.0, ws->u64, ws->v64, ws->used, ws->y64, ws->r64,
                       ws->partials, nullptr)))
        return rc;
    k_init_solve<<<1, 32, 0, s>>>(ws->sc, ws->sc_init, ws->partials, npart);
    k_center<<<ceil_div(ds->n_pad, 256), 256, 0, s>>>(ws->r64, ws->r64, ws->used, ds->n_pad, ws->sc,
                                                      ws->r32);
    note_launch(2);
    IHT_CUDA(cudaGetLastError());
    const int32_t *done = &ws->sc->done;
    if ((rc = launch_grad(ds, impl, done, false, hist, hflag))) return rc;
    if ((rc = select_topk(ds->ctx, ws->g, P, k, ws->S, done))) return rc;
    IHT_CUDA(cudaMemsetAsync(ws->bS, 0, sizeof(double) * k, s));
    return IHT_OK;
}

int run_solve(iht_dataset *ds, int k, const iht_options *opt, int n_rows, const TraceDev &tr,
              const SolveInit *init)
{
    Workspace *ws = ds->ws;
    cudaStream_t s = ds->ctx->stream;
    const int npart = zmul_blocks(ds);
    const int64_t P = ds->p + ds->q;                  // SNPs, then covariates
    const int K = (int)std::min<int64_t>(2 * (int64_t)k, P);
    const bool htp = opt->variant == IHT_VARIANT_HTP;
    int rc;

    Scalars h{};
    h.htp = htp ? 1 : 0;
    h.c = opt->c;
    h.kappa = opt->kappa;
    h.tol = opt->tol;
    h.max_iter = opt->max_iter;
    h.max_backtrack = opt->max_backtrack;
    h.k = k;
    h.n_rows = n_rows;
    h.status = IHT_ENOTCONV;
    h.iter = init ? init->iter : 0;
    h.bt_total = init ? init->backtracks : 0;
    h.done = opt->max_iter <= h.iter ? 1 : 0;
    const bool traced = tr.objective || tr.mu || tr.backtracks || tr.changed || tr.supp || tr.beta;
    if (!init && !traced && !htp && !opt->profile && fused_supported(ds, k, opt->grad_impl)) {
        // the whole solve as one graph launch and one host synchronisation;
        // the set-up kernels' flags are read with the final scalars
        ws->nprof = 0;
        ws->prof_ms = 0.0;
        rc = run_whole_fused_solve(ds, k, K, opt->grad_impl, h);
        if (rc != IHT_EAGAIN) {
            if (rc) return rc;
            const int32_t err = ws->sc_host->err;
            if (err) return (err & 1) ? IHT_ENUMERIC : IHT_EINVAL;
            ws->graph_replays = ws->sc_host->iter;
            return IHT_OK;
        }
    }
    IHT_CUDA(cudaMemcpyAsync(ws->sc_host, ws->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
    IHT_CUDA(cudaStreamSynchronize(s));
    h.err = ws->sc_host->err;        // row / input flags from the set-up kernels
    if (h.err) return (h.err & 1) ? IHT_ENUMERIC : IHT_EINVAL;
    if ((rc = grad_tc_reset_status(ds))) return rc;
    *ws->sc_host = h;
    IHT_CUDA(cudaMemcpyAsync(ws->sc, ws->sc_host, sizeof(Scalars), cudaMemcpyHostToDevice, s));

    // beta = 0: r = y, objective, centred residual, g^0, S^0 = top-k |g^0|.  A
    // resumed solve starts from its S and beta_S instead: r = y - Z_S beta_S by the
    // same product the accepted step of the interrupted solve used.
    if (init) {
        IHT_CUDA(cudaMemcpyAsync(ws->S, init->S, sizeof(int32_t) * k, cudaMemcpyHostToDevice, s));
        IHT_CUDA(cudaMemcpyAsync(ws->bS, init->bS, sizeof(double) * k, cudaMemcpyHostToDevice, s));
    }
    if ((rc = init ? zmul_run(ds, ws->S, k, ws->bS, -1.0, ws->u64, ws->v64, ws->used, ws->y64,
                              ws->r64, ws->partials, nullptr)
                   : zmul_run(ds, ws->cols, 0, ws->coef, -1.0, ws->u64, ws->v64, ws->used, ws->y64,
                              ws->r64, ws->partials, nullptr)))
        return rc;
    k_init_objective<<<1, 32, 0, s>>>(ws->sc, ws->partials, npart);
    k_center<<<ceil_div(ds->n_pad, 256), 256, 0, s>>>(ws->r64, ws->r64, ws->used, ds->n_pad, ws->sc,
                                                      ws->r32);
    note_launch(2);
    IHT_CUDA(cudaGetLastError());
    const int32_t *done = &ws->sc->done;
    const bool prof = opt->profile != 0;
    ws->nprof = 0;
    if (prof && !ws->prof_ev[0]) {
        for (int e = 0; e < 2 * kProfEvents; ++e) IHT_CUDA(cudaEventCreate(&ws->prof_ev[e]));
    }
    if ((rc = launch_grad(ds, opt->grad_impl, done, prof))) return rc;
    if (!init) {
        if ((rc = select_topk(ds->ctx, ws->g, P, k, ws->S, done))) return rc;
        IHT_CUDA(cudaMemsetAsync(ws->bS, 0, sizeof(double) * k, s));
    }

    ws->graph_replays = 0;
    double graph_ms = 0.0;
    int graph_n = 0;
    if (htp) {
        // HTP (Sec. 2.2), one host synchronisation per attempt: step over Gamma =
        // the k largest |g| with g_Gamma and ||g_Gamma||^2 from the selection's last
        // block, candidates, attempts on the projected candidate, then the
        // least-squares refit on S+, its residual, the stopping test and centring.
        if ((rc = ensure_htp_scratch(ds, k))) return rc;
        for (int it = 0; it < opt->max_iter; ++it) {
            if (it > 0 && (rc = launch_grad(ds, opt->grad_impl, done, prof))) return rc;
            if ((rc = select_topk(ds->ctx, ws->g, P, k, ws->gam, done, ws->gam, k, ws->coef, ws->sc)))
                return rc;
            if ((rc = zmul_run(ds, ws->gam, k, ws->coef, 1.0, ws->u64, ws->v64, ws->used, nullptr,
                               ws->zv, ws->partials, done)))
                return rc;
            if ((rc = select_topk(ds->ctx, ws->g, P, K, ws->cand, done))) return rc;
            for (int attempt = 0;; ++attempt) {
                if ((rc = enqueue_attempt(ds, k, K, attempt == 0, nullptr, tr))) return rc;
                IHT_CUDA(cudaMemcpyAsync(&ws->sc_host->done, &ws->sc->done, 2 * sizeof(int32_t),
                                         cudaMemcpyDeviceToHost, s));
                IHT_CUDA(cudaStreamSynchronize(s));
                if (ws->sc_host->done || !ws->sc_host->retry) break;
            }
            if (ws->sc_host->done) break;
            if ((rc = htp_refit(ds, k, ws->Sp, ws->bSp, done))) return rc;
            if ((rc = zmul_run(ds, ws->Sp, k, ws->bSp, -1.0, ws->u64, ws->v64, ws->used, ws->y64,
                               ws->rc64, ws->partials, done)))
                return rc;
            k_htp_finish<<<1, 256, 0, s>>>(ws->sc, ws->partials, npart, ws->S, ws->bS, ws->Sp, ws->bSp, tr);
            k_center<<<ceil_div(ds->n_pad, 256), 256, 0, s>>>(ws->rc64, ws->r64, ws->used, ds->n_pad,
                                                              ws->sc, ws->r32);
            note_launch(2);
            IHT_CUDA(cudaGetLastError());
            IHT_CUDA(cudaMemcpyAsync(&ws->sc_host->done, &ws->sc->done, sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, s));
            IHT_CUDA(cudaStreamSynchronize(s));
            if (ws->sc_host->done) break;
        }
    }
    bool fused = false;
    if (!traced && !htp && !prof && fused_supported(ds, k, opt->grad_impl)) {
        // the rest of the solve as one graph launch: one host synchronisation
        const int it0 = ws->sc_host->iter;
        rc = run_fused_solve(ds, k, K, opt->grad_impl);
        if (rc != IHT_EAGAIN) {
            if (rc) return rc;
            fused = true;
            IHT_CUDA(cudaMemcpyAsync(&ws->sc_host->iter, &ws->sc->iter, sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, s));
            IHT_CUDA(cudaStreamSynchronize(s));
            ws->graph_replays = ws->sc_host->iter - it0;
            note_launch(ws->fused_launches * std::max(ws->graph_replays, 1));
        }
    }
    if (!traced && !htp && !fused) {
        // one graph replay and one host synchronisation per iteration
        cudaGraphExec_t exec = nullptr;
        if ((rc = iteration_graph(ds, k, K, opt->grad_impl, prof, &exec))) return rc;
        for (int it = 0; it < opt->max_iter; ++it) {
            IHT_CUDA(cudaGraphLaunch(exec, s));
            note_launch(ws->iter_launches);
            ++ws->graph_replays;
            IHT_CUDA(cudaMemcpyAsync(&ws->sc_host->done, &ws->sc->done, 2 * sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, s));
            IHT_CUDA(cudaStreamSynchronize(s));
            int32_t dn = ws->sc_host->done, rt = ws->sc_host->retry;
            if (!dn && rt) {
                // rejected twice: further attempts one at a time, then the next gradient
                while (!dn && rt) {
                    if ((rc = enqueue_attempt(ds, k, K, 0, nullptr, tr))) return rc;
                    IHT_CUDA(cudaMemcpyAsync(&ws->sc_host->done, &ws->sc->done, 2 * sizeof(int32_t),
                                             cudaMemcpyDeviceToHost, s));
                    IHT_CUDA(cudaStreamSynchronize(s));
                    dn = ws->sc_host->done;
                    rt = ws->sc_host->retry;
                }
                if (!dn && (rc = launch_grad(ds, opt->grad_impl, done, prof))) return rc;
            } else if (prof && !dn) {
                float ms = 0.0f;                       // the graph's gradient pass ran
                IHT_CUDA(cudaEventElapsedTime(&ms, ws->gev[0], ws->gev[1]));
                graph_ms += ms;
                ++graph_n;
            }
            if (dn) break;
        }
    }
    for (int it = 0; traced && !htp && it < opt->max_iter; ++it) {
        if (it > 0 && (rc = launch_grad(ds, opt->grad_impl, done, prof))) return rc;
        if ((rc = select_topk(ds->ctx, ws->g, P, K, ws->cand, done))) return rc;
        k_gather_gS<<<1, 1024, 0, s>>>(ws->g, ws->S, k, ws->coef, ws->sc);
        note_launch();
        if ((rc = zmul_run(ds, ws->S, k, ws->coef, 1.0, ws->u64, ws->v64, ws->used, nullptr, ws->zv,
                           ws->partials, done)))
            return rc;
        for (int attempt = 0;; ++attempt) {
            if ((rc = enqueue_attempt(ds, k, K, attempt == 0, nullptr, tr))) return rc;
            IHT_CUDA(cudaMemcpyAsync(&ws->sc_host->done, &ws->sc->done, 2 * sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, s));
            IHT_CUDA(cudaStreamSynchronize(s));
            if (ws->sc_host->done || !ws->sc_host->retry) break;
        }
        if (ws->sc_host->done) break;
    }
    IHT_CUDA(cudaMemcpyAsync(ws->sc_host, ws->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
    int timed_out = 0;
    if ((rc = grad_tc_status(ds, &timed_out))) return rc;     // synchronises the stream
    if (timed_out) return IHT_ETIMEOUT;                        // a pass gave up: g was not formed
    ws->prof_ms = graph_ms;
    for (int e = 0; prof && e < ws->nprof; ++e) {
        float ms = 0.0f;
        IHT_CUDA(cudaEventElapsedTime(&ms, ws->prof_ev[2 * e], ws->prof_ev[2 * e + 1]));
        ws->prof_ms += ms;
    }
    ws->nprof += graph_n;
    return IHT_OK;
}

int run_solve_host(iht_dataset *ds, int k, const iht_options *opt, int n_rows, iht_trace *trace,
                   int max_iter, const SolveInit *init)
{
    TraceDev tr{};
    void *buf = nullptr;
    const size_t T = (size_t)std::max(max_iter, 1);
    if (trace) {
        const size_t bytes = T * (2 * sizeof(double) + 2 * sizeof(int32_t)) +
                             T * k * (sizeof(int32_t) + sizeof(double));
        IHT_CUDA(dev_malloc(&buf, bytes));
        char *p = (char *)buf;
        tr.objective = (double *)p; p += T * sizeof(double);
        tr.mu = (double *)p; p += T * sizeof(double);
        tr.beta = (double *)p; p += T * k * sizeof(double);
        tr.backtracks = (int32_t *)p; p += T * sizeof(int32_t);
        tr.changed = (int32_t *)p; p += T * sizeof(int32_t);
        tr.supp = (int32_t *)p;
    }
    int rc = run_solve(ds, k, opt, n_rows, tr, init);
    if (rc == IHT_OK && trace) {
        cudaStream_t s = ds->ctx->stream;
        const int it = ds->ws->sc_host->iter;
        auto get = [&](void *dst, const void *src, size_t bytes) -> int {
            if (dst && bytes) IHT_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
            return IHT_OK;
        };
        if ((rc = get(trace->objective, tr.objective, it * sizeof(double))) ||
            (rc = get(trace->mu, tr.mu, it * sizeof(double))) ||
            (rc = get(trace->backtracks, tr.backtracks, it * sizeof(int32_t))) ||
            (rc = get(trace->changed, tr.changed, it * sizeof(int32_t))) ||
            (rc = get(trace->supp, tr.supp, (size_t)it * k * sizeof(int32_t))) ||
            (rc = get(trace->beta, tr.beta, (size_t)it * k * sizeof(double)))) {
        }
        if (rc == IHT_OK) IHT_CUDA(cudaStreamSynchronize(s));
    }
    if (buf) cudaFree(buf);
    return rc;
}

int check_finite_y_sc(iht_dataset *ds, int64_t n_rows, const double *y_dev, Scalars *sc)
{
    if (n_rows > 0) {
        k_check_finite<<<ceil_div(n_rows, 256), 256, 0, ds->ctx->stream>>>(y_dev, n_rows, sc);
        note_launch();
    }
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

int check_finite_y(iht_dataset *ds, int64_t n_rows, const double *y_dev)
{
    return check_finite_y_sc(ds, n_rows, y_dev, ds->ws->sc);
}

}  // namespace iht

namespace iht {

__global__ void k_gather_rows(const int32_t *__restrict__ rows, int64_t n_rows,
                              const double *__restrict__ src, double *__restrict__ dst)
{
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a < n_rows) dst[a] = src[rows ? rows[a] : a];
}

int gather_rows_f64(iht_dataset *ds, const int32_t *rows_dev, int64_t n_rows, const double *src,
                    double *dst)
{
    if (n_rows > 0) {
        k_gather_rows<<<ceil_div(n_rows, 256), 256, 0, ds->ctx->stream>>>(rows_dev, n_rows, src, dst);
        note_launch();
    }
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

__global__ void k_scatter_beta(const int32_t *__restrict__ S, const double *__restrict__ bS, int k,
                               double *__restrict__ beta)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < k) beta[S[c]] = bS[c];
}

// beta_out (device, p doubles): zeros off the support, beta_S on it.
int write_beta_device(iht_dataset *ds, int k, double *beta_out)
{
    cudaStream_t s = ds->ctx->stream;
    IHT_CUDA(cudaMemsetAsync(beta_out, 0, sizeof(double) * (ds->p + ds->q), s));
    k_scatter_beta<<<ceil_div(k, 256), 256, 0, s>>>(ds->ws->S, ds->ws->bS, k, beta_out);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

}  // namespace iht

// ---------------------------------------------------------------------------
// Batched tails: the same bodies, one solve per block row (blockIdx.y, or
// blockIdx.x for single-block steps).  A solve takes part in an attempt when
// it is not done and either the attempt is its first of the iteration or its
// last candidate was rejected; k_merge_b records that in sc->live and the
// later kernels of the attempt read it.

namespace iht {

__global__ void __launch_bounds__(1024) k_gather_gS_b(const BSolve *bs)
{
    const BSolve &B = bs[blockIdx.x];
    if (B.sc->done) return;
    gather_gS_body(B.g, B.S, B.k, B.coef, B.sc);
}

__device__ __forceinline__ bool zmul_gate(const BSolve &B, int which)
{
    const Scalars *sc = B.sc;
    if (which == kZmulInit) return sc->fresh && !sc->done;
    if (which == kZmulStep) return !sc->done;
    return sc->live && !sc->done;
}

__global__ void __launch_bounds__(kZmulThreads) k_zmul_b(const uint8_t *__restrict__ G, int64_t stride,
                                                int64_t rowb, const BSolve *bs, int which,
                                                int64_t n_pad)
{
    const BSolve &B = bs[blockIdx.y];
    if (!zmul_gate(B, which)) return;
    if (which == kZmulInit)
        zmul_body(G, stride, rowb, nullptr, 0, nullptr, -1.0, B.u64, B.v64, B.used, B.y64, nullptr,
                  B.r64, B.partials, n_pad, 0, nullptr, (int)blockIdx.x);
    else if (which == kZmulStep)
        zmul_body(G, stride, rowb, B.S, B.k, B.coef, 1.0, B.u64, B.v64, B.used, nullptr, nullptr,
                  B.zv, B.partials, n_pad, 0, nullptr, (int)blockIdx.x);
    else
        zmul_body(G, stride, rowb, B.Sp, B.k, B.bSp, -1.0, B.u64, B.v64, B.used, B.y64, B.r64,
                  B.rc64, B.partials, n_pad, 0, nullptr, (int)blockIdx.x);
}

__global__ void k_init_objective_b(const BSolve *bs, int npart)
{
    const BSolve &B = bs[blockIdx.x];
    if (!B.sc->fresh || B.sc->done) return;
    init_objective_body(B.sc, B.partials, npart);
}

__global__ void k_center_b(const BSolve *bs, int64_t n_pad, int init)
{
    const BSolve &B = bs[blockIdx.y];
    const Scalars *sc = B.sc;
    if (init) {
        if (!sc->fresh || sc->done) return;
        center_body(B.r64, B.r64, B.used, n_pad, sc, B.r32);
    } else {
        if (!sc->live || sc->done || sc->retry) return;
        center_body(B.rc64, B.r64, B.used, n_pad, sc, B.r32);
    }
}

__global__ void __launch_bounds__(kMergeThreads) k_merge_b(const BSolve *bs, int first, int npart)
{
    const BSolve &B = bs[blockIdx.x];
    Scalars *sc = B.sc;
    const int live = !sc->done && (first || sc->retry);
    __syncthreads();   // flags read by every thread before thread 0 writes any
    if (threadIdx.x == 0) sc->live = live;
    if (!live) return;
    MergeArgs A;
    A.g = B.g;
    A.S = B.S;
    A.bS = B.bS;
    A.cand = B.cand;
    A.K = B.K;
    A.partials = B.partials;
    A.npart = npart;
    A.first = first;
    A.skip = nullptr;
    A.Sp = B.Sp;
    A.bSp = B.bSp;
    A.sc = sc;
    merge_body(A);
}

__global__ void __launch_bounds__(256) k_decide_b(const BSolve *bs, int npart)
{
    const BSolve &B = bs[blockIdx.x];
    Scalars *sc = B.sc;
    if (!sc->live || sc->done) return;
    decide_body(sc, B.partials, npart, B.S, B.bS, B.Sp, B.bSp, TraceDev{});
}

// Cross-validation (Sec. 2.4): the residual y - Z_S beta_S of each fitted
// solve over its partition's rows, standardised with its training rows'
// statistics (the sparse product above, one job per block row).
__global__ void __launch_bounds__(kZmulThreads) k_cv_resid(const uint8_t *__restrict__ G, int64_t stride,
                                                  int64_t rowb, const CvJob *jobs, int64_t n_pad)
{
    const CvJob &J = jobs[blockIdx.y];
    zmul_body(G, stride, rowb, J.S, J.k, J.bS, -1.0, J.u64, J.v64, J.used, J.y64, nullptr, J.out, J.partials,
              n_pad, 0, nullptr, (int)blockIdx.x);
}

int launch_cv_resid(iht_dataset *ds, const CvJob *jobs_dev, int njobs)
{
    if (njobs <= 0) return IHT_OK;
    k_cv_resid<<<dim3(zmul_blocks(ds), njobs), zmul_threads(ds), 0, ds->ctx->stream>>>(ds->G, ds->stride, ds->rowb,
                                                                                    jobs_dev, ds->n_pad);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

__global__ void k_scatter_beta_b(const BSolve *bs, int64_t p, double *__restrict__ betas)
{
    const BSolve &B = bs[blockIdx.y];
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= B.k) return;
    const int32_t j = B.S[c];
    if (j >= 0 && j < p) betas[(int64_t)blockIdx.y * p + j] = B.bS[c];
}

__global__ void k_compact_support_b(const BSolve *bs, int32_t *__restrict__ supports,
                                    double *__restrict__ beta_s)
{
    const BSolve &B = bs[blockIdx.y];
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= B.k) return;
    if (supports) supports[B.out_off + c] = B.S[c];
    if (beta_s) beta_s[B.out_off + c] = B.bS[c];
}

// After S^0 of newly set-up solves: beta_S = 0, set-up flag cleared.
__global__ void k_finish_fresh_b(const BSolve *bs)
{
    const BSolve &B = bs[blockIdx.x];
    Scalars *sc = B.sc;
    const int fresh = sc->fresh, done = sc->done;
    __syncthreads();   // flags read by every thread before thread 0 clears one
    if (!fresh) return;
    for (int c = threadIdx.x; c < B.k && !done; c += blockDim.x) B.bS[c] = 0.0;
    if (threadIdx.x == 0) sc->fresh = 0;
}

int launch_finish_fresh_batch(iht_dataset *ds, const BSolve *bs, int nb, int)
{
    k_finish_fresh_b<<<nb, 256, 0, ds->ctx->stream>>>(bs);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

int launch_compact_support_batch(iht_dataset *ds, const BSolve *bs, int nb, int kmax,
                                 int32_t *supports, double *beta_s)
{
    k_compact_support_b<<<dim3(ceil_div(kmax, 256), nb), 256, 0, ds->ctx->stream>>>(bs, supports,
                                                                                  beta_s);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

int launch_gather_gS_batch(iht_dataset *ds, const BSolve *bs, int nb)
{
    k_gather_gS_b<<<nb, 1024, 0, ds->ctx->stream>>>(bs);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

int launch_zmul_batch(iht_dataset *ds, const BSolve *bs, int nb, int, ZmulWhich which)
{
    k_zmul_b<<<dim3(zmul_blocks(ds), nb), zmul_threads(ds), 0, ds->ctx->stream>>>(ds->G, ds->stride, ds->rowb, bs,
                                                                   (int)which, ds->n_pad);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

int launch_init_objective_batch(iht_dataset *ds, const BSolve *bs, int nb)
{
    k_init_objective_b<<<nb, 32, 0, ds->ctx->stream>>>(bs, zmul_blocks(ds));
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

int launch_center_batch(iht_dataset *ds, const BSolve *bs, int nb, bool init)
{
    k_center_b<<<dim3(ceil_div(ds->n_pad, 256), nb), 256, 0, ds->ctx->stream>>>(bs, ds->n_pad,
                                                                              init ? 1 : 0);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

int launch_merge_batch(iht_dataset *ds, const BSolve *bs, int nb, int first)
{
    static thread_local int configured_dev = -1;
    const int smem = (int)sizeof(MergeShared);
    if (configured_dev != ds->ctx->device) {
        IHT_CUDA(cudaFuncSetAttribute(k_merge_b, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        configured_dev = ds->ctx->device;
    }
    k_merge_b<<<nb, kMergeThreads, smem, ds->ctx->stream>>>(bs, first, zmul_blocks(ds));
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

int launch_decide_batch(iht_dataset *ds, const BSolve *bs, int nb)
{
    k_decide_b<<<nb, 256, 0, ds->ctx->stream>>>(bs, zmul_blocks(ds));
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

// betas (device, nb x p doubles, zero-filled by the caller): beta_S of each solve.
int launch_scatter_beta_batch(iht_dataset *ds, const BSolve *bs, int nb, int kmax, double *betas)
{
    k_scatter_beta_b<<<dim3(ceil_div(kmax, 256), nb), 256, 0, ds->ctx->stream>>>(bs, ds->p, betas);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

}  // namespace iht
