// Internal declarations shared by the CUDA translation units of libiht.
//
// Device data layout (one dataset):
//   G        uint8[p][stride]   PLINK 2-bit codes, SNP-major; stride = ceil(n/4)
//                               rounded up to 128 bytes so rows start on DRAM
//                               sector boundaries; pad samples carry the
//                               missing code 01 so every sum skips them.
//   used     int32[n_pad]       1 for rows of the current solve, else 0
//                               (n_pad = 4 * stride samples).
//   rowmask  uint32[stride/4]   2-bit lanes 11 for used rows, 00 otherwise.
//   u64,v64  double[p]          per-SNP mean / inverse SD over the used rows.
//   u32,v32  float[p]           FP32 copies read by the gradient kernels.
//   y64,r64  double[n_pad]      phenotype and residual (0 off the used rows).
//   r32      float[n_pad]       centred FP32 residual the gradient pass reads.
//   g        float[p]           standardised gradient Z^T r.
#pragma once
#include <cuda_runtime.h>
#include <vector>
#include <stdint.h>

#include <algorithm>

#include "../../include/iht.h"

namespace iht {

constexpr int kMaxK = 1024;            // largest sparsity level accepted
constexpr int kMaxCand = 2 * kMaxK;    // candidate list of the projection
constexpr int kSelBins = 2048;         // radix-select histogram bins
constexpr int kSelCap = 4096;          // keys at or above the boundary bin the fast finish sorts
constexpr int kPartials = 2048;        // max blocks of per-block partial sums (3 values each)
constexpr int kMaxCov = 64;            // nongenetic covariates per dataset

struct Scalars {                       // device-resident state of one solve
    double num;                        // ||g_S||^2
    double mu;                         // step size of the current iteration
    double f;                          // objective after the last update
    double sum_r;                      // sum of r over used rows
    double sumsq_r;                    // sum of r^2 over used rows
    double step;                       // ||beta+ - beta|| / (||beta|| + 1)
    double c, kappa, tol;              // options
    double dd;                         // ||beta+ - beta||^2 of the candidate
    double bb;                         // ||beta||^2
    int32_t iter;                      // updates performed
    int32_t status;                    // IHT_OK / ENOTCONV / ENUMERIC
    int32_t done;                      // 1 once the solve has stopped
    int32_t retry;                     // 1: candidate rejected, mu shrunk (read with done)
    int32_t bt_total;                  // total shrinks
    int32_t bt_last;                   // shrinks of the last iteration
    int32_t changed;                   // support changed in the last iteration
    int32_t max_iter, max_backtrack;
    int32_t k, n_rows;
    int32_t err;                       // bit 0: non-finite input, bit 1: bad rows
    int32_t live;                      // batched solves: takes part in the current attempt
    int32_t fresh;                     // batched solves: beta = 0 set-up still to run
    int32_t skip1;                     // 1: no further attempt this iteration (accepted or stopped)
    int32_t skip2;                     // 1: no next gradient yet (stopped, or still rejecting)
    int32_t htp;                       // 1: HTP (the accepted support is refitted by least squares)
    int32_t pad_;
};

// Device descriptor of one solve of a batch (all pointers device memory).
struct BSolve {
    Scalars *sc;
    const int32_t *used;               // row set of the solve and its statistics
    const double *u64, *v64;
    double *y64, *r64, *rc64, *zv;     // n_pad each
    float *r32;                        // n_pad: centred residual read by the gradient
    float *g;                          // p: gradient
    int32_t *S, *Sp, *cand;            // k, k, K
    double *bS, *bSp, *coef;           // k, k, k
    double *partials;                  // 3 * zmul blocks
    int32_t k, K;
    int64_t out_off;                   // offset of this solve in concatenated outputs
};

// Optional CUDA-event timing of selected launches (pairs begin / end).
struct ProfEvents {
    cudaEvent_t *ev = nullptr;
    int cap = 0;                       // pairs available
    int n = 0;                         // pairs recorded
};
// Inside a stream capture the records are external, so they become event
// nodes of the graph (recorded again on every replay).
inline unsigned prof_flags(cudaStream_t s)
{
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &st) == cudaSuccess && st == cudaStreamCaptureStatusActive
               ? cudaEventRecordExternal
               : cudaEventRecordDefault;
}
inline void prof_begin(ProfEvents *pe, cudaStream_t s)
{
    if (pe && pe->n < pe->cap) cudaEventRecordWithFlags(pe->ev[2 * pe->n], s, prof_flags(s));
}
inline void prof_end(ProfEvents *pe, cudaStream_t s)
{
    if (pe && pe->n < pe->cap) {
        cudaEventRecordWithFlags(pe->ev[2 * pe->n + 1], s, prof_flags(s));
        ++pe->n;
    }
}

struct SelState {                      // top-K selection progress (zero between calls)
    uint32_t prefix, mask, need, count_gt;
    uint32_t n_gt, err;
    uint32_t ticket_a, ticket_b;       // blocks done in launch A / B
    uint32_t ncand;                    // keys at or above the boundary bin
    uint32_t pad[3];
};

// Host-side handles -------------------------------------------------------
struct Workspace;
struct TailWork;                       // fused per-iteration kernel's scratch (tail.cu)
struct TcParams;                       // limb scale, residual sum, error word (limbs.cuh)
struct BatchWork;
void free_batchwork(BatchWork *w);

// Makes a device current for the scope of an API call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

struct SelWork {                       // radix-select scratch, one per context
    uint32_t *hist = nullptr;          // kSelBins
    unsigned long long *cand = nullptr;    // kSelCap candidate words
    SelState *st = nullptr;
};

}  // namespace iht

struct iht_ctx {
    int device;
    cudaStream_t stream;
    int num_sms;
    iht::SelWork sel;
};

struct iht_dataset {
    iht_ctx *ctx;
    int64_t n, p;
    int64_t stride;      // row pitch in bytes: ceil(n/4) rounded up to 128 (sector aligned rows)
    int64_t rowb;        // bytes a kernel reads per row: ceil(n/4) rounded up to 16
    int64_t n_pad;       // 4 * stride samples
    uint8_t *G;
    // missing calls (code 01), built once at upload: sample offsets of SNP j
    // are miss_idx[miss_off[j] .. miss_off[j+1]) (uint16 when n <= 65536), in
    // residue classes (i - j) mod 8 = 0, 1, .., 7, ascending within a class (the
    // order every kernel sums them in: adjacent SNPs start on different shared-
    // memory banks when their lanes gather staged residuals)
    int64_t *miss_off;
    void *miss_idx;
    int64_t miss_total;
    bool miss_idx16;
    // the same lists padded for the multi-column finalisation (uint16, built
    // when a 4-column residual table with 8 zero rows fits in shared memory):
    // groups of kPadGroup consecutive SNPs; every SNP of group g has a sequence
    // of the same length L_g with the same class boundaries (class c padded to
    // the group's longest class c with zero-row indices n_pad + ((j + c) mod 8),
    // then to a multiple of 8 with n_pad + (j mod 8)); SNP j's sequence starts
    // at miss_goff[g] + (j mod 8) L_g, L_g = (miss_goff[g + 1] - miss_goff[g]) / 8
    int64_t *miss_goff = nullptr;
    uint16_t *miss_gidx = nullptr;
    // the same lists interleaved for the single-column missing-call sums
    // (uint16, built when r and 32 zero slots fit the sums kernel's shared
    // memory): groups of 32 consecutive SNPs, group g's sequences of common
    // length L_g (its longest list rounded up to a multiple of 8, padded with
    // the zero slot n_pad + (j mod 32)); entry t of SNP j at miss_ioff[g] +
    // 256 (t / 8) + 8 (j mod 32) + t mod 8, L_g = (miss_ioff[g + 1] -
    // miss_ioff[g]) / 32
    int64_t *miss_ioff = nullptr;
    uint16_t *miss_iidx = nullptr;
    // nongenetic covariates (iht_set_covariates): q dense columns, predictors
    // p .. p+q-1; cov[t * n_pad + i] = covariate t of subject i (0 on pad samples)
    int64_t q = 0;
    double *cov = nullptr;
    iht::Workspace *ws;
};

namespace iht {

struct Workspace {
    int64_t p = 0, n_pad = 0;
    int kcap = 0;
    bool rowset_all = false;               // used/rowmask/statistics hold the all-rows set
    int32_t *used = nullptr;
    uint32_t *rowmask = nullptr;
    int32_t *counts = nullptr;
    double *u64 = nullptr, *v64 = nullptr;
    float *u32 = nullptr, *v32 = nullptr;
    double *y64 = nullptr, *r64 = nullptr, *zv = nullptr;
    double *rc64 = nullptr;                // residual of the candidate update
    float *r32 = nullptr, *g = nullptr;    // g: p + kMaxCov entries (covariates after the SNPs)
    float *Mj = nullptr;                   // per-SNP sum of r over missing calls
    // covariates over the current row set: mean, inverse SD, standardised
    // values zc[t * n_pad + i] (0 off the used rows)
    double *cu64 = nullptr, *cv64 = nullptr, *zc = nullptr;
    // HTP refit scratch: Gamma, standardised support columns, Gram, Cholesky factor
    int32_t *gam = nullptr;
    double *zs = nullptr, *gram = nullptr, *chol = nullptr, *hvec = nullptr;
    int htp_k = 0;                         // support size the refit scratch holds
    double *partials = nullptr;        // kPartials * 2
    int32_t *rows_dev = nullptr;       // int32[n]: host row lists copied here
    double *ybuf = nullptr;            // double[n]: host phenotypes copied here
    float *fbuf = nullptr;             // float[n_pad]: scratch
    int32_t *cand = nullptr;           // kMaxCand
    // solver state
    int32_t *S = nullptr, *Sp = nullptr;   // current / next support (k, ascending)
    double *bS = nullptr, *bSp = nullptr;  // beta on S / S+
    double *coef = nullptr;                // scratch coefficients (kMaxCand)
    int32_t *cols = nullptr;               // scratch columns (kMaxCand)
    Scalars *sc = nullptr;
    Scalars *sc_host = nullptr;            // pinned mirror
    // optional timing of the gradient launches of a solve
    cudaEvent_t prof_ev[2 * 256] = {};
    int nprof = 0;
    double prof_ms = 0.0;
    // one iteration of a solve as a CUDA graph, replayed while its key matches
    cudaGraphExec_t iter_exec = nullptr;
    cudaStream_t cap_stream = nullptr;     // private stream the iteration is captured on
    uint64_t iter_key[8] = {};
    int iter_launches = 0;                 // kernel launches per replay
    cudaEvent_t gev[2] = {};               // around the gradient pass inside the graph
    int graph_replays = 0;                 // iterations of the last solve run as replays
    BatchWork *bw = nullptr;               // batched solves (batch.cu)
    // a whole solve as one graph: a conditional while loop over the fused
    // per-iteration kernel and the gradient pass (tail.cu)
    TailWork *tail = nullptr;
    int32_t *Sp2 = nullptr;                // the second candidate of the fused kernel (mu / kappa)
    double *bSp2 = nullptr, *rc64_2 = nullptr, *partials2 = nullptr;
    cudaGraphExec_t fused_exec = nullptr;
    uint64_t fused_key[12] = {};
    int fused_launches = 0;                // kernels per loop trip
    int fused_setup_launches = 0;          // kernels ahead of the loop (whole-solve graph)
    Scalars *sc_init = nullptr;            // device: a whole-solve graph's starting scalars
    int32_t *flags_host = nullptr;         // pinned: barrier and pass error words after a solve
    // pinned: a whole solve's support (kMaxK int32) then beta_S (kMaxK doubles),
    // copied with its final scalars ahead of its one synchronisation when the
    // caller wants host outputs (out_want); out_ready: they are there
    void *out_host = nullptr;
    int out_want = 0, out_ready = 0;
};
constexpr int kProfEvents = 256;

// error helpers -----------------------------------------------------------
void set_cuda_error(cudaError_t e, const char *where);
// Device allocations of the library go through these (host-side fault
// injection, iht_fault_inject, can make them fail as an exhausted device would).
cudaError_t dev_malloc_raw(void **ptr, size_t bytes);
cudaError_t dev_malloc_async_raw(void **ptr, size_t bytes, cudaStream_t s);
template <typename T> inline cudaError_t dev_malloc(T **ptr, size_t bytes)
{
    return dev_malloc_raw(reinterpret_cast<void **>(ptr), bytes);
}
template <typename T> inline cudaError_t dev_malloc_async(T **ptr, size_t bytes, cudaStream_t s)
{
    return dev_malloc_async_raw(reinterpret_cast<void **>(ptr), bytes, s);
}
// true (and one injected fault used up) when a fault of `kind` is pending
bool fault_take(int kind);
void note_launch(int n = 1);           // kernel launches issued (iht_kernel_launches)
uint64_t launches_noted();
#define IHT_CUDA(call)                                                  \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) {                                        \
            ::iht::set_cuda_error(e_, #call);                           \
            return e_ == cudaErrorMemoryAllocation ? IHT_ENOMEM : IHT_ECUDA; \
        }                                                               \
    } while (0)

int ensure_workspace(iht_dataset *ds, int kcap);
void free_workspace(Workspace *ws);

// Device arrays of one row set and its per-SNP statistics.
struct RowSet {
    int32_t *used = nullptr;       // int32[n_pad], 1 on the set's rows
    uint32_t *rowmask = nullptr;   // uint32[stride/4], 2-bit lanes 11 on the set's rows
    int32_t *counts = nullptr;     // int32[4p] or null
    double *u64 = nullptr, *v64 = nullptr;
    float *u32 = nullptr, *v32 = nullptr;
};

// kernels launched from the host side (stream-ordered) ---------------------
// geno.cu
RowSet workspace_rowset(iht_dataset *ds);
int setup_rowset(iht_dataset *ds, const int32_t *rows_dev, int64_t n_rows, const RowSet &rs,
                 int32_t *err);
int launch_counts_rowset(iht_dataset *ds, int64_t n_rows, const RowSet &rs);
int launch_counts_sets(iht_dataset *ds, const RowSet *sets, const int64_t *n_rows, int nsets);
int launch_fix_padding(iht_dataset *ds);
int build_missing_lists(iht_dataset *ds);
constexpr int kPadGroup = 8;
bool padded_lists_wanted(const iht_dataset *ds);
int launch_missing_sums(iht_dataset *ds, const float *r32, float *M, const int32_t *done);
// The missing-call sums plus the limb image of r for the next tensor-core pass
// (the fused solve); EINVAL when r does not fit the kernel's shared memory.
bool missing_limbs_supported(const iht_dataset *ds, int64_t nlim);
int launch_missing_sums_limbs(iht_dataset *ds, const float *r32, float *M, const int32_t *done,
                              uint8_t *bimg, TcParams *prm, int64_t nlim, bool programmatic = false);
int setup_rows(iht_dataset *ds, const int32_t *rows_dev, int64_t n_rows);
int launch_counts(iht_dataset *ds, int64_t n_rows);
int scatter_rows_f64(iht_dataset *ds, const int32_t *rows_dev, int64_t n_rows, const double *src,
                     double *dst);
int scatter_rows_f32(iht_dataset *ds, const int32_t *rows_dev, int64_t n_rows, const float *src,
                     float *dst);
// grad_simt.cu / grad_tc.cu
int launch_grad_simt(iht_dataset *ds, const float *r32, float *g, const int32_t *done);
int launch_grad_tc(iht_dataset *ds, const float *r32, float *g, const int32_t *done);
bool grad_tc_supported(const iht_dataset *ds);
int prepare_grad_tc(iht_dataset *ds, const float *r32, const int32_t *done);
// hist (optional): the selection's 2048-bin histogram of |g| bits 30..20 the
// pass adds its keys to (hflag bit 0: a non-finite g)
// (programmatic: launched with programmatic stream serialization -- it may
// start while the kernel before it runs, and waits for it before reading)
int launch_grad_tc_main(iht_dataset *ds, const float *r32, float *g, const int32_t *done,
                        uint32_t *hist = nullptr, uint32_t *hflag = nullptr, bool programmatic = false);
int prepare_grad_tc_to(iht_dataset *ds, const float *r32, float *Mj, const int32_t *done);
int launch_grad_tc_main_with(iht_dataset *ds, const float *r32, float *g, const float *u32,
                             const float *v32, const float *Mj, const int32_t *done,
                             uint32_t *hist = nullptr, uint32_t *hflag = nullptr, bool programmatic = false);
void grad_tc_release_thread();
uint64_t grad_tc_scratch_id();
int grad_tc_status(iht_dataset *ds, int *timed_out);
int grad_tc_reset_status(iht_dataset *ds);
int grad_tc_limb_buffers(iht_dataset *ds, uint8_t **bimg, TcParams **prm, int64_t *nlim);
// impl: 0 default (tensor cores when supported), 1 CUDA cores, 2 tensor cores
int launch_grad_impl(iht_dataset *ds, int impl, const float *r32, float *g, const int32_t *done);
int launch_grad_simt_stats(iht_dataset *ds, const float *r32, const float *u32, const float *v32,
                           float *g);
// grad_mrhs.cu: one residual column of a multi-column gradient pass (device)
struct MrCol {
    const float *r32;              // n_pad residual, zero off the column's rows
    const float *u32, *v32;        // statistics of the column's row set
    float *g;                      // p outputs
    float scale, R;                // set by the pass
};
int mrhs_max_cols();
bool grad_mrhs_supported(const iht_dataset *ds);
int launch_grad_mrhs(iht_dataset *ds, MrCol *cols_dev, int ncols, ProfEvents *prof = nullptr,
                     const MrCol *cols_host = nullptr);
int grad_mrhs_status(iht_dataset *ds, int *timed_out);
int grad_mrhs_reset_status(iht_dataset *ds);
void grad_mrhs_release_thread();
uint64_t grad_mrhs_scratch_id();
// solver.cu: out-of-fold residuals of fitted solves (cross-validation)
struct CvJob {
    const int32_t *S;          // k support indices of the fit
    const double *bS;          // beta on S
    int32_t k;
    const int32_t *used;       // n_pad, 1 on the partition's (test) rows
    const double *u64, *v64;   // statistics of the fit's training rows
    const double *y64;         // n_pad phenotype (all rows)
    double *out;               // n_pad: y - Z_S beta_S on the test rows, 0 elsewhere
    double *partials;          // 3 per block: sum, sum of squares, 0
};
int launch_cv_resid(iht_dataset *ds, const CvJob *jobs_dev, int njobs);
// tune.cu: cached launch shapes of the gradient passes (kind IHT_PASS_SINGLE /
// IHT_PASS_MULTI; bucket 0 for the single-column pass, else the largest
// accumulator width of the multi-column bucket)
constexpr int kTuneParams = 5;
bool autotune_enabled();
bool tune_lookup(const iht_dataset *ds, int kind, int bucket, int *params);
void tune_store(const iht_dataset *ds, int kind, int bucket, const int *params, double ms, int candidates);
bool stream_capturing(cudaStream_t s);
bool grad_tc_shape_fits(const iht_dataset *ds, const int *params);
bool grad_mrhs_shape_fits(int ncols, const int *params);
int grad_mrhs_bucket(int ncols);
// Events of one tuning run, destroyed with the set.
struct TuneEvents {
    std::vector<cudaEvent_t> ev;
    explicit TuneEvents(size_t n) : ev(n, nullptr) {}
    ~TuneEvents()
    {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
    cudaError_t create()
    {
        for (cudaEvent_t &e : ev)
            if (cudaError_t r = cudaEventCreate(&e)) return r;
        return cudaSuccess;
    }
    float ms(size_t a, size_t b) const
    {
        float t = 0.0f;
        return cudaEventElapsedTime(&t, ev[a], ev[b]) == cudaSuccess ? t : 1e30f;
    }
};
// select.cu
struct SelJob {                        // one problem of a batched top-K
    const float *keys;
    int32_t *out;
    SelState *st;
    uint32_t *hist;                    // kSelBins
    unsigned long long *cand;          // kSelCap candidate words
    const int32_t *done;               // skip the problem when *done (may be null)
    uint32_t K;
};
int select_topk_batch(iht_ctx *ctx, const SelJob *jobs, int nb, int64_t p);
int ensure_selwork(iht_ctx *ctx, int64_t p);
// gS .. gsc (optional): also form g_S and ||g_S||^2 of support gS (k = gk) in
// the selection's last block (gather_gS_body).
int select_topk(iht_ctx *ctx, const float *key_src, int64_t p, int32_t K, int32_t *out_idx,
                const int32_t *done, const int32_t *gS = nullptr, int gk = 0,
                double *gcoef = nullptr, Scalars *gsc = nullptr);
// solver.cu
int zmul_blocks(const iht_dataset *ds);
int launch_zmul(iht_dataset *ds, const int32_t *cols, int32_t m, const double *coef,
                const double *u, const double *v, const int32_t *used, const double *base,
                double *out, double *partials);
int gather_rows_f64(iht_dataset *ds, const int32_t *rows_dev, int64_t n_rows, const double *src,
                    double *dst);
int check_finite_y(iht_dataset *ds, int64_t n_rows, const double *y_dev);
int check_finite_y_sc(iht_dataset *ds, int64_t n_rows, const double *y_dev, Scalars *sc);
struct SolveInit {                     // resume a solve from its state (host arrays)
    const int32_t *S;                  // k, strictly ascending
    const double *bS;                  // beta on S
    int32_t iter, backtracks;          // counters so far
};
int run_solve_host(iht_dataset *ds, int k, const iht_options *opt, int n_rows, iht_trace *trace,
                   int max_iter, const SolveInit *init = nullptr);
int write_beta_device(iht_dataset *ds, int k, double *beta_out);
// tail.cu: the rest of a solve after its first gradient pass as one graph
// launch (no host synchronisation per iteration); false when the shape is not
// supported (then the per-iteration graph runs)
bool fused_supported(const iht_dataset *ds, int k, int impl);
int run_fused_solve(iht_dataset *ds, int k, int K, int impl);
// The whole solve from beta = 0 as one graph launch (set-up, then the loop):
// h is the solve's starting scalars; on return ws->sc_host holds the final
// ones.  EAGAIN (nothing enqueued) when the graph cannot be built.
int run_whole_fused_solve(iht_dataset *ds, int k, int K, int impl, const Scalars &h);
// (hist, hflag: the gradient pass's keys go to this histogram, as in launch_grad_tc_main)
int enqueue_solve_setup(iht_dataset *ds, int k, int impl, uint32_t *hist = nullptr,
                        uint32_t *hflag = nullptr);
bool grad_tc_shape_settled(const iht_dataset *ds);
void free_fused(Workspace *ws);
// htp.cu: covariates of the current row set, their gradient entries, and the
// least-squares refit of HTP
int cov_setup(iht_dataset *ds, int64_t n_rows);
int launch_cov_grad(iht_dataset *ds, const float *r32, float *g, const int32_t *done,
                    uint32_t *hist = nullptr, uint32_t *hflag = nullptr);
int htp_refit(iht_dataset *ds, int k, const int32_t *Sp, double *bSp, const int32_t *done);
int ensure_htp_scratch(iht_dataset *ds, int k);
// batched tails (blockIdx selects the solve; finished solves return at once)
enum ZmulWhich { kZmulInit = 0, kZmulStep = 1, kZmulResidual = 2 };
int launch_gather_gS_batch(iht_dataset *ds, const BSolve *bs, int nb);
int launch_zmul_batch(iht_dataset *ds, const BSolve *bs, int nb, int kmax, ZmulWhich which);
int launch_init_objective_batch(iht_dataset *ds, const BSolve *bs, int nb);
int launch_center_batch(iht_dataset *ds, const BSolve *bs, int nb, bool init);
int launch_merge_batch(iht_dataset *ds, const BSolve *bs, int nb, int first);
int launch_decide_batch(iht_dataset *ds, const BSolve *bs, int nb);
int launch_scatter_beta_batch(iht_dataset *ds, const BSolve *bs, int nb, int kmax, double *betas);
int launch_finish_fresh_batch(iht_dataset *ds, const BSolve *bs, int nb, int kmax);
int launch_compact_support_batch(iht_dataset *ds, const BSolve *bs, int nb, int kmax,
                                 int32_t *supports, double *beta_s);

// device helpers ------------------------------------------------------------
// Programmatic dependent launch (a kernel launched with programmatic stream
// serialization may start while the grid before it still runs): wait for the
// grids this one depends on to complete with their memory visible (at once
// when launched without such a dependency), and let the dependent grid launch
// once every block of this one has called it or exited.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ float warp_sum(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Fixed-order block sum (deterministic); every thread gets the result.
// `sh` needs blockDim.x / 32 doubles.
__device__ __forceinline__ double block_sum(double x, double *sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    x = warp_sum(x);
    __syncthreads();
    if (lane == 0) sh[wid] = x;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = lane < nw ? sh[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) sh[0] = t;
    }
    __syncthreads();
    t = sh[0];
    __syncthreads();
    return t;
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// g = v (S1 - u (R - M)) with every operation rounded on its own (no
// contraction), so the single- and multi-column passes give the same value.
__device__ __forceinline__ float standardise(float S1, float R, float M, float u, float v)
{
    return __fmul_rn(v, __fsub_rn(S1, __fmul_rn(u, __fsub_rn(R, M))));
}

// g_S (coef) and ||g_S||^2 (sc->num) for the step size: the first warp of the
// block, lanes strided over S then a shuffle tree, so the sum's order does not
// depend on the block size (the single-solve selection's last block and the
// batched kernel give the same bits).
// ||g_S||^2 from g_S by one warp: lane l adds its squares c = l, l + 32, ...
// in order with fused multiply-adds, then an xor shuffle tree (every caller
// forms it this way, so every path has the same bits).
__device__ __forceinline__ double gS_sumsq_warp(const double *coef, int k)
{
    double s = 0.0;
#pragma unroll 2
    for (int c = threadIdx.x & 31; c < k; c += 32) s = __fma_rn(coef[c], coef[c], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

__device__ __forceinline__ void gather_gS_body(const float *__restrict__ g,
                                               const int32_t *__restrict__ S, int k,
                                               double *__restrict__ coef, Scalars *sc)
{
    if (threadIdx.x >= 32) return;
    double s = 0.0;
#pragma unroll 2
    for (int c = threadIdx.x; c < k; c += 32) {
        const double x = (double)g[S[c]];
        coef[c] = x;
        s = __fma_rn(x, x, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) sc->num = s;
}

// The same from D = sum over all calls of (2 x + [call missing]) r, which is
// what the tensor-core dosage map yields (a missing call counts once):
// S1 = (D - M) / 2.
__device__ __forceinline__ float standardise_d(float D, float R, float M, float u, float v)
{
    return standardise(__fmul_rn(0.5f, __fsub_rn(D, M)), R, M, u, v);
}

}  // namespace iht
