/*
 * iht.h -- C ABI of the B300 (sm_103a) library for iterative hard
 * thresholding (IHT) least squares on PLINK-packed genotypes.
 *
 * Method: Keys, Chen & Lange, "Iterative Hard Thresholding for Model
 * Selection in Genome-Wide Association Studies".  The library minimises
 *   f(beta) = 1/2 ||y - Z beta||^2   subject to ||beta||_0 <= k
 * (Eq. leastsquaresloss, Sec. 2.2) by projected gradient steps
 *   beta+ = P_{S_k}[beta + mu g],  g = Z^T (y - Z beta)   (Eq. ihta, Eq. normal_grad)
 * with the normalized step size and its backtracking check (Sec. 2.3.1),
 * where Z is the genotype matrix standardised on the fly (Sec. 2.3.2).
 *
 * Conventions (every entry point):
 *   - Return an int status (iht_status).  No C++ exception crosses the ABI.
 *   - Work is ordered on the context's CUDA stream.  Calls that return host
 *     results synchronise that stream before returning.
 *   - The caller owns every input and output buffer.  The library owns the
 *     context, datasets and all scratch memory.
 *   - Genotype codes (PLINK .bed, SNP-major): 00 hom-ref (dosage 0),
 *     01 missing, 10 het (dosage 1), 11 hom-alt (dosage 2).
 *   - Standardisation: u_j = mean dosage over observed calls of the rows in
 *     use, v_j = 1/SD with an (n_obs - 1) denominator (v_j = 0 when the SD is
 *     0 or n_obs < 2); z_ij = v_j (x_ij - u_j) for observed calls, 0 for
 *     missing calls (Sec. 2.3.2 identity; Sec. 3.1).
 */
#ifndef IHT_H
#define IHT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum iht_status {
    IHT_OK = 0,
    IHT_EINVAL = 1,    /* bad argument: k < 1, k > p, n_rows < 2, bad .bed magic/size, ... */
    IHT_ENOMEM = 2,    /* device or host allocation failed                               */
    IHT_ENOTCONV = 3,  /* max_iter reached before convergence; results are valid          */
    IHT_ENUMERIC = 4,  /* NaN/Inf input, or a zero step-size denominator with g_S != 0    */
    IHT_ETIMEOUT = 5,  /* a bounded device wait gave up                                  */
    IHT_ECUDA = 6,     /* a CUDA runtime call failed (iht_last_cuda_error tells which)    */
    IHT_EAGAIN = 7     /* result not ready yet                                            */
} iht_status;

typedef enum iht_mem { IHT_HOST = 0, IHT_DEVICE = 1 } iht_mem;

typedef struct iht_ctx iht_ctx;
typedef struct iht_dataset iht_dataset;

/* Solver options (Sec. 2.3.1; readings of unstated constants in brackets). */
typedef struct iht_options {
    int32_t max_iter;      /* iteration cap [100]                                   */
    int32_t max_backtrack; /* step shrinks per iteration [50]                       */
    double tol;            /* stop when ||beta+ - beta|| / (||beta|| + 1) < tol [1e-4] */
    double c;              /* omega = (1-c)||d||^2/||Z d||^2, 0 < c << 1 [0.01]       */
    double kappa;          /* shrink mu <- mu / kappa while mu >= omega [2]           */
    int32_t in_mem;        /* where rows and y live: IHT_HOST or IHT_DEVICE          */
    int32_t out_mem;       /* where beta_out and support_out live                    */
    int32_t grad_impl;     /* gradient kernel: 0 default, 1 CUDA-core, 2 tensor-core  */
    int32_t profile;       /* 1: time every gradient launch with CUDA events [0]     */
    int32_t variant;       /* IHT_VARIANT_IHT [default] or IHT_VARIANT_HTP (below)   */
    int32_t flags;         /* IHT_FIT_* bits (below) [0]                              */
} iht_options;

/* iht_options.flags.
 *   IHT_FIT_BETA_ZEROED: a host beta_out holds zeros on entry, so iht_fit writes
 *     only its support entries (without it, iht_fit first writes zeros to all
 *     p + q entries: the bytes of a freshly allocated buffer are then all
 *     touched once).  Ignored for device outputs.  Other bits: EINVAL. */
enum { IHT_FIT_BETA_ZEROED = 1 };

/* Solver variants (iht_options.variant).
 *   IHT: the projected gradient step of Eq. ihta.
 *   HTP: hard thresholding pursuit (Sec. 2.2: the projection is followed by a
 *        least-squares solve of the normal equations, Eq. normal_equations, on
 *        the active set).  After a refit the gradient vanishes on the support,
 *        so the normalized step is taken over the k largest |g_j| (ties to the
 *        lower index); the backtracking check applies to the projected
 *        candidate, whose support S+ is then refitted by an FP64 Cholesky
 *        solve in ascending index order, a column with pivot <= 1e-10 times its
 *        diagonal entry (zero or dependent on earlier columns) getting 0.
 *        Supported by iht_fit and iht_fit_trace; the batched calls, iht_cv,
 *        the server and iht_fit_resume return EINVAL for it. */
enum { IHT_VARIANT_IHT = 0, IHT_VARIANT_HTP = 1 };

typedef struct iht_result {
    int32_t iterations;    /* updates performed                                */
    int32_t status;        /* iht_status of the solve                          */
    int32_t backtracks;    /* total step shrinks                               */
    int32_t reserved;
    double objective;      /* 1/2 ||y - Z beta||^2 at exit (FP64)              */
    double mu;             /* last accepted step size                          */
    double grad_ms;        /* total device time of the gradient launches (profile = 1) */
    int32_t grad_launches; /* gradient launches timed                          */
    int32_t graph_replays; /* iterations run as one CUDA graph replay          */
} iht_result;

/* Optional per-iteration record of iht_fit_trace (host arrays; any may be NULL).
 * Arrays have max_iter entries; supp and beta have max_iter * k. */
typedef struct iht_trace {
    double *objective;     /* f after each update                               */
    double *mu;            /* accepted step size                                */
    int32_t *backtracks;   /* shrinks in the iteration                          */
    int32_t *changed;      /* 1 if the support changed                          */
    int32_t *supp;         /* accepted support, ascending (k per iteration)     */
    double *beta;          /* beta on that support (k per iteration)           */
} iht_trace;

/* Fill *opt with the defaults in brackets above (host in/out, default kernels). */
void iht_default_options(iht_options *opt);

/* Static string for a status code. */
const char *iht_strerror(int status);

/* Name of the last CUDA error seen by this thread ("" if none). */
const char *iht_last_cuda_error(void);

/* Number of CUDA kernel launches this library has issued in this process
 * (all threads, all devices).  Host-only; lets callers count device work. */
uint64_t iht_kernel_launches(void);

/* Host-side fault injection, for testing how failures reach the caller (the
 * paper has no counterpart).  No device fault is made and no kernel changes:
 *   IHT_FAULT_ALLOC   : the next `count` device allocations made by the library
 *                       fail as on an exhausted device (calls return ENOMEM and
 *                       free what they had taken);
 *   IHT_FAULT_TIMEOUT : the next `count` reads of a gradient pass's bounded-wait
 *                       status find its error word set (the library writes it
 *                       from the host before the read, as a device wait that
 *                       gave up would have), so the call returns ETIMEOUT;
 *   IHT_FAULT_NONE    : clears pending faults (count ignored).
 * Process-wide, all threads.  EINVAL for another kind or count < 0. */
enum { IHT_FAULT_NONE = 0, IHT_FAULT_ALLOC = 1, IHT_FAULT_TIMEOUT = 2 };
int iht_fault_inject(int kind, int32_t count);

/* Create a context on CUDA device `device` that orders all work on `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * context.  EINVAL for a bad device, ECUDA if the device cannot be used. */
int iht_create(iht_ctx **out, int device, void *stream);

/* Free a context (datasets created from it must be freed first). */
int iht_destroy(iht_ctx *ctx);

/* a0 -- upload a PLINK .bed image once; the packed matrix then stays resident
 * on the device for every later call (Sec. 2.3.3 device data placement).
 *   bed, bed_bytes : the whole file image, 3-byte magic 0x6C 0x1B 0x01 then
 *                    p SNP rows of ceil(n/4) bytes; host or device memory
 *                    as `mem` says.  Read only during the call.
 *   n, p           : subjects and SNPs.
 * The library keeps a repacked copy: row stride rounded up to 16 bytes, pad
 * samples set to the missing code.  EINVAL on bad magic, size mismatch,
 * n < 1 or p < 1; ENOMEM if the copy does not fit. */
int iht_load_bed(iht_ctx *ctx, const uint8_t *bed, size_t bed_bytes, int mem, int64_t n,
                 int64_t p, iht_dataset **out);

/* Free a dataset and its device memory. */
int iht_dataset_free(iht_dataset *ds);

/* Dataset shape: n, p and the repacked row stride in bytes (any may be NULL). */
int iht_dataset_shape(const iht_dataset *ds, int64_t *n, int64_t *p, int64_t *stride);

/* Nongenetic covariates (Sec. 3: the predictors are the SNPs and the
 * covariates, and a model size k counts both).  Sets q dense columns that
 * iht_fit and iht_fit_trace append to the SNPs as predictors p .. p+q-1:
 * each is standardised over the rows of the solve (mean, (n_rows - 1)
 * denominator, a constant column is inert) and competes in the projection
 * like a SNP.  With covariates set, beta_out of those calls has p + q entries
 * and support entries >= p name covariates.
 *   cov : double[q][n], covariate t of subject i at cov[t * n + i], in memory
 *         of kind `mem`; copied (the caller keeps ownership).
 *   q   : 0..64; 0 removes the covariates.
 * A non-finite value on a used row makes the fit return ENUMERIC.  The
 * batched calls, iht_cv, the server and iht_fit_resume return EINVAL on a
 * dataset with covariates.  EINVAL for q outside 0..64 or cov NULL with q > 0;
 * ENOMEM if the copy does not fit. */
int iht_set_covariates(iht_dataset *ds, const double *cov, int32_t q, int mem);

/* a1 -- per-SNP code counts and the cached mean / inverse-SD vectors u, v of
 * Sec. 2.3.2, over a row set.
 *   rows       : n_rows distinct subject indices in [0, n), or NULL for all n.
 *   counts_out : int32[p][4] (index = code 0..3), may be NULL.
 *   u_out      : double[p] means, v_out: double[p] inverse SDs, may be NULL.
 * rows and the outputs live in memory of kind `mem`.  The FP64 statistics are
 * computed from the integer counts in the order n_obs = n_rows - n_miss,
 * s1 = n_het + 2 n_homalt, s2 = n_het + 4 n_homalt, u = s1/n_obs,
 * var = (s2 - s1*s1/n_obs)/(n_obs - 1), v = 1/sqrt(var). */
int iht_counts(iht_dataset *ds, const int32_t *rows, int64_t n_rows, int mem,
               int32_t *counts_out, double *u_out, double *v_out);

/* a2 -- one standardised gradient pass g = Z^T r (Eq. normal_grad; the
 * negative gradient of f at the beta whose residual is r).
 *   rows   : device int32[n_rows] subject indices or NULL (= all n); the
 *            statistics are those of this row set.
 *   r      : device float[n_rows], aligned with rows.
 *   g_out  : device float[p].
 *   impl   : 0 default, 1 CUDA-core kernel, 2 tensor-core kernel.
 * ETIMEOUT when a bounded wait of the tensor-core pass gave up (g_out invalid).
 * Computed as g_j = v_j (S1_j - u_j (R - M_j)), S1 = sum of dosage * r over
 * observed calls, M = sum of r over missing calls, R = sum of r. */
int iht_gradient(iht_dataset *ds, const int32_t *rows, int64_t n_rows, const float *r,
                 float *g_out, int impl);

/* a3 -- projection onto the k-sparse set (Eq. ihta): the k indices of the
 * largest |w_j|, ties to the lower index, returned ascending.
 *   w: device float[p]; idx_out: device int32[k].  EINVAL if k < 1 or k > p;
 *   ENUMERIC if w holds a NaN (idx_out is still written: NaN ranks above +Inf). */
int iht_topk(iht_ctx *ctx, const float *w, int64_t p, int32_t k, int32_t *idx_out);

/* Allocation-free variant of iht_topk (the paper has no counterpart; this is
 * an interface for callers that cannot allocate device memory -- for example a
 * host that hands all GPU memory to its own pool allocator, or a latency-
 * critical loop that must not call cudaMalloc, which can synchronise the device
 * or fail under memory pressure).  Same result as iht_topk: the k indices of
 * the largest |w_j|, ties to the lower index, ascending.
 *   device  : CUDA device the pointers belong to.
 *   stream  : cudaStream_t to order the work on (NULL = legacy default stream).
 *   w       : device float[p];  idx_out: device int32[k].
 * The selection's scratch is a static device array in the library (about
 * 41 KB, held on every GPU that loads the library until the process exits);
 * p is limited to 16 777 216 (a fixed maximum of this entry point, not a
 * bound set by the array, whose size does not depend on p); larger p returns
 * IHT_EINVAL without launching anything.  The first call on a device looks the
 * array's address up with cudaGetSymbolAddress and clears it with
 * cudaMemsetAsync on `stream`; make that first call before any stream capture.
 * The call only enqueues work on `stream` (it does not synchronise), so it
 * cannot report NaN keys: they rank above +Inf and the call returns IHT_OK.
 * All calls on a device share the scratch, so calls that overlap on the GPU
 * (other streams or other host threads) race.  Never calls cudaMalloc or
 * cudaFree. */
int iht_topk_noalloc(int device, void *stream, const float *w, int64_t p, int32_t k,
                     int32_t *idx_out);

/* a4/a6 -- sparse standardised product out = Z[rows, cols] coef: only the m
 * listed columns are decoded and standardised (Sec. 2.3.2-2.3.3, X_k beta_k).
 *   cols: device int32[m]; coef: device double[m]; out: device double[n_rows].
 *   u, v: device double[p] statistics to standardise with (e.g. a training
 *   fold's, for held-out rows); NULL = statistics of `rows`. */
int iht_zmul(iht_dataset *ds, const int32_t *rows, int64_t n_rows, const double *u,
             const double *v, const int32_t *cols, int32_t m, const double *coef, double *out);

/* a2-a6 -- IHT least squares to convergence (Sec. 2.2-2.3.1).
 *   rows        : int32[n_rows] subjects the solve uses, or NULL for all n.
 *   y           : double[n_rows] phenotype aligned with rows.
 *   k           : sparsity level, 1 <= k <= p (+ q with covariates), k <= 1024.
 *   opt         : options (NULL = defaults).  rows and y live in opt->in_mem,
 *                 beta_out and support_out in opt->out_mem.
 *   beta_out    : double[p] (p + q with covariates), written in full (zeros
 *                 off the support).
 *   support_out : int32[k], ascending.
 *   info        : host iht_result, may be NULL.
 * Starts from beta = 0 with S^0 = the top-k of |Z^T y|.  Returns the solve's
 * status: OK, ENOTCONV (results valid), ENUMERIC, EINVAL, ENOMEM, ECUDA, or
 * ETIMEOUT when a bounded wait of a tensor-core gradient pass gave up (the
 * outputs are then not valid). */
int iht_fit(iht_dataset *ds, const int32_t *rows, int64_t n_rows, const double *y, int32_t k,
            const iht_options *opt, double *beta_out, int32_t *support_out, iht_result *info);

/* iht_fit with a per-iteration record (host arrays, see iht_trace). */
int iht_fit_trace(iht_dataset *ds, const int32_t *rows, int64_t n_rows, const double *y,
                  int32_t k, const iht_options *opt, double *beta_out, int32_t *support_out,
                  iht_result *info, iht_trace *trace);

/* Checkpoint / resume.  Between iterations the method carries only the support
 * S, beta on S and its counters (Sec. 2.2: the residual, the gradient and the
 * step size are recomputed from them), so a solve stopped after m iterations
 * (max_iter = m, status ENOTCONV) and resumed from its state takes exactly the
 * iterations the uninterrupted solve takes: same supports, same beta bit for
 * bit, same count.
 *
 * The state image is a host byte string, little-endian: "IHTSTATE", version 1
 * (uint32), header size 80 (uint32), n, p, n_rows (int64), k, iterations,
 * backtracks, status (int32), objective, mu (double), an FNV-1a 64-bit
 * checksum of the image taken with this field zero (uint64), then support[k]
 * (int32, strictly ascending in [0, p)) and beta_s[k] (double, finite).
 * No device work and no CUDA device needed for these three:
 *   iht_state_bytes: image size for k (1 <= k <= 1024).
 *   iht_state_save : image of a solve's outputs -- host support_out, beta_out
 *                    on the support and info of iht_fit -- fitted on n_rows of a
 *                    dataset of shape (n, p) into buf.  EINVAL when buf_bytes is
 *                    too small or the support / values are not as above.
 *   iht_state_load : parses an image.  With support, beta_s and info all NULL
 *                    only the shape (n, p, n_rows, k) is returned; otherwise
 *                    support and beta_s receive k entries (k <= k_cap) and info
 *                    (optional) the counters.  EINVAL when the magic, version,
 *                    size or checksum is wrong, or the contents are invalid.
 * iht_fit_resume: iht_fit that starts from the image (state, state_bytes,
 * host memory) instead of beta = 0.  k is the image's; the image's n and p must
 * be the dataset's and its n_rows the rows given (EINVAL otherwise).  The
 * iteration count continues from the image's, so opt->max_iter caps the total
 * and info->iterations / backtracks are totals. */
int iht_state_bytes(int32_t k, size_t *bytes);
int iht_state_save(int64_t n, int64_t p, int64_t n_rows, int32_t k, const int32_t *support,
                   const double *beta_s, const iht_result *info, void *buf, size_t buf_bytes);
int iht_state_load(const void *buf, size_t buf_bytes, int32_t k_cap, int64_t *n, int64_t *p,
                   int64_t *n_rows, int32_t *k, int32_t *support, double *beta_s,
                   iht_result *info);
int iht_fit_resume(iht_dataset *ds, const int32_t *rows, int64_t n_rows, const double *y,
                   const void *state, size_t state_bytes, const iht_options *opt,
                   double *beta_out, int32_t *support_out, iht_result *info);

/* One solve of a batch: its row set (a CV training fold, a phenotype's
 * non-missing subjects, a serving request's subset), phenotype and k. */
typedef struct iht_solve_desc {
    const int32_t *rows;   /* int32[n_rows] distinct subjects, or NULL = all n   */
    int64_t n_rows;        /* rows in use (n when rows is NULL)                  */
    const double *y;       /* double[n_rows], aligned with rows                  */
    int32_t k;             /* sparsity level, 1 <= k <= min(p, 1024)             */
    int32_t reserved;
} iht_solve_desc;

/* a2-a7 -- b IHT solves on one dataset that share every pass over the packed
 * genotypes (Sec. 2.4 model selection: q-fold cross-validation over a path of
 * model sizes fits many solves on the same matrix).  Each solve follows
 * iht_fit exactly (same readings, same statistics over its own rows); the
 * gradient of all active solves is one multi-right-hand-side pass per
 * iteration, and every other step runs batched.  Solves retire independently.
 *   solves  : host array of b descriptors (rows, y in opt->in_mem memory).
 *   betas   : double[b][p] dense coefficients (opt->out_mem memory) or NULL.
 *   supports: int32[sum of k] concatenated in solve order (opt->out_mem).
 *   beta_s  : double[sum of k] beta on each support, aligned with supports
 *             (opt->out_mem), or NULL.
 *   infos   : host iht_result[b], may be NULL; with opt->profile, grad_ms and
 *             grad_launches describe the batch's multi-column passes.
 * Returns OK, EINVAL, ENOMEM, ETIMEOUT, ECUDA; per-solve status (OK,
 * ENOTCONV, ENUMERIC) is in infos[c].status.  A solve whose y is not finite
 * stops before its first step: beta row 0, support entries -1.  Identical
 * row sets (same rows pointer and n_rows) share one set of statistics. */
int iht_fit_batch(iht_dataset *ds, int32_t b, const iht_solve_desc *solves,
                  const iht_options *opt, double *betas, int32_t *supports, double *beta_s,
                  iht_result *infos);

/* Model selection -- q-fold cross-validation over a path of model sizes, then
 * the refit (Sec. 2.4).  Every (partition, size) pair is one solve of a single
 * iht_fit_batch: partition f's path is fitted on the other partitions' rows
 * (statistics of those rows); its mean squared error is taken on partition
 * f's rows on the device, z standardised with the training rows' statistics;
 * the errors are averaged over the q partitions, the first size in ks with the
 * least average is chosen and the model is refitted on all labelled rows.
 *   y           : host double[n]
 *   fold        : host int32[n], subject i's partition in 0..q-1, or -1 for
 *                 a subject outside both the selection and the refit (a
 *                 held-out test set); every partition needs a row and its
 *                 complement among the labelled subjects at least 2
 *   q           : partitions, 2..64
 *   ks, nk      : host int32[nk] model sizes, each in 1..min(p, 1024)
 *   opt         : solver options (in_mem, out_mem ignored: host in and out)
 *   mse         : host double[nk] averaged out-of-fold MSE, or NULL
 *   mse_fold    : host double[q][nk] each partition's MSE, or NULL
 *   k_best      : host int32, the chosen size, or NULL
 *   beta_out    : host double[p] refit coefficients, or NULL
 *   support_out : host int32[k_best] refit support (capacity max ks), or NULL
 *   info        : host iht_result of the refit, or NULL
 * Returns the refit's status (OK or ENOTCONV), or EINVAL, ENOMEM, ENUMERIC
 * (non-finite y), ETIMEOUT, ECUDA. */
int iht_cv(iht_dataset *ds, const double *y, const int32_t *fold, int32_t q, const int32_t *ks,
           int32_t nk, const iht_options *opt, double *mse, double *mse_fold, int32_t *k_best,
           double *beta_out, int32_t *support_out, iht_result *info);

/* a7 -- multi-right-hand-side standardised gradient G = Z^T R for b residual
 * columns, each with its own row set and statistics (exposes the batched
 * gradient for tests).
 *   rows_list : host array of b device pointers (int32 row lists or NULL = all)
 *   n_rows    : host int64[b]
 *   R         : device float, column c at R + c * n (aligned with its rows)
 *   G_out     : device float[b][p]
 *   impl      : 0 default (tensor cores; a single column runs the single-column
 *               pass, which gives the same bits), 1 one CUDA-core pass per
 *               column, 2 the multi-column tensor-core pass always. */
int iht_gradient_batch(iht_dataset *ds, int32_t b, const int32_t *const *rows_list,
                       const int64_t *n_rows, const float *R, float *G_out, int impl);

/* Launch shapes of the gradient passes and their autotuner.
 *
 * The tensor-core gradient passes (Sec. 2.2's g = Z^T r, one or many residual
 * columns) have staging knobs that change how genotype and residual tiles are
 * buffered, never the arithmetic or its order, so every shape writes the same
 * bits.  The first pass of a kind on a dataset shape (device, padded samples,
 * SNPs; for the multi-column pass also the accumulator-width bucket, 16..64,
 * 80..96, 112..128, 144..192 or 208..224 accumulator columns, 5 per residual
 * column)
 * runs every candidate shape on its real inputs, timed with CUDA events, and
 * caches the fastest for the life of the process; later passes, including
 * those captured into CUDA graphs, use the cached shape.  A pass launched
 * while its stream is being captured, or with tuning off, uses the cached
 * shape or else a fixed default.
 *
 * kind IHT_PASS_SINGLE (one residual column), params[0]: TMA stages per
 * warpgroup, 2 .. as many as shared memory holds beside the residual image.
 * kind IHT_PASS_MULTI (ncols residual columns in one pass), params[0]:
 * genotype stages 2..8 (4 at most with 4 tiles); params[1]: 1 = each decoder
 * step fills a pair of A buffers (needs four or more buffers: 192
 * accumulator columns at most with 2 tiles, 64 with 4);
 * params[2]: 1 = missing-call finalisation over 8 columns per block (when
 * more than 4 columns and the 8-column residual table fits in shared
 * memory); params[3]: 1 = finalisation over the padded missing-call lists
 * (groups of 8 SNPs with common residue-class boundaries, built at upload
 * when n is at most about 12 800; ignored otherwise); params[4]: 128-SNP
 * tiles per step of a CTA, each with its own MMA-issuing warp: 2, or 4 for
 * accumulators of at most 96 columns (19 residual columns). */
enum { IHT_PASS_SINGLE = 0, IHT_PASS_MULTI = 1 };

/* Tuning on (default) or off; IHT_AUTOTUNE=0 in the environment starts it off. */
void iht_set_autotune(int on);

/* Forgets every cached shape. */
void iht_tune_clear(void);

/* Pins the shape of passes of `kind` over ncols columns on this dataset
 * (params: host int32[nparams], nparams 1 for SINGLE, 5 for MULTI).  EINVAL for
 * a shape that does not fit the pass or an unknown kind. */
int iht_tune_pin(const iht_dataset *ds, int32_t kind, int32_t ncols, const int32_t *params,
                 int32_t nparams);

/* Cached shape of passes of `kind` over ncols columns on this dataset into
 * params (host int32[nparams]); EAGAIN when none is cached yet. */
int iht_tune_query(const iht_dataset *ds, int32_t kind, int32_t ncols, int32_t *params,
                   int32_t nparams);

/* Text listing of the cache, one line per entry.  buf NULL: returns the bytes
 * needed (with the terminating 0); otherwise writes at most buf_bytes bytes
 * (truncated, 0-terminated) and returns OK. */
int iht_tuning_summary(char *buf, size_t buf_bytes);

/* a8 -- continuous-batching IHT server on one dataset.
 *
 * Requests (a phenotype, a subject subset and k: iht_solve_desc with host
 * pointers, copied at submission) arrive at any time.  A worker thread owned
 * by the server admits a pending request when a slot is free and its device
 * footprint (per-SNP statistics, gradient, residuals and scratch of one solve,
 * about 28 p + 56 n bytes plus about 130 kB) fits in hbm_budget, then runs
 * every admitted solve together: one iteration per tick, one multi-column
 * gradient pass over the packed genotypes for all active solves (each solve is
 * a column), the O(nk) steps batched.  A solve retires when it stops (same
 * rule as iht_fit) and frees its slot and memory for the next request.  Each
 * solve's arithmetic does not depend on which other solves share its ticks.
 * The paper fits one model at a time; this is the serving form of the batched
 * cross-validation above (Sec. 2.4 fits many models on one matrix). */
typedef struct iht_server iht_server;

typedef struct iht_server_options {
    int32_t max_slots;       /* solves on the device at once, 1..1024 (default 64)     */
    int32_t reserved;
    uint64_t hbm_budget;     /* device bytes for admitted solves; 0 = no limit         */
    iht_options solve;       /* per-solve options; in_mem, out_mem, profile ignored    */
} iht_server_options;

typedef struct iht_server_stats {
    uint64_t submitted, admitted, completed, ticks;
    int32_t active, max_active;              /* solves on the device now / at most   */
    uint64_t bytes_in_use, max_bytes_in_use; /* footprint of the admitted solves     */
} iht_server_stats;

void iht_server_default_options(iht_server_options *o);

/* Starts the worker on its own stream of the dataset's device.  The dataset
 * must outlive the server; other calls on the same dataset while a server is
 * running are not supported.  Returns OK, EINVAL, ENOMEM, ECUDA. */
int iht_server_create(iht_dataset *ds, const iht_server_options *opt, iht_server **out);

/* Queues one request (host rows or NULL for all n, host y).  EINVAL for k
 * outside 1..min(p, 1024), n_rows < 2, a request that can never fit the
 * budget, or a server whose worker has failed (then ECUDA). */
int iht_server_submit(iht_server *s, const iht_solve_desc *req, uint64_t *ticket);

/* Result of a finished request: support (int32[k], ascending), beta on it
 * (double[k]), info (info->status: OK, ENOTCONV, ENUMERIC for non-finite y,
 * EINVAL for bad rows) and the time from submission to retirement in
 * seconds; any output may be NULL.  Returns EAGAIN while the request is queued
 * or running, EINVAL for an unknown (or already collected) ticket, ECUDA if
 * the worker failed.  A collected result is released. */
int iht_server_poll(iht_server *s, uint64_t ticket, int32_t *support, double *beta_s,
                    iht_result *info, double *latency_s);

int iht_server_get_stats(iht_server *s, iht_server_stats *out);

/* Stops the worker after its current tick; requests not yet finished are
 * dropped.  Frees everything the server holds. */
int iht_server_destroy(iht_server *s);

#ifdef __cplusplus
}
#endif
#endif /* IHT_H */
