/*
 * FP64 CPU oracle for iterative hard thresholding (IHT) least squares on
 * PLINK-packed genotypes -- Keys, Chen & Lange, "Iterative Hard Thresholding
 * for Model Selection in Genome-Wide Association Studies".
 *
 * TEST INFRASTRUCTURE.  This file is the plain, slow, obviously correct
 * statement of what the GPU path computes.  Only the tests, the smoke check
 * and the bench's CPU-baseline / reference arm may load it.  It shares no code,
 * header, table or constant with the CUDA library, and the CUDA library never
 * calls it.
 *
 * Every quantity is FP64.  Nothing is blocked, fused or reordered beyond the
 * definitions cited at each function.  OpenMP only splits independent SNP
 * columns of the dense gradient (the paper's multicore column split, Sec.
 * 2.3.3); each column's sum runs in sample order on one thread, so results do
 * not depend on the thread count.
 *
 * Readings of the paper fixed here (each also listed in the design notes):
 *  R1 step size: mu = ||g_S||^2 / ||Z_S g_S||^2 (normalized IHT, Sec. 2.3.1;
 *     the printed ||beta||^2/||X beta||^2 is 0/0 at beta = 0).  S^0 = top-k of
 *     |Z^T y|.  ||Z_S g_S|| = 0 with g_S != 0 -> ENUMERIC; g_S = 0 -> converged.
 *  R2 omega = (1-c) ||beta+ - beta||^2 / ||Z (beta+ - beta)||^2 (Sec. 2.3.1,
 *     parentheses garbled in print).
 *  R3 c = 0.01, kappa = 2 (mu <- mu/kappa), at most 50 shrinks; the check is
 *     applied only when the support changes; after the last shrink the
 *     candidate is taken as it is.
 *  R4 accept iff mu < omega (strict, Sec. 2.3.1).  ||Z d|| = 0 -> accept.
 *  R5 projection P_{S_k} (Eq. ihta): order by |w| descending, then index
 *     ascending; S always has k indices.
 *  R6 converged iff ||beta+ - beta||_2 / (||beta||_2 + 1) < tol.
 *  R7 per-SNP mean u over observed calls, variance with an (n_obs - 1)
 *     denominator, v = 1/sqrt(var); v = 0 when var = 0 or n_obs < 2.
 *  R8 statistics over the rows the solve uses.
 *  R9 code 00 = hom-ref (dosage 0), 01 = missing, 10 = het (1), 11 = hom-alt (2).
 *  R10 standardised dosage z = v (x - u) on observed calls, 0 on missing
 *     (Sec. 3.1 standardises the observed dosages and zeroes the missing
 *     ones; this equals the identity of Sec. 2.3.2 on mean-imputed
 *     genotypes).
 *  R11 HTP (Sec. 2.2: the projection solves the normal equations on the
 *     active set).  After a least-squares refit g vanishes on S, so the
 *     normalized step over S is 0/0; the step is taken over Gamma = the k
 *     largest |g_j| (ties to the lower index): mu = ||g_G||^2 / ||Z_G g_G||^2
 *     (at beta = 0, Gamma = S^0, so the first step is IHT's).  The
 *     backtracking check of R2-R4 applies to the projected candidate
 *     P_{S_k}(beta + mu g); the accepted support S+ is then refitted:
 *     beta+ = argmin ||y - Z_{S+} b||^2 by the normal equations (Eq.
 *     normal_equations).
 *  R12 the normal equations are solved by Cholesky in the ascending index
 *     order of S+; a column whose pivot is <= 1e-10 times its diagonal entry
 *     (a zero column, or one dependent on earlier columns of S+) gets
 *     coefficient 0 and leaves the solve.
 *  R13 nongenetic covariates (Sec. 3: p counts genetic predictors and
 *     covariates, k_best includes covariates): q dense columns appended as
 *     predictors p .. p+q-1, standardised like the SNPs over the used rows
 *     (mean, (n_rows - 1) denominator, v = 0 for a constant column) and
 *     subject to the same projection, so they count toward k.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2, OR_ENOTCONV = 3, OR_ENUMERIC = 4 };

typedef struct {
    int32_t max_iter;      /* iteration cap                            */
    int32_t max_backtrack; /* cap on step shrinks per iteration (R3)    */
    double tol;            /* convergence tolerance (R6)               */
    double c;              /* omega constant 0 < c << 1 (R2)           */
    double kappa;          /* shrink factor (R3)                       */
    int32_t variant;       /* 0 IHT, 1 HTP (R11)                        */
    int32_t pad;
} oracle_opts;

enum { OR_IHT = 0, OR_HTP = 1 };

typedef struct {
    int32_t iterations;    /* updates performed                        */
    int32_t status;        /* OR_*                                     */
    int32_t backtracks;    /* total shrinks                            */
    int32_t pad;
    double objective;      /* 1/2 ||y - Z beta||^2 at exit              */
    double mu;             /* last accepted step size                   */
} oracle_info;

/* Per-iteration record; every pointer may be NULL.  Arrays have max_iter
 * entries (supp/beta: max_iter * k). */
typedef struct {
    double *objective;     /* f after the update                        */
    double *mu;            /* accepted step size                         */
    double *omega;         /* last omega evaluated (NAN if none)         */
    int32_t *backtracks;   /* shrinks in this iteration                  */
    int32_t *changed;      /* support changed by the accepted update     */
    double *gap;           /* |w|_(k) - |w|_(k+1) of the accepted selection */
    double *wscale;        /* mu * max_j |g_j| of the accepted selection  */
    double *margin;        /* min over omega checks of |mu - omega| / omega */
    double *step;          /* ||beta+ - beta|| / (||beta|| + 1)           */
    int32_t *supp;         /* accepted support, ascending (k per iter)   */
    double *beta;          /* beta on that support (k per iter)          */
} oracle_trace;

/* ---------------------------------------------------------------------- */
/* Genotype access: PLINK .bed SNP-major 2-bit codes (Sec. 2.3.2).  Sample i
 * of SNP j is bits 2(i mod 4)..2(i mod 4)+1 of byte floor(i/4) of row j.    */
static inline int bed_code(const uint8_t *body, int64_t row_bytes, int64_t j, int64_t i)
{
    return (body[j * row_bytes + (i >> 2)] >> (2 * (i & 3))) & 3;
}

/* Dosage of a code (R9); returns -1 for missing. */
static inline int code_dosage(int code)
{
    switch (code) {
    case 0: return 0;
    case 2: return 1;
    case 3: return 2;
    default: return -1;
    }
}

/* Standardised genotype z_ij (R10; Sec. 2.3.2 identity, Sec. 3.1). */
static inline double zval(const uint8_t *body, int64_t rb, int64_t j, int64_t i,
                          const double *u, const double *v)
{
    int x = code_dosage(bed_code(body, rb, j, i));
    if (x < 0) return 0.0;
    return v[j] * ((double)x - u[j]);
}

static inline int64_t row_of(const int64_t *rows, int64_t a) { return rows ? rows[a] : a; }

void oracle_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* codes[j*n + i] for every SNP and sample (Sec. 2.3.2 packing). */
int oracle_decode(const uint8_t *body, int64_t row_bytes, int64_t n, int64_t p, int8_t *codes)
{
    if (!body || !codes || n < 0 || p < 0 || row_bytes < (n + 3) / 4) return OR_EINVAL;
    for (int64_t j = 0; j < p; ++j)
        for (int64_t i = 0; i < n; ++i)
            codes[j * n + i] = (int8_t)bed_code(body, row_bytes, j, i);
    return OR_OK;
}

/* Per-SNP code counts over the used rows and the statistics of R7
 * (mean and inverse SD vectors u, v of Sec. 2.3.2).
 * counts[4j + c] = number of used rows with code c. */
int oracle_counts(const uint8_t *body, int64_t row_bytes, int64_t n, int64_t p,
                  const int64_t *rows, int64_t n_rows, int32_t *counts, double *u, double *v)
{
    if (!body || n < 0 || p < 0 || row_bytes < (n + 3) / 4 || n_rows < 0) return OR_EINVAL;
    if (!rows && n_rows != n) return OR_EINVAL;
    for (int64_t a = 0; rows && a < n_rows; ++a)
        if (rows[a] < 0 || rows[a] >= n) return OR_EINVAL;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < p; ++j) {
        int64_t cnt[4] = {0, 0, 0, 0};
        for (int64_t a = 0; a < n_rows; ++a) cnt[bed_code(body, row_bytes, j, row_of(rows, a))]++;
        if (counts)
            for (int c = 0; c < 4; ++c) counts[4 * j + c] = (int32_t)cnt[c];
        const double n_obs = (double)(n_rows - cnt[1]);
        const double s1 = (double)(cnt[2] + 2 * cnt[3]);
        const double s2 = (double)(cnt[2] + 4 * cnt[3]);
        double mean = n_obs > 0 ? s1 / n_obs : 0.0;
        double inv_sd = 0.0;
        if (n_obs >= 2) {
            double var = (s2 - s1 * s1 / n_obs) / (n_obs - 1.0);
            if (var > 0) inv_sd = 1.0 / sqrt(var);
        }
        if (u) u[j] = mean;
        if (v) v[j] = inv_sd;
    }
    return OR_OK;
}

/* Negative gradient g = Z^T r (Eq. normal_grad, g = -grad f), r indexed like
 * rows.  One column per loop trip, samples in order. */
int oracle_gradient(const uint8_t *body, int64_t row_bytes, int64_t n, int64_t p,
                    const int64_t *rows, int64_t n_rows, const double *u, const double *v,
                    const double *r, double *g)
{
    if (!body || !u || !v || !r || !g || (!rows && n_rows != n)) return OR_EINVAL;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < p; ++j) {
        double acc = 0.0;
        for (int64_t a = 0; a < n_rows; ++a)
            acc += zval(body, row_bytes, j, row_of(rows, a), u, v) * r[a];
        g[j] = acc;
    }
    return OR_OK;
}

/* out = Z[:, cols] coef over the used rows (the sparse product X_k beta_k of
 * Sec. 2.3.2-2.3.3, with the standardisation identity applied per entry). */
int oracle_zmul(const uint8_t *body, int64_t row_bytes, int64_t n, const int64_t *rows,
                int64_t n_rows, const double *u, const double *v, const int32_t *cols,
                int32_t m, const double *coef, double *out)
{
    if (!body || !u || !v || !out || (m > 0 && (!cols || !coef)) || (!rows && n_rows != n))
        return OR_EINVAL;
    for (int64_t a = 0; a < n_rows; ++a) {
        double acc = 0.0;
        for (int32_t c = 0; c < m; ++c)
            acc += zval(body, row_bytes, cols[c], row_of(rows, a), u, v) * coef[c];
        out[a] = acc;
    }
    return OR_OK;
}

/* ---------------------------------------------------------------------- */
/* Projection onto the k-sparse set (Eq. ihta, R5): full sort of all indices
 * by (|w| descending, index ascending), keep the first k. */
static const double *g_sort_w;

static int cmp_abs_desc(const void *pa, const void *pb)
{
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    double fa = fabs(g_sort_w[a]), fb = fabs(g_sort_w[b]);
    if (fa > fb) return -1;
    if (fa < fb) return 1;
    return (a > b) - (a < b);
}

static int cmp_i32(const void *pa, const void *pb)
{
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    return (a > b) - (a < b);
}

/* order: int32[p] scratch.  idx_out: the k selected indices in selection
 * order.  Returns |w|_(k) - |w|_(k+1) through *gap (+inf when k == p). */
static void topk_sorted(const double *w, int64_t p, int32_t k, int32_t *order, int32_t *idx_out,
                        double *gap)
{
    for (int64_t j = 0; j < p; ++j) order[j] = (int32_t)j;
    g_sort_w = w;
    qsort(order, (size_t)p, sizeof(int32_t), cmp_abs_desc);
    memcpy(idx_out, order, sizeof(int32_t) * (size_t)k);
    if (gap) *gap = (k < p) ? fabs(w[order[k - 1]]) - fabs(w[order[k]]) : INFINITY;
}

int oracle_topk(const double *w, int64_t p, int32_t k, int32_t *idx_out)
{
    if (!w || !idx_out || k < 1 || k > p) return OR_EINVAL;
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)p);
    if (!order) return OR_ENOMEM;
    topk_sorted(w, p, k, order, idx_out, NULL);
    free(order);
    return OR_OK;
}

/* ---------------------------------------------------------------------- */
static double sumsq(const double *x, int64_t m)
{
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) s += x[i] * x[i];
    return s;
}

/* Covariate statistics over the used rows (R13): cov[t*n + i] is covariate t
 * of subject i; mean cu[t] and inverse SD cv[t] with an (n_rows - 1)
 * denominator (cv = 0 for a constant column or n_rows < 2). */
int oracle_cov_stats(const double *cov, int64_t n, int64_t q, const int64_t *rows, int64_t n_rows,
                     double *cu, double *cv)
{
    if ((q > 0 && (!cov || !cu || !cv)) || n_rows < 0 || (!rows && n_rows != n)) return OR_EINVAL;
    for (int64_t t = 0; t < q; ++t) {
        const double *c = cov + t * n;
        double m = 0.0;
        for (int64_t a = 0; a < n_rows; ++a) m += c[row_of(rows, a)];
        m = n_rows > 0 ? m / (double)n_rows : 0.0;
        double ss = 0.0;
        for (int64_t a = 0; a < n_rows; ++a) {
            const double d = c[row_of(rows, a)] - m;
            ss += d * d;
        }
        double inv_sd = 0.0;
        if (n_rows >= 2) {
            const double var = ss / (double)(n_rows - 1);
            if (var > 0) inv_sd = 1.0 / sqrt(var);
        }
        cu[t] = m;
        cv[t] = inv_sd;
    }
    return OR_OK;
}

/* The design of one solve: SNP predictors 0..p-1 (R10) and covariate
 * predictors p..p+q-1 (R13), over the used rows. */
typedef struct {
    const uint8_t *body;
    int64_t rb, n, p;
    const int64_t *rows;
    int64_t n_rows;
    const double *u, *v;         /* SNP statistics */
    const double *cov;           /* q x n, may be NULL when q = 0 */
    int64_t q;
    const double *cu, *cv;       /* covariate statistics */
} design;

/* Standardised predictor j at used row a. */
static inline double pred(const design *D, int64_t j, int64_t a)
{
    if (j < D->p) return zval(D->body, D->rb, j, row_of(D->rows, a), D->u, D->v);
    const int64_t t = j - D->p;
    return D->cv[t] * (D->cov[t * D->n + row_of(D->rows, a)] - D->cu[t]);
}

/* g = Z^T r over all p + q predictors (Eq. normal_grad). */
static void design_gradient(const design *D, const double *r, double *g)
{
    oracle_gradient(D->body, D->rb, D->n, D->p, D->rows, D->n_rows, D->u, D->v, r, g);
    for (int64_t t = 0; t < D->q; ++t) {
        double acc = 0.0;
        for (int64_t a = 0; a < D->n_rows; ++a) acc += pred(D, D->p + t, a) * r[a];
        g[D->p + t] = acc;
    }
}

/* out = Z[:, cols] coef over the used rows (columns in the given order). */
static void design_zmul(const design *D, const int32_t *cols, int32_t m, const double *coef,
                        double *out)
{
    for (int64_t a = 0; a < D->n_rows; ++a) {
        double acc = 0.0;
        for (int32_t c = 0; c < m; ++c) acc += pred(D, cols[c], a) * coef[c];
        out[a] = acc;
    }
}

/* Least squares on the columns S (k, ascending) by the normal equations
 * (Eq. normal_equations, R12): G = Z_S^T Z_S, h = Z_S^T y, Cholesky
 * G = L L^T in the order of S; a column whose pivot is <= 1e-10 G_aa is
 * dependent (or zero): its row of L is zero and its coefficient 0.
 * zs: k * n_rows scratch, L: k * k scratch. */
static void refit_ls(const design *D, const int32_t *S, int32_t k, const double *y, double *b,
                     double *zs, double *L, double *h)
{
    const int64_t nr = D->n_rows;
    for (int32_t c = 0; c < k; ++c)
        for (int64_t a = 0; a < nr; ++a) zs[(int64_t)c * nr + a] = pred(D, S[c], a);
    for (int32_t i = 0; i < k; ++i) {
        double acc = 0.0;
        for (int64_t a = 0; a < nr; ++a) acc += zs[(int64_t)i * nr + a] * y[a];
        h[i] = acc;
    }
    for (int32_t i = 0; i < k; ++i) {
        for (int32_t j = 0; j <= i; ++j) {
            double gij = 0.0;
            for (int64_t a = 0; a < nr; ++a) gij += zs[(int64_t)i * nr + a] * zs[(int64_t)j * nr + a];
            double sdot = 0.0;
            for (int32_t t = 0; t < j; ++t) sdot += L[(int64_t)i * k + t] * L[(int64_t)j * k + t];
            if (j < i) {
                const double ljj = L[(int64_t)j * k + j];
                L[(int64_t)i * k + j] = ljj > 0.0 ? (gij - sdot) / ljj : 0.0;
            } else {
                const double d = gij - sdot;
                L[(int64_t)i * k + i] = d > 1e-10 * gij ? sqrt(d) : 0.0;
                if (!(d > 1e-10 * gij))
                    for (int32_t t = 0; t < i; ++t) L[(int64_t)i * k + t] = 0.0;
            }
        }
        for (int32_t j = i + 1; j < k; ++j) L[(int64_t)i * k + j] = 0.0;
    }
    /* L z = h, then L^T b = z; dependent columns (zero pivot) take 0 */
    for (int32_t i = 0; i < k; ++i) {
        const double lii = L[(int64_t)i * k + i];
        double acc = h[i];
        for (int32_t t = 0; t < i; ++t) acc -= L[(int64_t)i * k + t] * b[t];
        b[i] = lii > 0.0 ? acc / lii : 0.0;
    }
    for (int32_t i = k - 1; i >= 0; --i) {
        const double lii = L[(int64_t)i * k + i];
        double acc = b[i];
        for (int32_t t = i + 1; t < k; ++t) acc -= L[(int64_t)t * k + i] * b[t];
        b[i] = lii > 0.0 ? acc / lii : 0.0;
    }
}

/*
 * IHT least squares (Eq. leastsquaresloss, Eq. ihta, Sec. 2.3.1):
 *   beta^0 = 0, r^0 = y, S^0 = top-k |Z^T y|.
 *   repeat: g = Z^T r;  mu = ||g_S||^2 / ||Z_S g_S||^2;
 *           w = beta + mu g;  S+ = top-k |w|;  beta+ = w on S+;
 *           if S+ != S and mu >= omega: mu <- mu / kappa, recompute w, S+, beta+;
 *           r+ = y - Z_{S+} beta+;  stop when ||beta+ - beta|| / (||beta|| + 1) < tol.
 * HTP (opt->variant = OR_HTP, R11-R12): mu over Gamma = top-k |g|, and the
 * accepted S+ is refitted by least squares before r+.
 * Predictors: the p SNPs, then the q covariates of cov (q x n, may be NULL
 * when q = 0; R13).  y has n_rows entries aligned with rows (rows == NULL: all
 * n subjects).  beta_out: p + q doubles; support_out: k indices ascending.
 */
int oracle_iht(const uint8_t *body, int64_t row_bytes, int64_t n, int64_t p, const int64_t *rows,
               int64_t n_rows, const double *y, int32_t k, const oracle_opts *opt,
               const double *cov, int64_t q, double *beta_out, int32_t *support_out,
               oracle_info *info, oracle_trace *tr)
{
    const int64_t P = p + q;
    if (!body || !y || !opt || !beta_out || !support_out || n < 1 || p < 1 || q < 0 ||
        (q > 0 && !cov) || k < 1 || k > P || n_rows < 2 || row_bytes < (n + 3) / 4 ||
        (!rows && n_rows != n) || opt->max_iter < 0 || opt->kappa <= 1.0 || opt->c < 0 ||
        opt->c >= 1 || opt->max_backtrack < 0 || (opt->variant != OR_IHT && opt->variant != OR_HTP))
        return OR_EINVAL;
    for (int64_t a = 0; a < n_rows; ++a)
        if (!isfinite(y[a])) return OR_ENUMERIC;
    for (int64_t a = 0; a < q * n; ++a)
        if (!isfinite(cov[a])) return OR_ENUMERIC;

    const int htp = opt->variant == OR_HTP;
    int status = OR_ENOTCONV;
    double *u = malloc(sizeof(double) * p), *v = malloc(sizeof(double) * p);
    double *cu = malloc(sizeof(double) * (q + 1)), *cv = malloc(sizeof(double) * (q + 1));
    double *g = malloc(sizeof(double) * P), *w = malloc(sizeof(double) * P);
    double *beta = calloc((size_t)P, sizeof(double)), *bplus = calloc((size_t)P, sizeof(double));
    double *r = malloc(sizeof(double) * n_rows), *zv = malloc(sizeof(double) * n_rows);
    int32_t *order = malloc(sizeof(int32_t) * P);
    int32_t *S = malloc(sizeof(int32_t) * k), *Sp = malloc(sizeof(int32_t) * k);
    int32_t *uni = malloc(sizeof(int32_t) * 2 * (size_t)k);
    double *coef = malloc(sizeof(double) * 2 * (size_t)k);
    uint8_t *inS = calloc((size_t)P, 1);
    int32_t *gam = htp ? malloc(sizeof(int32_t) * k) : NULL;
    double *zs = htp ? malloc(sizeof(double) * (size_t)k * n_rows) : NULL;
    double *Lm = htp ? malloc(sizeof(double) * (size_t)k * k) : NULL;
    double *hv = htp ? malloc(sizeof(double) * k) : NULL;
    double *bls = htp ? malloc(sizeof(double) * k) : NULL;
    if (!u || !v || !cu || !cv || !g || !w || !beta || !bplus || !r || !zv || !order || !S ||
        !Sp || !uni || !coef || !inS || (htp && (!gam || !zs || !Lm || !hv || !bls))) {
        status = OR_ENOMEM;
        goto done;
    }

    oracle_counts(body, row_bytes, n, p, rows, n_rows, NULL, u, v);
    oracle_cov_stats(cov, n, q, rows, n_rows, cu, cv);
    const design D = {body, row_bytes, n, p, rows, n_rows, u, v, cov, q, cu, cv};

    /* beta^0 = 0, r^0 = y, S^0 = top-k of |g^0| (R1). */
    memcpy(r, y, sizeof(double) * n_rows);
    design_gradient(&D, r, g);
    topk_sorted(g, P, k, order, S, NULL);
    qsort(S, (size_t)k, sizeof(int32_t), cmp_i32);
    double f = 0.5 * sumsq(r, n_rows);
    double mu = 0.0;
    int32_t it = 0, total_bt = 0;

    for (it = 0; it < opt->max_iter; ++it) {
        if (it > 0) design_gradient(&D, r, g);

        /* Normalized step size (R1); HTP over the k largest |g| (R11). */
        const int32_t *stepset = S;
        if (htp) {
            topk_sorted(g, P, k, order, gam, NULL);
            qsort(gam, (size_t)k, sizeof(int32_t), cmp_i32);
            stepset = gam;
        }
        for (int32_t c = 0; c < k; ++c) coef[c] = g[stepset[c]];
        double num = sumsq(coef, k);
        if (num == 0.0) { status = OR_OK; break; }
        design_zmul(&D, stepset, k, coef, zv);
        double den = sumsq(zv, n_rows);
        if (!(den > 0.0) || !isfinite(num) || !isfinite(den)) { status = OR_ENUMERIC; break; }
        mu = num / den;

        int32_t bt = 0, changed = 0;
        double omega = NAN, margin = INFINITY, gap = 0.0, gmax = 0.0;
        for (int64_t j = 0; j < P; ++j) gmax = fmax(gmax, fabs(g[j]));
        for (;;) {
            for (int64_t j = 0; j < P; ++j) w[j] = beta[j] + mu * g[j];
            topk_sorted(w, P, k, order, Sp, &gap);
            qsort(Sp, (size_t)k, sizeof(int32_t), cmp_i32);
            memset(bplus, 0, sizeof(double) * P);
            for (int32_t c = 0; c < k; ++c) bplus[Sp[c]] = w[Sp[c]];
            changed = memcmp(S, Sp, sizeof(int32_t) * k) != 0;
            if (!changed) break;
            /* Backtracking check on d = beta+ - beta over S u S+ (R2-R4). */
            int32_t m = 0;
            for (int32_t c = 0; c < k; ++c) { inS[S[c]] = 1; uni[m] = S[c]; coef[m] = bplus[S[c]] - beta[S[c]]; ++m; }
            for (int32_t c = 0; c < k; ++c)
                if (!inS[Sp[c]]) { uni[m] = Sp[c]; coef[m] = bplus[Sp[c]] - beta[Sp[c]]; ++m; }
            for (int32_t c = 0; c < k; ++c) inS[S[c]] = 0;
            double dd = sumsq(coef, m);
            design_zmul(&D, uni, m, coef, zv);
            double zz = sumsq(zv, n_rows);
            if (!(zz > 0.0)) { omega = INFINITY; break; }
            omega = (1.0 - opt->c) * dd / zz;
            margin = fmin(margin, fabs(mu - omega) / omega);
            if (mu < omega || bt >= opt->max_backtrack) break;
            mu /= opt->kappa;
            ++bt;
        }
        total_bt += bt;

        /* HTP: least squares on the accepted support (R11, R12). */
        if (htp) {
            refit_ls(&D, Sp, k, y, bls, zs, Lm, hv);
            memset(bplus, 0, sizeof(double) * P);
            for (int32_t c = 0; c < k; ++c) bplus[Sp[c]] = bls[c];
        }

        /* Residual from scratch and objective (Eq. leastsquaresloss). */
        for (int32_t c = 0; c < k; ++c) coef[c] = bplus[Sp[c]];
        design_zmul(&D, Sp, k, coef, zv);
        for (int64_t a = 0; a < n_rows; ++a) r[a] = y[a] - zv[a];
        f = 0.5 * sumsq(r, n_rows);

        double dn = 0.0, bn = 0.0;
        for (int64_t j = 0; j < P; ++j) {
            double d = bplus[j] - beta[j];
            dn += d * d;
            bn += beta[j] * beta[j];
        }
        double step = sqrt(dn) / (sqrt(bn) + 1.0);
        memcpy(beta, bplus, sizeof(double) * P);
        memcpy(S, Sp, sizeof(int32_t) * k);

        if (tr) {
            if (tr->objective) tr->objective[it] = f;
            if (tr->mu) tr->mu[it] = mu;
            if (tr->omega) tr->omega[it] = omega;
            if (tr->backtracks) tr->backtracks[it] = bt;
            if (tr->changed) tr->changed[it] = changed;
            if (tr->gap) tr->gap[it] = gap;
            if (tr->wscale) tr->wscale[it] = mu * gmax;
            if (tr->margin) tr->margin[it] = margin;
            if (tr->step) tr->step[it] = step;
            if (tr->supp) memcpy(tr->supp + (size_t)it * k, S, sizeof(int32_t) * k);
            if (tr->beta)
                for (int32_t c = 0; c < k; ++c) tr->beta[(size_t)it * k + c] = beta[S[c]];
        }
        if (step < opt->tol) { status = OR_OK; ++it; break; }
    }

    memcpy(beta_out, beta, sizeof(double) * P);
    memcpy(support_out, S, sizeof(int32_t) * k);
    if (info) {
        info->iterations = it;
        info->status = status;
        info->backtracks = total_bt;
        info->objective = f;
        info->mu = mu;
    }

done:
    free(u); free(v); free(cu); free(cv); free(g); free(w); free(beta); free(bplus); free(r);
    free(zv); free(order); free(S); free(Sp); free(uni); free(coef); free(inS); free(gam);
    free(zs); free(Lm); free(hv); free(bls);
    return status;
}
