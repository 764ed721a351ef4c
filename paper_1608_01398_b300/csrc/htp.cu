// Nongenetic covariates and the least-squares refit of HTP.
//
// Covariates (Sec. 3: the predictors are the SNPs and the covariates, and a
// model size counts both): q dense columns stored beside the packed matrix,
// standardised over the rows of the solve (mean, (n_rows - 1) denominator,
// inverse SD 0 for a constant column) into zc, and appended to the gradient as
// entries p .. p+q-1 of g, so the projection selects among p + q predictors.
//
// HTP (Sec. 2.2: the projection solves the normal equations, Eq.
// normal_equations, on the active set): the accepted support S+ is refitted by
// least squares.  The k standardised columns of S+ are formed once (FP64), the
// Gram matrix Z_S^T Z_S and Z_S^T y by fixed-order block sums, and the k x k
// system is solved by a Cholesky factorisation in the ascending index order of
// S+; a column whose pivot is at most 1e-10 times its diagonal entry (a zero
// column, or one that depends on earlier columns of S+) gets coefficient 0.
#include <math.h>

#include "common.cuh"

namespace iht {

// Mean, inverse SD and standardised values of each covariate over the used
// rows (one block per covariate); a non-finite value on a used row sets
// err bit 0 of the solve.
__global__ void __launch_bounds__(256) k_cov_setup(const double *__restrict__ cov, int64_t n_pad,
                                                   const int32_t *__restrict__ used, int64_t n_rows,
                                                   double *__restrict__ cu, double *__restrict__ cv,
                                                   double *__restrict__ zc, Scalars *sc)
{
    __shared__ double red[8];
    const int t = blockIdx.x;
    const double *c = cov + (int64_t)t * n_pad;
    double s = 0.0;
    bool bad = false;
    for (int64_t i = threadIdx.x; i < n_pad; i += blockDim.x)
        if (used[i]) {
            s += c[i];
            bad |= !isfinite(c[i]);
        }
    if (bad) atomicOr(&sc->err, 1);
    s = block_sum(s, red);
    const double m = s / (double)n_rows;
    double ss = 0.0;
    for (int64_t i = threadIdx.x; i < n_pad; i += blockDim.x)
        if (used[i]) {
            const double d = c[i] - m;
            ss += d * d;
        }
    ss = block_sum(ss, red);
    double inv_sd = 0.0;
    if (n_rows >= 2) {
        const double var = ss / (double)(n_rows - 1);
        if (var > 0.0) inv_sd = 1.0 / sqrt(var);
    }
    for (int64_t i = threadIdx.x; i < n_pad; i += blockDim.x)
        zc[(int64_t)t * n_pad + i] = used[i] ? inv_sd * (c[i] - m) : 0.0;
    if (threadIdx.x == 0) {
        cu[t] = m;
        cv[t] = inv_sd;
    }
}

// g[p + t] = sum_i zc_t,i r_i (FP64 sum, one block per covariate).
// (hist: also its key into the selection's histogram, as the SNPs' pass does)
__global__ void __launch_bounds__(256) k_cov_grad(const double *__restrict__ zc, int64_t n_pad,
                                                  const float *__restrict__ r32, float *__restrict__ g,
                                                  int64_t p, const int32_t *__restrict__ done,
                                                  uint32_t *hist, uint32_t *hflag)
{
    __shared__ double red[8];
    if (done && *done) return;
    const int t = blockIdx.x;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n_pad; i += blockDim.x)
        s += zc[(int64_t)t * n_pad + i] * (double)r32[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
        const float gv = (float)s;
        g[p + t] = gv;
        if (hist) {
            const uint32_t key = __float_as_uint(gv) & 0x7fffffffu;
            if (key > 0x7f800000u) atomicOr(hflag, 1u);
            atomicAdd(&hist[key >> 20], 1u);
        }
    }
}

int cov_setup(iht_dataset *ds, int64_t n_rows)
{
    if (ds->q <= 0) return IHT_OK;
    Workspace *ws = ds->ws;
    if (!ws->zc) {
        IHT_CUDA(dev_malloc(&ws->cu64, sizeof(double) * kMaxCov));
        IHT_CUDA(dev_malloc(&ws->cv64, sizeof(double) * kMaxCov));
        IHT_CUDA(dev_malloc(&ws->zc, sizeof(double) * kMaxCov * (size_t)ds->n_pad));
    }
    k_cov_setup<<<(int)ds->q, 256, 0, ds->ctx->stream>>>(ds->cov, ds->n_pad, ws->used, n_rows,
                                                        ws->cu64, ws->cv64, ws->zc, ws->sc);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

int launch_cov_grad(iht_dataset *ds, const float *r32, float *g, const int32_t *done, uint32_t *hist,
                    uint32_t *hflag)
{
    if (ds->q <= 0) return IHT_OK;
    k_cov_grad<<<(int)ds->q, 256, 0, ds->ctx->stream>>>(ds->ws->zc, ds->n_pad, r32, g, ds->p, done,
                                                       hist, hflag);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

// ---------------------------------------------------------------------------
// HTP refit.

// zs[c][i] = standardised predictor S[c] at sample i on the used rows, else 0.
__global__ void k_htp_cols(const uint8_t *__restrict__ G, int64_t stride, const int32_t *__restrict__ S,
                           const double *__restrict__ u64, const double *__restrict__ v64,
                           const double *__restrict__ zc, int64_t p, const int32_t *__restrict__ used,
                           int64_t n_pad, double *__restrict__ zs, const int32_t *__restrict__ done)
{
    if (done && *done) return;
    const int c = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pad) return;
    const int64_t j = S[c];
    double z = 0.0;
    if (used[i]) {
        if (j < p) {
            const uint32_t code = (G[j * stride + (i >> 2)] >> (2 * (int)(i & 3))) & 3u;
            if (code != 1u) {
                const double x = code == 0u ? 0.0 : (code == 2u ? 1.0 : 2.0);
                z = v64[j] * (x - u64[j]);
            }
        } else {
            z = zc[(j - p) * n_pad + i];
        }
    }
    zs[(int64_t)c * n_pad + i] = z;
}

// gram[a][b] = zs_a . zs_b for b <= a (blockIdx.y = b), h[a] = zs_a . y (b = k).
__global__ void __launch_bounds__(256) k_htp_gram(const double *__restrict__ zs, const double *__restrict__ y,
                                                  int k, int64_t n_pad, double *__restrict__ gram,
                                                  double *__restrict__ h, const int32_t *__restrict__ done)
{
    __shared__ double red[8];
    if (done && *done) return;
    const int a = blockIdx.x, b = blockIdx.y;
    if (b < k && b > a) return;
    const double *x = zs + (int64_t)a * n_pad;
    const double *z = b == k ? y : zs + (int64_t)b * n_pad;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n_pad; i += blockDim.x) s += x[i] * z[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
        if (b == k)
            h[a] = s;
        else
            gram[(int64_t)a * k + b] = s;
    }
}

// Cholesky L L^T = gram (lower triangle, columns left to right; a pivot
// <= 1e-10 gram_jj makes column j dependent: its row of L is zero), then
// L z = h and L^T b = z with b_j = 0 for dependent j.  One block.
__global__ void __launch_bounds__(1024) k_htp_solve(const double *__restrict__ gram,
                                                    const double *__restrict__ h, int k,
                                                    double *__restrict__ L, double *__restrict__ b,
                                                    const int32_t *__restrict__ done)
{
    if (done && *done) return;
    for (int j = 0; j < k; ++j) {
        if (threadIdx.x == 0) {
            const double gjj = gram[(int64_t)j * k + j];
            double sdot = 0.0;
            for (int t = 0; t < j; ++t) sdot += L[(int64_t)j * k + t] * L[(int64_t)j * k + t];
            const double d = gjj - sdot;
            const bool ok = d > 1e-10 * gjj;
            L[(int64_t)j * k + j] = ok ? sqrt(d) : 0.0;
            if (!ok)
                for (int t = 0; t < j; ++t) L[(int64_t)j * k + t] = 0.0;
        }
        __syncthreads();
        const double ljj = L[(int64_t)j * k + j];
        for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) {
            double sdot = 0.0;
            for (int t = 0; t < j; ++t) sdot += L[(int64_t)i * k + t] * L[(int64_t)j * k + t];
            L[(int64_t)i * k + j] = ljj > 0.0 ? (gram[(int64_t)i * k + j] - sdot) / ljj : 0.0;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < k; ++i) {
            const double lii = L[(int64_t)i * k + i];
            double acc = h[i];
            for (int t = 0; t < i; ++t) acc -= L[(int64_t)i * k + t] * b[t];
            b[i] = lii > 0.0 ? acc / lii : 0.0;
        }
        for (int i = k - 1; i >= 0; --i) {
            const double lii = L[(int64_t)i * k + i];
            double acc = b[i];
            for (int t = i + 1; t < k; ++t) acc -= L[(int64_t)t * k + i] * b[t];
            b[i] = lii > 0.0 ? acc / lii : 0.0;
        }
    }
}

int ensure_htp_scratch(iht_dataset *ds, int k)
{
    Workspace *ws = ds->ws;
    if (ws->htp_k >= k) return IHT_OK;
    void *ptrs[] = {ws->gam, ws->zs, ws->gram, ws->chol, ws->hvec};
    for (void *x : ptrs)
        if (x) cudaFree(x);
    ws->gam = nullptr;
    ws->zs = ws->gram = ws->chol = ws->hvec = nullptr;
    ws->htp_k = 0;
    IHT_CUDA(dev_malloc(&ws->gam, sizeof(int32_t) * k));
    IHT_CUDA(dev_malloc(&ws->zs, sizeof(double) * (size_t)k * ds->n_pad));
    IHT_CUDA(dev_malloc(&ws->gram, sizeof(double) * (size_t)k * k));
    IHT_CUDA(dev_malloc(&ws->chol, sizeof(double) * (size_t)k * k));
    IHT_CUDA(dev_malloc(&ws->hvec, sizeof(double) * (size_t)k));
    ws->htp_k = k;
    return IHT_OK;
}

// bSp <- least-squares coefficients on Sp (k, ascending) against y.
int htp_refit(iht_dataset *ds, int k, const int32_t *Sp, double *bSp, const int32_t *done)
{
    Workspace *ws = ds->ws;
    cudaStream_t s = ds->ctx->stream;
    k_htp_cols<<<dim3(ceil_div(ds->n_pad, 256), k), 256, 0, s>>>(ds->G, ds->stride, Sp, ws->u64, ws->v64,
                                                                 ws->zc, ds->p, ws->used, ds->n_pad,
                                                                 ws->zs, done);
    k_htp_gram<<<dim3(k, k + 1), 256, 0, s>>>(ws->zs, ws->y64, k, ds->n_pad, ws->gram, ws->hvec, done);
    k_htp_solve<<<1, 1024, 0, s>>>(ws->gram, ws->hvec, k, ws->chol, bSp, done);
    note_launch(3);
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

}  // namespace iht
