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

#include "common.cuh"

namespace iht {

__device__ __forceinline__ int dosage_of(uint32_t code)   // -1 = missing
{
    return code == 0u ? 0 : (code == 2u ? 1 : (code == 3u ? 2 : -1));
}

// Sums of the per-block partial triples (stride 3) by one full warp: lane l
// adds blocks l, l + 32, ... in order, then a fixed shuffle tree; every lane
// gets the totals (deterministic, and 32 loads in flight instead of one).
__device__ __forceinline__ void warp_partials(const double *__restrict__ partials, int npart,
                                              double &s, double &s2, double &d2)
{
    const int lane = threadIdx.x & 31;
    s = 0.0;
    s2 = 0.0;
    d2 = 0.0;
    for (int b = lane; b < npart; b += 32) {
        s += partials[3 * b];
        s2 += partials[3 * b + 1];
        d2 += partials[3 * b + 2];
    }
    s = warp_sum(s);
    s2 = warp_sum(s2);
    d2 = warp_sum(d2);
}


__global__ void __launch_bounds__(1024) k_gather_gS(const float *__restrict__ g,
                                                    const int32_t *__restrict__ S, int k,
                                                    double *__restrict__ coef, Scalars *sc)
{
    if (sc->done) return;
    gather_gS_body(g, S, k, coef, sc);
}

// out_i = base_i + sum_c a_c (x_i,col_c - u_col_c), a_c = sign coef_c v_col_c, over
// the observed calls (Z[:, cols] coef, Sec. 2.3.2-2.3.3), on used rows (0
// elsewhere); per-block sums of out, out^2 and (out - prev)^2 (0 without
// prev) go to partials[3 b .. 3 b + 2].  One thread per sample, 128 samples
// per block (smaller blocks only multiply the partial triples every consumer
// sums); each column's three possible terms a (x - u) for x = 0, 1, 2 are
// staged in shared memory kZmulChunk columns at a time, so a term costs one
// FP64 add, added in column order.  The product is a chain of dependent steps
// (global loads, FP64 adds, block reductions) on a few warps per SM, so the
// body shortens the chain: the row values (used, base, prev) are requested
// first; a thread loads the genotype bytes of a chunk's first kZmulFirst
// columns (column index, then byte) while the block stages the terms, and the
// rest kZmulBatch columns at a time; the three block sums share one
// reduction.
constexpr int kZmulChunk = 256;
constexpr int kZmulThreads = 128;           // largest block
constexpr int kZmulFirst = 64;
constexpr int kZmulBatch = 16;

__device__ __forceinline__ void zmul_body(const uint8_t *__restrict__ G, int64_t stride,
                                          int64_t rowb, const int32_t *__restrict__ cols, int m,
                                          const double *__restrict__ coef, double sign,
                                          const double *__restrict__ u64,
                                          const double *__restrict__ v64,
                                          const int32_t *__restrict__ used,
                                          const double *__restrict__ base,
                                          const double *__restrict__ prev, double *__restrict__ out,
                                          double *__restrict__ partials, int64_t n_pad,
                                          int64_t psnp = 0, const double *__restrict__ zc = nullptr)
{
    __shared__ double red[3 * (kZmulThreads / 32)];
    __shared__ double term[kZmulChunk][4];     // terms for codes 00, 01 (missing: 0), 10, 11
    __shared__ const uint8_t *srow[kZmulChunk];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t byte = i >> 2;
    const int shift = 2 * (int)(i & 3);
    const bool inb = i < n_pad && byte < rowb;
    const bool in = i < n_pad;
    const int32_t ui = in ? used[i] : 0;
    const double bi = in && base ? base[i] : 0.0;
    const double pi = in && prev ? prev[i] : 0.0;
    // covariate columns (index >= psnp, with zc) sort after the SNPs of an
    // ascending column list: the SNP loop takes the first msnp columns
    const int mall = m;
    if (zc)
        while (m > 0 && cols[m - 1] >= psnp) --m;
    double acc = 0.0;
    for (int c0 = 0; c0 < m; c0 += kZmulChunk) {
        const int mc = min(kZmulChunk, m - c0);
        const int mf = min(mc, kZmulFirst);
        uint32_t bf[kZmulFirst];
        if (inb) {
#pragma unroll
            for (int q = 0; q < kZmulFirst; ++q)
                if (q < mf) bf[q] = __ldg(G + (int64_t)__ldg(cols + c0 + q) * stride + byte);
        }
        __syncthreads();
        for (int c = threadIdx.x; c < mc; c += blockDim.x) {
            const int col = cols[c0 + c];
            const double a = sign * coef[c0 + c] * v64[col];
            const double b = a * u64[col];
            term[c][0] = a * 0.0 - b;
            term[c][1] = 0.0;
            term[c][2] = a * 1.0 - b;
            term[c][3] = a * 2.0 - b;
            srow[c] = G + (int64_t)col * stride;
        }
        __syncthreads();
        if (inb) {
#pragma unroll
            for (int q = 0; q < kZmulFirst; ++q)
                if (q < mf) acc += term[q][(bf[q] >> shift) & 3u];
            int c = mf;
            for (; c + kZmulBatch <= mc; c += kZmulBatch) {
                uint32_t b[kZmulBatch];
#pragma unroll
                for (int q = 0; q < kZmulBatch; ++q) b[q] = __ldg(srow[c + q] + byte);
#pragma unroll
                for (int q = 0; q < kZmulBatch; ++q) acc += term[c + q][(b[q] >> shift) & 3u];
            }
            for (; c + 4 <= mc; c += 4) {
                uint32_t b[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) b[q] = __ldg(srow[c + q] + byte);
#pragma unroll
                for (int q = 0; q < 4; ++q) acc += term[c + q][(b[q] >> shift) & 3u];
            }
            for (; c < mc; ++c) acc += term[c][((uint32_t)__ldg(srow[c] + byte) >> shift) & 3u];
        }
    }
    if (in)
        for (int c = m; c < mall; ++c) acc += (sign * coef[c]) * zc[(int64_t)(cols[c] - psnp) * n_pad + i];
    double o = 0.0, d = 0.0;
    if (in) {
        o = ui ? bi + acc : 0.0;
        out[i] = o;
        if (prev) d = o - pi;
    }
    double s = o, s2 = o * o, d2 = d * d;
    block_sum3(s, s2, d2, red);
    if (threadIdx.x == 0 && partials) {
        partials[3 * blockIdx.x] = s;
        partials[3 * blockIdx.x + 1] = s2;
        partials[3 * blockIdx.x + 2] = d2;
    }
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
              psnp, zc);
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

struct MergeArgs {
    const float *g;
    const int32_t *S;     // k, ascending
    const double *bS;     // beta on S
    const int32_t *cand;  // K, ascending
    int K;
    const double *partials;   // ||Z_S g_S||^2 pieces (first attempt)
    int npart;
    int first;                // 1: compute mu from num / den
    const int32_t *skip;      // not null: return when *skip (a speculative attempt not needed)
    int32_t *Sp;
    double *bSp;
    Scalars *sc;
};

constexpr int kMergeThreads = 1024;
constexpr int kMergeU = 3 * kMaxK;      // |S u C| <= k + 2k
constexpr int kMergeSort = 4 * kMaxK;   // power of two >= kMergeU
constexpr int kMergeRank = 768;         // up to this many candidates: selection by rank

struct MergeShared {
    int32_t sS[kMaxK];            // S, beta_S and the candidates, staged once
    double sbS[kMaxK];
    int32_t scand[kMaxCand];
    int32_t uidx[kMergeU];
    double ubeta[kMergeU];
    double ug[kMergeU];
    double uw[kMergeU];
    uint8_t inS[kMergeU];
    uint8_t inSp[kMergeU];
    unsigned long long skey[kMergeSort];
    int32_t spos[kMergeSort];
    double red[32];
    uint32_t wsum[32];
    int nS_extra;
    int stop;
};

__device__ __forceinline__ bool before(unsigned long long ka, int32_t ia, unsigned long long kb,
                                       int32_t ib)
{
    return ka > kb || (ka == kb && ia < ib);
}

__device__ int lower_bound_i32(const int32_t *a, int n, int32_t x)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Sort positions 0..nU-1 of U by (|w| descending, index ascending).
__device__ void sort_by_w(MergeShared &sh, int nU)
{
    int P = 1;
    while (P < nU) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        if (i < nU) {
            sh.skey[i] = (unsigned long long)__double_as_longlong(fabs(sh.uw[i]));
            sh.spos[i] = i;
        } else {
            sh.skey[i] = 0ull;
            sh.spos[i] = -1;
        }
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int st = size >> 1; st > 0; st >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int j = i ^ st;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const unsigned long long ki = sh.skey[i], kj = sh.skey[j];
                    const int32_t pi = sh.spos[i], pj = sh.spos[j];
                    const int32_t xi = pi < 0 ? 0x7fffffff : sh.uidx[pi];
                    const int32_t xj = pj < 0 ? 0x7fffffff : sh.uidx[pj];
                    const bool swap = up ? before(kj, xj, ki, xi) : before(ki, xi, kj, xj);
                    if (swap) {
                        sh.skey[i] = kj; sh.skey[j] = ki;
                        sh.spos[i] = pj; sh.spos[j] = pi;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// The projection proper for a live solve (every thread of the block calls it).
__device__ __forceinline__ void merge_body(const MergeArgs &A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MergeShared &sh = *reinterpret_cast<MergeShared *>(smem_raw);
    Scalars *sc = A.sc;
    const int k = sc->k;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        sh.sS[i] = A.S[i];
        sh.sbS[i] = A.bS[i];
    }
    for (int i = threadIdx.x; i < A.K; i += blockDim.x) sh.scand[i] = A.cand[i];

    double den = 0.0;
    if (A.first && threadIdx.x < 32) {
        double s_, d2_;
        warp_partials(A.partials, A.npart, s_, den, d2_);
    }
    if (threadIdx.x == 0) {
        sh.stop = 0;
        sh.nS_extra = 0;
        if (A.first) {
            // step size mu = ||g_S||^2 / ||Z_S g_S||^2 (reading of Sec. 2.3.1)
            const double num = sc->num;
            sc->bt_last = 0;
            if (num == 0.0) {
                sc->status = IHT_OK;            // g_S = 0: fixed point
                sc->done = 1;
                sc->skip1 = sc->skip2 = 1;
                sh.stop = 1;
            } else if (!(den > 0.0) || !isfinite(den) || !isfinite(num)) {
                sc->status = IHT_ENUMERIC;
                sc->done = 1;
                sc->skip1 = sc->skip2 = 1;
                sh.stop = 1;
            } else {
                sc->mu = num / den;
            }
        }
    }
    __syncthreads();
    if (sh.stop) return;
    const double mu = sc->mu;

    // U = C (ascending) followed by S \ C (in S order)
    const int K = A.K;
    for (int b = threadIdx.x; b < K; b += blockDim.x) {
        const int32_t j = sh.scand[b];
        const int pos = lower_bound_i32(sh.sS, k, j);
        const bool on = pos < k && sh.sS[pos] == j;
        sh.uidx[b] = j;
        sh.inS[b] = on;
        sh.ubeta[b] = on ? sh.sbS[pos] : 0.0;
        sh.ug[b] = (double)A.g[j];
    }
    {
        const int a = threadIdx.x;
        int32_t j = 0;
        bool extra = false;
        if (a < k) {
            j = sh.sS[a];
            const int pos = lower_bound_i32(sh.scand, K, j);
            extra = !(pos < K && sh.scand[pos] == j);
        }
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        const unsigned bal = __ballot_sync(0xffffffffu, extra);
        if (lane == 0) sh.wsum[wid] = __popc(bal);
        __syncthreads();
        int off = 0;
        for (int w = 0; w < wid; ++w) off += sh.wsum[w];
        off += __popc(bal & ((1u << lane) - 1u));
        if (extra) {
            const int u = K + off;
            sh.uidx[u] = j;
            sh.inS[u] = 1;
            sh.ubeta[u] = sh.sbS[a];
            sh.ug[u] = (double)A.g[j];
        }
        if (threadIdx.x == blockDim.x - 1) sh.nS_extra = off + (extra ? 1 : 0);
    }
    __syncthreads();
    const int nU = K + sh.nS_extra;

    for (int u = threadIdx.x; u < nU; u += blockDim.x) {
        sh.uw[u] = __dadd_rn(sh.ubeta[u], __dmul_rn(mu, sh.ug[u]));
        sh.skey[u] = (unsigned long long)__double_as_longlong(fabs(sh.uw[u]));
    }
    __syncthreads();
    const bool small = nU <= kMergeRank;
    if (small) {
        // S+ by rank: u is in S+ iff fewer than k entries come before it
        // (|w| descending, index ascending); every thread reads the same v
        // at the same time (shared-memory broadcast)
        for (int u = threadIdx.x; u < nU; u += blockDim.x) {
            const unsigned long long ku = sh.skey[u];
            const int32_t iu = sh.uidx[u];
            int rank = 0;
            for (int v = 0; v < nU; ++v) rank += before(sh.skey[v], sh.uidx[v], ku, iu) ? 1 : 0;
            sh.inSp[u] = rank < k ? 1 : 0;
        }
        __syncthreads();
    } else {
        sort_by_w(sh, nU);
        for (int u = threadIdx.x; u < nU; u += blockDim.x) sh.inSp[u] = 0;
        __syncthreads();
        for (int r = threadIdx.x; r < k; r += blockDim.x) sh.inSp[sh.spos[r]] = 1;
        __syncthreads();
    }
    // ||beta+ - beta||^2, ||beta||^2 and |S n S+| by one warp (FP64 issue is
    // scarce: a block-wide reduction would spend it on empty threads); only
    // thread 0 uses them
    int kept = 0;
    double dd = 0.0, bb = 0.0;
    if (threadIdx.x < 32) {
        for (int u = threadIdx.x; u < nU; u += 32) {
            kept += sh.inS[u] && sh.inSp[u];
            const double d = (sh.inSp[u] ? sh.uw[u] : 0.0) - sh.ubeta[u];
            dd += d * d;
            bb += sh.ubeta[u] * sh.ubeta[u];
        }
        kept = __reduce_add_sync(0xffffffffu, kept);
        dd = warp_sum(dd);
        bb = warp_sum(bb);
    }

    // S+ in index order with beta+
    if (small) {
        // position of u among the members of S+ = members with a lower index
        for (int u = threadIdx.x; u < nU; u += blockDim.x) {
            if (!sh.inSp[u]) continue;
            const int32_t iu = sh.uidx[u];
            int pos = 0;
            for (int v = 0; v < nU; ++v) pos += (sh.inSp[v] && sh.uidx[v] < iu) ? 1 : 0;
            A.Sp[pos] = iu;
            A.bSp[pos] = sh.uw[u];
        }
        if (threadIdx.x == 0) {
            sc->changed = kept < k ? 1 : 0;
            sc->dd = dd;
            sc->bb = bb;
        }
        return;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < kMergeSort; r += blockDim.x) sh.skey[r] = ~0ull;
    __syncthreads();
    for (int r = threadIdx.x; r < k; r += blockDim.x) {
        const int u = sh.spos[r];
        sh.skey[r] = ((unsigned long long)(uint32_t)sh.uidx[u] << 32) | (uint32_t)u;
    }
    __syncthreads();
    {
        int P = 1;
        while (P < k) P <<= 1;
        for (int size = 2; size <= P; size <<= 1)
            for (int st = size >> 1; st > 0; st >>= 1) {
                for (int i = threadIdx.x; i < P; i += blockDim.x) {
                    const int j = i ^ st;
                    if (j > i) {
                        const bool up = (i & size) == 0;
                        const unsigned long long a = sh.skey[i], b = sh.skey[j];
                        if ((a > b) == up) { sh.skey[i] = b; sh.skey[j] = a; }
                    }
                }
                __syncthreads();
            }
    }
    for (int r = threadIdx.x; r < k; r += blockDim.x) {
        const int u = (int)(uint32_t)(sh.skey[r] & 0xffffffffull);
        A.Sp[r] = sh.uidx[u];
        A.bSp[r] = sh.uw[u];
    }
    if (threadIdx.x == 0) {
        sc->changed = kept < k ? 1 : 0;
        sc->dd = dd;
        sc->bb = bb;
    }
}

__global__ void __launch_bounds__(kMergeThreads) k_merge(MergeArgs A)
{
    const int d = A.sc->done || (A.skip && *A.skip);
    __syncthreads();   // every thread has read the flag before thread 0 may set it
    if (d) return;
    merge_body(A);
}

// ---------------------------------------------------------------------------
struct TraceDev {
    double *objective, *mu;
    int32_t *backtracks, *changed, *supp;
    double *beta;
};

// Backtracking decision for the candidate of k_merge, whose residual r+ the
// preceding pass wrote (partials: sum r+, sum r+^2, sum (r+ - r)^2).
__device__ __forceinline__ void decide_body(Scalars *sc, const double *partials, int npart,
                                            int32_t *S, double *bS, const int32_t *Sp,
                                            const double *bSp, const TraceDev &tr)
{
    __shared__ int accept;
    const int k = sc->k;
    double s = 0.0, s2 = 0.0, zz = 0.0;
    if (threadIdx.x < 32) warp_partials(partials, npart, s, s2, zz);
    if (threadIdx.x == 0) {
        accept = 1;
        if (sc->changed && zz > 0.0) {
            const double omega = (1.0 - sc->c) * sc->dd / zz;
            if (sc->mu >= omega && sc->bt_last < sc->max_backtrack) {
                sc->mu = sc->mu / sc->kappa;
                sc->bt_last += 1;
                accept = 0;
            }
        }
        sc->retry = accept ? 0 : 1;
        if (accept && sc->htp) {
            // HTP: the step is accepted; the refit on S+ and its residual give the
            // objective and the stopping test (k_htp_finish)
            const int it = sc->iter;
            sc->bt_total += sc->bt_last;
            if (tr.mu) tr.mu[it] = sc->mu;
            if (tr.backtracks) tr.backtracks[it] = sc->bt_last;
            if (tr.changed) tr.changed[it] = sc->changed;
            sc->skip1 = 1;
            sc->skip2 = 1;
        } else if (accept) {
            const int it = sc->iter;
            sc->bt_total += sc->bt_last;
            sc->sum_r = s;
            sc->sumsq_r = s2;
            sc->f = 0.5 * s2;
            sc->step = sqrt(sc->dd) / (sqrt(sc->bb) + 1.0);
            if (tr.objective) tr.objective[it] = sc->f;
            if (tr.mu) tr.mu[it] = sc->mu;
            if (tr.backtracks) tr.backtracks[it] = sc->bt_last;
            if (tr.changed) tr.changed[it] = sc->changed;
        }
    }
    __syncthreads();
    if (!accept) {
        if (threadIdx.x == 0) {
            sc->skip1 = 0;                     // another attempt with the shrunk mu
            sc->skip2 = 1;
        }
        return;
    }
    if (sc->htp) return;
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
        sc->skip1 = 1;                         // accepted: no further attempt
        sc->skip2 = sc->done;                  // the next gradient unless stopped
    }
}

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

// Objective of beta = 0 (r = y) before the first iteration (one thread).
// One full warp; lane 0 writes.
__device__ __forceinline__ void init_objective_body(Scalars *sc, const double *partials, int npart)
{
    double s, s2, d2;
    warp_partials(partials, npart, s, s2, d2);
    if (threadIdx.x == 0) {
        sc->sum_r = s;
        sc->sumsq_r = s2;
        sc->f = 0.5 * s2;
    }
}

__global__ void k_init_objective(Scalars *sc, const double *partials, int npart)
{
    if (sc->done) return;
    init_objective_body(sc, partials, npart);
}

// Accepted residual: r64 <- src, r32 <- src - mean on the used rows.
__device__ __forceinline__ void center_body(const double *__restrict__ src, double *__restrict__ r64,
                                            const int32_t *__restrict__ used, int64_t n_pad,
                                            const Scalars *sc, float *__restrict__ r32)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pad) return;
    const double mean = sc->sum_r / (double)sc->n_rows;
    const double v = src[i];
    if (src != r64) r64[i] = v;
    r32[i] = used[i] ? (float)(v - mean) : 0.0f;
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
static int launch_grad_ev(iht_dataset *ds, int impl, const int32_t *done, cudaEvent_t e0, cudaEvent_t e1)
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
    rc = tc ? launch_grad_tc_main(ds, ws->r32, ws->g, done) : launch_grad_simt(ds, ws->r32, ws->g, done);
    if (rc) return rc;
    if (e1) IHT_CUDA(cudaEventRecordWithFlags(e1, s, flags));
    return launch_cov_grad(ds, ws->r32, ws->g, done);       // covariate entries p .. p+q-1
}

int launch_grad(iht_dataset *ds, int impl, const int32_t *done, bool profile)
{
    Workspace *ws = ds->ws;
    const bool rec = profile && ws->nprof < kProfEvents;
    const int rc = launch_grad_ev(ds, impl, done, rec ? ws->prof_ev[2 * ws->nprof] : nullptr,
                                  rec ? ws->prof_ev[2 * ws->nprof + 1] : nullptr);
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

    const bool traced = tr.objective || tr.mu || tr.backtracks || tr.changed || tr.supp || tr.beta;
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
    if (!traced && !htp) {
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
                  B.r64, B.partials, n_pad);
    else if (which == kZmulStep)
        zmul_body(G, stride, rowb, B.S, B.k, B.coef, 1.0, B.u64, B.v64, B.used, nullptr, nullptr,
                  B.zv, B.partials, n_pad);
    else
        zmul_body(G, stride, rowb, B.Sp, B.k, B.bSp, -1.0, B.u64, B.v64, B.used, B.y64, B.r64,
                  B.rc64, B.partials, n_pad);
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
              n_pad);
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
