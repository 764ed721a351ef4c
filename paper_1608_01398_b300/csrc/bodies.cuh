// Device bodies of the O(nk) steps of an IHT iteration (a4-a6), shared by the
// kernels of solver.cu (one solve, and one solve per block row of a batch) and
// the fused per-iteration kernel of tail.cu, so every path performs the same
// operations in the same order and gives the same bits.
//
//   zmul_body     out = base + sign * Z[:, cols] coef over one 128-sample block,
//                 per-block partial sums of out, out^2 and (out - prev)^2
//                 (sparse product X_k beta_k, Sec. 2.3.2-2.3.3)
//   merge_body    mu = num / den on the first attempt; w = beta + mu g on S u C;
//                 S+ = top-k |w|, beta+ = w on S+ (Eq. ihta)
//   decide_body   backtracking test mu < omega (Sec. 2.3.1), objective,
//                 stopping test, state copy
//   center_body   r32 = r - mean(r) on the used rows
#pragma once
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
__device__ __forceinline__ void warp_partials(const double *partials, int npart,
                                              double &s, double &s2, double &d2)
{
    const int lane = threadIdx.x & 31;
    s = 0.0;
    s2 = 0.0;
    d2 = 0.0;
#pragma unroll 2
    for (int b = lane; b < npart; b += 32) {
        s += partials[3 * b];
        s2 += partials[3 * b + 1];
        d2 += partials[3 * b + 2];
    }
    s = warp_sum(s);
    s2 = warp_sum(s2);
    d2 = warp_sum(d2);
}

// out_i = base_i + sum_c a_c (x_i,col_c - u_col_c), a_c = sign coef_c v_col_c, over
// the observed calls (Z[:, cols] coef, Sec. 2.3.2-2.3.3), on used rows (0
// elsewhere); per-block sums of out, out^2 and (out - prev)^2 (0 without
// prev) go to partials[3 b .. 3 b + 2].  One thread per sample, 128 samples
// per block (every caller launches kZmulThreads threads; smaller blocks would
// only multiply the partial triples every consumer sums).
//
// The sum over columns is exact: each column's three possible terms
// a (x - u), x = 0, 1, 2, are rounded once to multiples of 2^-E and added as
// 64-bit integers, E chosen from the largest |a| and the column count so that
// no partial sum can reach 2^62 (|x - u| <= 2); the integer sum is rounded
// once back to FP64.  Its error is below that of any FP64 summation order,
// and the FP64 unit (a few operations per clock per SM on this part) is
// left to the per-sample base add and the block sums.  A non-finite a or u
// makes every output NaN.  Per chunk of kZmulChunk columns the block stages
// the integer terms and its 32 genotype bytes of each column (two 16-byte
// loads, one per thread, all in flight at once) in shared memory; a thread
// then adds one staged term per column.  The body runs once per pass of a
// launch that is itself run once per iteration, so its code is fetched cold
// each time: the loops stay rolled (a few lines of code).
constexpr int kZmulChunk = 256;
constexpr int kZmulThreads = 128;           // the block every caller launches
constexpr int kZmulBytes = kZmulThreads / 4;   // genotype bytes of a block per column

// a_c of column c of the list (the expression every pass uses)
__device__ __forceinline__ double zmul_coef(const double *coef, int c, double sign, double v)
{
    return sign * coef[c] * v;
}

// vb: the 128-sample block to compute (blockIdx.x in a kernel of its own; a
// fused kernel passes its own index).  The column list, coefficients, base,
// prev and outputs may be written earlier in the same launch by a fused
// kernel, so they are read with ordinary (coherent) loads.
__device__ __forceinline__ void zmul_body(const uint8_t *__restrict__ G, int64_t stride,
                                          int64_t rowb, const int32_t *cols, int m,
                                          const double *coef, double sign,
                                          const double *__restrict__ u64,
                                          const double *__restrict__ v64,
                                          const int32_t *__restrict__ used,
                                          const double *base,
                                          const double *prev, double *out,
                                          double *partials, int64_t n_pad,
                                          int64_t psnp, const double *zc, int vb)
{
    __shared__ double red[3 * (kZmulThreads / 32)];
    __shared__ long long term[kZmulChunk][4];  // terms for codes 00, 01 (missing: 0), 10, 11
    __shared__ double sa[kZmulChunk], su[kZmulChunk];
    __shared__ __align__(16) uint8_t gtile[kZmulChunk][kZmulBytes];
    __shared__ int s_ebits, s_bad;             // largest biased exponent of |a|; a non-finite input
    const int64_t i = (int64_t)vb * kZmulThreads + threadIdx.x;
    const int64_t b0 = (int64_t)vb * kZmulBytes;     // first byte of the block in a row (< stride)
    const int bl = threadIdx.x >> 2;                   // this sample's byte in the tile
    const int shift = 2 * (int)(threadIdx.x & 3);
    const bool inb = i < n_pad && b0 + bl < rowb;
    const bool in = i < n_pad;
    const int32_t ui = in ? used[i] : 0;
    const double bi = in && base ? base[i] : 0.0;
    const double pi = in && prev ? prev[i] : 0.0;
    // covariate columns (index >= psnp, with zc) sort after the SNPs of an
    // ascending column list: the SNP loop takes the first msnp columns
    const int mall = m;
    if (zc)
        while (m > 0 && cols[m - 1] >= psnp) --m;
    if (threadIdx.x == 0) {
        s_ebits = 0;
        s_bad = 0;
    }
    __syncthreads();
    // a chunk's bytes, a and u into shared memory (thread t: half t & 1 of
    // column t >> 1's 32 bytes -- rows are 128-byte aligned and b0 + 32 <=
    // stride, so the loads stay inside the row; the even thread takes a, u)
    auto stage = [&](int c0, int mc) {
#pragma unroll 2
        for (int t = threadIdx.x; t < 2 * mc; t += kZmulThreads) {
            const int c = t >> 1;
            const int col = cols[c0 + c];
            const uint4 *src = reinterpret_cast<const uint4 *>(G + (int64_t)col * stride + b0) + (t & 1);
            reinterpret_cast<uint4 *>(gtile[c])[t & 1] = __ldg(src);
            if (!(t & 1)) {
                const double a = zmul_coef(coef, c0 + c, sign, v64[col]);
                const double u = u64[col];
                sa[c] = a;
                su[c] = u;
                if (!isfinite(a) || !isfinite(u)) s_bad = 1;
                atomicMax(&s_ebits, (int)((__double_as_longlong(a) >> 52) & 0x7ff));
            }
        }
    };
    // the scale 2^E: m 2^(emax + 1) 2^E <= 2^62 with |a| < 2^emax, from every
    // column (the first chunk's while it is staged)
    if (m > 0) stage(0, min(m, kZmulChunk));
#pragma unroll 1
    for (int c = kZmulChunk + threadIdx.x; c < m; c += kZmulThreads) {
        const int col = cols[c];
        const double a = zmul_coef(coef, c, sign, v64[col]);
        if (!isfinite(a) || !isfinite(u64[col])) s_bad = 1;
        atomicMax(&s_ebits, (int)((__double_as_longlong(a) >> 52) & 0x7ff));
    }
    __syncthreads();
    int L = 0;
    while ((1 << L) < m) ++L;
    const int emax = s_ebits - 1022;                   // |a| < 2^emax (0 bits: every a is 0 or tiny)
    const int E = max(-1000, min(1000, 61 - L - emax));
    const double scale = __longlong_as_double((long long)(E + 1023) << 52);
    const bool bad = s_bad != 0;
    long long acc = 0;
#pragma unroll 1
    for (int c0 = 0; c0 < m && !bad; c0 += kZmulChunk) {
        const int mc = min(kZmulChunk, m - c0);
        if (c0 > 0) {
            __syncthreads();                       // the previous chunk's reads are done
            stage(c0, mc);
            __syncthreads();
        }
#pragma unroll 1
        for (int c = threadIdx.x; c < mc; c += kZmulThreads) {
            const double a = sa[c], u = su[c];
            term[c][0] = __double2ll_rn((a * (0.0 - u)) * scale);
            term[c][1] = 0;
            term[c][2] = __double2ll_rn((a * (1.0 - u)) * scale);
            term[c][3] = __double2ll_rn((a * (2.0 - u)) * scale);
        }
        __syncthreads();
        if (inb) {
#pragma unroll 4
            for (int c = 0; c < mc; ++c) acc += term[c][((uint32_t)gtile[c][bl] >> shift) & 3u];
        }
    }
    double sum = bad ? __longlong_as_double(0x7ff8000000000000ll)
                     : __ll2double_rn(acc) * __longlong_as_double((long long)(1023 - E) << 52);
    if (in)
#pragma unroll 1
        for (int c = m; c < mall; ++c) sum += (sign * coef[c]) * zc[(int64_t)(cols[c] - psnp) * n_pad + i];
    double o = 0.0, d = 0.0;
    if (in) {
        o = ui ? bi + sum : 0.0;
        out[i] = o;
        if (prev) d = o - pi;
    }
    // the block's sums of out, out^2 and (out - prev)^2: a shuffle tree per
    // warp, then lanes 0..2 each add one quantity's warp sums in warp order
    double s = o, s2 = o * o, d2 = d * d;
    constexpr int nw = kZmulThreads / 32;
#pragma unroll
    for (int q = 16; q > 0; q >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, q);
        s2 += __shfl_xor_sync(0xffffffffu, s2, q);
        d2 += __shfl_xor_sync(0xffffffffu, d2, q);
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = s;
        red[nw + (threadIdx.x >> 5)] = s2;
        red[2 * nw + (threadIdx.x >> 5)] = d2;
    }
    __syncthreads();
    if (threadIdx.x < 3 && partials) {
        double t = red[threadIdx.x * nw];
#pragma unroll
        for (int w = 1; w < nw; ++w) t += red[threadIdx.x * nw + w];
        partials[3 * vb + threadIdx.x] = t;
    }
    __syncthreads();                                   // red is free for the next call
}

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
    int shrinks = 0;          // first attempt only: mu / kappa this many times after num / den
                              // (a later attempt evaluated ahead of the decision on this one)
    const float *gS = nullptr;    // g on S in S order, when the caller has it at hand
};

constexpr int kMergeThreads = 1024;
// Up to this many entries of S u C the selection is by rank (each thread counts
// the entries before its own), above it by a bitonic sort of the block; both
// choose the same set in the same order (measured: the rank is the faster of
// the two at the sizes of the single-solve workload, with 128 threads or 1024).
constexpr int kMergeRank = 768;

// Shared memory of the projection for supports of at most KM indices (the
// candidates are at most 2 KM, |S u C| at most 3 KM).
template <int KM> struct MergeSharedT {
    static constexpr int kU = 3 * KM;   // |S u C| <= k + 2k
    static constexpr int kSort = 4 * KM;    // power of two >= kU
    int32_t sS[KM];               // S, beta_S and the candidates, staged once
    double sbS[KM];
    int32_t scand[2 * KM];
    int32_t uidx[kU];
    double ubeta[kU];
    double ug[kU];
    double uw[kU];
    uint8_t inS[kU];
    uint8_t inSp[kU];
    // sort keys and positions; the rank reads skey and spos together as one
    // array of kU 16-byte keys (16 kU = 12 kSort bytes)
    alignas(16) unsigned long long skey[kSort];
    int32_t spos[kSort];
    double red[32];
    uint32_t wsum[32];
    double mu;                    // the step of this attempt, read once
    int nS_extra;
    int stop;
};
using MergeShared = MergeSharedT<kMaxK>;

__device__ __forceinline__ bool before(unsigned long long ka, int32_t ia, unsigned long long kb,
                                       int32_t ib)
{
    return ka > kb || (ka == kb && ia < ib);
}

// 96-bit unsigned (a.z, a.y, a.x) < (v.z, v.y, v.x): all ones if so, else 0
// (the borrow of a - v).
__device__ __forceinline__ uint32_t lt96(uint4 a, uint4 v)
{
    uint32_t b;
    asm("{\n.reg .u32 t, z;\nmov.u32 z, 0;\nsub.cc.u32 t, %1, %4;\nsubc.cc.u32 t, %2, %5;\n"
        "subc.cc.u32 t, %3, %6;\nsubc.u32 %0, z, z;\n}"
        : "=r"(b)
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(v.x), "r"(v.y), "r"(v.z));
    return b;
}

__device__ __forceinline__ int lower_bound_i32(const int32_t *a, int n, int32_t x)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Sort positions 0..nU-1 of U by (|w| descending, index ascending).
template <typename SH> __device__ void sort_by_w(SH &sh, int nU)
{
    int P = 1;
    while (P < nU) P <<= 1;
#pragma unroll 1
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
#pragma unroll 1
    for (int size = 2; size <= P; size <<= 1) {
#pragma unroll 1
        for (int st = size >> 1; st > 0; st >>= 1) {
#pragma unroll 1
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

// The projection proper for a live solve (every thread of the block calls it;
// SH bounds k; the block may have fewer threads than k).
template <typename SH = MergeShared> __device__ __forceinline__ void merge_body(const MergeArgs &A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SH &sh = *reinterpret_cast<SH *>(smem_raw);
    Scalars *sc = A.sc;
    const int k = sc->k;
#pragma unroll 1
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        sh.sS[i] = A.S[i];
        sh.sbS[i] = A.bS[i];
    }
#pragma unroll 1
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
#pragma unroll 1
                for (int q = 0; q < A.shrinks; ++q) sc->mu = sc->mu / sc->kappa;   // as the decision shrinks it
            }
        }
    }
    if (threadIdx.x == 0 && !sh.stop) sh.mu = sc->mu;
    __syncthreads();
    if (sh.stop) return;
    const double mu = sh.mu;

    // U = C (ascending) followed by S \ C (in S order)
    const int K = A.K;
#pragma unroll 1
    for (int b = threadIdx.x; b < K; b += blockDim.x) {
        const int32_t j = sh.scand[b];
        const int pos = lower_bound_i32(sh.sS, k, j);
        const bool on = pos < k && sh.sS[pos] == j;
        sh.uidx[b] = j;
        sh.inS[b] = on;
        sh.ubeta[b] = on ? sh.sbS[pos] : 0.0;
        sh.ug[b] = (double)A.g[j];
    }
    // members of S not among the candidates, appended in S order (blockDim.x
    // at a time: a running offset carries the count of earlier chunks)
    {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        int base = 0;
#pragma unroll 1
        for (int a0 = 0; a0 < k; a0 += blockDim.x) {
            const int a = a0 + threadIdx.x;
            int32_t j = 0;
            bool extra = false;
            if (a < k) {
                j = sh.sS[a];
                const int pos = lower_bound_i32(sh.scand, K, j);
                extra = !(pos < K && sh.scand[pos] == j);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, extra);
            if (lane == 0) sh.wsum[wid] = __popc(bal);
            __syncthreads();
            int off = base, tot = 0;
#pragma unroll 1
            for (int w = 0; w < nw; ++w) {
                if (w < wid) off += sh.wsum[w];
                tot += sh.wsum[w];
            }
            off += __popc(bal & ((1u << lane) - 1u));
            if (extra) {
                const int u = K + off;
                sh.uidx[u] = j;
                sh.inS[u] = 1;
                sh.ubeta[u] = sh.sbS[a];
                sh.ug[u] = (double)(A.gS ? A.gS[a] : A.g[j]);
            }
            base += tot;
            __syncthreads();              // wsum is reused by the next chunk
        }
        if (threadIdx.x == 0) sh.nS_extra = base;
    }
    __syncthreads();
    const int nU = K + sh.nS_extra;

    const bool small = nU <= kMergeRank;
    // rank keys {~index, |w| low word, |w| high word, 0}: v comes before u
    // (|w| descending, index ascending) iff key u < key v as 96-bit integers
    uint4 *rk = reinterpret_cast<uint4 *>(sh.skey);
#pragma unroll 1
    for (int u = threadIdx.x; u < nU; u += blockDim.x) {
        const double w = __dadd_rn(sh.ubeta[u], __dmul_rn(mu, sh.ug[u]));
        sh.uw[u] = w;
        if (small) {
            const unsigned long long kb = (unsigned long long)__double_as_longlong(fabs(w));
            rk[u] = make_uint4(~(uint32_t)sh.uidx[u], (uint32_t)kb, (uint32_t)(kb >> 32), 0u);
        }
    }
    __syncthreads();
    if (small) {
        // S+ by rank: u is in S+ iff fewer than k entries come before it; a
        // thread ranks two entries in one sweep over v, and every thread reads
        // the same v at the same time (shared-memory broadcast)
#pragma unroll 1
        for (int ub = 0; ub < nU; ub += 2 * (int)blockDim.x) {
            const int ua = ub + threadIdx.x, uc = ua + blockDim.x;
            const bool two = __any_sync(0xffffffffu, uc < nU);   // one path per warp
            if (ua >= nU) continue;               // (a large block: most threads have none)
            const uint4 ka = rk[ua], kc = rk[min(uc, nU - 1)];
            int ra = 0, rc = 0;
            if (two) {
#pragma unroll 4
                for (int v = 0; v < nU; ++v) {
                    const uint4 kv = rk[v];
                    ra -= (int)lt96(ka, kv);
                    rc -= (int)lt96(kc, kv);
                }
            } else {
#pragma unroll 4
                for (int v = 0; v < nU; ++v) ra -= (int)lt96(ka, rk[v]);
            }
            if (ua < nU) sh.inSp[ua] = ra < k ? 1 : 0;
            if (uc < nU) sh.inSp[uc] = rc < k ? 1 : 0;
        }
        __syncthreads();
    } else {
        sort_by_w(sh, nU);
#pragma unroll 1
        for (int u = threadIdx.x; u < nU; u += blockDim.x) sh.inSp[u] = 0;
        __syncthreads();
#pragma unroll 1
        for (int r = threadIdx.x; r < k; r += blockDim.x) sh.inSp[sh.spos[r]] = 1;
        __syncthreads();
    }
    // ||beta+ - beta||^2 by warp 0, ||beta||^2 by warp 1 and |S n S+| by warp 2
    // (all three by warp 0 in a block of fewer warps), each over u = lane
    // (mod 32) and a shuffle tree: FP64 issue is scarce, and a block-wide
    // reduction would spend it on empty threads.  Only thread 0 uses them
    // (warps 1 and 2 hand theirs over in shared memory, read after the
    // barriers below).
    int kept = 0;
    double dd = 0.0, bb = 0.0;
    {
        const int wq = threadIdx.x >> 5;
        const bool split = blockDim.x >= 96;
        const bool do_dd = wq == 0, do_bb = split ? wq == 1 : wq == 0, do_kept = split ? wq == 2 : wq == 0;
        if (do_dd || do_bb || do_kept) {
#pragma unroll 2
            for (int u = threadIdx.x & 31; u < nU; u += 32) {
                if (do_kept) kept += sh.inS[u] && sh.inSp[u];
                if (do_dd) {
                    const double d = (sh.inSp[u] ? sh.uw[u] : 0.0) - sh.ubeta[u];
                    dd += d * d;
                }
                if (do_bb) bb += sh.ubeta[u] * sh.ubeta[u];
            }
            if (do_kept) kept = __reduce_add_sync(0xffffffffu, kept);
            if (do_dd) dd = warp_sum(dd);
            if (do_bb) bb = warp_sum(bb);
            if (split && (threadIdx.x == 32)) sh.red[0] = bb;
            if (split && (threadIdx.x == 64)) sh.red[1] = (double)kept;
        }
    }

    // S+ in index order with beta+
    if (small) {
        // position of u among the members of S+ = members with a lower index.
        // U is two ascending runs, C (positions < K) and S \ C (K .. nU - 1):
        // pre[u] = members of S+ before position u (a block scan), and the
        // members of the other run with a lower index are found by a binary
        // search of that run
        int32_t *pre = sh.spos;
        {
            const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
            int base = 0;
#pragma unroll 1
            for (int a0 = 0; a0 < nU; a0 += blockDim.x) {
                const int u = a0 + threadIdx.x;
                const bool f = u < nU && sh.inSp[u];
                const unsigned bal = __ballot_sync(0xffffffffu, f);
                __syncthreads();          // the previous chunk's wsum reads are done
                if (lane == 0) sh.wsum[wid] = __popc(bal);
                __syncthreads();
                int off = base, tot = 0;
#pragma unroll 1
                for (int w = 0; w < nw; ++w) {
                    if (w < wid) off += sh.wsum[w];
                    tot += sh.wsum[w];
                }
                if (u < nU) pre[u] = off + __popc(bal & ((1u << lane) - 1u));
                base += tot;
            }
            if (threadIdx.x == 0) pre[nU] = base;
        }
        __syncthreads();
#pragma unroll 1
        for (int u = threadIdx.x; u < nU; u += blockDim.x) {
            if (!sh.inSp[u]) continue;
            const int32_t iu = sh.uidx[u];
            int pos;
            if (u < K) {
                const int lb = lower_bound_i32(sh.uidx + K, nU - K, iu);
                pos = pre[u] + (pre[K + lb] - pre[K]);
            } else {
                const int lb = lower_bound_i32(sh.uidx, K, iu);
                pos = (pre[u] - pre[K]) + pre[lb];
            }
            A.Sp[pos] = iu;
            A.bSp[pos] = sh.uw[u];
        }
        if (threadIdx.x == 0) {
            if (blockDim.x >= 96) {
                bb = sh.red[0];
                kept = (int)sh.red[1];
            }
            sc->changed = kept < k ? 1 : 0;
            sc->dd = dd;
            sc->bb = bb;
        }
        return;
    }
    __syncthreads();
#pragma unroll 1
    for (int r = threadIdx.x; r < SH::kSort; r += blockDim.x) sh.skey[r] = ~0ull;
    __syncthreads();
#pragma unroll 1
    for (int r = threadIdx.x; r < k; r += blockDim.x) {
        const int u = sh.spos[r];
        sh.skey[r] = ((unsigned long long)(uint32_t)sh.uidx[u] << 32) | (uint32_t)u;
    }
    __syncthreads();
    {
        int P = 1;
        while (P < k) P <<= 1;
#pragma unroll 1
        for (int size = 2; size <= P; size <<= 1)
#pragma unroll 1
            for (int st = size >> 1; st > 0; st >>= 1) {
#pragma unroll 1
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
#pragma unroll 1
    for (int r = threadIdx.x; r < k; r += blockDim.x) {
        const int u = (int)(uint32_t)(sh.skey[r] & 0xffffffffull);
        A.Sp[r] = sh.uidx[u];
        A.bSp[r] = sh.uw[u];
    }
    if (threadIdx.x == 0) {
        if (blockDim.x >= 96) {
            bb = sh.red[0];
            kept = (int)sh.red[1];
        }
        sc->changed = kept < k ? 1 : 0;
        sc->dd = dd;
        sc->bb = bb;
    }
}

struct TraceDev {
    double *objective, *mu;
    int32_t *backtracks, *changed, *supp;
    double *beta;
};

// Backtracking decision for the candidate of k_merge, whose residual r+ the
// preceding pass wrote (partials: sum r+, sum r+^2, sum (r+ - r)^2).
//
// pre (optional): the values the body would compute, formed ahead by the
// caller with the same expressions -- {sum r+, sum r+^2, ||ZΔ||^2, omega,
// the stopping measure, mu / kappa} -- so a fused kernel can form them for
// both candidates at once.
__device__ __forceinline__ void decide_body(Scalars *sc, const double *partials, int npart,
                                            int32_t *S, double *bS, const int32_t *Sp,
                                            const double *bSp, const TraceDev &tr,
                                            const double *pre = nullptr)
{
    __shared__ int accept;
    const int k = sc->k;
    double s = 0.0, s2 = 0.0, zz = 0.0;
    if (pre) {
        s = pre[0];
        s2 = pre[1];
        zz = pre[2];
    } else if (threadIdx.x < 32) {
        warp_partials(partials, npart, s, s2, zz);
    }
    if (threadIdx.x == 0) {
        accept = 1;
        if (sc->changed && zz > 0.0) {
            const double omega = pre ? pre[3] : (1.0 - sc->c) * sc->dd / zz;
            if (sc->mu >= omega && sc->bt_last < sc->max_backtrack) {
                sc->mu = pre ? pre[5] : sc->mu / sc->kappa;
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
            sc->step = pre ? pre[4] : sqrt(sc->dd) / (sqrt(sc->bb) + 1.0);
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
#pragma unroll 1
    for (int c = threadIdx.x; c < k && S; c += blockDim.x) {    // (S null: only the scalars)
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

}  // namespace iht
