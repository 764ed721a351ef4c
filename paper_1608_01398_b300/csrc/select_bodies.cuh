// Device pieces of the top-K selection by |key| with ties to the lower index
// (Eq. ihta's projection P_{S_k}), shared by the selection kernels of
// select.cu and the fused per-iteration kernel of tail.cu.  For non-negative
// floats the IEEE bit pattern orders like the value, so |x| is keyed by its
// bits 30..0.
#pragma once
#include "common.cuh"

namespace iht {

__device__ __forceinline__ uint32_t sel_key(float x) { return __float_as_uint(x) & 0x7fffffffu; }

constexpr int kSelAThreads = 256;
constexpr int kSelBThreads = 512;
constexpr int kSelKeysPerBlock = 4096;     // keys per block of A and B (fewer blocks: fewer atomics)

// Exclusive scan of x over the block (blockDim.x <= 1024); wsum: 32 words.
__device__ __forceinline__ uint32_t sel_excl_scan(uint32_t x, uint32_t *wsum, uint32_t *total = nullptr)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t t = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += v;
    }
    if (lane == 31) wsum[wid] = t;
    __syncthreads();
    if (wid == 0) {
        uint32_t q = lane < nw ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, q, o);
            if (lane >= o) q += v;
        }
        wsum[lane] = q;
    }
    __syncthreads();
    const uint32_t r = t - x + (wid ? wsum[wid - 1] : 0u);
    if (total) *total = wsum[nw - 1];
    __syncthreads();
    return r;
}

// Bins h[0..nbins) (shared) scanned from the top: res = {bin, keys above it,
// keys in it} for the bin where the running count reaches need.
__device__ __forceinline__ void sel_find(const uint32_t *h, int nbins, uint32_t need, uint32_t *wsum,
                                         uint32_t *res)
{
    const int per = nbins / (int)blockDim.x;
    const int t = threadIdx.x;
    if (t == 0) res[0] = res[1] = res[2] = 0;
    uint32_t tot = 0;
#pragma unroll 1
    for (int i = 0; i < per; ++i) tot += h[nbins - 1 - (per * t + i)];
    uint32_t before = sel_excl_scan(tot, wsum);
#pragma unroll 1
    for (int i = 0; i < per; ++i) {
        const int bin = nbins - 1 - (per * t + i);
        const uint32_t c = h[bin];
        if (before < need && before + c >= need) {
            res[0] = (uint32_t)bin;
            res[1] = before;
            res[2] = c;
        }
        before += c;
    }
    __syncthreads();
}

// sel_find over a histogram of kPer * blockDim.x bins held in registers:
// thread t holds bins nbins - 1 - (kPer t + i) in c[i], i = 0 .. kPer-1 --
// the same scan in the same order, so the same result.
template <int kPer>
__device__ __forceinline__ void sel_find_regs(const uint32_t (&c)[kPer], uint32_t need, uint32_t *wsum,
                                              uint32_t *res)
{
    const int t = threadIdx.x, nbins = kPer * (int)blockDim.x;
    if (t == 0) res[0] = res[1] = res[2] = 0;
    uint32_t tot = 0;
#pragma unroll
    for (int i = 0; i < kPer; ++i) tot += c[i];
    uint32_t before = sel_excl_scan(tot, wsum);
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        if (before < need && before + c[i] >= need) {
            res[0] = (uint32_t)(nbins - 1 - (kPer * t + i));
            res[1] = before;
            res[2] = c[i];
        }
        before += c[i];
    }
    __syncthreads();
}

// Calls f(key, index) for every key; 16-byte loads, two in flight per thread,
// over the 16-byte aligned middle, the (at most 3 + 3) keys around it one at a
// time.
// (b, nb: this block's index among the nb blocks that share the keys; by
// default the grid's)
template <typename F>
__device__ __forceinline__ void sel_each(const float *__restrict__ keys, int64_t p, F &&f, int b = -1,
                                         int nb = -1)
{
    if (nb < 0) {
        b = blockIdx.x;
        nb = gridDim.x;
    }
    const int64_t head = std::min<int64_t>(p, (int64_t)((16u - ((uintptr_t)keys & 15u)) & 15u) >> 2);
    const float4 *k4 = reinterpret_cast<const float4 *>(keys + head);
    const int64_t n4 = (p - head) >> 2, step = (int64_t)nb * blockDim.x;
    const int64_t tid = (int64_t)b * blockDim.x + threadIdx.x;
    int64_t q = tid;
    for (; q + step < n4; q += 2 * step) {
        const float4 a = k4[q], b = k4[q + step];
        const int64_t ja = head + 4 * q, jb = head + 4 * (q + step);
        f(a.x, ja); f(a.y, ja + 1); f(a.z, ja + 2); f(a.w, ja + 3);
        f(b.x, jb); f(b.y, jb + 1); f(b.z, jb + 2); f(b.w, jb + 3);
    }
    if (q < n4) {
        const float4 a = k4[q];
        const int64_t ja = head + 4 * q;
        f(a.x, ja); f(a.y, ja + 1); f(a.z, ja + 2); f(a.w, ja + 3);
    }
    if (tid < head) f(keys[tid], tid);
    const int64_t t = head + (n4 << 2) + tid;
    if (t < p) f(keys[t], t);
}

// Exact finish in one block (keys in or above the boundary bin > kSelCap):
// the other two digits of the K-th key T, then every key > T in any order and
// the lowest-index keys == T in index order after them.
static __device__ void sel_exact_block(const float *__restrict__ keys, int64_t p, const SelState *st,
                                int32_t *out, uint32_t K, uint32_t *wsum)
{
    __shared__ uint32_t h[1024];
    __shared__ uint32_t res[3];
    __shared__ uint32_t s_prefix, s_mask, s_need, s_gt, s_cnt;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_prefix = st->prefix;
        s_mask = st->mask;
        s_need = st->need;
        s_gt = st->count_gt;
        s_cnt = 0;
    }
    __syncthreads();
#pragma unroll 1
    for (int ps = 0; ps < 2; ++ps) {
        const int shift = ps == 0 ? 10 : 0;
#pragma unroll 1
        for (int b = tid; b < 1024; b += blockDim.x) h[b] = 0;
        __syncthreads();
        const uint32_t prefix = s_prefix, mask = s_mask;
#pragma unroll 1
        for (int64_t j = tid; j < p; j += blockDim.x) {
            const uint32_t k = sel_key(keys[j]);
            if ((k & mask) == prefix) atomicAdd(&h[(k >> shift) & 0x3ffu], 1u);
        }
        __syncthreads();
        sel_find(h, 1024, s_need, wsum, res);
        if (tid == 0) {
            s_prefix |= res[0] << shift;
            s_mask |= 0x3ffu << shift;
            s_gt += res[1];
            s_need -= res[1];
        }
        __syncthreads();
    }
    const uint32_t T = s_prefix, gt = s_gt, need = s_need;
#pragma unroll 1
    for (int64_t j = tid; j < p; j += blockDim.x) {
        if (sel_key(keys[j]) > T) {
            const uint32_t slot = atomicAdd(&s_cnt, 1u);
            if (slot < K) out[slot] = (int32_t)j;
        }
    }
    uint32_t taken = 0;
#pragma unroll 1
    for (int64_t base = 0; base < p && taken < need; base += blockDim.x) {
        const int64_t j = base + tid;
        const uint32_t f = (j < p && sel_key(keys[j]) == T) ? 1u : 0u;
        uint32_t tot = 0;
        const uint32_t r = sel_excl_scan(f, wsum, &tot);
        if (f && taken + r < need && gt + taken + r < K) out[gt + taken + r] = (int32_t)j;
        taken += tot;
    }
    __syncthreads();
}

// Sort K (<= kMaxCand) indices ascending in one block (bitonic in shared memory).
__device__ __forceinline__ void sort_idx_body(int32_t *idx, int K)
{
    __shared__ int32_t s[kMaxCand];
    int P = 1;
    while (P < K) P <<= 1;
#pragma unroll 1
    for (int i = threadIdx.x; i < P; i += blockDim.x) s[i] = i < K ? idx[i] : 0x7fffffff;
    __syncthreads();
#pragma unroll 1
    for (int size = 2; size <= P; size <<= 1) {
#pragma unroll 1
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
#pragma unroll 1
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int jx = i ^ stride;
                if (jx > i) {
                    const bool up = (i & size) == 0;
                    const int32_t a = s[i], b = s[jx];
                    if ((a > b) == up) {
                        s[i] = b;
                        s[jx] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
#pragma unroll 1
    for (int i = threadIdx.x; i < K; i += blockDim.x) idx[i] = s[i];
}


// Up to this many candidate words the finish ranks them instead of sorting.
constexpr int kSelRank = 512;

// s_sel[e] = 1 iff fewer than K words of w are larger than w[e]: Q words per
// thread in one sweep over w.
template <int Q>
__device__ __forceinline__ void sel_rank_sweep(const unsigned long long *w, int n, uint32_t K, uint8_t *s_sel)
{
    const int bd = (int)blockDim.x;
#pragma unroll 1
    for (int ub = 0; ub < n; ub += Q * bd) {
        const int e0 = ub + (int)threadIdx.x;
        if (e0 >= n) continue;                   // (a large block: most threads have none)
        unsigned long long we[Q];
        uint32_t r[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            we[q] = w[min(e0 + q * bd, n - 1)];
            r[q] = 0u;
        }
#pragma unroll 4
        for (int v = 0; v < n; ++v) {
            const unsigned long long wv = w[v];
#pragma unroll
            for (int q = 0; q < Q; ++q) r[q] += wv > we[q] ? 1u : 0u;
        }
#pragma unroll
        for (int q = 0; q < Q; ++q)
            if (e0 + q * bd < n) s_sel[e0 + q * bd] = r[q] < K ? 1 : 0;
    }
}

// The K largest of n <= kSelRank distinct words w (shared memory; key << 32 |
// ~index, so larger key first and lower index first among equal keys), their
// indices written to out in ascending index order: a word is among the K iff
// fewer than K words are larger.  One sweep over w ranks two words per thread,
// or four when there are more than two per thread (every thread reads the
// same word at the same time: a broadcast);
// the chosen indices are then compacted, and each one's place is the number
// of chosen indices below it -- a sweep over the K chosen, not over all n.
__device__ __forceinline__ void sel_rank_finish(const unsigned long long *w, int n, int32_t *out,
                                                uint32_t K)
{
    __shared__ uint8_t s_sel[kSelRank];
    __shared__ uint32_t s_ix[kSelRank];
    __shared__ uint32_t s_ws[32];
    const int bd = (int)blockDim.x;
    if (n <= 2 * bd)
        sel_rank_sweep<2>(w, n, K, s_sel);
    else
        sel_rank_sweep<4>(w, n, K, s_sel);
    __syncthreads();
    // the chosen indices, compacted in word order (thread t: words per t ..)
    const int per = (n + bd - 1) / bd;
    uint32_t c = 0, m = 0;
#pragma unroll 1
    for (int q = 0; q < per; ++q) {
        const int e = per * (int)threadIdx.x + q;
        if (e < n) c += s_sel[e];
    }
    uint32_t o = sel_excl_scan(c, s_ws, &m);
#pragma unroll 1
    for (int q = 0; q < per; ++q) {
        const int e = per * (int)threadIdx.x + q;
        if (e < n && s_sel[e]) s_ix[o++] = ~(uint32_t)(w[e] & 0xffffffffull);
    }
    __syncthreads();
#pragma unroll 1
    for (int t = threadIdx.x; t < (int)m; t += bd) {
        const uint32_t ia = s_ix[t];
        uint32_t pa = 0;
#pragma unroll 4
        for (int v = 0; v < (int)m; ++v) pa += s_ix[v] < ia ? 1u : 0u;
        out[pa] = (int32_t)ia;
    }
    __syncthreads();
}

// One block: the K indices from the candidate words (larger key first, lower
// index first among equal keys): ranked up to kSelRank words, else a bitonic
// sort descending, or the exact radix finish when more than kSelCap keys lie
// in or above the boundary bin; the K indices come out ascending.  sk: kSelCap
// words of shared memory.
__device__ __forceinline__ void sel_finish(const float *keys, int64_t p, const SelState *st,
                                           const unsigned long long *cand, uint32_t ncand,
                                           int32_t *out, uint32_t K, unsigned long long *sk,
                                           uint32_t *wsum, bool staged = false)
{
    if (ncand <= (uint32_t)kSelRank) {
        // (staged: the caller has copied the words into sk already)
        if (!staged)
#pragma unroll 1
            for (int i = threadIdx.x; i < (int)ncand; i += blockDim.x) sk[i] = __ldcg(&cand[i]);
        __syncthreads();
        sel_rank_finish(sk, (int)ncand, out, K);
        return;
    }
    if (ncand <= (uint32_t)kSelCap) {
        int P = 1;
        while (P < (int)ncand) P <<= 1;
        for (int i = threadIdx.x; i < P; i += blockDim.x) sk[i] = i < (int)ncand ? __ldcg(&cand[i]) : 0ull;
        __syncthreads();
#pragma unroll 1
        for (int size = 2; size <= P; size <<= 1) {               // bitonic, descending
#pragma unroll 1
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
#pragma unroll 1
                for (int i = threadIdx.x; i < P; i += blockDim.x) {
                    const int jx = i ^ stride;
                    if (jx > i) {
                        const bool up = (i & size) == 0;
                        const unsigned long long a = sk[i], b = sk[jx];
                        if ((a < b) == up) {
                            sk[i] = b;
                            sk[jx] = a;
                        }
                    }
                }
                __syncthreads();
            }
        }
#pragma unroll 1
        for (int i = threadIdx.x; i < (int)K; i += blockDim.x)
            out[i] = (int32_t)(~(uint32_t)(sk[i] & 0xffffffffull));
        __syncthreads();
    } else {
        sel_exact_block(keys, p, st, out, K, wsum);
    }
    sort_idx_body(out, (int)K);
}

// The same result as sel_finish for a block with few threads: with more than
// kSelRank candidates, a histogram of bits 19..10 of the boundary bin's keys
// finds the sub-bin holding the K-th key; only the keys above it and in it
// (every key that can be among the K, ties included) are ranked or sorted.  sk: room for kSelCap
// words plus `extra` words (the kept keys are compacted there); when they do
// not fit, all candidates are sorted as in sel_finish.
__device__ __forceinline__ void sel_finish_narrow(const float *keys, int64_t p, const SelState *st,
                                                  const unsigned long long *cand, uint32_t ncand,
                                                  int32_t *out, uint32_t K, unsigned long long *sk,
                                                  int extra, uint32_t *wsum, bool staged = false)
{
    __shared__ uint32_t h[1024];
    __shared__ uint32_t res[3];
    if (ncand <= (uint32_t)kSelRank || ncand > (uint32_t)kSelCap) {
        sel_finish(keys, p, st, cand, ncand, out, K, sk, wsum, staged && ncand <= (uint32_t)kSelRank);
        return;
    }
    const uint32_t bin = st->prefix >> 20;
#pragma unroll 1
    for (int b = threadIdx.x; b < 1024; b += blockDim.x) h[b] = 0;
    for (int i = threadIdx.x; i < (int)ncand; i += blockDim.x) sk[i] = __ldcg(&cand[i]);
    __syncthreads();
#pragma unroll 1
    for (int i = threadIdx.x; i < (int)ncand; i += blockDim.x) {
        const uint32_t key = (uint32_t)(sk[i] >> 32);
        if ((key >> 20) == bin) atomicAdd(&h[(key >> 10) & 0x3ffu], 1u);
    }
    __syncthreads();
    sel_find(h, 1024, st->need, wsum, res);
    const uint32_t lo = (bin << 20) | (res[0] << 10);          // keys >= lo can be among the K
    // compact the keys >= lo after the candidates (order kept: a block-wide scan)
    unsigned long long *kept = sk + kSelCap;
    uint32_t nk = 0;
#pragma unroll 1
    for (int base = 0; base < (int)ncand; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const uint32_t f = (i < (int)ncand && (uint32_t)(sk[i] >> 32) >= lo) ? 1u : 0u;
        uint32_t tot = 0;
        const uint32_t r = sel_excl_scan(f, wsum, &tot);
        if (f && nk + r < (uint32_t)extra) kept[nk + r] = sk[i];
        nk += tot;
    }
    __syncthreads();
    if (nk > (uint32_t)extra) {                                 // no room: sort them all
        sel_finish(keys, p, st, cand, ncand, out, K, sk, wsum);
        return;
    }
    if (nk <= (uint32_t)kSelRank) {
        sel_rank_finish(kept, (int)nk, out, K);
        return;
    }
    int P = 1;
    while (P < (int)nk) P <<= 1;
#pragma unroll 1
    for (int i = (int)nk + threadIdx.x; i < P; i += blockDim.x) kept[i] = 0ull;
    __syncthreads();
#pragma unroll 1
    for (int size = 2; size <= P; size <<= 1) {                 // bitonic, descending
#pragma unroll 1
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
#pragma unroll 1
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int jx = i ^ stride;
                if (jx > i) {
                    const bool up = (i & size) == 0;
                    const unsigned long long a = kept[i], b = kept[jx];
                    if ((a < b) == up) {
                        kept[i] = b;
                        kept[jx] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
#pragma unroll 1
    for (int i = threadIdx.x; i < (int)K; i += blockDim.x)
        out[i] = (int32_t)(~(uint32_t)(kept[i] & 0xffffffffull));
    __syncthreads();
    sort_idx_body(out, (int)K);
}

}  // namespace iht
