// a3: top-K selection by |key| with ties to the lower index (Eq. ihta's
// projection P_{S_k}; the paper only asks for a fast sort, the tie rule is
// this library's reading).
//
// Radix select on the IEEE bits of |x| (for non-negative floats the unsigned
// bit pattern is monotone in the value):
//   pass 0 histograms bits 30..20 (2048 bins), pass 1 bits 19..10, pass 2
//   bits 9..0, each restricted to keys matching the digits fixed so far; a
//   single-CTA scan after each pass picks the digit where the running count
//   from the top reaches K.  The result is the K-th largest key T, the number
//   of keys above it, and how many keys equal to T are still needed.
// Collection writes every key > T (unordered) and the lowest-index keys == T
// (ordered by a per-chunk count and an exclusive scan), then one CTA sorts the
// K indices ascending.  NaN keys set SelState::err bit 0.
#include <mutex>

#include "common.cuh"

namespace iht {

__device__ __forceinline__ uint32_t sel_key(float x) { return __float_as_uint(x) & 0x7fffffffu; }

constexpr int kSelThreads = 256;
constexpr int kSelItems = 16;                          // consecutive indices per thread
constexpr int kSelChunk = kSelThreads * kSelItems;     // indices per collection block

__device__ __forceinline__ void sel_init_body(SelState *st, uint32_t K, uint32_t *hist)
{
    if (threadIdx.x == 0) {
        st->prefix = 0;
        st->mask = 0;
        st->need = K;
        st->count_gt = 0;
        st->n_gt = 0;
        st->err = 0;
    }
    for (int b = threadIdx.x; b < kSelBins; b += blockDim.x) hist[b] = 0;
}

__global__ void k_sel_init(SelState *st, uint32_t K, uint32_t *hist, const int32_t *done)
{
    if (done && *done) return;
    sel_init_body(st, K, hist);
}

// Histogram pass over keys[0..p) with the digits fixed so far; blockIdx.x
// strides over the keys.
__device__ __forceinline__ void sel_hist_body(const float *__restrict__ keys, int64_t p,
                                              SelState *st, uint32_t *hist, int shift,
                                              uint32_t dmask)
{
    __shared__ uint32_t sh[kSelBins];
    for (int b = threadIdx.x; b < kSelBins; b += blockDim.x) sh[b] = 0;
    __syncthreads();
    const uint32_t prefix = st->prefix, mask = st->mask;
    bool nan = false;
    // 16-byte loads, two in flight per thread, over the 16-byte aligned middle of
    // keys; the (at most 3 + 3) keys before and after it one at a time
    auto one = [&](float x) {
        const uint32_t k = sel_key(x);
        nan |= k > 0x7f800000u;
        if ((k & mask) == prefix) atomicAdd(&sh[(k >> shift) & dmask], 1u);
    };
    const int64_t head = std::min<int64_t>(p, (int64_t)((16u - ((uintptr_t)keys & 15u)) & 15u) >> 2);
    const float4 *k4 = reinterpret_cast<const float4 *>(keys + head);
    const int64_t n4 = (p - head) >> 2, step = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t q = tid;
    for (; q + step < n4; q += 2 * step) {
        const float4 a = k4[q], b = k4[q + step];
        one(a.x); one(a.y); one(a.z); one(a.w);
        one(b.x); one(b.y); one(b.z); one(b.w);
    }
    if (q < n4) {
        const float4 a = k4[q];
        one(a.x); one(a.y); one(a.z); one(a.w);
    }
    if (tid < head) one(keys[tid]);
    const int64_t t = head + (n4 << 2) + tid;
    if (t < p) one(keys[t]);
    if (nan && shift == 20) atomicOr(&st->err, 1u);
    __syncthreads();
    for (int b = threadIdx.x; b < kSelBins; b += blockDim.x)
        if (sh[b]) atomicAdd(&hist[b], sh[b]);
}

__global__ void __launch_bounds__(kSelThreads) k_sel_hist(const float *__restrict__ keys, int64_t p,
                                                          SelState *st, uint32_t *hist, int shift,
                                                          uint32_t dmask, const int32_t *done)
{
    if (done && *done) return;
    sel_hist_body(keys, p, st, hist, shift, dmask);
}

// Inclusive scan over a block of 1024 threads, 2 items per thread (fixed order).
__device__ __forceinline__ void scan2(uint32_t &a, uint32_t &b, uint32_t *wsum)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    b += a;
    uint32_t t = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += v;
    }
    if (lane == 31) wsum[wid] = t;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += v;
        }
        wsum[lane] = s;
    }
    __syncthreads();
    const uint32_t off = (t - b) + (wid ? wsum[wid - 1] : 0u);
    a += off;
    b += off;
    __syncthreads();
}

// Single block of 1024 threads: bins scanned from the top.
__device__ __forceinline__ void sel_scan_body(SelState *st, uint32_t *hist, int shift, uint32_t dmask,
                                              int nbins)
{
    __shared__ uint32_t wsum[32];
    const int t = threadIdx.x;
    // reversed order: position q holds bin nbins-1-q
    const int q0 = 2 * t, q1 = 2 * t + 1;
    const uint32_t h0 = q0 < nbins ? hist[nbins - 1 - q0] : 0u;
    const uint32_t h1 = q1 < nbins ? hist[nbins - 1 - q1] : 0u;
    uint32_t c0 = h0, c1 = h1;
    scan2(c0, c1, wsum);     // inclusive cumulative counts from the top
    const uint32_t need = st->need;
    __syncthreads();
    int hit = -1;
    uint32_t above = 0;
    if (q0 < nbins && c0 >= need && c0 - h0 < need) { hit = nbins - 1 - q0; above = c0 - h0; }
    if (q1 < nbins && c1 >= need && c1 - h1 < need) { hit = nbins - 1 - q1; above = c1 - h1; }
    if (hit >= 0) {
        st->count_gt += above;
        st->need = need - above;
        st->prefix |= (uint32_t)hit << shift;
        st->mask |= dmask << shift;
    }
    if (q0 < nbins) hist[nbins - 1 - q0] = 0;
    if (q1 < nbins) hist[nbins - 1 - q1] = 0;
}

__global__ void __launch_bounds__(1024) k_sel_scan(SelState *st, uint32_t *hist, int shift,
                                                   uint32_t dmask, int nbins, const int32_t *done)
{
    if (done && *done) return;
    sel_scan_body(st, hist, shift, dmask, nbins);
}

// Keys > T go to out[0..count_gt) in any order; per-chunk counts of keys == T
// (chunk = blockIdx.x).
__device__ __forceinline__ void sel_collect_gt_body(const float *__restrict__ keys, int64_t p,
                                                    SelState *st, int32_t *__restrict__ out,
                                                    uint32_t *__restrict__ chunk_eq)
{
    __shared__ uint32_t sh_eq;
    if (threadIdx.x == 0) sh_eq = 0;
    __syncthreads();
    const uint32_t T = st->prefix;
    const int64_t base = (int64_t)blockIdx.x * kSelChunk;
    uint32_t eq = 0;
    for (int it = 0; it < kSelItems; ++it) {
        const int64_t j = base + it * kSelThreads + threadIdx.x;
        if (j < p) {
            const uint32_t k = sel_key(keys[j]);
            if (k > T) out[atomicAdd(&st->n_gt, 1u)] = (int32_t)j;
            eq += k == T;
        }
    }
    if (eq) atomicAdd(&sh_eq, eq);
    __syncthreads();
    if (threadIdx.x == 0) chunk_eq[blockIdx.x] = sh_eq;
}

__global__ void __launch_bounds__(kSelThreads) k_sel_collect_gt(const float *__restrict__ keys,
                                                                int64_t p, SelState *st,
                                                                int32_t *__restrict__ out,
                                                                uint32_t *__restrict__ chunk_eq,
                                                                const int32_t *done)
{
    if (done && *done) return;
    sel_collect_gt_body(keys, p, st, out, chunk_eq);
}

// Exclusive scan of chunk_eq in place (single block of 1024 threads).
__device__ __forceinline__ void sel_scan_chunks_body(uint32_t *chunk_eq, int64_t nchunks)
{
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nchunks; base += 2048) {
        const int64_t i0 = base + 2 * threadIdx.x, i1 = i0 + 1;
        const uint32_t h0 = i0 < nchunks ? chunk_eq[i0] : 0u;
        const uint32_t h1 = i1 < nchunks ? chunk_eq[i1] : 0u;
        uint32_t c0 = h0, c1 = h1;
        scan2(c0, c1, wsum);
        const uint32_t cr = carry;
        if (i0 < nchunks) chunk_eq[i0] = cr + c0 - h0;
        if (i1 < nchunks) chunk_eq[i1] = cr + c1 - h1;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = cr + c1;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) k_sel_scan_chunks(uint32_t *chunk_eq, int64_t nchunks,
                                                          const int32_t *done)
{
    if (done && *done) return;
    sel_scan_chunks_body(chunk_eq, nchunks);
}

// The lowest-index keys == T, in index order, after the keys > T.
__device__ __forceinline__ void sel_collect_eq_body(const float *__restrict__ keys, int64_t p,
                                                    const SelState *st, int32_t *__restrict__ out,
                                                    const uint32_t *__restrict__ chunk_off)
{
    __shared__ uint32_t wsum[kSelThreads / 32];
    const uint32_t T = st->prefix, need = st->need, gt = st->count_gt;
    const uint32_t off0 = chunk_off[blockIdx.x];
    if (off0 >= need) return;                 // uniform over the block
    const int64_t base = (int64_t)blockIdx.x * kSelChunk + (int64_t)threadIdx.x * kSelItems;
    uint32_t mine = 0;
    for (int it = 0; it < kSelItems; ++it) {
        const int64_t j = base + it;
        mine += (j < p) && sel_key(keys[j]) == T;
    }
    // exclusive scan of `mine` over the block
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t t = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += v;
    }
    if (lane == 31) wsum[wid] = t;
    __syncthreads();
    uint32_t woff = 0;
    for (int w = 0; w < wid; ++w) woff += wsum[w];
    uint32_t rank = off0 + woff + t - mine;
    for (int it = 0; it < kSelItems && rank < need; ++it) {
        const int64_t j = base + it;
        if (j < p && sel_key(keys[j]) == T) out[gt + rank++] = (int32_t)j;
    }
}

__global__ void __launch_bounds__(kSelThreads) k_sel_collect_eq(const float *__restrict__ keys,
                                                                int64_t p, const SelState *st,
                                                                int32_t *__restrict__ out,
                                                                const uint32_t *__restrict__ chunk_off,
                                                                const int32_t *done)
{
    if (done && *done) return;
    sel_collect_eq_body(keys, p, st, out, chunk_off);
}

// Sort K (<= kMaxCand) indices ascending in one block (bitonic in shared memory).
__device__ __forceinline__ void sort_idx_body(int32_t *idx, int K)
{
    __shared__ int32_t s[kMaxCand];
    int P = 1;
    while (P < K) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) s[i] = i < K ? idx[i] : 0x7fffffff;
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
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
    for (int i = threadIdx.x; i < K; i += blockDim.x) idx[i] = s[i];
}

__global__ void __launch_bounds__(1024) k_sort_idx(int32_t *idx, int K, const int32_t *done)
{
    if (done && *done) return;
    sort_idx_body(idx, K);
}

// ---------------------------------------------------------------------------
// Batched selection: blockIdx.y (or blockIdx.x for the single-block steps)
// indexes the problem; each problem has its own keys, K, output and scratch.

__global__ void k_bsel_init(const SelJob *jobs)
{
    const SelJob &J = jobs[blockIdx.x];
    if (J.done && *J.done) return;
    sel_init_body(J.st, J.K, J.hist);
}

__global__ void __launch_bounds__(kSelThreads) k_bsel_hist(const SelJob *jobs, int64_t p, int shift,
                                                           uint32_t dmask)
{
    const SelJob &J = jobs[blockIdx.y];
    if (J.done && *J.done) return;
    sel_hist_body(J.keys, p, J.st, J.hist, shift, dmask);
}

__global__ void __launch_bounds__(1024) k_bsel_scan(const SelJob *jobs, int shift, uint32_t dmask,
                                                    int nbins)
{
    const SelJob &J = jobs[blockIdx.x];
    if (J.done && *J.done) return;
    sel_scan_body(J.st, J.hist, shift, dmask, nbins);
}

__global__ void __launch_bounds__(kSelThreads) k_bsel_collect_gt(const SelJob *jobs, int64_t p)
{
    const SelJob &J = jobs[blockIdx.y];
    if (J.done && *J.done) return;
    sel_collect_gt_body(J.keys, p, J.st, J.out, J.chunk_eq);
}

__global__ void __launch_bounds__(1024) k_bsel_scan_chunks(const SelJob *jobs, int64_t nchunks)
{
    const SelJob &J = jobs[blockIdx.x];
    if (J.done && *J.done) return;
    sel_scan_chunks_body(J.chunk_eq, nchunks);
}

__global__ void __launch_bounds__(kSelThreads) k_bsel_collect_eq(const SelJob *jobs, int64_t p)
{
    const SelJob &J = jobs[blockIdx.y];
    if (J.done && *J.done) return;
    sel_collect_eq_body(J.keys, p, J.st, J.out, J.chunk_eq);
}

__global__ void __launch_bounds__(1024) k_bsort_idx(const SelJob *jobs)
{
    const SelJob &J = jobs[blockIdx.x];
    if (J.done && *J.done) return;
    sort_idx_body(J.out, (int)J.K);
}

int64_t sel_nchunks(int64_t p) { return (p + kSelChunk - 1) / kSelChunk; }

// Top-K of |keys| for nb problems at once (jobs: device array of nb SelJob;
// every job's chunk_eq holds sel_nchunks(p) counts).
int select_topk_batch(iht_ctx *ctx, const SelJob *jobs, int nb, int64_t p)
{
    if (nb < 1) return IHT_OK;
    cudaStream_t s = ctx->stream;
    const int64_t nchunks = (p + kSelChunk - 1) / kSelChunk;
    const int hblocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(p, kSelThreads),
                                                                     ((int64_t)ctx->num_sms * 4 + nb - 1) / nb));
    k_bsel_init<<<nb, 256, 0, s>>>(jobs);
    const int shifts[3] = {20, 10, 0};
    const uint32_t dmasks[3] = {0x7ffu, 0x3ffu, 0x3ffu};
    for (int ps = 0; ps < 3; ++ps) {
        k_bsel_hist<<<dim3(hblocks, nb), kSelThreads, 0, s>>>(jobs, p, shifts[ps], dmasks[ps]);
        k_bsel_scan<<<nb, 1024, 0, s>>>(jobs, shifts[ps], dmasks[ps], (int)dmasks[ps] + 1);
    }
    k_bsel_collect_gt<<<dim3((unsigned)nchunks, nb), kSelThreads, 0, s>>>(jobs, p);
    k_bsel_scan_chunks<<<nb, 1024, 0, s>>>(jobs, nchunks);
    k_bsel_collect_eq<<<dim3((unsigned)nchunks, nb), kSelThreads, 0, s>>>(jobs, p);
    k_bsort_idx<<<nb, 1024, 0, s>>>(jobs);
    note_launch(11);
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

int ensure_selwork(iht_ctx *ctx, int64_t p)
{
    SelWork &w = ctx->sel;
    const int64_t nchunks = (p + kSelChunk - 1) / kSelChunk;
    if (!w.hist) {
        IHT_CUDA(cudaMalloc(&w.hist, sizeof(uint32_t) * kSelBins));
        IHT_CUDA(cudaMalloc(&w.st, sizeof(SelState)));
        IHT_CUDA(cudaMemsetAsync(w.hist, 0, sizeof(uint32_t) * kSelBins, ctx->stream));
    }
    if (nchunks > w.nchunks_cap) {
        if (w.chunk_eq) cudaFree(w.chunk_eq);
        w.chunk_eq = nullptr;
        w.nchunks_cap = 0;
        IHT_CUDA(cudaMalloc(&w.chunk_eq, sizeof(uint32_t) * nchunks));
        w.nchunks_cap = nchunks;
    }
    return IHT_OK;
}

int select_topk(iht_ctx *ctx, const float *keys, int64_t p, int32_t K, int32_t *out,
                const int32_t *done)
{
    SelWork *ws = &ctx->sel;
    cudaStream_t s = ctx->stream;
    if (K < 1 || K > p || K > kMaxCand) return IHT_EINVAL;
    const int64_t nchunks = (p + kSelChunk - 1) / kSelChunk;
    if (nchunks > ws->nchunks_cap) return IHT_EINVAL;
    const int hblocks = (int)std::min<int64_t>(ceil_div(p, kSelThreads), (int64_t)ctx->num_sms * 4);
    k_sel_init<<<1, 256, 0, s>>>(ws->st, (uint32_t)K, ws->hist, done);
    const int shifts[3] = {20, 10, 0};
    const uint32_t dmasks[3] = {0x7ffu, 0x3ffu, 0x3ffu};
    for (int ps = 0; ps < 3; ++ps) {
        k_sel_hist<<<hblocks, kSelThreads, 0, s>>>(keys, p, ws->st, ws->hist, shifts[ps], dmasks[ps],
                                                   done);
        k_sel_scan<<<1, 1024, 0, s>>>(ws->st, ws->hist, shifts[ps], dmasks[ps],
                                      (int)dmasks[ps] + 1, done);
    }
    k_sel_collect_gt<<<(int)nchunks, kSelThreads, 0, s>>>(keys, p, ws->st, out, ws->chunk_eq, done);
    k_sel_scan_chunks<<<1, 1024, 0, s>>>(ws->chunk_eq, nchunks, done);
    k_sel_collect_eq<<<(int)nchunks, kSelThreads, 0, s>>>(keys, p, ws->st, out, ws->chunk_eq, done);
    k_sort_idx<<<1, 1024, 0, s>>>(out, K, done);
    note_launch(11);
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free top-k (iht_topk_noalloc).
//
// For callers that must not allocate device memory: the scratch of the
// selection (radix histogram, selection state, per-chunk tie counts) lives in
// this file-scope device array, sized for p <= kNoAllocMaxP.  Every GPU that
// loads the library holds it (about 24 KB) until the process exits.  The array
// is shared by all calls on a device and keeps the last call's contents; the
// first kernel of each call clears the histogram and the state, and the chunk
// counts are written in full before they are read.  Calls that overlap on the
// GPU (different streams, or several host threads) race on it.

constexpr int64_t kNoAllocMaxP = int64_t(1) << 24;                 // 16 777 216 entries
constexpr int64_t kNoAllocChunks = kNoAllocMaxP / kSelChunk;      // 4096 tie-count chunks
constexpr size_t kNoAllocHist = sizeof(uint32_t) * kSelBins;      // 8 KB
constexpr size_t kNoAllocState = 256;                             // SelState, padded
constexpr size_t kNoAllocBytes = kNoAllocHist + kNoAllocState + sizeof(uint32_t) * kNoAllocChunks;

static __device__ __align__(256) unsigned char g_topk_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static unsigned char *g_noalloc_addr[kNoAllocMaxDevices] = {};
static int g_noalloc_sms[kNoAllocMaxDevices] = {};

// Device address of the scratch array on `device` (looked up once per device,
// with that device current; the caller's current device is restored).
static int noalloc_scratch(int device, unsigned char **addr, int *num_sms)
{
    if (device < 0 || device >= kNoAllocMaxDevices) return IHT_EINVAL;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        int prev = -1;
        IHT_CUDA(cudaGetDevice(&prev));
        IHT_CUDA(cudaSetDevice(device));
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_topk_scratch);
        int sms = 0;
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        cudaSetDevice(prev);
        if (e != cudaSuccess) {
            set_cuda_error(e, "cudaGetSymbolAddress(top-k scratch)");
            return IHT_ECUDA;
        }
        g_noalloc_addr[device] = static_cast<unsigned char *>(ptr);
        g_noalloc_sms[device] = sms;
    }
    *addr = g_noalloc_addr[device];
    *num_sms = g_noalloc_sms[device];
    return IHT_OK;
}

}  // namespace iht

extern "C" int iht_topk_noalloc(int device, void *stream, const float *w, int64_t p, int32_t k,
                                int32_t *idx_out)
{
    using namespace iht;
    if (!w || !idx_out || p < 1 || k < 1 || k > p || k > kMaxCand) return IHT_EINVAL;
    if (p > kNoAllocMaxP) return IHT_EINVAL;   // beyond the size of the static scratch
    unsigned char *scratch = nullptr;
    int sms = 0;
    int rc = noalloc_scratch(device, &scratch, &sms);
    if (rc) return rc;
    int prev = -1;
    IHT_CUDA(cudaGetDevice(&prev));
    if (prev != device) IHT_CUDA(cudaSetDevice(device));
    uint32_t *hist = reinterpret_cast<uint32_t *>(scratch);
    SelState *st = reinterpret_cast<SelState *>(scratch + kNoAllocHist);
    uint32_t *chunk_eq = reinterpret_cast<uint32_t *>(scratch + kNoAllocHist + kNoAllocState);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nchunks = (p + kSelChunk - 1) / kSelChunk;
    const int hblocks = (int)std::min<int64_t>(ceil_div(p, kSelThreads), (int64_t)sms * 4);
    k_sel_init<<<1, 256, 0, s>>>(st, (uint32_t)k, hist, nullptr);
    const int shifts[3] = {20, 10, 0};
    const uint32_t dmasks[3] = {0x7ffu, 0x3ffu, 0x3ffu};
    for (int ps = 0; ps < 3; ++ps) {
        k_sel_hist<<<hblocks, kSelThreads, 0, s>>>(w, p, st, hist, shifts[ps], dmasks[ps], nullptr);
        k_sel_scan<<<1, 1024, 0, s>>>(st, hist, shifts[ps], dmasks[ps], (int)dmasks[ps] + 1, nullptr);
    }
    k_sel_collect_gt<<<(int)nchunks, kSelThreads, 0, s>>>(w, p, st, idx_out, chunk_eq, nullptr);
    k_sel_scan_chunks<<<1, 1024, 0, s>>>(chunk_eq, nchunks, nullptr);
    k_sel_collect_eq<<<(int)nchunks, kSelThreads, 0, s>>>(w, p, st, idx_out, chunk_eq, nullptr);
    k_sort_idx<<<1, 1024, 0, s>>>(idx_out, k, nullptr);
    note_launch(11);
    const cudaError_t e = cudaGetLastError();
    if (prev != device) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        set_cuda_error(e, "iht_topk_noalloc launch");
        return IHT_ECUDA;
    }
    return IHT_OK;
}
