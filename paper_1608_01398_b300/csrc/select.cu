// a3: top-K selection by |key| with ties to the lower index (Eq. ihta's
// projection P_{S_k}; the paper only asks for a fast sort, the tie rule is
// this library's reading).
//
// Two launches per call (per problem in the batched form), no host round trip:
//   A  histograms bits 30..20 of |x| (2048 bins; for non-negative floats the
//      unsigned bit pattern is monotone in the value).  The last block to
//      finish (an atomic ticket) scans the bins from the top for the boundary
//      bin b: fewer than K keys lie above it, at least K at or above it.
//   B  copies every key in bin b or above -- typically a few hundred -- as the
//      64-bit word (key << 32 | ~index) into a candidate buffer; the last block
//      sorts the words descending (larger key first, lower index first among
//      equal keys), takes the first K indices and sorts them ascending.
// When more than kSelCap keys lie in or above the boundary bin (heavy ties),
// B's last block finishes alone with the exact radix select: bits 19..10 and
// 9..0 within the boundary bin give the K-th key T, then every key > T and the
// lowest-index keys == T.  The tickets, the histogram and the candidate count
// are zero again when a call ends (the scratch is zeroed once when allocated).
// A NaN key sets SelState::err bit 0 (the bit stays set until a caller clears
// it); its bit pattern orders above +Inf, so NaN keys are selected first.
#include <mutex>

#include "select_bodies.cuh"

namespace iht {

// Launch A: histogram of bits 30..20; the last block finds the boundary bin.
__device__ __forceinline__ void sel_count_body(const float *__restrict__ keys, int64_t p, SelState *st,
                                               uint32_t *hist, uint32_t K)
{
    __shared__ uint32_t sh[kSelBins];
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t res[3];
    __shared__ int last;
    for (int b = threadIdx.x; b < kSelBins; b += blockDim.x) sh[b] = 0;
    __syncthreads();
    bool nan = false;
    sel_each(keys, p, [&](float x, int64_t) {
        const uint32_t k = sel_key(x);
        nan |= k > 0x7f800000u;
        atomicAdd(&sh[k >> 20], 1u);
    });
    if (nan) atomicOr(&st->err, 1u);
    __syncthreads();
    for (int b = threadIdx.x; b < kSelBins; b += blockDim.x)
        if (sh[b]) atomicAdd(&hist[b], sh[b]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&st->ticket_a, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int b = threadIdx.x; b < kSelBins; b += blockDim.x) {
        sh[b] = __ldcg(&hist[b]);
        hist[b] = 0;                                  // clean for the next call
    }
    __syncthreads();
    sel_find(sh, kSelBins, K, wsum, res);
    if (threadIdx.x == 0) {
        st->prefix = res[0] << 20;
        st->mask = 0x7ffu << 20;
        st->count_gt = res[1];
        st->need = K - res[1];
        st->ncand = res[1] + res[2];
        st->n_gt = 0;
        st->ticket_a = 0;
    }
}

// Launch B: candidates at or above the boundary bin; the last block finishes.
// gS (optional): the single solve's support; the last block then also forms
// g_S and ||g_S||^2 (gather_gS_body) for the step size, saving a launch.
__device__ __forceinline__ void sel_pick_body(const float *__restrict__ keys, int64_t p, SelState *st,
                                              unsigned long long *cand, int32_t *out, uint32_t K,
                                              const int32_t *gS = nullptr, int gk = 0,
                                              double *gcoef = nullptr, Scalars *gsc = nullptr)
{
    __shared__ unsigned long long sk[kSelCap];
    __shared__ uint32_t wsum[32];
    __shared__ int last;
    const uint32_t ncand = st->ncand;
    const bool fast = ncand <= (uint32_t)kSelCap;
    if (fast) {
        const uint32_t lo = st->prefix;               // bin b << 20: keys >= lo are the candidates
        sel_each(keys, p, [&](float x, int64_t j) {
            const uint32_t k = sel_key(x);
            if (k >= lo) {
                const uint32_t slot = atomicAdd(&st->n_gt, 1u);
                if (slot < (uint32_t)kSelCap)
                    cand[slot] = ((unsigned long long)k << 32) | (unsigned long long)(~(uint32_t)j);
            }
        });
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&st->ticket_b, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    sel_finish(keys, p, st, cand, ncand, out, K, sk, wsum);
    if (threadIdx.x == 0) {
        st->n_gt = 0;
        st->ticket_b = 0;
    }
    if (gS) {
        __syncthreads();          // gS may be the output just written (HTP's step set)
        gather_gS_body(keys, gS, gk, gcoef, gsc);
    }
}

__global__ void __launch_bounds__(kSelAThreads) k_sel_count(const float *__restrict__ keys, int64_t p,
                                                            SelState *st, uint32_t *hist, uint32_t K,
                                                            const int32_t *done)
{
    if (done && *done) return;
    sel_count_body(keys, p, st, hist, K);
}

__global__ void __launch_bounds__(kSelBThreads) k_sel_pick(const float *__restrict__ keys, int64_t p,
                                                           SelState *st, unsigned long long *cand,
                                                           int32_t *out, uint32_t K, const int32_t *done,
                                                           const int32_t *gS, int gk, double *gcoef,
                                                           Scalars *gsc)
{
    if (done && *done) return;
    sel_pick_body(keys, p, st, cand, out, K, gS, gk, gcoef, gsc);
}

// Batched selection: blockIdx.y indexes the problem; each problem has its own
// keys, K, output and scratch.
__global__ void __launch_bounds__(kSelAThreads) k_bsel_count(const SelJob *jobs, int64_t p)
{
    const SelJob &J = jobs[blockIdx.y];
    if (J.done && *J.done) return;
    sel_count_body(J.keys, p, J.st, J.hist, J.K);
}

__global__ void __launch_bounds__(kSelBThreads) k_bsel_pick(const SelJob *jobs, int64_t p)
{
    const SelJob &J = jobs[blockIdx.y];
    if (J.done && *J.done) return;
    sel_pick_body(J.keys, p, J.st, J.cand, J.out, J.K);
}

static int sel_blocks(int64_t p, int num_sms, int nb)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((p + kSelKeysPerBlock - 1) / kSelKeysPerBlock,
                                                        ((int64_t)num_sms * 8 + nb - 1) / nb));
}

// Top-K of |keys| for nb problems at once (jobs: device array of nb SelJob
// whose scratch was zeroed when allocated).
int select_topk_batch(iht_ctx *ctx, const SelJob *jobs, int nb, int64_t p)
{
    if (nb < 1) return IHT_OK;
    cudaStream_t s = ctx->stream;
    const int blocks = sel_blocks(p, ctx->num_sms, nb);
    k_bsel_count<<<dim3(blocks, nb), kSelAThreads, 0, s>>>(jobs, p);
    k_bsel_pick<<<dim3(blocks, nb), kSelBThreads, 0, s>>>(jobs, p);
    note_launch(2);
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

int ensure_selwork(iht_ctx *ctx, int64_t p)
{
    (void)p;
    SelWork &w = ctx->sel;
    if (!w.hist) {
        IHT_CUDA(dev_malloc(&w.hist, sizeof(uint32_t) * kSelBins));
        IHT_CUDA(dev_malloc(&w.st, sizeof(SelState)));
        IHT_CUDA(dev_malloc(&w.cand, sizeof(unsigned long long) * kSelCap));
        IHT_CUDA(cudaMemsetAsync(w.hist, 0, sizeof(uint32_t) * kSelBins, ctx->stream));
        IHT_CUDA(cudaMemsetAsync(w.st, 0, sizeof(SelState), ctx->stream));
    }
    return IHT_OK;
}

int select_topk(iht_ctx *ctx, const float *keys, int64_t p, int32_t K, int32_t *out,
                const int32_t *done, const int32_t *gS, int gk, double *gcoef, Scalars *gsc)
{
    SelWork *ws = &ctx->sel;
    cudaStream_t s = ctx->stream;
    if (K < 1 || K > p || K > kMaxCand || !ws->hist) return IHT_EINVAL;
    const int blocks = sel_blocks(p, ctx->num_sms, 1);
    k_sel_count<<<blocks, kSelAThreads, 0, s>>>(keys, p, ws->st, ws->hist, (uint32_t)K, done);
    k_sel_pick<<<blocks, kSelBThreads, 0, s>>>(keys, p, ws->st, ws->cand, out, (uint32_t)K, done, gS, gk,
                                               gcoef, gsc);
    note_launch(2);
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free top-k (iht_topk_noalloc).
//
// For callers that must not allocate device memory: the scratch of the
// selection (histogram, selection state, candidate buffer) lives in this
// file-scope device array.  Every GPU that loads the library holds it (about
// 41 KB) until the process exits.  The first call on a device clears it on the
// caller's stream (cudaMemsetAsync, ahead of its kernels), and every call
// leaves it clean again; a call whose clear or launches fail marks the device
// so that the next call clears it again.  The array is shared by all calls on
// a device: calls that overlap on the GPU (different streams, or several host
// threads) race on it.  The call does not synchronise, so it cannot report NaN
// keys: they rank above +Inf (their bit patterns are larger), and the NaN bit
// of the selection state is cleared at the start of every call.

// The entry point's chosen fixed maximum p.  It is not set by the array: the
// histogram, the state and the candidate buffer have the same size for any p.
constexpr int64_t kNoAllocMaxP = int64_t(1) << 24;                 // 16 777 216 entries
constexpr size_t kNoAllocHist = sizeof(uint32_t) * kSelBins;      // 8 KB
constexpr size_t kNoAllocState = 256;                             // SelState, padded
constexpr size_t kNoAllocBytes = kNoAllocHist + kNoAllocState + sizeof(unsigned long long) * kSelCap;

static_assert(sizeof(SelState) <= kNoAllocState, "selection state must fit its slot");

static __device__ __align__(256) unsigned char g_topk_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static unsigned char *g_noalloc_addr[kNoAllocMaxDevices] = {};
static int g_noalloc_sms[kNoAllocMaxDevices] = {};
static bool g_noalloc_cleared[kNoAllocMaxDevices] = {};

// Device address of the scratch array on `device` (looked up once per device,
// with that device current; the caller's current device is restored).
// first: set while no call on the device has enqueued the clear yet (the
// caller clears the scratch on its stream, then calls noalloc_mark_cleared).
static int noalloc_scratch(int device, unsigned char **addr, int *num_sms, bool *first)
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
    *first = !g_noalloc_cleared[device];
    return IHT_OK;
}

static void noalloc_mark_cleared(int device, bool cleared)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    g_noalloc_cleared[device] = cleared;
}

}  // namespace iht

extern "C" int iht_topk_noalloc(int device, void *stream, const float *w, int64_t p, int32_t k,
                                int32_t *idx_out)
{
    using namespace iht;
    if (!w || !idx_out || p < 1 || k < 1 || k > p || k > kMaxCand) return IHT_EINVAL;
    if (p > kNoAllocMaxP) return IHT_EINVAL;   // above the entry point's fixed maximum
    unsigned char *scratch = nullptr;
    int sms = 0;
    bool first = false;
    int rc = noalloc_scratch(device, &scratch, &sms, &first);
    if (rc) return rc;
    int prev = -1;
    IHT_CUDA(cudaGetDevice(&prev));
    if (prev != device) IHT_CUDA(cudaSetDevice(device));
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *hist = reinterpret_cast<uint32_t *>(scratch);
    SelState *st = reinterpret_cast<SelState *>(scratch + kNoAllocHist);
    unsigned long long *cand = reinterpret_cast<unsigned long long *>(scratch + kNoAllocHist + kNoAllocState);
    cudaError_t e = first ? cudaMemsetAsync(scratch, 0, kNoAllocBytes, s)
                          : cudaMemsetAsync(&st->err, 0, sizeof(st->err), s);
    if (e != cudaSuccess) {
        if (prev != device) cudaSetDevice(prev);
        set_cuda_error(e, "iht_topk_noalloc scratch clear");
        return IHT_ECUDA;
    }
    if (first) noalloc_mark_cleared(device, true);
    const int blocks = sel_blocks(p, sms, 1);
    k_sel_count<<<blocks, kSelAThreads, 0, s>>>(w, p, st, hist, (uint32_t)k, nullptr);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_sel_pick<<<blocks, kSelBThreads, 0, s>>>(w, p, st, cand, idx_out, (uint32_t)k, nullptr,
                                                   nullptr, 0, nullptr, nullptr);
        e = cudaGetLastError();
    }
    note_launch(2);
    if (prev != device) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        noalloc_mark_cleared(device, false);   // the scratch may be left dirty: clear it next time
        set_cuda_error(e, "iht_topk_noalloc launch");
        return IHT_ECUDA;
    }
    return IHT_OK;
}
