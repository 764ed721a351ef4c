// a2, tensor-core variant (tcgen05, sm_103a): g_j = v_j (S1_j - u_j (R - M_j)).
//
// The O(np) products S1_j = sum of dosage*r and M_j = sum of r over missing
// calls run on the 5th-generation tensor cores; the CUDA cores only turn the
// 2-bit codes into FP8 operands.  Decoding is the bottleneck of a CUDA-core
// version (about a dozen instructions per genotype), so the MMA unit absorbs
// the multiply-adds while the kernel stays bound by the HBM stream of packed
// genotypes.
//
// The dense part runs on the tensor cores (kind::f8f6f4, FP32 accumulate,
// M = 128 SNPs, N = 16, K = 32 samples):
//   A: the dosage map in E5M2.  The 2-bit code masked into bits 2-3 (the two
//      low exponent bits) reads 0, 2^-14, 2^-13, 2^-12 for codes 00, 01, 10,
//      11, i.e. 2^-14 (2x + [missing]); one AND, plus a shift for three of the
//      four fields, per output word of a 16-code input word (byte k of output
//      word j = sample 4k+j).
//   B: the residual as L = 5 E4M3 limbs, r ~ sum_l s_l q_l with s_l =
//      s_0 2^(-4l), in the same permuted sample order; limb l is row l of the
//      K-step's first 8-row group and the second group is one shared all-zero
//      group (8 bytes per sample).
// So D = 2^14 sum_l s_l acc[l] = sum of (2x + [missing]) r over the calls, and
// S1_j = sum over observed calls of x_ij r_i = (D - M_j) / 2.  The missing-call
// sums M_j (1-2 % of calls) come from a per-SNP list of missing sample offsets
// built at upload (a small warp-per-SNP pass before this one); they are needed
// for R - M_j anyway, and with them in the hot loop the data-dependent
// per-call branches cost more than the whole dense pass.
//
// Each tcgen05 instruction (an MMA or a commit) costs the SM's tensor front
// end about 45 cycles whatever the operand size, so the kernel issues one MMA
// per 4096 genotypes and one commit per four MMAs.
//
// Data movement (one persistent CTA per SM, four decoder warpgroups):
//   * producer warps stream 128-row x 64-byte tiles of packed genotypes
//     (256 samples of 128 SNPs) into shared memory with TMA (64-byte
//     swizzle, up to six stages per warpgroup, as many as shared memory
//     holds next to B and r: the stream is latency-bound, so the bytes in
//     flight per SM set the bandwidth), one producer warp per warpgroup;
//   * decoder thread r of a warpgroup owns row r of the tile: it reads its
//     16-byte chunks from shared memory (the swizzle makes the 8 rows of a
//     bank group distinct) and writes the FP8 map straight from registers to
//     tensor memory (tcgen05.st);
//   * one MMA warp per warpgroup issues the tcgen05.mma and commits;
//   * B (8 bytes per sample) stays in shared memory.
// Per warpgroup, tensor memory holds one 16-column accumulator and three
// 32-column A buffers of four K-steps each.  Every hand-off is an mbarrier
// (TMA transaction counts, tcgen05.commit for MMA completion), never a
// block-wide barrier, and every wait is bounded: a timeout is reported
// through TcParams::err instead of hanging.
#include <cuda.h>
#include <cuda_fp8.h>

#include "limbs.cuh"

namespace iht {

constexpr int kTcN = 16;
constexpr int kTcStepSamples = 32;                 // K of one MMA (bytes of FP8)
constexpr int kTcGroupBytes = 16;                  // packed bytes per chunk = 2 K-steps
constexpr int kTcStageBytes = 64;                  // packed bytes per row per TMA stage
constexpr int kTcStageSteps = 8;                   // K-steps per stage
constexpr int kTcMaxStages = 6;                    // TMA stages per warpgroup (as smem allows)
constexpr int kTcBufs = 3;                         // A buffers of kTcBufSteps K-steps
constexpr int kTcBufSteps = 4;                     // K-steps per A buffer (one commit)
constexpr int kTcNWG = 4;                          // decoder warpgroups per CTA
constexpr int kTcThreads = kTcNWG * (128 + 32 + 32);   // decoders, MMA warps, TMA warps
constexpr int kTcStageTile = 128 * kTcStageBytes;  // 8 KB

constexpr uint32_t kTcSpin = 1u << 24;             // bounded waits (each poll may suspend up to 128 ns)
constexpr int kTcHistBins = 2048;                  // bits 30..20 of |g| (the selection's histogram)


__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}


__global__ void __launch_bounds__(1024) k_limbs(const float *__restrict__ r32, int64_t n_pad,
                                                uint8_t *__restrict__ bimg, TcParams *prm,
                                                const int32_t *__restrict__ done)
{
    __shared__ float smax[32];
    __shared__ double red[32];
    if (done && *done) return;
    float m = 0.0f;
    for (int64_t i = threadIdx.x; i < n_pad; i += blockDim.x) m = fmaxf(m, fabsf(r32[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? smax[threadIdx.x] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) smax[0] = m;
    }
    __syncthreads();
    m = smax[0];
    const float s0 = limb_scale(m);
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n_pad; i += blockDim.x) {
        const float res = r32[i];
        acc += (double)res;
        limb_encode(res, s0, bimg, i);
    }
    // the trailing zero group may hold limbs of an earlier, longer residual
    for (int64_t b = threadIdx.x; b < 256; b += blockDim.x) bimg[256 + 256 * (n_pad >> 5) + b] = 0;
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) {             // (err is left as it is: set by a pass that timed out)
        prm->s0 = s0;
        prm->R = (float)acc;
    }
}

// ---------------------------------------------------------------------------
// mbarrier / TMA / tcgen05 helpers

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}

// true when the phase with the given parity has completed; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t a = smem_addr(bar);
    for (uint32_t it = 0; it < kTcSpin; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity), "n"(128)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// The decoders' waits, on barriers that have almost always passed by then:
// one poll in line, the bounded loop out of line (shared-space addresses).
__device__ __noinline__ bool mbar_wait_slow(uint32_t a, uint32_t parity)
{
    for (uint32_t it = 0; it < kTcSpin; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity), "n"(128)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ bool mbar_wait_fast(uint32_t a, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity), "n"(128)
        : "memory");
    return ok ? true : mbar_wait_slow(a, parity);
}

__device__ __forceinline__ void mbar_arrive_at(uint32_t a)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// An L2 policy that evicts first what it covers: the panel is read once per
// pass, so its lines go before anything else in L2 (the residual, the
// gradient, and the code and data of the kernels that run between passes).
__device__ __forceinline__ uint64_t l2_evict_first()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar, uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
        "%13,%14,%15,%16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
        "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void mma_f8(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc,
                                       uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

// K-major, no swizzle: core matrices of 8 rows x 16 bytes; LBO = 128 bytes
// between the two K halves, SBO = bytes between the two 8-row groups.
__device__ __forceinline__ uint64_t b_desc(uint32_t saddr, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// D FP32 (bit 4), A E5M2 (1 at bit 7), B E4M3 (0 at bit 10), K-major,
// N = 16 (N>>3 at bit 17), M = 128 (M>>4 at bit 24)
constexpr uint32_t kIdescF8 = (1u << 4) | (1u << 7) | ((uint32_t)(kTcN >> 3) << 17) |
                              ((uint32_t)(128 >> 4) << 24);

// Dosage map of one 16-code input word: each 2-bit field moved to bits 2-3 of
// its byte, E5M2 2^-14 (2x + [missing]).  Output word j holds samples 4k+j
// (byte k).
__device__ __forceinline__ void decode_word(uint32_t w, uint32_t *a)
{
    const uint32_t m = 0x0C0C0C0Cu;
    a[0] = (w << 2) & m;
    a[1] = w & m;
    a[2] = (w >> 2) & m;
    a[3] = (w >> 4) & m;
}

struct TcPipe {
    uint64_t tma_full[kTcMaxStages];   // producer -> decoders: stage landed (tx count)
    uint64_t tma_empty[kTcMaxStages];  // decoders -> producer: stage read (128 arrivals)
    uint64_t full[kTcBufs];         // decoders -> MMA warp: A buffer written (128 arrivals)
    uint64_t empty[kTcBufs];        // MMA warp -> decoders: MMAs reading the buffer done
    uint64_t accfull;               // MMA warp -> decoders: tile accumulators complete
    uint64_t accempty;              // decoders -> MMA warp: accumulators read out (128)
};

// One group of two 16-byte chunks (128 samples = 4 K-steps) of the row into A
// buffer `buf` with two 16-column stores, one per chunk (x1 is zero past the
// row's last chunk).
__device__ __forceinline__ void tc_put_group(uint32_t taddr, uint4 x0, uint4 x1)
{
    uint32_t v[16], u[16];
    decode_word(x0.x, &v[0]);
    decode_word(x0.y, &v[4]);
    decode_word(x0.z, &v[8]);
    decode_word(x0.w, &v[12]);
    tmem_st16(taddr, v);                 // (the second chunk decodes while this store runs)
    decode_word(x1.x, &u[0]);
    decode_word(x1.y, &u[4]);
    decode_word(x1.z, &u[8]);
    decode_word(x1.w, &u[12]);
    tmem_st16(taddr + 16, u);
}

// Read out the accumulator of local tile t and write g for this thread's row.
__device__ __forceinline__ bool tc_epilogue(TcPipe &P, uint32_t tb, uint32_t lane_off, int t,
                                            int64_t row, int64_t p, float s0, float R,
                                            const float *__restrict__ Mj,
                                            const float *__restrict__ u32,
                                            const float *__restrict__ v32, float *__restrict__ g,
                                            volatile int &abort_flag, uint32_t *s_hist, bool &nan)
{
    bool ok = true;
    if (!mbar_wait(&P.accfull, (uint32_t)t & 1u)) {
        abort_flag = 1;
        ok = false;
    }
    tc_fence_after();
    uint32_t acc[16];
    tmem_ld16(tb + lane_off, acc);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    tc_fence_before();
    mbar_arrive(&P.accempty);
    if (ok && row >= 0 && row < p) {
        float Ssum = 0.0f, s = s0;
#pragma unroll
        for (int l = 0; l < kTcLimbs; ++l) {
            Ssum = fmaf(s, __uint_as_float(acc[l]), Ssum);
            s *= 0.0625f;
        }
        const float D = 16384.0f * Ssum;
        const float gv = standardise_d(D, R, Mj[row], u32[row], v32[row]);
        g[row] = gv;
        if (s_hist) {
            const uint32_t key = __float_as_uint(gv) & 0x7fffffffu;
            nan |= key > 0x7f800000u;
            atomicAdd(&s_hist[key >> 20], 1u);
        }
    }
    return ok;
}

// Warp roles: warps 0..15 decoders (four warpgroups), warps 16..19 MMA issuers
// (one per warpgroup, lane 0), warps 20..23 TMA producers (one per warpgroup,
// lane 0; warp 20 also owns the tensor-memory allocation).  Tensor memory of warpgroup w, from column
// 128 w: accumulators D-even, S-even, D-odd, S-odd (16 each), then A buffers.
__global__ void __launch_bounds__(kTcThreads, 1) k_grad_tc(const __grid_constant__ CUtensorMap gmap,
                                                           int64_t p, int ngroups, int nst,
                                                           const uint8_t *__restrict__ bimg,
                                                           int bbytes, const float *__restrict__ Mj,
                                                           const float *__restrict__ u32,
                                                           const float *__restrict__ v32,
                                                           float *__restrict__ g, TcParams *prm,
                                                           const int32_t *__restrict__ done,
                                                           uint32_t *hist, uint32_t *hflag)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) TcPipe pipe[kTcNWG];
    __shared__ uint32_t s_hist[kTcHistBins];     // with hist: this CTA's counts of |g| bits 30..20
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    constexpr int kDecoders = kTcNWG * 128;
    constexpr int kProducerWarp = kTcNWG * 5;          // first TMA warp

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t *stages = smem;                      // kTcNWG * nst stages, 1024-aligned
    uint8_t *bsm = smem + kTcNWG * nst * kTcStageTile;   // B image

    if (tid == 0) {
        for (int w = 0; w < kTcNWG; ++w) {
            for (int b = 0; b < nst; ++b) {
                mbar_init(&pipe[w].tma_full[b], 1);
                mbar_init(&pipe[w].tma_empty[b], 128);
            }
            for (int b = 0; b < kTcBufs; ++b) {
                mbar_init(&pipe[w].full[b], 128);
                mbar_init(&pipe[w].empty[b], 1);
            }
            mbar_init(&pipe[w].accfull, 1);
            mbar_init(&pipe[w].accempty, 128);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (hist)
        for (int b = tid; b < kTcHistBins; b += blockDim.x) s_hist[b] = 0;
    if (warp == kProducerWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&tmem_base)),
                     "r"(kTcNWG * 128));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    const int64_t ntiles_all = (p + 127) / 128;
    const int ksteps = 2 * ngroups;
    const int spt = (ksteps + kTcStageSteps - 1) / kTcStageSteps;   // TMA stages per tile
    // warpgroup w of CTA b takes tiles w gridDim.x + b, then every tile_step on:
    // a round's tiles go first to one warpgroup of every CTA, so in the last,
    // partial round every SM keeps some warpgroups busy and each runs faster
    // with fewer decoders beside it
    const int64_t tile_step = (int64_t)gridDim.x * kTcNWG;

    // TMA producer state (lane 0 of the producer warps): the panel depends on
    // nothing the grids before this one write, so each producer fills its
    // first stages before this grid waits for them
    const bool producer = warp >= kProducerWarp && lane == 0;
    const int pw = warp - kProducerWarp;
    int64_t kk = 0, total = 0, ptile = 0;
    uint32_t pslot = 0, pphase = 0;
    int pst = 0;
    auto issue = [&](int64_t upto) {
        TcPipe &P = pipe[pw];
        const uint64_t policy = l2_evict_first();
        for (; kk < upto && !abort_flag; ++kk) {
            if (kk >= nst && !mbar_wait(&P.tma_empty[pslot], pphase ^ 1u)) {
                abort_flag = 1;
                break;
            }
            mbar_expect_tx(&P.tma_full[pslot], kTcStageTile);
            tma_load_2d(stages + (pw * nst + pslot) * kTcStageTile, &gmap, pst * kTcStageBytes,
                        (int)(ptile * 128), &P.tma_full[pslot], policy);
            if (++pslot == (uint32_t)nst) {
                pslot = 0;
                pphase ^= 1u;
            }
            if (++pst == spt) {
                pst = 0;
                ptile += tile_step;
            }
        }
    };
    if (producer) {
        const int64_t first = (int64_t)pw * gridDim.x + blockIdx.x;
        total = first < ntiles_all ? ((ntiles_all - 1 - first) / tile_step + 1) * spt : 0;
        ptile = first;
        issue(std::min<int64_t>(total, (int64_t)nst));
    }

    grid_dep_wait();   // the missing-call sums and limb image when launched programmatically
    const bool stop = done && *done;             // (the solve has stopped: no pass)
    if (!stop) {
        const uint4 *src = reinterpret_cast<const uint4 *>(bimg);
        uint4 *dst = reinterpret_cast<uint4 *>(bsm);
        for (int i = tid; i < bbytes / 16; i += blockDim.x) dst[i] = src[i];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    const int64_t ntiles = stop ? 0 : ntiles_all;
    if (stop) total = 0;                         // (the stages already requested are waited for below)

    if (tid < kDecoders) {
        // ------------------------------------------------------------ decoders
        const int w = warp >> 2, r = tid & 127;
        TcPipe &P = pipe[w];
        const uint32_t tb = tmem_base + (uint32_t)(w * 128);
        const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
        const float s0 = prm->s0, R = prm->R;
        uint32_t slot = 0, sphase = 0;          // TMA stage ring (slot, phase bit)
        uint32_t buf = 0, bphase = 0;           // A-buffer ring
        int T = 0;
        bool ok = true;
        bool nan = false;                       // a non-finite g among this thread's rows
        // swizzled offsets of the stage's four 16-byte chunks in this thread's row
        const int swz = (r >> 1) & 3;
        const uint32_t off0 = (uint32_t)((0 ^ swz) << 4), off1 = (uint32_t)((1 ^ swz) << 4);
        const uint32_t off2 = (uint32_t)((2 ^ swz) << 4), off3 = (uint32_t)((3 ^ swz) << 4);
        const uint32_t abase = tb + 32 + lane_off;
        // this row of slot 0, and the barriers' shared-space addresses (slot
        // or buffer b at + 8 b), set once
        const uint8_t *row0 = stages + (size_t)w * nst * kTcStageTile + (size_t)r * kTcStageBytes;
        const uint8_t *sp = row0;
        const uint32_t tfull0 = smem_addr(&P.tma_full[0]), tempty0 = smem_addr(&P.tma_empty[0]);
        const uint32_t afull0 = smem_addr(&P.full[0]), aempty0 = smem_addr(&P.empty[0]);
        // one A group (two chunks) into buffer buf
        auto put = [&](uint4 x0, uint4 x1) -> bool {
            // (a fresh barrier passes the wait on parity 1: the first round is free)
            if (!mbar_wait_fast(aempty0 + 8u * buf, bphase ^ 1u)) return false;
            tc_fence_after();
            tc_put_group(abase + 32u * buf, x0, x1);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            mbar_arrive_at(afull0 + 8u * buf);
            if (++buf == kTcBufs) {
                buf = 0;
                bphase ^= 1u;
            }
            return true;
        };
        // one TMA stage of nch chunks (4 but at the row's end): the row's chunks
        // into registers, the stage handed back to the producer before they are
        // decoded, then one A group per pair of chunks
        auto stage = [&](int nch) -> bool {
            if (!mbar_wait_fast(tfull0 + 8u * slot, sphase)) return false;
            const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
            uint4 xc[4];
            xc[0] = *reinterpret_cast<const uint4 *>(sp + off0);
            xc[1] = nch > 1 ? *reinterpret_cast<const uint4 *>(sp + off1) : zero;
            xc[2] = nch > 2 ? *reinterpret_cast<const uint4 *>(sp + off2) : zero;
            xc[3] = nch > 3 ? *reinterpret_cast<const uint4 *>(sp + off3) : zero;
            mbar_arrive_at(tempty0 + 8u * slot);
            sp += kTcStageTile;
            if (++slot == (uint32_t)nst) {
                slot = 0;
                sphase ^= 1u;
                sp = row0;
            }
            if (!put(xc[0], xc[1])) return false;
            return nch <= 2 || put(xc[2], xc[3]);
        };
        const int nfull = ngroups / 4, ntail = ngroups - 4 * nfull;   // stages of a row: full, then the rest
        for (int64_t tile = (int64_t)w * gridDim.x + blockIdx.x; tile < ntiles && ok; tile += tile_step, ++T) {
            const int64_t row = tile * 128 + r;
#pragma unroll 2
            for (int st = 0; st < nfull && ok; ++st) ok = stage(4);
            if (ok && ntail) ok = stage(ntail);
            if (!ok || abort_flag) {                     // this warp's wait gave up, or another's
                ok = false;
                break;
            }
            ok &= tc_epilogue(P, tb, lane_off, T, row, p, s0, R, Mj, u32, v32, g, abort_flag,
                              hist ? s_hist : nullptr, nan);
        }
        if (!ok) abort_flag = 1;
        if (nan && hflag) atomicOr(hflag, 1u);
    } else if (warp < kProducerWarp) {
        // ------------------------------------------------------------ MMA issuers
        const int w = warp - kTcNWG * 4;
        TcPipe &P = pipe[w];
        const uint32_t tb = tmem_base + (uint32_t)(w * 128);
        const uint32_t b_addr = smem_addr(bsm);
        const uint32_t za = 256u + 256u * (uint32_t)ksteps;   // trailing zero group
        if (lane == 0) {
            uint32_t buf = 0, use = 0;                                   // A-buffer ring
            uint64_t *last_bar = nullptr;            // barrier of the last commit, and its phase
            uint32_t last_par = 0;
            int T = 0;
            bool ok = true;
            const int ngrp = (ngroups + 1) / 2;                          // A groups per tile
            for (int64_t tile = (int64_t)w * gridDim.x + blockIdx.x; tile < ntiles && ok; tile += tile_step, ++T) {
                if (T >= 1) {
                    if (!mbar_wait(&P.accempty, (uint32_t)(T - 1) & 1u)) { abort_flag = 1; ok = false; }
                    tc_fence_after();
                }
                // B descriptor of K-step s: start b_addr + 256 (s + 1), 8-row-group
                // stride za - 256 (s + 1) (to the shared zero group); both fields
                // move by 256 bytes per step, so one 64-bit add advances it.
                uint64_t bd = b_desc(b_addr + 256u, za - 256u);
                constexpr uint64_t kBdStep = (uint64_t)(256 >> 4) - ((uint64_t)(256 >> 4) << 32);
                for (int gg = 0; gg < ngrp && ok; ++gg) {
                    if (!mbar_wait(&P.full[buf], use & 1u)) { abort_flag = 1; ok = false; break; }
                    tc_fence_after();
                    const int s0 = gg * kTcBufSteps;
                    const uint32_t a0 = tb + 32 + 32 * buf;
                    if (s0 + kTcBufSteps <= ksteps) {
#pragma unroll
                        for (int q = 0; q < kTcBufSteps; ++q) {
                            mma_f8(tb, a0 + 8 * q, bd, kIdescF8, (s0 + q) > 0 ? 1u : 0u);
                            bd += kBdStep;
                        }
                    } else {
                        for (int q = 0; s0 + q < ksteps; ++q) {
                            mma_f8(tb, a0 + 8 * q, bd, kIdescF8, (s0 + q) > 0 ? 1u : 0u);
                            bd += kBdStep;
                        }
                    }
                    mma_commit(&P.empty[buf]);
                    last_bar = &P.empty[buf];
                    last_par = use & 1u;
                    if (gg == ngrp - 1) mma_commit(&P.accfull);
                    if (++buf == kTcBufs) {
                        buf = 0;
                        use ^= 1u;
                    }
                }
                if (abort_flag) ok = false;
            }
            // MMAs still running after an abort write tensor memory: wait (bounded)
            // for the last commit, which tracks every MMA issued before it, so the
            // allocation is not released under them (on a normal exit it has
            // completed long ago)
            if (last_bar) mbar_wait(last_bar, last_par);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ TMA producers
        if (producer) {
            issue(total);
            // copies still in flight (after an abort, or when the solve had
            // stopped) are waited for, bounded
            TcPipe &P = pipe[pw];
            for (int64_t j = kk - nst; j < kk; ++j)
                if (j >= 0) mbar_wait(&P.tma_full[j % nst], (uint32_t)(j / nst) & 1u);
        }
        __syncwarp();
    }
    if (abort_flag && tid == 0) atomicExch(&prm->err, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (hist)                                    // this CTA's counts into the selection's histogram
        for (int b = tid; b < kTcHistBins; b += blockDim.x)
            if (s_hist[b]) atomicAdd(&hist[b], s_hist[b]);
    if (warp == kProducerWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"(kTcNWG * 128));
}

// ---------------------------------------------------------------------------

struct TcWork {
    uint8_t *bimg = nullptr;
    size_t bbytes = 0;
    TcParams *prm = nullptr;
    int dev = -1;
    cudaStream_t side = nullptr;            // missing-call sums beside the limb kernel
    cudaEvent_t fork = nullptr, join = nullptr;
};
static thread_local TcWork g_tc;

static int tc_ngroups(const iht_dataset *ds)
{
    return (int)(((ds->n + 3) / 4 + kTcGroupBytes - 1) / kTcGroupBytes);
}

static size_t tc_bbytes(const iht_dataset *ds) { return 512 + 256 * (size_t)(2 * tc_ngroups(ds)); }

constexpr size_t kTcSmemMax = 212 * 1024;   // dynamic; the static part (histogram, pipes) fits beside it

// TMA stages per warpgroup that fit beside B and r (0: the pass does not fit).
static int tc_stages(const iht_dataset *ds)
{
    const size_t fixed = tc_bbytes(ds);   // B
    if (fixed >= kTcSmemMax) return 0;
    const size_t ns = (kTcSmemMax - fixed) / ((size_t)kTcNWG * kTcStageTile);
    return (int)std::min<size_t>(ns, kTcMaxStages);
}

static size_t tc_smem(const iht_dataset *ds)
{
    return (size_t)kTcNWG * tc_stages(ds) * kTcStageTile + tc_bbytes(ds);
}

bool grad_tc_supported(const iht_dataset *ds)
{
    return tc_stages(ds) >= 2 && ds->p < (1ll << 31);
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                 const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                 const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Tensor map of the packed matrix: uint8 [p][stride], boxes of 64 bytes x
// 128 rows, 64-byte swizzle; rows past p read as zeros.
static int make_gmap(const iht_dataset *ds, CUtensorMap *map)
{
    static EncodeTiled encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        IHT_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                  cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !fn) return IHT_ECUDA;
        encode = (EncodeTiled)fn;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)ds->stride, (cuuint64_t)ds->p};
    const cuuint64_t strides[1] = {(cuuint64_t)ds->stride};
    const cuuint32_t box[2] = {(cuuint32_t)kTcStageBytes, 128};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, ds->G, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? IHT_OK : IHT_ECUDA;
}

// The calling thread's limb image and parameter block, sized for this dataset.
static int tc_ensure(iht_dataset *ds)
{
    cudaStream_t s = ds->ctx->stream;
    const size_t bbytes = tc_bbytes(ds);
    TcWork &w = g_tc;
    if (w.dev != ds->ctx->device || w.bbytes < bbytes) {
        if (w.bimg) cudaFree(w.bimg);
        if (w.prm) cudaFree(w.prm);
        if (w.dev != ds->ctx->device) {
            if (w.side) cudaStreamDestroy(w.side);
            if (w.fork) cudaEventDestroy(w.fork);
            if (w.join) cudaEventDestroy(w.join);
            w.side = nullptr;
            w.fork = w.join = nullptr;
        }
        w.bimg = nullptr;
        w.prm = nullptr;
        w.bbytes = 0;
        IHT_CUDA(dev_malloc(&w.bimg, bbytes));
        IHT_CUDA(dev_malloc(&w.prm, sizeof(TcParams)));
        IHT_CUDA(cudaMemsetAsync(w.bimg, 0, bbytes, s));   // zero groups and unused limb rows
        IHT_CUDA(cudaMemsetAsync(w.prm, 0, sizeof(TcParams), s));
        if (!w.side) {
            IHT_CUDA(cudaStreamCreateWithFlags(&w.side, cudaStreamNonBlocking));
            IHT_CUDA(cudaEventCreateWithFlags(&w.fork, cudaEventDisableTiming));
            IHT_CUDA(cudaEventCreateWithFlags(&w.join, cudaEventDisableTiming));
        }
        w.bbytes = bbytes;
        w.dev = ds->ctx->device;
    }
    return IHT_OK;
}

int grad_tc_limb_buffers(iht_dataset *ds, uint8_t **bimg, TcParams **prm, int64_t *nlim)
{
    if (!grad_tc_supported(ds)) return IHT_EINVAL;
    if (int rc = tc_ensure(ds)) return rc;
    *bimg = g_tc.bimg;
    *prm = g_tc.prm;
    *nlim = (int64_t)2 * tc_ngroups(ds) * kTcStepSamples;
    return IHT_OK;
}

// Residual -> limb image (and its scale and sum) for the next tensor-core pass,
// and the missing-call sums of r into Mj (p floats).
int prepare_grad_tc_to(iht_dataset *ds, const float *r32, float *Mj, const int32_t *done)
{
    if (!grad_tc_supported(ds)) return IHT_EINVAL;
    cudaStream_t s = ds->ctx->stream;
    const int ksteps = 2 * tc_ngroups(ds);
    if (int rc = tc_ensure(ds)) return rc;
    TcWork &w = g_tc;
    // The limb kernel (one block) and the missing-call sums read the same
    // residual and nothing of each other: the sums run on a side stream forked
    // from and joined back to the caller's (two branches of a captured graph).
    IHT_CUDA(cudaEventRecord(w.fork, s));
    IHT_CUDA(cudaStreamWaitEvent(w.side, w.fork, 0));
    ds->ctx->stream = w.side;
    const int rc = launch_missing_sums(ds, r32, Mj, done);
    ds->ctx->stream = s;
    if (rc) return rc;
    IHT_CUDA(cudaEventRecord(w.join, w.side));
    k_limbs<<<1, 1024, 0, s>>>(r32, (int64_t)ksteps * kTcStepSamples, w.bimg, w.prm, done);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    IHT_CUDA(cudaStreamWaitEvent(s, w.join, 0));
    return IHT_OK;
}

int prepare_grad_tc(iht_dataset *ds, const float *r32, const int32_t *done)
{
    return prepare_grad_tc_to(ds, r32, ds->ws->Mj, done);
}

bool grad_tc_shape_fits(const iht_dataset *ds, const int *params)
{
    return params[0] >= 2 && params[0] <= tc_stages(ds);
}

static int tc_launch(iht_dataset *ds, const CUtensorMap &map, int nst, float *g, const float *u32,
                     const float *v32, const float *Mj, const int32_t *done, uint32_t *hist = nullptr,
                     uint32_t *hflag = nullptr, bool programmatic = false)
{
    const int64_t tiles = (ds->p + 127) / 128;
    const int grid = (int)std::min<int64_t>((tiles + kTcNWG - 1) / kTcNWG, (int64_t)ds->ctx->num_sms);
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)grid);
    lc.blockDim = dim3(kTcThreads);
    lc.dynamicSmemBytes = (size_t)kTcNWG * nst * kTcStageTile + tc_bbytes(ds);
    lc.stream = ds->ctx->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = programmatic ? 1 : 0;
    const cudaError_t e = cudaLaunchKernelEx(&lc, k_grad_tc, map, ds->p, tc_ngroups(ds), nst,
                                             (const uint8_t *)g_tc.bimg, (int)tc_bbytes(ds), Mj, u32, v32, g,
                                             g_tc.prm, done, hist, hflag);
    note_launch();
    IHT_CUDA(e);
    return IHT_OK;
}

// First pass on a dataset shape: every stage count from 3 up to the most that
// fit, twice in turn (each run writes the same g), timed with events; the
// fastest is cached.  Nothing is cached when the solve had already stopped
// (the runs returned at once and timed nothing).
static int tc_tune(iht_dataset *ds, const CUtensorMap &map, float *g, const float *u32, const float *v32,
                   const float *Mj, const int32_t *done)
{
    cudaStream_t s = ds->ctx->stream;
    const int hi = tc_stages(ds), lo = std::min(3, hi);
    const int nc = hi - lo + 1, rounds = 2;
    TuneEvents te(2 * nc * rounds);
    IHT_CUDA(te.create());
    for (int r = 0; r < rounds; ++r)
        for (int c = 0; c < nc; ++c) {
            const int i = 2 * (r * nc + c);
            IHT_CUDA(cudaEventRecord(te.ev[i], s));
            if (int rc = tc_launch(ds, map, lo + c, g, u32, v32, Mj, done)) return rc;
            IHT_CUDA(cudaEventRecord(te.ev[i + 1], s));
        }
    int32_t stopped = 0;
    if (done) IHT_CUDA(cudaMemcpyAsync(&stopped, done, sizeof(stopped), cudaMemcpyDeviceToHost, s));
    IHT_CUDA(cudaStreamSynchronize(s));
    float best = 1e30f;
    int prm[kTuneParams] = {hi, 0, 0, 0};
    for (int r = 0; r < rounds; ++r)
        for (int c = 0; c < nc; ++c) {
            const float ms = te.ms(2 * (r * nc + c), 2 * (r * nc + c) + 1);
            if (ms < best) {
                best = ms;
                prm[0] = lo + c;
            }
        }
    if (!stopped) tune_store(ds, IHT_PASS_SINGLE, 0, prm, best, nc * rounds);
    return IHT_OK;
}

// The gradient pass proper (after prepare_grad_tc on the same stream) with
// explicit statistics and missing-call sums.  The TMA stage count is the
// cached tuned one (tuned on this call when none is cached, tuning is on and
// the stream is not being captured), else the most that fit.
int launch_grad_tc_main_with(iht_dataset *ds, const float *r32, float *g, const float *u32,
                             const float *v32, const float *Mj, const int32_t *done, uint32_t *hist,
                             uint32_t *hflag, bool programmatic)
{
    cudaStream_t s = ds->ctx->stream;
    CUtensorMap map;
    int rc = make_gmap(ds, &map);
    if (rc) return rc;
    static thread_local int cfg = -1;
    if (cfg != ds->ctx->device) {
        IHT_CUDA(cudaFuncSetAttribute(k_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kTcSmemMax));
        cfg = ds->ctx->device;
    }
    int prm[kTuneParams];
    if (tune_lookup(ds, IHT_PASS_SINGLE, 0, prm) && grad_tc_shape_fits(ds, prm))
        return tc_launch(ds, map, prm[0], g, u32, v32, Mj, done, hist, hflag, programmatic);
    if (!hist && autotune_enabled() && !stream_capturing(s)) return tc_tune(ds, map, g, u32, v32, Mj, done);
    return tc_launch(ds, map, tc_stages(ds), g, u32, v32, Mj, done, hist, hflag, programmatic);
}

// True when a pass launched now would take its settled shape (a tuned one is
// cached, or tuning is off): a graph captured now keeps what an eager pass
// would have used.
bool grad_tc_shape_settled(const iht_dataset *ds)
{
    int prm[kTuneParams];
    return !autotune_enabled() || (tune_lookup(ds, IHT_PASS_SINGLE, 0, prm) && grad_tc_shape_fits(ds, prm));
}

int launch_grad_tc_main(iht_dataset *ds, const float *r32, float *g, const int32_t *done,
                        uint32_t *hist, uint32_t *hflag, bool programmatic)
{
    return launch_grad_tc_main_with(ds, r32, g, ds->ws->u32, ds->ws->v32, ds->ws->Mj, done, hist, hflag,
                                    programmatic);
}

// Identifies the calling thread's pass scratch (changes when it is reallocated).
uint64_t grad_tc_scratch_id()
{
    return (uint64_t)(uintptr_t)g_tc.bimg ^ ((uint64_t)(uintptr_t)g_tc.prm << 1);
}

// Frees the calling thread's pass scratch (a server's worker before it exits).
void grad_tc_release_thread()
{
    TcWork &w = g_tc;
    if (w.bimg) cudaFree(w.bimg);
    if (w.prm) cudaFree(w.prm);
    if (w.side) cudaStreamDestroy(w.side);
    if (w.fork) cudaEventDestroy(w.fork);
    if (w.join) cudaEventDestroy(w.join);
    w = TcWork();
}

int launch_grad_tc(iht_dataset *ds, const float *r32, float *g, const int32_t *done)
{
    int rc = prepare_grad_tc(ds, r32, done);
    if (rc) return rc;
    return launch_grad_tc_main(ds, r32, g, done);
}

// Bounded-wait status of the tensor-core passes since the last reset (1 = a
// wait timed out); synchronises the stream.  An injected timeout
// (iht_fault_inject) writes the error word from the host first.
int grad_tc_status(iht_dataset *ds, int *timed_out)
{
    *timed_out = 0;
    if (!g_tc.prm) {                     // no tensor-core pass yet: nothing to read
        IHT_CUDA(cudaStreamSynchronize(ds->ctx->stream));
        return IHT_OK;
    }
    if (fault_take(IHT_FAULT_TIMEOUT))
        IHT_CUDA(cudaMemsetAsync(&g_tc.prm->err, 0x01, sizeof(int), ds->ctx->stream));
    TcParams h;
    IHT_CUDA(cudaMemcpyAsync(&h, g_tc.prm, sizeof(h), cudaMemcpyDeviceToHost, ds->ctx->stream));
    IHT_CUDA(cudaStreamSynchronize(ds->ctx->stream));
    *timed_out = h.err != 0;
    return IHT_OK;
}

// Clears the error word of the calling thread's tensor-core pass (stream-ordered).
int grad_tc_reset_status(iht_dataset *ds)
{
    if (g_tc.prm) IHT_CUDA(cudaMemsetAsync(&g_tc.prm->err, 0, sizeof(int), ds->ctx->stream));
    return IHT_OK;
}

}  // namespace iht
