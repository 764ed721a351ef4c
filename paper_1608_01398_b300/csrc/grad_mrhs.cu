// a7: multi-right-hand-side standardised gradient (tcgen05, sm_103a).
//
// b solves on one genotype matrix (q-fold cross-validation over a path of
// model sizes, Sec. 2.4; several phenotypes) each need g_c = Z_c^T r_c per
// iteration, with Z_c standardised over the solve's own rows.  Per column c
// and SNP j
//     g_cj = v_cj (S1_cj - u_cj (R_c - M_cj)),
// S1_cj = sum_i x_ij r_ci over observed calls, M_cj = sum of r_ci over the
// missing calls of SNP j, R_c = sum_i r_ci (r_c is zero off the solve's rows,
// so one dense product serves every row set).  The dense part S1 = X0^T R is a
// GEMM of the 2-bit matrix against the b residual columns: one pass over the
// packed genotypes serves all b solves.
//
// Operands (kind::f8f6f4, A E5M2, B E4M3, FP32 accumulate, M = 128 SNPs,
// K = 32), the same numbers as the single-column pass (grad_tc.cu), column by
// column:
//   A: the dosage map in tensor memory, decoded by CUDA-core warps from the
//      TMA-staged 2-bit codes: a code moved to bits 2-3 of a byte (the low
//      exponent bits) is the E5M2 value 2^-14 (2x + [missing]); output word j
//      of an input word holds samples 4k + j (byte k).
//   B: each residual column as 5 E4M3 limbs r ~ sum_l s_l q_l, s_l = s_0 2^-4l,
//      s_0 = 2^ceil(log2(max|r| / 448)) (the single-column pass's limbs), one
//      B row per limb (row 5c + l for column c), N = 5 b rounded up to 16,
//      stored per K-step in the canonical K-major layout (8-row x 16-byte core
//      matrices) in the same permuted sample order as A.
//   So D = 2^14 sum_l s_l acc_l (summed over l in the single-column order) is
//   the sum of (2x + [missing]) r over all calls, and S1 = (D - M) / 2.
//
// One persistent CTA per SM handles two 128-SNP tiles at a time, so every B
// chunk it streams from L2 feeds two MMAs.  Warps 0-15 decode (warps 8t..8t+7
// own tile t, thread = SNP row = tensor-memory lane; two groups of four per
// tile take alternate A buffers) and run the epilogue, warps 16 and 17 issue
// the MMAs of tiles 0 and 1 (one issuing warp per tile: with a single one,
// passes of few columns were bound by its MMA issue), warp 18 streams genotype
// tiles (TMA 2D, 64-byte swizzle), warp 19 streams B chunks (bulk copies; a
// chunk is free again once both tiles' MMAs reading it have completed).  Tensor memory (512
// columns): accumulator of tile t at column 256 t, its A buffers right after
// it.  The epilogue writes D; a second pass (k_miss_finalize) forms the
// missing-call sums from the per-SNP lists, S1 and g, so this kernel's
// epilogue only stores.  Every wait is bounded and reports a timeout through
// an error word instead of hanging.
#include <cuda.h>
#include <cuda_fp8.h>

#include "common.cuh"

namespace iht {

// A CTA takes kTiles 128-SNP tiles per step, each with its own MMA-issuing
// warp and its own kTiles-th of tensor memory, and kGroups decoder groups of
// 128 threads per tile (512 decoders either way): 2 tiles x 2 groups, or, for
// accumulators of at most 96 columns, 4 tiles x 1 group -- one MMA-issuing
// warp sustains about one MMA per few hundred cycles, so with few columns the
// pass is bound by the number of issuing warps per SM.
constexpr int kMrMaxTiles = 4;
constexpr int kMrDecoders = 512;                             // decoder / epilogue threads
constexpr int kMrBufArrivals = 128;                          // decoders that fill one tile's A buffer
constexpr int kMrMmaWarp = kMrDecoders / 32;                 // MMA warps kMrMmaWarp + t, one per tile
__host__ __device__ constexpr int mr_threads(int tiles) { return kMrDecoders + 32 * (tiles + 2); }
constexpr int kMrStepSamples = 32;          // K of one MMA
constexpr int kMrLimbs = 5;                 // E4M3 limbs per residual column
constexpr int kMrGStageBytes = 64;          // packed bytes per row per TMA stage (256 samples)
constexpr int kMrGTile = 128 * kMrGStageBytes;
constexpr int kMrMaxGStages = 8;          // genotype stages (launch parameter ngs <= this)
constexpr int kMrChunkSteps = 4;            // K-steps per B chunk
constexpr int kMrMaxBStages = 6;
constexpr int kMrMaxBufs = 8;               // A buffers of 2 K-steps
constexpr int kMrMaxN = 224;                // accumulator columns per tile
constexpr int kMrMaxCols = kMrMaxN / kMrLimbs;   // residual columns per pass (44)
constexpr size_t kMrSmemMax = 220 * 1024;
constexpr uint32_t kMrSpin = 1u << 24;             // bounded waits (each poll may suspend up to 128 ns)

__device__ __forceinline__ uint32_t mr_smem(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// ---------------------------------------------------------------------------
// Residual columns -> E4M3 limb image.  One block per column; the scale, the
// limbs and the sum R (FP64, fixed order) follow the single-column pass's
// arithmetic exactly.

// Byte offset of sample i, limb row q: K-step s = i / 32; inside the step,
// sample 16 wi + 4 k + j sits at K position 4 (4 wi + j) + k, the order in
// which the decoded A words hold it.
__device__ __forceinline__ int64_t mr_b_offset(int64_t i, int q, int N)
{
    const int64_t s = i >> 5;
    const int ii = (int)(i & 31);
    const int wi = ii >> 4, q16 = ii & 15;
    const int k = q16 >> 2, j = q16 & 3;
    const int kpos = 4 * (4 * wi + j) + k;
    return s * (int64_t)N * 32 + (q >> 3) * 256 + (kpos >> 4) * 128 + (q & 7) * 16 + (kpos & 15);
}

__global__ void __launch_bounds__(1024) k_mr_limbs(MrCol *cols, int64_t nsamp, int N,
                                                   uint8_t *__restrict__ bimg)
{
    __shared__ float smax[32];
    __shared__ double red[32];
    MrCol &C = cols[blockIdx.x];
    const float *__restrict__ r = C.r32;
    float m = 0.0f;
    for (int64_t i = threadIdx.x; i < nsamp; i += blockDim.x) m = fmaxf(m, fabsf(r[i]));
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
    float s0 = 1.0f;
    if (m > 0.0f) {
        int e;
        frexpf(m / 448.0f, &e);          // m/448 <= 2^e
        s0 = ldexpf(1.0f, e);
    }
    const int q0 = kMrLimbs * blockIdx.x;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < nsamp; i += blockDim.x) {
        float res = r[i];
        float sc = s0;
        acc += (double)res;
#pragma unroll
        for (int l = 0; l < kMrLimbs; ++l) {
            const __nv_fp8_e4m3 q(res / sc);
            const float qf = (float)q;
            bimg[mr_b_offset(i, q0 + l, N)] = q.__x;
            res -= sc * qf;
            sc *= 0.0625f;
        }
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) {
        C.scale = s0;                    // limb l scale: s0 16^-l; D = 2^14 sum_l s_l acc_l
        C.R = (float)acc;
    }
}

// ---------------------------------------------------------------------------
// mbarrier / TMA / tcgen05 helpers (all waits bounded)

__device__ __forceinline__ void mr_bar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mr_smem(bar)), "r"(count));
}

__device__ __forceinline__ bool mr_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t a = mr_smem(bar);
    for (uint32_t it = 0; it < kMrSpin; ++it) {
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

__device__ __forceinline__ void mr_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mr_smem(bar)) : "memory");
}

__device__ __forceinline__ void mr_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mr_smem(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mr_tma_2d(void *dst, const CUtensorMap *map, int x, int y,
                                          uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
        "%3}], [%4];" ::"r"(mr_smem(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mr_smem(bar))
        : "memory");
}

__device__ __forceinline__ void mr_bulk(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            mr_smem(dst)),
        "l"(src), "r"(bytes), "r"(mr_smem(bar))
        : "memory");
}

__device__ __forceinline__ void mr_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void mr_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mr_st32(uint32_t taddr, const uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
        "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
        "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]),
        "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]),
        "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}

__device__ __forceinline__ void mr_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
        "%13,%14,%15,%16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
        "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void mr_ld16(uint32_t taddr, uint32_t (&v)[16])
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

__device__ __forceinline__ void mr_mma(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc,
                                       uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mr_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     mr_smem(bar))
                 : "memory");
}

// K-major, no swizzle: LBO 128 bytes (the two K halves), SBO 256 bytes (8-row groups).
__device__ __forceinline__ uint64_t mr_b_desc(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) |
           ((uint64_t)(256u >> 4) << 32) | (1ull << 46);
}

// E5M2 dosage map of one word of 16 codes (as the single-column pass): each
// 2-bit field in bits 2-3 of its byte, value 2^-14 (2x + [missing]); output j
// holds samples 4k + j (byte k).
__device__ __forceinline__ void mr_decode(uint32_t w, uint32_t *a)
{
    const uint32_t m = 0x0C0C0C0Cu;
    a[0] = (w << 2) & m;
    a[1] = w & m;
    a[2] = (w >> 2) & m;
    a[3] = (w >> 4) & m;
}

struct MrPipe {
    uint64_t gfull[kMrMaxGStages], gempty[kMrMaxGStages];
    uint64_t bfull[kMrMaxBStages], bempty[kMrMaxBStages];   // B chunks: shared by the tiles
    uint64_t afull[kMrMaxTiles][kMrMaxBufs], aempty[kMrMaxTiles][kMrMaxBufs];
    uint64_t accfull[kMrMaxTiles], accempty[kMrMaxTiles];
};

template <bool kPairs, int kTiles, int kGroups>
__global__ void __launch_bounds__(mr_threads(kTiles), 1) k_grad_mrhs(
    const __grid_constant__ CUtensorMap gmap, int64_t p, int ksteps, int N, int ncols, int nbufs,
    int nbst, int ngs, const uint8_t *__restrict__ bimg, const MrCol *__restrict__ cols,
    uint32_t idesc, int *err)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ MrPipe pipe;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;

    static_assert(kTiles * kGroups * 128 == kMrDecoders && kTiles <= kMrMaxTiles, "decoder layout");
    constexpr int kGWarp = kMrMmaWarp + kTiles;                // genotype TMA warp (B warp after it)
    constexpr uint32_t kTmemPerTile = 512u / kTiles;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t *gst = smem;                                        // ngs x kTiles tiles x 8 KB
    uint8_t *bst = smem + ngs * kTiles * kMrGTile;              // nbst x chunk
    const uint32_t chunk_bytes = (uint32_t)kMrChunkSteps * (uint32_t)N * 32u;
    const uint32_t step_bytes = (uint32_t)N * 32u;

    if (tid == 0) {
        for (int s = 0; s < ngs; ++s) {
            mr_bar_init(&pipe.gfull[s], 1);
            mr_bar_init(&pipe.gempty[s], kMrDecoders);
        }
        for (int s = 0; s < nbst; ++s) {
            mr_bar_init(&pipe.bfull[s], 1);
            mr_bar_init(&pipe.bempty[s], kTiles);             // one commit per tile's MMA warp
        }
        for (int t = 0; t < kTiles; ++t) {
            for (int b = 0; b < nbufs; ++b) {
                mr_bar_init(&pipe.afull[t][b], kMrBufArrivals);
                mr_bar_init(&pipe.aempty[t][b], 1);
            }
            mr_bar_init(&pipe.accfull[t], 1);
            mr_bar_init(&pipe.accempty[t], kMrDecoders / kTiles);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMrMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
            mr_smem(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    mr_fence_before();
    __syncthreads();
    mr_fence_after();

    const int64_t ntiles = (p + 128 * kTiles - 1) / (128 * kTiles);
    const int spt = (ksteps + 7) / 8;                   // genotype stages per tile (8 K-steps each)
    const int cpt = ksteps / kMrChunkSteps;             // B chunks per tile

    // Ring positions advance by increment and compare (slot, phase bit): the
    // single-thread roles issue work every few hundred cycles, so no division
    // or modulo sits on their path.
    if (tid < kMrDecoders) {
        // ------------------------------------------------------- decoders + epilogue
        // warps 4 kGroups t .. serve tile t; with two groups, group dg = 0 fills
        // the even A buffers of the sequence and dg = 1 the odd ones, so two
        // buffers are in flight per lane quarter and each group's latency chain
        // (decode, tcgen05.st, wait, arrive) overlaps the other's
        const int t = warp / (4 * kGroups), dg = (warp >> 2) % kGroups, r = tid & 127;
        const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
        const uint32_t tb = tmem_base + kTmemPerTile * (uint32_t)t + lane_off;
        const uint32_t abase = tb + (uint32_t)N;
        const int swz = (r >> 1) & 3;
        uint32_t gslot = 0, gphase = 0;           // genotype stage ring
        // A buffer ring position of this group's next buffer (sequence number aseq)
        // (pairs: group dg's first pair is pair dg, buffers 2 dg and 2 dg + 1)
        const uint32_t first = kPairs ? 2u * (uint32_t)dg : (uint32_t)dg;
        uint32_t aslot = first % (uint32_t)nbufs, aphase = first / (uint32_t)nbufs;
        uint32_t aseq = first;
        int T = 0;
        bool ok = true;
        uint32_t gseq = 0;                         // sequence number of the stage's first buffer
        for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++T) {
            int left = ksteps >> 1;                 // A buffers (2 K-steps, 16 packed bytes) left in the tile
            for (int st = 0; st < spt && ok; ++st) {
                if (!mr_wait(&pipe.gfull[gslot], gphase)) {
                    abort_flag = 1;
                    ok = false;
                    break;
                }
                const uint8_t *rowp = gst + (gslot * kTiles + t) * kMrGTile + r * kMrGStageBytes;
                const int nb = min(4, left);
                left -= nb;
                if (kPairs) {
                    // group dg fills the buffer pairs (2 adjacent buffers, 128
                    // samples, one 32-column store) whose pair number has parity
                    // dg; buffers per tile and per stage are even, so no pair
                    // straddles a stage or the ring's end (nbufs even)
                    for (int q2 = (int)(((uint32_t)dg - (gseq >> 1)) & (kGroups - 1)); 2 * q2 < nb; q2 += kGroups) {
                        if (aseq >= (uint32_t)nbufs) {
                            if (!mr_wait(&pipe.aempty[t][aslot], aphase ^ 1u) ||
                                !mr_wait(&pipe.aempty[t][aslot + 1], aphase ^ 1u)) {
                                abort_flag = 1;
                                ok = false;
                                break;
                            }
                            mr_fence_after();
                        }
                        const uint4 x0 = *reinterpret_cast<const uint4 *>(rowp + (((2 * q2) ^ swz) << 4));
                        const uint4 x1 = *reinterpret_cast<const uint4 *>(rowp + (((2 * q2 + 1) ^ swz) << 4));
                        uint32_t v[32];
                        mr_decode(x0.x, &v[0]);
                        mr_decode(x0.y, &v[4]);
                        mr_decode(x0.z, &v[8]);
                        mr_decode(x0.w, &v[12]);
                        mr_decode(x1.x, &v[16]);
                        mr_decode(x1.y, &v[20]);
                        mr_decode(x1.z, &v[24]);
                        mr_decode(x1.w, &v[28]);
                        mr_st32(abase + 16u * aslot, v);
                        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                        mr_fence_before();
                        mr_arrive(&pipe.afull[t][aslot]);
                        mr_arrive(&pipe.afull[t][aslot + 1]);
                        aseq += 2 * kGroups;
                        aslot += 2 * kGroups;
                        while (aslot >= (uint32_t)nbufs) {
                            aslot -= (uint32_t)nbufs;
                            aphase ^= 1u;
                        }
                    }
                } else
                // group dg fills the buffers whose sequence number is dg mod kGroups
                for (int q4 = (int)(((uint32_t)dg - gseq) & (kGroups - 1)); q4 < nb; q4 += kGroups) {
                    if (aseq >= (uint32_t)nbufs) {
                        if (!mr_wait(&pipe.aempty[t][aslot], aphase ^ 1u)) {
                            abort_flag = 1;
                            ok = false;
                            break;
                        }
                        mr_fence_after();
                    }
                    const uint4 x = *reinterpret_cast<const uint4 *>(rowp + ((q4 ^ swz) << 4));
                    uint32_t v[16];
                    mr_decode(x.x, &v[0]);
                    mr_decode(x.y, &v[4]);
                    mr_decode(x.z, &v[8]);
                    mr_decode(x.w, &v[12]);
                    mr_st16(abase + 16u * aslot, v);
                    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                    mr_fence_before();
                    mr_arrive(&pipe.afull[t][aslot]);
                    aseq += kGroups;
                    aslot += kGroups;
                    while (aslot >= (uint32_t)nbufs) {       // at most twice (nbufs >= 2)
                        aslot -= (uint32_t)nbufs;
                        aphase ^= 1u;
                    }
                }
                gseq += (uint32_t)nb;
                mr_arrive(&pipe.gempty[gslot]);
                if (++gslot == (uint32_t)ngs) {
                    gslot = 0;
                    gphase ^= 1u;
                }
                if (abort_flag) ok = false;
            }
            if (!ok) break;
            // epilogue: D of each column for this thread's SNP
            if (!mr_wait(&pipe.accfull[t], (uint32_t)T & 1u)) {
                abort_flag = 1;
                ok = false;
                break;
            }
            mr_fence_after();
            const int64_t j = tile * (128 * kTiles) + 128 * t + r;
            {
                // the groups take halves of the solves (one group: all); solve c's
                // limbs are the accumulator columns 5c .. 5c+4, combined in limb
                // order as the single-column epilogue does: D = 2^14 sum_l s0 16^-l acc_l
                const int half = kGroups == 1 ? ncols : (ncols + 1) / 2;
                const int c_lo = dg == 0 ? 0 : half, c_hi = dg == 0 ? half : ncols;
                int c = c_lo, l = 0;
                float ssum = 0.0f, sc = c < c_hi ? cols[c].scale : 0.0f;
                const int col_lo = kMrLimbs * c_lo, col_hi = kMrLimbs * c_hi;
                for (int cg = col_lo >> 4; (cg << 4) < col_hi; ++cg) {
                    uint32_t acc[16];
                    mr_ld16(tb + 16u * cg, acc);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int col = 16 * cg + e;
                        if (col < col_lo || col >= col_hi) continue;
                        ssum = fmaf(sc, __uint_as_float(acc[e]), ssum);
                        sc *= 0.0625f;
                        if (++l == kMrLimbs) {
                            if (j < p) cols[c].g[j] = 16384.0f * ssum;     // D
                            ++c;
                            l = 0;
                            ssum = 0.0f;
                            sc = c < c_hi ? cols[c].scale : 0.0f;
                        }
                    }
                }
            }
            mr_fence_before();
            mr_arrive(&pipe.accempty[t]);
        }
    } else if (warp < kGWarp) {
        // ------------------------------------------------------- MMA issuers (one per tile)
        const int t = warp - kMrMmaWarp;
        if (lane == 0) {
            uint32_t aslot = 0, aphase = 0, bslot = 0, bphase = 0;
            uint64_t *last_bar = nullptr;           // barrier of the last commit, and its phase
            uint32_t last_par = 0;
            int T = 0;
            bool ok = true;
            const uint32_t b0 = mr_smem(bst);
            const uint32_t tb = tmem_base + kTmemPerTile * (uint32_t)t;
            for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++T) {
                if (T >= 1) {
                    if (!mr_wait(&pipe.accempty[t], (uint32_t)(T - 1) & 1u)) { abort_flag = 1; break; }
                    mr_fence_after();
                }
                for (int ch = 0; ch < cpt && ok; ++ch) {
                    if (!mr_wait(&pipe.bfull[bslot], bphase)) { abort_flag = 1; ok = false; break; }
                    uint32_t baddr = b0 + bslot * chunk_bytes;
#pragma unroll
                    for (int h = 0; h < kMrChunkSteps / 2; ++h) {     // two A buffers per chunk
                        if (!mr_wait(&pipe.afull[t][aslot], aphase)) { abort_flag = 1; ok = false; break; }
                        mr_fence_after();
#pragma unroll
                        for (int s2 = 0; s2 < 2; ++s2) {
                            const uint32_t acc = (ch | h | s2) ? 1u : 0u;
                            mr_mma(tb, tb + (uint32_t)N + 16u * aslot + 8u * (uint32_t)s2, mr_b_desc(baddr),
                                   idesc, acc);
                            baddr += step_bytes;
                        }
                        mr_commit(&pipe.aempty[t][aslot]);
                        last_bar = &pipe.aempty[t][aslot];
                        last_par = aphase;
                        if (++aslot == (uint32_t)nbufs) {
                            aslot = 0;
                            aphase ^= 1u;
                        }
                    }
                    if (!ok) break;
                    mr_commit(&pipe.bempty[bslot]);
                    if (++bslot == (uint32_t)nbst) {
                        bslot = 0;
                        bphase ^= 1u;
                    }
                }
                if (!ok) break;
                mr_commit(&pipe.accfull[t]);
                if (abort_flag) ok = false;
            }
            // MMAs still running after an abort write tensor memory: wait (bounded)
            // for the last commit, which tracks every MMA issued before it, so the
            // allocation is not released under them (on a normal exit it has
            // completed long ago)
            if (last_bar) mr_wait(last_bar, last_par);
        }
        __syncwarp();
    } else if (warp == kGWarp) {
        // ------------------------------------------------------- genotype tiles (TMA)
        if (lane == 0) {
            uint32_t slot = 0, phase = 0;
            int64_t issued = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                const int y0 = (int)(tile * (128 * kTiles));
                for (int st = 0; st < spt; ++st, ++issued) {
                    if (abort_flag || (issued >= ngs && !mr_wait(&pipe.gempty[slot], phase ^ 1u))) {
                        abort_flag = 1;
                        ok = false;
                        break;
                    }
                    mr_expect_tx(&pipe.gfull[slot], (uint32_t)(kTiles * kMrGTile));
#pragma unroll
                    for (int t = 0; t < kTiles; ++t)
                        mr_tma_2d(gst + (slot * kTiles + t) * kMrGTile, &gmap, st * kMrGStageBytes,
                                  y0 + 128 * t, &pipe.gfull[slot]);
                    if (++slot == (uint32_t)ngs) {
                        slot = 0;
                        phase ^= 1u;
                    }
                }
            }
            // copies still in flight after an abort: wait for them (bounded)
            for (int64_t q = issued - ngs; q < issued; ++q)
                if (q >= 0) mr_wait(&pipe.gfull[q % ngs], (uint32_t)(q / ngs) & 1u);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------- B chunks (bulk copies)
        if (lane == 0) {
            uint32_t slot = 0, phase = 0;
            int64_t issued = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                const uint8_t *src = bimg;
                for (int ch = 0; ch < cpt; ++ch, ++issued) {
                    if (abort_flag || (issued >= nbst && !mr_wait(&pipe.bempty[slot], phase ^ 1u))) {
                        abort_flag = 1;
                        ok = false;
                        break;
                    }
                    mr_expect_tx(&pipe.bfull[slot], chunk_bytes);
                    mr_bulk(bst + slot * chunk_bytes, src, chunk_bytes, &pipe.bfull[slot]);
                    src += chunk_bytes;
                    if (++slot == (uint32_t)nbst) {
                        slot = 0;
                        phase ^= 1u;
                    }
                }
            }
            for (int64_t q = issued - nbst; q < issued; ++q)
                if (q >= 0) mr_wait(&pipe.bfull[q % nbst], (uint32_t)(q / nbst) & 1u);
        }
        __syncwarp();
    }
    if (abort_flag && tid == 0) atomicExch(err, 1);
    mr_fence_before();
    __syncthreads();
    mr_fence_after();
    if (warp == kMrMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem_base));
}

// ---------------------------------------------------------------------------
// Missing-call sums and the standardisation: g_cj = v (S1 - u (R - M_cj)),
// with S1 = (D - M_cj) / 2 and D read from g_c.  A block stages CG residual
// columns in shared memory, interleaved (CG floats per sample); each lane owns
// one SNP, reads its missing-call list 16 bytes at a time (8 or 4 sample
// indices) and gathers the
// CG residual values of every listed sample, so a list entry costs one
// shared-memory vector load for all CG columns; the lane then writes the CG
// finished gradient entries of its SNP (consecutive SNPs across the warp).

template <int CG>
struct MrVec;
template <>
struct MrVec<1> { using T = float; };
template <>
struct MrVec<2> { using T = float2; };
template <>
struct MrVec<4> { using T = float4; };

__device__ __forceinline__ void mr_addv(float *m, float v) { m[0] += v; }
__device__ __forceinline__ void mr_addv(float *m, float2 v) { m[0] += v.x; m[1] += v.y; }
__device__ __forceinline__ void mr_addv(float *m, float4 v)
{
    m[0] += v.x; m[1] += v.y; m[2] += v.z; m[3] += v.w;
}

constexpr int kFinThreads = 512;

template <int CG, typename IdxT, bool kStage>
__global__ void __launch_bounds__(kFinThreads) k_miss_finalize(const int64_t *__restrict__ off,
                                                               const IdxT *__restrict__ idx, int64_t p,
                                                               int64_t n_pad,
                                                               const MrCol *__restrict__ cols,
                                                               int ncols)
{
    using V = typename MrVec<CG>::T;
    constexpr int kPer = 16 / (int)sizeof(IdxT);               // indices per 16-byte load
    extern __shared__ __align__(16) unsigned char mr_sh[];
    V *rs = reinterpret_cast<V *>(mr_sh);
    const int c0 = blockIdx.y * CG;
    if (kStage) {
        for (int64_t i = threadIdx.x; i < n_pad; i += blockDim.x) {
            float v[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int e = 0; e < CG; ++e)
                if (c0 + e < ncols) v[e] = cols[c0 + e].r32[i];
            V x;
            if constexpr (CG == 1) x = v[0];
            else if constexpr (CG == 2) x = make_float2(v[0], v[1]);
            else x = make_float4(v[0], v[1], v[2], v[3]);
            rs[i] = x;
        }
        __syncthreads();
    }
    const float *__restrict__ rg = cols[c0].r32;        // unstaged path: CG == 1
    const uint4 *__restrict__ idx4 = reinterpret_cast<const uint4 *>(idx);
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * 32; base < p; base += nwarps * 32) {
        const int64_t j = base + lane;
        const bool live = j < p;
        const int64_t e0 = live ? off[j] : 0, e1 = live ? off[j + 1] : 0;
        const int64_t a0 = e0 & ~(int64_t)(kPer - 1);
        const int lo = (int)(e0 - a0), hi = (int)(e1 - a0);   // valid positions [lo, hi) from a0
        const uint4 *__restrict__ src = idx4 + a0 / kPer;
        float m[CG];
#pragma unroll
        for (int e = 0; e < CG; ++e) m[e] = 0.0f;
        uint4 w = src[0];                                      // next piece requested a step ahead
        for (int q = 0; q * kPer < hi; ++q) {
            const uint4 wn = (q + 1) * kPer < hi ? src[q + 1] : w;
            const IdxT *ent = reinterpret_cast<const IdxT *>(&w);
#pragma unroll
            for (int t = 0; t < kPer; ++t) {
                const int pos = q * kPer + t;
                if (pos >= lo && pos < hi) {
                    if (kStage) mr_addv(m, rs[ent[t]]);
                    else m[0] += __ldg(rg + ent[t]);
                }
            }
            w = wn;
        }
        if (live) {
#pragma unroll
            for (int e = 0; e < CG; ++e) {
                if (c0 + e < ncols) {
                    const MrCol &C = cols[c0 + e];
                    const float d = C.g[j];
                    C.g[j] = standardise_d(d, C.R, m[e], C.u32[j], C.v32[j]);
                }
            }
        }
    }
}

// Eight columns per block: sample i's eight residual values form one 32-byte
// row of the shared table, and a pair of lanes owns one SNP, lane h of the pair
// reading half h (columns 4h .. 4h+3) of every listed row, so a quarter-warp's
// 16-byte loads touch four rows instead of eight.  List positions outside the
// SNP's range in its first and last 16-byte piece read an all-zero row (index
// n_pad); every sum still runs over the SNP's list in order from 0.0f.
constexpr int kFin8Threads = 1024;

template <typename IdxT>
__global__ void __launch_bounds__(kFin8Threads) k_miss_finalize8(const int64_t *__restrict__ off,
                                                                 const IdxT *__restrict__ idx, int64_t p,
                                                                 int64_t n_pad,
                                                                 const MrCol *__restrict__ cols,
                                                                 int ncols)
{
    constexpr int kPer = 16 / (int)sizeof(IdxT);               // indices per 16-byte load
    extern __shared__ __align__(16) unsigned char mr_sh[];
    float4 *rs = reinterpret_cast<float4 *>(mr_sh);            // 2 (n_pad + 1) float4
    const int c0 = blockIdx.y * 8;
    for (int64_t i = threadIdx.x; i <= n_pad; i += blockDim.x) {
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = (i < n_pad && c0 + e < ncols) ? cols[c0 + e].r32[i] : 0.0f;
        rs[2 * i] = make_float4(v[0], v[1], v[2], v[3]);
        rs[2 * i + 1] = make_float4(v[4], v[5], v[6], v[7]);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, h = lane & 1;
    const uint32_t zrow = (uint32_t)n_pad;
    const uint4 *__restrict__ idx4 = reinterpret_cast<const uint4 *>(idx);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * 16; base < p; base += nwarps * 16) {
        const int64_t j = base + (lane >> 1);
        const bool live = j < p;
        const int64_t e0 = live ? off[j] : 0, e1 = live ? off[j + 1] : 0;
        const int64_t a0 = e0 & ~(int64_t)(kPer - 1);
        const int lo = (int)(e0 - a0), hi = (int)(e1 - a0);   // valid positions [lo, hi) from a0
        const uint4 *__restrict__ src = idx4 + a0 / kPer;
        float m0 = 0.0f, m1 = 0.0f, m2 = 0.0f, m3 = 0.0f;
        uint4 w = src[0];                                      // next piece requested a step ahead
        for (int q = 0; q * kPer < hi; ++q) {
            const uint4 wn = (q + 1) * kPer < hi ? src[q + 1] : w;
            const IdxT *ent = reinterpret_cast<const IdxT *>(&w);
#pragma unroll
            for (int t = 0; t < kPer; ++t) {
                const int pos = q * kPer + t;
                const uint32_t row = (pos >= lo && pos < hi) ? (uint32_t)ent[t] : zrow;
                const float4 x = rs[2 * row + h];
                m0 += x.x;
                m1 += x.y;
                m2 += x.z;
                m3 += x.w;
            }
            w = wn;
        }
        if (live) {
            const float m[4] = {m0, m1, m2, m3};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = c0 + 4 * h + e;
                if (c < ncols) {
                    const MrCol &C = cols[c];
                    const float d = C.g[j];
                    C.g[j] = standardise_d(d, C.R, m[e], C.u32[j], C.v32[j]);
                }
            }
        }
    }
}

// The same two finalisations over the padded lists (groups of 8 SNPs with
// common class boundaries, pads pointing at zero rows n_pad + ((j + c) mod 8)):
// at every step the SNPs of a quarter-warp read rows of one residue class c,
// (j + c) mod 8 for consecutive j, so their rows fall in distinct bank groups
// (32-byte rows: 4 per 128 bytes; 16-byte rows: 8); no bounds tests.  Zero
// rows add +0.0f, which leaves a sum that starts at 0.0f unchanged, so every
// SNP's sum is the one the unpadded lists give.
template <bool kWide>
__global__ void __launch_bounds__(kWide ? kFin8Threads : kFinThreads) k_miss_finalize_pad(
    const int64_t *__restrict__ goff, const uint16_t *__restrict__ gidx, int64_t p, int64_t n_pad,
    const MrCol *__restrict__ cols, int ncols)
{
    constexpr int kCols = kWide ? 8 : 4;                       // columns per block
    constexpr int kSnps = kWide ? 16 : 32;                     // SNPs per warp
    extern __shared__ __align__(16) unsigned char mr_sh[];
    float4 *rs = reinterpret_cast<float4 *>(mr_sh);            // (n_pad + 8) rows of kCols floats
    const int c0 = blockIdx.y * kCols;
    for (int64_t i = threadIdx.x; i < n_pad + 8; i += blockDim.x) {
        float v[kCols];
#pragma unroll
        for (int e = 0; e < kCols; ++e) v[e] = (i < n_pad && c0 + e < ncols) ? cols[c0 + e].r32[i] : 0.0f;
#pragma unroll
        for (int h = 0; h < kCols / 4; ++h)
            rs[(kCols / 4) * i + h] = make_float4(v[4 * h], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3]);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, h = kWide ? (lane & 1) : 0;
    const int64_t ngroups = (p + kPadGroup - 1) / kPadGroup;
    const uint4 *__restrict__ g4 = reinterpret_cast<const uint4 *>(gidx);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * kSnps; base < p; base += nwarps * kSnps) {
        const int64_t j = base + (kWide ? (lane >> 1) : lane);
        const int64_t g = j / kPadGroup;
        int64_t start = 0, L = 0;
        if (g < ngroups) {
            const int64_t g0 = goff[g];
            L = (goff[g + 1] - g0) / kPadGroup;
            start = g0 + (j % kPadGroup) * L;
        }
        const uint4 *__restrict__ src = g4 + start / 8;
        const int nq = (int)(L / 8);
        float m0 = 0.0f, m1 = 0.0f, m2 = 0.0f, m3 = 0.0f;
        uint4 w = src[0];                                      // next piece requested a step ahead
        for (int q = 0; q < nq; ++q) {
            const uint4 wn = q + 1 < nq ? src[q + 1] : w;
            const uint16_t *ent = reinterpret_cast<const uint16_t *>(&w);
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const float4 x = rs[(kCols / 4) * (uint32_t)ent[t] + h];
                m0 += x.x;
                m1 += x.y;
                m2 += x.z;
                m3 += x.w;
            }
            w = wn;
        }
        if (j < p) {
            const float m[4] = {m0, m1, m2, m3};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = c0 + 4 * h + e;
                if (c < ncols) {
                    const MrCol &C = cols[c];
                    const float d = C.g[j];
                    C.g[j] = standardise_d(d, C.R, m[e], C.u32[j], C.v32[j]);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------

struct MrWork {
    uint8_t *bimg = nullptr;
    size_t bbytes = 0;
    int *err = nullptr;
    int dev = -1;
    float *mj = nullptr;                   // missing-call sums of a one-column pass (p)
    int64_t mj_cap = 0;
    int mj_dev = -1;
};
static thread_local MrWork g_mr;

// 16-byte groups of packed samples per row (2 K-steps of 32 samples each)
static int64_t mr_ngroups(const iht_dataset *ds) { return ((ds->n + 3) / 4 + 15) / 16; }

// K-steps of a pass: the single-column pass's 2 ngroups, rounded up to whole
// B chunks (the extra K-steps multiply zero limbs and add exactly 0).
static int mr_ksteps(const iht_dataset *ds)
{
    return (int)((2 * mr_ngroups(ds) + kMrChunkSteps - 1) / kMrChunkSteps * kMrChunkSteps);
}

static int mr_n(int ncols) { return (kMrLimbs * ncols + 15) / 16 * 16; }

// Launch shape of a pass: staging only, so every shape writes the same bits.
struct MrShape {
    int ngs;      // genotype stages (tiles x 8 KB each)
    int pairs;    // 1: each decoder step fills a pair of A buffers
    int fin8;     // 1: missing-call finalisation over 8 columns per block
    int padded;   // 1: finalisation over the padded lists (when the dataset has them)
    int tiles;    // 128-SNP tiles per CTA step: 2 (two decoder groups each) or 4 (one)
};

// B stages and A buffers of shape sh at N accumulator columns (false: it does
// not fit).  B stages: as many chunks as shared memory holds beside the
// genotype stages, up to kMrMaxBStages; A buffers: as many 16-column buffers
// as a tile's share of tensor memory holds beside its accumulator.
static bool mr_shape_launch(int N, const MrShape &sh, int *nbst, int *nbufs)
{
    if (sh.ngs < 2 || sh.ngs > kMrMaxGStages || sh.pairs < 0 || sh.pairs > 1 || sh.fin8 < 0 || sh.fin8 > 1 ||
        sh.padded < 0 || sh.padded > 1 || (sh.tiles != 2 && sh.tiles != 4))
        return false;
    const size_t gb = (size_t)sh.ngs * sh.tiles * kMrGTile;
    const size_t chunk = (size_t)kMrChunkSteps * N * 32;
    if (gb + 2 * chunk > kMrSmemMax) return false;
    int nb = std::min(kMrMaxBufs, (512 / sh.tiles - N) / 16);
    if (sh.pairs) {
        if (nb < 4) return false;
        nb &= ~1;
    }
    if (nb < 2) return false;
    *nbst = (int)std::min<size_t>(kMrMaxBStages, (kMrSmemMax - gb) / chunk);
    *nbufs = nb;
    return true;
}

// Default shape: with at most 64 accumulator columns four tiles per step (four
// MMA-issuing warps); above, two tiles, with many genotype stages in flight up
// to 96 columns and B chunks given the room beyond (the pass is tensor-bound
// there).  Pairs whenever there are four or more A buffers.
static MrShape mr_default_shape(int N)
{
    if (N <= 64) return MrShape{4, 1, 1, 1, 4};
    return MrShape{N <= 96 ? kMrMaxGStages : 4, 1, 1, 1, 2};
}

// A cached shape made to fit N (pairs dropped when there are too few buffers;
// the default when the stages or tiles do not fit; last, two tiles, four
// stages, no pairs, which fit at any N <= kMrMaxN).
static MrShape mr_fit_shape(int N, MrShape sh, int *nbst, int *nbufs)
{
    if (mr_shape_launch(N, sh, nbst, nbufs)) return sh;
    sh.pairs = 0;
    if (mr_shape_launch(N, sh, nbst, nbufs)) return sh;
    sh = mr_default_shape(N);
    if (mr_shape_launch(N, sh, nbst, nbufs)) return sh;
    sh = MrShape{4, 0, 1, 1, 2};
    mr_shape_launch(N, sh, nbst, nbufs);
    return sh;
}

// Tuning buckets of accumulator widths: 16..64, 80..96 (four tiles possible),
// 112..128, 144..192 (pairs possible) and 208..224.
static int mr_bucket_of(int N)
{
    return N <= 64 ? 64 : N <= 96 ? 96 : N <= 128 ? 128 : N <= 192 ? 192 : kMrMaxN;
}

int grad_mrhs_bucket(int ncols) { return mr_bucket_of(mr_n(std::min(ncols, kMrMaxCols))); }

bool grad_mrhs_shape_fits(int ncols, const int *params)
{
    int nbst, nbufs;
    return mr_shape_launch(mr_n(std::min(ncols, kMrMaxCols)),
                           MrShape{params[0], params[1], params[2], params[3], params[4]}, &nbst, &nbufs);
}

int mrhs_max_cols() { return kMrMaxCols; }

bool grad_mrhs_supported(const iht_dataset *ds) { return ds->p < (1ll << 31) && mr_ksteps(ds) > 0; }

using MrEncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static int mr_gmap(const iht_dataset *ds, CUtensorMap *map)
{
    static MrEncodeTiled encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        IHT_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                  cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !fn) return IHT_ECUDA;
        encode = (MrEncodeTiled)fn;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)ds->stride, (cuuint64_t)ds->p};
    const cuuint64_t strides[1] = {(cuuint64_t)ds->stride};
    const cuuint32_t box[2] = {(cuuint32_t)kMrGStageBytes, 128};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, ds->G, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? IHT_OK : IHT_ECUDA;
}

template <int CG, typename IdxT, bool kStage>
static int mr_launch_finalize(iht_dataset *ds, const MrCol *cols, int ncols, size_t smem)
{
    auto kern = k_miss_finalize<CG, IdxT, kStage>;
    static thread_local int configured_dev = -1;          // limit raised once (not during a capture)
    if (configured_dev != ds->ctx->device) {
        IHT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        configured_dev = ds->ctx->device;
    }
    const int groups = (ncols + CG - 1) / CG;
    const int per_sm = smem > 110 * 1024 ? 1 : 2;
    // one wave: at most per_sm resident blocks on every SM
    const int gx = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ds->p, kFinThreads),
                                                               (int64_t)ds->ctx->num_sms * per_sm / groups));
    kern<<<dim3(gx, groups), kFinThreads, smem, ds->ctx->stream>>>(ds->miss_off, (const IdxT *)ds->miss_idx,
                                                           ds->p, ds->n_pad, cols, ncols);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

constexpr size_t kFin8SmemMax = 220 * 1024;

template <typename IdxT>
static int mr_launch_finalize8(iht_dataset *ds, const MrCol *cols, int ncols, size_t smem)
{
    auto kern = k_miss_finalize8<IdxT>;
    static thread_local int configured_dev = -1;
    if (configured_dev != ds->ctx->device) {
        IHT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFin8SmemMax));
        configured_dev = ds->ctx->device;
    }
    const int groups = (ncols + 7) / 8;
    // one wave: one block per SM (the table takes most of shared memory)
    const int gx = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ds->p, kFin8Threads / 2),
                                                               (int64_t)ds->ctx->num_sms / groups));
    kern<<<dim3(gx, groups), kFin8Threads, smem, ds->ctx->stream>>>(ds->miss_off, (const IdxT *)ds->miss_idx,
                                                                    ds->p, ds->n_pad, cols, ncols);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

template <bool kWide>
static int mr_launch_finalize_pad(iht_dataset *ds, const MrCol *cols, int ncols, size_t smem)
{
    auto kern = k_miss_finalize_pad<kWide>;
    static thread_local int configured_dev = -1;
    if (configured_dev != ds->ctx->device) {
        IHT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFin8SmemMax));
        configured_dev = ds->ctx->device;
    }
    const int cg = kWide ? 8 : 4, threads = kWide ? kFin8Threads : kFinThreads;
    const int groups = (ncols + cg - 1) / cg;
    const int per_sm = kWide || smem > 110 * 1024 ? 1 : 2;
    const int64_t per_block = kWide ? threads / 2 : threads;     // SNPs per block and sweep
    const int gx = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ds->p, per_block),
                                                               (int64_t)ds->ctx->num_sms * per_sm / groups));
    kern<<<dim3(gx, groups), threads, smem, ds->ctx->stream>>>(ds->miss_goff, ds->miss_gidx, ds->p, ds->n_pad,
                                                               cols, ncols);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

template <typename IdxT>
static int mr_finalize(iht_dataset *ds, const MrCol *cols, int ncols, bool fin8, bool padded)
{
    if (padded && ds->miss_gidx) {
        const size_t p8 = 32 * ((size_t)ds->n_pad + 8), p4 = 16 * ((size_t)ds->n_pad + 8);
        if (fin8 && ncols > 4 && p8 <= kFin8SmemMax) return mr_launch_finalize_pad<true>(ds, cols, ncols, p8);
        if (p4 <= 200 * 1024) return mr_launch_finalize_pad<false>(ds, cols, ncols, p4);
    }
    const size_t f8 = 32 * ((size_t)ds->n_pad + 1);
    if (fin8 && ncols > 4 && f8 <= kFin8SmemMax) return mr_launch_finalize8<IdxT>(ds, cols, ncols, f8);
    const size_t f = sizeof(float) * (size_t)ds->n_pad;
    if (4 * f <= 200 * 1024) return mr_launch_finalize<4, IdxT, true>(ds, cols, ncols, 4 * f);
    if (2 * f <= 200 * 1024) return mr_launch_finalize<2, IdxT, true>(ds, cols, ncols, 2 * f);
    if (f <= 200 * 1024) return mr_launch_finalize<1, IdxT, true>(ds, cols, ncols, f);
    return mr_launch_finalize<1, IdxT, false>(ds, cols, ncols, 0);
}

// One pass of nc <= kMrMaxCols columns after its limbs are staged.
struct MrPass {
    iht_dataset *ds;
    const CUtensorMap *map;
    int ksteps, N, nc;
    MrCol *cols;
};

// The multi-column pass and its finalisation in shape sh; with events, ev[e0],
// ev[e0 + 1] bracket the pass and ev[e0 + 2], ev[e0 + 3] the finalisation.
static int mr_pass(const MrPass &P, MrShape sh, const TuneEvents *te, size_t e0, ProfEvents *prof)
{
    cudaStream_t s = P.ds->ctx->stream;
    int nbst = 0, nbufs = 0;
    sh = mr_fit_shape(P.N, sh, &nbst, &nbufs);
    // at least 116 KB, so one CTA per SM: the kernel allocates all 512 columns of tensor memory
    const size_t smem = std::max<size_t>(116 * 1024, (size_t)sh.ngs * sh.tiles * kMrGTile +
                                                         (size_t)nbst * kMrChunkSteps * P.N * 32);
    // D FP32, A E5M2, B E4M3, K-major, N, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | ((uint32_t)(P.N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    const int64_t ntiles = (P.ds->p + 128 * sh.tiles - 1) / (128 * sh.tiles);
    const int grid = (int)std::min<int64_t>(ntiles, P.ds->ctx->num_sms);
    if (te) IHT_CUDA(cudaEventRecord(te->ev[e0], s));
    prof_begin(prof, s);
    auto kern = sh.tiles == 4 ? (sh.pairs ? k_grad_mrhs<true, 4, 1> : k_grad_mrhs<false, 4, 1>)
                              : (sh.pairs ? k_grad_mrhs<true, 2, 2> : k_grad_mrhs<false, 2, 2>);
    kern<<<grid, mr_threads(sh.tiles), smem, s>>>(*P.map, P.ds->p, P.ksteps, P.N, P.nc, nbufs, nbst, sh.ngs,
                                                  g_mr.bimg, P.cols, idesc, g_mr.err);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    prof_end(prof, s);
    if (te) IHT_CUDA(cudaEventRecord(te->ev[e0 + 1], s));
    if (te) IHT_CUDA(cudaEventRecord(te->ev[e0 + 2], s));
    const int rc = P.ds->miss_idx16 ? mr_finalize<uint16_t>(P.ds, P.cols, P.nc, sh.fin8 != 0, sh.padded != 0)
                                    : mr_finalize<int32_t>(P.ds, P.cols, P.nc, sh.fin8 != 0, sh.padded != 0);
    if (rc) return rc;
    if (te) IHT_CUDA(cudaEventRecord(te->ev[e0 + 3], s));
    return IHT_OK;
}

// First pass of a bucket: the pass and its finalisation once per run, the
// pass cycling through the candidate shapes (2 or 4 tiles per CTA step x
// genotype stages 4, 6, 8 x pairs on, off, as they fit) and the finalisation
// through its variants (8 or 4 columns per block x plain or padded lists),
// each run writing the same g (the
// finalisation reads the pass's output in place, so each run does both).  The
// fastest pass shape and the fastest finalisation are cached.  prof brackets
// the first run's pass.
static int mr_tune(const MrPass &P, ProfEvents *prof)
{
    std::vector<MrShape> cand;
    for (int tiles : {2, 4})
        for (int ngs : {4, 6, 8})
            for (int pairs : {1, 0}) {
                const MrShape sh{ngs, pairs, 1, 0, tiles};
                int nbst, nbufs;
                if (mr_shape_launch(P.N, sh, &nbst, &nbufs)) cand.push_back(sh);
            }
    const int fins[4][2] = {{1, 1}, {0, 1}, {1, 0}, {0, 0}};    // (fin8, padded)
    const int nfin = P.ds->miss_gidx ? 4 : 2;
    const size_t runs = std::max(cand.size(), (size_t)nfin);
    TuneEvents te(4 * runs);
    IHT_CUDA(te.create());
    for (size_t r = 0; r < runs; ++r) {
        MrShape sh = cand[r % cand.size()];
        sh.fin8 = fins[(P.ds->miss_gidx ? 0 : 2) + r % nfin][0];
        sh.padded = fins[(P.ds->miss_gidx ? 0 : 2) + r % nfin][1];
        if (int rc = mr_pass(P, sh, &te, 4 * r, r == 0 ? prof : nullptr)) return rc;
    }
    IHT_CUDA(cudaStreamSynchronize(P.ds->ctx->stream));
    float best = 1e30f, fin_best = 1e30f;
    int prm[kTuneParams] = {0, 0, 1, 0, 2};
    for (size_t r = 0; r < runs; ++r) {
        const float k = te.ms(4 * r, 4 * r + 1), f = te.ms(4 * r + 2, 4 * r + 3);
        if (r < cand.size() && k < best) {
            best = k;
            prm[0] = cand[r].ngs;
            prm[1] = cand[r].pairs;
            prm[4] = cand[r].tiles;
        }
        if (f < fin_best) {
            fin_best = f;
            prm[2] = fins[(P.ds->miss_gidx ? 0 : 2) + r % nfin][0];
            prm[3] = fins[(P.ds->miss_gidx ? 0 : 2) + r % nfin][1];
        }
    }
    tune_store(P.ds, IHT_PASS_MULTI, mr_bucket_of(P.N), prm, best + fin_best, (int)runs);
    return IHT_OK;
}

// G of ncols residual columns (cols: device array; r32, u32, v32 and g set by
// the caller; cols_host, optional, the same descriptors on the host).  Passes
// of at most kMrMaxCols columns, each in its bucket's cached shape (tuned on
// this call when none is cached, tuning is on and the stream is not being
// captured; else the default shape).  A single column with its host descriptor
// goes through the single-column pass instead (same arithmetic, so the same
// bits, at about half the cost of a one-column multi-column pass).
int launch_grad_mrhs(iht_dataset *ds, MrCol *cols, int ncols, ProfEvents *prof, const MrCol *cols_host)
{
    if (ncols <= 0) return IHT_OK;
    if (!grad_mrhs_supported(ds)) return IHT_EINVAL;
    cudaStream_t s = ds->ctx->stream;
    if (ncols == 1 && cols_host && grad_tc_supported(ds)) {
        MrWork &w = g_mr;
        if (w.mj_dev != ds->ctx->device || w.mj_cap < ds->p) {
            if (w.mj) cudaFree(w.mj);
            w.mj = nullptr;
            w.mj_cap = 0;
            IHT_CUDA(dev_malloc(&w.mj, sizeof(float) * (size_t)ds->p));
            w.mj_cap = ds->p;
            w.mj_dev = ds->ctx->device;
        }
        const MrCol &C = cols_host[0];
        int rc = prepare_grad_tc_to(ds, C.r32, w.mj, nullptr);
        if (rc) return rc;
        prof_begin(prof, s);
        rc = launch_grad_tc_main_with(ds, C.r32, C.g, C.u32, C.v32, w.mj, nullptr);
        prof_end(prof, s);
        return rc;
    }
    const int ksteps = mr_ksteps(ds);
    const size_t need = (size_t)ksteps * mr_n(kMrMaxCols) * 32;
    MrWork &w = g_mr;
    if (w.dev != ds->ctx->device || w.bbytes < need) {
        if (w.bimg) cudaFree(w.bimg);
        if (w.err) cudaFree(w.err);
        w.bimg = nullptr;
        w.err = nullptr;
        w.bbytes = 0;
        IHT_CUDA(dev_malloc(&w.bimg, need));
        IHT_CUDA(dev_malloc(&w.err, sizeof(int)));
        IHT_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), s));
        w.bbytes = need;
        w.dev = ds->ctx->device;
    }
    CUtensorMap map;
    int rc = mr_gmap(ds, &map);
    if (rc) return rc;
    static thread_local int cfg = -1;
    if (cfg != ds->ctx->device) {
        for (auto kern : {k_grad_mrhs<true, 2, 2>, k_grad_mrhs<false, 2, 2>, k_grad_mrhs<true, 4, 1>,
                          k_grad_mrhs<false, 4, 1>})
            IHT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMrSmemMax));
        cfg = ds->ctx->device;
    }
    const bool may_tune = autotune_enabled() && !stream_capturing(s);
    for (int c0 = 0; c0 < ncols; c0 += kMrMaxCols) {
        const int nc = std::min(kMrMaxCols, ncols - c0);
        const int N = mr_n(nc);
        const size_t bbytes = (size_t)ksteps * N * 32;
        IHT_CUDA(cudaMemsetAsync(w.bimg, 0, bbytes, s));
        // scale, limbs and R over the single-column pass's samples (the rest are 0)
        k_mr_limbs<<<nc, 1024, 0, s>>>(cols + c0, 2 * mr_ngroups(ds) * kMrStepSamples, N, w.bimg);
        note_launch();
        IHT_CUDA(cudaGetLastError());
        const MrPass pass{ds, &map, ksteps, N, nc, cols + c0};
        int prm[kTuneParams];
        if (tune_lookup(ds, IHT_PASS_MULTI, mr_bucket_of(N), prm))
            rc = mr_pass(pass, MrShape{prm[0], prm[1], prm[2], prm[3], prm[4]}, nullptr, 0, prof);
        else if (may_tune)
            rc = mr_tune(pass, prof);
        else
            rc = mr_pass(pass, mr_default_shape(N), nullptr, 0, prof);
        if (rc) return rc;
    }
    return IHT_OK;
}

// Identifies the calling thread's pass scratch (changes when it is reallocated).
uint64_t grad_mrhs_scratch_id()
{
    return (uint64_t)(uintptr_t)g_mr.bimg ^ ((uint64_t)(uintptr_t)g_mr.err << 1) ^
           ((uint64_t)(uintptr_t)g_mr.mj << 2) ^ ((uint64_t)g_mr.bbytes << 3);
}

// Frees the calling thread's pass scratch (a server's worker before it exits).
void grad_mrhs_release_thread()
{
    MrWork &w = g_mr;
    if (w.bimg) cudaFree(w.bimg);
    if (w.err) cudaFree(w.err);
    if (w.mj) cudaFree(w.mj);
    w = MrWork();
}

// Bounded-wait status of the multi-column passes since the last reset (1 = a
// wait timed out); synchronises the stream.  An injected timeout
// (iht_fault_inject) writes the error word from the host first.
int grad_mrhs_status(iht_dataset *ds, int *timed_out)
{
    *timed_out = 0;
    if (!g_mr.err) {                     // no multi-column pass yet: nothing to read
        IHT_CUDA(cudaStreamSynchronize(ds->ctx->stream));
        return IHT_OK;
    }
    if (fault_take(IHT_FAULT_TIMEOUT))
        IHT_CUDA(cudaMemsetAsync(g_mr.err, 0x01, sizeof(int), ds->ctx->stream));
    int h = 0;
    IHT_CUDA(cudaMemcpyAsync(&h, g_mr.err, sizeof(int), cudaMemcpyDeviceToHost, ds->ctx->stream));
    IHT_CUDA(cudaStreamSynchronize(ds->ctx->stream));
    *timed_out = h != 0;
    return IHT_OK;
}

// Clears the error word of the calling thread's multi-column pass (stream-ordered).
int grad_mrhs_reset_status(iht_dataset *ds)
{
    if (g_mr.err) IHT_CUDA(cudaMemsetAsync(g_mr.err, 0, sizeof(int), ds->ctx->stream));
    return IHT_OK;
}

}  // namespace iht
