// a2, CUDA-core variant: g_j = v_j (S1_j - u_j (R - M_j)) over every SNP.
//
// Standardisation is applied on the fly (Sec. 2.3.2): S1_j = sum of dosage*r
// over observed calls, M_j = sum of r over missing calls, R = sum of r, so no
// standardised genotype is ever stored.  Layout of the work:
//   * each CTA stages the whole residual r (n_pad floats) in shared memory,
//     16-byte slots rotated within groups of 8 so that the 32 lanes of a warp
//     reading 4 consecutive slots each hit distinct banks;
//   * one warp owns one SNP row at a time (grid-stride over SNPs); lane l reads
//     32-bit words l, l+32, ... of the row (coalesced 128-byte requests), with
//     8 words per lane in flight before any arithmetic;
//   * the two per-SNP sums are reduced with warp shuffles in a fixed order, so
//     results are identical run to run.
// R is summed per CTA from the staged residual (every CTA gets the same value).
#include "common.cuh"

namespace iht {

__device__ __forceinline__ int rslot(int f) { return (f & ~7) | ((f + (f >> 3)) & 7); }

constexpr int kSimtWords = 8;   // 32-bit words per lane per chunk (128 samples)

__device__ __forceinline__ void accum_byte(uint32_t byte, float4 r, float &s1, float &m)
{
    const float rv[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t code = (byte >> (2 * q)) & 3u;
        const float x = code == 3u ? 2.0f : (code == 2u ? 1.0f : 0.0f);
        s1 = fmaf(x, rv[q], s1);
        m += code == 1u ? rv[q] : 0.0f;
    }
}

__global__ void __launch_bounds__(256) k_grad_simt(const uint8_t *__restrict__ G, int64_t p,
                                                   int64_t stride, int64_t rowb,
                                                   const float *__restrict__ r32,
                                                   int64_t n_pad, const float *__restrict__ u32,
                                                   const float *__restrict__ v32,
                                                   float *__restrict__ g,
                                                   const int32_t *__restrict__ done)
{
    extern __shared__ float4 rs[];
    __shared__ double red[8];
    if (done && *done) return;

    const int nslot = (int)(n_pad / 4);
    const float4 *r4 = reinterpret_cast<const float4 *>(r32);
    double acc = 0.0;
    for (int f = threadIdx.x; f < nslot; f += blockDim.x) {
        const float4 v = r4[f];
        acc += ((double)v.x + (double)v.y) + ((double)v.z + (double)v.w);
        rs[rslot(f)] = v;
    }
    const float R = (float)block_sum(acc, red);   // synchronises the block

    const int lane = threadIdx.x & 31;
    const int64_t nw = rowb / 4;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < p;
         j += nwarps) {
        const uint32_t *row = reinterpret_cast<const uint32_t *>(G + j * stride);
        float s1 = 0.0f, m = 0.0f;
        for (int64_t base = 0; base < nw; base += 32 * kSimtWords) {
            uint32_t w[kSimtWords];
#pragma unroll
            for (int t = 0; t < kSimtWords; ++t) {
                const int64_t c = base + lane + 32 * t;
                w[t] = c < nw ? __ldcs(row + c) : 0u;
            }
#pragma unroll
            for (int t = 0; t < kSimtWords; ++t) {
                const int64_t c = base + lane + 32 * t;
                if (c < nw) {
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        accum_byte(w[t] >> (8 * b), rs[rslot((int)(4 * c + b))], s1, m);
                }
            }
        }
        s1 = warp_sum(s1);
        m = warp_sum(m);
        if (lane == 0) g[j] = v32[j] * (s1 - u32[j] * (R - m));
    }
}

static int grad_simt_run(iht_dataset *ds, const float *r32, const float *u32, const float *v32,
                         float *g, const int32_t *done)
{
    static thread_local int configured_dev = -1;
    static thread_local size_t configured_smem = 0;
    const size_t smem = sizeof(float) * (size_t)ds->n_pad;
    if (configured_dev != ds->ctx->device || configured_smem < smem) {
        IHT_CUDA(cudaFuncSetAttribute(k_grad_simt, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)std::max<size_t>(smem, 48 * 1024)));
        configured_dev = ds->ctx->device;
        configured_smem = std::max<size_t>(smem, 48 * 1024);
    }
    int per_sm = 0;
    IHT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grad_simt, 256, smem));
    if (per_sm < 1) return IHT_EINVAL;   // residual does not fit in shared memory
    const int64_t want = (ds->p + 7) / 8;
    const int blocks = (int)std::min<int64_t>(want, (int64_t)per_sm * ds->ctx->num_sms);
    k_grad_simt<<<blocks, 256, smem, ds->ctx->stream>>>(ds->G, ds->p, ds->stride, ds->rowb, r32,
                                                        ds->n_pad, u32, v32, g, done);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

int launch_grad_simt(iht_dataset *ds, const float *r32, float *g, const int32_t *done)
{
    return grad_simt_run(ds, r32, ds->ws->u32, ds->ws->v32, g, done);
}

int launch_grad_simt_stats(iht_dataset *ds, const float *r32, const float *u32, const float *v32,
                           float *g)
{
    return grad_simt_run(ds, r32, u32, v32, g, nullptr);
}

int launch_grad_impl(iht_dataset *ds, int impl, const float *r32, float *g, const int32_t *done)
{
    if (impl == 2 || (impl == 0 && grad_tc_supported(ds))) return launch_grad_tc(ds, r32, g, done);
    return launch_grad_simt(ds, r32, g, done);
}

}  // namespace iht
