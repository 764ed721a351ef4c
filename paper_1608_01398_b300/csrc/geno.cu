// a0/a1: genotype upload fix-up, row sets, per-SNP counts and statistics.
//
// Counts come from popcounts on 32-bit words of 16 codes: with lo = even bits
// and hi = odd bits of each 2-bit code, code 11 = lo&hi, 01 = lo&~hi,
// 10 = hi&~lo; unused rows are masked to 00 and code 00 is n_rows minus the
// rest.  The FP64 statistics then follow the integer counts in the fixed
// order of Sec. 2.3.2's u, v vectors (mean over observed calls, variance with
// an (n_obs - 1) denominator), with every operation correctly rounded so the
// values match any IEEE FP64 evaluation of the same expression bit for bit.
#include "common.cuh"
#include "limbs.cuh"

namespace iht {

// Pad samples (n .. 4*stride-1) get code 01 (missing), so no kernel ever
// needs a bounds test on the sample axis.
__global__ void k_fix_padding(uint8_t *__restrict__ G, int64_t p, int64_t stride, int64_t nbytes,
                              int rem)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= p) return;
    uint8_t *row = G + j * stride;
    if (rem) {
        const unsigned keep = (1u << (2 * rem)) - 1u;
        row[nbytes - 1] = (uint8_t)((row[nbytes - 1] & keep) | (0x55u & ~keep));
    }
    for (int64_t b = nbytes; b < stride; ++b) row[b] = 0x55;
}

int launch_fix_padding(iht_dataset *ds)
{
    const int64_t nbytes = (ds->n + 3) / 4;
    const int rem = (int)(ds->n & 3);
    if (rem == 0 && nbytes == ds->stride) return IHT_OK;
    k_fix_padding<<<ceil_div(ds->p, 256), 256, 0, ds->ctx->stream>>>(ds->G, ds->p, ds->stride,
                                                                     nbytes, rem);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

__global__ void k_mark_rows(const int32_t *__restrict__ rows, int64_t n_rows, int64_t n,
                            int32_t *__restrict__ used, int32_t *__restrict__ err)
{
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_rows) return;
    const int32_t i = rows[a];
    if (i < 0 || i >= n) {
        atomicOr(err, 2);
        return;
    }
    if (atomicExch(&used[i], 1) != 0) atomicOr(err, 2);   // duplicate row
}

__global__ void k_mark_all(int64_t n, int64_t n_pad, int32_t *__restrict__ used)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_pad) used[i] = i < n ? 1 : 0;
}

__global__ void k_rowmask(const int32_t *__restrict__ used, uint32_t *__restrict__ rowmask,
                          int64_t nwords)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nwords) return;
    uint32_t m = 0;
#pragma unroll
    for (int q = 0; q < 16; ++q)
        if (used[16 * c + q]) m |= 3u << (2 * q);
    rowmask[c] = m;
}

// Marks the rows of a row set (rows_dev == nullptr: all n) and builds its
// 2-bit row mask.  Bad or duplicate indices set bit 1 of *err.
int setup_rowset(iht_dataset *ds, const int32_t *rows_dev, int64_t n_rows, const RowSet &rs,
                 int32_t *err)
{
    cudaStream_t s = ds->ctx->stream;
    if (rows_dev) {
        IHT_CUDA(cudaMemsetAsync(rs.used, 0, sizeof(int32_t) * ds->n_pad, s));
        if (n_rows > 0) {
            k_mark_rows<<<ceil_div(n_rows, 256), 256, 0, s>>>(rows_dev, n_rows, ds->n, rs.used, err);
            note_launch();
        }
    } else {
        k_mark_all<<<ceil_div(ds->n_pad, 256), 256, 0, s>>>(ds->n, ds->n_pad, rs.used);
        note_launch();
    }
    const int64_t nwords = ds->stride / 4;
    k_rowmask<<<ceil_div(nwords, 256), 256, 0, s>>>(rs.used, rs.rowmask, nwords);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

RowSet workspace_rowset(iht_dataset *ds)
{
    Workspace *ws = ds->ws;
    RowSet rs;
    rs.used = ws->used;
    rs.rowmask = ws->rowmask;
    rs.counts = ws->counts;
    rs.u64 = ws->u64;
    rs.v64 = ws->v64;
    rs.u32 = ws->u32;
    rs.v32 = ws->v32;
    return rs;
}

int setup_rows(iht_dataset *ds, const int32_t *rows_dev, int64_t n_rows)
{
    return setup_rowset(ds, rows_dev, n_rows, workspace_rowset(ds), &ds->ws->sc->err);
}

constexpr int kCountUnroll = 4;        // 16-byte words per lane and SNP in flight (2 KB of a row)

// FP64 statistics from the integer counts, every operation correctly rounded
// (Sec. 2.3.2: mean over observed calls, variance with n_obs - 1).
__device__ __forceinline__ void snp_stats(int64_t n_rows, int c1, int c2, int c3, double &mean,
                                          double &inv_sd)
{
    const double n_obs = (double)(n_rows - c1);
    const double s1 = (double)(c2 + 2 * c3);
    const double s2 = (double)(c2 + 4 * c3);
    mean = n_obs > 0.0 ? __ddiv_rn(s1, n_obs) : 0.0;
    inv_sd = 0.0;
    if (n_obs >= 2.0) {
        const double var = __ddiv_rn(__dsub_rn(s2, __ddiv_rn(__dmul_rn(s1, s1), n_obs)),
                                     __dsub_rn(n_obs, 1.0));
        if (var > 0.0) inv_sd = __ddiv_rn(1.0, __dsqrt_rn(var));
    }
}

// This lane's masked counts (missing, het, hom-alt) over one pass of a row.
__device__ __forceinline__ void count_words(const uint4 (&w4)[kCountUnroll], const uint4 *mask4,
                                            int64_t c0, int lane, int64_t nw4, int &c1, int &c2,
                                            int &c3)
{
#pragma unroll
    for (int u = 0; u < kCountUnroll; ++u) {
        const int64_t c = c0 + lane + 32 * u;
        if (c >= nw4) break;
        const uint4 m4 = __ldg(mask4 + c);
        const uint32_t ws[4] = {w4[u].x & m4.x, w4[u].y & m4.y, w4[u].z & m4.z, w4[u].w & m4.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t lo = ws[q] & 0x55555555u, hi = (ws[q] >> 1) & 0x55555555u;
            c3 += __popc(lo & hi);
            c1 += __popc(lo & ~hi);
            c2 += __popc(hi & ~lo);
        }
    }
}

__device__ __forceinline__ void load_pass(const uint4 *row4, int64_t c0, int lane, int64_t nw4,
                                          uint4 (&w4)[kCountUnroll])
{
#pragma unroll
    for (int u = 0; u < kCountUnroll; ++u) {
        const int64_t c = c0 + lane + 32 * u;
        w4[u] = c < nw4 ? __ldcs(row4 + c) : make_uint4(0u, 0u, 0u, 0u);
    }
}

// A warp takes 32 consecutive SNPs: two at a time it counts (all loads of
// both rows in flight) and reduces across the lanes, lane s keeping SNP s's
// totals; then every lane computes its SNP's FP64 statistics at once and the
// warp writes 32 consecutive entries.
__global__ void __launch_bounds__(256) k_counts(const uint8_t *__restrict__ G, int64_t p,
                                                int64_t stride, int64_t rowb,
                                                const uint32_t *__restrict__ rowmask,
                                                int64_t n_rows, int32_t *__restrict__ counts,
                                                double *__restrict__ u64, double *__restrict__ v64,
                                                float *__restrict__ u32, float *__restrict__ v32)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t nw4 = rowb / 16;
    const uint4 *mask4 = reinterpret_cast<const uint4 *>(rowmask);
    for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < p;
         base += nwarps * 32) {
        int m1 = 0, m2 = 0, m3 = 0;                 // totals of SNP base + lane
        for (int s = 0; s < 32 && base + s < p; s += 2) {
            const int64_t ja = base + s;
            const bool two = s + 1 < 32 && ja + 1 < p;
            const uint4 *ra = reinterpret_cast<const uint4 *>(G + ja * stride);
            const uint4 *rb = reinterpret_cast<const uint4 *>(G + (two ? ja + 1 : ja) * stride);
            int a1 = 0, a2 = 0, a3 = 0, b1 = 0, b2 = 0, b3 = 0;
            for (int64_t c0 = 0; c0 < nw4; c0 += 32 * kCountUnroll) {
                uint4 wa[kCountUnroll], wb[kCountUnroll];
                load_pass(ra, c0, lane, nw4, wa);
                load_pass(rb, c0, lane, nw4, wb);
                count_words(wa, mask4, c0, lane, nw4, a1, a2, a3);
                count_words(wb, mask4, c0, lane, nw4, b1, b2, b3);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a1 += __shfl_xor_sync(0xffffffffu, a1, o);
                a2 += __shfl_xor_sync(0xffffffffu, a2, o);
                a3 += __shfl_xor_sync(0xffffffffu, a3, o);
                b1 += __shfl_xor_sync(0xffffffffu, b1, o);
                b2 += __shfl_xor_sync(0xffffffffu, b2, o);
                b3 += __shfl_xor_sync(0xffffffffu, b3, o);
            }
            if (lane == s) { m1 = a1; m2 = a2; m3 = a3; }
            if (two && lane == s + 1) { m1 = b1; m2 = b2; m3 = b3; }
        }
        const int64_t j = base + lane;
        if (j < p) {
            if (counts) {
                counts[4 * j + 0] = (int32_t)(n_rows - m1 - m2 - m3);
                counts[4 * j + 1] = m1;
                counts[4 * j + 2] = m2;
                counts[4 * j + 3] = m3;
            }
            double mean, inv_sd;
            snp_stats(n_rows, m1, m2, m3, mean, inv_sd);
            u64[j] = mean;
            v64[j] = inv_sd;
            u32[j] = (float)mean;
            v32[j] = (float)inv_sd;
        }
    }
}

int launch_counts_rowset(iht_dataset *ds, int64_t n_rows, const RowSet &rs)
{
    const int blocks = (int)std::min<int64_t>(ceil_div(ds->p, 8 * 32), (int64_t)ds->ctx->num_sms * 8);
    k_counts<<<blocks, 256, 0, ds->ctx->stream>>>(ds->G, ds->p, ds->stride, ds->rowb, rs.rowmask,
                                                  n_rows, rs.counts, rs.u64, rs.v64, rs.u32, rs.v32);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

int launch_counts(iht_dataset *ds, int64_t n_rows)
{
    return launch_counts_rowset(ds, n_rows, workspace_rowset(ds));
}

// Several row sets in one pass over the genotypes: a warp reads SNP j's row
// once and applies up to kMultiSets row masks (same arithmetic as k_counts).
constexpr int kMultiSets = 8;

struct MultiSets {
    const uint32_t *rowmask[kMultiSets];
    int64_t n_rows[kMultiSets];
    double *u64[kMultiSets], *v64[kMultiSets];
    float *u32[kMultiSets], *v32[kMultiSets];
};

template <int NS>
__global__ void __launch_bounds__(256) k_counts_multi(const uint8_t *__restrict__ G, int64_t p,
                                                      int64_t stride, int64_t rowb, MultiSets ms)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t nw4 = rowb / 16;
    for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < p;
         base += nwarps * 32) {
        int m1[NS], m2[NS], m3[NS];                 // totals of SNP base + lane, per set
#pragma unroll
        for (int q = 0; q < NS; ++q) m1[q] = m2[q] = m3[q] = 0;
        for (int s = 0; s < 32 && base + s < p; ++s) {
            const uint4 *row4 = reinterpret_cast<const uint4 *>(G + (base + s) * stride);
            int c1[NS], c2[NS], c3[NS];
#pragma unroll
            for (int q = 0; q < NS; ++q) c1[q] = c2[q] = c3[q] = 0;
            for (int64_t c0 = 0; c0 < nw4; c0 += 32 * kCountUnroll) {
                uint4 w4[kCountUnroll];
                load_pass(row4, c0, lane, nw4, w4);
#pragma unroll
                for (int u = 0; u < kCountUnroll; ++u) {
                    const int64_t c = c0 + lane + 32 * u;
                    if (c >= nw4) break;
                    // the genotype word split once into its lo / hi bit planes
                    const uint32_t wv[4] = {w4[u].x, w4[u].y, w4[u].z, w4[u].w};
                    uint32_t lo[4], hi[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        lo[e] = wv[e] & 0x55555555u;
                        hi[e] = (wv[e] >> 1) & 0x55555555u;
                    }
#pragma unroll
                    for (int q = 0; q < NS; ++q) {
                        const uint4 mk = __ldg(reinterpret_cast<const uint4 *>(ms.rowmask[q]) + c);
                        const uint32_t mv[4] = {mk.x & 0x55555555u, mk.y & 0x55555555u,
                                                mk.z & 0x55555555u, mk.w & 0x55555555u};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const uint32_t l = lo[e] & mv[e], h = hi[e] & mv[e];
                            c3[q] += __popc(l & h);
                            c1[q] += __popc(l & ~h);
                            c2[q] += __popc(h & ~l);
                        }
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < NS; ++q) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    c1[q] += __shfl_xor_sync(0xffffffffu, c1[q], o);
                    c2[q] += __shfl_xor_sync(0xffffffffu, c2[q], o);
                    c3[q] += __shfl_xor_sync(0xffffffffu, c3[q], o);
                }
                if (lane == s) {
                    m1[q] = c1[q];
                    m2[q] = c2[q];
                    m3[q] = c3[q];
                }
            }
        }
        const int64_t j = base + lane;
        if (j < p) {
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                double mean, inv_sd;
                snp_stats(ms.n_rows[q], m1[q], m2[q], m3[q], mean, inv_sd);
                ms.u64[q][j] = mean;
                ms.v64[q][j] = inv_sd;
                ms.u32[q][j] = (float)mean;
                ms.v32[q][j] = (float)inv_sd;
            }
        }
    }
}

template <int NS>
static int launch_counts_multi_n(iht_dataset *ds, const MultiSets &ms)
{
    const int blocks = (int)std::min<int64_t>(ceil_div(ds->p, 8 * 32), (int64_t)ds->ctx->num_sms * 8);
    k_counts_multi<NS><<<blocks, 256, 0, ds->ctx->stream>>>(ds->G, ds->p, ds->stride, ds->rowb, ms);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

// Statistics of several row sets (rowmasks already built), kMultiSets per pass.
int launch_counts_sets(iht_dataset *ds, const RowSet *sets, const int64_t *n_rows, int nsets)
{
    for (int s0 = 0; s0 < nsets; s0 += kMultiSets) {
        const int ns = std::min(kMultiSets, nsets - s0);
        MultiSets ms{};
        for (int q = 0; q < ns; ++q) {
            const RowSet &r = sets[s0 + q];
            ms.rowmask[q] = r.rowmask;
            ms.n_rows[q] = n_rows[s0 + q];
            ms.u64[q] = r.u64;
            ms.v64[q] = r.v64;
            ms.u32[q] = r.u32;
            ms.v32[q] = r.v32;
        }
        int rc;
        switch (ns) {
        case 1: rc = launch_counts_multi_n<1>(ds, ms); break;
        case 2: rc = launch_counts_multi_n<2>(ds, ms); break;
        case 3: rc = launch_counts_multi_n<3>(ds, ms); break;
        case 4: rc = launch_counts_multi_n<4>(ds, ms); break;
        case 5: rc = launch_counts_multi_n<5>(ds, ms); break;
        case 6: rc = launch_counts_multi_n<6>(ds, ms); break;
        case 7: rc = launch_counts_multi_n<7>(ds, ms); break;
        default: rc = launch_counts_multi_n<8>(ds, ms); break;
        }
        if (rc) return rc;
    }
    return IHT_OK;
}

template <typename T>
__global__ void k_scatter(const int32_t *__restrict__ rows, int64_t n_rows, const T *__restrict__ src,
                          T *__restrict__ dst, int64_t n)
{
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_rows) return;
    const int64_t i = rows ? rows[a] : a;
    if (i >= 0 && i < n) dst[i] = src[a];
}

int scatter_rows_f64(iht_dataset *ds, const int32_t *rows_dev, int64_t n_rows, const double *src,
                     double *dst)
{
    cudaStream_t s = ds->ctx->stream;
    IHT_CUDA(cudaMemsetAsync(dst, 0, sizeof(double) * ds->n_pad, s));
    if (n_rows > 0) {
        k_scatter<double><<<ceil_div(n_rows, 256), 256, 0, s>>>(rows_dev, n_rows, src, dst, ds->n);
        note_launch();
    }
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

int scatter_rows_f32(iht_dataset *ds, const int32_t *rows_dev, int64_t n_rows, const float *src,
                     float *dst)
{
    cudaStream_t s = ds->ctx->stream;
    IHT_CUDA(cudaMemsetAsync(dst, 0, sizeof(float) * ds->n_pad, s));
    if (n_rows > 0) {
        k_scatter<float><<<ceil_div(n_rows, 256), 256, 0, s>>>(rows_dev, n_rows, src, dst, ds->n);
        note_launch();
    }
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

// ---------------------------------------------------------------------------
// Missing-call lists: the gradient needs M_j = sum of r over the missing calls
// of SNP j; missing calls are rare (1-2 %), so a per-SNP list of their sample
// offsets, built once, lets a small pass form M_j and keeps the dense pass free
// of data-dependent branches.

// Missing-code mask of word c (samples 16c..16c+15) restricted to samples < n.
__device__ __forceinline__ uint32_t missing_mask(uint32_t w, int64_t c, int64_t n)
{
    uint32_t mm = w & ~(w >> 1) & 0x55555555u;
    const int64_t left = n - 16 * c;
    if (left < 16) mm &= left > 0 ? (uint32_t)((1ull << (2 * left)) - 1ull) : 0u;
    return mm;
}

__global__ void __launch_bounds__(256) k_miss_count(const uint8_t *__restrict__ G, int64_t p,
                                                    int64_t stride, int64_t n,
                                                    int32_t *__restrict__ cnt)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t nw = (n + 15) / 16;
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < p; j += nwarps) {
        const uint32_t *row = reinterpret_cast<const uint32_t *>(G + j * stride);
        int c = 0;
        for (int64_t w = lane; w < nw; w += 32) c += __popc(missing_mask(__ldg(row + w), w, n));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) cnt[j] = c;
    }
}

template <typename IdxT>
__global__ void __launch_bounds__(256) k_miss_fill(const uint8_t *__restrict__ G, int64_t p,
                                                   int64_t stride, int64_t n,
                                                   const int64_t *__restrict__ off,
                                                   IdxT *__restrict__ idx)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t nw = (n + 15) / 16;
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < p; j += nwarps) {
        const uint32_t *row = reinterpret_cast<const uint32_t *>(G + j * stride);
        int64_t pos = off[j];
        // residue classes (i - j) mod 8 in turn, ascending within a class: the
        // samples of class rho are fields rho and rho + 8 of every 16-sample word
        for (int cls = 0; cls < 8; ++cls)
        for (int64_t base = 0; base < nw; base += 32) {
            const int rho = (int)((j + cls) & 7);
            const uint32_t cmask = (1u << (2 * rho)) | (1u << (2 * rho + 16));
            const int64_t w = base + lane;
            uint32_t mm = w < nw ? missing_mask(__ldg(row + w), w, n) & cmask : 0u;
            const int c = __popc(mm);
            int x = c;   // inclusive warp scan
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            int64_t q = pos + x - c;
            while (mm) {
                const int b = __ffs(mm) - 1;
                idx[q++] = (IdxT)(16 * w + (b >> 1));
                mm &= mm - 1;
            }
            pos += __shfl_sync(0xffffffffu, x, 31);
        }
    }
}

// Padded lists (see iht_dataset): class counts of this lane's SNP j (0 past p)
// and, over the lane's group of kPadGroup lanes, the longest count of every
// class.  Called by all 32 lanes of a warp, j = 32 w + lane.
__device__ __forceinline__ int pad_classes(const int64_t *__restrict__ off, const uint16_t *__restrict__ idx,
                                           int64_t j, int64_t p, int (&cnt)[8], int (&len)[8])
{
#pragma unroll
    for (int c = 0; c < 8; ++c) cnt[c] = 0;
    if (j < p)
        for (int64_t e = off[j]; e < off[j + 1]; ++e) {
            const int cls = (int)(((int64_t)idx[e] - j) & 7);
#pragma unroll
            for (int c = 0; c < 8; ++c) cnt[c] += cls == c;
        }
    int L = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        int t = cnt[c];
#pragma unroll
        for (int o = 1; o < kPadGroup; o <<= 1) t = max(t, __shfl_xor_sync(0xffffffffu, t, o));
        len[c] = t;
        L += t;
    }
    return (L + 7) & ~7;
}

__global__ void __launch_bounds__(256) k_pad_len(const int64_t *__restrict__ off, const uint16_t *__restrict__ idx,
                                                 int64_t p, int32_t *__restrict__ glen)
{
    const int lane = threadIdx.x & 31;
    const int64_t ngroups = (p + kPadGroup - 1) / kPadGroup;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w * 32 < p; w += nwarps) {
        const int64_t j = 32 * w + lane;
        int cnt[8], len[8];
        const int L = pad_classes(off, idx, j, p, cnt, len);
        if ((lane & (kPadGroup - 1)) == 0 && j / kPadGroup < ngroups) glen[j / kPadGroup] = L;
    }
}

__global__ void __launch_bounds__(256) k_pad_fill(const int64_t *__restrict__ off, const uint16_t *__restrict__ idx,
                                                  int64_t p, int64_t n_pad, const int64_t *__restrict__ goff,
                                                  uint16_t *__restrict__ gidx)
{
    const int lane = threadIdx.x & 31;
    const int64_t ngroups = (p + kPadGroup - 1) / kPadGroup;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w * 32 < p; w += nwarps) {
        const int64_t j = 32 * w + lane;
        int cnt[8], len[8];
        const int L = pad_classes(off, idx, j, p, cnt, len);
        const int64_t g = j / kPadGroup;
        if (g >= ngroups) continue;
        uint16_t *dst = gidx + goff[g] + (j % kPadGroup) * (int64_t)L;
        int64_t e = j < p ? off[j] : 0;
        int pos = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            for (int t = 0; t < cnt[c]; ++t) dst[pos++] = idx[e++];
            const uint16_t z = (uint16_t)(n_pad + ((j + c) & 7));
            for (int t = cnt[c]; t < len[c]; ++t) dst[pos++] = z;
        }
        const uint16_t z = (uint16_t)(n_pad + (j & 7));
        while (pos < L) dst[pos++] = z;
    }
}

bool padded_lists_wanted(const iht_dataset *ds)
{
    return ds->miss_idx16 && 16 * ((size_t)ds->n_pad + 8) <= 200 * 1024;
}

static int build_padded_lists(iht_dataset *ds)
{
    cudaStream_t s = ds->ctx->stream;
    const int64_t p = ds->p, ngroups = (p + kPadGroup - 1) / kPadGroup;
    const int blocks = (int)std::min<int64_t>(ceil_div(p, 256), (int64_t)ds->ctx->num_sms * 8);
    int32_t *glen = nullptr;
    IHT_CUDA(dev_malloc(&glen, sizeof(int32_t) * ngroups));
    k_pad_len<<<blocks, 256, 0, s>>>(ds->miss_off, (const uint16_t *)ds->miss_idx, p, glen);
    note_launch();
    std::vector<int32_t> hl(ngroups);
    std::vector<int64_t> ho(ngroups + 1);
    cudaError_t e = cudaMemcpyAsync(hl.data(), glen, sizeof(int32_t) * ngroups, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(glen);
    if (e != cudaSuccess) {
        set_cuda_error(e, "padded list lengths");
        return IHT_ECUDA;
    }
    ho[0] = 0;
    for (int64_t g = 0; g < ngroups; ++g) ho[g + 1] = ho[g] + (int64_t)kPadGroup * hl[g];
    e = dev_malloc(&ds->miss_goff, sizeof(int64_t) * (ngroups + 1));
    // 16 spare entries: readers request the next 16-byte piece before they know it is needed
    if (e == cudaSuccess) e = dev_malloc(&ds->miss_gidx, sizeof(uint16_t) * (ho[ngroups] + 16));
    if (e == cudaSuccess) e = cudaMemsetAsync(ds->miss_gidx + ho[ngroups], 0, 16 * sizeof(uint16_t), s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ds->miss_goff, ho.data(), sizeof(int64_t) * (ngroups + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_cuda_error(e, "padded lists");
        return e == cudaErrorMemoryAllocation ? IHT_ENOMEM : IHT_ECUDA;
    }
    k_pad_fill<<<blocks, 256, 0, s>>>(ds->miss_off, (const uint16_t *)ds->miss_idx, p, ds->n_pad, ds->miss_goff,
                                      ds->miss_gidx);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

// Interleaved lists (see iht_dataset): group g's sequence length L_g, the
// longest list of its 32 SNPs rounded up to a multiple of 8.  One warp per group.
__global__ void __launch_bounds__(256) k_ilv_len(const int64_t *__restrict__ off, int64_t p,
                                                 int32_t *__restrict__ glen)
{
    const int lane = threadIdx.x & 31;
    const int64_t ngroups = (p + 31) / 32;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < ngroups; g += nwarps) {
        const int64_t j = 32 * g + lane;
        const int len = j < p ? (int)(off[j + 1] - off[j]) : 0;
        const int L = __reduce_max_sync(0xffffffffu, len);
        if (lane == 0) glen[g] = (L + 7) & ~7;
    }
}

// Entry t of lane l's sequence in group g sits at ioff[g] + 256 (t / 8) +
// 8 l + t mod 8; past the lane's list (and for lanes past p) it is the zero
// slot n_pad + l.
__global__ void __launch_bounds__(256) k_ilv_fill(const int64_t *__restrict__ off, const uint16_t *__restrict__ idx,
                                                  int64_t p, int64_t n_pad, const int64_t *__restrict__ ioff,
                                                  uint16_t *__restrict__ iidx)
{
    const int lane = threadIdx.x & 31;
    const int64_t ngroups = (p + 31) / 32;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < ngroups; g += nwarps) {
        const int64_t j = 32 * g + lane;
        const int64_t e0 = j < p ? off[j] : 0;
        const int len = j < p ? (int)(off[j + 1] - e0) : 0;
        const int L = (int)((ioff[g + 1] - ioff[g]) / 32);
        uint16_t *dst = iidx + ioff[g] + 8 * lane;
        const uint16_t z = (uint16_t)(n_pad + lane);
        for (int t = 0; t < L; ++t) dst[256 * (t >> 3) + (t & 7)] = t < len ? idx[e0 + t] : z;
    }
}

bool interleaved_lists_wanted(const iht_dataset *ds)
{
    return ds->miss_idx16 && ds->n_pad + 32 <= 65536 && sizeof(float) * (size_t)(ds->n_pad + 32) <= 160 * 1024;
}

static int build_interleaved_lists(iht_dataset *ds)
{
    cudaStream_t s = ds->ctx->stream;
    const int64_t p = ds->p, ngroups = (p + 31) / 32;
    const int blocks = (int)std::min<int64_t>(ceil_div(ngroups, 8), (int64_t)ds->ctx->num_sms * 8);
    int32_t *glen = nullptr;
    IHT_CUDA(dev_malloc(&glen, sizeof(int32_t) * ngroups));
    k_ilv_len<<<blocks, 256, 0, s>>>(ds->miss_off, p, glen);
    note_launch();
    std::vector<int32_t> hl(ngroups);
    std::vector<int64_t> ho(ngroups + 1);
    cudaError_t e = cudaMemcpyAsync(hl.data(), glen, sizeof(int32_t) * ngroups, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(glen);
    if (e != cudaSuccess) {
        set_cuda_error(e, "interleaved list lengths");
        return IHT_ECUDA;
    }
    ho[0] = 0;
    for (int64_t g = 0; g < ngroups; ++g) ho[g + 1] = ho[g] + 32 * (int64_t)hl[g];
    e = dev_malloc(&ds->miss_ioff, sizeof(int64_t) * (ngroups + 1));
    if (e == cudaSuccess) e = dev_malloc(&ds->miss_iidx, sizeof(uint16_t) * std::max<int64_t>(ho[ngroups], 8));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ds->miss_ioff, ho.data(), sizeof(int64_t) * (ngroups + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_cuda_error(e, "interleaved lists");
        return e == cudaErrorMemoryAllocation ? IHT_ENOMEM : IHT_ECUDA;
    }
    k_ilv_fill<<<blocks, 256, 0, s>>>(ds->miss_off, (const uint16_t *)ds->miss_idx, p, ds->n_pad, ds->miss_ioff,
                                      ds->miss_iidx);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

int build_missing_lists(iht_dataset *ds)
{
    cudaStream_t s = ds->ctx->stream;
    const int64_t p = ds->p;
    int32_t *cnt = nullptr;
    IHT_CUDA(dev_malloc(&cnt, sizeof(int32_t) * p));
    const int blocks = (int)std::min<int64_t>(ceil_div(p, 8), (int64_t)ds->ctx->num_sms * 16);
    k_miss_count<<<blocks, 256, 0, s>>>(ds->G, p, ds->stride, ds->n, cnt);
    note_launch();
    int32_t *hc = (int32_t *)malloc(sizeof(int32_t) * p);
    int64_t *ho = (int64_t *)malloc(sizeof(int64_t) * (p + 1));
    if (!hc || !ho) {
        free(hc);
        free(ho);
        cudaFree(cnt);
        return IHT_ENOMEM;
    }
    cudaError_t e = cudaMemcpyAsync(hc, cnt, sizeof(int32_t) * p, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(cnt);
    if (e != cudaSuccess) {
        free(hc);
        free(ho);
        set_cuda_error(e, "missing-call counts");
        return IHT_ECUDA;
    }
    ho[0] = 0;
    for (int64_t j = 0; j < p; ++j) ho[j + 1] = ho[j] + hc[j];
    free(hc);
    ds->miss_total = ho[p];
    e = dev_malloc(&ds->miss_off, sizeof(int64_t) * (p + 1));
    if (e == cudaSuccess)
        // 16 spare entries: readers load the lists in aligned 16-byte pieces
        e = dev_malloc(&ds->miss_idx, (ds->miss_total + 16) * (ds->miss_idx16 ? 2 : 4));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ds->miss_off, ho, sizeof(int64_t) * (p + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    free(ho);
    if (e != cudaSuccess) {
        set_cuda_error(e, "missing-call lists");
        return e == cudaErrorMemoryAllocation ? IHT_ENOMEM : IHT_ECUDA;
    }
    if (ds->miss_idx16)
        k_miss_fill<uint16_t><<<blocks, 256, 0, s>>>(ds->G, p, ds->stride, ds->n, ds->miss_off,
                                                     (uint16_t *)ds->miss_idx);
    else
        k_miss_fill<int32_t><<<blocks, 256, 0, s>>>(ds->G, p, ds->stride, ds->n, ds->miss_off,
                                                    (int32_t *)ds->miss_idx);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    if (interleaved_lists_wanted(ds)) {
        const int rc = build_interleaved_lists(ds);
        if (rc != IHT_OK) return rc;
    }
    return padded_lists_wanted(ds) ? build_padded_lists(ds) : IHT_OK;
}

// Limb image of the residual staged in shared memory (512-thread blocks): every
// block finds max |r| (the limbs' scale) itself and encodes its own share of
// the samples; block 0 forms R in the limb kernel's order.
__device__ __noinline__ void missing_limb_image(const float *rs, int64_t nlim, uint8_t *__restrict__ bimg,
                                                   TcParams *prm)
{
    __shared__ float smax[16];
    __shared__ double wsr[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float m = 0.0f;
    for (int64_t i = threadIdx.x; i < nlim; i += blockDim.x) m = fmaxf(m, fabsf(rs[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) smax[warp] = m;
    __syncthreads();
    m = 0.0f;
#pragma unroll 1
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, smax[w]);
    const float s0 = limb_scale(m);
    const int64_t per = (nlim + gridDim.x - 1) / gridDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * per, i1 = min(nlim, i0 + per);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) limb_encode(rs[i], s0, bimg, i);
    if (blockIdx.x == 0) {
        // thread h holds the limb kernel's residues t = h and t = h + 512
        double a0 = 0.0, a1 = 0.0;
        for (int64_t i = threadIdx.x; i < nlim; i += 1024) a0 += (double)rs[i];
        for (int64_t i = threadIdx.x + 512; i < nlim; i += 1024) a1 += (double)rs[i];
        a0 = warp_sum(a0);
        a1 = warp_sum(a1);
        if (lane == 0) {
            wsr[warp] = a0;
            wsr[warp + 16] = a1;
        }
        for (int b = threadIdx.x; b < 256; b += blockDim.x) bimg[256 + 256 * (nlim >> 5) + b] = 0;
        __syncthreads();
        if (warp == 0) {
            const double R = warp_sum(wsr[lane]);
            if (lane == 0) {
                prm->s0 = s0;
                prm->R = (float)R;
            }
        }
    }
}

// M_j = sum of r over the missing calls of SNP j.  The block stages r in
// shared memory; each lane owns one SNP and reads its list 16 bytes (8 or 4
// sample offsets) at a time, adding in list order; the next 16-byte piece is
// requested before the current one is summed, so one list latency is exposed
// per SNP rather than one per piece.
//
// With kLimbs (the fused solve), the blocks also write the next tensor-core
// pass's limb image of r, which otherwise the limb kernel writes: every block
// has all of r in shared memory, so each finds max |r| (the limbs' scale) by
// itself and encodes its own share of the samples, and block 0 forms R = sum
// of r in the limb kernel's order (a running FP64 sum per residue of i mod
// 1024, a shuffle tree per 32 residues, the same tree over the 32 warp sums)
// -- the limb kernel's bytes and R, bit for bit.
template <typename IdxT, bool kLimbs>
__global__ void __launch_bounds__(512) k_missing_sum_smem(const int64_t *__restrict__ off,
                                                          const IdxT *__restrict__ idx, int64_t p,
                                                          const float *__restrict__ r32,
                                                          int64_t n_pad, float *__restrict__ M,
                                                          const int32_t *__restrict__ done,
                                                          uint8_t *__restrict__ bimg, TcParams *prm,
                                                          int64_t nlim)
{
    extern __shared__ float rs_miss[];
    if (done && *done) return;
    constexpr int kPer = 16 / (int)sizeof(IdxT);
    for (int64_t i = threadIdx.x; i < n_pad; i += blockDim.x) rs_miss[i] = r32[i];
    __syncthreads();
    if constexpr (kLimbs) missing_limb_image(rs_miss, nlim, bimg, prm);
    const uint4 *__restrict__ idx4 = reinterpret_cast<const uint4 *>(idx);
    constexpr int kBatch = 8;                                 // 16-byte list pieces in flight
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e0 = __ldcs(&off[j]), e1 = __ldcs(&off[j + 1]);
        const int64_t a0 = e0 & ~(int64_t)(kPer - 1);
        const int lo = (int)(e0 - a0), hi = (int)(e1 - a0);   // valid positions [lo, hi) from a0
        const uint4 *__restrict__ src = idx4 + a0 / kPer;     // (lists end with 16 spare entries)
        const int nq = (hi + kPer - 1) / kPer;                // pieces holding the list
        float m = 0.0f;
        for (int q0 = 0; q0 < nq; q0 += kBatch) {
            uint4 w[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u)
                if (q0 + u < nq) w[u] = __ldcs(src + q0 + u);   // read once a pass: evict first
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                if (q0 + u >= nq) break;
                const IdxT *ent = reinterpret_cast<const IdxT *>(&w[u]);
#pragma unroll
                for (int t = 0; t < kPer; ++t) {
                    const int pos = (q0 + u) * kPer + t;
                    if (pos >= lo && pos < hi) m += rs_miss[ent[t]];
                }
            }
        }
        M[j] = m;
    }
}

// The same sums over the interleaved lists (iht_dataset::miss_ioff): a warp
// takes whole groups of 32 SNPs, lane l SNP 32 g + l, and piece q of group g
// -- 512 contiguous bytes, entries 8q .. 8q+7 of every lane's sequence -- is
// one coalesced request of the warp instead of 32 scattered 16-byte ones.
// Two pieces are requested ahead of the two being summed, and the next
// group's offsets ahead of the group.  Pads index the 32 zero slots after r
// (lane l's at n_pad + l, a bank of its own); adding +0.0f to a sum that
// starts at 0.0f leaves it unchanged, so every M_j is the plain lists' sum in
// the same order, bit for bit.
__device__ __forceinline__ float miss_sum8(float m, uint4 w, const float *rs)
{
    m += rs[w.x & 0xffffu];
    m += rs[w.x >> 16];
    m += rs[w.y & 0xffffu];
    m += rs[w.y >> 16];
    m += rs[w.z & 0xffffu];
    m += rs[w.z >> 16];
    m += rs[w.w & 0xffffu];
    m += rs[w.w >> 16];
    return m;
}

template <bool kLimbs>
__global__ void __launch_bounds__(512, 3) k_missing_sum_ilv(const int64_t *__restrict__ ioff,
                                                            const uint16_t *__restrict__ iidx, int64_t p,
                                                            const float *__restrict__ r32, int64_t n_pad,
                                                            float *__restrict__ M,
                                                            const int32_t *__restrict__ done,
                                                            uint8_t *__restrict__ bimg, TcParams *prm,
                                                            int64_t nlim)
{
    extern __shared__ __align__(16) float rs_miss[];   // r, then 32 zero slots
    grid_dep_launch();
    const int lane = threadIdx.x & 31;
    const int64_t ngroups = (p + 31) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint4 *__restrict__ i4 = reinterpret_cast<const uint4 *>(iidx);
    // the first group's offsets and first two pieces are requested before r is staged
    int64_t a = 0, b = 0;
    if (g < ngroups) {
        a = __ldg(&ioff[g]);
        b = __ldg(&ioff[g + 1]);
    }
    uint4 w0 = make_uint4(0u, 0u, 0u, 0u), w1 = w0;
    if (b - a > 0) w0 = __ldcs(i4 + (a >> 3) + lane);
    if (b - a > 256) w1 = __ldcs(i4 + (a >> 3) + 32 + lane);
    grid_dep_wait();   // r and the stop flag, when launched programmatically after the kernel forming them
    if (done && *done) return;
    if ((reinterpret_cast<uintptr_t>(r32) & 15u) == 0 && (n_pad & 3) == 0) {
        const float4 *__restrict__ r4 = reinterpret_cast<const float4 *>(r32);
        float4 *rs4 = reinterpret_cast<float4 *>(rs_miss);
        for (int64_t i = threadIdx.x; i < (n_pad >> 2); i += blockDim.x) rs4[i] = __ldcg(r4 + i);
    } else {
        for (int64_t i = threadIdx.x; i < n_pad; i += blockDim.x) rs_miss[i] = __ldcg(r32 + i);
    }
    if (threadIdx.x < 32) rs_miss[n_pad + threadIdx.x] = 0.0f;
    __syncthreads();
    if constexpr (kLimbs) missing_limb_image(rs_miss, nlim, bimg, prm);
    for (; g < ngroups; g += nwarps) {
        const int64_t gn = g + nwarps;
        int64_t an = 0, bn = 0;
        if (gn < ngroups) {
            an = __ldg(&ioff[gn]);
            bn = __ldg(&ioff[gn + 1]);
        }
        const int nq = (int)((b - a) >> 8);                 // pieces of 256 entries
        const uint4 *__restrict__ src = i4 + (a >> 3) + lane;
        float m = 0.0f;
#pragma unroll 1
        for (int q = 0; q < nq; q += 2) {
            uint4 n0 = w0, n1 = w1;
            if (q + 2 < nq) n0 = __ldcs(src + 32 * (q + 2));
            if (q + 3 < nq) n1 = __ldcs(src + 32 * (q + 3));
            m = miss_sum8(m, w0, rs_miss);
            if (q + 1 < nq) m = miss_sum8(m, w1, rs_miss);
            w0 = n0;
            w1 = n1;
        }
        const int64_t j = (g << 5) + lane;
        if (j < p) M[j] = m;
        a = an;
        b = bn;
        if (b - a > 0) w0 = __ldcs(i4 + (a >> 3) + lane);
        if (b - a > 256) w1 = __ldcs(i4 + (a >> 3) + 32 + lane);
    }
}

// (global-memory variant for residuals too long for shared memory)
// M_j = sum of r over the missing calls of SNP j.  Four lanes per SNP (eight
// SNPs per warp, 16 list entries in flight per group), fixed summation order.
template <typename IdxT>
__global__ void __launch_bounds__(256) k_missing_sum(const int64_t *__restrict__ off,
                                                     const IdxT *__restrict__ idx, int64_t p,
                                                     const float *__restrict__ r32,
                                                     float *__restrict__ M,
                                                     const int32_t *__restrict__ done)
{
    if (done && *done) return;
    const int lane = threadIdx.x & 31, q = lane & 3;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * 8; base < p; base += nwarps * 8) {      // warp-uniform
        const int64_t j = base + (lane >> 2);
        const bool live = j < p;
        const int64_t e0 = live ? off[j] : 0, e1 = live ? off[j + 1] : 0;
        float m = 0.0f;
        for (int64_t e = e0 + q; e < e1; e += 16) {
            IdxT i[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) i[t] = e + 4 * t < e1 ? idx[e + 4 * t] : (IdxT)0;
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (e + 4 * t < e1) m += __ldg(r32 + i[t]);
        }
        m += __shfl_xor_sync(0xffffffffu, m, 1);
        m += __shfl_xor_sync(0xffffffffu, m, 2);
        if (live && q == 0) M[j] = m;
    }
}

bool missing_limbs_supported(const iht_dataset *ds, int64_t nlim)
{
    return sizeof(float) * (size_t)ds->n_pad <= 160 * 1024 && nlim <= ds->n_pad;
}

template <bool kLimbs>
static int launch_missing_ilv(iht_dataset *ds, const float *r32, float *M, const int32_t *done,
                              uint8_t *bimg, TcParams *prm, int64_t nlim, bool programmatic)
{
    const size_t smem = sizeof(float) * (size_t)(ds->n_pad + 32);
    static thread_local int configured = -1, per_sm = 1;
    static thread_local size_t sized = 0;
    if (configured != ds->ctx->device) {
        IHT_CUDA(cudaFuncSetAttribute(k_missing_sum_ilv<kLimbs>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      160 * 1024));
        configured = ds->ctx->device;
        sized = 0;
    }
    if (sized != smem) {   // resident blocks per SM for this residual length
        IHT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_missing_sum_ilv<kLimbs>, 512, smem));
        per_sm = std::max(per_sm, 1);
        sized = smem;
    }
    const int64_t ngroups = (ds->p + 31) / 32;
    const int blocks = (int)std::min<int64_t>(std::max<int64_t>(ceil_div(ngroups, 16), 1),
                                              (int64_t)ds->ctx->num_sms * per_sm);
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)blocks);
    lc.blockDim = dim3(512);
    lc.dynamicSmemBytes = smem;
    lc.stream = ds->ctx->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = programmatic ? 1 : 0;
    const cudaError_t e = cudaLaunchKernelEx(&lc, k_missing_sum_ilv<kLimbs>, (const int64_t *)ds->miss_ioff,
                                             (const uint16_t *)ds->miss_iidx, ds->p, r32, ds->n_pad, M, done,
                                             bimg, prm, nlim);
    note_launch();
    IHT_CUDA(e);
    return IHT_OK;
}

template <bool kLimbs>
static int launch_missing_smem(iht_dataset *ds, const float *r32, float *M, const int32_t *done,
                               uint8_t *bimg, TcParams *prm, int64_t nlim, bool programmatic = false)
{
    if (ds->miss_iidx) return launch_missing_ilv<kLimbs>(ds, r32, M, done, bimg, prm, nlim, programmatic);
    cudaStream_t s = ds->ctx->stream;
    const size_t smem = sizeof(float) * (size_t)ds->n_pad;
    static thread_local int configured = -1;
    if (configured != ds->ctx->device) {
        IHT_CUDA(cudaFuncSetAttribute(k_missing_sum_smem<uint16_t, kLimbs>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
        IHT_CUDA(cudaFuncSetAttribute(k_missing_sum_smem<int32_t, kLimbs>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
        configured = ds->ctx->device;
    }
    int per_sm = 1;   // resident blocks per SM (registers and shared memory)
    if (ds->miss_idx16)
        IHT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_missing_sum_smem<uint16_t, kLimbs>, 512,
                                                               smem));
    else
        IHT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_missing_sum_smem<int32_t, kLimbs>, 512,
                                                               smem));
    const int blocks = (int)std::min<int64_t>(std::max<int64_t>(ceil_div(ds->p, 512), 1),
                                              (int64_t)ds->ctx->num_sms * std::max(per_sm, 1));
    if (ds->miss_idx16)
        k_missing_sum_smem<uint16_t, kLimbs><<<blocks, 512, smem, s>>>(
            ds->miss_off, (const uint16_t *)ds->miss_idx, ds->p, r32, ds->n_pad, M, done, bimg, prm, nlim);
    else
        k_missing_sum_smem<int32_t, kLimbs><<<blocks, 512, smem, s>>>(
            ds->miss_off, (const int32_t *)ds->miss_idx, ds->p, r32, ds->n_pad, M, done, bimg, prm, nlim);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

int launch_missing_sums_limbs(iht_dataset *ds, const float *r32, float *M, const int32_t *done,
                              uint8_t *bimg, TcParams *prm, int64_t nlim, bool programmatic)
{
    if (!missing_limbs_supported(ds, nlim)) return IHT_EINVAL;
    return launch_missing_smem<true>(ds, r32, M, done, bimg, prm, nlim, programmatic);
}

int launch_missing_sums(iht_dataset *ds, const float *r32, float *M, const int32_t *done)
{
    cudaStream_t s = ds->ctx->stream;
    const size_t smem = sizeof(float) * (size_t)ds->n_pad;
    if (smem <= 160 * 1024) return launch_missing_smem<false>(ds, r32, M, done, nullptr, nullptr, 0);
    const int blocks = (int)std::min<int64_t>(ceil_div(ds->p, 64), (int64_t)ds->ctx->num_sms * 16);
    if (ds->miss_idx16)
        k_missing_sum<uint16_t><<<blocks, 256, 0, s>>>(ds->miss_off, (const uint16_t *)ds->miss_idx,
                                                       ds->p, r32, M, done);
    else
        k_missing_sum<int32_t><<<blocks, 256, 0, s>>>(ds->miss_off, (const int32_t *)ds->miss_idx,
                                                      ds->p, r32, M, done);
    note_launch();
    IHT_CUDA(cudaGetLastError());
    return IHT_OK;
}

}  // namespace iht
