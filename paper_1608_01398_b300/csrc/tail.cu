// One IHT iteration after its gradient pass as a single cooperative kernel,
// and a whole solve as one CUDA graph launch.
//
// Between two gradient passes an iteration (Sec. 2.2-2.3.1) is a chain of small
// dependent steps: the top-2k candidates of |g|, g_S and Z_S g_S for the step
// size, the projection, the residual of the candidate, the backtracking test
// (repeated while it rejects) and the centred residual.  As separate launches
// each step costs a launch and a drain of the GPU; here they are the phases of
// one kernel whose blocks meet at grid barriers (a cooperative launch, so every
// block is resident; every wait is bounded and a barrier that gives up stops
// the solve with an error word the host reads).  Where every block can form
// the same result from the same inputs (the candidates, the projection, the
// decisions), the blocks that need it do so, instead of one block doing it
// between two barriers.  Each phase runs the same device code as the separate
// kernels (bodies.cuh, select_bodies.cuh), so a solve gives the same bits on
// either path and in a batch.
//
// The solve graph holds the solve's set-up (first gradient pass, S^0) and a
// conditional while node whose body is this kernel, the missing-call sums
// (which also write the next pass's limb image) and the gradient pass; the
// kernel clears the condition once the solve has stopped, so the host
// synchronises once per solve.
#include "bodies.cuh"
#include "limbs.cuh"
#include "select_bodies.cuh"

namespace iht {

constexpr int kTailThreads = kZmulThreads;    // one 128-sample block of the sparse product per pass
constexpr int kTailKM = 256;                  // largest k of the fused path
constexpr int kTailKept = 1024;               // candidates the selection's narrow finish sorts
constexpr int kFusedUnroll = 2;               // iterations per trip of the fused solve's conditional loop
constexpr uint32_t kBarSpin = 1u << 22;       // bounded barrier waits (polls; sleeps up to 256 ns each)

struct TailWork {                     // zeroed before every solve
    unsigned long long bar_count;     // grid barrier: arrivals since the solve began (+ kBarAbort)
    int bar_err, pad_;                // 1: a barrier wait gave up
    double num;                       // ||g_S||^2, from the blocks that form Z_S g_S
    Scalars spec;                     // the second candidate's projection scalars (mu / kappa)
    SelState st;                      // selection state (boundary bin, candidate count)
    alignas(16) uint32_t hist[kSelBins];   // histogram of |g| bits 30..20
    unsigned long long cand[kSelCap]; // candidate words (key << 32 | ~index)
};

struct TailArgs {
    const uint8_t *G;
    int64_t stride, rowb, n_pad, p, P;   // P = p + covariates
    const double *zc;                    // standardised covariates, or null
    Scalars *sc;
    const float *g;
    int32_t *S, *Sp, *Sp2;
    double *bS, *bSp, *coef, *bSp2;
    const double *u64, *v64;
    const int32_t *used;
    const double *y64;
    double *r64, *rc64, *zv, *rc64_2;
    float *r32;
    double *partials, *partials2;
    int npart;                           // 128-sample blocks of the sparse product
    int k, K;
    TailWork *T;
    uint8_t *bimg;                       // limb image of the next pass (the missing-call sums write it)
    TcParams *prm;
    int64_t nlim;                        // samples the limb image covers
    int own_hist;                        // 1: phase A forms the histogram of |g| (else the
                                         //   gradient pass before this kernel counted its keys)
    cudaGraphConditionalHandle cond;
};

// Grid-wide barrier on one monotone arrival count: every block of every
// launch passes the same barriers, so the count is a multiple of the grid at
// each barrier's start and the barrier the arrival old + 1 belongs to ends at
// the next multiple.  Thread 0 arrives after the block's writes (block
// barrier, then a device-scope fence) and, unless it is the last to arrive,
// polls the count with a bounded number of short sleeps; a block that gives up
// adds kBarAbort, which every waiter (now and at later barriers) sees at once.
// One atomic per block and no reset: the last block to arrive leaves at once.
// Returns false when this block or another gave up.
constexpr unsigned long long kBarAbort = 1ull << 62;

__device__ __forceinline__ bool grid_sync(TailWork *T)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long G = gridDim.x;
        __threadfence();
        const unsigned long long old = atomicAdd(&T->bar_count, 1ull);
        int ok = old < kBarAbort;
        if (ok) {
            const unsigned long long target = (old / G + 1) * G;
            volatile unsigned long long *cnt = &T->bar_count;
            unsigned long long now = old + 1;
            uint32_t it = 0, ns = 32;
            while (now < target) {
                if (++it > kBarSpin) {
                    atomicAdd(&T->bar_count, kBarAbort);
                    atomicExch(&T->bar_err, 1);
                    break;
                }
                // back off: the blocks still at work (often block 0 alone) do
                // not queue behind the polls in L2
                __nanosleep(ns);
                if (ns < 256) ns <<= 1;
                now = *cnt;
            }
            ok = now >= target && now < kBarAbort;
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Block 0 runs the serial steps (step size, projection, decisions) on a
// shared-memory copy of the solve's scalars and writes it back before every
// grid barrier, so the other blocks read the current values after it; no
// other block writes them.
constexpr int kScWords = (int)(sizeof(Scalars) / sizeof(unsigned long long));
static_assert(sizeof(Scalars) % sizeof(unsigned long long) == 0, "Scalars: whole words");

__device__ __forceinline__ bool grid_sync_put(TailWork *T, Scalars *sc, const Scalars *ssc, bool b0)
{
    __syncthreads();
    if (b0 && threadIdx.x < kScWords)
        reinterpret_cast<unsigned long long *>(sc)[threadIdx.x] =
            reinterpret_cast<const unsigned long long *>(ssc)[threadIdx.x];
    return grid_sync(T);
}

__device__ __forceinline__ void tail_stop(const TailArgs &A)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicExch(&A.T->bar_err, 1);
        A.sc->done = 1;
        cudaGraphSetConditional(A.cond, 0u);
    }
}

__global__ void __launch_bounds__(kTailThreads) k_tail(const __grid_constant__ TailArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t res[3];
    __shared__ int s_state;
    TailWork *T = A.T;
    Scalars *sc = A.sc;
    const int tid = threadIdx.x;
    const bool b0 = blockIdx.x == 0;

    __shared__ Scalars ssc;               // the block's working copy of the scalars (block 0's is the solve's)
    grid_dep_launch();   // the missing-call sums may launch now; they wait for this grid before reading

    // Z_S g_S for the step size, in B: on the nden blocks no candidate needs
    // (which then leave the candidate scan to the others), or, when every
    // block forms a candidate's residual, on the last blocks besides their scan
    const int nfree = (int)gridDim.x - 2 * A.npart;
    const int nden = nfree > 0 ? min(nfree, A.npart) : 0;
    const bool den_block = nden > 0 && (int)blockIdx.x >= 2 * A.npart && (int)blockIdx.x < 2 * A.npart + nden;

    // the histogram of |g| for B in registers, thread t holding bins 2047 -
    // (16 t + i) in hc[i]; requested first when the pass before this kernel
    // counted it
    static_assert(kTailThreads * 16 == kSelBins, "one 16-bin slice of the histogram per thread");
    uint32_t hc[16];
    auto load_hist = [&]() {
        const uint4 *h4 = reinterpret_cast<const uint4 *>(T->hist + kSelBins - 16 * (tid + 1));
        const uint4 q0 = __ldcg(h4), q1 = __ldcg(h4 + 1), q2 = __ldcg(h4 + 2), q3 = __ldcg(h4 + 3);
        const uint32_t w[16] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w,
                                q2.x, q2.y, q2.z, q2.w, q3.x, q3.y, q3.z, q3.w};
#pragma unroll
        for (int i = 0; i < 16; ++i) hc[i] = w[15 - i];
    };
    if (!A.own_hist && !den_block) load_hist();
    // S for Z_S g_S, requested first on the blocks that form it (the barrier
    // after the scalars' copy makes it visible)
    __shared__ int32_t s_Sd[kTailKM];
    if (den_block)
#pragma unroll 1
        for (int c = tid; c < A.k; c += blockDim.x) s_Sd[c] = A.S[c];
    if (tid == 0) s_state = *(volatile int32_t *)&sc->done;
    if (tid < kScWords)
        reinterpret_cast<unsigned long long *>(&ssc)[tid] =
            reinterpret_cast<const volatile unsigned long long *>(sc)[tid];
    __syncthreads();
    if (s_state) {
        if (b0 && tid == 0) cudaGraphSetConditional(A.cond, 0u);
        return;
    }

    // A (when the gradient pass before this kernel did not count its keys): the
    // histogram of |g| over every block
    if (A.own_hist) {
        uint32_t *hs = reinterpret_cast<uint32_t *>(smem_raw);
#pragma unroll 1
        for (int b = tid; b < kSelBins; b += blockDim.x) hs[b] = 0;
        __syncthreads();
        bool nan = false;
        sel_each(A.g, A.P, [&](float x, int64_t) {
            const uint32_t key = sel_key(x);
            nan |= key > 0x7f800000u;
            atomicAdd(&hs[key >> 20], 1u);
        });
        if (nan) atomicOr(&T->st.err, 1u);
        __syncthreads();
#pragma unroll 1
        for (int b = tid; b < kSelBins; b += blockDim.x)
            if (hs[b]) atomicAdd(&T->hist[b], hs[b]);
        if (!grid_sync_put(T, sc, &ssc, b0)) return tail_stop(A);
    }

    // g_S (in shared memory) for the blocks that form Z_S g_S; the one that
    // forms sample block 0 publishes ||g_S||^2 in T->num before it is counted
    // g_S (and, for sample block 0, ||g_S||^2 to T->num) and this block's
    // samples of Z_S g_S; S in s_Sd (staged by the caller), the genotype bytes
    // of the columns requested into L2 together with g_S
    __shared__ double s_coef[kTailKM];
    auto zsgs = [&](int vb) {
        const uint8_t *gb = A.G + (int64_t)vb * kZmulBytes;
#pragma unroll 1
        for (int c = tid; c < A.k; c += blockDim.x) {
            const int32_t j = s_Sd[c];
            s_coef[c] = (double)A.g[j];
            if (j < A.p) asm volatile("prefetch.global.L2 [%0];" ::"l"(gb + (int64_t)j * A.stride));
        }
        __syncthreads();
        if (vb == 0 && tid < 32) {
            const double s = gS_sumsq_warp(s_coef, A.k);
            if (tid == 0) T->num = s;
        }
        zmul_body(A.G, A.stride, A.rowb, s_Sd, A.k, s_coef, 1.0, A.u64, A.v64, A.used, nullptr, nullptr,
                  A.zv, A.partials, A.n_pad, A.p, A.zc, vb);
    };

    // B: the boundary bin (every scanning block, from the whole histogram) and
    // the keys in or above it as candidate words
    if (den_block) {
#pragma unroll 1
        for (int vb = (int)blockIdx.x - 2 * A.npart; vb < A.npart; vb += nden) zsgs(vb);
    } else {
        if (A.own_hist) load_hist();
        sel_find_regs<16>(hc, (uint32_t)A.K, wsum, res);
        const uint32_t lo = res[0] << 20, ncand = res[1] + res[2];
        const int sb = (int)blockIdx.x < 2 * A.npart ? (int)blockIdx.x : (int)blockIdx.x - nden;
        if (ncand <= (uint32_t)kSelCap)
            sel_each(A.g, A.P, [&](float x, int64_t j) {
                const uint32_t key = sel_key(x);
                if (key >= lo) {
                    const uint32_t slot = atomicAdd(&T->st.n_gt, 1u);
                    if (slot < (uint32_t)kSelCap)
                        T->cand[slot] = ((unsigned long long)key << 32) | (unsigned long long)(~(uint32_t)j);
                }
            }, sb, (int)gridDim.x - nden);
        if (b0 && tid == 0) {
            T->st.prefix = res[0] << 20;
            T->st.mask = 0x7ffu << 20;
            T->st.count_gt = res[1];
            T->st.need = (uint32_t)A.K - res[1];
            T->st.ncand = ncand;
        }
        if (nden == 0 && (int)gridDim.x - 1 - (int)blockIdx.x < A.npart) {
#pragma unroll 1
            for (int c = tid; c < A.k; c += blockDim.x) s_Sd[c] = A.S[c];
            __syncthreads();
#pragma unroll 1
            for (int vb = (int)gridDim.x - 1 - (int)blockIdx.x; vb < A.npart; vb += gridDim.x) zsgs(vb);
        }
    }
    if (!grid_sync_put(T, sc, &ssc, b0)) return tail_stop(A);

    // C: every block that forms a candidate's residual selects the K candidates
    // and projects for itself (the same inputs give every block the same
    // result, so no barrier separates the steps): blocks v < npart take the
    // step mu, blocks npart <= v < 2 npart mu / kappa (the step the decision
    // takes when it rejects the first), and each forms its 128 samples of that
    // candidate's residual.  Block 0 keeps the first candidate (its scalars
    // are the solve's); the block of v = npart publishes the second one's.
    // The decisions then run in order on block 0 -- the same arithmetic as one
    // attempt after the other; later attempts, when both are rejected, run one
    // at a time.
    __shared__ int32_t s_cand[2 * kTailKM];
    __shared__ int32_t s_S[kTailKM];
    __shared__ double s_bS[kTailKM];
    __shared__ float s_gS[kTailKM];
    __shared__ int32_t s_Sp[2][kTailKM];
    __shared__ double s_bSp[2][kTailKM];
    __shared__ Scalars ssc2;              // the second candidate's scalars
    {
        bool want[2] = {false, false};
#pragma unroll 1
        for (int v = blockIdx.x; v < 2 * A.npart; v += gridDim.x) want[v >= A.npart] = true;
        if (b0) want[0] = true;
        if (want[0] || want[1]) {
            // the solve's scalars as block 0 wrote them back (||g_S||^2 follows
            // from T->num, published in B)
            if (tid < kScWords && !b0)
                reinterpret_cast<unsigned long long *>(&ssc)[tid] =
                    reinterpret_cast<const volatile unsigned long long *>(sc)[tid];
            const uint32_t ncand = res[1] + res[2];
            // the candidate words (when few enough to rank) requested first,
            // into registers, so their loads and S's are in flight together
            static_assert(4 * kTailThreads >= kSelRank, "four candidate words per thread");
            const bool stage_cand = ncand <= (uint32_t)kSelRank;
            unsigned long long cw[4] = {0ull, 0ull, 0ull, 0ull};
            if (stage_cand)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int i = tid + q * kTailThreads;
                    if (i < (int)ncand) cw[q] = __ldcg(&T->cand[i]);
                }
            // S, beta_S and g_S into shared memory for the projection, and the
            // genotype bytes of this block's residual on their way to L2, while
            // the candidates are chosen (S+ mostly repeats S)
            {
                const int vb0 = (int)blockIdx.x < A.npart ? (int)blockIdx.x : (int)blockIdx.x - A.npart;
                const uint8_t *gb = A.G + (int64_t)vb0 * kZmulBytes;
#pragma unroll 1
                for (int c = tid; c < A.k; c += blockDim.x) {
                    const int32_t j = A.S[c];
                    s_S[c] = j;
                    s_bS[c] = A.bS[c];
                    s_gS[c] = A.g[j];
                    if (j < A.p) asm volatile("prefetch.global.L2 [%0];" ::"l"(gb + (int64_t)j * A.stride));
                }
            }
            if (stage_cand) {
                unsigned long long *sk = reinterpret_cast<unsigned long long *>(smem_raw);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int i = tid + q * kTailThreads;
                    if (i < (int)ncand) sk[i] = cw[q];
                }
            }
            sel_finish_narrow(A.g, A.P, &T->st, T->cand, ncand, s_cand, (uint32_t)A.K,
                              reinterpret_cast<unsigned long long *>(smem_raw), kTailKept, wsum,
                              stage_cand);
            __syncthreads();
            if (tid == 0) ssc.num = *(volatile double *)&T->num;    // the step size's numerator
            __syncthreads();
#pragma unroll 1
            for (int c = 0; c < 2; ++c) {
                if (!want[c]) continue;
                if (c == 1 && tid < kScWords)
                    reinterpret_cast<unsigned long long *>(&ssc2)[tid] =
                        reinterpret_cast<const unsigned long long *>(&ssc)[tid];
                __syncthreads();
                MergeArgs M;
                M.g = A.g;
                M.S = s_S;
                M.bS = s_bS;
                M.cand = s_cand;
                M.K = A.K;
                M.partials = A.partials;
                M.npart = A.npart;
                M.first = 1;
                M.shrinks = c;
                M.skip = nullptr;
                M.Sp = s_Sp[c];
                M.bSp = s_bSp[c];
                M.sc = c ? &ssc2 : &ssc;
                M.gS = s_gS;
                merge_body<MergeSharedT<kTailKM>>(M);
                __syncthreads();
                const Scalars &ms = c ? ssc2 : ssc;
                if (ms.done) continue;            // g_S = 0 or a non-finite step: no candidate
                // block 0 decides on the first candidate from its own copy; the
                // block of v = npart publishes the second for it
                if (c == 1 && (int)(A.npart % gridDim.x) == (int)blockIdx.x) {
#pragma unroll 1
                    for (int i = tid; i < A.k; i += blockDim.x) {
                        A.Sp2[i] = s_Sp[1][i];
                        A.bSp2[i] = s_bSp[1][i];
                    }
                    if (tid < kScWords)
                        reinterpret_cast<unsigned long long *>(&T->spec)[tid] =
                            reinterpret_cast<const unsigned long long *>(&ssc2)[tid];
                }
#pragma unroll 1
                for (int v = blockIdx.x; v < 2 * A.npart; v += gridDim.x) {
                    if ((v >= A.npart) != (c == 1)) continue;
                    zmul_body(A.G, A.stride, A.rowb, s_Sp[c], A.k, s_bSp[c], -1.0, A.u64, A.v64, A.used,
                              A.y64, A.r64, c ? A.rc64_2 : A.rc64, c ? A.partials2 : A.partials, A.n_pad,
                              A.p, A.zc, c ? v - A.npart : v);
                }
            }
        }
        if (b0) {
#pragma unroll 1
            for (int b = tid; b < kSelBins; b += blockDim.x) T->hist[b] = 0;
            if (tid == 0) T->st.n_gt = 0;
        }
    }
    if (!grid_sync_put(T, sc, &ssc, b0)) return tail_stop(A);

    // D: every block takes the decisions itself -- the scalars block 0 wrote
    // back, both candidates' partial sums and the second one's scalars give
    // every block the same outcome -- so the centring needs no barrier; block
    // 0's scalars remain the solve's and only block 0 copies S+ into S.
    // Later attempts (both candidates rejected) run one at a time: projection
    // on block 0, residual on all, decision on block 0.
    __shared__ int s_acc2;                // 1: the second candidate was accepted
    if (!b0 && tid < kScWords)
        reinterpret_cast<unsigned long long *>(&ssc)[tid] =
            reinterpret_cast<const volatile unsigned long long *>(sc)[tid];
    __syncthreads();
    if (tid == 0) {
        s_state = ssc.done;
        s_acc2 = 0;
    }
    __syncthreads();
    if (!s_state) {
        __shared__ int s_second;
        // both candidates' decision values at once, with the body's own
        // expressions: warp c sums candidate c's partials and forms omega,
        // warp 2 + c its stopping measure and mu / kappa
        __shared__ double s_pre[2][6];
        {
            const int w = tid >> 5, c = w & 1, lane = tid & 31;
            const double dd = c ? T->spec.dd : ssc.dd;
            if (w < 2) {
                double ps, ps2, pzz;
                warp_partials(c ? A.partials2 : A.partials, A.npart, ps, ps2, pzz);
                if (lane == 0) {
                    s_pre[c][0] = ps;
                    s_pre[c][1] = ps2;
                    s_pre[c][2] = pzz;
                    s_pre[c][3] = (1.0 - ssc.c) * dd / pzz;
                }
            } else if (lane == 0) {
                const double bb = c ? T->spec.bb : ssc.bb, mu = c ? T->spec.mu : ssc.mu;
                s_pre[c][4] = sqrt(dd) / (sqrt(bb) + 1.0);
                s_pre[c][5] = mu / ssc.kappa;
            }
        }
        __syncthreads();
        int32_t *dS = b0 ? A.S : nullptr;
        double *dbS = b0 ? A.bS : nullptr;
        decide_body(&ssc, A.partials, A.npart, dS, dbS, s_Sp[0], s_bSp[0], TraceDev{}, s_pre[0]);
        __syncthreads();
        if (tid == 0) {
            s_second = ssc.retry && !ssc.done && ssc.bt_last == 1;
            if (s_second) {                      // the second candidate is the shrunk step
                ssc.changed = T->spec.changed;
                ssc.dd = T->spec.dd;
                ssc.bb = T->spec.bb;
            }
        }
        __syncthreads();
        if (s_second) {
            decide_body(&ssc, A.partials2, A.npart, dS, dbS, A.Sp2, A.bSp2, TraceDev{}, s_pre[1]);
            __syncthreads();
            if (tid == 0) s_acc2 = !ssc.retry;
        }
        if (tid == 0) s_state = (ssc.done ? 1 : 0) | (ssc.retry ? 2 : 0);
        __syncthreads();
        if (!(s_state & 1) && (s_state & 2)) {
            while (!(s_state & 1) && (s_state & 2)) {
                if (b0) {
                    MergeArgs M;
                    M.g = A.g;
                    M.S = A.S;
                    M.bS = A.bS;
                    M.cand = s_cand;
                    M.K = A.K;
                    M.partials = A.partials;
                    M.npart = A.npart;
                    M.first = 0;
                    M.skip = nullptr;
                    M.Sp = A.Sp;
                    M.bSp = A.bSp;
                    M.sc = &ssc;
                    merge_body<MergeSharedT<kTailKM>>(M);
                }
                if (!grid_sync_put(T, sc, &ssc, b0)) return tail_stop(A);
#pragma unroll 1
                for (int vb = blockIdx.x; vb < A.npart; vb += gridDim.x)
                    zmul_body(A.G, A.stride, A.rowb, A.Sp, A.k, A.bSp, -1.0, A.u64, A.v64, A.used, A.y64,
                              A.r64, A.rc64, A.partials, A.n_pad, A.p, A.zc, vb);
                if (!grid_sync_put(T, sc, &ssc, b0)) return tail_stop(A);
                if (b0) decide_body(&ssc, A.partials, A.npart, A.S, A.bS, A.Sp, A.bSp, TraceDev{});
                if (!grid_sync_put(T, sc, &ssc, b0)) return tail_stop(A);
                if (tid == 0)
                    s_state = (*(volatile int32_t *)&sc->done ? 1 : 0) | (*(volatile int32_t *)&sc->retry ? 2 : 0);
                __syncthreads();
            }
            // the scalars block 0 wrote back at the last barrier
            if (!b0 && tid < kScWords)
                reinterpret_cast<unsigned long long *>(&ssc)[tid] =
                    reinterpret_cast<const volatile unsigned long long *>(sc)[tid];
            if (tid == 0) s_acc2 = 0;
            __syncthreads();
        }
    }

    // E: the accepted residual, centred (the next pass's limb image follows in
    // the missing-call sums kernel, which holds all of r in shared memory)
    if (tid == 0) s_state = ssc.done;
    __syncthreads();
    if (!s_state) {
        const double *acc = s_acc2 ? A.rc64_2 : A.rc64;
        const double mean = ssc.sum_r / (double)ssc.n_rows;
#pragma unroll 1
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + tid; i < A.n_pad;
             i += (int64_t)gridDim.x * blockDim.x) {
            const double v = acc[i];
            if (acc != A.r64) A.r64[i] = v;
            A.r32[i] = A.used[i] ? (float)(v - mean) : 0.0f;
        }
    }
    if (b0) {                             // block 0's scalars are the solve's
        __syncthreads();
        if (tid < kScWords)
            reinterpret_cast<unsigned long long *>(sc)[tid] = reinterpret_cast<const unsigned long long *>(&ssc)[tid];
        __syncthreads();
    }
    if (b0 && tid == 0) cudaGraphSetConditional(A.cond, ssc.done ? 0u : 1u);
}

// ---------------------------------------------------------------------------
// Host side.

static size_t tail_smem()
{
    return std::max(sizeof(MergeSharedT<kTailKM>), sizeof(unsigned long long) * (kSelCap + kTailKept));
}

bool fused_supported(const iht_dataset *ds, int k, int impl)
{
    return (impl == 0 || impl == 2) && grad_tc_supported(ds) && k <= kTailKM &&
           zmul_blocks(ds) <= kPartials;
}

void free_fused(Workspace *ws)
{
    if (ws->fused_exec) cudaGraphExecDestroy(ws->fused_exec);
    void *ptrs[] = {ws->tail, ws->Sp2, ws->bSp2, ws->rc64_2, ws->partials2, ws->sc_init};
    for (void *x : ptrs)
        if (x) cudaFree(x);
    if (ws->flags_host) cudaFreeHost(ws->flags_host);
    if (ws->out_host) cudaFreeHost(ws->out_host);
    ws->out_host = nullptr;
    ws->fused_exec = nullptr;
    ws->tail = nullptr;
    ws->Sp2 = nullptr;
    ws->bSp2 = ws->rc64_2 = ws->partials2 = nullptr;
    ws->sc_init = nullptr;
    ws->flags_host = nullptr;
}

// Blocks of the cooperative launch: one per SM when it fits (more blocks
// lengthen the barriers and multiply the histogram's global atomics).
static int tail_grid(iht_dataset *ds)
{
    static thread_local int cfg_dev = -1, per_sm = 0;
    if (cfg_dev != ds->ctx->device) {
        if (cudaFuncSetAttribute(k_tail, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tail_smem()) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tail, kTailThreads, tail_smem()) !=
                cudaSuccess)
            per_sm = 0;
        cfg_dev = ds->ctx->device;
    }
    return std::min(per_sm, 1) * ds->ctx->num_sms;
}

// Captures the solve loop: while (condition) { fused iteration; missing-call
// sums; gradient pass }.
// whole: the solve's set-up (enqueue_solve_setup, after clearing the kernel's
// work area) is captured as a child graph the loop depends on.
static int build_fused_graph(iht_dataset *ds, int k, int K, int impl, const TailArgs &args,
                             int grid, cudaGraphExec_t *exec, bool whole)
{
    Workspace *ws = ds->ws;
    cudaGraph_t graph = nullptr;
    IHT_CUDA(cudaGraphCreate(&graph, 0));
    cudaError_t e = cudaSuccess;
    if (!ws->cap_stream) {
        e = cudaStreamCreateWithFlags(&ws->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            cudaGraphDestroy(graph);
            set_cuda_error(e, "capture stream");
            return IHT_ECUDA;
        }
    }
    cudaGraphNode_t setup_node = nullptr;
    if (whole) {
        cudaStream_t user0 = ds->ctx->stream;
        ds->ctx->stream = ws->cap_stream;
        const uint64_t before0 = launches_noted();
        cudaGraph_t setup = nullptr;
        int rc0 = IHT_OK;
        e = cudaStreamBeginCapture(ws->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            e = cudaMemsetAsync(ws->tail, 0, sizeof(TailWork), ws->cap_stream);
            if (e == cudaSuccess) rc0 = enqueue_solve_setup(ds, k, impl, ws->tail->hist, &ws->tail->st.err);
            const cudaError_t e2 = cudaStreamEndCapture(ws->cap_stream, &setup);
            if (e == cudaSuccess) e = e2;
        }
        ds->ctx->stream = user0;
        ws->fused_setup_launches = (int)(launches_noted() - before0);
        note_launch(-ws->fused_setup_launches);            // captured, not run
        if (e == cudaSuccess && rc0 == IHT_OK)
            e = cudaGraphAddChildGraphNode(&setup_node, graph, nullptr, 0, setup);
        if (setup) cudaGraphDestroy(setup);
        if (e != cudaSuccess || rc0 != IHT_OK) {
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) set_cuda_error(e, "fused solve set-up capture");
            return rc0 != IHT_OK ? rc0 : IHT_ECUDA;
        }
    }
    cudaGraphConditionalHandle cond;
    e = cudaGraphConditionalHandleCreate(&cond, graph, 1u, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t node;
    if (e == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&node, graph, whole ? &setup_node : nullptr, nullptr, whole ? 1 : 0, &cp);
    }
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        set_cuda_error(e, "fused solve graph");
        return IHT_ECUDA;
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t user = ds->ctx->stream;
    ds->ctx->stream = ws->cap_stream;
    const uint64_t before = launches_noted();
    e = cudaStreamBeginCaptureToGraph(ws->cap_stream, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    int rc = IHT_OK;
    if (e == cudaSuccess) {
        TailArgs a = args;
        a.cond = cond;
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3((unsigned)grid);
        lc.blockDim = dim3(kTailThreads);
        lc.dynamicSmemBytes = tail_smem();
        lc.stream = ws->cap_stream;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        lc.attrs = at;
        lc.numAttrs = 1;
        // kFusedUnroll iterations per trip of the conditional loop (a trip's
        // relaunch of the body costs more than a few kernels that return at
        // once after the solve has stopped)
        const int32_t *done = &ws->sc->done;
        // the pass counts its keys into the next trip's histogram unless the
        // kernel forms it itself
        uint32_t *hist = args.own_hist ? nullptr : ws->tail->hist;
        uint32_t *hflag = args.own_hist ? nullptr : &ws->tail->st.err;
#pragma unroll 1
        for (int u = 0; u < kFusedUnroll && rc == IHT_OK; ++u) {
            e = cudaLaunchKernelEx(&lc, k_tail, a);
            note_launch();
            if (e != cudaSuccess) {
                set_cuda_error(e, "fused iteration launch");
                rc = IHT_ECUDA;
            }
            if (rc == IHT_OK)
                rc = launch_missing_sums_limbs(ds, ws->r32, ws->Mj, done, args.bimg, args.prm, args.nlim, true);
            if (rc == IHT_OK) rc = launch_grad_tc_main(ds, ws->r32, ws->g, done, hist, hflag, true);
            if (rc == IHT_OK) rc = launch_cov_grad(ds, ws->r32, ws->g, done, hist, hflag);
        }
        cudaGraph_t captured = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(ws->cap_stream, &captured);
        if (rc == IHT_OK && e2 != cudaSuccess) {
            set_cuda_error(e2, "fused solve capture");
            rc = IHT_ECUDA;
        }
    } else {
        set_cuda_error(e, "fused solve capture");
        rc = IHT_ECUDA;
    }
    ds->ctx->stream = user;
    const int n = (int)(launches_noted() - before);
    note_launch(-n);                                   // captured, not run
    if (rc == IHT_OK) {
        e = cudaGraphInstantiate(exec, graph, 0);
        if (e != cudaSuccess) {
            set_cuda_error(e, "fused solve instantiate");
            *exec = nullptr;
            rc = IHT_ECUDA;
        }
    }
    cudaGraphDestroy(graph);
    if (rc == IHT_OK) ws->fused_launches = n / kFusedUnroll;   // per iteration
    (void)k;
    (void)K;
    return rc;
}

// The fused graph for this solve's shape, built when its key changes: the
// loop alone (after a first gradient pass run outside), or with the solve's
// set-up ahead of it (whole).  EAGAIN when it cannot be built here.
static int ensure_fused_exec(iht_dataset *ds, int k, int K, int impl, bool whole, TcParams **prm_out)
{
    Workspace *ws = ds->ws;
    const int grid = tail_grid(ds);
    if (grid < 1) return IHT_EAGAIN;
    if (!ws->tail) {
        IHT_CUDA(dev_malloc(&ws->tail, sizeof(TailWork)));
        IHT_CUDA(dev_malloc(&ws->Sp2, sizeof(int32_t) * kTailKM));
        IHT_CUDA(dev_malloc(&ws->bSp2, sizeof(double) * kTailKM));
        IHT_CUDA(dev_malloc(&ws->rc64_2, sizeof(double) * ds->n_pad));
        IHT_CUDA(dev_malloc(&ws->partials2, sizeof(double) * 3 * kPartials));
    }
    uint8_t *bimg = nullptr;
    TcParams *prm = nullptr;
    int64_t nlim = 0;
    int rc = grad_tc_limb_buffers(ds, &bimg, &prm, &nlim);
    if (rc) return rc;
    if (!missing_limbs_supported(ds, nlim)) return IHT_EAGAIN;   // (the pass's B operand fits first)
    TailArgs a = {};
    a.G = ds->G;
    a.stride = ds->stride;
    a.rowb = ds->rowb;
    a.n_pad = ds->n_pad;
    a.p = ds->p;
    a.P = ds->p + ds->q;
    a.zc = ds->q > 0 ? ws->zc : nullptr;
    a.sc = ws->sc;
    a.g = ws->g;
    a.S = ws->S;
    a.Sp = ws->Sp;
    a.Sp2 = ws->Sp2;
    a.bS = ws->bS;
    a.bSp = ws->bSp;
    a.bSp2 = ws->bSp2;
    a.rc64_2 = ws->rc64_2;
    a.partials2 = ws->partials2;
    a.coef = ws->coef;
    a.u64 = ws->u64;
    a.v64 = ws->v64;
    a.used = ws->used;
    a.y64 = ws->y64;
    a.r64 = ws->r64;
    a.rc64 = ws->rc64;
    a.zv = ws->zv;
    a.r32 = ws->r32;
    a.partials = ws->partials;
    a.npart = zmul_blocks(ds);
    a.k = k;
    a.K = K;
    a.T = ws->tail;
    a.bimg = bimg;
    a.prm = prm;
    a.nlim = nlim;
    a.own_hist = whole ? 0 : 1;
    *prm_out = prm;
    const uint64_t key[12] = {(uint64_t)k | ((uint64_t)ds->q << 32),
                              (uint64_t)K, (uint64_t)impl | ((uint64_t)whole << 8),
                              (uint64_t)(uintptr_t)ws->tail, (uint64_t)(uintptr_t)bimg,
                              grad_tc_scratch_id(), (uint64_t)(uintptr_t)ws->S,
                              (uint64_t)(uintptr_t)ws->used, (uint64_t)grid,
                              (uint64_t)(uintptr_t)ds->G, (uint64_t)(uintptr_t)ds->ctx->sel.st,
                              (uint64_t)(uintptr_t)ws->zc};
    if (!ws->fused_exec || !std::equal(key, key + 12, ws->fused_key)) {
        if (ws->fused_exec) cudaGraphExecDestroy(ws->fused_exec);
        ws->fused_exec = nullptr;
        if (build_fused_graph(ds, k, K, impl, a, grid, &ws->fused_exec, whole) != IHT_OK) {
            cudaGetLastError();                        // the per-iteration graph runs instead
            return IHT_EAGAIN;
        }
        std::copy(key, key + 12, ws->fused_key);
    }
    return IHT_OK;
}

// After the first gradient pass and S (a resumed support): the rest of the
// solve as one graph launch.  Returns IHT_EAGAIN, with nothing enqueued, when
// the graph cannot be built here (the caller then runs the per-iteration
// graph); ETIMEOUT when a barrier of the fused kernel gave up.
int run_fused_solve(iht_dataset *ds, int k, int K, int impl)
{
    Workspace *ws = ds->ws;
    cudaStream_t s = ds->ctx->stream;
    TcParams *prm = nullptr;
    int rc = ensure_fused_exec(ds, k, K, impl, false, &prm);
    if (rc) return rc;
    IHT_CUDA(cudaMemsetAsync(ws->tail, 0, sizeof(TailWork), s));   // barrier, histogram, state
    IHT_CUDA(cudaGraphLaunch(ws->fused_exec, s));
    int err = 0;
    IHT_CUDA(cudaMemcpyAsync(&err, &ws->tail->bar_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    IHT_CUDA(cudaStreamSynchronize(s));
    return err ? IHT_ETIMEOUT : IHT_OK;
}

// A solve from beta = 0 as one graph launch: the starting scalars go to
// ws->sc_init (the graph's first kernel merges them with the set-up kernels'
// flags); the final scalars and both error words come back with one host
// synchronisation.
int run_whole_fused_solve(iht_dataset *ds, int k, int K, int impl, const Scalars &h)
{
    Workspace *ws = ds->ws;
    cudaStream_t s = ds->ctx->stream;
    if (!ws->sc_init) IHT_CUDA(dev_malloc(&ws->sc_init, sizeof(Scalars)));
    if (!ws->flags_host) {
        const cudaError_t e = cudaMallocHost((void **)&ws->flags_host, 2 * sizeof(int32_t));
        if (e != cudaSuccess) {
            set_cuda_error(e, "pinned error words");
            return e == cudaErrorMemoryAllocation ? IHT_ENOMEM : IHT_ECUDA;
        }
    }
    if (ws->out_want && !ws->out_host) {
        const cudaError_t e = cudaMallocHost(&ws->out_host, (size_t)kMaxK * (sizeof(int32_t) + sizeof(double)));
        if (e != cudaSuccess) {
            set_cuda_error(e, "pinned outputs");
            return e == cudaErrorMemoryAllocation ? IHT_ENOMEM : IHT_ECUDA;
        }
    }
    // (the first solve of a panel tunes its pass outside a graph)
    if (!grad_tc_shape_settled(ds)) return IHT_EAGAIN;
    TcParams *prm = nullptr;
    int rc = ensure_fused_exec(ds, k, K, impl, true, &prm);
    if (rc) return rc;
    *ws->sc_host = h;
    IHT_CUDA(cudaMemcpyAsync(ws->sc_init, ws->sc_host, sizeof(Scalars), cudaMemcpyHostToDevice, s));
    if ((rc = grad_tc_reset_status(ds))) return rc;
    IHT_CUDA(cudaGraphLaunch(ws->fused_exec, s));
    if (fault_take(IHT_FAULT_TIMEOUT))                 // (host-injected: a pass that gave up)
        IHT_CUDA(cudaMemsetAsync(&prm->err, 0x01, sizeof(int), s));
    IHT_CUDA(cudaMemcpyAsync(ws->sc_host, ws->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
    IHT_CUDA(cudaMemcpyAsync(&ws->flags_host[0], &ws->tail->bar_err, sizeof(int32_t),
                             cudaMemcpyDeviceToHost, s));
    IHT_CUDA(cudaMemcpyAsync(&ws->flags_host[1], &prm->err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (ws->out_want) {                                  // the host outputs, before the same synchronisation
        int32_t *hS = static_cast<int32_t *>(ws->out_host);
        IHT_CUDA(cudaMemcpyAsync(hS, ws->S, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, s));
        IHT_CUDA(cudaMemcpyAsync(reinterpret_cast<double *>(hS + kMaxK), ws->bS, sizeof(double) * k,
                                 cudaMemcpyDeviceToHost, s));
    }
    IHT_CUDA(cudaStreamSynchronize(s));
    ws->out_ready = ws->out_want;
    note_launch(ws->fused_setup_launches + ws->fused_launches * std::max(ws->sc_host->iter, 1));
    return (ws->flags_host[0] || ws->flags_host[1]) ? IHT_ETIMEOUT : IHT_OK;
}

}  // namespace iht
