// The centred residual as FP8 E4M3 limbs for the single-column tensor-core
// pass (the B operand of its MMAs), shared by the pass's limb kernel and the
// fused per-iteration kernel of tail.cu so both write the same bytes.
//
// r ~ sum_l s_l q_l with s_l = s_0 2^(-4l), l = 0..4, q_l in E4M3; s_0 is the
// power of two with max|r| / 448 <= s_0 (448 = the largest E4M3 value).  The
// B image holds, per K-step of 32 samples, 256 bytes in the permuted K order of
// the dosage map: [256 unused bytes][K-step 0]...[K-step S-1][256 zero bytes].
#pragma once
#include <cuda_fp8.h>

#include "common.cuh"

namespace iht {

constexpr int kTcLimbs = 5;

struct TcParams {
    float s0;        // scale of limb 0 (limb l: s0 * 2^-4l)
    float R;         // sum of the residual over the samples
    int err;         // 1: a bounded wait of the pass timed out
    int pad;
};

__device__ __forceinline__ int b_offset(int64_t i, int limb)
{
    const int64_t s = i >> 5;                       // K-step
    const int ii = (int)(i & 31);
    const int wi = ii >> 4, q = ii & 15;            // 16-sample word, position in it
    const int k = q >> 2, j = q & 3;                // output byte k of decoded word j
    const int c = 4 * wi + j;                       // TMEM column within the step
    const int kpos = 4 * c + k;                     // K index within the step
    return 256 + (int)(s * 256) + (kpos >> 4) * 128 + limb * 16 + (kpos & 15);
}

// s_0 from m = max |r|.
__device__ __forceinline__ float limb_scale(float m)
{
    float s0 = 1.0f;
    if (m > 0.0f) {
        int e;
        frexpf(m / 448.0f, &e);          // m/448 <= 2^e
        s0 = ldexpf(1.0f, e);
    }
    return s0;
}

// The five limbs of sample i's residual into the B image.
__device__ __forceinline__ void limb_encode(float res, float s0, uint8_t *bimg, int64_t i)
{
    float s = s0;
#pragma unroll
    for (int l = 0; l < kTcLimbs; ++l) {
        const __nv_fp8_e4m3 q(res / s);
        const float qf = (float)q;
        bimg[b_offset(i, l)] = q.__x;
        res -= s * qf;
        s *= 0.0625f;
    }
}

}  // namespace iht
