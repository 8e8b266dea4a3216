// learned_common.cuh -- input featurisation and step buckets of the learned
// exit proposal, shared by first-passage data generation (training) and the
// walk's proposal step (inference).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace rddmc {

constexpr int kFeat = 16;
constexpr int kStepBuckets = 32;

// Constants of the input featurisation shared by training and inference.
struct FeatConst {
    float log_b;     // log10(brick cells per edge)
    float log_a;     // log10(damping parameter a)
    float inv_xs;    // 1 / max |x| of the frequency grid
};

// Network inputs for a brick of line-centre cell optical depth 10^lk (k0 dz)
// entered at a bin with log10 bin-mean profile lp and centre frequency x:
// region size in tau at line centre and at the entry bin, region a*tau, the
// entry frequency and eight Fourier features of it.
__device__ __forceinline__ void features(float lk, float lp, float x, const FeatConst& C, __nv_bfloat16* out) {
    float f[kFeat];
    f[0] = (lk + C.log_b) * 0.1f;
    f[1] = (lk + lp + C.log_b) * 0.2f;
    f[2] = (lk + C.log_b + C.log_a) * 0.1f;
    const float xs = x * C.inv_xs;
    f[3] = xs;
    f[4] = fabsf(xs);
#pragma unroll
    for (int k = 1; k <= 4; ++k) {
        float sn, cs;
        sincospif((float)k * xs, &sn, &cs);
        f[3 + 2 * k] = sn;
        f[4 + 2 * k] = cs;
    }
    f[13] = f[14] = f[15] = 0.0f;
#pragma unroll
    for (int i = 0; i < kFeat; ++i) out[i] = __float2bfloat16(f[i]);
}

__device__ __forceinline__ int step_bucket(unsigned long long t) {
    int k = 63 - __clzll((long long)(t | 1ull));
    return k < kStepBuckets - 1 ? k : kStepBuckets - 1;
}

}  // namespace rddmc
