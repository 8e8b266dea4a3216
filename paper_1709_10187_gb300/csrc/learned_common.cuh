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

// Fold of a brick cell into the fundamental domain of the cube's symmetry
// group: each coordinate l becomes c = min(l, b-1-l) (flip[a] records the
// reflection), then the axes are sorted so that c[perm[0]] <= c[perm[1]] <=
// c[perm[2]]; canonical axis k is world axis perm[k].
__device__ __forceinline__ void fold_cell(const int l[3], int b, int C[3], int perm[3], bool flip[3]) {
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        flip[a] = b - 1 - l[a] < l[a];
        c[a] = flip[a] ? b - 1 - l[a] : l[a];
    }
    int p0 = 0, p1 = 1, p2 = 2, t;
    if (c[p1] < c[p0]) { t = p0; p0 = p1; p1 = t; }
    if (c[p2] < c[p1]) { t = p1; p1 = p2; p2 = t; }
    if (c[p1] < c[p0]) { t = p0; p0 = p1; p1 = t; }
    perm[0] = p0; perm[1] = p1; perm[2] = p2;
    C[0] = c[p0]; C[1] = c[p1]; C[2] = c[p2];
}

// Network inputs for a brick of line-centre cell optical depth 10^lk (k0 dz)
// at a bin with log10 bin-mean profile lp and centre frequency x, at the cell
// with folded brick coordinates c[3]: region size in tau at line centre and at
// the bin, region a*tau, the frequency and eight Fourier features of it, and
// the cell's position, (2c + 1) / b - 1 per axis.
__device__ __forceinline__ void features(float lk, float lp, float x, const int c[3], int b, const FeatConst& C,
                                         __nv_bfloat16* out) {
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
    const float inv_b = 1.0f / (float)b;
#pragma unroll
    for (int a = 0; a < 3; ++a) f[13 + a] = (float)(2 * c[a] + 1) * inv_b - 1.0f;
#pragma unroll
    for (int i = 0; i < kFeat; ++i) out[i] = __float2bfloat16(f[i]);
}

// Summary of a region (a brick's inner cube) of a medium that varies from cell
// to cell, kRegionSum floats per brick, computed by the caller from the medium:
// [0] log10(k0 dz) at the region's geometric-mean density, [1] the standard
// deviation of log10 n over its cells, [2..4] the least-squares slope of
// log10 n per axis against the cell position (2l + 1)/r - 1, [5] the mean and
// [6] the rms of the comoving shift f_mu (v_c - v_nb).e_a / v_th over the
// region's interior faces (in Doppler widths; the same for both directions of
// a crossing), [7] unused.
constexpr int kRegionSum = 8;

// Network inputs for a packet in such a region, in the world frame (no
// symmetry fold: the region has none): region size in tau at line centre and
// at the bin, the start cell's log10 density relative to the region's mean,
// the frequency (x / x_max, |x| / x_max, one Fourier pair), the region's
// density spread and slopes, its mean and rms Doppler shift per crossing, and
// the cell's position (2 l + 1) / r - 1 per axis.
__device__ __forceinline__ void features_region(const float* __restrict__ sm, float lp, float x, float dlog,
                                                const int l[3], int r, const FeatConst& C, __nv_bfloat16* out) {
    float f[kFeat];
    f[0] = (sm[0] + C.log_b) * 0.1f;
    f[1] = (sm[0] + lp + C.log_b) * 0.2f;
    f[2] = dlog;
    const float xs = x * C.inv_xs;
    f[3] = xs;
    f[4] = fabsf(xs);
    float sn, cs;
    sincospif(xs, &sn, &cs);
    f[5] = sn;
    f[6] = cs;
    f[7] = sm[1] * 2.0f;
    f[8] = sm[2];
    f[9] = sm[3];
    f[10] = sm[4];
    f[11] = sm[5] * 4.0f;
    f[12] = sm[6] * 4.0f;
    const float inv_r = 1.0f / (float)r;
#pragma unroll
    for (int a = 0; a < 3; ++a) f[13 + a] = (float)(2 * l[a] + 1) * inv_r - 1.0f;
#pragma unroll
    for (int i = 0; i < kFeat; ++i) out[i] = __float2bfloat16(f[i]);
}

__device__ __forceinline__ int step_bucket(unsigned long long t) {
    int k = 63 - __clzll((long long)(t | 1ull));
    return k < kStepBuckets - 1 ? k : kStepBuckets - 1;
}

}  // namespace rddmc
