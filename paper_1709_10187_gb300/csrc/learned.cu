// learned.cu -- the learned exit proposal: first-passage data generation, the
// BF16 MLP (forward, backward, softmax cross-entropy, Adam) on tensor cores,
// and batched inference that samples exits for parked packets.
//
// First passages: sample i picks a density level, a start bin and a cell of a
// b^3 brick of uniform medium from its event stream, folds the cell into the
// fundamental domain of the cube's symmetry group and walks from it with the
// rows of an interior cell of that medium (the same rows and transition
// stream as the walk) until a spatial move leaves the brick.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "grid.h"
#include "learned_common.cuh"
#include "umma.cuh"

namespace rddmc {
namespace {

constexpr int kMaxLevels = 64;

struct FpParams {
    const uint4* rows[kMaxLevels];  // 3D rows (two uint4) of the interior class, J per level
    const uint2* fast[kMaxLevels];
    int jlo[kMaxLevels], jhi[kMaxLevels];
    int L, J, b;
    uint32_t k0, k1;
    unsigned long long p0, n, cap;
    int* out;                    // 8 ints per sample (rddmc_fp_generate)
    unsigned long long* steps;   // transitions per sample
    // optional training tensors: inputs (bf16, 16 per sample), targets
    __nv_bfloat16* X;
    int* tA;                     // exit face * J + exit bin, -1 when the step cap was reached
    int* tB;                     // log2 step bucket
    int* tC;                     // exit face * b^2 + exit position, -1 when the step cap was reached
    const float* lk;             // per level: log10(k0 dz)
    const float* lp;             // per bin: log10 of the bin-mean profile
    const float* xc;             // per bin: centre frequency
    FeatConst fc;
};

__device__ __forceinline__ uint4 fp_philox(uint4 c, uint32_t k0, uint32_t k1) { return philox4x32_10(c, k0, k1); }

__global__ void __launch_bounds__(256) fp_kernel(const FpParams P) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += stride) {
        const unsigned long long pk = P.p0 + i;
        const uint32_t pl = (uint32_t)pk, ph = (uint32_t)(pk >> 32);
        const uint4 ew = fp_philox(make_uint4(0u, 0u, pl, ph | 0x80000000u), P.k0, P.k1);  // event words 0..3
        const int l = min((int)(((unsigned long long)ew.x * (unsigned long long)P.L) >> 32), P.L - 1);
        const int nb = P.jhi[l] - P.jlo[l] + 1;
        int j = P.jlo[l] + (int)(((unsigned long long)ew.y * (unsigned long long)nb) >> 32);
        const int m = (int)(((unsigned long long)ew.z * (unsigned long long)(P.b * P.b * P.b)) >> 32);
        const int lw[3] = {m % P.b, (m / P.b) % P.b, m / (P.b * P.b)};
        int idx[3], perm[3];
        bool flip[3];
        fold_cell(lw, P.b, idx, perm, flip);
        const uint4* rows = P.rows[l];
        const uint2* fast = P.fast[l];
        const int j0 = j;
        const int start = idx[0] + P.b * (idx[1] + P.b * idx[2]);
        const int c0[3] = {idx[0], idx[1], idx[2]};
        int face = 6, pos = -1;
        unsigned long long t = 0;
        const unsigned J1 = (unsigned)P.J - 1u;
        while (t < P.cap && face == 6) {
            const unsigned long long blk = t >> 2;
            const uint4 r = fp_philox(make_uint4((uint32_t)blk, (uint32_t)(blk >> 32), pl, ph), P.k0, P.k1);
            for (unsigned q = (unsigned)(t & 3u); q < 4u && t < P.cap; ++q) {
                const unsigned w = q == 0 ? r.x : (q == 1 ? r.y : (q == 2 ? r.z : r.w));
                ++t;
                const unsigned jj = min((unsigned)j, J1);
                const uint2 f = __ldg(&fast[jj]);
                if (w < f.y) { j += (w >= f.x) ? 1 : -1; continue; }
                const uint4 a = __ldg(&rows[2 * jj]), c = __ldg(&rows[2 * jj + 1]);
                const unsigned o = (unsigned)(w >= a.x) + (unsigned)(w >= a.y) + (unsigned)(w >= a.z) +
                                   (unsigned)(w >= c.x) + (unsigned)(w >= c.y) + (unsigned)(w >= c.z) +
                                   (unsigned)(w >= c.w);
                if (o < 2u) { j += o ? 1 : -1; continue; }
                const int fc = (int)o - 2, ax = fc >> 1, side = (fc & 1) ? 1 : -1;
                if (idx[ax] + side < 0 || idx[ax] + side >= P.b) {
                    face = fc;
                    const int u = ax == 0 ? 1 : 0, v = ax == 2 ? 1 : 2;  // the other two axes, lower first
                    pos = idx[u] + P.b * idx[v];
                    break;
                }
                idx[ax] += side;
            }
        }
        int* o8 = P.out + 8 * i;
        o8[0] = l;
        o8[1] = j0;
        o8[2] = start;
        o8[3] = face;
        o8[4] = j;
        o8[5] = pos;
        o8[6] = 0;
        o8[7] = 0;
        P.steps[i] = t;
        if (P.X) {
            features(P.lk[l], P.lp[j0], P.xc[j0], c0, P.b, P.fc, P.X + kFeat * i);
            P.tA[i] = face < 6 ? face * P.J + min(max(j, 0), P.J - 1) : -1;
            P.tB[i] = step_bucket(t);
            if (P.tC) P.tC[i] = face < 6 ? face * P.b * P.b + pos : -1;
        }
    }
}

}  // namespace
}  // namespace rddmc

using namespace rddmc;

extern "C" {

int rddmc_cell_tau(const rddmc_grid* g, const void* d_table, int64_t cell, float* tau, void* stream) {
    if (!g || !d_table || !tau || cell < 0 || cell >= g->ncell) return RDDMC_ERR_ARG;
    if (!g->precomputed) return RDDMC_ERR_TABLE;
    const uint32_t cls = g->cell_class[cell];
    if (cls == UINT32_MAX) return RDDMC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const char* src = (const char*)d_table + g->off_tau + (uint64_t)cls * g->J * 4;
    if (cudaMemcpyAsync(tau, src, (size_t)g->J * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) return RDDMC_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? RDDMC_OK : RDDMC_ERR_CUDA;
}

int rddmc_fp_generate(const rddmc_grid* const* grids, const void* const* d_tables, int L, int b, const int32_t* jlo,
                      const int32_t* jhi, uint64_t seed, uint64_t p0, uint64_t n, uint64_t cap, int32_t* d_out,
                      uint64_t* d_steps, const rddmc_fp_train* train, void* stream) {
    if (!grids || !d_tables || !jlo || !jhi || !d_out || !d_steps) return RDDMC_ERR_ARG;
    if (L < 1 || L > kMaxLevels || b < 1 || b > 64 || n == 0 || cap == 0) return RDDMC_ERR_ARG;
    FpParams P;
    std::memset(&P, 0, sizeof(P));
    int J = -1;
    for (int l = 0; l < L; ++l) {
        const rddmc_grid* g = grids[l];
        if (!g || !d_tables[l]) return RDDMC_ERR_ARG;
        if (!g->precomputed) return RDDMC_ERR_TABLE;
        if (g->ndim != 3 || g->params.mode != RDDMC_MODE_DDMC || g->dusty() || g->weighted())
            return RDDMC_ERR_UNSUPPORTED;
        if (J < 0) J = g->J;
        if (g->J != J) return RDDMC_ERR_ARG;
        int idx[3] = {g->n[0] / 2, g->n[1] / 2, g->n[2] / 2};
        for (int a = 0; a < 3; ++a)
            for (int sd = -1; sd <= 1; sd += 2) {
                int nidx[3] = {idx[0], idx[1], idx[2]};
                nidx[a] += sd;
                if (!g->in_medium(nidx)) return RDDMC_ERR_ARG;  // the centre cell must be interior
            }
        const uint32_t cls = g->cell_class[g->cell_of(idx)];
        const char* tb = (const char*)d_tables[l];
        P.rows[l] = (const uint4*)(tb + g->off_rows) + (uint64_t)cls * J * 2;
        P.fast[l] = (const uint2*)(tb + g->off_fast) + (uint64_t)cls * J;
        if (jlo[l] < 0 || jhi[l] >= J || jlo[l] > jhi[l]) return RDDMC_ERR_ARG;
        P.jlo[l] = jlo[l];
        P.jhi[l] = jhi[l];
    }
    P.L = L; P.J = J; P.b = b;
    P.k0 = (uint32_t)seed; P.k1 = (uint32_t)(seed >> 32);
    P.p0 = p0; P.n = n; P.cap = cap;
    P.out = d_out;
    P.steps = (unsigned long long*)d_steps;
    if (train) {
        if (!train->d_x || !train->d_ta || !train->d_tb || !train->d_lk || !train->d_lp || !train->d_xc)
            return RDDMC_ERR_ARG;
        P.X = (__nv_bfloat16*)train->d_x;
        P.tA = train->d_ta;
        P.tB = train->d_tb;
        P.tC = train->d_tc;
        P.lk = train->d_lk;
        P.lp = train->d_lp;
        P.xc = train->d_xc;
        P.fc.log_b = log10f((float)b);
        P.fc.log_a = (float)log10(grids[0]->a);
        P.fc.inv_xs = (float)(1.0 / std::max(std::fabs(grids[0]->edges.front()), std::fabs(grids[0]->edges.back())));
    }
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return RDDMC_ERR_CUDA;
    const unsigned long long want = (n + 255) / 256;
    const unsigned blocks = (unsigned)(want < (unsigned long long)nsm * 8 ? want : (unsigned long long)nsm * 8);
    fp_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(P);
    return cudaGetLastError() == cudaSuccess ? RDDMC_OK : RDDMC_ERR_CUDA;
}

}  // extern "C"

// ===================================================================== MLP
// Architecture: n_in = 16 inputs -> 3 hidden layers of 128 (ReLU) -> n_out
// logits (a multiple of 16): head A over [0, nA) (exit face x exit bin),
// head B over [nA, nA + nB) (log2 step bucket) and head C over
// [nA + nB, nA + nB + 6 S) (exit cell on each face, S = b^2 per face, used
// one slice at a time); columns past the heads are padding.  Parameters, FP32 master copy and BF16 copy in the same order:
// W1[128x16] b1[128] W2[128x128] b2[128] W3[128x128] b3[128] W4[n_out x 128]
// b4[n_out].  Every matrix product runs on the tcgen05 tensor cores
// (umma.cuh: BF16 operands, FP32 accumulators in tensor memory), the backward
// ones on transposed copies so that both operands are K-major; softmax,
// cross-entropy, bias sums and Adam in FP32.
namespace rddmc {
namespace {

constexpr int kIn = 16, kHid = 128;

struct MlpOffsets {
    uint64_t W[4], b[4], total;
};

MlpOffsets mlp_offsets(int n_out) {
    MlpOffsets o;
    const int fan_in[4] = {kIn, kHid, kHid, kHid}, fan_out[4] = {kHid, kHid, kHid, n_out};
    uint64_t off = 0;
    for (int l = 0; l < 4; ++l) {
        o.W[l] = off; off += (uint64_t)fan_in[l] * fan_out[l];
        o.b[l] = off; off += (uint64_t)fan_out[l];
    }
    o.total = off;
    return o;
}

// Softmax cross-entropy of the heads, one warp per row: loss += CE_A + CE_B
// (+ CE_C over the S logits of the target's slice when head C is present and
// its target is >= 0), summed over the batch; dlogits = (softmax - onehot) / B
// on the logits a head used, zero elsewhere.
__global__ void softmax_ce_kernel(const float* __restrict__ logits, int n_out, int nA, int nB, int nC, int S,
                                  const int* __restrict__ tA, const int* __restrict__ tB, const int* __restrict__ tC,
                                  int Bsz, float* __restrict__ dlogf, __nv_bfloat16* __restrict__ dlogb,
                                  float* loss) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= Bsz) return;
    const float* z = logits + (size_t)row * n_out;
    float* gf = dlogf + (size_t)row * n_out;
    __nv_bfloat16* gb = dlogb + (size_t)row * n_out;
    float total = 0.0f;
    const bool skip = tA[row] < 0;  // ignored sample: no loss, no gradient
    // zero everything past heads A and B (head C's unused slices, padding)
    for (int k = (skip ? 0 : nA + nB) + lane; k < n_out; k += 32) {
        gf[k] = 0.0f;
        gb[k] = __float2bfloat16(0.0f);
    }
    if (skip) return;
    __syncwarp();
    int tc = (nC > 0 && tC) ? tC[row] : -1;
    if (tc >= nC) tc = -1;
    const int nh = tc >= 0 ? 3 : 2;
    for (int h = 0; h < nh; ++h) {
        int lo, hi, tgt;
        if (h == 0) { lo = 0; hi = nA; tgt = tA[row]; }
        else if (h == 1) { lo = nA; hi = nA + nB; tgt = nA + tB[row]; }
        else { lo = nA + nB + (tc / S) * S; hi = lo + S; tgt = nA + nB + tc; }
        float mx = -3.0e38f;
        for (int k = lo + lane; k < hi; k += 32) mx = fmaxf(mx, z[k]);
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        float se = 0.0f;
        for (int k = lo + lane; k < hi; k += 32) se += __expf(z[k] - mx);
        for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
        const float lse = mx + __logf(se);
        total += lse - z[tgt];
        for (int k = lo + lane; k < hi; k += 32) {
            const float g = (__expf(z[k] - lse) - (k == tgt ? 1.0f : 0.0f)) / (float)Bsz;
            gf[k] = g;
            gb[k] = __float2bfloat16(g);
        }
    }
    if (lane == 0) atomicAdd(loss, total);
}

// db[n] += sum over the block's rows of dY[b, n]: blocks of 32 columns x 8 row
// lanes, each block a contiguous range of rows; db must start at zero.
__global__ void colsum_kernel(const float* __restrict__ dy, int Bsz, int N, int rows_per_block,
                              float* __restrict__ db) {
    __shared__ float part[8][33];
    const int n = blockIdx.x * 32 + threadIdx.x;
    const int r0 = blockIdx.y * rows_per_block, r1 = min(Bsz, r0 + rows_per_block);
    float acc = 0.0f;
    if (n < N)
        for (int r = r0 + (int)threadIdx.y; r < r1; r += 8) acc += dy[(size_t)r * N + n];
    part[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.y == 0 && n < N) {
        float t = 0.0f;
#pragma unroll
        for (int i = 0; i < 8; ++i) t += part[i][threadIdx.x];
        atomicAdd(&db[n], t);
    }
}

cudaError_t colsum(const float* dy, int Bsz, int N, float* db, cudaStream_t s) {
    const int rpb = 256;
    dim3 grid((N + 31) / 32, (Bsz + rpb - 1) / rpb);
    colsum_kernel<<<grid, dim3(32, 8), 0, s>>>(dy, Bsz, N, rpb, db);
    return cudaGetLastError();
}

// K splits for a weight-gradient product (K = batch rows) on 128 x min(N, 256)
// tensor-core tiles: about two waves of CTAs over the GPU, at most one split
// per 64-column panel of K.
int ksplit_for(int M, int N, int K) {
    const int nt = std::min(256, N);
    const int tiles = ((M + 127) / 128) * ((N + nt - 1) / nt);
    return std::max(1, std::min((K + 63) / 64, (304 + tiles - 1) / tiles));
}

__global__ void adam_kernel(uint64_t n, float* __restrict__ w, __nv_bfloat16* __restrict__ wb,
                            const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi, vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16(wi);
}

__global__ void to_bf16_kernel(uint64_t n, const float* __restrict__ w, __nv_bfloat16* __restrict__ wb) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wb[i] = __float2bfloat16(w[i]);
}

// Work buffer (bytes, rows B a multiple of 64): H1 H2 H3 bf16 [B x 128] each,
// dHf f32 [B x 128], dHb bf16 [B x 128] x2, logits f32 [B x n_out],
// dlogf f32 [B x n_out], dlogb bf16 [B x n_out].
struct MlpWork {
    __nv_bfloat16 *H[3], *dHb[2], *dlogb;
    float *dHf, *logits, *dlogf;
    __nv_bfloat16 *dZT, *HT, *WT;  // transposed copies for the K-major products of the backward pass
};

// The transposed copies serve every layer: dZT holds [n_out x B] and [128 x B],
// WT holds [128 x n_out] and [128 x 128], so both take max(n_out, 128) rows.
uint64_t mlp_work_bytes(int Bsz, int n_out) {
    const uint64_t bh = (uint64_t)Bsz * kHid;
    const uint64_t wide = (uint64_t)std::max(n_out, kHid);
    return align256(bh * 2) * 5 + align256(bh * 4) + align256((uint64_t)Bsz * n_out * 4) * 2 +
           align256((uint64_t)Bsz * n_out * 2) + align256((uint64_t)Bsz * wide * 2) + align256(bh * 2) +
           align256(wide * kHid * 2);
}

MlpWork mlp_work(void* d_work, int Bsz, int n_out) {
    char* p = (char*)d_work;
    const uint64_t bh = (uint64_t)Bsz * kHid;
    MlpWork w;
    for (int i = 0; i < 3; ++i) { w.H[i] = (__nv_bfloat16*)p; p += align256(bh * 2); }
    for (int i = 0; i < 2; ++i) { w.dHb[i] = (__nv_bfloat16*)p; p += align256(bh * 2); }
    w.dHf = (float*)p; p += align256(bh * 4);
    w.logits = (float*)p; p += align256((uint64_t)Bsz * n_out * 4);
    w.dlogf = (float*)p; p += align256((uint64_t)Bsz * n_out * 4);
    w.dlogb = (__nv_bfloat16*)p; p += align256((uint64_t)Bsz * n_out * 2);
    w.dZT = (__nv_bfloat16*)p; p += align256((uint64_t)Bsz * std::max(n_out, kHid) * 2);  // [n_out or 128 x B]
    w.HT = (__nv_bfloat16*)p; p += align256(bh * 2);                          // [128 x B] or [16 x B]
    w.WT = (__nv_bfloat16*)p;                                                 // [128 x n_out or 128]
    return w;
}

// Device status of the tensor-core products (set when a bounded wait runs out).
__device__ unsigned g_tc_err = 0;

// The status word's device address, looked up on every call (a cheap host
// call; a cached address would go stale when the device is reset and the
// module loaded again).
unsigned* tc_err_ptr() {
    void* a = nullptr;
    if (cudaGetSymbolAddress(&a, g_tc_err) != cudaSuccess) return nullptr;
    return (unsigned*)a;
}

// C = epi(A W^T (+ bias)) on tcgen05 (umma.cuh): A [M x K], W [N x K], both K
// contiguous; ksplit > 1 only with F32_ADD.  K <= 128 and not a multiple of 64
// is staged by the threads, everything else by TMA.
template <int EPI>
cudaError_t gemm_tc(int M, int N, int K, const __nv_bfloat16* A, int lda, const __nv_bfloat16* W, int ldw,
                    const float* bias, const __nv_bfloat16* mask, int ldmask, __nv_bfloat16* outb, float* outf,
                    int ldc, cudaStream_t s, int ksplit = 1) {
    unsigned* err = tc_err_ptr();
    if (!err || K % 16 || N % 16 || ksplit < 1 || (ksplit > 1 && EPI != umma::F32_ADD)) return cudaErrorInvalidValue;
    const int NT = std::min(256, N);
    // two staging areas when a split has more than one K block of 128 (the copy
    // of the next block overlaps the products of this one)
    const int kpanels = (K + umma::kPanel - 1) / umma::kPanel;
    const int per_split = (kpanels + ksplit - 1) / ksplit;
    const bool staged_k = K <= 128 && K % umma::kPanel != 0;
    const int nstage = (!staged_k && per_split > umma::kMaxPanels) ? 2 : 1;
    // at least 80 KiB of shared memory: at most two CTAs per SM, so their TMEM
    // accumulators (<= 256 columns each) always fit the SM's 512 columns
    const size_t smem = std::max<size_t>(umma::smem_bytes(NT, nstage), 80 * 1024);
    dim3 grid((N + NT - 1) / NT, (M + umma::kTileM - 1) / umma::kTileM, ksplit);
    CUtensorMap mapA, mapW;
    std::memset(&mapA, 0, sizeof(mapA));
    std::memset(&mapW, 0, sizeof(mapW));
    const bool staged = K <= 128 && K % umma::kPanel != 0;
    if (staged && ksplit != 1) return cudaErrorInvalidValue;
    if (!staged && !(umma::make_map(&mapA, A, M, K, lda, umma::kTileM) && umma::make_map(&mapW, W, N, K, ldw, NT)))
        return cudaErrorInvalidValue;
    auto kern = staged ? umma::gemm_tc_kernel<EPI, false> : umma::gemm_tc_kernel<EPI, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, umma::kThreads, smem, s>>>(M, N, K, NT, A, lda, W, ldw, mapA, mapW, bias, mask, ldmask, outb, outf,
                                            ldc, nstage, err);
    return cudaGetLastError();
}

cudaError_t transpose(const __nv_bfloat16* in, int rows, int cols, int ld_in, __nv_bfloat16* out, int ld_out,
                      cudaStream_t s) {
    dim3 grid((cols + 31) / 32, (rows + 31) / 32);
    umma::transpose_bf16_kernel<<<grid, dim3(32, 8), 0, s>>>(in, rows, cols, ld_in, out, ld_out);
    return cudaGetLastError();
}

cudaError_t mlp_forward(int n_out, const float* wf, const __nv_bfloat16* wb, const __nv_bfloat16* X, int Bsz,
                        const MlpWork& w, cudaStream_t s) {
    const MlpOffsets o = mlp_offsets(n_out);
    cudaError_t e;
    if ((e = gemm_tc<umma::RELU_BF16>(Bsz, kHid, kIn, X, kIn, wb + o.W[0], kIn, wf + o.b[0], nullptr, 0, w.H[0],
                                      nullptr, kHid, s)) != cudaSuccess)
        return e;
    for (int l = 1; l < 3; ++l)
        if ((e = gemm_tc<umma::RELU_BF16>(Bsz, kHid, kHid, w.H[l - 1], kHid, wb + o.W[l], kHid, wf + o.b[l],
                                          nullptr, 0, w.H[l], nullptr, kHid, s)) != cudaSuccess)
            return e;
    return gemm_tc<umma::LINEAR_F32>(Bsz, n_out, kHid, w.H[2], kHid, wb + o.W[3], kHid, wf + o.b[3], nullptr, 0,
                                     nullptr, w.logits, n_out, s);
}

}  // namespace
}  // namespace rddmc

extern "C" {

uint64_t rddmc_mlp_param_count(int n_out) { return (n_out > 0 && n_out % 16 == 0) ? mlp_offsets(n_out).total : 0; }

uint64_t rddmc_mlp_work_bytes(int batch, int n_out) {
    return (batch > 0 && batch % 64 == 0 && n_out > 0 && n_out % 16 == 0) ? mlp_work_bytes(batch, n_out) : 0;
}

int rddmc_mlp_to_bf16(int n_out, const float* d_wf, void* d_wb, void* stream) {
    const uint64_t n = rddmc_mlp_param_count(n_out);
    if (!n || !d_wf || !d_wb) return RDDMC_ERR_ARG;
    to_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, d_wf, (__nv_bfloat16*)d_wb);
    return cudaGetLastError() == cudaSuccess ? RDDMC_OK : RDDMC_ERR_CUDA;
}

int rddmc_mlp_forward(int n_out, const float* d_wf, const void* d_wb, const void* d_x, int batch, void* d_work,
                      float* d_logits, void* stream) {
    if (!rddmc_mlp_param_count(n_out) || !rddmc_mlp_work_bytes(batch, n_out) || !d_wf || !d_wb || !d_x || !d_work)
        return RDDMC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const MlpWork w = mlp_work(d_work, batch, n_out);
    if (mlp_forward(n_out, d_wf, (const __nv_bfloat16*)d_wb, (const __nv_bfloat16*)d_x, batch, w, s) != cudaSuccess)
        return RDDMC_ERR_CUDA;
    if (d_logits && cudaMemcpyAsync(d_logits, w.logits, (size_t)batch * n_out * 4, cudaMemcpyDeviceToDevice, s) !=
                        cudaSuccess)
        return RDDMC_ERR_CUDA;
    return RDDMC_OK;
}

int rddmc_mlp_loss_grad(int n_out, int nA, int nB, int nC, int S, const float* d_wf, const void* d_wb,
                        const void* d_x, const int32_t* d_ta, const int32_t* d_tb, const int32_t* d_tc, int batch,
                        void* d_work, float* d_grad, float* d_loss, void* stream) {
    if (!rddmc_mlp_param_count(n_out) || !rddmc_mlp_work_bytes(batch, n_out) || nA < 1 || nB < 1 || nC < 0 ||
        nA + nB + nC > n_out || !d_wf || !d_wb || !d_x || !d_ta || !d_tb || !d_work || !d_grad || !d_loss)
        return RDDMC_ERR_ARG;
    if (nC > 0 && (S < 1 || nC != 6 * S || !d_tc)) return RDDMC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const MlpOffsets o = mlp_offsets(n_out);
    const __nv_bfloat16* wb = (const __nv_bfloat16*)d_wb;
    const __nv_bfloat16* X = (const __nv_bfloat16*)d_x;
    const MlpWork w = mlp_work(d_work, batch, n_out);
    if (mlp_forward(n_out, d_wf, wb, X, batch, w, s) != cudaSuccess) return RDDMC_ERR_CUDA;
    if (cudaMemsetAsync(d_loss, 0, 4, s) != cudaSuccess) return RDDMC_ERR_CUDA;
    softmax_ce_kernel<<<(batch + 7) / 8, 256, 0, s>>>(w.logits, n_out, nA, nB, nC, S, d_ta, d_tb,
                                                       nC > 0 ? d_tc : nullptr, batch, w.dlogf, w.dlogb, d_loss);
    // gradients accumulate (split-K products, column sums) into a zeroed buffer
    if (cudaMemsetAsync(d_grad, 0, o.total * sizeof(float), s) != cudaSuccess) return RDDMC_ERR_CUDA;
    // Every product runs on tcgen05 with K contiguous in both operands:
    //   dW = dZ^T H     as (dZ^T [out x B]) (H^T [in x B])^T, K = batch, split over K
    //   dH = (dZ W) .* [H > 0]  as (dZ [B x out]) (W^T [in x out])^T, K = out
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    // output layer
    chk(transpose(w.dlogb, batch, n_out, n_out, w.dZT, batch, s));
    chk(transpose(w.H[2], batch, kHid, kHid, w.HT, batch, s));
    chk(gemm_tc<umma::F32_ADD>(n_out, kHid, batch, w.dZT, batch, w.HT, batch, nullptr, nullptr, 0, nullptr,
                               d_grad + o.W[3], kHid, s, ksplit_for(n_out, kHid, batch)));
    chk(colsum(w.dlogf, batch, n_out, d_grad + o.b[3], s));
    chk(transpose(wb + o.W[3], n_out, kHid, kHid, w.WT, n_out, s));
    chk(gemm_tc<umma::MASK_BF16>(batch, kHid, n_out, w.dlogb, n_out, w.WT, n_out, nullptr, w.H[2], kHid, w.dHb[0],
                                 w.dHf, kHid, s));
    int cur = 0;
    for (int l = 2; l >= 1; --l) {
        // layer l (W[l]: H[l-1] -> H[l]); dHb[cur] holds dL/d(pre-activation of H[l])
        chk(transpose(w.dHb[cur], batch, kHid, kHid, w.dZT, batch, s));
        chk(transpose(w.H[l - 1], batch, kHid, kHid, w.HT, batch, s));
        chk(gemm_tc<umma::F32_ADD>(kHid, kHid, batch, w.dZT, batch, w.HT, batch, nullptr, nullptr, 0, nullptr,
                                   d_grad + o.W[l], kHid, s, ksplit_for(kHid, kHid, batch)));
        chk(colsum(w.dHf, batch, kHid, d_grad + o.b[l], s));
        chk(transpose(wb + o.W[l], kHid, kHid, kHid, w.WT, kHid, s));
        chk(gemm_tc<umma::MASK_BF16>(batch, kHid, kHid, w.dHb[cur], kHid, w.WT, kHid, nullptr, w.H[l - 1], kHid,
                                     w.dHb[cur ^ 1], w.dHf, kHid, s));
        cur ^= 1;
    }
    // input layer: dW1 = dZ1^T X
    chk(transpose(w.dHb[cur], batch, kHid, kHid, w.dZT, batch, s));
    chk(transpose(X, batch, kIn, kIn, w.HT, batch, s));
    chk(gemm_tc<umma::F32_ADD>(kHid, kIn, batch, w.dZT, batch, w.HT, batch, nullptr, nullptr, 0, nullptr,
                               d_grad + o.W[0], kIn, s, ksplit_for(kHid, kIn, batch)));
    chk(colsum(w.dHf, batch, kHid, d_grad + o.b[0], s));
    if (e != cudaSuccess) return RDDMC_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? RDDMC_OK : RDDMC_ERR_CUDA;
}

int rddmc_mlp_status(void* stream) {
    unsigned* p = tc_err_ptr();
    if (!p) return RDDMC_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned v = 0;
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaMemcpy(&v, p, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return RDDMC_ERR_CUDA;
    if (v && cudaMemset(p, 0, 4) != cudaSuccess) return RDDMC_ERR_CUDA;
    return v ? RDDMC_ERR_TIMEOUT : RDDMC_OK;
}

int rddmc_mlp_adam(int n_out, float* d_wf, void* d_wb, const float* d_grad, float* d_m, float* d_v, int step, float lr,
                   float beta1, float beta2, float eps, void* stream) {
    const uint64_t n = rddmc_mlp_param_count(n_out);
    if (!n || !d_wf || !d_wb || !d_grad || !d_m || !d_v || step < 1) return RDDMC_ERR_ARG;
    const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
    adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        n, d_wf, (__nv_bfloat16*)d_wb, d_grad, d_m, d_v, lr, beta1, beta2, eps, c1, c2);
    return cudaGetLastError() == cudaSuccess ? RDDMC_OK : RDDMC_ERR_CUDA;
}

}  // extern "C"
