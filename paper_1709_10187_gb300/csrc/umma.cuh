// umma.cuh -- dense BF16 products on the 5th-generation tensor cores
// (tcgen05.mma, FP32 accumulators in tensor memory) for the learned proposal's
// network: C[M x N] = A[M x K] W[N x K]^T (+ bias, epilogue), both operands
// row-major with K contiguous ("K-major"), K a multiple of 16.
//
// One CTA of 128 threads computes a 128 x NT tile (NT <= 256, a multiple of
// 16), over K in blocks of 128 (two 64-column panels), optionally a range of
// K per blockIdx.z (split-K).  A block of A and W is staged in shared memory
// in the 128-byte swizzled K-major layout (rows of 64 BF16 = 128 B, eight-row
// atoms of 1 KiB, 16-byte chunk c of row r stored at chunk c ^ (r mod 8)): by
// TMA (cp.async.bulk.tensor with 128-byte swizzle; rows and columns past the
// matrix filled with zeros by the copy engine), or by the threads for a single
// block with K not a multiple of 64.  One elected thread issues the block's
// tcgen05.mma instructions into a TMEM accumulator of 128 lanes x NT columns,
// commits them to an mbarrier and waits before reusing the shared memory;
// after the last block every warp reads its 32 lanes back with tcgen05.ld and
// turns each 32 x 32 block around in shared memory, so that the epilogue's
// stores run along rows.  Waits are bounded: a wait that runs out sets the
// error word and the tile's outputs are left unwritten.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rddmc {
namespace umma {

constexpr int kTileM = 128;
constexpr int kThreads = 128;
constexpr int kPanel = 64;  // BF16 per 128-byte swizzled row
constexpr int kMaxPanels = 2;  // a K block is at most 128 wide

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading byte offset (unused
// by swizzled K-major layouts, set to 16 B), stride byte offset between
// eight-row atoms (1 KiB), descriptor version 1, 128-byte swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)(16u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)2u << 61;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t instr_desc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__host__ __device__ constexpr int tmem_cols(int nt) {
    return nt <= 32 ? 32 : (nt <= 64 ? 64 : (nt <= 128 ? 128 : 256));
}

// Copy rows [row0, row0 + rows) x K of a row-major BF16 matrix into the
// swizzled K-major layout at dst (1 KiB aligned; rows a multiple of 8); rows
// past `valid` are zero.
__device__ __forceinline__ void stage(const __nv_bfloat16* __restrict__ src, int ld, int row0, int rows, int valid,
                                      int K, unsigned char* dst) {
    const int chunks_per_row = K / 8;  // 16-byte chunks of K
    const int total = rows * chunks_per_row;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const int r = i / chunks_per_row, q = i % chunks_per_row;
        const int p = q >> 3, c = q & 7;  // panel, chunk in the 128-byte row
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (r < valid) v = *reinterpret_cast<const uint4*>(src + (size_t)(row0 + r) * ld + q * 8);
        unsigned char* d = dst + (size_t)p * rows * 128 + (size_t)(r >> 3) * 1024 + (r & 7) * 128 +
                           ((c ^ (r & 7)) << 4);
        *reinterpret_cast<uint4*>(d) = v;
    }
}

enum Epi { RELU_BF16 = 0, LINEAR_F32 = 1, MASK_BF16 = 2, F32_ADD = 3 };

// Bounded wait for the given phase parity of an mbarrier; false when it ran out.
__device__ __forceinline__ bool wait_parity(uint64_t* mbar, uint32_t parity) {
    uint32_t done = 0;
    for (int it = 0; it < (1 << 22) && !done; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(smem_u32(mbar)), "r"(parity));
    }
    return done != 0;
}

// TMA copy of the box at element coordinates (x, y) of a 2D tensor map into
// shared memory, counted on the mbarrier's transaction bytes.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        :: "r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(mbar))
        : "memory");
}

// Issue the tcgen05.mma instructions of one staged block: `slices` K-slices of
// 16 (four per 64-column panel), the first of them overwriting the accumulator
// when `first`.
__device__ __forceinline__ void mma_block(uint32_t tmem, unsigned char* sA, unsigned char* sB, int NT, int slices,
                                          bool first) {
    const uint32_t idesc = instr_desc(kTileM, NT);
    for (int s = 0; s < slices; ++s) {
        const int p = s >> 2, off = (s & 3) * 32;  // panel, byte offset of the 16-wide K slice
        const uint64_t ad = smem_desc(smem_u32(sA + (size_t)p * kTileM * 128 + off));
        const uint64_t bd = smem_desc(smem_u32(sB + (size_t)p * NT * 128 + off));
        const uint32_t acc = (first && s == 0) ? 0u : 1u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
            :: "r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
}

// C = epi(A W^T (+ bias)) for A [M x K], W [N x K], both K contiguous.
// Grid: (ceil(N / NT), ceil(M / 128), ksplit); blockIdx.z takes a range of K
// in blocks of 128 (64-column panels).  TMA path: tensor maps mapA (box 64 x
// 128) and mapW (box 64 x NT), any K (columns past K are zero-filled);
// thread-staged path: K <= 128.  Epilogues: RELU_BF16 and LINEAR_F32 add the
// bias; MASK_BF16 keeps entries where mask > 0 and writes them to outb (BF16)
// and outf (FP32); F32_ADD adds into outf (split-K partial sums).  err: set
// to 1 when a wait ran out (the tile's outputs are then left unwritten).
template <int EPI, bool TMA>
__global__ void __launch_bounds__(kThreads) gemm_tc_kernel(int M, int N, int K, int NT,
                                                           const __nv_bfloat16* __restrict__ A, int lda,
                                                           const __nv_bfloat16* __restrict__ W, int ldw,
                                                           const __grid_constant__ CUtensorMap mapA,
                                                           const __grid_constant__ CUtensorMap mapW,
                                                           const float* __restrict__ bias,
                                                           const __nv_bfloat16* __restrict__ mask, int ldmask,
                                                           __nv_bfloat16* __restrict__ outb, float* __restrict__ outf,
                                                           int ldc, int nstage, unsigned* err) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    // nstage (1 or 2) staging areas of one K block each: A panels, then W panels
    const size_t stage_bytes = (size_t)kMaxPanels * (kTileM + NT) * 128;
    unsigned char* sA = base;  // stage 0's A panels (also the epilogue's scratch)
    auto stage_a = [&](int st) { return base + (size_t)st * stage_bytes; };
    auto stage_b = [&](int st) { return base + (size_t)st * stage_bytes + (size_t)kMaxPanels * kTileM * 128; };
    // per stage: tbar (its TMA copy landed) and mbar (its products completed)
    uint64_t* tbar = reinterpret_cast<uint64_t*>(base + (size_t)nstage * stage_bytes);
    uint64_t* mbar = tbar + 2;
    uint32_t* taddr_s = reinterpret_cast<uint32_t*>(tbar + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kTileM, n0 = blockIdx.x * NT;
    const int ncols = tmem_cols(NT);
    // this split's range of K, in whole 64-column panels
    const int kpanels = (K + kPanel - 1) / kPanel;
    const int per = (kpanels + (int)gridDim.z - 1) / (int)gridDim.z;
    const int p_begin = (int)blockIdx.z * per, p_end = min(kpanels, p_begin + per);
    if (p_begin >= p_end) return;  // an empty split adds nothing

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(taddr_s)), "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < 4; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(tbar + i)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (!TMA) {  // one block: K <= 128
        stage(A, lda, m0, kTileM, min(kTileM, M - m0), K, stage_a(0));
        stage(W, ldw, n0, NT, min(NT, N - n0), K, stage_b(0));
        asm volatile("fence.proxy.async.shared::cta;");  // generic-proxy stores -> tensor-core reads
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *taddr_s;

    // One thread stages (TMA), issues and waits.  With two stages the copy of
    // K block b+1 is issued as soon as its stage is free (the products of block
    // b-1 completed), so it lands while block b's products run; with one stage
    // each block is copied, multiplied and waited for in turn.  Use k of a
    // stage completes phase k of its two mbarriers (parity k & 1); a stage is
    // rewritten only after its previous use was waited for, so no barrier runs
    // two phases ahead of its wait.
    __shared__ int ok_s;
    if (threadIdx.x == 0) {
        bool ok = true;
        if (TMA) {
            const int nb = (p_end - p_begin + kMaxPanels - 1) / kMaxPanels;
            auto issue = [&](int blk) {
                const int st = nstage == 2 ? (blk & 1) : 0;
                const int p = p_begin + blk * kMaxPanels;
                const int np = min(kMaxPanels, p_end - p);
                const uint32_t bytes = (uint32_t)(np * (kTileM + NT) * 128);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                             :: "r"(smem_u32(tbar + st)), "r"(bytes) : "memory");
                for (int q = 0; q < np; ++q) {
                    tma_load_2d(stage_a(st) + (size_t)q * kTileM * 128, &mapA, (p + q) * kPanel, m0, tbar + st);
                    tma_load_2d(stage_b(st) + (size_t)q * NT * 128, &mapW, (p + q) * kPanel, n0, tbar + st);
                }
            };
            int pend = 0;  // copies issued and not yet waited for
            issue(0);
            pend = 1;
            int b = 0;
            for (; b < nb; ++b) {
                const int st = nstage == 2 ? (b & 1) : 0;
                const uint32_t use = nstage == 2 ? (uint32_t)(b >> 1) : (uint32_t)b;
                if (nstage == 2 && b + 1 < nb) {
                    // stage of block b+1 last held block b-1: wait for its products
                    if (b >= 1 && !(ok = wait_parity(mbar + ((b + 1) & 1), (uint32_t)((b - 1) >> 1) & 1u))) break;
                    issue(b + 1);
                    ++pend;
                }
                if (!(ok = wait_parity(tbar + st, use & 1u))) break;
                --pend;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const int np = min(kMaxPanels, p_end - (p_begin + b * kMaxPanels));
                mma_block(tmem, stage_a(st), stage_b(st), NT, 4 * np, b == 0);  // columns past K were zero-filled
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             :: "r"(smem_u32(mbar + st)));
                if (nstage == 1) {
                    if (!(ok = wait_parity(mbar, use & 1u))) break;
                    if (b + 1 < nb) {
                        issue(b + 1);
                        ++pend;
                    }
                }
            }
            if (ok && nstage == 2) {
                // the last commit covers every product issued before it
                const int bl = nb - 1;
                ok = wait_parity(mbar + (bl & 1), (uint32_t)(bl >> 1) & 1u);
            }
            if (!ok) {
                // a wait ran out: give the copies still in flight another bounded
                // wait before the CTA leaves (their stages' next phases)
                for (int i = 0; i < pend && i < 2; ++i) {
                    const int blk = b + i;  // the copies of blocks b (and b+1) were issued, not waited
                    const int st = nstage == 2 ? (blk & 1) : 0;
                    const uint32_t use = nstage == 2 ? (uint32_t)(blk >> 1) : (uint32_t)blk;
                    wait_parity(tbar + st, use & 1u);
                }
            }
        } else {
            mma_block(tmem, stage_a(0), stage_b(0), NT, K / 16, true);  // only the staged K columns
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(mbar)));
            ok = wait_parity(mbar, 0);
        }
        if (!ok) atomicOr(err, 1u);
        ok_s = ok ? 1 : 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok_s) {
        // warp w reads TMEM lanes 32w..32w+31 (thread t holds row m0 + 32w + t,
        // 32 columns at a time), then turns each 32 x 32 block around through
        // shared memory (the operand staging area, free now that the products
        // completed; 33-float rows keep both passes free of bank conflicts) so
        // that lane l writes column c0 + l: every store covers consecutive
        // columns of one row
        float* st = reinterpret_cast<float*>(sA) + warp * (32 * 33);
        for (int c0 = 0; c0 < NT; c0 += 32) {
            // the ReLU mask of this warp's 32 rows at column n0 + c0 + lane, loaded
            // before the accumulator so that the 32 loads are in flight together
            // (indices clamped into the matrix: rows and columns past it are
            // loaded but not stored)
            float mk[32];
            if (EPI == MASK_BF16) {
                const int nn = min(n0 + c0 + lane, N - 1);
#pragma unroll
                for (int r = 0; r < 32; ++r) {
                    const int row = min(m0 + warp * 32 + r, M - 1);
                    mk[r] = __bfloat162float(mask[(size_t)row * ldmask + nn]);
                }
            }
            uint32_t v[32];
            const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                  "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                  "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
            for (int j = 0; j < 32; ++j) st[lane * 33 + j] = __uint_as_float(v[j]);
            __syncwarp();
            const int n = n0 + c0 + lane;
            const bool col_ok = c0 + lane < NT && n < N;
            const float b = (col_ok && (EPI == RELU_BF16 || EPI == LINEAR_F32)) ? bias[n] : 0.0f;
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                const int row = m0 + warp * 32 + r;
                if (row >= M || !col_ok) continue;
                const float x = st[r * 33 + lane];
                const size_t o = (size_t)row * ldc + n;
                if (EPI == RELU_BF16) {
                    outb[o] = __float2bfloat16(fmaxf(x + b, 0.0f));
                } else if (EPI == LINEAR_F32) {
                    outf[o] = x + b;
                } else if (EPI == MASK_BF16) {
                    const float y = mk[r] > 0.0f ? x : 0.0f;
                    outb[o] = __float2bfloat16(y);
                    outf[o] = y;
                } else {
                    atomicAdd(&outf[o], x);
                }
            }
            __syncwarp();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(ncols));
    }
}

// BF16 transpose: out[c][r] = in[r][c] for in [rows x cols] (leading dims
// ld_in, ld_out), 32 x 32 tiles through shared memory.
__global__ void transpose_bf16_kernel(const __nv_bfloat16* __restrict__ in, int rows, int cols, int ld_in,
                                      __nv_bfloat16* __restrict__ out, int ld_out) {
    __shared__ __nv_bfloat16 t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        t[i][threadIdx.x] = (r < rows && c < cols) ? in[(size_t)r * ld_in + c] : __float2bfloat16(0.0f);
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (c < cols && r < rows) out[(size_t)c * ld_out + r] = t[threadIdx.x][i];
    }
}

// Dynamic shared memory of a 128 x NT tile with `stages` staging areas of two
// 64-column panels of A and W each (+1 KiB alignment slack, four mbarriers and
// the TMEM address).
__host__ __device__ constexpr size_t smem_bytes(int nt, int stages) {
    return 1024 + (size_t)stages * kMaxPanels * (kTileM + nt) * 128 + 64;
}

// 2D BF16 tensor map of a row-major [rows x cols] matrix with leading
// dimension ld, box of box_rows x 64 columns, 128-byte swizzle, zero fill.
inline bool make_map(CUtensorMap* map, const void* ptr, int rows, int cols, int ld, int box_rows) {
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = (Encode)fn;
    }
    if (((uintptr_t)ptr & 15u) || ((size_t)ld * 2) % 16) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kPanel, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace umma
}  // namespace rddmc
