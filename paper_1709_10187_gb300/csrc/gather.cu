// gather.cu -- random dependent gathers: the memory system's rate for the
// access the walk makes once per transition.
//
// The walk reads one row of its leakage table per transition (an 8-byte fast
// head, or a 16/32-byte row) at an address that depends on the previous read.
// This probe measures how many such gathers per second the GPU serves when
// every thread chases its own chain through a table of a given footprint: in
// shared memory, or through L1/L2/HBM depending on the table's size.  The rate
// times the walk's bytes per transition is the gather roofline of the walk.
//
// Row r of the table holds, in its first word, the index of the next row:
// (a r + c) mod n with a = 1 (mod 4) and c odd, a single cycle through all
// n = 2^k rows (Hull-Dobell).  Each thread starts at a hashed row, so the 32
// lanes of a warp read 32 unrelated rows.  The other words of each row are
// folded into a checksum that keeps the loads alive.
#include <cstdint>

#include "grid.h"

namespace rddmc {
namespace {

constexpr uint32_t kLcgA = 1664525u;     // = 1 (mod 4)
constexpr uint32_t kLcgC = 1013904223u;  // odd

template <int RB>
struct Row;
template <>
struct Row<8> {
    using T = uint2;
};
template <>
struct Row<16> {
    using T = uint4;
};

__global__ void gather_fill_kernel(uint32_t* __restrict__ table, uint32_t mask, int words_per_row) {
    const uint64_t n = (uint64_t)mask + 1ull;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t* row = table + r * (uint64_t)words_per_row;
        row[0] = (kLcgA * (uint32_t)r + kLcgC) & mask;
        for (int w = 1; w < words_per_row; ++w) row[w] = (uint32_t)r * 0x9E3779B9u + (uint32_t)w;
    }
}

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7FEB352Du;
    x ^= x >> 15;
    x *= 0x846CA68Bu;
    x ^= x >> 16;
    return x;
}

__device__ __forceinline__ uint32_t fold(const uint2& v) { return v.y; }
__device__ __forceinline__ uint32_t fold(const uint4& v) { return v.y ^ v.z ^ v.w; }

// Every thread follows `chain` links of the cycle from its own start row.
// SMEM: the CTA first copies the whole table into shared memory and chases
// there; otherwise the loads go through L1 (ld.global.nc).
template <int RB, bool SMEM>
__global__ void gather_chase_kernel(const typename Row<RB>::T* __restrict__ table, uint32_t mask, uint32_t chain,
                                    uint32_t seed, unsigned long long* __restrict__ sink) {
    using T = typename Row<RB>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s_table = reinterpret_cast<T*>(smem_raw);
    if (SMEM) {
        const uint32_t n = mask + 1u;
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) s_table[i] = table[i];
        __syncthreads();
    }
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t r = mix32(tid ^ seed) & mask;
    uint32_t acc = 0;
#pragma unroll 4
    for (uint32_t i = 0; i < chain; ++i) {
        const T v = SMEM ? s_table[r] : __ldg(&table[r]);
        acc ^= fold(v);
        r = v.x & mask;
    }
    // a value the loads produce, written only in the (never expected) case that
    // it matches the seed, so that no load can be dropped
    if ((acc ^ r) == seed) atomicAdd(sink, 1ull);
}

// Launches ctas_per_sm CTAs per SM (0 or more than fit: as many as fit) and
// returns the number of threads it launched in *n_threads.
template <int RB, bool SMEM>
cudaError_t launch_chase(const void* table, uint32_t mask, uint32_t chain, int ctas_per_sm, int threads,
                         uint32_t seed, unsigned long long* sink, cudaStream_t s, uint64_t* n_threads) {
    const size_t smem = SMEM ? (size_t)(mask + 1u) * RB : 0;
    cudaError_t e = cudaFuncSetAttribute(gather_chase_kernel<RB, SMEM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, fit = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, gather_chase_kernel<RB, SMEM>, threads, smem)) !=
        cudaSuccess)
        return e;
    if (fit < 1) return cudaErrorInvalidConfiguration;
    const int ctas = ctas_per_sm > 0 ? (ctas_per_sm < fit ? ctas_per_sm : fit) : fit;
    gather_chase_kernel<RB, SMEM><<<(unsigned)(ctas * nsm), threads, smem, s>>>(
        reinterpret_cast<const typename Row<RB>::T*>(table), mask, chain, seed, sink);
    *n_threads = (uint64_t)ctas * (uint64_t)nsm * (uint64_t)threads;
    return cudaGetLastError();
}

}  // namespace
}  // namespace rddmc

using namespace rddmc;

extern "C" int rddmc_gather_probe(void* d_table, uint64_t table_bytes, int row_bytes, int in_smem, uint32_t chain,
                                  int ctas_per_sm, int threads_per_cta, uint64_t seed, int fill,
                                  unsigned long long* d_sink, uint64_t* gathers, void* stream) {
    if (!d_table || !d_sink || !gathers) return RDDMC_ERR_ARG;
    if (row_bytes != 8 && row_bytes != 16) return RDDMC_ERR_ARG;
    if (((uintptr_t)d_table & 255u) || ((uintptr_t)d_sink & 7u)) return RDDMC_ERR_ARG;
    if (threads_per_cta < 32 || threads_per_cta > 1024 || threads_per_cta % 32 || ctas_per_sm < 0 || chain == 0)
        return RDDMC_ERR_ARG;
    // a power-of-two number of rows, at least 64 and at most 2^32
    const uint64_t rows = table_bytes / (uint64_t)row_bytes;
    if (rows < 64 || rows > (1ull << 32) || (rows & (rows - 1)) || rows * (uint64_t)row_bytes != table_bytes)
        return RDDMC_ERR_ARG;
    if (in_smem && table_bytes > 200u * 1024u) return RDDMC_ERR_SIZE;
    const uint32_t mask = (uint32_t)(rows - 1ull);
    cudaStream_t s = (cudaStream_t)stream;
    if (fill) {
        gather_fill_kernel<<<1216, 256, 0, s>>>((uint32_t*)d_table, mask, row_bytes / 4);
        if (cudaGetLastError() != cudaSuccess) return RDDMC_ERR_CUDA;
    }
    cudaError_t e;
    uint64_t nt = 0;
    const uint32_t sd = (uint32_t)(seed ^ (seed >> 32));
    if (row_bytes == 8)
        e = in_smem ? launch_chase<8, true>(d_table, mask, chain, ctas_per_sm, threads_per_cta, sd, d_sink, s, &nt)
                    : launch_chase<8, false>(d_table, mask, chain, ctas_per_sm, threads_per_cta, sd, d_sink, s, &nt);
    else
        e = in_smem ? launch_chase<16, true>(d_table, mask, chain, ctas_per_sm, threads_per_cta, sd, d_sink, s, &nt)
                    : launch_chase<16, false>(d_table, mask, chain, ctas_per_sm, threads_per_cta, sd, d_sink, s, &nt);
    if (e != cudaSuccess) return RDDMC_ERR_CUDA;
    *gathers = nt * (uint64_t)chain;
    return RDDMC_OK;
}
