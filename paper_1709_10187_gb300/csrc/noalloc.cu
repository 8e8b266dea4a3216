// noalloc.cu -- rddmc_launch_packets_noalloc: the packet walk without a
// caller-allocated state buffer.
//
// The ordinary rddmc_launch_packets needs a caller-owned device buffer for the
// packet cursor and the saved per-packet state.  Some callers cannot provide
// one, because they cannot call cudaMalloc at all: a plug-in running inside a
// host application that owns every byte of device memory and hands the plug-in
// none, or a latency-sensitive caller that must not trigger the implicit
// device-wide synchronisation cudaMalloc can cause.  This entry point keeps that
// scratch in a fixed-size array compiled into the library instead.
//
// The array is RDDMC_NOALLOC_SCRATCH_BYTES (32 MiB) of device memory that every
// GPU that loads the library holds until the process exits.  Every call shares
// it and it keeps the previous call's contents: the launch zeroes the packet
// cursor before the kernel runs, and time-sliced runs resume from the state the
// previous call left there.  Calls whose work overlaps on the GPU (different
// streams, or different grids at the same time) race on the array.
#include <mutex>

#include "grid.h"

namespace {

// Packet cursor and saved per-packet state of the no-allocation launch.
static __device__ __align__(256) unsigned char g_walk_scratch[RDDMC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 128;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_walk_scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress, once per device, with that device current.
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RDDMC_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_walk_scratch) != cudaSuccess || !p) return RDDMC_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return RDDMC_OK;
}

}  // namespace

extern "C" int rddmc_launch_packets_noalloc(const rddmc_grid* g, const void* d_table, const rddmc_run_opts* o,
                                            void* d_tallies, size_t tally_bytes, void* stream) {
    // The same argument rules as rddmc_launch_packets, except for the state
    // buffer, which is the library's own array here.
    if (!g || !d_table || !o || !d_tallies) return RDDMC_ERR_ARG;
    if (!g->precomputed) return RDDMC_ERR_TABLE;
    if (((uintptr_t)d_table & 255u) || ((uintptr_t)d_tallies & 7u)) return RDDMC_ERR_ARG;
    if (o->n_packets == 0 || o->n_packets >= (1ull << 63)) return RDDMC_ERR_ARG;
    if (o->steps_per_launch % 4 != 0) return RDDMC_ERR_ARG;
    if (o->chunk < 0 || o->chunk % 4 != 0 || o->ctas_per_sm < 0 || o->threads_per_cta < 0) return RDDMC_ERR_ARG;
    if (o->threads_per_cta && (o->threads_per_cta % 32 != 0 || o->threads_per_cta > 256)) return RDDMC_ERR_ARG;
    if (o->resume != 0 && o->resume != 1) return RDDMC_ERR_ARG;
    if (o->time_slice_us < 0) return RDDMC_ERR_ARG;
    if (o->time_slice_us > 0 && o->steps_per_launch == 0 && o->resume == 0) return RDDMC_ERR_ARG;
    if (o->proposal) return RDDMC_ERR_UNSUPPORTED;  // parked packets need a caller-owned state buffer
    if (tally_bytes < rddmc::tally_bytes_for(g->J)) return RDDMC_ERR_SIZE;
    // A run to completion only uses the packet cursor; time-sliced or resumed
    // runs keep every packet's state in the array, which bounds their packet
    // count (about 1 million packets).
    const bool sliced = o->steps_per_launch != 0 || o->resume != 0 || o->time_slice_us != 0;
    const uint64_t need = sliced ? rddmc::state_bytes_for(o->n_packets) : 256ull;
    if (need > (uint64_t)RDDMC_NOALLOC_SCRATCH_BYTES) return RDDMC_ERR_SIZE;
    void* scratch = nullptr;
    const int rc = scratch_address(&scratch);
    if (rc != RDDMC_OK) return rc;
    rddmc::WalkLaunch w{d_table, scratch, (unsigned long long*)d_tallies, *o};
    return rddmc::launch_walk(*g, w, (cudaStream_t)stream) == cudaSuccess ? RDDMC_OK : RDDMC_ERR_CUDA;
}
