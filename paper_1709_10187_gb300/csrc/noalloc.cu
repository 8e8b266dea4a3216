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
#include "grid.h"

namespace {

// Packet cursor and saved per-packet state of the no-allocation launch.
static __device__ __align__(256) unsigned char g_walk_scratch[RDDMC_NOALLOC_SCRATCH_BYTES];

// Device address of g_walk_scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress, with that device current.  It is looked up on every
// call (a host-side query): a cached address would go stale once the device's
// context is destroyed and created again (cudaDeviceReset), which loads the
// library's device code, and the array, anew.
int scratch_address(void** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_walk_scratch) != cudaSuccess || !p) return RDDMC_ERR_CUDA;
    *out = p;
    return RDDMC_OK;
}

}  // namespace

extern "C" int rddmc_launch_packets_noalloc(const rddmc_grid* g, const void* d_table, const rddmc_run_opts* o,
                                            void* d_tallies, size_t tally_bytes, void* stream) {
    // Parked packets of a learned proposal need a caller-owned state buffer.
    if (o && o->proposal) return RDDMC_ERR_UNSUPPORTED;
    // Every other rule is rddmc_launch_packets' own (one shared check), with
    // the library's array in place of the state buffer.
    const int rc = rddmc::check_walk_launch(g, d_table, o, nullptr, true, d_tallies, tally_bytes);
    if (rc != RDDMC_OK) return rc;
    // A run to completion only uses the packet cursor; time-sliced or resumed
    // runs keep every packet's state in the array, which bounds their packet
    // count (about 1 million packets).
    const bool sliced = o->steps_per_launch != 0 || o->resume != 0 || o->time_slice_us != 0;
    const uint64_t need = sliced ? rddmc::state_bytes_for(o->n_packets) : 256ull;
    if (need > (uint64_t)RDDMC_NOALLOC_SCRATCH_BYTES) return RDDMC_ERR_SIZE;
    void* scratch = nullptr;
    const int ra = scratch_address(&scratch);
    if (ra != RDDMC_OK) return ra;
    rddmc::WalkLaunch w{d_table, scratch, (unsigned long long*)d_tallies, *o};
    return rddmc::launch_walk(*g, w, (cudaStream_t)stream) == cudaSuccess ? RDDMC_OK : RDDMC_ERR_CUDA;
}
