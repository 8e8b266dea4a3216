// walk_common.cuh -- what the DDMC walk kernels share: their parameter block,
// Philox4x32-10 with precomputed round keys, shared-memory tallies and the
// escape geometry of a packet that leaves the grid.
#pragma once
#include <cstdint>

#include "escape.cuh"
#include "grid.h"

namespace rddmc {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kSmemHistMax = 8192;  // histogram entries kept in shared memory

struct WalkParams {
    const uint4* rows;
    const uint2* fast;
    const float* tau_row;     // tau_ij = k_ij dz per row (hybrid conversions)
    const float2* upar;       // u_par envelope split points
    const ClassDesc* cdesc;
    const uint32_t* cell_class;
    const Rebin* rebin;
    const double* cell_v;     // km/s, 3 per cell (moving media)
    const double* edges;
    const uint32_t* abs_thr;  // per row: where dust absorption starts (dust only)
    int dust;                 // the draw has the absorption outcome (Sec. 2.6)
    const uint32_t* redist;   // hybrid: frequency-grouped MC (Sec. 5.3), J rows of J-1 thresholds, or null
    float inv_dzmin;          // 1 / dz_min: k of a row = tau_row / dz_min
    const unsigned long long* wq;  // dust weight method: -ln(weight kept per dwell) per row, 2^-40 units
    unsigned long long* st_lw;     // per packet: accumulated -ln(weight), 2^-40 units
    int weights;                   // the dust weight method is on (Sec. 2.6)
    int hist_off_w;                // tally word of the escaped weight (then one per escape bin)
    unsigned long long* cursor;
    uint32_t* st_cell;
    uint32_t* st_bin;
    unsigned long long* st_t;
    unsigned long long* st_e;
    uint8_t* st_status;
    unsigned long long* tally;
    unsigned long long n_packets, max_steps, slice, mc_cap;
    unsigned long long time_slice_ns;  // wall-time slice of the launch (0 = none)
    uint32_t k0, k1;
    uint32_t rk0[10], rk1[10];  // Philox round keys k + r * (Weyl constant)
    int J, n_rows, n_class, ncell, chunk;
    int n0, n01;
    double R, dz[3], vth;
    int resume, save_state, hist_in_smem, moving, hybrid;
    int n[3];
    float a, lambda;
    int src_ncand[3], src_cand[3][2], src_nbin, src_bin[2];
    // learned exit proposal (3D DDMC): bricks of prop_b^3 cells, brick
    // coordinate (i + prop_sh) / prop_b of cell index i on every axis; the
    // served region of a brick is its inner cube of side prop_r = prop_b -
    // 2 prop_m
    int prop_b, prop_sh, prop_nbx, prop_nby, prop_m, prop_r;
    const float* prop_lk;
    const float* prop_lp;
    float prop_llo, prop_lhi;
    unsigned long long* prop_qcount;
    unsigned long long* prop_qpid;
    // region mode (media that vary from cell to cell): kRegionSum floats per
    // brick summarising its inner cube; null for uniform bricks (symmetry fold)
    const float* prop_sum;
};

// Philox4x32-10 with precomputed round keys (held in the kernel's parameter bank).
__device__ __forceinline__ uint4 philox_rk(uint4 c, const WalkParams& P) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ P.rk0[r], lo1, hi0 ^ c.w ^ P.rk1[r], lo0);
    }
    return c;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned word_of(const uint4& r, unsigned q) {
    return q == 0 ? r.x : (q == 1 ? r.y : (q == 2 ? r.z : r.w));
}

// Shared-memory tally update aggregated over the lanes that hit the same index.
__device__ __forceinline__ void smem_tally(unsigned long long* s, unsigned idx) {
    const unsigned active = __activemask();
    const unsigned peers = __match_any_sync(active, idx);
    const int leader = __ffs(peers) - 1;
    if ((int)(threadIdx.x & 31) == leader) atomicAdd(&s[idx], (unsigned long long)__popc(peers));
}

// Escape through `face` of `cell` at `bin`.  A static slab cell tallies its
// bin; otherwise the escape geometry (escape.cuh) decides the bins.  OOL:
// the geometry is an out-of-line call and the rest inline (the persistent
// walk, measured faster this way); otherwise the whole function is out of
// line (the time-dependent walk, whose hot loop keeps its registers then).
template <int NDIM, bool OOL>
__device__ __forceinline__ EscapeBins escape_bins_body(const WalkParams& P, unsigned cell, unsigned bin,
                                                       unsigned face, unsigned long long pid, unsigned long long e,
                                                       bool moving) {
    if (NDIM == 1 && !moving) {
        EscapeBins out;
        out.hist = (int)bin + 1;
        out.sb = -1;
        return out;
    }
    int idx[3];
    idx[0] = (int)(cell % (unsigned)P.n0);
    idx[1] = NDIM == 3 ? (int)((cell / (unsigned)P.n0) % (unsigned)(P.n01 / P.n0)) : 0;
    idx[2] = NDIM == 3 ? (int)(cell / (unsigned)P.n01) : 0;
    const EscapeFrame F{NDIM, P.J, P.R, P.vth, P.dz, P.edges, moving ? P.cell_v + 3ull * cell : nullptr};
    return OOL ? escape_geometry_ool(F, idx, bin, face, pid, e, P.k0, P.k1)
               : escape_geometry(F, idx, bin, face, pid, e, P.k0, P.k1);
}

template <int NDIM>
__device__ __noinline__ EscapeBins escape_bins(const WalkParams& P, unsigned cell, unsigned bin, unsigned face,
                                               unsigned long long pid, unsigned long long e, bool moving) {
    return escape_bins_body<NDIM, false>(P, cell, bin, face, pid, e, moving);
}

template <int NDIM>
__device__ __forceinline__ EscapeBins escape_bins_inl(const WalkParams& P, unsigned cell, unsigned bin, unsigned face,
                                                      unsigned long long pid, unsigned long long e, bool moving) {
    return escape_bins_body<NDIM, true>(P, cell, bin, face, pid, e, moving);
}

// Parameter block of a walk launch (tables, state arrays, stream keys, source).
void fill_walk_params(const rddmc_grid& g, const WalkLaunch& w, WalkParams& P);

}  // namespace rddmc
