// grid.h -- host-side grid handle shared by the library's translation units.
#pragma once
#include <cstdint>
#include <vector>

#include "../../include/rddmc.h"
#include "rddmc_internal.cuh"

struct rddmc_grid {
    int ndim = 1;
    int n[3] = {1, 1, 1};
    int J = 0;
    int layout = RDDMC_LAYOUT_DEDUP;
    int64_t ncell = 0;
    int n_class = 0;
    int K = 4;          // outcomes per state
    int nfaces = 2;
    int row_bytes = 16;
    double R = 1.0, tau0 = 0.0, T = 1.0e4, a = 0.0;
    bool moving = false;
    bool uniform_bins = true;
    std::vector<double> edges;
    std::vector<uint32_t> cell_class;   // UINT32_MAX for vacuum cells
    std::vector<int64_t> class_rep;     // a representative cell per class
    std::vector<double> n_rel;          // per cell (copied)
    std::vector<double> v;              // per cell x3, km/s (empty if static)
    double vth = 12.85;                 // thermal velocity, km/s
    std::vector<uint8_t> mask;          // per cell (empty = all medium)
    // source (centre cells and bins containing x0 = 0)
    int src_ncand[3] = {1, 1, 1};
    int src_cand[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    int src_nbin = 0;
    int src_bin[2] = {0, 0};
    // table layout (byte offsets)
    uint64_t off_class = 0, off_cdesc = 0, off_rebin = 0, off_vel = 0, off_edges = 0, off_phi = 0,
             off_rows = 0, off_fast = 0, off_tau = 0, off_upar = 0, off_rk = 0, off_abs = 0, off_wq = 0, off_ka = 0, table_bytes = 0;
    // leakage parameters of the last precompute
    rddmc_leak_params params{};
    bool precomputed = false;
    // dust absorption as an outcome of the draw, or by packet weights (Sec. 2.6)
    bool dusty() const { return params.dust_abs > 0.0 && params.dust_method == RDDMC_DUST_PROBABILISTIC; }
    bool weighted() const { return params.dust_abs > 0.0 && params.dust_method == RDDMC_DUST_WEIGHTS; }

    bool in_medium(const int idx[3]) const;
    int64_t cell_of(const int idx[3]) const { return idx[0] + (int64_t)n[0] * (idx[1] + (int64_t)n[1] * idx[2]); }
    void idx_of(int64_t c, int idx[3]) const {
        idx[0] = (int)(c % n[0]);
        idx[1] = (int)((c / n[0]) % n[1]);
        idx[2] = (int)(c / ((int64_t)n[0] * n[1]));
    }
};

namespace rddmc {

// Kernel launch wrappers (defined next to their kernels).
cudaError_t launch_precompute(const rddmc_grid& g, void* d_table, cudaStream_t s);

struct WalkLaunch {
    const void* d_table;
    void* d_state;
    unsigned long long* d_tally;
    rddmc_run_opts opts;
};
cudaError_t launch_walk(const rddmc_grid& g, const WalkLaunch& w, cudaStream_t s);
cudaError_t launch_scatter_samples(const rddmc_grid& g, const void* d_table, double x_in, uint64_t seed, uint64_t n,
                                   float* d_out, cudaStream_t s);

// Argument checks of a walk launch, shared by rddmc_launch_packets and
// rddmc_launch_packets_noalloc: everything but the size of the packet-state
// buffer.  library_state: the state is the library's own array, so d_state is
// not checked.  Returns RDDMC_OK or the status the entry point returns.
int check_walk_launch(const rddmc_grid* g, const void* d_table, const rddmc_run_opts* o, const void* d_state,
                      bool library_state, const void* d_tallies, size_t tally_bytes);

uint64_t state_bytes_for(uint64_t n_packets);
uint64_t tally_bytes_for(int J);
int tally_words(int J);

// Bricks (partial ones included) of a proposal's lattice on grid g.
inline int64_t proposal_bricks(const rddmc_grid& g, const rddmc_proposal& pr) {
    const int sh = (pr.brick - pr.offset % pr.brick) % pr.brick;
    int64_t nb = 1;
    for (int a = 0; a < 3; ++a) nb *= (g.n[a] + sh + pr.brick - 1) / pr.brick;
    return nb;
}

}  // namespace rddmc
