// api.cu -- host side of the C-ABI declared in include/rddmc.h.
//
// Builds the host grid handle (validation, class deduplication, table layout),
// uploads the per-class inputs of the leakage precompute, validates launches and
// reads tallies.  All device compute lives in precompute.cu and walk.cu.
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "grid.h"

using namespace rddmc;

namespace {

constexpr double kTwo32 = 4294967296.0;

uint32_t quantise(double C) {
    double t = std::nearbyint(C * kTwo32);
    if (t < 0.0) t = 0.0;
    if (t > kTwo32 - 1.0) t = kTwo32 - 1.0;
    return (uint32_t)t;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? RDDMC_OK : RDDMC_ERR_CUDA; }

}  // namespace

bool rddmc_grid::in_medium(const int idx[3]) const {
    for (int a = 0; a < 3; ++a)
        if (idx[a] < 0 || idx[a] >= n[a]) return false;
    if (mask.empty()) return true;
    return mask[cell_of(idx)] != 0;
}

namespace rddmc {

uint64_t state_bytes_for(uint64_t np) {
    uint64_t b = 256;                     // cursor + spare words
    b += align256(np * 4);                // cell
    b += align256(np * 4);                // bin
    b += align256(np * 8);                // transitions so far
    b += align256(np * 8);                // event draws so far
    b += align256(np * 1);                // status
    b += align256(np * 8);                // -ln(weight) in 2^-40 units (dust weight method)
    return b;
}

// counters, faces, escape histogram, impact parameters, then the escaped
// weight (u64, 2^-32 units): total and per escape-histogram bin
int tally_words(int J) { return kHistOff + J + 2 + kNsb + J + 3; }
uint64_t tally_bytes_for(int J) { return (uint64_t)tally_words(J) * 8ull; }

}  // namespace rddmc

extern "C" {

int rddmc_version(void) { return 100; }

const char* rddmc_status_string(int s) {
    switch (s) {
        case RDDMC_OK: return "ok";
        case RDDMC_ERR_ARG: return "invalid argument";
        case RDDMC_ERR_UNSUPPORTED: return "unsupported input";
        case RDDMC_ERR_SIZE: return "buffer too small";
        case RDDMC_ERR_CUDA: return "CUDA error";
        case RDDMC_ERR_STEP_LIMIT: return "packets aborted by the step watchdog";
        case RDDMC_ERR_TABLE: return "table not precomputed for this grid";
        case RDDMC_ERR_TIMEOUT: return "a bounded device wait ran out";
        default: return "unknown status";
    }
}

int rddmc_build_grid(const rddmc_grid_desc* d, rddmc_grid** out) {
    if (!d || !out) return RDDMC_ERR_ARG;
    *out = nullptr;
    if (d->geometry != RDDMC_GEOM_SLAB_1D && d->geometry != RDDMC_GEOM_CART_3D) return RDDMC_ERR_ARG;
    if (d->layout != RDDMC_LAYOUT_DEDUP && d->layout != RDDMC_LAYOUT_DENSE) return RDDMC_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (d->n[a] < 1 || d->n[a] > (1 << 20)) return RDDMC_ERR_ARG;
    if (d->geometry == RDDMC_GEOM_SLAB_1D && (d->n[1] != 1 || d->n[2] != 1)) return RDDMC_ERR_ARG;
    if (d->nbins < 1 || d->nbins > 65535) return RDDMC_ERR_ARG;
    if (!(d->R > 0.0) || !(d->tau0 >= 0.0) || !(d->T > 0.0) || !std::isfinite(d->tau0) || !std::isfinite(d->R) ||
        !std::isfinite(d->T))
        return RDDMC_ERR_ARG;
    if (!d->freq_edges) return RDDMC_ERR_ARG;
    const int64_t ncell = (int64_t)d->n[0] * d->n[1] * d->n[2];
    if (ncell > ((int64_t)1 << 31) - 1) return RDDMC_ERR_ARG;
    const int J = d->nbins;
    for (int j = 0; j <= J; ++j)
        if (!std::isfinite(d->freq_edges[j])) return RDDMC_ERR_ARG;
    for (int j = 0; j < J; ++j)
        if (!(d->freq_edges[j + 1] > d->freq_edges[j])) return RDDMC_ERR_ARG;
    if (d->n_rel)
        for (int64_t c = 0; c < ncell; ++c)
            if (!(d->n_rel[c] >= 0.0) || !std::isfinite(d->n_rel[c])) return RDDMC_ERR_ARG;
    if (d->v_kms)
        for (int64_t c = 0; c < 3 * ncell; ++c)
            if (!std::isfinite(d->v_kms[c])) return RDDMC_ERR_ARG;

    rddmc_grid* g = new (std::nothrow) rddmc_grid();
    if (!g) return RDDMC_ERR_ARG;
    g->ndim = d->geometry == RDDMC_GEOM_SLAB_1D ? 1 : 3;
    for (int a = 0; a < 3; ++a) g->n[a] = d->n[a];
    g->J = J;
    g->layout = d->layout;
    g->ncell = ncell;
    g->K = 2 + 2 * g->ndim;
    g->nfaces = 2 * g->ndim;
    g->row_bytes = g->ndim == 1 ? 16 : 32;
    g->R = d->R;
    g->tau0 = d->tau0;
    g->T = d->T;
    g->a = 4.702e-4 / std::sqrt(d->T / 1.0e4);  // Sec. 2.1
    g->edges.assign(d->freq_edges, d->freq_edges + J + 1);
    const double dx0 = g->edges[1] - g->edges[0];
    for (int j = 0; j < J; ++j)
        if (std::fabs((g->edges[j + 1] - g->edges[j]) - dx0) > 1e-9 * std::fabs(dx0)) g->uniform_bins = false;
    g->n_rel.resize(ncell);
    for (int64_t c = 0; c < ncell; ++c) g->n_rel[c] = d->n_rel ? d->n_rel[c] : 1.0;
    if (d->mask) g->mask.assign(d->mask, d->mask + ncell);
    g->vth = 12.85 * std::sqrt(d->T / 1.0e4);  // Sec. 2.1
    if (d->v_kms) {
        bool any = false;
        for (int64_t i = 0; i < 3 * ncell; ++i) any |= d->v_kms[i] != 0.0;
        g->moving = any;
        if (any) g->v.assign(d->v_kms, d->v_kms + 3 * ncell);
    }
    if (g->moving && !g->uniform_bins) { delete g; return RDDMC_ERR_UNSUPPORTED; }

    // Source: the centre cell(s) per axis and the bin(s) containing x0 = 0.
    for (int a = 0; a < 3; ++a) {
        const int m = g->n[a];
        if (m % 2) { g->src_ncand[a] = 1; g->src_cand[a][0] = g->src_cand[a][1] = m / 2; }
        else { g->src_ncand[a] = 2; g->src_cand[a][0] = m / 2 - 1; g->src_cand[a][1] = m / 2; }
    }
    g->src_nbin = 0;
    for (int j = 1; j < J; ++j)
        if (g->edges[j] == 0.0) { g->src_nbin = 2; g->src_bin[0] = j - 1; g->src_bin[1] = j; }
    if (!g->src_nbin)
        for (int j = 0; j < J; ++j)
            if (g->edges[j] < 0.0 && 0.0 < g->edges[j + 1]) { g->src_nbin = 1; g->src_bin[0] = g->src_bin[1] = j; }
    if (!g->src_nbin) { delete g; return RDDMC_ERR_ARG; }
    {
        int idx[3];
        for (int a = 0; a < 3; ++a) idx[a] = g->src_cand[a][0];
        for (int b = 0; b < 8; ++b) {
            for (int a = 0; a < 3; ++a) idx[a] = g->src_cand[a][(b >> a) & 1];
            if (!g->in_medium(idx)) { delete g; return RDDMC_ERR_ARG; }
        }
    }

    // Classes of cells with identical rows.  A row depends only on the cell's
    // density and on whether it moves and, per face, on whether the neighbour is
    // medium, on its density and on the normal velocity difference across the
    // face (the Doppler shift of eq. velocity-shift), so equal keys give equal
    // rows.  The cell's own velocity is only needed at escape and is read from
    // a per-cell array.
    g->cell_class.assign(ncell, UINT32_MAX);
    if (g->layout == RDDMC_LAYOUT_DENSE) {
        for (int64_t c = 0; c < ncell; ++c) g->cell_class[c] = (uint32_t)c;
        g->class_rep.resize(ncell);
        for (int64_t c = 0; c < ncell; ++c) g->class_rep[c] = c;
    } else {
        std::map<std::vector<double>, uint32_t> ids;
        std::vector<double> key;
        for (int64_t c = 0; c < ncell; ++c) {
            int idx[3];
            g->idx_of(c, idx);
            if (!g->in_medium(idx)) continue;
            key.clear();
            key.push_back(g->n_rel[c]);
            key.push_back((!g->v.empty() && (g->v[3 * c] != 0.0 || g->v[3 * c + 1] != 0.0 || g->v[3 * c + 2] != 0.0))
                              ? 1.0 : 0.0);
            for (int ax = 0; ax < g->ndim; ++ax)
                for (int sd = 0; sd < 2; ++sd) {
                    int nidx[3] = {idx[0], idx[1], idx[2]};
                    nidx[ax] += sd ? 1 : -1;
                    if (!g->in_medium(nidx)) { key.push_back(1.0); key.push_back(0.0); key.push_back(0.0); continue; }
                    const int64_t nb = g->cell_of(nidx);
                    key.push_back(0.0);
                    key.push_back(g->n_rel[nb]);
                    key.push_back(g->v.empty() ? 0.0 : g->v[3 * c + ax] - g->v[3 * nb + ax]);
                }
            auto it = ids.find(key);
            if (it == ids.end()) {
                const uint32_t id = (uint32_t)g->class_rep.size();
                ids.emplace(key, id);
                g->class_rep.push_back(c);
                g->cell_class[c] = id;
            } else {
                g->cell_class[c] = it->second;
            }
        }
    }
    g->n_class = (int)g->class_rep.size();
    if ((uint64_t)g->n_class * (uint64_t)J > (1ull << 40)) { delete g; return RDDMC_ERR_UNSUPPORTED; }

    // Table layout.
    uint64_t off = align256(sizeof(TableHeader));
    g->off_class = off; off += align256((uint64_t)ncell * 4);
    g->off_cdesc = off; off += align256((uint64_t)g->n_class * sizeof(ClassDesc));
    g->off_rebin = off; off += align256((uint64_t)g->n_class * g->nfaces * sizeof(Rebin));
    g->off_vel = off; off += align256(g->moving ? (uint64_t)ncell * 24 : 0);
    g->off_edges = off; off += align256((uint64_t)(J + 1) * 8);
    g->off_phi = off; off += align256((uint64_t)J * 8);
    g->off_rows = off; off += align256((uint64_t)g->n_class * J * g->row_bytes);
    g->off_fast = off; off += align256((uint64_t)g->n_class * J * 8);
    g->off_tau = off; off += align256((uint64_t)g->n_class * J * 4);
    g->off_upar = off; off += align256((uint64_t)kUparN * 8);
    g->off_rk = off; off += align256((uint64_t)g->n_class * J * 4);
    g->off_abs = off; off += align256((uint64_t)g->n_class * J * 4);
    g->off_wq = off; off += align256((uint64_t)g->n_class * J * 8);
    g->off_ka = off; off += align256((uint64_t)g->n_class * J * 4);
    g->table_bytes = off;
    *out = g;
    return RDDMC_OK;
}

void rddmc_destroy_grid(rddmc_grid* g) { delete g; }

int rddmc_grid_sizes(const rddmc_grid* g, uint64_t n_packets, rddmc_sizes* out) {
    if (!g || !out) return RDDMC_ERR_ARG;
    if (n_packets >= (1ull << 63)) return RDDMC_ERR_ARG;
    out->table_bytes = g->table_bytes;
    out->tally_bytes = tally_bytes_for(g->J);
    out->state_bytes = state_bytes_for(n_packets);
    out->n_class = g->n_class;
    out->row_bytes = g->row_bytes;
    out->n_outcomes = g->K + (g->precomputed && g->dusty() ? 1 : 0);
    out->reserved = 0;
    return RDDMC_OK;
}

int rddmc_precompute_leakage(rddmc_grid* g, const rddmc_leak_params* p, void* d_table, size_t table_bytes,
                             void* stream) {
    if (!g || !p || !d_table) return RDDMC_ERR_ARG;
    if (((uintptr_t)d_table & 255u) != 0) return RDDMC_ERR_ARG;
    if (table_bytes < g->table_bytes) return RDDMC_ERR_SIZE;
    if (!(p->tau_ddmc > 0.0) || !(p->lambda >= 0.0) || !(p->f_mu >= 0.0 && p->f_mu <= 1.0) ||
        (p->mode != RDDMC_MODE_DDMC && p->mode != RDDMC_MODE_HYBRID))
        return RDDMC_ERR_ARG;
    if (!(p->dust_abs >= 0.0) || !(p->dust_scat >= 0.0) || !std::isfinite(p->dust_abs) ||
        !std::isfinite(p->dust_scat))
        return RDDMC_ERR_ARG;
    if (p->dust_method != RDDMC_DUST_PROBABILISTIC && p->dust_method != RDDMC_DUST_WEIGHTS) return RDDMC_ERR_ARG;
    if (p->dust_abs > 0.0 && p->mode != RDDMC_MODE_DDMC) return RDDMC_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    g->params = *p;

    // Per-class inputs of the FP64 precompute kernel.
    std::vector<ClassDesc> cd(g->n_class);
    std::vector<Rebin> rb((size_t)g->n_class * g->nfaces);
    const double dx0 = g->edges[1] - g->edges[0];
    for (int k = 0; k < g->n_class; ++k) {
        const int64_t c = g->class_rep[k];
        int idx[3];
        g->idx_of(c, idx);
        ClassDesc& D = cd[k];
        std::memset(&D, 0, sizeof(D));
        D.k0 = g->tau0 / g->R * g->n_rel[c];
        D.ks = p->dust_scat / g->R * g->n_rel[c];
        D.ka = p->dust_abs / g->R * g->n_rel[c];
        D.moving = (!g->v.empty() && (g->v[3 * c] != 0.0 || g->v[3 * c + 1] != 0.0 || g->v[3 * c + 2] != 0.0)) ? 1 : 0;
        for (int ax = 0; ax < g->ndim; ++ax)
            for (int sd = 0; sd < 2; ++sd) {
                const int side = sd ? 1 : -1, f = 2 * ax + sd;
                int nidx[3] = {idx[0], idx[1], idx[2]};
                nidx[ax] += side;
                double delta = 0.0;
                if (!g->in_medium(nidx)) {
                    D.face[f].exterior = 1;
                } else {
                    const int64_t nb = g->cell_of(nidx);
                    D.face[f].exterior = 0;
                    D.face[f].k0_nb = g->tau0 / g->R * g->n_rel[nb];
                    D.face[f].ks_nb = p->dust_scat / g->R * g->n_rel[nb];
                    if (!g->v.empty())
                        delta = p->f_mu * (double)side * ((g->v[3 * c + ax] - g->v[3 * nb + ax]) / g->vth);
                }
                D.face[f].delta = delta;
                const double q = delta / dx0, m = std::floor(q), fr = q - m;
                rb[(size_t)k * g->nfaces + f].m = (int32_t)m;
                rb[(size_t)k * g->nfaces + f].thr = quantise(1.0 - fr);
            }
    }
    TableHeader h;
    std::memset(&h, 0, sizeof(h));
    h.magic = kMagic;
    h.filled = 1;
    h.ndim = g->ndim; h.J = g->J; h.ncell = (int32_t)g->ncell; h.n_class = g->n_class; h.K = g->K;
    h.row_bytes = g->row_bytes;
    for (int a = 0; a < 3; ++a) { h.n[a] = g->n[a]; h.dz[a] = 2.0 * g->R / g->n[a]; }
    h.mode = p->mode;
    h.off_class = g->off_class; h.off_cdesc = g->off_cdesc; h.off_rebin = g->off_rebin; h.off_vel = g->off_vel;
    h.off_edges = g->off_edges; h.off_phi = g->off_phi; h.off_rows = g->off_rows; h.off_fast = g->off_fast;
    h.off_tau = g->off_tau; h.off_upar = g->off_upar;
    h.total = g->table_bytes;
    h.tau_ddmc = p->tau_ddmc; h.lambda = p->lambda; h.f_mu = p->f_mu; h.a = g->a; h.vth = g->vth;

    char* base = (char*)d_table;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(base, &h, sizeof(h), cudaMemcpyHostToDevice, s)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaMemcpyAsync(base + g->off_class, g->cell_class.data(), g->cell_class.size() * 4,
                             cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_status(e);
    if ((e = cudaMemcpyAsync(base + g->off_cdesc, cd.data(), cd.size() * sizeof(ClassDesc), cudaMemcpyHostToDevice,
                             s)) != cudaSuccess)
        return cuda_status(e);
    if ((e = cudaMemcpyAsync(base + g->off_rebin, rb.data(), rb.size() * sizeof(Rebin), cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
        return cuda_status(e);
    if (g->moving && (e = cudaMemcpyAsync(base + g->off_vel, g->v.data(), g->v.size() * 8, cudaMemcpyHostToDevice,
                                          s)) != cudaSuccess)
        return cuda_status(e);
    if ((e = cudaMemcpyAsync(base + g->off_edges, g->edges.data(), g->edges.size() * 8, cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
        return cuda_status(e);
    // Pageable-memory copies are staged before cudaMemcpyAsync returns, so the
    // host vectors above may go out of scope; the kernels follow in stream order.
    if ((e = launch_precompute(*g, d_table, s)) != cudaSuccess) return cuda_status(e);
    g->precomputed = true;
    return RDDMC_OK;
}

int rddmc_reset_tallies(const rddmc_grid* g, void* d_tallies, size_t tally_bytes, void* stream) {
    if (!g || !d_tallies) return RDDMC_ERR_ARG;
    if (((uintptr_t)d_tallies & 7u) != 0) return RDDMC_ERR_ARG;
    if (tally_bytes < tally_bytes_for(g->J)) return RDDMC_ERR_SIZE;
    return cuda_status(cudaMemsetAsync(d_tallies, 0, tally_bytes_for(g->J), (cudaStream_t)stream));
}

int rddmc_launch_packets(const rddmc_grid* g, const void* d_table, const rddmc_run_opts* o, void* d_state,
                         size_t state_bytes, void* d_tallies, size_t tally_bytes, void* stream) {
    const int rc = check_walk_launch(g, d_table, o, d_state, false, d_tallies, tally_bytes);
    if (rc != RDDMC_OK) return rc;
    if (state_bytes < state_bytes_for(o->n_packets)) return RDDMC_ERR_SIZE;
    WalkLaunch w{d_table, d_state, (unsigned long long*)d_tallies, *o};
    return cuda_status(launch_walk(*g, w, (cudaStream_t)stream));
}

}  // extern "C"

namespace rddmc {

int check_walk_launch(const rddmc_grid* g, const void* d_table, const rddmc_run_opts* o, const void* d_state,
                      bool library_state, const void* d_tallies, size_t tally_bytes) {
    if (!g || !d_table || !o || (!library_state && !d_state) || !d_tallies) return RDDMC_ERR_ARG;
    if (!g->precomputed) return RDDMC_ERR_TABLE;
    if (((uintptr_t)d_table & 255u) || (!library_state && ((uintptr_t)d_state & 255u)) ||
        ((uintptr_t)d_tallies & 7u))
        return RDDMC_ERR_ARG;
    if (o->n_packets == 0 || o->n_packets >= (1ull << 63)) return RDDMC_ERR_ARG;
    if (o->steps_per_launch % 4 != 0) return RDDMC_ERR_ARG;
    if (o->chunk < 0 || o->chunk % 4 != 0 || o->ctas_per_sm < 0 || o->threads_per_cta < 0) return RDDMC_ERR_ARG;
    if (o->threads_per_cta && (o->threads_per_cta % 32 != 0 || o->threads_per_cta > 256)) return RDDMC_ERR_ARG;
    if (o->resume != 0 && o->resume != 1) return RDDMC_ERR_ARG;
    if (o->time_slice_us < 0) return RDDMC_ERR_ARG;
    // frequency-grouped MC needs thin states, i.e. a hybrid table
    if (o->redist && (g->params.mode != RDDMC_MODE_HYBRID || ((uintptr_t)o->redist & 3u))) return RDDMC_ERR_ARG;
    if (o->time_slice_us > 0 && o->steps_per_launch == 0 && o->resume == 0 && !o->proposal) return RDDMC_ERR_ARG;
    if (o->proposal) {
        const rddmc_proposal* pr = o->proposal;
        // the learned proposal samples first passages without absorption
        if (g->ndim != 3 || g->params.mode != RDDMC_MODE_DDMC || g->dusty() || g->weighted())
            return RDDMC_ERR_UNSUPPORTED;
        if (o->steps_per_launch == 0 && o->resume == 0 && o->time_slice_us == 0) return RDDMC_ERR_ARG;
        if (pr->brick < 1 || pr->brick > 64 || pr->offset < 0 || pr->offset >= pr->brick) return RDDMC_ERR_ARG;
        if (pr->margin < 0 || 2 * pr->margin >= pr->brick) return RDDMC_ERR_ARG;
        if ((int64_t)pr->n_bricks != proposal_bricks(*g, *pr)) return RDDMC_ERR_ARG;
        if (!pr->d_brick_lk || !pr->d_lp || !pr->d_xc || !pr->d_queue_count || !pr->d_queue_pid)
            return RDDMC_ERR_ARG;
    }
    if (tally_bytes < tally_bytes_for(g->J)) return RDDMC_ERR_SIZE;
    return RDDMC_OK;
}

}  // namespace rddmc

extern "C" {

int rddmc_read_tallies(const rddmc_grid* g, const void* d_tallies, rddmc_tallies* out, uint64_t* hist,
                       uint64_t* faces, uint64_t* sb, void* stream) {
    if (!g || !d_tallies || !out) return RDDMC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<uint64_t> t(tally_words(g->J));
    cudaError_t e = cudaMemcpyAsync(t.data(), d_tallies, t.size() * 8, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return RDDMC_ERR_CUDA;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return RDDMC_ERR_CUDA;
    out->emitted = t[C_EMITTED];
    out->escaped = t[C_ESCAPED];
    out->aborted = t[C_ABORTED];
    out->steps = t[C_STEPS];
    out->mc_events = t[C_MC_EVENTS];
    out->conversions = t[C_CONVERSIONS];
    out->clamps = t[C_CLAMPS];
    out->event_draws = t[C_EVENT_DRAWS];
    out->proposals = t[C_PROPOSALS];
    out->proposed_steps = t[C_PROPOSED_STEPS];
    out->absorbed = t[C_ABSORBED];
    out->escaped_weight = (double)t[kHistOff + g->J + 2 + kNsb] * (1.0 / 4294967296.0);
    out->status = RDDMC_OK;
    if (t[C_ABORTED]) out->status = RDDMC_ERR_STEP_LIMIT;
    if (t[C_STATUS_BITS] & STATUS_UNSUPPORTED_EVENT) out->status = RDDMC_ERR_UNSUPPORTED;
    out->nbins = g->J;
    out->nfaces = g->nfaces;
    out->nsb = kNsb;
    if (hist) std::memcpy(hist, t.data() + kHistOff, (size_t)(g->J + 2) * 8);
    if (faces) std::memcpy(faces, t.data() + kFaceOff, (size_t)g->nfaces * 8);
    if (sb) std::memcpy(sb, t.data() + kHistOff + g->J + 2, (size_t)kNsb * 8);
    return RDDMC_OK;
}

int rddmc_read_escape_weights(const rddmc_grid* g, const void* d_tallies, double* whist, void* stream) {
    if (!g || !d_tallies || !whist) return RDDMC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<uint64_t> t(g->J + 2);
    const uint64_t off = (uint64_t)(kHistOff + g->J + 2 + kNsb + 1) * 8;
    if (cudaMemcpyAsync(t.data(), (const char*)d_tallies + off, t.size() * 8, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return RDDMC_ERR_CUDA;
    for (size_t i = 0; i < t.size(); ++i) whist[i] = (double)t[i] * (1.0 / 4294967296.0);
    return RDDMC_OK;
}

int rddmc_table_rows(const rddmc_grid* g, const void* d_table, uint32_t* thr, uint32_t* flags, void* stream) {
    if (!g || !d_table || !thr || !flags) return RDDMC_ERR_ARG;
    if (!g->precomputed) return RDDMC_ERR_TABLE;
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t nrow = (uint64_t)g->n_class * g->J;
    std::vector<uint32_t> rows(nrow * g->row_bytes / 4);
    cudaError_t e = cudaMemcpyAsync(rows.data(), (const char*)d_table + g->off_rows, rows.size() * 4,
                                    cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return RDDMC_ERR_CUDA;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return RDDMC_ERR_CUDA;
    const int wpr = g->row_bytes / 4, K = g->K + (g->dusty() ? 1 : 0);
    std::vector<uint32_t> ab;
    if (g->dusty()) {
        ab.resize(nrow);
        if (cudaMemcpyAsync(ab.data(), (const char*)d_table + g->off_abs, nrow * 4, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return RDDMC_ERR_CUDA;
    }
    for (int64_t c = 0; c < g->ncell; ++c) {
        const uint32_t k = g->cell_class[c];
        for (int j = 0; j < g->J; ++j) {
            const uint64_t s_ = (uint64_t)c * g->J + j;
            if (k == UINT32_MAX) {
                for (int o = 0; o < K - 1; ++o) thr[s_ * (K - 1) + o] = 0;
                flags[s_] = 0;
                continue;
            }
            // stored words: thr0, thr1, thr2, flags[, thr3..thr6]; FLAG_FASTX is
            // an encoding detail of the walk and is not returned
            const uint32_t* r = &rows[((uint64_t)k * g->J + j) * wpr];
            for (int o = 0; o < g->K - 1; ++o) thr[s_ * (K - 1) + o] = o < 3 ? r[o] : r[o + 1];
            if (g->dusty()) thr[s_ * (K - 1) + g->K - 1] = ab[(uint64_t)k * g->J + j];
            flags[s_] = r[3] & ~FLAG_FASTX;
        }
    }
    return RDDMC_OK;
}

int rddmc_read_packet_states(const rddmc_grid* g, const void* d_state, uint64_t np, uint64_t first, uint64_t count,
                             uint32_t* cell, uint32_t* bin, uint64_t* steps, uint64_t* edraws, uint8_t* status,
                             void* stream) {
    if (!g || !d_state) return RDDMC_ERR_ARG;
    if (np == 0 || first > np || count > np - first) return RDDMC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const char* sb = (const char*)d_state;
    uint64_t off = 256;
    const uint64_t o_cell = off; off += align256(np * 4);
    const uint64_t o_bin = off; off += align256(np * 4);
    const uint64_t o_t = off; off += align256(np * 8);
    const uint64_t o_e = off; off += align256(np * 8);
    const uint64_t o_st = off;
    cudaError_t e = cudaSuccess;
    if (cell && e == cudaSuccess) e = cudaMemcpyAsync(cell, sb + o_cell + first * 4, count * 4, cudaMemcpyDeviceToHost, s);
    if (bin && e == cudaSuccess) e = cudaMemcpyAsync(bin, sb + o_bin + first * 4, count * 4, cudaMemcpyDeviceToHost, s);
    if (steps && e == cudaSuccess) e = cudaMemcpyAsync(steps, sb + o_t + first * 8, count * 8, cudaMemcpyDeviceToHost, s);
    if (edraws && e == cudaSuccess) e = cudaMemcpyAsync(edraws, sb + o_e + first * 8, count * 8, cudaMemcpyDeviceToHost, s);
    if (status && e == cudaSuccess) e = cudaMemcpyAsync(status, sb + o_st + first, count, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? RDDMC_OK : RDDMC_ERR_CUDA;
}

int rddmc_scatter_samples(const rddmc_grid* g, const void* d_table, double x_in, uint64_t seed, uint64_t n,
                          float* d_out, void* stream) {
    if (!g || !d_table || !d_out || n == 0 || !std::isfinite(x_in)) return RDDMC_ERR_ARG;
    if (!g->precomputed) return RDDMC_ERR_TABLE;
    if (g->params.mode != RDDMC_MODE_HYBRID) return RDDMC_ERR_UNSUPPORTED;  // no envelope table in DDMC mode
    return cuda_status(launch_scatter_samples(*g, d_table, x_in, seed, n, d_out, (cudaStream_t)stream));
}

}  // extern "C"
