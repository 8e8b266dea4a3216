// batch.cu -- many independent grids (instances) walked by one persistent
// kernel, a CUDA-graph wrapper for the launch sequence, and a host autotuner
// for the launch schedule.
//
// Instances keep their own precomputed tables (any mix of slabs and 3D grids,
// DDMC mode).  Their packets form one global id space: instance i owns ids
// [off_i, off_i + n_i) and its packet p uses the streams of global id off_i + p
// under the batch seed, so one Philox key schedule serves every lane.  A lane
// maps a refilled id to its instance by binary search over the offsets and
// walks it exactly as the single-grid kernel does (the 8-byte fast head for
// frequency moves, the full row otherwise).  Counters are kept per lane and
// added to the instance's tally block when the lane changes instance;
// escapes go straight to the instance's histograms with global atomics (they
// are rare and instances differ in size, so per-CTA shared histograms would
// not fit every instance).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "escape.cuh"
#include "grid.h"

namespace rddmc {
namespace {

constexpr unsigned FULL = 0xffffffffu;

struct InstDesc {
    const uint4* rows;
    const uint2* fast;
    const uint32_t* cell_class;
    const Rebin* rebin;
    const double* edges;
    const double* cell_v;
    unsigned long long tally_off;   // word offset of the instance's tally block
    unsigned long long pkt_begin;   // first global packet id
    double R, dz[3], vth;
    int J, n_rows, n_class, ncell, n0, n1, n01, ndim, moving;
    int src_ncand[3], src_cand[3][2], src_nbin, src_bin[2];
};

struct BatchParams {
    const InstDesc* desc;
    const unsigned long long* off;  // n_inst + 1 prefix offsets of the packets to run
    int n_inst;
    unsigned long long* cursor;
    unsigned long long* tally;
    unsigned long long total, max_steps;
    uint32_t k0, k1;
    uint32_t rk0[10], rk1[10];
    int chunk;
};

__device__ __forceinline__ uint4 bphilox(uint4 c, const BatchParams& P) {
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

__device__ __forceinline__ unsigned bword(const uint4& r, unsigned q) {
    return q == 0 ? r.x : (q == 1 ? r.y : (q == 2 ? r.z : r.w));
}

// Escape geometry of an instance (see the single-grid walk): static slab cells
// tally their bin; 3D grids and moving slab cells draw a face point, an
// isotropic outward direction and x in the bin (five event words).
__device__ __noinline__ void batch_escape(const BatchParams& P, const InstDesc& D, unsigned cell, unsigned bin,
                                          unsigned face, unsigned long long gid, unsigned long long e, bool moving) {
    unsigned long long* T = P.tally + D.tally_off;
    int hist, sb = -1;
    if (D.ndim == 1 && !moving) {
        hist = (int)bin + 1;
    } else {
        int idx[3];
        idx[0] = (int)(cell % (unsigned)D.n0);
        idx[1] = D.ndim == 3 ? (int)((cell / (unsigned)D.n0) % (unsigned)D.n1) : 0;
        idx[2] = D.ndim == 3 ? (int)(cell / (unsigned)D.n01) : 0;
        const EscapeFrame F{D.ndim, D.J, D.R, D.vth, D.dz, D.edges, moving ? D.cell_v + 3ull * cell : nullptr};
        const EscapeBins eb = escape_geometry(F, idx, bin, face, gid, e, P.k0, P.k1);
        hist = eb.hist;
        sb = eb.sb;
    }
    atomicAdd(&T[kHistOff + hist], 1ull);
    atomicAdd(&T[kFaceOff + face], 1ull);
    if (sb >= 0) atomicAdd(&T[kHistOff + D.J + 2 + sb], 1ull);
}

__global__ void __launch_bounds__(256, 3) batch_kernel(const BatchParams P) {
    const unsigned lane = threadIdx.x & 31u;
    bool have = false, exhausted = false;
    int inst = -1;
    // instance parameters held by the lane
    const uint2* fast = nullptr;
    const uint4* rows = nullptr;
    const uint32_t* cell_class = nullptr;
    unsigned J = 1, nr1 = 0, ncell1 = 0, ncls1 = 0, n0 = 1, n01 = 1, ndim = 1;
    unsigned long long gid = 0, t = 0, e = 0;
    unsigned cell = 0, cls = 0, s = 0;
    unsigned long long n_steps = 0, n_edraw = 0;
    unsigned n_emit = 0, n_esc = 0, n_abort = 0, n_clamp = 0;

    auto flush = [&]() {
        if (inst < 0) return;
        unsigned long long* T = P.tally + P.desc[inst].tally_off;
        if (n_emit) atomicAdd(&T[C_EMITTED], (unsigned long long)n_emit);
        if (n_esc) atomicAdd(&T[C_ESCAPED], (unsigned long long)n_esc);
        if (n_abort) atomicAdd(&T[C_ABORTED], (unsigned long long)n_abort);
        if (n_steps) atomicAdd(&T[C_STEPS], n_steps);
        if (n_clamp) atomicAdd(&T[C_CLAMPS], (unsigned long long)n_clamp);
        if (n_edraw) atomicAdd(&T[C_EVENT_DRAWS], n_edraw);
        n_emit = n_esc = n_abort = n_clamp = 0;
        n_steps = n_edraw = 0;
    };

    auto generic = [&](unsigned w) -> bool {
        const unsigned rw = ndim == 1 ? 1u : 2u;
        const unsigned ri = min(s, nr1);
        const uint4 a = __ldg(&rows[ri * rw]);
        unsigned o = (unsigned)(w >= a.x) + (unsigned)(w >= a.y) + (unsigned)(w >= a.z);
        if (ndim == 3) {
            const uint4 b = __ldg(&rows[ri * rw + 1]);
            o += (unsigned)(w >= b.x) + (unsigned)(w >= b.y) + (unsigned)(w >= b.z) + (unsigned)(w >= b.w);
        }
        const unsigned fl = a.w;
        const unsigned act = (fl >> (2u * o)) & 3u;
        const unsigned bin = min(s - cls * J, J - 1u);
        if (o < 2u) {
            if (act == ACT_MOVE) { s += o ? 1u : 0xffffffffu; return false; }
            ++n_abort;  // a hand-off to MC: batches run the DDMC walk only
            return true;
        }
        const unsigned face = o - 2u;
        if (act == ACT_ESCAPE) {
            batch_escape(P, P.desc[inst], cell, bin, face, gid, e, (fl & FLAG_MOVING) != 0u);
            if (ndim == 3 || (fl & FLAG_MOVING)) e += 5;
            ++n_esc;
            return true;
        }
        if (act == ACT_TO_MC) { ++n_abort; return true; }
        unsigned nbin = bin;
        if (act == ACT_REBIN) {
            const Rebin rb = P.desc[inst].rebin[min(cls, ncls1) * (2u * ndim) + face];
            const unsigned w1 = event_word(gid, e++, P.k0, P.k1);
            int jn = (int)bin + rb.m + (w1 >= rb.thr ? 1 : 0);
            if (jn < 0) { jn = 0; ++n_clamp; }
            if (jn > (int)J - 1) { jn = (int)J - 1; ++n_clamp; }
            nbin = (unsigned)jn;
        }
        const unsigned ax = face >> 1;
        const unsigned stride = ax == 0 ? 1u : (ax == 1 ? n0 : n01);
        cell = min((face & 1u) ? cell + stride : cell - stride, ncell1);
        cls = __ldg(&cell_class[cell]);
        s = cls * J + nbin;
        return false;
    };

    for (;;) {
        const unsigned need = __ballot_sync(FULL, !have && !exhausted);
        if (need) {
            const int leader = __ffs(need) - 1;
            unsigned long long first = 0;
            if ((int)lane == leader) first = atomicAdd(P.cursor, (unsigned long long)__popc(need));
            first = __shfl_sync(FULL, first, leader);
            if (!have && !exhausted) {
                const unsigned long long q = first + (unsigned long long)__popc(need & ((1u << lane) - 1u));
                if (q >= P.total) {
                    exhausted = true;
                } else {
                    int lo = 0, hi = P.n_inst;  // off[lo] <= q < off[hi]
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (q >= P.off[mid]) lo = mid; else hi = mid;
                    }
                    if (lo != inst) {
                        flush();
                        inst = lo;
                        const InstDesc& D = P.desc[inst];
                        fast = D.fast; rows = D.rows; cell_class = D.cell_class;
                        J = (unsigned)D.J; nr1 = (unsigned)D.n_rows - 1u; ncell1 = (unsigned)D.ncell - 1u;
                        ncls1 = (unsigned)D.n_class - 1u; n0 = (unsigned)D.n0; n01 = (unsigned)D.n01;
                        ndim = (unsigned)D.ndim;
                    }
                    const InstDesc& D = P.desc[inst];
                    gid = D.pkt_begin + (q - P.off[inst]);
                    const unsigned w = event_word(gid, 0, P.k0, P.k1);
                    unsigned idx[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        idx[a] = (unsigned)D.src_cand[a][(D.src_ncand[a] == 2) ? ((w >> (31 - a)) & 1u) : 0u];
                    cell = min(idx[0] + n0 * idx[1] + n01 * idx[2], ncell1);
                    const unsigned bin = (unsigned)D.src_bin[(D.src_nbin == 2) ? ((w >> 28) & 1u) : 0u];
                    cls = __ldg(&cell_class[cell]);
                    s = cls * J + min(bin, J - 1u);
                    t = 0;
                    e = 1;
                    ++n_emit;
                    ++n_edraw;
                    have = true;
                }
            }
        }
        if (__all_sync(FULL, exhausted && !have)) break;
        if (!have) continue;

        unsigned long long lim = t + (unsigned long long)P.chunk;
        lim = lim < P.max_steps ? lim : P.max_steps;
        const unsigned long long t0 = t, e0 = e;
        bool fin = false;
        {
            const uint32_t pl = (uint32_t)gid, ph = (uint32_t)(gid >> 32);
            unsigned long long blk = t >> 2;
            const unsigned ng = (unsigned)((lim - t) >> 2);
            uint4 rn = bphilox(make_uint4((uint32_t)blk, (uint32_t)(blk >> 32), pl, ph), P);
            unsigned g = 0;
            while (g < ng) {
                const uint4 r = rn;
                ++blk;
                rn = bphilox(make_uint4((uint32_t)blk, (uint32_t)(blk >> 32), pl, ph), P);
                unsigned q;
                {
                    // four transitions as one branch-free chain of head loads
                    // (clamped speculative states), checked at its end, as in
                    // the single-grid walk
                    const unsigned s0 = s;
                    const uint2 f0 = __ldg(&fast[min(s0, nr1)]);
                    const unsigned s1 = s0 + ((r.x >= f0.x) ? 1u : 0xffffffffu);
                    const uint2 f1 = __ldg(&fast[min(s1, nr1)]);
                    const unsigned s2 = s1 + ((r.y >= f1.x) ? 1u : 0xffffffffu);
                    const uint2 f2 = __ldg(&fast[min(s2, nr1)]);
                    const unsigned s3 = s2 + ((r.z >= f2.x) ? 1u : 0xffffffffu);
                    const uint2 f3 = __ldg(&fast[min(s3, nr1)]);
                    const unsigned s4 = s3 + ((r.w >= f3.x) ? 1u : 0xffffffffu);
                    const bool ok0 = r.x < f0.y, ok1 = r.y < f1.y, ok2 = r.z < f2.y, ok3 = r.w < f3.y;
                    if (ok0 && ok1 && ok2 && ok3) {
                        s = s4;
                        ++g;
                        continue;
                    }
                    q = !ok0 ? 0u : (!ok1 ? 1u : (!ok2 ? 2u : 3u));
                    s = !ok0 ? s0 : (!ok1 ? s1 : (!ok2 ? s2 : s3));
                    goto slow;
                }
                ++g;
                continue;
            slow:
                for (; q < 4u; ++q) {
                    if (generic(bword(r, q))) {
                        fin = true;
                        t += 4ull * g + q + 1ull;
                        goto chunk_done;
                    }
                }
                ++g;
            }
            t += 4ull * ng;
            while (t < lim) {
                const unsigned long long b = t >> 2;
                const uint4 r = bphilox(make_uint4((uint32_t)b, (uint32_t)(b >> 32), pl, ph), P);
                const bool f = generic(bword(r, (unsigned)t & 3u));
                ++t;
                if (f) { fin = true; break; }
            }
        }
    chunk_done:
        n_steps += t - t0;
        n_edraw += e - e0;
        if (fin) {
            have = false;
        } else if (t >= P.max_steps) {
            ++n_abort;
            have = false;
        }
    }
    flush();
}

}  // namespace
}  // namespace rddmc

using namespace rddmc;

struct rddmc_batch {
    std::vector<const rddmc_grid*> grids;
    std::vector<InstDesc> desc;
    std::vector<unsigned long long> off;        // full runs
    std::vector<unsigned long long> off_trial;  // autotuner subsets
    std::vector<uint64_t> n_packets;
    uint64_t tally_words = 0, total = 0;
    uint64_t desc_bytes = 0;
    int default_ctas = 0;
};

namespace {

uint64_t off_array_bytes(size_t n_inst) { return align256((n_inst + 1) * 8ull); }

void fill_params(const rddmc_batch* b, const void* d_desc, bool trial, const rddmc_run_opts* o, void* d_scratch,
                 void* d_tallies, BatchParams& P) {
    std::memset(&P, 0, sizeof(P));
    const char* base = (const char*)d_desc;
    const size_t n = b->desc.size();
    P.desc = (const InstDesc*)base;
    const uint64_t o_full = align256(n * sizeof(InstDesc));
    P.off = (const unsigned long long*)(base + o_full + (trial ? off_array_bytes(n) : 0));
    P.n_inst = (int)n;
    P.cursor = (unsigned long long*)d_scratch;
    P.tally = (unsigned long long*)d_tallies;
    P.total = trial ? b->off_trial.back() : b->off.back();
    P.max_steps = o->max_steps ? o->max_steps : (1ull << 62);
    P.k0 = (uint32_t)o->seed;
    P.k1 = (uint32_t)(o->seed >> 32);
    for (int r = 0; r < 10; ++r) {
        P.rk0[r] = P.k0 + (uint32_t)r * 0x9E3779B9u;
        P.rk1[r] = P.k1 + (uint32_t)r * 0xBB67AE85u;
    }
    P.chunk = o->chunk ? o->chunk : 256;
}

cudaError_t enqueue(const rddmc_batch* b, const BatchParams& P, const rddmc_run_opts* o, cudaStream_t s) {
    int nsm = 0, dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int threads = o->threads_per_cta ? o->threads_per_cta : 256;
    const int ctas = o->ctas_per_sm ? o->ctas_per_sm : std::max(1, b->default_ctas);
    if ((e = cudaMemsetAsync(P.cursor, 0, 8, s)) != cudaSuccess) return e;
    batch_kernel<<<(unsigned)(ctas * nsm), threads, 0, s>>>(P);
    return cudaGetLastError();
}

// The buffers of a batched launch (the same rules for a launch, a graph and the
// autotuner's trials, checked before anything is written to them).
int check_buffers(const rddmc_batch* b, const void* d_desc, const void* d_scratch, size_t scratch_bytes,
                  const void* d_tallies, size_t tally_bytes) {
    if (!b || !d_desc || !d_scratch || !d_tallies) return RDDMC_ERR_ARG;
    if (((uintptr_t)d_desc & 255u) || ((uintptr_t)d_scratch & 7u) || ((uintptr_t)d_tallies & 7u)) return RDDMC_ERR_ARG;
    if (scratch_bytes < 256 || tally_bytes < b->tally_words * 8ull) return RDDMC_ERR_SIZE;
    return RDDMC_OK;
}

int check_opts(const rddmc_run_opts* o) {
    if (!o) return RDDMC_ERR_ARG;
    if (o->steps_per_launch != 0 || o->resume != 0 || o->time_slice_us != 0) return RDDMC_ERR_UNSUPPORTED;
    if (o->chunk < 0 || o->chunk % 4 != 0 || o->ctas_per_sm < 0 || o->threads_per_cta < 0) return RDDMC_ERR_ARG;
    if (o->threads_per_cta && (o->threads_per_cta % 32 != 0 || o->threads_per_cta > 256)) return RDDMC_ERR_ARG;
    return RDDMC_OK;
}

}  // namespace

extern "C" {

int rddmc_batch_create(const rddmc_grid* const* grids, const void* const* d_tables, const uint64_t* n_packets,
                       int n_inst, rddmc_batch** out) {
    if (!grids || !d_tables || !n_packets || !out || n_inst < 1 || n_inst > (1 << 20)) return RDDMC_ERR_ARG;
    *out = nullptr;
    rddmc_batch* b = new (std::nothrow) rddmc_batch();
    if (!b) return RDDMC_ERR_ARG;
    b->off.push_back(0);
    b->off_trial.push_back(0);
    uint64_t tw = 0;
    for (int i = 0; i < n_inst; ++i) {
        const rddmc_grid* g = grids[i];
        if (!g || !d_tables[i] || ((uintptr_t)d_tables[i] & 255u) || n_packets[i] == 0 ||
            n_packets[i] >= (1ull << 62) - b->off.back()) {  // global packet ids stay below 2^62
            delete b;
            return RDDMC_ERR_ARG;
        }
        if (!g->precomputed) { delete b; return RDDMC_ERR_TABLE; }
        if (g->params.mode != RDDMC_MODE_DDMC || g->dusty() || g->weighted()) { delete b; return RDDMC_ERR_UNSUPPORTED; }
        const char* tb = (const char*)d_tables[i];
        InstDesc D;
        std::memset(&D, 0, sizeof(D));
        D.rows = (const uint4*)(tb + g->off_rows);
        D.fast = (const uint2*)(tb + g->off_fast);
        D.cell_class = (const uint32_t*)(tb + g->off_class);
        D.rebin = (const Rebin*)(tb + g->off_rebin);
        D.edges = (const double*)(tb + g->off_edges);
        D.cell_v = (const double*)(tb + g->off_vel);
        D.tally_off = tw;
        D.pkt_begin = b->off.back();
        D.R = g->R;
        for (int a = 0; a < 3; ++a) D.dz[a] = 2.0 * g->R / g->n[a];
        D.vth = g->vth;
        D.J = g->J; D.n_rows = g->n_class * g->J; D.n_class = g->n_class; D.ncell = (int)g->ncell;
        D.n0 = g->n[0]; D.n1 = g->n[1]; D.n01 = g->n[0] * g->n[1]; D.ndim = g->ndim; D.moving = g->moving ? 1 : 0;
        for (int a = 0; a < 3; ++a) {
            D.src_ncand[a] = g->src_ncand[a];
            D.src_cand[a][0] = g->src_cand[a][0];
            D.src_cand[a][1] = g->src_cand[a][1];
        }
        D.src_nbin = g->src_nbin; D.src_bin[0] = g->src_bin[0]; D.src_bin[1] = g->src_bin[1];
        b->desc.push_back(D);
        b->grids.push_back(g);
        b->n_packets.push_back(n_packets[i]);
        tw += (uint64_t)tally_words(g->J);
        b->off.push_back(b->off.back() + n_packets[i]);
    }
    b->tally_words = tw;
    b->total = b->off.back();
    b->desc_bytes = align256(b->desc.size() * sizeof(InstDesc)) + 2 * off_array_bytes(b->desc.size());
    int ctas = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas, batch_kernel, 256, 0) != cudaSuccess) ctas = 1;
    b->default_ctas = std::max(1, ctas);
    *out = b;
    return RDDMC_OK;
}

void rddmc_batch_destroy(rddmc_batch* b) { delete b; }

int rddmc_batch_sizes(const rddmc_batch* b, uint64_t* desc_bytes, uint64_t* tally_bytes, uint64_t* scratch_bytes,
                      uint64_t* total_packets) {
    if (!b) return RDDMC_ERR_ARG;
    if (desc_bytes) *desc_bytes = b->desc_bytes;
    if (tally_bytes) *tally_bytes = b->tally_words * 8ull;
    if (scratch_bytes) *scratch_bytes = 256;
    if (total_packets) *total_packets = b->total;
    return RDDMC_OK;
}

int rddmc_batch_upload(rddmc_batch* b, double trial_fraction, void* d_desc, size_t desc_bytes, void* stream) {
    if (!b || !d_desc || ((uintptr_t)d_desc & 255u)) return RDDMC_ERR_ARG;
    if (desc_bytes < b->desc_bytes) return RDDMC_ERR_SIZE;
    if (!(trial_fraction > 0.0 && trial_fraction <= 1.0)) return RDDMC_ERR_ARG;
    b->off_trial.assign(1, 0);
    for (size_t i = 0; i < b->desc.size(); ++i) {
        const uint64_t n = std::max<uint64_t>(1, (uint64_t)std::ceil((double)b->n_packets[i] * trial_fraction));
        b->off_trial.push_back(b->off_trial.back() + std::min(n, b->n_packets[i]));
    }
    cudaStream_t s = (cudaStream_t)stream;
    char* base = (char*)d_desc;
    const size_t n = b->desc.size();
    const uint64_t o_full = align256(n * sizeof(InstDesc));
    cudaError_t e = cudaMemcpyAsync(base, b->desc.data(), n * sizeof(InstDesc), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_full, b->off.data(), (n + 1) * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + o_full + off_array_bytes(n), b->off_trial.data(), (n + 1) * 8,
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? RDDMC_OK : RDDMC_ERR_CUDA;
}

int rddmc_batch_launch(const rddmc_batch* b, const void* d_desc, const rddmc_run_opts* o, int trial, void* d_scratch,
                       size_t scratch_bytes, void* d_tallies, size_t tally_bytes, void* stream) {
    int rc = check_buffers(b, d_desc, d_scratch, scratch_bytes, d_tallies, tally_bytes);
    if (rc != RDDMC_OK) return rc;
    rc = check_opts(o);
    if (rc != RDDMC_OK) return rc;
    BatchParams P;
    fill_params(b, d_desc, trial != 0, o, d_scratch, d_tallies, P);
    return enqueue(b, P, o, (cudaStream_t)stream) == cudaSuccess ? RDDMC_OK : RDDMC_ERR_CUDA;
}

int rddmc_batch_read_tallies(const rddmc_batch* b, const void* d_tallies, int inst, rddmc_tallies* out, uint64_t* hist,
                             uint64_t* faces, uint64_t* sb, void* stream) {
    if (!b || !d_tallies || !out || inst < 0 || inst >= (int)b->desc.size()) return RDDMC_ERR_ARG;
    return rddmc_read_tallies(b->grids[inst], (const uint64_t*)d_tallies + b->desc[inst].tally_off, out, hist, faces,
                              sb, stream);
}

// Build a CUDA graph of {zero the tallies, launch the batch} on `stream` and
// instantiate it; replay with rddmc_batch_graph_launch.
int rddmc_batch_graph_create(const rddmc_batch* b, const void* d_desc, const rddmc_run_opts* o, void* d_scratch,
                             size_t scratch_bytes, void* d_tallies, size_t tally_bytes, void* stream,
                             void** graph_exec) {
    if (!graph_exec) return RDDMC_ERR_ARG;
    *graph_exec = nullptr;
    int rc = check_buffers(b, d_desc, d_scratch, scratch_bytes, d_tallies, tally_bytes);
    if (rc != RDDMC_OK) return rc;
    rc = check_opts(o);
    if (rc != RDDMC_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (!s) return RDDMC_ERR_ARG;  // the legacy default stream cannot be captured
    BatchParams P;
    fill_params(b, d_desc, false, o, d_scratch, d_tallies, P);
    int nsm = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return RDDMC_ERR_CUDA;
    const int threads = o->threads_per_cta ? o->threads_per_cta : 256;
    const int ctas = o->ctas_per_sm ? o->ctas_per_sm : std::max(1, b->default_ctas);
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return RDDMC_ERR_CUDA;
    cudaMemsetAsync(d_tallies, 0, b->tally_words * 8ull, s);
    cudaMemsetAsync(d_scratch, 0, 8, s);
    batch_kernel<<<(unsigned)(ctas * nsm), threads, 0, s>>>(P);
    const cudaError_t le = cudaGetLastError();
    const cudaError_t ce = cudaStreamEndCapture(s, &graph);
    if (le != cudaSuccess || ce != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        return RDDMC_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return RDDMC_ERR_CUDA;
    *graph_exec = (void*)exec;
    return RDDMC_OK;
}

int rddmc_batch_graph_launch(void* graph_exec, void* stream) {
    if (!graph_exec) return RDDMC_ERR_ARG;
    return cudaGraphLaunch((cudaGraphExec_t)graph_exec, (cudaStream_t)stream) == cudaSuccess ? RDDMC_OK
                                                                                               : RDDMC_ERR_CUDA;
}

void rddmc_batch_graph_destroy(void* graph_exec) {
    if (graph_exec) cudaGraphExecDestroy((cudaGraphExec_t)graph_exec);
}

// Time every candidate schedule on the trial subset (trial_fraction of each
// instance's packets, set by rddmc_batch_upload) with CUDA events and return
// the one with the highest transitions/s in *best.  A trial walks each of its
// packets for at most kTrialSteps transitions (or base->max_steps if lower):
// it measures the schedule's throughput on the run's own instances while the
// GPU is full, not the time to the last escape, so a run without a watchdog
// is tuned in a bounded time.  Clobbers d_tallies.
constexpr unsigned long long kTrialSteps = 1ull << 16;  // transitions per trial packet

int rddmc_batch_autotune(const rddmc_batch* b, const void* d_desc, const rddmc_run_opts* base, void* d_scratch,
                         size_t scratch_bytes, void* d_tallies, size_t tally_bytes, void* stream,
                         rddmc_run_opts* best, double* best_rate) {
    if (!b || !base || !best) return RDDMC_ERR_ARG;
    // every trial zeroes and reads the whole tally buffer: check it first
    int rc = check_buffers(b, d_desc, d_scratch, scratch_bytes, d_tallies, tally_bytes);
    if (rc != RDDMC_OK) return rc;
    rc = check_opts(base);
    if (rc != RDDMC_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int threads_c[] = {128, 256};
    const int chunk_c[] = {64, 256, 1024};
    int occ128 = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ128, batch_kernel, 128, 0) != cudaSuccess) occ128 = 6;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return RDDMC_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return RDDMC_ERR_CUDA; }
    double best_r = -1.0;
    rddmc_run_opts bo = *base;
    for (int th : threads_c) {
        const int occ = th == 128 ? std::max(1, occ128) : std::max(1, b->default_ctas);
        for (int ctas : {occ, std::max(1, occ - 1)}) {
            for (int ch : chunk_c) {
                rddmc_run_opts o = *base;
                o.max_steps = (base->max_steps && base->max_steps < kTrialSteps) ? base->max_steps : kTrialSteps;
                o.threads_per_cta = th;
                o.ctas_per_sm = ctas;
                o.chunk = ch;
                if (cudaMemsetAsync(d_tallies, 0, b->tally_words * 8ull, s) != cudaSuccess) { rc = RDDMC_ERR_CUDA; break; }
                cudaEventRecord(e0, s);
                rc = rddmc_batch_launch(b, d_desc, &o, 1, d_scratch, scratch_bytes, d_tallies, tally_bytes, stream);
                cudaEventRecord(e1, s);
                if (rc != RDDMC_OK) break;
                if (cudaEventSynchronize(e1) != cudaSuccess) { rc = RDDMC_ERR_CUDA; break; }
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                std::vector<uint64_t> t(b->tally_words);
                if (cudaMemcpy(t.data(), d_tallies, t.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
                    rc = RDDMC_ERR_CUDA;
                    break;
                }
                uint64_t steps = 0;
                for (const InstDesc& D : b->desc) steps += t[D.tally_off + C_STEPS];
                const double r = ms > 0.0f ? (double)steps / (ms * 1e-3) : 0.0;
                if (r > best_r) { best_r = r; bo = o; }
            }
            if (rc != RDDMC_OK) break;
        }
        if (rc != RDDMC_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != RDDMC_OK) return rc;
    bo.max_steps = base->max_steps;  // the trials' transition cap is not the run's watchdog
    *best = bo;
    if (best_rate) *best_rate = best_r;
    return RDDMC_OK;
}

}  // extern "C"
