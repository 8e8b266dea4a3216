// walk.cu -- persistent DDMC walk kernel (Sec. 2.4) for slabs.
//
// One packet per thread.  A transition draws one 32-bit word of the packet's
// transition stream (lane t&3 of Philox4x32-10 keyed by (t>>2, packet); every
// lane's t stays a multiple of 4 at a refill, so a warp makes one Philox call
// per four transitions without divergence), gathers the 16-byte row
// {thr0, thr1, thr2, flags} of its state (cell class, bin) and takes outcome
// o = #{k : w >= thr_k}: the categorical form of the competing exponentials of
// eq. l_min_1/2.  Outcomes are bin-1, bin+1, cell-1, cell+1; the 2-bit action
// of the outcome selects a plain move (the fast path) or the slow path
// (escape through an exterior face, Doppler rebin across a face).
//
// Lanes whose packet escaped, was aborted by the watchdog or reached the end of
// its time slice take new packet ids from a global cursor, one atomicAdd per
// warp (__ballot_sync / __popc prefix).  Tallies are integer: per-thread
// registers for counters, warp-aggregated (__match_any_sync) shared-memory
// atomics for the escape histogram and faces, flushed to the u64 tally buffer
// in global memory when the CTA finishes.
#include <cstring>

#include "grid.h"

namespace rddmc {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kSmemHistMax = 8192;  // histogram entries kept in shared memory

struct SlabWalkParams {
    const uint4* rows;
    const uint32_t* cell_class;
    const Rebin* rebin;
    const ClassDesc* cdesc;
    const double* edges;
    unsigned long long* cursor;
    uint32_t* st_cell;
    uint32_t* st_bin;
    unsigned long long* st_t;
    unsigned long long* st_e;
    uint8_t* st_status;
    unsigned long long* tally;
    unsigned long long n_packets, max_steps, slice;
    uint32_t k0, k1;
    int J, n_rows, ncell, chunk;
    int resume, save_state, hist_in_smem;
    int src_ncell, src_cell0, src_cell1, src_nbin, src_bin0, src_bin1;
};

// Shared-memory tally update aggregated over the lanes that hit the same index.
__device__ __forceinline__ void smem_tally(unsigned long long* s, unsigned idx) {
    const unsigned active = __activemask();
    const unsigned peers = __match_any_sync(active, idx);
    const int leader = __ffs(peers) - 1;
    if ((int)(threadIdx.x & 31) == leader) atomicAdd(&s[idx], (unsigned long long)__popc(peers));
}

// Observer-frame escape bin of a packet leaving a moving cell through face
// (axis 0, side): a point on the face (two draws, unused by a slab), an
// isotropic outward direction (mu uniform on (0,1], azimuth uniform), x uniform
// in the bin; x_obs = x + n.u (FP64).  Returns the histogram index.
__device__ __noinline__ int moving_escape_bin(const SlabWalkParams& P, const ClassDesc& D, unsigned bin, int side,
                                 unsigned long long pid, unsigned long long& e) {
    (void)event_word(pid, e++, P.k0, P.k1);
    (void)event_word(pid, e++, P.k0, P.k1);
    const double inv = 1.0 / 4294967296.0;
    const double mu = 1.0 - ((double)event_word(pid, e++, P.k0, P.k1) + 0.5) * inv;
    const double ph = 2.0 * 3.14159265358979323846 * (((double)event_word(pid, e++, P.k0, P.k1) + 0.5) * inv);
    const double xu = ((double)event_word(pid, e++, P.k0, P.k1) + 0.5) * inv;
    const double x = P.edges[bin] + xu * (P.edges[bin + 1] - P.edges[bin]);
    const double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    const double nu = (double)side * mu * D.u[0] + st * (cos(ph) * D.u[1] + sin(ph) * D.u[2]);
    const double xo = x + nu;
    if (xo < P.edges[0]) return 0;
    if (xo >= P.edges[P.J]) return P.J + 1;
    int lo = 0, hi = P.J;  // find j with edges[j] <= xo < edges[j+1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (xo >= P.edges[mid]) lo = mid; else hi = mid;
    }
    return lo + 1;
}

template <bool SMEM_ROWS>
__global__ void __launch_bounds__(256, 3) slab_walk_kernel(const SlabWalkParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long* s_cnt = reinterpret_cast<unsigned long long*>(smem_raw);  // kCounters
    unsigned long long* s_face = s_cnt + kCounters;                              // 8
    unsigned long long* s_hist = s_face + 8;                                      // J+2 if in smem
    const int nhist = P.J + 2;
    uint4* s_rows = reinterpret_cast<uint4*>(s_hist + (P.hist_in_smem ? ((nhist + 1) & ~1) : 0));

    for (int i = threadIdx.x; i < kCounters + 8; i += blockDim.x) s_cnt[i] = 0ull;
    if (P.hist_in_smem)
        for (int i = threadIdx.x; i < nhist; i += blockDim.x) s_hist[i] = 0ull;
    if (SMEM_ROWS)
        for (int i = threadIdx.x; i < P.n_rows; i += blockDim.x) s_rows[i] = __ldg(&P.rows[i]);
    __syncthreads();

    const unsigned lane = threadIdx.x & 31u;
    const int J = P.J;
    bool have = false, exhausted = false;
    unsigned long long pid = 0, t = 0, e = 0, t_stop = 0;
    unsigned cell = 0, bin = 0, cls = 0, base = 0;
    unsigned long long n_steps = 0, n_edraw = 0;
    unsigned n_emit = 0, n_esc = 0, n_abort = 0, n_clamp = 0, status_bits = 0;

    for (;;) {
        // ---- warp-cooperative refill
        const unsigned need = __ballot_sync(FULL, !have && !exhausted);
        if (need) {
            const int leader = __ffs(need) - 1;
            unsigned long long first = 0;
            if ((int)lane == leader) first = atomicAdd(P.cursor, (unsigned long long)__popc(need));
            first = __shfl_sync(FULL, first, leader);
            if (!have && !exhausted) {
                pid = first + (unsigned long long)__popc(need & ((1u << lane) - 1u));
                if (pid >= P.n_packets) {
                    exhausted = true;
                } else {
                    const uint8_t st = P.resume ? P.st_status[pid] : (uint8_t)PK_FRESH;
                    if (st == PK_INFLIGHT) {
                        cell = P.st_cell[pid];
                        bin = P.st_bin[pid];
                        t = P.st_t[pid];
                        e = P.st_e[pid];
                        have = true;
                    } else if (st == PK_FRESH) {
                        // event draw 0: bit 31 picks the centre cell, bit 28 the bin
                        const unsigned w = event_word(pid, 0, P.k0, P.k1);
                        cell = (P.src_ncell == 2 && ((w >> 31) & 1u)) ? P.src_cell1 : P.src_cell0;
                        bin = (P.src_nbin == 2 && ((w >> 28) & 1u)) ? P.src_bin1 : P.src_bin0;
                        t = 0;
                        e = 1;
                        ++n_emit;
                        have = true;
                    }
                    if (have) {
                        cell = min(cell, (unsigned)P.ncell - 1u);
                        bin = min(bin, (unsigned)J - 1u);
                        cls = __ldg(&P.cell_class[cell]);
                        base = cls * (unsigned)J;
                        t_stop = P.slice ? t + P.slice : ~0ull;
                    }
                }
            }
        }
        if (__all_sync(FULL, exhausted && !have)) break;
        if (!have) continue;

        // ---- run up to `chunk` transitions
        unsigned long long lim = t + (unsigned long long)P.chunk;
        lim = lim < t_stop ? lim : t_stop;
        lim = lim < P.max_steps ? lim : P.max_steps;
        const unsigned long long t0 = t;
        const unsigned long long e0 = e;
        bool fin = false;
        while (t < lim) {
            const unsigned long long blk = t >> 2;
            const uint4 r = philox4x32_10(make_uint4((uint32_t)blk, (uint32_t)(blk >> 32), (uint32_t)pid,
                                                     (uint32_t)(pid >> 32)),
                                          P.k0, P.k1);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const unsigned w = q == 0 ? r.x : (q == 1 ? r.y : (q == 2 ? r.z : r.w));
                // every index below is clamped into its buffer, so no table content
                // can send a read or a tally outside its array
                const unsigned ri = min(base + bin, (unsigned)P.n_rows - 1u);
                const uint4 row = SMEM_ROWS ? s_rows[ri] : __ldg(&P.rows[ri]);
                const unsigned o = (unsigned)(w >= row.x) + (unsigned)(w >= row.y) + (unsigned)(w >= row.z);
                const unsigned act = (row.w >> (2u * o)) & 3u;
                ++t;
                if (act == ACT_MOVE) {
                    if (o < 2u) {
                        bin = bin + 2u * o - 1u;
                    } else {
                        cell = min(cell + 2u * (o - 2u) - 1u, (unsigned)P.ncell - 1u);
                        cls = __ldg(&P.cell_class[cell]);
                        base = cls * (unsigned)J;
                    }
                } else if (act == ACT_REBIN) {
                    const int face = (int)o - 2;
                    const Rebin rb = P.rebin[min(cls, (unsigned)P.n_rows / (unsigned)J - 1u) * 2u + (unsigned)face];
                    const unsigned w1 = event_word(pid, e++, P.k0, P.k1);
                    int jn = (int)bin + rb.m + (w1 >= rb.thr ? 1 : 0);
                    if (jn < 0) { jn = 0; ++n_clamp; }
                    if (jn > J - 1) { jn = J - 1; ++n_clamp; }
                    bin = (unsigned)jn;
                    cell = min(cell + 2u * (o - 2u) - 1u, (unsigned)P.ncell - 1u);
                    cls = __ldg(&P.cell_class[cell]);
                    base = cls * (unsigned)J;
                } else if (act == ACT_ESCAPE) {
                    const int face = (int)o - 2;
                    int h = (int)min(bin, (unsigned)J - 1u) + 1;
                    if (row.w & FLAG_MOVING)
                        h = moving_escape_bin(P, P.cdesc[min(cls, (unsigned)P.n_rows / (unsigned)J - 1u)],
                                              min(bin, (unsigned)J - 1u), face ? 1 : -1, pid, e);
                    if (P.hist_in_smem) smem_tally(s_hist, (unsigned)h);
                    else atomicAdd(&P.tally[kHistOff + h], 1ull);
                    smem_tally(s_face, (unsigned)face);
                    ++n_esc;
                    fin = true;
                } else {
                    // hand-off to continuous MC: not available in this walk
                    status_bits |= (unsigned)STATUS_UNSUPPORTED_EVENT;
                    ++n_abort;
                    fin = true;
                }
                if (fin || t >= lim) break;
            }
            if (fin) break;
        }
        n_steps += t - t0;
        n_edraw += e - e0;
        if (fin) {
            have = false;
            if (P.save_state) P.st_status[pid] = PK_DONE;
        } else if (t >= P.max_steps) {
            ++n_abort;
            have = false;
            if (P.save_state) P.st_status[pid] = PK_DONE;
        } else if (t >= t_stop) {
            P.st_cell[pid] = cell;
            P.st_bin[pid] = bin;
            P.st_t[pid] = t;
            P.st_e[pid] = e;
            P.st_status[pid] = PK_INFLIGHT;
            have = false;
        }
    }

    // ---- flush: warp sums of the per-thread counters, then CTA totals to HBM
    n_edraw += n_emit;  // the source draw of each emitted packet
    unsigned long long v[7] = {n_emit, n_esc, n_abort, n_steps, n_clamp, n_edraw, status_bits};
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        unsigned long long x = v[i];
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(FULL, x, off);
        v[i] = x;
    }
    if (lane == 0) {
        atomicAdd(&s_cnt[C_EMITTED], v[0]);
        atomicAdd(&s_cnt[C_ESCAPED], v[1]);
        atomicAdd(&s_cnt[C_ABORTED], v[2]);
        atomicAdd(&s_cnt[C_STEPS], v[3]);
        atomicAdd(&s_cnt[C_CLAMPS], v[4]);
        atomicAdd(&s_cnt[C_EVENT_DRAWS], v[5]);
        if (v[6]) atomicOr(&s_cnt[C_STATUS_BITS], v[6]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kCounters; i += blockDim.x) {
        if (!s_cnt[i]) continue;
        if (i == C_STATUS_BITS) atomicOr(&P.tally[i], s_cnt[i]);
        else atomicAdd(&P.tally[i], s_cnt[i]);
    }
    for (int i = threadIdx.x; i < 2; i += blockDim.x)
        if (s_face[i]) atomicAdd(&P.tally[kFaceOff + i], s_face[i]);
    if (P.hist_in_smem)
        for (int i = threadIdx.x; i < nhist; i += blockDim.x)
            if (s_hist[i]) atomicAdd(&P.tally[kHistOff + i], s_hist[i]);
}

}  // namespace

cudaError_t launch_walk(const rddmc_grid& g, const WalkLaunch& w, cudaStream_t s) {
    const rddmc_run_opts& o = w.opts;
    const char* tb = (const char*)w.d_table;
    char* sb = (char*)w.d_state;
    SlabWalkParams P;
    std::memset(&P, 0, sizeof(P));
    P.rows = (const uint4*)(tb + g.off_rows);
    P.cell_class = (const uint32_t*)(tb + g.off_class);
    P.rebin = (const Rebin*)(tb + g.off_rebin);
    P.cdesc = (const ClassDesc*)(tb + g.off_cdesc);
    P.edges = (const double*)(tb + g.off_edges);
    const uint64_t np = o.n_packets;
    uint64_t off = 256;
    P.cursor = (unsigned long long*)sb;
    P.st_cell = (uint32_t*)(sb + off); off += align256(np * 4);
    P.st_bin = (uint32_t*)(sb + off); off += align256(np * 4);
    P.st_t = (unsigned long long*)(sb + off); off += align256(np * 8);
    P.st_e = (unsigned long long*)(sb + off); off += align256(np * 8);
    P.st_status = (uint8_t*)(sb + off);
    P.tally = w.d_tally;
    P.n_packets = np;
    P.max_steps = o.max_steps ? o.max_steps : (1ull << 62);
    P.slice = o.steps_per_launch;
    P.k0 = (uint32_t)o.seed;
    P.k1 = (uint32_t)(o.seed >> 32);
    P.J = g.J;
    P.n_rows = g.n_class * g.J;
    P.ncell = (int)g.ncell;
    P.chunk = o.chunk ? o.chunk : 64;
    P.resume = o.resume;
    P.save_state = (o.steps_per_launch != 0 || o.resume) ? 1 : 0;
    P.hist_in_smem = (g.J + 2 <= kSmemHistMax) ? 1 : 0;
    P.src_ncell = g.src_ncand[0];
    P.src_cell0 = g.src_cand[0][0];
    P.src_cell1 = g.src_cand[0][1];
    P.src_nbin = g.src_nbin;
    P.src_bin0 = g.src_bin[0];
    P.src_bin1 = g.src_bin[1];

    int dev = 0, nsm = 0, smem_optin = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
        return e;
    const int threads = o.threads_per_cta ? o.threads_per_cta : 256;
    size_t smem = (size_t)(kCounters + 8) * 8;
    if (P.hist_in_smem) smem += (size_t)((g.J + 2 + 1) & ~1) * 8;
    const size_t rows_bytes = (size_t)P.n_rows * 16;
    const bool use_smem_rows = o.table_in_smem && smem + rows_bytes <= (size_t)smem_optin;
    if (use_smem_rows) smem += rows_bytes;
    int ctas = o.ctas_per_sm;
    if (use_smem_rows) {
        if ((e = cudaFuncSetAttribute(slab_walk_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess)
            return e;
        if (!ctas && (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas, slab_walk_kernel<true>, threads,
                                                                        smem)) != cudaSuccess)
            return e;
    } else {
        if ((e = cudaFuncSetAttribute(slab_walk_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess)
            return e;
        if (!ctas && (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas, slab_walk_kernel<false>, threads,
                                                                        smem)) != cudaSuccess)
            return e;
    }
    if (ctas < 1) ctas = 1;
    if ((e = cudaMemsetAsync(P.cursor, 0, 8, s)) != cudaSuccess) return e;
    const unsigned blocks = (unsigned)(ctas * nsm);
    if (use_smem_rows)
        slab_walk_kernel<true><<<blocks, threads, smem, s>>>(P);
    else
        slab_walk_kernel<false><<<blocks, threads, smem, s>>>(P);
    return cudaGetLastError();
}

}  // namespace rddmc
