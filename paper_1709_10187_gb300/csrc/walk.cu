// walk.cu -- persistent DDMC walk kernel (Sec. 2.3) for slabs and 3D grids.
//
// One packet per thread.  A transition draws one 32-bit word of the packet's
// transition stream (lane t&3 of Philox4x32-10 keyed by (t>>2, packet); every
// lane's t is a multiple of 4 when a chunk starts, so a warp makes one Philox
// call per four transitions without divergence, and the call for the next four
// is issued while the current four are walked).  The word w selects outcome
// o = #{k : w >= thr_k} of the state's row: the categorical form of the
// competing exponentials of eq. l_min_1/2.
//
// Frequency moves dominate (the core of the line, Sec. 4.2), so the fast path
// reads only the state's 8-byte fast head {thr0, thr1 or 0} (through L1, or
// staged in shared memory): when w < thr1 the packet moves one bin down
// (w < thr0) or up.  A group of four transitions runs as one branch-free chain
// of head loads, checked at its end.
// Everything else -- spatial moves, Doppler rebins, escapes through exterior
// faces, and frequency outcomes that are not plain moves (their head holds 0)
// -- goes through one generic step that reads the full row (through L1) and
// evaluates every threshold and the outcome's 2-bit action.
//
// Lanes whose packet escaped, was aborted by the watchdog or reached the end of
// its time slice take new packet ids from a global cursor, one atomicAdd per
// warp (__ballot_sync / __popc prefix).  Tallies are integer: per-thread
// registers for counters, warp-aggregated (__match_any_sync) shared-memory
// atomics for the escape histograms and faces, flushed to the u64 tally buffer
// in global memory when the CTA finishes.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "grid.h"
#include "learned_common.cuh"
#include "mc.cuh"
#include "walk_common.cuh"

namespace rddmc {
namespace {

// weight method: -ln(1e-10) in 2^-40 units, the elimination weight of Sec. 2.6
constexpr unsigned long long kLwMin = 25317190836906ull;

#ifndef RDDMC_WALK_MIN_BLOCKS
#define RDDMC_WALK_MIN_BLOCKS 4  // resident 256-thread CTAs per SM the register budget targets
#endif

// ---------------------------------------------------------------- hybrid MC
// Continuous MC of a packet in thin states (Sec. 5.1, Sec. 5.2), in FP32.  It
// runs from a DDMC hand-off until the packet converts back to DDMC, escapes or
// meets the event watchdog; time slices only count DDMC transitions, so an
// excursion always finishes within the transition that started it.
struct McResult {
    int status;            // 0 back to DDMC at (cell, bin), 1 escaped, 2 aborted
    unsigned cell, bin;
    int hist, sb, face;    // escape tallies
};

struct McPacket {
    int idx[3];
    unsigned cell;
    float r[3], n[3], x;
    int bin;  // frequency grouping: the bin of x when known, else -1
};

__device__ __forceinline__ int bin_of(const WalkParams& P, float xf) {
    const double x = (double)xf;
    if (x < P.edges[0]) return -1;
    if (x >= P.edges[P.J]) return P.J;
    int lo = 0, hi = P.J;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (x >= P.edges[mid]) lo = mid; else hi = mid;
    }
    return lo;
}

template <int NDIM>
__device__ __forceinline__ bool thick_state(const WalkParams& P, unsigned cell, int j) {
    if (j < 0 || j >= P.J) return false;
    const unsigned cls = min(__ldg(&P.cell_class[min(cell, (unsigned)P.ncell - 1u)]), (unsigned)P.n_class - 1u);
    const uint4 a = __ldg(&P.rows[(cls * (unsigned)P.J + (unsigned)j) * (NDIM == 1 ? 1u : 2u)]);
    return (a.w & FLAG_THIN) == 0u;
}

__device__ __forceinline__ float cell_u(const WalkParams& P, unsigned cell, int a) {
    return P.moving ? (float)(P.cell_v[3ull * cell + a] / P.vth) : 0.0f;
}

template <int NDIM>
__device__ __forceinline__ float face_coord(const WalkParams& P, int ax, int i) {
    return (float)(-P.R + (double)i * P.dz[ax]);
}

template <int NDIM>
__device__ void mc_escape_bins(const WalkParams& P, const McPacket& m, int ax, int side, McResult& res) {
    const float xo = m.x + m.n[0] * cell_u(P, m.cell, 0) + m.n[1] * cell_u(P, m.cell, 1) +
                     m.n[2] * cell_u(P, m.cell, 2);
    const int b = bin_of(P, xo);
    res.status = 1;
    res.hist = b < 0 ? 0 : (b >= P.J ? P.J + 1 : b + 1);
    res.face = 2 * ax + (side > 0 ? 1 : 0);
    res.sb = -1;
    if (NDIM == 3) {
        const float rr = m.r[0] * m.r[0] + m.r[1] * m.r[1] + m.r[2] * m.r[2];
        const float rn = m.r[0] * m.n[0] + m.r[1] * m.n[1] + m.r[2] * m.n[2];
        const float b2 = sqrtf(fmaxf(0.0f, rr - rn * rn)) / (float)P.R;
        res.sb = min((int)(b2 / (float)kSbMax * kNsb), kNsb - 1);
    }
}

// Cross from m's cell through face (ax, side): escape, continue into a thin
// neighbour, convert into a thick neighbour with probability
// 2/(tau + 2 lambda) (2/3 + mu), or reflect (random point on the face,
// isotropic inward direction; a reflection into a thick state converts).
// Returns true when the excursion ends (res filled).
template <int NDIM>
__device__ bool mc_cross(const WalkParams& P, McPacket& m, int ax, int side, EventStream& es, unsigned& n_conv,
                         McResult& res) {
    int nidx[3] = {m.idx[0], m.idx[1], m.idx[2]};
    nidx[ax] += side;
    bool inside = nidx[ax] >= 0 && nidx[ax] < P.n[ax];
    unsigned nb = 0;
    if (inside) {
        nb = (unsigned)nidx[0] + (unsigned)P.n0 * (unsigned)nidx[1] + (unsigned)P.n01 * (unsigned)nidx[2];
        inside = __ldg(&P.cell_class[min(nb, (unsigned)P.ncell - 1u)]) != 0xffffffffu;
    }
    if (!inside) { mc_escape_bins<NDIM>(P, m, ax, side, res); return true; }
    float xn = m.x;
    if (P.moving)
        xn += m.n[0] * (cell_u(P, m.cell, 0) - cell_u(P, nb, 0)) + m.n[1] * (cell_u(P, m.cell, 1) - cell_u(P, nb, 1)) +
              m.n[2] * (cell_u(P, m.cell, 2) - cell_u(P, nb, 2));
    const int jn = bin_of(P, xn);
    if (!thick_state<NDIM>(P, nb, jn)) {
        m.idx[ax] = nidx[ax];
        m.cell = nb;
        m.x = xn;
        return false;
    }
    const unsigned clsn = min(__ldg(&P.cell_class[nb]), (unsigned)P.n_class - 1u);
    const float tau = P.tau_row[clsn * (unsigned)P.J + (unsigned)jn];
    const float prob = 2.0f / (tau + 2.0f * P.lambda) * (0.6666667f + fabsf(m.n[ax]));
    if (es.u01() < prob) {
        ++n_conv;
        res.status = 0; res.cell = nb; res.bin = (unsigned)jn;
        return true;
    }
    const int t1 = (ax + 1) % 3, t2 = (ax + 2) % 3;
    const float p1 = es.u01(), p2 = es.u01();
    if (t1 < NDIM) m.r[t1] = (float)(-P.R + ((double)m.idx[t1] + p1) * P.dz[t1]);
    if (t2 < NDIM) m.r[t2] = (float)(-P.R + ((double)m.idx[t2] + p2) * P.dz[t2]);
    half_dir(es, ax, -side, m.n);
    const int j = bin_of(P, m.x);
    if (thick_state<NDIM>(P, m.cell, j)) {
        ++n_conv;
        res.status = 0; res.cell = m.cell; res.bin = (unsigned)j;
        return true;
    }
    return false;
}

// DDMC hand-off at (cell, bin) and the MC excursion that follows.  face >= 0:
// a leak into a thin neighbour through that face (random point on the face,
// isotropic outward direction, x uniform in bin, then the crossing); face < 0:
// a leak into the thin bin `bin` of the same cell, or a thin source state
// (random point in the cell, isotropic direction, x uniform in bin).
template <int NDIM>
__device__ __noinline__ McResult mc_excursion(const WalkParams& P, unsigned cell, unsigned bin, int face,
                                              unsigned long long pid, unsigned long long& e,
                                              unsigned long long& n_mc, unsigned& n_conv) {
    EventStream es;
    es.init(pid, e, P.k0, P.k1);
    McPacket m;
    m.cell = cell;
    m.idx[0] = (int)(cell % (unsigned)P.n0);
    m.idx[1] = NDIM == 3 ? (int)((cell / (unsigned)P.n0) % (unsigned)P.n[1]) : 0;
    m.idx[2] = NDIM == 3 ? (int)(cell / (unsigned)P.n01) : 0;
    m.r[0] = m.r[1] = m.r[2] = 0.0f;
    m.bin = (int)bin;
    McResult res;
    res.status = 2; res.cell = cell; res.bin = bin; res.hist = 0; res.sb = -1; res.face = 0;
    ++n_conv;
    bool done = false;
    if (face >= 0) {
        const int ax = face >> 1, side = (face & 1) ? 1 : -1;
        const int t1 = (ax + 1) % 3, t2 = (ax + 2) % 3;
        m.r[ax] = face_coord<NDIM>(P, ax, m.idx[ax] + (side > 0 ? 1 : 0));
        const float p1 = es.u01(), p2 = es.u01();
        if (t1 < NDIM) m.r[t1] = (float)(-P.R + ((double)m.idx[t1] + p1) * P.dz[t1]);
        if (t2 < NDIM) m.r[t2] = (float)(-P.R + ((double)m.idx[t2] + p2) * P.dz[t2]);
        half_dir(es, ax, side, m.n);
        m.x = (float)(P.edges[bin] + (double)es.u01() * (P.edges[bin + 1] - P.edges[bin]));
        done = mc_cross<NDIM>(P, m, ax, side, es, n_conv, res);
    } else {
        const float p0 = es.u01(), p1 = es.u01(), p2 = es.u01();
        const float pp[3] = {p0, p1, p2};
        for (int ax = 0; ax < NDIM; ++ax) m.r[ax] = (float)(-P.R + ((double)m.idx[ax] + pp[ax]) * P.dz[ax]);
        iso_dir(es, m.n);
        m.x = (float)(P.edges[bin] + (double)es.u01() * (P.edges[bin + 1] - P.edges[bin]));
    }
    for (unsigned long long ev = 0; !done; ++ev) {
        if (ev >= P.mc_cap) { res.status = 2; break; }
        const unsigned cls = min(__ldg(&P.cell_class[min(m.cell, (unsigned)P.ncell - 1u)]), (unsigned)P.n_class - 1u);
        // frequency grouping (Sec. 5.3): the bin-mean opacity of the packet's bin
        // (the end bin past the grid, where the leakage has no flux either)
        unsigned jb = 0;
        float k;
        if (P.redist) {
            if (m.bin < 0) m.bin = min(max(bin_of(P, m.x), 0), P.J - 1);  // after a face crossing
            jb = (unsigned)m.bin;
            k = __ldg(&P.tau_row[cls * (unsigned)P.J + jb]) * P.inv_dzmin;
        } else {
            k = (float)P.cdesc[cls].k0 * voigt_H_f32(P.a, m.x);
        }
        const float sflight = -__logf(es.u01()) / k;
        float dmin = 3.0e38f;
        int fax = 0, fside = 1;
#pragma unroll
        for (int ax = 0; ax < NDIM; ++ax) {
            if (m.n[ax] == 0.0f) continue;
            const float lo = face_coord<NDIM>(P, ax, m.idx[ax]), hi = face_coord<NDIM>(P, ax, m.idx[ax] + 1);
            float d = m.n[ax] > 0.0f ? (hi - m.r[ax]) / m.n[ax] : (lo - m.r[ax]) / m.n[ax];
            d = fmaxf(d, 0.0f);
            if (d < dmin) { dmin = d; fax = ax; fside = m.n[ax] > 0.0f ? 1 : -1; }
        }
        ++n_mc;
        if (sflight < dmin) {
#pragma unroll
            for (int q = 0; q < 3; ++q) m.r[q] += sflight * m.n[q];
            if (P.redist) {
                // the new bin from row jb of eq. R_discrete (categorical draw on
                // its cumulative thresholds), x uniform in it, a new direction
                const unsigned w = es.next();
                const uint32_t* row = P.redist + (size_t)jb * (unsigned)(P.J - 1);
                int lo = 0, hi = P.J - 1;  // number of thresholds <= w
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (w >= __ldg(&row[mid])) lo = mid + 1; else hi = mid;
                }
                m.x = (float)(P.edges[lo] + (double)es.u01() * (P.edges[lo + 1] - P.edges[lo]));
                iso_dir(es, m.n);
                m.bin = lo;
            } else {
                m.x = scatter(P.a, m.x, m.n, P.upar, es);
            }
            const int j = P.redist ? m.bin : bin_of(P, m.x);
            if (thick_state<NDIM>(P, m.cell, j)) {
                ++n_conv;
                res.status = 0; res.cell = m.cell; res.bin = (unsigned)j;
                break;
            }
            continue;
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) m.r[q] += dmin * m.n[q];
        m.r[fax] = face_coord<NDIM>(P, fax, m.idx[fax] + (fside > 0 ? 1 : 0));
        done = mc_cross<NDIM>(P, m, fax, fside, es, n_conv, res);
        m.bin = -1;  // a crossing may shift x (Doppler, reflection): look the bin up again
    }
    e = es.e;
    return res;
}

__device__ __forceinline__ void cell_coords(const WalkParams& P, unsigned cell, unsigned ic[3]) {
    ic[0] = cell % (unsigned)P.n0;
    ic[1] = (cell / (unsigned)P.n0) % (unsigned)P.n[1];
    ic[2] = cell / (unsigned)P.n01;
}

__device__ __forceinline__ unsigned brick_of(const WalkParams& P, unsigned cell) {
    unsigned ic[3];
    cell_coords(P, cell, ic);
    const unsigned b = (unsigned)P.prop_b, sh = (unsigned)P.prop_sh;
    return (ic[0] + sh) / b + (unsigned)P.prop_nbx * ((ic[1] + sh) / b + (unsigned)P.prop_nby * ((ic[2] + sh) / b));
}

// Whether a packet at (cell, bin) is served by the proposal: its brick lies
// wholly inside the grid, the cell lies in the brick's inner cube (margin
// prop_m), the brick is eligible (brick_lk above -1e29) and the bin's cell
// optical depth 10^(brick_lk + lp[bin]) lies in [10^llo, 10^lhi].
__device__ __forceinline__ bool prop_takes(const WalkParams& P, unsigned cell, unsigned bin) {
    unsigned ic[3];
    cell_coords(P, cell, ic);
    const int b = P.prop_b, sh = P.prop_sh, m = P.prop_m;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int lo = (((int)ic[a] + sh) / b) * b - sh;
        if (lo < 0 || lo + b > P.n[a]) return false;
        const int l = (int)ic[a] - lo;
        if (l < m || l > b - 1 - m) return false;
    }
    const float lkb = __ldg(&P.prop_lk[brick_of(P, cell)]);
    if (!(lkb > -1.0e29f)) return false;
    const float l = lkb + __ldg(&P.prop_lp[min(bin, (unsigned)P.J - 1u)]);
    return l >= P.prop_llo && l <= P.prop_lhi;
}

template <int NDIM, bool SMEM_ROWS, bool HYBRID, bool PROPOSE, bool WEIGHT>
__global__ void __launch_bounds__(256, RDDMC_WALK_MIN_BLOCKS) walk_kernel(const WalkParams P) {
    constexpr int RW = NDIM == 1 ? 1 : 2;  // uint4 per row
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long* s_cnt = reinterpret_cast<unsigned long long*>(smem_raw);  // kCounters
    unsigned long long* s_face = s_cnt + kCounters;                              // 8
    unsigned long long* s_sb = s_face + 8;                                        // kNsb
    unsigned long long* s_hist = s_sb + kNsb;                                     // J+2 if in smem
    const int nhist = P.J + 2;
    uint2* s_fast = reinterpret_cast<uint2*>(s_hist + (P.hist_in_smem ? ((nhist + 1) & ~1) : 0));

    for (int i = threadIdx.x; i < kCounters + 8 + kNsb; i += blockDim.x) s_cnt[i] = 0ull;
    if (P.hist_in_smem)
        for (int i = threadIdx.x; i < nhist; i += blockDim.x) s_hist[i] = 0ull;
    if (SMEM_ROWS)
        for (int i = threadIdx.x; i < P.n_rows; i += blockDim.x) s_fast[i] = __ldg(&P.fast[i]);
    __syncthreads();
    const uint4* rows = P.rows;
    const uint2* fast = SMEM_ROWS ? s_fast : P.fast;

    const unsigned lane = threadIdx.x & 31u;
    const unsigned J = (unsigned)P.J;
    const unsigned nr1 = (unsigned)P.n_rows - 1u;
    const unsigned long long t_begin = P.time_slice_ns ? global_ns() : 0ull;
    bool have = false, exhausted = false;
    unsigned long long pid = 0, t = 0, e = 0, t_stop = 0;
    unsigned long long lw = 0;  // weight method: -ln(packet weight) in 2^-40 units
    unsigned cell = 0, cls = 0, s = 0;  // s = cls * J + bin: the row of the state
    unsigned long long n_steps = 0, n_edraw = 0, n_mc = 0;
    unsigned n_emit = 0, n_esc = 0, n_abort = 0, n_clamp = 0, status_bits = 0, n_conv = 0;

    // Outcome of an MC excursion: back to DDMC (returns false) or finished.
    auto after_mc = [&](const McResult& res) -> bool {
        if (res.status == 0) {
            cell = res.cell;
            cls = __ldg(&P.cell_class[min(cell, (unsigned)P.ncell - 1u)]);
            s = cls * J + min(res.bin, J - 1u);
            return false;
        }
        if (res.status == 1) {
            if (P.hist_in_smem) smem_tally(s_hist, (unsigned)res.hist);
            else atomicAdd(&P.tally[kHistOff + res.hist], 1ull);
            if (res.sb >= 0) smem_tally(s_sb, (unsigned)res.sb);
            smem_tally(s_face, (unsigned)res.face);
            ++n_esc;
            return true;
        }
        ++n_abort;
        return true;
    };

    // Weight method of dust absorption (Sec. 2.6): a packet whose weight fell
    // below 1e-10 is eliminated and counted absorbed.
    auto faded = [&]() -> bool {
        if (WEIGHT && lw > kLwMin) {
            atomicAdd(&s_cnt[C_ABSORBED], 1ull);
            return true;
        }
        return false;
    };

    // One full transition: every threshold, the outcome's action, spatial moves
    // with the class lookup, Doppler rebins and escapes.  Returns true when the
    // packet has finished.
    auto generic = [&](unsigned w) -> bool {
        const unsigned ri = min(s, nr1);
        if (WEIGHT) lw += __ldg(&P.wq[ri]);  // the weight kept over the dwell in this state
        const uint4 a = __ldg(&rows[ri * RW]);
        unsigned o = (unsigned)(w >= a.x) + (unsigned)(w >= a.y) + (unsigned)(w >= a.z);
        if (NDIM == 3) {
            const uint4 b = __ldg(&rows[ri * RW + 1]);
            o += (unsigned)(w >= b.x) + (unsigned)(w >= b.y) + (unsigned)(w >= b.z) + (unsigned)(w >= b.w);
        }
        if (P.dust && o == 2u * NDIM + 1u && w >= __ldg(&P.abs_thr[ri])) {  // absorbed by dust (Sec. 2.6)
            atomicAdd(&s_cnt[C_ABSORBED], 1ull);
            return true;
        }
        const unsigned fl = a.w;
        const unsigned act = (fl >> (2u * o)) & 3u;
        const unsigned bin = min(s - cls * J, J - 1u);
        if (o < 2u) {
            if (act == ACT_MOVE) { s += o ? 1u : 0xffffffffu; return faded(); }
            if (HYBRID && act == ACT_TO_MC)  // leak into a thin bin of this cell
                return after_mc(mc_excursion<NDIM>(P, cell, o ? min(bin + 1u, J - 1u) : (bin ? bin - 1u : 0u), -1,
                                                   pid, e, n_mc, n_conv));
            status_bits |= (unsigned)STATUS_UNSUPPORTED_EVENT;
            ++n_abort;
            return true;
        }
        const unsigned face = o - 2u;
        if (act == ACT_ESCAPE) {
            // the hybrid kernel takes the escape wholly out of line: its inlined MC
            // excursion already fills the register budget, and the inline wrapper
            // more than doubled its stack frame (measured 16 % slower on C2)
            const EscapeBins eb = HYBRID ? escape_bins<NDIM>(P, cell, bin, face, pid, e, (fl & FLAG_MOVING) != 0u)
                                         : escape_bins_inl<NDIM>(P, cell, bin, face, pid, e, (fl & FLAG_MOVING) != 0u);
            if (NDIM == 3 || (fl & FLAG_MOVING)) e += 5;
            if (P.hist_in_smem) smem_tally(s_hist, (unsigned)eb.hist);
            else atomicAdd(&P.tally[kHistOff + eb.hist], 1ull);
            if (eb.sb >= 0) smem_tally(s_sb, (unsigned)eb.sb);
            smem_tally(s_face, face);
            if (WEIGHT) {  // the escaped weight, 2^-32 units
                const unsigned long long ww =
                    (unsigned long long)llrint(exp(-(double)lw * 9.094947017729282e-13) * 4294967296.0);
                atomicAdd(&P.tally[P.hist_off_w], ww);
                atomicAdd(&P.tally[P.hist_off_w + 1 + eb.hist], ww);
            }
            ++n_esc;
            return true;
        }
        if (act == ACT_TO_MC) {
            if (HYBRID)  // leak into a thin neighbour cell
                return after_mc(mc_excursion<NDIM>(P, cell, bin, (int)face, pid, e, n_mc, n_conv));
            status_bits |= (unsigned)STATUS_UNSUPPORTED_EVENT;
            ++n_abort;
            return true;
        }
        unsigned nbin = bin;
        if (act == ACT_REBIN) {
            const Rebin rb = P.rebin[min(cls, (unsigned)P.n_class - 1u) * (2u * NDIM) + face];
            const unsigned w1 = event_word(pid, e++, P.k0, P.k1);
            int jn = (int)bin + rb.m + (w1 >= rb.thr ? 1 : 0);
            if (jn < 0) { jn = 0; ++n_clamp; }
            if (jn > (int)J - 1) { jn = (int)J - 1; ++n_clamp; }
            nbin = (unsigned)jn;
        }
        const unsigned ax = face >> 1;
        const unsigned stride = NDIM == 1 ? 1u : (ax == 0 ? 1u : (ax == 1 ? (unsigned)P.n0 : (unsigned)P.n01));
        cell = min((face & 1u) ? cell + stride : cell - stride, (unsigned)P.ncell - 1u);
        cls = __ldg(&P.cell_class[cell]);
        s = cls * J + nbin;
        return faded();
    };

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
                    unsigned bin = 0;
                    if (st == PK_INFLIGHT) {
                        cell = P.st_cell[pid];
                        bin = P.st_bin[pid];
                        t = P.st_t[pid];
                        e = P.st_e[pid];
                        if (WEIGHT) lw = P.st_lw[pid];
                        have = true;
                    } else if (st == PK_FRESH) {
                        // event draw 0: bit 31-a picks the centre cell on axis a, bit 28 the bin
                        const unsigned w = event_word(pid, 0, P.k0, P.k1);
                        unsigned idx[3];
#pragma unroll
                        for (int a = 0; a < 3; ++a)
                            idx[a] = (unsigned)P.src_cand[a][(P.src_ncand[a] == 2) ? ((w >> (31 - a)) & 1u) : 0u];
                        cell = idx[0] + (unsigned)P.n0 * idx[1] + (unsigned)P.n01 * idx[2];
                        bin = (unsigned)P.src_bin[(P.src_nbin == 2) ? ((w >> 28) & 1u) : 0u];
                        t = 0;
                        e = 1;
                        lw = 0;
                        ++n_emit;
                        have = true;
                    }
                    if (have) {
                        cell = min(cell, (unsigned)P.ncell - 1u);
                        cls = __ldg(&P.cell_class[cell]);
                        s = cls * J + min(bin, J - 1u);
                        t_stop = P.slice ? t + P.slice : ~0ull;
                        if (HYBRID && st == PK_FRESH) {
                            // a thin source state starts as MC
                            const uint4 a0 = __ldg(&rows[min(s, nr1) * RW]);
                            if (a0.w & FLAG_THIN) {
                                const unsigned long long e0 = e;
                                const McResult res = mc_excursion<NDIM>(P, cell, min(bin, J - 1u), -1, pid, e, n_mc,
                                                                        n_conv);
                                n_edraw += e - e0;
                                if (after_mc(res)) have = false;
                            }
                        }
                    }
                }
            }
        }
        if (__all_sync(FULL, exhausted && !have)) break;
        if (!have) continue;
        if (P.time_slice_ns && global_ns() - t_begin > P.time_slice_ns) {
            // end of the wall-time slice: save the packet, take no new one
            P.st_cell[pid] = cell;
            P.st_bin[pid] = min(s - cls * J, J - 1u);
            P.st_t[pid] = t;
            P.st_e[pid] = e;
            if (WEIGHT) P.st_lw[pid] = lw;
            P.st_status[pid] = PK_INFLIGHT;
            have = false;
            exhausted = true;
            continue;
        }
        if (PROPOSE && prop_takes(P, cell, min(s - cls * J, J - 1u))) {
            // the walk is Markov in (cell, bin): a packet in a state the proposal
            // serves waits for it (checked once per chunk of transitions)
            P.st_cell[pid] = cell;
            P.st_bin[pid] = min(s - cls * J, J - 1u);
            P.st_t[pid] = t;
            P.st_e[pid] = e;
            if (WEIGHT) P.st_lw[pid] = lw;
            P.st_status[pid] = PK_PARKED;
            // one queue atomic per warp: the lanes parking now share a block of slots
            const unsigned grp = __activemask();
            const int lead = __ffs(grp) - 1;
            unsigned long long k0q = 0;
            if ((int)lane == lead) k0q = atomicAdd(P.prop_qcount, (unsigned long long)__popc(grp));
            k0q = __shfl_sync(grp, k0q, lead);
            const unsigned long long k = k0q + (unsigned long long)__popc(grp & ((1u << lane) - 1u));
            P.prop_qpid[min(k, P.n_packets - 1ull)] = pid;
            have = false;
            continue;
        }

        // ---- run up to `chunk` transitions (with a proposal, up to the next
        // multiple of chunk, so the parking checkpoints do not depend on slicing)
        unsigned long long lim = PROPOSE ? (t / (unsigned long long)P.chunk + 1ull) * (unsigned long long)P.chunk
                                         : t + (unsigned long long)P.chunk;
        lim = lim < t_stop ? lim : t_stop;
        lim = lim < P.max_steps ? lim : P.max_steps;
        const unsigned long long t0 = t;
        const unsigned long long e0 = e;
        bool fin = false;
        {
            const uint32_t pl = (uint32_t)pid, ph = (uint32_t)(pid >> 32);
            unsigned long long blk = t >> 2;
            const unsigned ng = (unsigned)((lim - t) >> 2);  // full groups of four
            uint4 rn = philox_rk(make_uint4((uint32_t)blk, (uint32_t)(blk >> 32), pl, ph), P);
            unsigned g = 0;
            while (g < ng) {
                const uint4 r = rn;
                ++blk;
                rn = philox_rk(make_uint4((uint32_t)blk, (uint32_t)(blk >> 32), pl, ph), P);
                unsigned q;
#define RDDMC_FAST(W, Q)                                                                  \
    {                                                                                     \
        const uint2 f_ = SMEM_ROWS ? fast[min(s, nr1)] : __ldg(&fast[min(s, nr1)]);       \
        const unsigned long long wq_ = WEIGHT ? __ldg(&P.wq[min(s, nr1)]) : 0ull;         \
        if ((W) < f_.y && (!WEIGHT || lw + wq_ <= kLwMin)) {                              \
            if (WEIGHT) lw += wq_;                                                        \
            s += ((W) >= f_.x) ? 1u : 0xffffffffu;                                        \
        } else {                                                                          \
            q = (Q);                                                                      \
            goto slow;                                                                    \
        }                                                                                 \
    }
                if (!WEIGHT) {
                    // The group's four transitions as one branch-free chain: each
                    // head is loaded at the state the previous transition would
                    // reach by a frequency move (index clamped, so a speculative
                    // state past a non-move stays in bounds), then the chain is
                    // checked.  With no branch between the loads the scheduler
                    // fills their latency with the next group's Philox rounds.
                    const unsigned s0 = s;
                    const uint2 f0 = SMEM_ROWS ? fast[min(s0, nr1)] : __ldg(&fast[min(s0, nr1)]);
                    const unsigned s1 = s0 + ((r.x >= f0.x) ? 1u : 0xffffffffu);
                    const uint2 f1 = SMEM_ROWS ? fast[min(s1, nr1)] : __ldg(&fast[min(s1, nr1)]);
                    const unsigned s2 = s1 + ((r.y >= f1.x) ? 1u : 0xffffffffu);
                    const uint2 f2 = SMEM_ROWS ? fast[min(s2, nr1)] : __ldg(&fast[min(s2, nr1)]);
                    const unsigned s3 = s2 + ((r.z >= f2.x) ? 1u : 0xffffffffu);
                    const uint2 f3 = SMEM_ROWS ? fast[min(s3, nr1)] : __ldg(&fast[min(s3, nr1)]);
                    const unsigned s4 = s3 + ((r.w >= f3.x) ? 1u : 0xffffffffu);
                    const bool ok0 = r.x < f0.y, ok1 = r.y < f1.y, ok2 = r.z < f2.y, ok3 = r.w < f3.y;
                    if (ok0 && ok1 && ok2 && ok3) {
                        s = s4;
                        ++g;
                        continue;
                    }
                    // the first transition that is not a plain frequency move
                    // takes the generic step from the state before it
                    q = !ok0 ? 0u : (!ok1 ? 1u : (!ok2 ? 2u : 3u));
                    s = !ok0 ? s0 : (!ok1 ? s1 : (!ok2 ? s2 : s3));
                    goto slow;
                }
                RDDMC_FAST(r.x, 0u)
                RDDMC_FAST(r.y, 1u)
                RDDMC_FAST(r.z, 2u)
                RDDMC_FAST(r.w, 3u)
#undef RDDMC_FAST
                ++g;
                continue;
            slow:
                for (; q < 4u; ++q) {
                    if (generic(word_of(r, q))) {
                        fin = true;
                        t += 4ull * g + q + 1ull;
                        goto chunk_done;
                    }
                }
                ++g;
            }
            t += 4ull * ng;
            // at most three transitions left before the watchdog limit
            while (t < lim) {
                const unsigned long long b = t >> 2;
                const uint4 r = philox_rk(make_uint4((uint32_t)b, (uint32_t)(b >> 32), pl, ph), P);
                const bool f = generic(word_of(r, (unsigned)t & 3u));
                ++t;
                if (f) { fin = true; break; }
            }
        }
    chunk_done:
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
            P.st_bin[pid] = min(s - cls * J, J - 1u);
            P.st_t[pid] = t;
            P.st_e[pid] = e;
            if (WEIGHT) P.st_lw[pid] = lw;
            P.st_status[pid] = PK_INFLIGHT;
            have = false;
        }
    }

    // ---- flush: warp sums of the per-thread counters, then CTA totals to HBM
    n_edraw += n_emit;  // the source draw of each emitted packet
    unsigned long long v[9] = {n_emit, n_esc, n_abort, n_steps, n_clamp, n_edraw, status_bits, n_mc, n_conv};
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        unsigned long long x = v[i];
#pragma unroll
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
        atomicAdd(&s_cnt[C_MC_EVENTS], v[7]);
        atomicAdd(&s_cnt[C_CONVERSIONS], v[8]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kCounters; i += blockDim.x) {
        if (!s_cnt[i]) continue;
        if (i == C_STATUS_BITS) atomicOr(&P.tally[i], s_cnt[i]);
        else atomicAdd(&P.tally[i], s_cnt[i]);
    }
    for (int i = threadIdx.x; i < 2 * NDIM; i += blockDim.x)
        if (s_face[i]) atomicAdd(&P.tally[kFaceOff + i], s_face[i]);
    if (P.hist_in_smem)
        for (int i = threadIdx.x; i < nhist; i += blockDim.x)
            if (s_hist[i]) atomicAdd(&P.tally[kHistOff + i], s_hist[i]);
    for (int i = threadIdx.x; i < kNsb; i += blockDim.x)
        if (s_sb[i]) atomicAdd(&P.tally[kHistOff + nhist + i], s_sb[i]);
}

template <int NDIM, bool SMEM, bool HYBRID, bool PROPOSE, bool WEIGHT>
cudaError_t launch_variant(const WalkParams& P, int threads, size_t smem, int ctas, int nsm, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(walk_kernel<NDIM, SMEM, HYBRID, PROPOSE, WEIGHT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (!ctas) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas, walk_kernel<NDIM, SMEM, HYBRID, PROPOSE, WEIGHT>,
                                                          threads, smem);
        if (e != cudaSuccess) return e;
    }
    if (ctas < 1) ctas = 1;
    walk_kernel<NDIM, SMEM, HYBRID, PROPOSE, WEIGHT><<<(unsigned)(ctas * nsm), threads, smem, s>>>(P);
    return cudaGetLastError();
}

template <int NDIM, bool SMEM>
cudaError_t launch_mode(const WalkParams& P, int threads, size_t smem, int ctas, int nsm, cudaStream_t s) {
    if (NDIM == 3 && P.prop_b) return launch_variant<NDIM, SMEM, false, true, false>(P, threads, smem, ctas, nsm, s);
    if (P.weights) return launch_variant<NDIM, SMEM, false, false, true>(P, threads, smem, ctas, nsm, s);
    return P.hybrid ? launch_variant<NDIM, SMEM, true, false, false>(P, threads, smem, ctas, nsm, s)
                    : launch_variant<NDIM, SMEM, false, false, false>(P, threads, smem, ctas, nsm, s);
}

// One scattering per thread at x_in with incoming direction +e_z; sample i
// reads the event stream of packet i.
__global__ void scatter_samples_kernel(float a, float x_in, const float2* __restrict__ upar, uint32_t k0,
                                       uint32_t k1, unsigned long long n, float* __restrict__ out) {
    const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    EventStream es;
    es.init(i, 0, k0, k1);
    float d[3] = {0.0f, 0.0f, 1.0f};
    out[i] = scatter(a, x_in, d, upar, es);
}

// ------------------------------------------------------------ proposals
// A parked packet's cell, folded into the fundamental domain of its brick (the
// frame the network was trained in): a uniform static brick is invariant
// under the cube's reflections and axis permutations, so the exit sampled in
// the folded frame is mapped back by the inverse transform.
// First cell, per axis, of the inner cube (the served region) of the brick
// holding a cell.
__device__ __forceinline__ void brick_base(const WalkParams& P, const unsigned ic[3], int base[3]) {
    const int b = P.prop_b, sh = P.prop_sh;
#pragma unroll
    for (int a = 0; a < 3; ++a) base[a] = (((int)ic[a] + sh) / b) * b - sh + P.prop_m;
}

// A cell's inner-cube base and its local coordinates there (world frame).
__device__ __forceinline__ void region_local(const WalkParams& P, unsigned cell, int base[3], int l[3]) {
    unsigned ic[3];
    cell_coords(P, cell, ic);
    brick_base(P, ic, base);
#pragma unroll
    for (int a = 0; a < 3; ++a) l[a] = min(max((int)ic[a] - base[a], 0), P.prop_r - 1);
}

__device__ __forceinline__ void fold_parked(const WalkParams& P, unsigned cell, int base[3], int C[3], int perm[3],
                                            bool flip[3]) {
    unsigned ic[3];
    cell_coords(P, cell, ic);
    brick_base(P, ic, base);
    int l[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) l[a] = min(max((int)ic[a] - base[a], 0), P.prop_r - 1);
    fold_cell(l, P.prop_r, C, perm, flip);
}

// Network inputs of queued packets q0 .. q0+cnt (rows past cnt are zeroed).
// Negative frequencies are mirrored: a static uniform brick is symmetric under
// x -> -x and the network was trained on x >= 0.
__global__ void propose_features_kernel(const WalkParams P, const float* __restrict__ xc, FeatConst fc,
                                        unsigned long long q0, unsigned long long cnt, int batch,
                                        __nv_bfloat16* __restrict__ X) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= batch) return;
    if ((unsigned long long)r >= cnt) {
        for (int i = 0; i < kFeat; ++i) X[r * kFeat + i] = __float2bfloat16(0.0f);
        return;
    }
    const unsigned long long pid = P.prop_qpid[q0 + r];
    const unsigned cell = min(P.st_cell[pid], (unsigned)P.ncell - 1u);
    unsigned j = min(P.st_bin[pid], (unsigned)P.J - 1u);
    if (P.prop_sum) {
        // region mode: world frame, the region's summary and the cell's own density
        int base[3], l[3];
        region_local(P, cell, base, l);
        const float* sm = P.prop_sum + (size_t)brick_of(P, cell) * kRegionSum;
        const unsigned cls = min(__ldg(&P.cell_class[cell]), (unsigned)P.n_class - 1u);
        const float dlog = log10f((float)(P.cdesc[cls].k0 * P.dz[0])) - sm[0];
        features_region(sm, P.prop_lp[j], xc[j], dlog, l, P.prop_r, fc, X + r * kFeat);
        return;
    }
    if (xc[j] < 0.0f) j = (unsigned)P.J - 1u - j;
    int base[3], C[3], perm[3];
    bool flip[3];
    fold_parked(P, cell, base, C, perm, flip);
    features(P.prop_lk[brick_of(P, cell)], P.prop_lp[j], xc[j], C, P.prop_r, fc, X + r * kFeat);
}

// Inverse-CDF draw from softmax(z[0..n)) with uniform u in (0,1), by one
// warp: every lane reads a strided share of the row (coalesced), the maximum
// and the sum of exponentials are warp reductions (the sum broadcast from lane
// 0 so that every lane holds the same value), and the running sum advances 32
// entries at a time by a warp scan; the first entry whose running sum reaches
// u times the total is drawn.  Warp-uniform result.
__device__ __forceinline__ int softmax_draw_warp(const float* __restrict__ z, int n, float u, unsigned lane) {
    float mx = -3.0e38f;
    for (int c = (int)lane; c < n; c += 32) mx = fmaxf(mx, z[c]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
    float sum = 0.0f;
    for (int c = (int)lane; c < n; c += 32) sum += __expf(z[c] - mx);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(FULL, sum, o);
    const float target = u * __shfl_sync(FULL, sum, 0);
    float acc = 0.0f;
    for (int c0 = 0; c0 < n; c0 += 32) {
        const int c = c0 + (int)lane;
        float v = c < n ? __expf(z[c] - mx) : 0.0f;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float y = __shfl_up_sync(FULL, v, o);
            if ((int)lane >= o) v += y;
        }
        const unsigned hit = __ballot_sync(FULL, c < n && acc + v >= target);
        if (hit) return c0 + __ffs(hit) - 1;
        acc += __shfl_sync(FULL, v, 31);
    }
    return n - 1;
}

// Sample an exit for each queued packet from its logits and place the packet
// across the exit face; one warp per packet (blockDim a multiple of 32).  The
// warp reads the packet's logits together and every lane takes the same event
// draws, in order: the exit (face, bin) of head A, the step bucket of head B
// and a uniform inside it, then the exit cell on the face -- one draw from
// head C's slice of that face when nC > 0, else two uniform coordinates --
// then lane 0 makes the crossing with its own draws (a Doppler rebin, or the
// five of an escape).
__global__ void propose_place_kernel(const WalkParams P, const float* __restrict__ xc,
                                     const float* __restrict__ logits, int n_out, int nA, int nB, int nC,
                                     unsigned long long q0, unsigned long long cnt) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned long long r = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= cnt) return;  // warp-uniform
    const unsigned J = (unsigned)P.J;
    const unsigned long long pid = P.prop_qpid[q0 + r];
    const unsigned cell = min(P.st_cell[pid], (unsigned)P.ncell - 1u);
    const unsigned bin = min(P.st_bin[pid], J - 1u);
    const bool region = P.prop_sum != nullptr;  // world frame: no fold, no mirror
    const bool mirror = !region && xc[bin] < 0.0f;
    EventStream es;
    es.init(pid, P.st_e[pid], P.k0, P.k1);
    const unsigned long long e_start = es.e;
    const float* z = logits + r * (unsigned long long)n_out;
    // head A: exit face (folded frame) x exit bin
    const int ca = softmax_draw_warp(z, nA, es.u01(), lane);
    // head B: log2 step bucket
    const int kb = min(softmax_draw_warp(z + nA, nB, es.u01(), lane), 40);
    const unsigned long long steps = (1ull << kb) + (unsigned long long)(es.u01() * (float)(1ull << kb));
    const int b = P.prop_r;  // side of the served inner cube
    const int fc_ = ca / (int)J;
    unsigned jo = (unsigned)(ca % (int)J);
    if (mirror) jo = J - 1u - jo;
    // exit cell on the folded frame's face: coordinates (q1, q2) along the
    // other two axes, lower axis first
    int q1, q2;
    if (nC > 0) {
        const int S = b * b;
        const int pq = softmax_draw_warp(z + nA + nB + fc_ * S, S, es.u01(), lane);
        q1 = pq % b;
        q2 = pq / b;
    } else {
        q1 = min((int)(es.u01() * (float)b), b - 1);
        q2 = min((int)(es.u01() * (float)b), b - 1);
    }
    if (lane != 0u) return;
    int base[3], C[3], perm[3];
    bool flip[3];
    if (region) {
        region_local(P, cell, base, C);
        perm[0] = 0; perm[1] = 1; perm[2] = 2;
        flip[0] = flip[1] = flip[2] = false;
    } else {
        fold_parked(P, cell, base, C, perm, flip);
    }
    const int cax = fc_ >> 1, cside = fc_ & 1;
    int cc[3];
    cc[cax] = cside ? b - 1 : 0;
    cc[cax == 0 ? 1 : 0] = q1;
    cc[cax == 2 ? 1 : 2] = q2;
    // folded -> world: folded axis k is world axis perm[k], reflected when flip[perm[k]]
    int wc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int wa = perm[k];
        const int loc = flip[wa] ? b - 1 - cc[k] : cc[k];
        wc[wa] = min(max(base[wa] + loc, 0), P.n[wa] - 1);
    }
    const int fa = perm[cax];
    const int fs = cside ^ (flip[fa] ? 1 : 0);
    const unsigned f = (unsigned)(2 * fa + fs);
    const unsigned cin = min((unsigned)wc[0] + (unsigned)P.n0 * (unsigned)wc[1] + (unsigned)P.n01 * (unsigned)wc[2],
                             (unsigned)P.ncell - 1u);
    const unsigned cls = min(__ldg(&P.cell_class[cin]), (unsigned)P.n_class - 1u);
    const uint4 a0 = __ldg(&P.rows[(cls * J + jo) * 2u]);
    const unsigned act = (a0.w >> (2u * (2u + f))) & 3u;
    unsigned long long* T = P.tally;
    if (act == ACT_ESCAPE) {
        const EscapeBins eb = escape_bins<3>(P, cin, jo, f, pid, es.e, (a0.w & FLAG_MOVING) != 0u);
        es.e += 5;
        atomicAdd(&T[kHistOff + eb.hist], 1ull);
        atomicAdd(&T[kFaceOff + f], 1ull);
        if (eb.sb >= 0) atomicAdd(&T[kHistOff + P.J + 2 + eb.sb], 1ull);
        atomicAdd(&T[C_ESCAPED], 1ull);
        P.st_status[pid] = PK_DONE;
    } else {
        unsigned j2 = jo;
        if (act == ACT_REBIN) {
            const Rebin rb = P.rebin[cls * 6u + f];
            const unsigned w1 = es.next();
            int jn = (int)jo + rb.m + (w1 >= rb.thr ? 1 : 0);
            if (jn < 0) { jn = 0; atomicAdd(&T[C_CLAMPS], 1ull); }
            if (jn > (int)J - 1) { jn = (int)J - 1; atomicAdd(&T[C_CLAMPS], 1ull); }
            j2 = (unsigned)jn;
        }
        const unsigned stride = fa == 0 ? 1u : (fa == 1 ? (unsigned)P.n0 : (unsigned)P.n01);
        const unsigned nb = min(fs ? cin + stride : cin - stride, (unsigned)P.ncell - 1u);
        P.st_cell[pid] = nb;
        P.st_bin[pid] = j2;
        P.st_status[pid] = PK_INFLIGHT;
    }
    P.st_e[pid] = es.e;
    atomicAdd(&T[C_PROPOSALS], 1ull);
    atomicAdd(&T[C_PROPOSED_STEPS], steps);
    atomicAdd(&T[C_EVENT_DRAWS], es.e - e_start);
}

// First passages out of the regions (brick inner cubes) of the grid's own
// medium, for training the proposal on media that vary from cell to cell.
// Sample i is packet p0 + i: event draws 0-2 pick the brick (from the listed
// ones), the start cell of its region and the start bin (from the brick's
// listed bins); the packet then takes the walk's transitions on the grid's
// table (transition stream; Doppler rebins take the next event draws) until an
// outcome would carry it out of the region.  That crossing is not made: the
// sample records the face, the bin and the cell on the face it would leave
// from (the proposal's placement makes the crossing).
struct FpRegionParams {
    const int32_t* bricks;
    const int32_t* bin_off;
    const int32_t* bins;
    int n_el;
    unsigned long long p0, n, cap;
    int32_t* out;
    unsigned long long* steps;
    // training targets and features (null: records only)
    __nv_bfloat16* X;
    int32_t *tA, *tB, *tC;
    const float* lp;
    const float* xc;
    FeatConst fc;
};

__global__ void __launch_bounds__(256) fp_region_kernel(const WalkParams P, const FpRegionParams F) {
    const unsigned J = (unsigned)P.J, nr1 = (unsigned)P.n_rows - 1u;
    const int r = P.prop_r, bl = P.prop_b;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < F.n; i += stride) {
        const unsigned long long pid = F.p0 + i;
        EventStream es;
        es.init(pid, 0, P.k0, P.k1);
        const unsigned w0 = es.next(), w1 = es.next(), w2 = es.next();
        const int k = min((int)(((unsigned long long)w0 * (unsigned long long)F.n_el) >> 32), F.n_el - 1);
        const int br = F.bricks[k];
        const int bc[3] = {br % P.prop_nbx, (br / P.prop_nbx) % P.prop_nby, br / (P.prop_nbx * P.prop_nby)};
        const int mc = (int)(((unsigned long long)w1 * (unsigned long long)(r * r * r)) >> 32);
        int l[3] = {mc % r, (mc / r) % r, mc / (r * r)};
        int base[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) base[a] = bc[a] * bl - P.prop_sh + P.prop_m;
        const int cnt = F.bin_off[k + 1] - F.bin_off[k];
        int j = F.bins[F.bin_off[k] + min((int)(((unsigned long long)w2 * (unsigned long long)cnt) >> 32), cnt - 1)];
        const int j0 = j;
        const int l0[3] = {l[0], l[1], l[2]};
        const uint32_t pl = (uint32_t)pid, ph = (uint32_t)(pid >> 32);
        int face = 6, pos = -1;
        unsigned long long t = 0;
        while (t < F.cap && face == 6) {
            const unsigned long long blk = t >> 2;
            const uint4 rw = philox_rk(make_uint4((uint32_t)blk, (uint32_t)(blk >> 32), pl, ph), P);
            bool stop = false;
            for (unsigned q = (unsigned)(t & 3u); q < 4u && t < F.cap; ++q) {
                const unsigned w = word_of(rw, q);
                ++t;
                int wc[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) wc[a] = min(max(base[a] + l[a], 0), P.n[a] - 1);
                const unsigned cell = (unsigned)wc[0] + (unsigned)P.n0 * (unsigned)wc[1] + (unsigned)P.n01 * (unsigned)wc[2];
                const unsigned cls = min(__ldg(&P.cell_class[min(cell, (unsigned)P.ncell - 1u)]), (unsigned)P.n_class - 1u);
                const unsigned sidx = min(cls * J + (unsigned)j, nr1);
                const uint2 f = __ldg(&P.fast[sidx]);
                if (w < f.y) { j += (w >= f.x) ? 1 : -1; continue; }
                const uint4 a = __ldg(&P.rows[2u * sidx]), c = __ldg(&P.rows[2u * sidx + 1u]);
                const unsigned o = (unsigned)(w >= a.x) + (unsigned)(w >= a.y) + (unsigned)(w >= a.z) +
                                   (unsigned)(w >= c.x) + (unsigned)(w >= c.y) + (unsigned)(w >= c.z) +
                                   (unsigned)(w >= c.w);
                if (o < 2u) { j += o ? 1 : -1; continue; }
                const int fc_ = (int)o - 2, ax = fc_ >> 1, side = (fc_ & 1) ? 1 : -1;
                if (l[ax] + side < 0 || l[ax] + side >= r) {
                    face = fc_;
                    const int u = ax == 0 ? 1 : 0, v = ax == 2 ? 1 : 2;  // the other two axes, lower first
                    pos = l[u] + r * l[v];
                    break;
                }
                const unsigned act = (a.w >> (2u * o)) & 3u;
                if (act == ACT_ESCAPE || act == ACT_TO_MC) { stop = true; break; }  // not inside a region
                if (act == ACT_REBIN) {
                    const Rebin rb = P.rebin[cls * 6u + (unsigned)fc_];
                    const unsigned wr = es.next();
                    const int jn = j + rb.m + (wr >= rb.thr ? 1 : 0);
                    j = jn < 0 ? 0 : (jn > (int)J - 1 ? (int)J - 1 : jn);
                }
                l[ax] += side;
            }
            if (stop) break;
        }
        int32_t* o8 = F.out + 8 * i;
        o8[0] = br;
        o8[1] = j0;
        o8[2] = mc;
        o8[3] = face;
        o8[4] = j;
        o8[5] = pos;
        o8[6] = (int32_t)(es.e - 3ull);
        o8[7] = 0;
        F.steps[i] = t;
        if (F.X) {
            int wc0[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) wc0[a] = min(max(base[a] + l0[a], 0), P.n[a] - 1);
            const unsigned c0 = (unsigned)wc0[0] + (unsigned)P.n0 * (unsigned)wc0[1] + (unsigned)P.n01 * (unsigned)wc0[2];
            const unsigned cls0 = min(__ldg(&P.cell_class[min(c0, (unsigned)P.ncell - 1u)]), (unsigned)P.n_class - 1u);
            const float* sm = P.prop_sum + (size_t)br * kRegionSum;
            const float dlog = log10f((float)(P.cdesc[cls0].k0 * P.dz[0])) - sm[0];
            features_region(sm, F.lp[j0], F.xc[j0], dlog, l0, r, F.fc, F.X + kFeat * i);
            F.tA[i] = face < 6 ? face * (int)J + min(max(j, 0), (int)J - 1) : -1;
            F.tB[i] = step_bucket(t);
            if (F.tC) F.tC[i] = face < 6 ? face * r * r + pos : -1;
        }
    }
}

}  // namespace

cudaError_t launch_scatter_samples(const rddmc_grid& g, const void* d_table, double x_in, uint64_t seed, uint64_t n,
                                   float* d_out, cudaStream_t s) {
    const float2* upar = (const float2*)((const char*)d_table + g.off_upar);
    const unsigned blocks = (unsigned)((n + 255) / 256);
    scatter_samples_kernel<<<blocks, 256, 0, s>>>((float)g.a, (float)x_in, upar, (uint32_t)seed,
                                                  (uint32_t)(seed >> 32), n, d_out);
    return cudaGetLastError();
}

void fill_walk_params(const rddmc_grid& g, const WalkLaunch& w, WalkParams& P) {
    const rddmc_run_opts& o = w.opts;
    const char* tb = (const char*)w.d_table;
    char* sb = (char*)w.d_state;
    std::memset(&P, 0, sizeof(P));
    P.rows = (const uint4*)(tb + g.off_rows);
    P.fast = (const uint2*)(tb + g.off_fast);
    P.tau_row = (const float*)(tb + g.off_tau);
    P.upar = (const float2*)(tb + g.off_upar);
    P.cdesc = (const ClassDesc*)(tb + g.off_cdesc);
    P.hybrid = g.params.mode == RDDMC_MODE_HYBRID ? 1 : 0;
    P.a = (float)g.a;
    P.lambda = (float)g.params.lambda;
    for (int a = 0; a < 3; ++a) P.n[a] = g.n[a];
    P.cell_class = (const uint32_t*)(tb + g.off_class);
    P.rebin = (const Rebin*)(tb + g.off_rebin);
    P.cell_v = (const double*)(tb + g.off_vel);
    P.edges = (const double*)(tb + g.off_edges);
    P.abs_thr = (const uint32_t*)(tb + g.off_abs);
    P.dust = g.dusty() ? 1 : 0;
    P.redist = o.redist;
    P.wq = (const unsigned long long*)(tb + g.off_wq);
    P.weights = g.weighted() ? 1 : 0;
    P.hist_off_w = kHistOff + g.J + 2 + kNsb;
    {
        double dzmin = 2.0 * g.R / g.n[0];
        for (int a = 1; a < g.ndim; ++a) dzmin = std::min(dzmin, 2.0 * g.R / g.n[a]);
        P.inv_dzmin = (float)(1.0 / dzmin);
    }
    const uint64_t np = o.n_packets;
    uint64_t off = 256;
    if (sb) {  // the packet-state arrays (first-passage generation has none)
        P.cursor = (unsigned long long*)sb;
        P.st_cell = (uint32_t*)(sb + off); off += align256(np * 4);
        P.st_bin = (uint32_t*)(sb + off); off += align256(np * 4);
        P.st_t = (unsigned long long*)(sb + off); off += align256(np * 8);
        P.st_e = (unsigned long long*)(sb + off); off += align256(np * 8);
        P.st_status = (uint8_t*)(sb + off); off += align256(np * 1);
        P.st_lw = (unsigned long long*)(sb + off);
    }
    P.tally = w.d_tally;
    P.n_packets = np;
    P.max_steps = o.max_steps ? o.max_steps : (1ull << 62);
    P.mc_cap = o.max_steps ? o.max_steps : 100000000ull;  // events per MC excursion
    P.slice = o.steps_per_launch;
    P.time_slice_ns = o.time_slice_us > 0 ? (unsigned long long)o.time_slice_us * 1000ull : 0ull;
    P.k0 = (uint32_t)o.seed;
    P.k1 = (uint32_t)(o.seed >> 32);
    for (int r = 0; r < 10; ++r) {
        P.rk0[r] = P.k0 + (uint32_t)r * 0x9E3779B9u;
        P.rk1[r] = P.k1 + (uint32_t)r * 0xBB67AE85u;
    }
    P.J = g.J;
    P.n_class = g.n_class;
    P.n_rows = g.n_class * g.J;
    P.ncell = (int)g.ncell;
    P.n0 = g.n[0];
    P.n01 = g.n[0] * g.n[1];
    P.R = g.R;
    for (int a = 0; a < 3; ++a) P.dz[a] = 2.0 * g.R / g.n[a];
    P.vth = g.vth;
    P.chunk = o.chunk ? o.chunk : 256;
    P.resume = o.resume;
    P.save_state = (o.steps_per_launch != 0 || o.resume || o.time_slice_us > 0) ? 1 : 0;
    P.hist_in_smem = (g.J + 2 <= kSmemHistMax) ? 1 : 0;
    P.moving = g.moving ? 1 : 0;
    for (int a = 0; a < 3; ++a) {
        P.src_ncand[a] = g.src_ncand[a];
        P.src_cand[a][0] = g.src_cand[a][0];
        P.src_cand[a][1] = g.src_cand[a][1];
    }
    P.src_nbin = g.src_nbin;
    P.src_bin[0] = g.src_bin[0];
    P.src_bin[1] = g.src_bin[1];
    if (o.proposal) {
        const rddmc_proposal* pr = o.proposal;
        P.prop_b = pr->brick;
        P.prop_sh = (pr->brick - pr->offset % pr->brick) % pr->brick;
        P.prop_nbx = (g.n[0] + P.prop_sh + pr->brick - 1) / pr->brick;
        P.prop_nby = (g.n[1] + P.prop_sh + pr->brick - 1) / pr->brick;
        P.prop_m = pr->margin;
        P.prop_r = pr->brick - 2 * pr->margin;
        P.prop_lk = pr->d_brick_lk;
        P.prop_lp = pr->d_lp;
        P.prop_llo = (float)pr->log_tau_lo;
        P.prop_lhi = (float)pr->log_tau_hi;
        P.prop_qcount = pr->d_queue_count;
        P.prop_qpid = pr->d_queue_pid;
        P.prop_sum = pr->d_summary;
        P.save_state = 1;
    }
}

cudaError_t launch_walk(const rddmc_grid& g, const WalkLaunch& w, cudaStream_t s) {
    const rddmc_run_opts& o = w.opts;
    WalkParams P;
    fill_walk_params(g, w, P);

    int dev = 0, nsm = 0, smem_optin = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
        return e;
    const int threads = o.threads_per_cta ? o.threads_per_cta : 256;
    size_t smem = (size_t)(kCounters + 8 + kNsb) * 8;
    if (P.hist_in_smem) smem += (size_t)((g.J + 2 + 1) & ~1) * 8;
    const size_t rows_bytes = (size_t)P.n_rows * 8;  // fast heads
    const bool use_smem_rows = o.table_in_smem && smem + rows_bytes <= (size_t)smem_optin;
    if (use_smem_rows) smem += rows_bytes;
    if ((e = cudaMemsetAsync(P.cursor, 0, 8, s)) != cudaSuccess) return e;
    if (P.save_state && !o.resume && (e = cudaMemsetAsync(P.st_status, PK_FRESH, o.n_packets, s)) != cudaSuccess)
        return e;
    if (g.ndim == 1)
        return use_smem_rows ? launch_mode<1, true>(P, threads, smem, o.ctas_per_sm, nsm, s)
                             : launch_mode<1, false>(P, threads, smem, o.ctas_per_sm, nsm, s);
    return use_smem_rows ? launch_mode<3, true>(P, threads, smem, o.ctas_per_sm, nsm, s)
                         : launch_mode<3, false>(P, threads, smem, o.ctas_per_sm, nsm, s);
}

}  // namespace rddmc

extern "C" int rddmc_mlp_forward(int n_out, const float* d_wf, const void* d_wb, const void* d_x, int batch,
                                 void* d_work, float* d_logits, void* stream);
extern "C" uint64_t rddmc_mlp_work_bytes(int batch, int n_out);

extern "C" int rddmc_propose(const rddmc_grid* g, const void* d_table, const rddmc_proposal* pr, uint64_t seed,
                             uint64_t n_packets, void* d_state, void* d_tallies, int n_out, int nA, int nB, int nC,
                             const float* d_wf, const void* d_wb, int batch, void* d_work, uint64_t* n_served,
                             void* stream) {
    using namespace rddmc;
    if (!g || !d_table || !pr || !d_state || !d_tallies || !d_wf || !d_wb || !d_work) return RDDMC_ERR_ARG;
    if (!g->precomputed) return RDDMC_ERR_TABLE;
    if (g->ndim != 3 || g->params.mode != RDDMC_MODE_DDMC || g->dusty() || g->weighted())
        return RDDMC_ERR_UNSUPPORTED;
    // the buffers the walk with this proposal was launched on (as rddmc_launch_packets checks them)
    if (((uintptr_t)d_table & 255u) || ((uintptr_t)d_state & 255u) || ((uintptr_t)d_tallies & 7u) ||
        ((uintptr_t)d_work & 255u))
        return RDDMC_ERR_ARG;
    if (n_packets == 0 || n_packets >= (1ull << 63)) return RDDMC_ERR_ARG;
    if (!pr->d_brick_lk || !pr->d_lp || !pr->d_xc || !pr->d_queue_count || !pr->d_queue_pid) return RDDMC_ERR_ARG;
    if (batch < 64 || batch % 64 || nA != 6 * g->J || nB < 1 || nB > 41 || nC < 0 || nA + nB + nC > n_out ||
        n_out % 16)
        return RDDMC_ERR_ARG;
    if (pr->brick < 1 || pr->brick > 64 || pr->offset < 0 || pr->offset >= pr->brick) return RDDMC_ERR_ARG;
    if (pr->margin < 0 || 2 * pr->margin >= pr->brick) return RDDMC_ERR_ARG;
    const int side = pr->brick - 2 * pr->margin;
    if (nC != 0 && nC != 6 * side * side) return RDDMC_ERR_ARG;
    if ((int64_t)pr->n_bricks != proposal_bricks(*g, *pr)) return RDDMC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    WalkLaunch w;
    std::memset(&w, 0, sizeof(w));
    w.d_table = d_table;
    w.d_state = d_state;
    w.d_tally = (unsigned long long*)d_tallies;
    w.opts.seed = seed;
    w.opts.n_packets = n_packets;
    w.opts.proposal = pr;
    w.opts.steps_per_launch = 4;
    WalkParams P;
    fill_walk_params(*g, w, P);
    unsigned long long cnt = 0;
    if (cudaMemcpyAsync(&cnt, pr->d_queue_count, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return RDDMC_ERR_CUDA;
    const uint64_t mlp_bytes = align256(rddmc_mlp_work_bytes(batch, n_out));
    __nv_bfloat16* X = (__nv_bfloat16*)((char*)d_work + mlp_bytes);
    float* logits = (float*)((char*)X + align256((uint64_t)batch * kFeat * 2));
    FeatConst fc;
    fc.log_b = log10f((float)(pr->brick - 2 * pr->margin));
    fc.log_a = (float)log10(g->a);
    fc.inv_xs = (float)(1.0 / std::max(std::fabs(g->edges.front()), std::fabs(g->edges.back())));
    for (unsigned long long q0 = 0; q0 < cnt; q0 += (unsigned long long)batch) {
        const unsigned long long c = std::min<unsigned long long>(batch, cnt - q0);
        const int rows = (int)((c + 63) / 64 * 64);  // forward only the rows in use
        propose_features_kernel<<<(rows + 127) / 128, 128, 0, s>>>(P, pr->d_xc, fc, q0, c, rows, X);
        if (cudaGetLastError() != cudaSuccess) return RDDMC_ERR_CUDA;
        const int rc = rddmc_mlp_forward(n_out, d_wf, d_wb, X, rows, d_work, logits, stream);
        if (rc != RDDMC_OK) return rc;
        propose_place_kernel<<<(unsigned)((c + 3) / 4), 128, 0, s>>>(P, pr->d_xc, logits, n_out, nA, nB, nC, q0,
                                                                      c);  // a warp per packet
        if (cudaGetLastError() != cudaSuccess) return RDDMC_ERR_CUDA;
    }
    if (cudaMemsetAsync(pr->d_queue_count, 0, 8, s) != cudaSuccess) return RDDMC_ERR_CUDA;
    if (n_served) *n_served = cnt;
    // no final synchronisation: work queued next on `stream` runs after these kernels
    return cudaGetLastError() == cudaSuccess ? RDDMC_OK : RDDMC_ERR_CUDA;
}

extern "C" int rddmc_fp_region_generate(const rddmc_grid* g, const void* d_table, const rddmc_fp_region* reg,
                                        uint64_t seed, uint64_t p0, uint64_t n, uint64_t cap, int32_t* d_out,
                                        uint64_t* d_steps, const rddmc_fp_train* train, void* stream) {
    using namespace rddmc;
    if (!g || !d_table || !reg || !d_out || !d_steps || n == 0 || cap == 0) return RDDMC_ERR_ARG;
    if (!g->precomputed) return RDDMC_ERR_TABLE;
    if (g->ndim != 3 || g->params.mode != RDDMC_MODE_DDMC || g->dusty() || g->weighted())
        return RDDMC_ERR_UNSUPPORTED;
    if (reg->brick < 1 || reg->brick > 64 || reg->offset < 0 || reg->offset >= reg->brick) return RDDMC_ERR_ARG;
    if (reg->margin < 0 || 2 * reg->margin >= reg->brick) return RDDMC_ERR_ARG;
    if (reg->n_eligible < 1 || !reg->d_bricks || !reg->d_bin_off || !reg->d_bins || !reg->d_summary)
        return RDDMC_ERR_ARG;
    rddmc_proposal pr;
    std::memset(&pr, 0, sizeof(pr));
    pr.brick = reg->brick;
    pr.offset = reg->offset;
    pr.margin = reg->margin;
    pr.d_summary = reg->d_summary;
    WalkLaunch w;
    std::memset(&w, 0, sizeof(w));
    w.d_table = d_table;
    w.opts.seed = seed;
    w.opts.n_packets = 1;
    w.opts.proposal = &pr;
    WalkParams P;
    fill_walk_params(*g, w, P);
    FpRegionParams F;
    std::memset(&F, 0, sizeof(F));
    F.bricks = reg->d_bricks;
    F.bin_off = reg->d_bin_off;
    F.bins = reg->d_bins;
    F.n_el = reg->n_eligible;
    F.p0 = p0;
    F.n = n;
    F.cap = cap;
    F.out = d_out;
    F.steps = (unsigned long long*)d_steps;
    if (train) {
        if (!train->d_x || !train->d_ta || !train->d_tb || !train->d_lp || !train->d_xc) return RDDMC_ERR_ARG;
        F.X = (__nv_bfloat16*)train->d_x;
        F.tA = train->d_ta;
        F.tB = train->d_tb;
        F.tC = train->d_tc;
        F.lp = train->d_lp;
        F.xc = train->d_xc;
        F.fc.log_b = log10f((float)(reg->brick - 2 * reg->margin));
        F.fc.log_a = (float)log10(g->a);
        F.fc.inv_xs = (float)(1.0 / std::max(std::fabs(g->edges.front()), std::fabs(g->edges.back())));
    }
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return RDDMC_ERR_CUDA;
    const unsigned long long want = (n + 255) / 256;
    const unsigned blocks = (unsigned)(want < (unsigned long long)nsm * 8 ? want : (unsigned long long)nsm * 8);
    fp_region_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(P, F);
    return cudaGetLastError() == cudaSuccess ? RDDMC_OK : RDDMC_ERR_CUDA;
}
