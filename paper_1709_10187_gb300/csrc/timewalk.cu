// timewalk.cu -- time-dependent DDMC walk (Sec. 2.3, causality within a time
// step; eq. E_estimator, bin and path estimates of the energy density).
//
// One launch advances every live packet through one time step [t_n, t_{n+1}].
// In state s a packet draws a dwell path dl = -ln(xi) / K_s, K_s the sum of the
// state's leakage coefficients: by eq. l_min_1/2 the smallest of the competing
// exponential lengths is Exp(K_s), independent of which process wins, and the
// categorical draw of the persistent walk picks the winner.  A dwell that
// passes t_{n+1} leaves the packet in its state, without leaking, until then;
// the next step draws a fresh dwell (the exponential is memoryless).  Lengths
// and times share one unit (c = 1).
//
// Time inside a step is an unsigned count of ticks, 2^31 per step.  The dwell
// is formed in FP32 (log2 of the 32-bit uniform on the special-function unit,
// times the state's 1/K_s and the step's ticks per unit length) and rounded to
// the nearest tick: a packet's clock and every path tally are integer sums, so
// the path estimate of a state does not depend on the order in which atomics
// land, and rounding moves each dwell by at most half a tick (2^-32 of the
// step), without bias.
//
// Streams: transition word t is lane t&3 of Philox4x32-10(ctr = (t>>2, p_lo,
// p_hi)), as in the persistent walk; dwell word d is lane d&3 of
// Philox4x32-10(ctr = (d>>2, p_lo, p_hi | 2^30)); packet ids stay below 2^62.
// Transitions run in groups of four with t a multiple of four at the start of
// each group (one transition call per group; a packet resumed at another t
// first walks single transitions up to the next multiple of four), and the
// dwell words of a group come from at most two dwell blocks, the lower one
// usually the block cached from the group before: two Philox calls per four
// transitions in all.  Lanes take packets from a global cursor (one atomicAdd
// per warp) and run at most `chunk` transitions between refills (256 by
// default), so a lane whose packet stopped early in its step takes a new one
// while long-running packets continue.  When fewer than `regroup` lanes of a
// warp are still walking (8 by default), they break off after their group of
// four, keeping packet, clock and cached blocks in registers, so that the
// stopped lanes take new packets before the warp walks on: in thick media a
// packet takes only a few transitions per step, and without the break a warp
// waits for its slowest lane.
//
// Tallies: the path and bin estimates go to shared memory when the grid's
// states fit (ticks as a u32 low word plus a u32 carry count, so every update
// is a native 32-bit shared atomic, and u32 bin counts; flushed with one
// atomic per touched state), else straight to global memory; the escape
// tallies of the walk use the tally buffer's shared-memory staging, as in the
// persistent walk.  With a leak buffer, the leaks of eq. a_estimator are summed
// per cell face in FP64 (shared memory when small), in their own kernel
// instantiation.  With dust by packet weights (Sec. 2.6), another
// instantiation attenuates each path l by exp(-k_a l), keeps the weight with
// the packet between steps, eliminates packets below 1e-10 and sums weighted
// bin and path estimates in FP64 (the path weighted by the weight averaged
// along it).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "grid.h"
#include "walk_common.cuh"

namespace rddmc {
namespace {

constexpr uint32_t kTicks = 1u << 31;  // ticks per time step
constexpr size_t kSmemTallyMax = 110 * 1024;  // shared-memory budget per CTA for the per-state tallies
constexpr int kRegroupDefault = 8;  // a warp regroups when fewer than a quarter of its lanes still walk

struct TimeParams {
    const float* rk;                 // 1 / K_s per row
    unsigned long long* st_d;        // dwell words drawn per packet
    unsigned long long* bins;        // [ncell * J] packets per state at t_{n+1}
    unsigned long long* path;        // [ncell * J] ticks spent per state during the step
    unsigned long long* counts;      // [5] escaped during the step, dwells, transitions, alive at t_{n+1}, absorbed
    double* leak;                    // [ncell * 2 NDIM * 2] k x ticks of leaks out of / into each face, or null
    float inv_dz;                    // 1 / dz_min: k of a row = tau_row / dz_min
    int leak_in_smem;
    int leak_smem_off;               // byte offset of the leak block in dynamic shared memory
    float x_scale;                   // ln 2 * ticks per unit length: dwell ticks = -log2(u) * x_scale / K_s
    int start;                       // every packet starts at the source at t_n
    int n_states;
    // dust by packet weights (Sec. 2.6): k_a per row (1/R units), the packet
    // weights, and the weighted bin and path estimates (FP64; path in ticks)
    const float* ka;
    float* st_w;
    double* wbins;
    double* wpath;
    float tick_len;                  // step length / 2^31
    int regroup;                     // lanes break off their packets when fewer than this many walk (0: never)
};

__device__ __forceinline__ uint4 time_block(unsigned long long b, uint32_t pl, uint32_t ph, const WalkParams& P) {
    return philox_rk(make_uint4((uint32_t)b, (uint32_t)(b >> 32), pl, ph | 0x40000000u), P);
}

__device__ __forceinline__ uint4 trans_block(unsigned long long b, uint32_t pl, uint32_t ph, const WalkParams& P) {
    return philox_rk(make_uint4((uint32_t)b, (uint32_t)(b >> 32), pl, ph), P);
}

// MINB: resident 256-thread CTAs per SM the register budget targets (2: no
// spills, 16 warps per SM; 3: 24 warps with a few spilled registers).
template <int NDIM, bool SMEM_TALLY, int MINB, bool LEAK, bool WEIGHT>
__global__ void __launch_bounds__(256, MINB) time_kernel(const WalkParams P, const TimeParams T) {
    constexpr int RW = NDIM == 1 ? 1 : 2;  // uint4 per row
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long* s_cnt = reinterpret_cast<unsigned long long*>(smem_raw);  // kCounters
    unsigned long long* s_face = s_cnt + kCounters;                              // 8
    unsigned long long* s_sb = s_face + 8;                                        // kNsb
    unsigned long long* s_hist = s_sb + kNsb;                                     // J+2 if in smem
    const int nhist = P.J + 2;
    // per-state tallies: path ticks as two u32 words (low word and carries, so
    // that every update is a native 32-bit shared atomic) and the bin counts
    unsigned* s_plo = reinterpret_cast<unsigned*>(s_hist + (P.hist_in_smem ? nhist : 0));  // n_states if SMEM_TALLY
    unsigned* s_phi = s_plo + (SMEM_TALLY ? T.n_states : 0);
    unsigned* s_bins = s_phi + (SMEM_TALLY ? T.n_states : 0);
    const int n_leak = LEAK ? P.ncell * 2 * NDIM * 2 : 0;
    double* s_leak = reinterpret_cast<double*>(smem_raw + T.leak_smem_off);  // n_leak if leak_in_smem

    for (int i = threadIdx.x; i < kCounters + 8 + kNsb; i += blockDim.x) s_cnt[i] = 0ull;
    if (P.hist_in_smem)
        for (int i = threadIdx.x; i < nhist; i += blockDim.x) s_hist[i] = 0ull;
    if (SMEM_TALLY)
        for (int i = threadIdx.x; i < T.n_states; i += blockDim.x) {
            s_plo[i] = 0u;
            s_phi[i] = 0u;
            s_bins[i] = 0u;
        }
    if (LEAK && T.leak_in_smem)
        for (int i = threadIdx.x; i < n_leak; i += blockDim.x) s_leak[i] = 0.0;
    __syncthreads();

    const uint4* rows = P.rows;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned J = (unsigned)P.J;
    const unsigned nr1 = (unsigned)P.n_rows - 1u;
    const unsigned ns1 = (unsigned)T.n_states - 1u;
    bool have = false, exhausted = false;
    unsigned long long pid = 0, t = 0, e = 0, d = 0;
    unsigned cell = 0, cls = 0, s = 0;  // s = cls * J + bin: the row of the state
    unsigned el = 0;                    // ticks elapsed in this step
    uint32_t pl = 0, ph = 0;
    unsigned long long tbc = ~0ull;     // index of the cached dwell block
    uint4 rtc = make_uint4(0u, 0u, 0u, 0u);
    float wgt = 1.0f;                   // dust by weights: the packet weight
    unsigned long long tnc = ~0ull;     // index of the cached transition block
    uint4 rnc = make_uint4(0u, 0u, 0u, 0u);
    unsigned long long n_steps = 0, n_edraw = 0, n_dwell = 0;
    unsigned n_emit = 0, n_esc = 0, n_abort = 0, n_clamp = 0, n_alive = 0, n_absorbed = 0, status_bits = 0;

    auto add_path = [&](unsigned ticks) {
        if (!ticks) return;
        const unsigned st = min(cell * J + min(s - cls * J, J - 1u), ns1);
        if (SMEM_TALLY) {
            const unsigned old = atomicAdd(&s_plo[st], ticks);  // ticks <= 2^31: at most one carry
            if (old + ticks < old) atomicAdd(&s_phi[st], 1u);
        } else {
            atomicAdd(&T.path[st], (unsigned long long)ticks);
        }
    };

    // Leak of eq. a_estimator through face slot `f` (cell * 2 NDIM + face) of a
    // packet whose dwell was `ticks`: k of the row times the ticks.
    auto add_leak = [&](unsigned f, unsigned io, unsigned row, unsigned ticks) {
        const double v = (double)(__ldg(&P.tau_row[min(row, nr1)]) * T.inv_dz * (float)ticks);
        const unsigned i = min(2u * f + io, (unsigned)n_leak - 1u);
        if (T.leak_in_smem) atomicAdd(&s_leak[i], v);
        else atomicAdd(&T.leak[i], v);
    };

    // One transition of the state on word w after a dwell of `ticks`: every
    // threshold, the outcome's action, spatial moves with the class lookup,
    // Doppler rebins and escapes.  Returns true when the packet escaped or met
    // an unsupported event.
    auto generic = [&](unsigned w, unsigned ticks) -> bool {
        const unsigned ri = min(s, nr1);
        const uint4 a = __ldg(&rows[ri * RW]);
        unsigned o = (unsigned)(w >= a.x) + (unsigned)(w >= a.y) + (unsigned)(w >= a.z);
        if (NDIM == 3) {
            const uint4 b = __ldg(&rows[ri * RW + 1]);
            o += (unsigned)(w >= b.x) + (unsigned)(w >= b.y) + (unsigned)(w >= b.z) + (unsigned)(w >= b.w);
        }
        if (P.dust && o == 2u * NDIM + 1u && w >= __ldg(&P.abs_thr[ri])) {  // absorbed by dust (Sec. 2.6)
            atomicAdd(&s_cnt[C_ABSORBED], 1ull);
            ++n_absorbed;
            return true;
        }
        const unsigned fl = a.w;
        const unsigned act = (fl >> (2u * o)) & 3u;
        const unsigned bin = min(s - cls * J, J - 1u);
        if (o < 2u) {
            if (act == ACT_MOVE) { s += o ? 1u : 0xffffffffu; return false; }
            status_bits |= (unsigned)STATUS_UNSUPPORTED_EVENT;  // MC hand-offs are not part of this walk
            ++n_abort;
            return true;
        }
        const unsigned face = o - 2u;
        if (LEAK && act != ACT_TO_MC) add_leak(cell * (2u * NDIM) + face, 0u, ri, ticks);
        if (act == ACT_ESCAPE) {
            const EscapeBins eb = escape_bins<NDIM>(P, cell, bin, face, pid, e, (fl & FLAG_MOVING) != 0u);
            if (NDIM == 3 || (fl & FLAG_MOVING)) e += 5;
            if (P.hist_in_smem) smem_tally(s_hist, (unsigned)eb.hist);
            else atomicAdd(&P.tally[kHistOff + eb.hist], 1ull);
            if (eb.sb >= 0) smem_tally(s_sb, (unsigned)eb.sb);
            smem_tally(s_face, face);
            ++n_esc;
            return true;
        }
        if (act == ACT_TO_MC) {
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
        if (LEAK) add_leak(cell * (2u * NDIM) + (face ^ 1u), 1u, s, ticks);
        return false;
    };

    // One dwell on dwell word wd and, if the packet is still inside the step,
    // one transition on word wt.  Returns 0 (moved), 1 (stopped at t_{n+1}) or
    // 2 (finished: escaped or unsupported event).
    // Dust by weights: over `ticks` of path the weight falls by exp(-k_a l);
    // the weighted path estimate takes the weight averaged along the path.
    auto attenuate = [&](unsigned ri, unsigned ticks) {
        const float l = (float)ticks;
        const float ta = __ldg(&T.ka[ri]) * l * T.tick_len;
        const float avg = ta > 1e-4f ? -expm1f(-ta) / ta : 1.0f - 0.5f * ta;
        const unsigned st = min(cell * J + min(s - cls * J, J - 1u), ns1);
        atomicAdd(&T.wpath[st], (double)(wgt * l * avg));
        wgt *= expf(-ta);
    };

    auto dwell_then_move = [&](unsigned wd, unsigned wt) -> int {
        const unsigned ri = min(s, nr1);
        ++d;
        ++n_dwell;
        const float u = fmaf((float)wd, 0x1p-32f, 0x1p-33f);
        const float x = -__log2f(u) * (T.x_scale * __ldg(&T.rk[ri]));
        const unsigned dt = x < 4.0e9f ? __float2uint_rn(x) : 0xffffffffu;
        const unsigned rem = kTicks - el;
        if (dt > rem) {  // causality: the packet stays in its state until t_{n+1}
            add_path(rem);
            if (WEIGHT) attenuate(ri, rem);
            el = kTicks;
            return 1;
        }
        add_path(dt);
        if (WEIGHT) attenuate(ri, dt);
        el += dt;
        ++t;
        const uint2 f = __ldg(&P.fast[ri]);
        int r;
        if (wt < f.y) {
            s += (wt >= f.x) ? 1u : 0xffffffffu;
            r = 0;
        } else {
            r = generic(wt, dt) ? 2 : 0;
        }
        if (WEIGHT && r == 0 && wgt < 1e-10f) {  // eliminated below the paper's w_min
            atomicAdd(&s_cnt[C_ABSORBED], 1ull);
            ++n_absorbed;
            r = 2;
        }
        return r;
    };

    auto dwell_word = [&](unsigned long long dd) -> unsigned {
        const unsigned long long b = dd >> 2;
        if (b != tbc) { rtc = time_block(b, pl, ph, P); tbc = b; }
        return word_of(rtc, (unsigned)dd & 3u);
    };

    auto trans_word = [&](unsigned long long tt) -> unsigned {
        const unsigned long long b = tt >> 2;
        if (b != tnc) { rnc = trans_block(b, pl, ph, P); tnc = b; }
        return word_of(rnc, (unsigned)tt & 3u);
    };

    for (;;) {
        // ---- warp-cooperative refill, repeated while lanes draw finished packets
        for (;;) {
            const unsigned need = __ballot_sync(FULL, !have && !exhausted);
            if (!need) break;
            const int leader = __ffs(need) - 1;
            unsigned long long first = 0;
            if ((int)lane == leader) first = atomicAdd(P.cursor, (unsigned long long)__popc(need));
            first = __shfl_sync(FULL, first, leader);
            if (!have && !exhausted) {
                pid = first + (unsigned long long)__popc(need & ((1u << lane) - 1u));
                if (pid >= P.n_packets) {
                    exhausted = true;
                } else {
                    const uint8_t st = T.start ? (uint8_t)PK_FRESH : P.st_status[pid];
                    unsigned bin = 0;
                    if (st == PK_INFLIGHT) {
                        cell = P.st_cell[pid];
                        bin = P.st_bin[pid];
                        t = P.st_t[pid];
                        e = P.st_e[pid];
                        d = T.st_d[pid];
                        if (WEIGHT) wgt = T.st_w[pid];
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
                        d = 0;
                        wgt = 1.0f;
                        ++n_emit;
                        ++n_edraw;  // the source draw
                        have = true;
                    }
                    if (have) {
                        cell = min(cell, (unsigned)P.ncell - 1u);
                        cls = __ldg(&P.cell_class[cell]);
                        s = cls * J + min(bin, J - 1u);
                        el = 0;
                        pl = (uint32_t)pid;
                        ph = (uint32_t)(pid >> 32);
                        tbc = ~0ull;
                        tnc = ~0ull;
                    }
                }
            }
        }
        if (__all_sync(FULL, !have)) break;  // every lane is out of packets
        // once the cursor has run dry, lanes that stop cannot take new packets
        const bool dry = __any_sync(FULL, exhausted);
        if (!have) continue;

        // ---- up to `chunk` dwells: single ones up to t = 0 mod 4, then groups of four
        const unsigned long long t0 = t, e0 = e;
        const unsigned long long lim = min(t + (unsigned long long)P.chunk, P.max_steps);
        int r = 0;
        bool cut = false;
        while (r == 0 && (t & 3ull) && t < lim) r = dwell_then_move(dwell_word(d), trans_word(t));
        while (r == 0 && t + 4ull <= lim) {
            // Regroup: packets take different numbers of dwells to reach t_{n+1},
            // so once fewer than `regroup` lanes are still walking, they break
            // off (keeping their packets, blocks and clocks in registers) and the
            // stopped lanes take new packets before the warp walks on.
            if (T.regroup && !dry && __popc(__activemask()) < (unsigned)T.regroup) {
                cut = true;
                break;
            }
            const uint4 rn = trans_block(t >> 2, pl, ph, P);
            tnc = t >> 2;
            rnc = rn;
            const unsigned long long b0 = d >> 2;
            const unsigned p = (unsigned)d & 3u;
            const uint4 lo = (b0 == tbc) ? rtc : time_block(b0, pl, ph, P);
            uint4 hi = lo;
            if (p) hi = time_block(b0 + 1ull, pl, ph, P);
            tbc = p ? b0 + 1ull : b0;
            rtc = hi;
#pragma unroll
            for (unsigned k = 0; k < 4u; ++k) {
                const unsigned q = p + k;
                const unsigned wd = q < 4u ? word_of(lo, q) : word_of(hi, q - 4u);
                r = dwell_then_move(wd, word_of(rn, k));
                if (r) break;
            }
        }
        if (!cut)
            while (r == 0 && t < lim) r = dwell_then_move(dwell_word(d), trans_word(t));  // short chunk end
        n_steps += t - t0;
        n_edraw += e - e0;
        if (r == 0 && t >= P.max_steps) {
            ++n_abort;
            r = 2;
        }
        if (r == 2) {
            have = false;
            P.st_status[pid] = PK_DONE;
        } else if (r == 1) {
            const unsigned bin = min(s - cls * J, J - 1u);
            const unsigned st = min(cell * J + bin, ns1);
            if (SMEM_TALLY) atomicAdd(&s_bins[st], 1u);
            else atomicAdd(&T.bins[st], 1ull);
            if (WEIGHT) {
                atomicAdd(&T.wbins[st], (double)wgt);
                T.st_w[pid] = wgt;
            }
            ++n_alive;
            P.st_cell[pid] = cell;
            P.st_bin[pid] = bin;
            P.st_t[pid] = t;
            P.st_e[pid] = e;
            T.st_d[pid] = d;
            P.st_status[pid] = PK_INFLIGHT;
            have = false;
        }
    }

    // ---- flush: warp sums of the per-thread counters, then CTA totals to HBM
    unsigned long long v[10] = {n_emit, n_esc,  n_abort, n_steps, n_clamp,
                                n_edraw, status_bits, n_dwell, n_alive, n_absorbed};
#pragma unroll
    for (int i = 0; i < 10; ++i) {
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
        if (v[1]) atomicAdd(&T.counts[0], v[1]);
        if (v[7]) atomicAdd(&T.counts[1], v[7]);
        if (v[3]) atomicAdd(&T.counts[2], v[3]);
        if (v[8]) atomicAdd(&T.counts[3], v[8]);
        if (v[9]) atomicAdd(&T.counts[4], v[9]);
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
    if (LEAK && T.leak_in_smem)
        for (int i = threadIdx.x; i < n_leak; i += blockDim.x)
            if (s_leak[i] != 0.0) atomicAdd(&T.leak[i], s_leak[i]);
    if (SMEM_TALLY)
        for (int i = threadIdx.x; i < T.n_states; i += blockDim.x) {
            const unsigned long long v = ((unsigned long long)s_phi[i] << 32) | s_plo[i];
            if (v) atomicAdd(&T.path[i], v);
            if (s_bins[i]) atomicAdd(&T.bins[i], (unsigned long long)s_bins[i]);
        }
}

template <int NDIM, bool SMEM_TALLY, int MINB, bool LEAK, bool WEIGHT>
cudaError_t launch_time_minb(const WalkParams& P, const TimeParams& T, int threads, size_t smem, int ctas, int nsm,
                             cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(time_kernel<NDIM, SMEM_TALLY, MINB, LEAK, WEIGHT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    if (!ctas) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas, time_kernel<NDIM, SMEM_TALLY, MINB, LEAK, WEIGHT>, threads, smem);
        if (e != cudaSuccess) return e;
    }
    if (ctas < 1) ctas = 1;
    time_kernel<NDIM, SMEM_TALLY, MINB, LEAK, WEIGHT><<<(unsigned)(ctas * nsm), threads, smem, s>>>(P, T);
    return cudaGetLastError();
}

template <int NDIM, bool SMEM_TALLY>
cudaError_t launch_time(const WalkParams& P, const TimeParams& T, int threads, size_t smem, int ctas, int nsm,
                        cudaStream_t s) {
    // default and ctas_per_sm >= 3: the 24-warp variant (faster on short steps);
    // ctas_per_sm 1 or 2: the spill-free 16-warp one
    // the leak tally of eq. a_estimator is its own instantiation, so the default
    // kernel carries none of its registers
    if (T.wbins)  // dust by weights: its own instantiation (no leak tally alongside)
        return launch_time_minb<NDIM, SMEM_TALLY, 3, false, true>(P, T, threads, smem, ctas, nsm, s);
    if (T.leak)
        return (ctas == 0 || ctas >= 3)
                   ? launch_time_minb<NDIM, SMEM_TALLY, 3, true, false>(P, T, threads, smem, ctas, nsm, s)
                   : launch_time_minb<NDIM, SMEM_TALLY, 2, true, false>(P, T, threads, smem, ctas, nsm, s);
    return (ctas == 0 || ctas >= 3) ? launch_time_minb<NDIM, SMEM_TALLY, 3, false, false>(P, T, threads, smem, ctas, nsm, s)
                                    : launch_time_minb<NDIM, SMEM_TALLY, 2, false, false>(P, T, threads, smem, ctas, nsm, s);
}

}  // namespace

// walk state | dwell counters u64[np] | packet weights f32[np] (dust by weights)
uint64_t time_state_bytes_for(uint64_t np) { return state_bytes_for(np) + align256(np * 8) + align256(np * 4); }

}  // namespace rddmc

extern "C" uint64_t rddmc_time_state_bytes(uint64_t n_packets) {
    if (n_packets >= (1ull << 62)) return 0;
    return rddmc::time_state_bytes_for(n_packets);
}

extern "C" int rddmc_time_step_launch(const rddmc_grid* g, const void* d_table, const rddmc_time_step* ts,
                                      void* d_state, size_t state_bytes, void* d_tallies, size_t tally_bytes,
                                      uint64_t* d_bins, uint64_t* d_path, uint64_t* d_counts, double* d_leak,
                                      double* d_wbins, double* d_wpath, void* stream) {
    using namespace rddmc;
    if (!g || !d_table || !ts || !d_state || !d_tallies || !d_bins || !d_path || !d_counts) return RDDMC_ERR_ARG;
    if (((uintptr_t)d_state & 255u) || ((uintptr_t)d_tallies & 7u) || ((uintptr_t)d_bins & 7u) ||
        ((uintptr_t)d_path & 7u) || ((uintptr_t)d_counts & 7u) || ((uintptr_t)d_leak & 7u))
        return RDDMC_ERR_ARG;
    if (!g->precomputed) return RDDMC_ERR_TABLE;
    // dust by packet weights is the persistent walk's method only
    if (g->params.mode != RDDMC_MODE_DDMC) return RDDMC_ERR_UNSUPPORTED;
    // weighted estimates exactly with dust by weights, and not with the leak tally
    if ((!d_wbins) != (!d_wpath) || ((d_wbins != nullptr) != g->weighted()) || ((uintptr_t)d_wbins & 7u) ||
        ((uintptr_t)d_wpath & 7u))
        return RDDMC_ERR_ARG;
    if (d_wbins && d_leak) return RDDMC_ERR_UNSUPPORTED;
    if (ts->n_packets < 1 || ts->n_packets >= (1ull << 62)) return RDDMC_ERR_ARG;
    if (!(std::isfinite(ts->t_begin) && std::isfinite(ts->t_end) && ts->t_end > ts->t_begin)) return RDDMC_ERR_ARG;
    if (ts->chunk < 0 || ts->chunk % 4 || ts->chunk > (1 << 20)) return RDDMC_ERR_ARG;
    if (ts->threads_per_cta < 0 || ts->threads_per_cta % 32 || ts->threads_per_cta > 256 || ts->ctas_per_sm < 0 ||
        ts->ctas_per_sm > 32 || (ts->start != 0 && ts->start != 1))
        return RDDMC_ERR_ARG;
    if (ts->regroup < -1 || ts->regroup > 32 || ts->reserved != 0) return RDDMC_ERR_ARG;
    if ((uint64_t)g->ncell * (uint64_t)g->J > 0xffffffffull) return RDDMC_ERR_UNSUPPORTED;
    if (state_bytes < time_state_bytes_for(ts->n_packets)) return RDDMC_ERR_SIZE;
    if (tally_bytes < tally_bytes_for(g->J)) return RDDMC_ERR_SIZE;
    cudaStream_t s = (cudaStream_t)stream;

    WalkLaunch w;
    std::memset(&w, 0, sizeof(w));
    w.d_table = d_table;
    w.d_state = d_state;
    w.d_tally = (unsigned long long*)d_tallies;
    w.opts.seed = ts->seed;
    w.opts.n_packets = ts->n_packets;
    w.opts.max_steps = ts->max_steps;
    w.opts.chunk = ts->chunk ? ts->chunk : 256;
    WalkParams P;
    fill_walk_params(*g, w, P);
    TimeParams T;
    std::memset(&T, 0, sizeof(T));
    T.rk = (const float*)((const char*)d_table + g->off_rk);
    T.st_d = (unsigned long long*)((char*)d_state + state_bytes_for(ts->n_packets));
    T.bins = (unsigned long long*)d_bins;
    T.path = (unsigned long long*)d_path;
    T.counts = (unsigned long long*)d_counts;
    T.x_scale = (float)(0.69314718055994530942 * (double)kTicks / (ts->t_end - ts->t_begin));
    T.start = ts->start;
    T.leak = d_leak;
    T.ka = (const float*)((const char*)d_table + g->off_ka);
    T.st_w = (float*)((char*)T.st_d + align256(ts->n_packets * 8));
    T.wbins = d_wbins;
    T.wpath = d_wpath;
    T.tick_len = (float)((ts->t_end - ts->t_begin) / (double)kTicks);
    T.regroup = ts->regroup < 0 ? 0 : (ts->regroup ? ts->regroup : kRegroupDefault);
    double dzmin = 2.0 * g->R / g->n[0];
    for (int a = 1; a < g->ndim; ++a) dzmin = std::min(dzmin, 2.0 * g->R / g->n[a]);
    T.inv_dz = (float)(1.0 / dzmin);
    T.n_states = (int)std::min<uint64_t>((uint64_t)g->ncell * g->J, 0x7fffffffull);

    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RDDMC_ERR_CUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RDDMC_ERR_CUDA;
    const int threads = ts->threads_per_cta ? ts->threads_per_cta : 256;
    size_t smem = (size_t)(kCounters + 8 + kNsb) * 8;
    if (P.hist_in_smem) smem += (size_t)(g->J + 2) * 8;
    // per-state tallies in shared memory while they fit the budget (u32 bin
    // counts: a CTA walks fewer than 2^32 packets per step)
    const bool smem_path = smem + (size_t)T.n_states * 12 <= kSmemTallyMax && ts->n_packets < (1ull << 32);
    if (smem_path) smem += (size_t)T.n_states * 12;
    // the leak block (eq. a_estimator) in shared memory when it is small
    const size_t leak_bytes = d_leak ? (size_t)g->ncell * 2 * g->ndim * 2 * 8 : 0;
    if (d_leak && leak_bytes <= 16384) {
        smem = (smem + 15) & ~(size_t)15;
        T.leak_smem_off = (int)smem;
        T.leak_in_smem = 1;
        smem += leak_bytes;
    }
    if (cudaMemsetAsync(P.cursor, 0, 8, s) != cudaSuccess) return RDDMC_ERR_CUDA;
    cudaError_t e;
    if (g->ndim == 1)
        e = smem_path ? launch_time<1, true>(P, T, threads, smem, ts->ctas_per_sm, nsm, s)
                      : launch_time<1, false>(P, T, threads, smem, ts->ctas_per_sm, nsm, s);
    else
        e = smem_path ? launch_time<3, true>(P, T, threads, smem, ts->ctas_per_sm, nsm, s)
                      : launch_time<3, false>(P, T, threads, smem, ts->ctas_per_sm, nsm, s);
    return e == cudaSuccess ? RDDMC_OK : RDDMC_ERR_CUDA;
}
