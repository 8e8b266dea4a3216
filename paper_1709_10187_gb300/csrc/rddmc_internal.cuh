// rddmc_internal.cuh -- internal layout and device helpers of the CUDA library.
//
// Device table buffer (caller-owned, filled by rddmc_precompute_leakage):
//   [TableHeader | cell_class u32[ncell] | ClassDesc[n_class] | Rebin[n_class*nfaces]
//    | cell velocity f64[3*ncell] (moving media only) | edges f64[J+1] | phi f64[J] | rows
//    | fast heads uint2[n_class*J] | tau f32[n_class*J] | u_par split points f32x2[kUparN]
//    | 1/K_s f32[n_class*J] | dust absorption thresholds u32[n_class*J]]
// With dust absorption (Sec. 2.6) the categorical draw has one more outcome,
// absorption, after the leakage outcomes: the row thresholds are cumulative over
// the leakage rates plus k_a, and the absorption threshold (where absorption
// starts) is kept apart so that rows keep their size.
// every region 256-byte aligned.  Rows are n_class blocks of J rows; a row is
// 16 bytes in a slab {thr0, thr1, thr2, flags} and 32 bytes in 3D
// {thr0, thr1, thr2, flags, thr3, thr4, thr5, thr6}: the first 16 bytes always
// hold both frequency thresholds and the flags, which is all the frequency-move
// fast path needs.  A fast head {thr0, thr1 or 0} repeats the two frequency
// thresholds of each row in 8 bytes, with thr1 replaced by 0 when a frequency
// outcome is not a plain move, so that a frequency move reads 8 bytes and one
// failed compare sends every other case to the full row.  Outcome order:
// bin-1, bin+1, then -e_a, +e_a per axis.
//
// Tally buffer (u64): [0, 16) counters, [16, 22) faces, [22, 22+J+2) escape
// histogram, then kNsb impact-parameter bins.
// State buffer: [0, 256) cursor and spare words, then SoA per-packet arrays.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace rddmc {

constexpr uint32_t kMagic = 0x52444d43u;  // "RDMC"
constexpr int kMaxFaces = 6;
constexpr int kCounters = 16;
constexpr int kFaceOff = 16;
constexpr int kHistOff = 22;
constexpr int kNsb = 64;            // impact-parameter bins over b/R in [0, kSbMax)
constexpr double kSbMax = 1.28;
constexpr int kUparN = 1024;        // |x| grid of the u_par envelope split points
constexpr float kUparStep = 1.0f / 16.0f;

enum Counter : int {
    C_EMITTED = 0, C_ESCAPED = 1, C_ABORTED = 2, C_STEPS = 3, C_MC_EVENTS = 4,
    C_CONVERSIONS = 5, C_CLAMPS = 6, C_EVENT_DRAWS = 7, C_STATUS_BITS = 8, C_PROPOSALS = 9,
    C_PROPOSED_STEPS = 10, C_ABSORBED = 11,
};

// 2-bit actions per outcome in the flags word.
constexpr uint32_t ACT_MOVE = 0u, ACT_ESCAPE = 1u, ACT_TO_MC = 2u, ACT_REBIN = 3u;
constexpr uint32_t FLAG_FASTX = 1u << 29;   // both frequency outcomes are plain moves
constexpr uint32_t FLAG_MOVING = 1u << 30;
constexpr uint32_t FLAG_THIN = 1u << 31;

// Device-side status bits (C_STATUS_BITS).
constexpr uint64_t STATUS_UNSUPPORTED_EVENT = 1ull << 0;

enum PacketStatus : uint8_t { PK_FRESH = 0, PK_INFLIGHT = 1, PK_DONE = 2, PK_PARKED = 3 };

struct FaceDesc {
    int32_t exterior;   // 1: the neighbour is outside the grid or vacuum
    int32_t pad;
    double k0_nb;       // neighbour's line-centre coefficient (tau0/R * n_rel)
    double ks_nb;       // neighbour's dust scattering coefficient
    double delta;       // comoving shift x' = x + delta on crossing (eq. velocity-shift)
};

struct ClassDesc {
    double k0;          // tau0/R * n_rel of the cells in this class
    double ks, ka;      // grey dust scattering and absorption coefficients (Sec. 2.6)
    int32_t moving;     // the cells have non-zero bulk velocity
    int32_t pad;
    FaceDesc face[kMaxFaces];
};

struct Rebin {          // new bin = j + m + [w >= thr] on crossing the face
    int32_t m;
    uint32_t thr;
};

struct TableHeader {
    uint32_t magic;
    uint32_t filled;
    int32_t ndim, J, ncell, n_class, K, row_bytes;
    int32_t n[3], mode;
    uint64_t off_class, off_cdesc, off_rebin, off_vel, off_edges, off_phi, off_rows, off_fast, off_tau, off_upar,
        total;
    double tau_ddmc, lambda, f_mu, a, dz[3], vth;
};

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two 32x32->64
// multiplies with the published constants, xor of the high halves with the
// other counter words and the round key, key bumped by the Weyl constants.
struct KeySched {
    uint32_t k0, k1;
};

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Word `n` of the event stream of packet `p` (top counter bit set).
__device__ __forceinline__ uint32_t event_word(uint64_t p, uint64_t n, uint32_t k0, uint32_t k1) {
    const uint64_t b = n >> 2;
    uint4 r = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)(b >> 32), (uint32_t)p,
                                       (uint32_t)(p >> 32) | 0x80000000u), k0, k1);
    const uint32_t l = (uint32_t)n & 3u;
    return l == 0 ? r.x : (l == 1 ? r.y : (l == 2 ? r.z : r.w));
}

__host__ __device__ __forceinline__ uint64_t align256(uint64_t v) { return (v + 255ull) & ~255ull; }

}  // namespace rddmc
