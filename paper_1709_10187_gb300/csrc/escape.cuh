// escape.cuh -- FP64 geometry of a packet escaping through an exterior face,
// shared by the single-grid walk, the time-dependent walk and the batched walk.
#pragma once
#include <cstdint>

#include "rddmc_internal.cuh"

namespace rddmc {

struct EscapeBins {
    int hist;   // escape-frequency bin (0 below the grid, J+1 above)
    int sb;     // impact-parameter bin, -1 if not tallied
};

// FP64 escape geometry of a packet leaving through `face` of the cell at
// index idx, at bin `bin`, in the observer frame of Sec. 2.5: a point on the
// face (two event draws for the tangential axes), an isotropic outward
// direction (mu uniform on (0,1], azimuth uniform), x uniform in the bin;
// x_obs = x + n.(v/v_th) binned over the edges and, in 3D, the impact
// parameter b = |r x n|.  Every product that meets a sum is rounded on its own
// (__dmul_rn / __dadd_rn are never contracted into fused multiply-adds), so
// the bins follow the arithmetic as written, whatever the compiler's
// contraction setting, and equal the FP64 oracle's.  Callers keep it out of
// their hot loops: inlined into an out-of-line escape function, or called
// through escape_geometry_ool.
struct EscapeFrame {
    int ndim, J;
    double R, vth;
    const double* dz;      // cell width per axis
    const double* edges;   // J + 1 frequency edges
    const double* v;       // the cell's bulk velocity (km/s, 3 values), or null when static
};

static __device__ __forceinline__ EscapeBins escape_geometry(const EscapeFrame& F, const int idx[3], unsigned bin,
                                                             unsigned face, unsigned long long pid,
                                                             unsigned long long e, uint32_t k0, uint32_t k1) {
    EscapeBins out;
    out.sb = -1;
    const int ax = (int)(face >> 1), side = (face & 1u) ? 1 : -1;
    const int t1 = (ax + 1) % 3, t2 = (ax + 2) % 3;
    const double inv = 1.0 / 4294967296.0;
    double r[3];
    r[ax] = __dadd_rn(-F.R, __dmul_rn((double)(idx[ax] + (side > 0 ? 1 : 0)), F.dz[ax]));
    const double p1 = ((double)event_word(pid, e, k0, k1) + 0.5) * inv;
    const double p2 = ((double)event_word(pid, e + 1, k0, k1) + 0.5) * inv;
    r[t1] = (t1 < F.ndim) ? __dadd_rn(-F.R, __dmul_rn((double)idx[t1] + p1, F.dz[t1])) : 0.0;
    r[t2] = (t2 < F.ndim) ? __dadd_rn(-F.R, __dmul_rn((double)idx[t2] + p2, F.dz[t2])) : 0.0;
    // (w + 0.5) 2^-32 is exact, so the subtraction below has nothing to fuse
    const double mu = 1.0 - ((double)event_word(pid, e + 2, k0, k1) + 0.5) * inv;
    const double ph = 2.0 * 3.14159265358979323846 * (((double)event_word(pid, e + 3, k0, k1) + 0.5) * inv);
    const double xu = ((double)event_word(pid, e + 4, k0, k1) + 0.5) * inv;
    const double x = __dadd_rn(F.edges[bin], __dmul_rn(xu, F.edges[bin + 1] - F.edges[bin]));
    const double st = sqrt(fmax(0.0, __dadd_rn(1.0, -__dmul_rn(mu, mu))));
    double n[3];
    n[ax] = (double)side * mu;
    n[t1] = st * cos(ph);
    n[t2] = st * sin(ph);
    double nu = 0.0;
    if (F.v) {
        nu = __dadd_rn(__dadd_rn(__dmul_rn(n[0], F.v[0] / F.vth), __dmul_rn(n[1], F.v[1] / F.vth)),
                       __dmul_rn(n[2], F.v[2] / F.vth));
    }
    const double xo = x + nu;
    if (xo < F.edges[0]) {
        out.hist = 0;
    } else if (xo >= F.edges[F.J]) {
        out.hist = F.J + 1;
    } else {
        int lo = 0, hi = F.J;  // edges[lo] <= xo < edges[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (xo >= F.edges[mid]) lo = mid; else hi = mid;
        }
        out.hist = lo + 1;
    }
    if (F.ndim == 3) {
        const double rr = __dadd_rn(__dadd_rn(__dmul_rn(r[0], r[0]), __dmul_rn(r[1], r[1])), __dmul_rn(r[2], r[2]));
        const double rn = __dadd_rn(__dadd_rn(__dmul_rn(r[0], n[0]), __dmul_rn(r[1], n[1])), __dmul_rn(r[2], n[2]));
        const double b = sqrt(fmax(0.0, __dadd_rn(rr, -__dmul_rn(rn, rn)))) / F.R;
        int k = (int)(b / kSbMax * kNsb);
        out.sb = k > kNsb - 1 ? kNsb - 1 : k;
    }
    return out;
}

// The same, as an out-of-line call.
static __device__ __noinline__ EscapeBins escape_geometry_ool(const EscapeFrame& F, const int idx[3], unsigned bin,
                                                             unsigned face, unsigned long long pid,
                                                             unsigned long long e, uint32_t k0, uint32_t k1) {
    return escape_geometry(F, idx, bin, face, pid, e, k0, k1);
}

}  // namespace rddmc
