// redist.cu -- discrete frequency redistribution (Sec. 5.3, eq. R_discrete) for
// the frequency-grouped MC of the hybrid scheme, in FP64.
//
// R(x' -> x) is the angle-averaged redistribution of isotropic coherent
// scattering without recoil (Appendix A), proportional in x to
//   g(x; x') = int_zeta^inf e^{-u^2} [atan((x_min + u)/a) - atan((x_max - u)/a)] du,
// zeta = |x - x'|/2, x_max/min = max/min(x, x').  Row j' of eq. R_discrete,
// kept as cumulative probabilities at the interior edges e_1..e_{J-1}, is the
// average over x' in bin j' of F(e | x') = int_{-inf}^{e} g dx / int g dx (the
// normalisation by the total stands for the 1/(pi H(x')) of the density).
// Outgoing frequencies beyond the grid fall in the end bins.  The x' average
// takes n_sub Gauss-Legendre nodes of the incoming bin (uniform weight, the
// equation's 1/dx_j'); thresholds are round-half-even(C 2^32) saturated at
// 2^32 - 1, as for the leakage.
//
// Quadrature.  In x: pieces between x' - 14 and x' + 14 cut at the integers,
// at the bin edges (where F is read), at x' and at -x' (the kinks of g), 16
// Gauss-Legendre nodes each.  In u: up to zeta + 6; the two atan terms jump
// by pi across u = x_max and u = -x_min within a width a, so the u range is cut
// there and at a 4^k (k = 1..7) on either side, 8 nodes per piece.  One thread
// per (incoming bin, node) sweeps x once; a block per incoming bin averages
// its nodes in a fixed order (deterministic thresholds).
#include <cmath>

#include "grid.h"

namespace rddmc {
namespace {

constexpr int kMaxSub = 8;       // incoming-bin nodes
constexpr double kSpan = 14.0;   // x range around x'
constexpr double kUSpan = 6.0;   // u range above zeta

__device__ __forceinline__ void gl16(int i, double& x, double& w) {
    // 16-point Gauss-Legendre nodes and weights on [-1, 1] (positive half)
    const double X[8] = {0.0950125098376374, 0.2816035507792589, 0.4580167776572274, 0.6178762444026438,
                         0.7554044083550030, 0.8656312023878318, 0.9445750230732326, 0.9894009349916499};
    const double Wt[8] = {0.1894506104550685, 0.1826034150449236, 0.1691565193950025, 0.1495959888165767,
                          0.1246289712555339, 0.0951585116824928, 0.0622535239386479, 0.0271524594117541};
    const int k = i < 8 ? 7 - i : i - 8;
    x = i < 8 ? -X[k] : X[k];
    w = Wt[k];
}

__device__ __forceinline__ void gl8(int i, double& x, double& w) {
    const double X[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
    const double Wt[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};
    const int k = i < 4 ? 3 - i : i - 4;
    x = i < 4 ? -X[k] : X[k];
    w = Wt[k];
}

__device__ double u_piece(double lo, double hi, double xmin, double xmax, double a) {
    if (!(hi > lo)) return 0.0;
    const double h = 0.5 * (hi - lo), c = 0.5 * (hi + lo);
    double s = 0.0;
    for (int i = 0; i < 8; ++i) {
        double t, w;
        gl8(i, t, w);
        const double u = c + h * t;
        s += w * exp(-u * u) * (atan((xmin + u) / a) - atan((xmax - u) / a));
    }
    return s * h;
}

// g(x; x') by pieces of the u range: [zeta, zeta + 6] cut at the two jumps and
// geometrically around them.
__device__ double g_of(double x, double xp, double a) {
    const double xmax = fmax(x, xp), xmin = fmin(x, xp);
    const double z0 = 0.5 * fabs(x - xp), z1 = z0 + kUSpan;
    double cut[2 + 2 * 15];
    int n = 0;
    cut[n++] = z0;
    cut[n++] = z1;
    const double jumps[2] = {xmax, -xmin};
    for (int q = 0; q < 2; ++q) {
        const double p = jumps[q];
        if (p > z0 && p < z1) cut[n++] = p;
        double d = 4.0 * a;
        for (int k = 0; k < 7; ++k, d *= 4.0) {
            if (p - d > z0 && p - d < z1) cut[n++] = p - d;
            if (p + d > z0 && p + d < z1) cut[n++] = p + d;
        }
    }
    // insertion sort of the few cut points
    for (int i = 1; i < n; ++i) {
        const double v = cut[i];
        int j = i - 1;
        while (j >= 0 && cut[j] > v) { cut[j + 1] = cut[j]; --j; }
        cut[j + 1] = v;
    }
    double s = 0.0;
    for (int i = 0; i + 1 < n; ++i) s += u_piece(cut[i], cut[i + 1], xmin, xmax, a);
    return s;
}

__device__ double x_piece(double lo, double hi, double xp, double a) {
    if (!(hi > lo)) return 0.0;
    const double h = 0.5 * (hi - lo), c = 0.5 * (hi + lo);
    double s = 0.0;
    for (int i = 0; i < 16; ++i) {
        double t, w;
        gl16(i, t, w);
        s += w * g_of(c + h * t, xp, a);
    }
    return s * h;
}

// Block j' (incoming bin), thread q < n_sub (node): F(e_i | x'_q) for the J-1
// interior edges, into shared memory; then the node average, thresholds.
__global__ void redist_kernel(const double* __restrict__ edges, int J, double a, int n_sub,
                              uint32_t* __restrict__ thr) {
    extern __shared__ double sF[];  // n_sub x (J - 1)
    const int jp = blockIdx.x;
    const int q = threadIdx.x;
    double gxn[kMaxSub], gwn[kMaxSub];
    // Gauss-Legendre nodes of order n_sub by Newton iteration on P_n
    for (int i = 0; i < n_sub; ++i) {
        double z = cos(3.14159265358979323846 * (i + 0.75) / (n_sub + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n_sub; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n_sub == 1) { p1 = z; p0 = 1.0; }
            dp = n_sub * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-15) break;
        }
        gxn[i] = z;
        gwn[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    if (n_sub == 1) { gxn[0] = 0.0; gwn[0] = 2.0; }
    if (q < n_sub) {
        const double lo_b = edges[jp], hi_b = edges[jp + 1];
        const double xp = 0.5 * (hi_b - lo_b) * gxn[q] + 0.5 * (hi_b + lo_b);
        const double lo = xp - kSpan, hi = xp + kSpan;
        // sweep x from lo to hi: cut points are the integers, the edges, x', -x'
        double x = lo, cum = 0.0;
        int ie = 1;  // next interior edge to record
        while (ie < J && edges[ie] <= lo) sF[q * (J - 1) + (ie++ - 1)] = 0.0;
        for (int guard = 0; guard < 4 * (J + 64) && x < hi; ++guard) {
            double nx = fmin(hi, floor(x) + 1.0);
            if (ie < J && edges[ie] > x && edges[ie] < nx) nx = edges[ie];
            if (xp > x && xp < nx) nx = xp;
            if (-xp > x && -xp < nx) nx = -xp;
            cum += x_piece(x, nx, xp, a);
            x = nx;
            while (ie < J && edges[ie] <= x) sF[q * (J - 1) + (ie++ - 1)] = cum;
        }
        while (ie < J) sF[q * (J - 1) + (ie++ - 1)] = cum;
        const double inv = cum > 0.0 ? 1.0 / cum : 0.0;
        for (int i = 0; i < J - 1; ++i) sF[q * (J - 1) + i] *= inv;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < J - 1; i += blockDim.x) {
        double C = 0.0;
        for (int k = 0; k < n_sub; ++k) C += 0.5 * gwn[k] * sF[k * (J - 1) + i];
        double t = rint(C * 4294967296.0);
        t = fmin(fmax(t, 0.0), 4294967295.0);
        thr[(size_t)jp * (J - 1) + i] = (uint32_t)t;
    }
}

}  // namespace
}  // namespace rddmc

extern "C" uint64_t rddmc_redistribution_bytes(const rddmc_grid* g) {
    if (!g || g->J < 2) return 0;
    return rddmc::align256((uint64_t)g->J * (uint64_t)(g->J - 1) * 4ull);
}

extern "C" int rddmc_precompute_redistribution(const rddmc_grid* g, const void* d_table, int n_sub, void* d_redist,
                                               size_t bytes, void* stream) {
    using namespace rddmc;
    if (!g || !d_table || !d_redist || ((uintptr_t)d_table & 255u) || ((uintptr_t)d_redist & 3u)) return RDDMC_ERR_ARG;
    if (n_sub < 1 || n_sub > kMaxSub || g->J < 2) return RDDMC_ERR_ARG;
    if (bytes < (size_t)g->J * (size_t)(g->J - 1) * 4u) return RDDMC_ERR_SIZE;
    if (!g->precomputed) return RDDMC_ERR_TABLE;  // the bin edges are read from the table
    const size_t smem = (size_t)n_sub * (size_t)(g->J - 1) * 8u;
    if (smem > 200u * 1024u) return RDDMC_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    const double* edges = (const double*)((const char*)d_table + g->off_edges);
    if (cudaFuncSetAttribute(redist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return RDDMC_ERR_CUDA;
    redist_kernel<<<(unsigned)g->J, 32, smem, s>>>(edges, g->J, g->a, n_sub, (uint32_t*)d_redist);
    return cudaGetLastError() == cudaSuccess ? RDDMC_OK : RDDMC_ERR_CUDA;
}
