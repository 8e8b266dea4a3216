// precompute.cu -- FP64 leakage-table kernels (Sec. 2.2, Sec. 2.5, Sec. 5.1).
//
// Kernel 1: phi[j] = bin mean of H(a,x) over bin j (k_ij = k0_i phi_j).
// Kernel 2: one thread per (class, bin) row: leakage coefficients of
//   eq. x-leakage and eq. z-leakage, the boundary / thin-neighbour form
//   2/(3 dz (k dz + 2 lambda)), probabilities p_X = k_X / sum k accumulated in
//   outcome order, 32-bit thresholds round-half-even(C 2^32) saturated at
//   2^32 - 1, the flag word (2-bit action per outcome, moving, thin) and the
//   mean dwell path 1 / sum_X k_X of the state.  Grey dust (Sec. 2.6): k_s adds
//   to every k_ij; k_a is one more outcome after the leakage ones.
// FP64 throughout: 1 - p of thick states and far-wing bin means (dcalH ~ a dx /
// (sqrt(pi) x^2) ~ 1e-8 against calH ~ 0.886) are below FP32 resolution.  This
// file is compiled without fused multiply-adds so every product and sum is
// rounded as written.
#include <cstring>

#include "grid.h"
#include "voigt.cuh"

namespace rddmc {
namespace {

__global__ void phi_kernel(const double* __restrict__ edges, double* __restrict__ phi, int J, double a) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= J) return;
    phi[j] = voigt_bin_mean_f64(a, edges[j], edges[j + 1]);
}

__device__ __forceinline__ uint32_t quantise_dev(double C) {
    double t = rint(C * 4294967296.0);
    t = fmax(t, 0.0);
    t = fmin(t, 4294967295.0);
    return (uint32_t)t;
}

template <int NDIM>
__global__ void rows_kernel(const TableHeader h, const ClassDesc* __restrict__ cdesc,
                            const double* __restrict__ edges, const double* __restrict__ phi,
                            uint32_t* __restrict__ rows, uint2* __restrict__ fast, float* __restrict__ tau_row,
                            float* __restrict__ rk, uint32_t* __restrict__ abs_thr, int dusty,
                            unsigned long long* __restrict__ wq, float* __restrict__ ka_row, int weighted,
                            int64_t nrow) {
    constexpr int K = 2 + 2 * NDIM;
    constexpr int W = NDIM == 1 ? 4 : 8;  // words per row, the last holding the flags
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrow) return;
    const int J = h.J;
    const int cls = (int)(r / J);
    const int j = (int)(r - (int64_t)cls * J);
    const ClassDesc& D = cdesc[cls];
    const bool hybrid = h.mode == RDDMC_MODE_HYBRID;
    double dzmin = h.dz[0];
    for (int ax = 1; ax < NDIM; ++ax) dzmin = fmin(dzmin, h.dz[ax]);

    const double dxj = edges[j + 1] - edges[j];
    const double k = D.k0 * phi[j] + D.ks;  // dust scattering adds to every k_ij (Sec. 2.6)
    double rate[K];
    uint32_t act[K];
    // frequency leakage, eq. x-leakage; zero flux beyond the grid ends
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
        const int jn = j + (sd ? 1 : -1);
        if (jn < 0 || jn >= J) { rate[sd] = 0.0; act[sd] = ACT_MOVE; continue; }
        const double dxn = edges[jn + 1] - edges[jn];
        const double kn = D.k0 * phi[jn] + D.ks;
        rate[sd] = 1.0 / (dxj * (dxj / k + dxn / kn));
        act[sd] = (hybrid && kn * dzmin < h.tau_ddmc) ? ACT_TO_MC : ACT_MOVE;
    }
    // spatial leakage, eq. z-leakage; exterior faces and thin neighbours use the
    // extrapolation-distance form of Sec. 5.1
#pragma unroll
    for (int ax = 0; ax < NDIM; ++ax) {
        const double dz = h.dz[ax];
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
            const int o = 2 + 2 * ax + sd;
            const FaceDesc& F = D.face[2 * ax + sd];
            const double r_bnd = 1.0 / (3.0 * dz) * 2.0 / (k * dz + 2.0 * h.lambda);
            if (F.exterior) { rate[o] = r_bnd; act[o] = ACT_ESCAPE; continue; }
            // neighbour opacity over the Doppler-shifted bin (eq. velocity-shift)
            const double knb = F.k0_nb * (F.delta == 0.0 ? phi[j]
                                                         : voigt_bin_mean_f64(h.a, edges[j] + F.delta,
                                                                              edges[j + 1] + F.delta)) +
                               F.ks_nb;
            const double dznb = dz;
            if (hybrid && knb * dznb < h.tau_ddmc) { rate[o] = r_bnd; act[o] = ACT_TO_MC; continue; }
            rate[o] = 1.0 / (3.0 * dz) * 2.0 / (k * dz + knb * dznb);
            act[o] = F.delta != 0.0 ? ACT_REBIN : ACT_MOVE;
        }
    }
    double tot = 0.0;
#pragma unroll
    for (int o = 0; o < K; ++o) tot += rate[o];
    // dust absorption: one more competing process, the last outcome; its lower
    // threshold (the end of the last leakage outcome) is stored apart
    if (dusty) tot += D.ka;
    uint32_t out[W - 1];
    double C = 0.0;
#pragma unroll
    for (int o = 0; o < K - 1; ++o) {
        C += rate[o] / tot;
        out[o] = quantise_dev(C);
    }
    abs_thr[r] = dusty ? quantise_dev(C + rate[K - 1] / tot) : 0xffffffffu;
    // weight method: -ln of the weight kept over one dwell, ln(1 + k_a / K_s),
    // in 2^-40 units (the walk sums these exactly)
    wq[r] = weighted ? (unsigned long long)llrint(log1p(D.ka / tot) * 1099511627776.0) : 0ull;
    ka_row[r] = weighted ? (float)D.ka : 0.0f;  // the time walk attenuates by exp(-k_a l)
    uint32_t fl = 0;
#pragma unroll
    for (int o = 0; o < K; ++o) fl |= (act[o] & 3u) << (2 * o);
    if (act[0] == ACT_MOVE && act[1] == ACT_MOVE) fl |= FLAG_FASTX;
    if (D.moving) fl |= FLAG_MOVING;
    if (hybrid && k * dzmin < h.tau_ddmc) fl |= FLAG_THIN;
    // word order: thr0, thr1, thr2, flags[, thr3..thr6] so that the first 16
    // bytes carry everything a frequency move needs
    fast[r] = make_uint2(out[0], (fl & FLAG_FASTX) ? out[1] : 0u);
    tau_row[r] = (float)(k * dzmin);
    rk[r] = (float)(1.0 / tot);  // mean dwell path 1 / K_s of the state (time-dependent walk)
    if (NDIM == 1) {
        reinterpret_cast<uint4*>(rows)[r] = make_uint4(out[0], out[1], out[2], fl);
    } else {
        uint4* p = reinterpret_cast<uint4*>(rows) + 2 * r;
        p[0] = make_uint4(out[0], out[1], out[2], fl);
        p[1] = make_uint4(out[3], out[4], out[5], out[6]);
    }
}

// Split points (u1, u0) of the three-part rejection envelope of the parallel
// atom velocity, f(u) = e^{-u^2} / (a^2 + (x-u)^2) (Sec. 5.2), for |x| = i/16:
//   u < u1: e^{-u^2} g(u1);  u1 <= u <= u0: c g(u), c = max e^{-u^2} on [u1,u0];
//   u > u0: e^{-u0^2} g(u),  g(u) = 1/(a^2 + (x-u)^2),  u1 <= u0 <= x, u0 >= 0.
// Each piece bounds f, so any such pair samples f exactly; the pair with the
// smallest envelope mass on a grid of candidates gives the best acceptance.
__global__ void upar_kernel(float2* __restrict__ tab, double a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kUparN) return;
    const double x = (double)i / 16.0;
    double best = 1e300, b1 = -30.0, b0 = 0.0;
    for (int p = 0; p <= 32; ++p) {
        const double u0 = x * p / 32.0;
        const double th0 = atan((u0 - x) / a);
        const double m3 = exp(-u0 * u0) * (1.5707963267948966 - th0) / a;
        for (int q = 0; q <= 33; ++q) {
            const double u1 = (q == 33) ? -30.0 : -4.0 + (u0 + 4.0) * q / 32.0;
            const double g1 = 1.0 / (a * a + (x - u1) * (x - u1));
            const double m1 = g1 * 0.88622692545275801365 * (1.0 + erf(u1));
            const double c = u1 <= 0.0 ? 1.0 : exp(-u1 * u1);
            const double m2 = c * (th0 - atan((u1 - x) / a)) / a;
            const double m = m1 + m2 + m3;
            if (m < best) { best = m; b1 = u1; b0 = u0; }
        }
    }
    tab[i] = make_float2((float)b1, (float)fmin(b0, x));
}

}  // namespace

cudaError_t launch_precompute(const rddmc_grid& g, void* d_table, cudaStream_t s) {
    char* base = (char*)d_table;
    const double* edges = (const double*)(base + g.off_edges);
    double* phi = (double*)(base + g.off_phi);
    phi_kernel<<<(g.J + 127) / 128, 128, 0, s>>>(edges, phi, g.J, g.a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    TableHeader h;
    std::memset(&h, 0, sizeof(h));
    h.J = g.J;
    h.mode = g.params.mode;
    h.tau_ddmc = g.params.tau_ddmc;
    h.lambda = g.params.lambda;
    h.f_mu = g.params.f_mu;
    h.a = g.a;
    for (int a = 0; a < 3; ++a) h.dz[a] = 2.0 * g.R / g.n[a];
    const int64_t nrow = (int64_t)g.n_class * g.J;
    const int threads = 128;
    const int64_t blocks = (nrow + threads - 1) / threads;
    const ClassDesc* cd = (const ClassDesc*)(base + g.off_cdesc);
    uint32_t* rows = (uint32_t*)(base + g.off_rows);
    uint2* fast = (uint2*)(base + g.off_fast);
    float* tau_row = (float*)(base + g.off_tau);
    float* rk = (float*)(base + g.off_rk);
    uint32_t* abs_thr = (uint32_t*)(base + g.off_abs);
    const int dusty = g.dusty() ? 1 : 0;
    unsigned long long* wq = (unsigned long long*)(base + g.off_wq);
    const int weighted = g.weighted() ? 1 : 0;
    float* ka_row = (float*)(base + g.off_ka);
    if (g.ndim == 1)
        rows_kernel<1><<<(unsigned)blocks, threads, 0, s>>>(h, cd, edges, phi, rows, fast, tau_row, rk, abs_thr,
                                                            dusty, wq, ka_row, weighted, nrow);
    else
        rows_kernel<3><<<(unsigned)blocks, threads, 0, s>>>(h, cd, edges, phi, rows, fast, tau_row, rk, abs_thr,
                                                            dusty, wq, ka_row, weighted, nrow);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the u_par envelope table serves only the continuous MC of the hybrid scheme
    if (g.params.mode == RDDMC_MODE_HYBRID)
        upar_kernel<<<(kUparN + 127) / 128, 128, 0, s>>>((float2*)(base + g.off_upar), g.a);
    return cudaGetLastError();
}

}  // namespace rddmc
