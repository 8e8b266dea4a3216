// voigt.cuh -- device line-profile functions (Sec. 2.1, Sec. 2.2) in FP64.
//
// dawson_f64: F(x) = int_0^x exp(y^2 - x^2) dy.  |x| < 0.5: its power series
//   F(x) = sum_k (-2)^k x^(2k+1) / (2k+1)!!.  Elsewhere Rybicki's (1989,
//   Computers in Physics 3(2)) series F(x) ~ pi^-1/2 sum_{n odd} e^{-(x-nh)^2}/n,
//   re-centred on the even multiple n0 of h closest to x; here h = 1/4 (aliasing
//   error ~ e^{-(2 pi)^2} ~ 7e-18 relative), 34 odd terms on each side summed
//   from the smallest.
// voigt_hint_diff_f64: calH(a, hi) - calH(a, lo) with
//   calH(a,x) = (sqrt(pi)/2) erf x - (2a/sqrt(pi)) F(x) + a^2 x e^{-x^2}
//   (integral of eq. H_approx); the erf difference is taken from erfc on the
//   side away from line centre.
#pragma once
#include <cuda_runtime.h>

namespace rddmc {

__device__ __forceinline__ double dawson_f64(double x) {
    const double ax = fabs(x);
    double res;
    if (ax < 0.5) {
        const double x2 = ax * ax;
        double term = ax, sum = ax;
        for (int k = 1; k < 30; ++k) {
            term = term * (-2.0 * x2) / (double)(2 * k + 1);
            sum += term;
        }
        res = sum;
    } else {
        const double h = 0.25;
        const double n0 = 2.0 * rint(ax / (2.0 * h));
        const double xp = ax - n0 * h;                 // |xp| <= h
        // pairs n' = +m and n' = -m for odd m = 1, 3, ..., 67
        double sum = 0.0;
        for (int i = 33; i >= 0; --i) {
            const double m = (double)(2 * i + 1);
            const double dp = xp - m * h, dm = xp + m * h;
            sum += exp(-dp * dp) / (n0 + m) + exp(-dm * dm) / (n0 - m);
        }
        res = sum * 0.56418958354775628695;            // 1/sqrt(pi)
    }
    return x < 0.0 ? -res : res;
}

__device__ __forceinline__ double voigt_hint_diff_f64(double a, double lo, double hi) {
    double derf;
    if (lo >= 0.0)
        derf = erfc(lo) - erfc(hi);
    else if (hi <= 0.0)
        derf = erfc(-hi) - erfc(-lo);
    else
        derf = erf(hi) - erf(lo);
    const double dF = dawson_f64(hi) - dawson_f64(lo);
    const double dG = hi * exp(-hi * hi) - lo * exp(-lo * lo);
    return 0.88622692545275801365 * derf - 2.0 * a * 0.56418958354775628695 * dF + a * a * dG;
}

// Bin mean of H over [lo, hi] (k_j / k0 of Sec. 2.2).
__device__ __forceinline__ double voigt_bin_mean_f64(double a, double lo, double hi) {
    return voigt_hint_diff_f64(a, lo, hi) / (hi - lo);
}

}  // namespace rddmc
