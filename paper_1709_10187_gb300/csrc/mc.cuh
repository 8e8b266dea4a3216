// mc.cuh -- FP32 building blocks of the continuous MC of the hybrid scheme
// (Sec. 5.1, Sec. 5.2): the Voigt profile, the parallel atom velocity of a
// scattering, coherent isotropic scattering, and an event-stream reader.
#pragma once
#include <cuda_runtime.h>

#include "rddmc_internal.cuh"

namespace rddmc {

// Reader of a packet's event stream (lane e&3 of Philox4x32-10 keyed by
// (e>>2, packet | 2^63)), holding the current four-word block.
struct EventStream {
    unsigned long long pid, e, blk;
    uint4 buf;
    uint32_t k0, k1;
    __device__ __forceinline__ void init(unsigned long long p, unsigned long long e0, uint32_t a, uint32_t b) {
        pid = p; e = e0; blk = ~0ull; k0 = a; k1 = b;
    }
    __device__ __forceinline__ unsigned next() {
        const unsigned long long b = e >> 2;
        if (b != blk) {
            buf = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)(b >> 32), (uint32_t)pid,
                                           (uint32_t)(pid >> 32) | 0x80000000u), k0, k1);
            blk = b;
        }
        const unsigned l = (unsigned)e & 3u;
        ++e;
        return l == 0 ? buf.x : (l == 1 ? buf.y : (l == 2 ? buf.z : buf.w));
    }
    // uniform in (0,1) from the top 24 bits
    __device__ __forceinline__ float u01() { return ((float)(next() >> 8) + 0.5f) * 5.9604645e-8f; }
};

// Dawson integral in FP32: power series near 0, asymptotic series beyond 10,
// Rybicki's sampling series (h = 0.4, aliasing error ~ e^{-(pi/2h)^2} ~ 2e-7)
// between.
__device__ __forceinline__ float dawson_f32(float x) {
    const float ax = fabsf(x);
    float r;
    if (ax < 0.2f) {
        const float x2 = ax * ax;
        r = ax * (1.0f - x2 * (0.6666667f - x2 * (0.26666668f - x2 * 0.07619048f)));
    } else if (ax > 10.0f) {
        const float i2 = 1.0f / (ax * ax);
        r = 0.5f / ax * (1.0f + i2 * (0.5f + i2 * (0.75f + i2 * 1.875f)));
    } else {
        const float h = 0.4f;
        const float n0 = 2.0f * rintf(ax / (2.0f * h));
        const float xp = ax - n0 * h;
        float s = 0.0f;
#pragma unroll
        for (int i = 6; i >= 0; --i) {
            const float m = (float)(2 * i + 1);
            const float dp = xp - m * h, dm = xp + m * h;
            s += __expf(-dp * dp) / (n0 + m) + __expf(-dm * dm) / (n0 - m);
        }
        r = s * 0.5641896f;
    }
    return x < 0.0f ? -r : r;
}

// H(a,x) to second order in a (eq. H_approx); beyond |x| = 10 the combination
// 2xF(x) - 1 is taken from its asymptotic series to avoid cancellation.
__device__ __forceinline__ float voigt_H_f32(float a, float x) {
    const float ax = fabsf(x);
    const float g = ax < 10.0f ? __expf(-x * x) : 0.0f;
    float q;  // 2 x F(x) - 1
    if (ax > 10.0f) {
        const float i2 = 1.0f / (ax * ax);
        q = i2 * (0.5f + i2 * (0.75f + i2 * (1.875f + i2 * 6.5625f)));
    } else {
        q = 2.0f * x * dawson_f32(x) - 1.0f;
    }
    return g + 1.1283792f * a * q + a * a * g * (1.0f - 2.0f * x * x);
}

// Parallel atom velocity u for a scattering at frequency x: density
// e^{-u^2} / (a^2 + (x-u)^2), by rejection from the three-part envelope whose
// split points (u1, u0) are tabulated per |x|.  The Lorentzian pieces are
// sampled in phi = atan(a / (x - u)) (u = x - a / tan(phi)), which stays
// accurate in FP32 far from resonance.
__device__ __noinline__ float sample_upar(float a, float xin, const float2* __restrict__ tab, EventStream& es) {
    const float x = fabsf(xin);
    const int i = min((int)(x * 16.0f), kUparN - 1);
    const float2 t = tab[i];
    const float u1 = t.x, u0 = fminf(t.y, x);
    const float d1 = x - u1, d0 = x - u0;
    const float g1 = 1.0f / (a * a + d1 * d1);
    const float phi1 = atanf(a / d1);
    const float phi0 = d0 > 0.0f ? atanf(a / d0) : 1.5707964f;
    const float c2 = u1 <= 0.0f ? 1.0f : __expf(-u1 * u1);
    const float w1 = g1 * 0.8862269f * (1.0f + erff(u1));
    const float w2 = c2 * (phi0 - phi1) / a;
    const float w3 = __expf(-u0 * u0) * (3.1415927f - phi0) / a;
    const float sig = 0.70710678f;
    for (int it = 0; it < 1000000; ++it) {
        const float pick = es.u01() * (w1 + w2 + w3);
        float u, acc;
        if (pick < w1) {
            if (u1 >= 0.0f) {  // the Gaussian below u1 >= 0: at least half of it
                u = u1 - 1.0f;
                for (int k = 0; k < 4096; ++k) {
                    const float r1 = es.u01(), r2 = es.u01();
                    const float g = sig * sqrtf(-2.0f * __logf(r1)) * cospif(2.0f * r2);
                    if (g < u1) { u = g; break; }
                }
            } else {  // Marsaglia's tail method beyond c = -u1/sigma
                const float c = -u1 / sig;
                float X = c;
                for (int k = 0; k < 4096; ++k) {
                    const float r1 = es.u01(), r2 = es.u01();
                    const float Xk = sqrtf(c * c - 2.0f * __logf(r1));
                    if (r2 * Xk < c) { X = Xk; break; }
                }
                u = -sig * X;
            }
            const float du = x - u;
            acc = (1.0f / (a * a + du * du)) / g1;
        } else if (pick < w1 + w2) {
            const float ph = phi1 + es.u01() * (phi0 - phi1);
            u = x - a / tanf(ph);
            acc = __expf(-u * u) / c2;
        } else {
            const float ph = phi0 + es.u01() * (3.1415927f - phi0);
            u = x - a / tanf(ph);
            acc = __expf(u0 * u0 - u * u);
        }
        if (es.u01() < acc) return xin < 0.0f ? -u : u;
    }
    return xin;
}

__device__ __forceinline__ void iso_dir(EventStream& es, float n[3]) {
    const float mu = 2.0f * es.u01() - 1.0f;
    float sp, cp;
    sincospif(2.0f * es.u01(), &sp, &cp);
    const float st = sqrtf(fmaxf(0.0f, 1.0f - mu * mu));
    n[0] = st * cp;
    n[1] = st * sp;
    n[2] = mu;
}

// Direction uniform over the half-space around side * e_ax.
__device__ __forceinline__ void half_dir(EventStream& es, int ax, int side, float n[3]) {
    const float mu = 1.0f - es.u01();
    float sp, cp;
    sincospif(2.0f * es.u01(), &sp, &cp);
    const float st = sqrtf(fmaxf(0.0f, 1.0f - mu * mu));
    n[ax] = (float)side * mu;
    n[(ax + 1) % 3] = st * cp;
    n[(ax + 2) % 3] = st * sp;
}

// Coherent isotropic scattering without recoil:
// x' = x + u_par (mu - 1) + u_perp sqrt(1 - mu^2), u_perp ~ N(0, 1/2), mu = n.n'.
__device__ __forceinline__ float scatter(float a, float x, float n[3], const float2* tab, EventStream& es) {
    const float up = sample_upar(a, x, tab, es);
    const float r1 = es.u01(), r2 = es.u01();
    const float uperp = 0.70710678f * sqrtf(-2.0f * __logf(r1)) * cospif(2.0f * r2);
    float nn[3];
    iso_dir(es, nn);
    float mu = n[0] * nn[0] + n[1] * nn[1] + n[2] * nn[2];
    mu = fminf(1.0f, fmaxf(-1.0f, mu));
    n[0] = nn[0]; n[1] = nn[1]; n[2] = nn[2];
    return x + up * (mu - 1.0f) + uperp * sqrtf(1.0f - mu * mu);
}

}  // namespace rddmc
