/*
 * rddmc_oracle.c -- FP64 CPU oracle for resonant discrete diffusion Monte Carlo
 * (Smith, Tsang, Bromm & Milosavljevic 2017, "Discrete diffusion Lyman alpha
 * radiative transfer").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call this
 * file: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code, header or constant table with the CUDA
 * library; the two are written independently from the paper.
 *
 * Everything here is plain, slow, double precision and follows the paper's
 * order of operations:
 *   - Dawson integral F(x): Maclaurin series near 0, Rybicki's (1989,
 *     Computers in Physics 3(2), 85) sampling-theorem series elsewhere.
 *   - Hjerting-Voigt H(a,x) to second order in a, and its integral calH(a,x)
 *     (Sec. 2.2, eq. H_approx and the integrated form below it).
 *   - bin-mean opacity k_j = k0 (calH(x_j+) - calH(x_j-)) / dx_j (Sec. 2.2).
 *   - leakage coefficients eq. z-leakage, eq. x-leakage; the hybrid
 *     DDMC->MC boundary coefficient with extrapolation distance lambda (Sec. 5.1);
 *     the comoving Doppler shift of bin edges across faces, eq. velocity-shift.
 *   - Philox4x32-10 (Salmon, Moraes, Dror & Shaw 2011, SC'11).
 *   - the DDMC walk of Sec. 2.3: the leakage with the smallest sampled distance
 *     is executed.  Two forms are provided: the literal competing exponentials
 *     (eq. l_min_1, l_min_2) and the equivalent categorical draw on quantised
 *     cumulative probabilities, which defines the random-stream contract shared
 *     (as a specification, not as code) with the GPU walk.
 *
 * Random-stream contract (fixed by this project; not in the paper):
 *   key = (seed_lo, seed_hi).  Each packet p (< 2^63) owns two streams of 32-bit
 *   words, selected by the top bit of the last counter word:
 *     transition stream: transition t of p uses lane t&3 of
 *       Philox4x32-10(ctr = ((t>>2)_lo, (t>>2)_hi, p_lo, p_hi), key);
 *     event stream: event draw e of p uses lane e&3 of
 *       Philox4x32-10(ctr = ((e>>2)_lo, (e>>2)_hi, p_lo, p_hi | 2^31), key).
 *   Event draw 0 picks the source cell/bin; a Doppler rebin takes the next event
 *   draw; a DDMC escape takes five (face point 2, mu, phi, x in bin) in 3D or
 *   from a moving slab cell, none from a static slab cell.  A uniform in (0,1)
 *   is (w + 0.5) * 2^-32.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define ORC_SQRTPI 1.77245385090551602730
#define ORC_TWO32 4294967296.0

/* ------------------------------------------------------------------------- */
/* Physics (Sec. 2.1, Sec. 2.2)                                               */
/* ------------------------------------------------------------------------- */

/* Damping parameter a = 4.702e-4 * (T / 1e4 K)^(-1/2)  (Sec. 2.1). */
double orc_damping(double T) { return 4.702e-4 / sqrt(T / 1.0e4); }

/* Dawson integral F(x) = int_0^x exp(y^2 - x^2) dy.
 * |x| < 0.2: Maclaurin series F(x) = sum_n (-1)^n 2^n x^(2n+1) / (2n+1)!!.
 * otherwise: Rybicki (1989): F(x) = lim_{h->0} pi^(-1/2) sum_{n odd} e^{-(x-nh)^2}/n,
 * re-centred on the even multiple n0 of h nearest to x, h = 0.2 (aliasing error
 * ~ exp(-(pi/2h)^2) ~ 1e-27), terms with |n'| h <= 8.2 kept. */
double orc_dawson(double x) {
    double ax = fabs(x), sgn = (x < 0.0) ? -1.0 : 1.0;
    if (ax < 0.2) {
        double x2 = ax * ax, term = ax, sum = ax;
        for (int n = 1; n < 40; ++n) {
            term *= -2.0 * x2 / (2.0 * n + 1.0);
            sum += term;
            if (fabs(term) < 1e-18 * fabs(sum)) break;
        }
        return sgn * sum;
    }
    const double h = 0.2;
    const int N = 41;
    long n0 = 2L * lround(ax / (2.0 * h));
    double xp = ax - (double)n0 * h;
    double sum = 0.0;
    for (int k = -N; k <= N; ++k) {
        long np = 2L * k + 1L;
        long den = np + n0;
        if (den == 0) continue;
        double d = xp - (double)np * h;
        sum += exp(-d * d) / (double)den;
    }
    return sgn * sum / ORC_SQRTPI;
}

/* H(a,x) to second order in a (eq. H_approx). */
double orc_voigt_H(double a, double x) {
    double e = exp(-x * x);
    return e + 2.0 * a / ORC_SQRTPI * (2.0 * x * orc_dawson(x) - 1.0) + a * a * e * (1.0 - 2.0 * x * x);
}

/* calH(a,x) = int_0^x H(a,y) dy = (sqrt(pi)/2) erf(x) - (2a/sqrt(pi)) F(x) + a^2 x e^{-x^2}. */
double orc_voigt_Hint(double a, double x) {
    return 0.5 * ORC_SQRTPI * erf(x) - 2.0 * a / ORC_SQRTPI * orc_dawson(x) + a * a * x * exp(-x * x);
}

/* Bin mean of H over [xlo, xhi]: (calH(xhi) - calH(xlo)) / (xhi - xlo).
 * The erf difference is formed from erfc on the side away from line centre,
 * where erf(x) -> 1 would cancel in double precision. */
double orc_bin_mean_H(double a, double xlo, double xhi) {
    double derf;
    if (xlo >= 0.0)
        derf = erfc(xlo) - erfc(xhi);
    else if (xhi <= 0.0)
        derf = erfc(-xhi) - erfc(-xlo);
    else
        derf = erf(xhi) - erf(xlo);
    double dF = orc_dawson(xhi) - orc_dawson(xlo);
    double dG = xhi * exp(-xhi * xhi) - xlo * exp(-xlo * xlo);
    return (0.5 * ORC_SQRTPI * derf - 2.0 * a / ORC_SQRTPI * dF + a * a * dG) / (xhi - xlo);
}

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al. 2011)                                        */
/* ------------------------------------------------------------------------- */

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Word n of stream `which` (0 transitions, 1 events) of packet p (see the
 * contract in the header comment). */
static uint32_t orc_word(uint64_t seed, uint64_t p, int which, uint64_t n) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint64_t b = n >> 2;
    uint32_t ctr[4] = {(uint32_t)b, (uint32_t)(b >> 32), (uint32_t)p,
                       (uint32_t)(p >> 32) | (which == 1 ? 0x80000000u : (which == 2 ? 0x40000000u : 0u))};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[n & 3];
}
#define ORC_TRANS 0
#define ORC_EVENT 1
#define ORC_TIME 2   /* dwell draws of the time-dependent walk (packet ids < 2^62) */

static double orc_unif(uint32_t w) { return ((double)w + 0.5) / ORC_TWO32; }

/* ------------------------------------------------------------------------- */
/* Grid and leakage table (Sec. 2.2, Sec. 2.5, Sec. 5.1)                      */
/* ------------------------------------------------------------------------- */

typedef struct orc_grid {
    int32_t ndim;     /* 1: slab (axis 0 only), 3: Cartesian cube */
    int32_t n[3];     /* cells per axis; unused axes hold 1 */
    int32_t J;        /* frequency bins */
    int32_t hybrid;   /* 0: DDMC in every state; 1: thin states hand off to MC */
    double R;         /* half-width of the domain [-R, R]^ndim */
    double tau0;      /* k0 * R for unit density */
    double T;         /* gas temperature (K), isothermal */
    double tau_ddmc;  /* thick threshold on tau_ij = k_ij dz */
    double lambda;    /* extrapolation distance of the DDMC->MC coefficient */
    double f_mu;      /* flux directionality factor of eq. velocity-shift */
    const double* edges;  /* J+1 ascending comoving frequency edges */
    const double* n_rel;  /* per-cell density scale, NULL = 1 */
    const double* v;      /* per-cell bulk velocity in km/s, 3 per cell, NULL = static */
    const uint8_t* mask;  /* per-cell 1 = medium, 0 = vacuum, NULL = all medium */
    double dust_abs;      /* dust absorption k_a R at unit density (grey; Sec. 2.6), 0 = none */
    double dust_scat;     /* dust scattering k_s R at unit density (grey), added to k_ij */
    const uint32_t* redist; /* hybrid only: frequency-grouped MC (Sec. 5.3) with these cumulative
                               thresholds of eq. R_discrete, J rows of J-1; NULL = continuous MC */
    int32_t dust_weights; /* 1: continuous absorption (Sec. 2.6): no absorption outcome; the
                             packet weight is multiplied by K_s / (K_s + k_a) per transition */
    int32_t pad;
} orc_grid;

/* Actions stored two bits per outcome in the flags word. */
#define ORC_ACT_MOVE 0u
#define ORC_ACT_ESCAPE 1u
#define ORC_ACT_TO_MC 2u
#define ORC_ACT_REBIN 3u
#define ORC_FLAG_MOVING (1u << 30) /* the cell has non-zero bulk velocity */
#define ORC_FLAG_THIN (1u << 31)   /* hybrid mode: the state is an MC state */

static int64_t orc_ncell(const orc_grid* g) { return (int64_t)g->n[0] * g->n[1] * g->n[2]; }
static int orc_nout(const orc_grid* g) { return 2 + 2 * g->ndim; }
/* Dust absorption is one more outcome, K = orc_nout, after the leakage
 * outcomes: thresholds per state orc_nthr = K - 1 (+1 with absorption). */
static int orc_dusty(const orc_grid* g) { return g->dust_abs > 0.0 && !g->dust_weights; }
#define ORC_W_MIN 1e-10  /* packets below this weight are eliminated (Sec. 2.6) */
static int orc_nthr(const orc_grid* g) { return orc_nout(g) - 1 + orc_dusty(g); }

static int orc_in_medium(const orc_grid* g, const int idx[3]) {
    for (int a = 0; a < 3; ++a)
        if (idx[a] < 0 || idx[a] >= g->n[a]) return 0;
    int64_t c = idx[0] + (int64_t)g->n[0] * (idx[1] + (int64_t)g->n[1] * idx[2]);
    return g->mask ? (g->mask[c] != 0) : 1;
}

static int64_t orc_cell_of(const orc_grid* g, const int idx[3]) {
    return idx[0] + (int64_t)g->n[0] * (idx[1] + (int64_t)g->n[1] * idx[2]);
}

static void orc_idx_of(const orc_grid* g, int64_t c, int idx[3]) {
    idx[0] = (int)(c % g->n[0]);
    idx[1] = (int)((c / g->n[0]) % g->n[1]);
    idx[2] = (int)(c / ((int64_t)g->n[0] * g->n[1]));
}

/* Line-centre absorption coefficient k0 of cell c (tau0 = k0 R at unit density). */
static double orc_k0(const orc_grid* g, int64_t c) {
    return g->tau0 / g->R * (g->n_rel ? g->n_rel[c] : 1.0);
}

static double orc_dz(const orc_grid* g, int axis) { return 2.0 * g->R / g->n[axis]; }

/* Thermal velocity v_th = 12.85 (T/1e4 K)^(1/2) km/s (Sec. 2.1). */
static double orc_vth(const orc_grid* g) { return 12.85 * sqrt(g->T / 1.0e4); }

/* Comoving frequency shift for crossing from cell c to cell nb through the face
 * with unit normal +/- e_axis: x' = x + f_mu n.(v_c - v_nb)/v_th, the
 * isothermal form of eq. velocity-shift. */
static double orc_face_shift(const orc_grid* g, int64_t c, int64_t nb, int axis, int side) {
    if (!g->v) return 0.0;
    double dv = g->v[3 * c + axis] - g->v[3 * nb + axis];
    return g->f_mu * (double)side * (dv / orc_vth(g));
}

/* Quantise a cumulative probability to a 32-bit threshold: round half to even
 * of C * 2^32, saturating at 2^32 - 1 so that the last outcome always keeps at
 * least one count. */
static uint32_t orc_quantise(double C) {
    double t = nearbyint(C * ORC_TWO32);
    if (t < 0.0) t = 0.0;
    if (t > ORC_TWO32 - 1.0) t = ORC_TWO32 - 1.0;
    return (uint32_t)t;
}

/*
 * Build the dense leakage table: one row per state s = c*J + j.
 * Outcome order: 0 bin-1, 1 bin+1, then for each axis a: 2+2a (-e_a), 3+2a (+e_a).
 * thr[s*(K-1) + k]: quantised cumulative probability of outcomes 0..k.
 * flags[s]: 2-bit action per outcome, ORC_FLAG_MOVING, ORC_FLAG_THIN.
 * rebin_m / rebin_thr [c*2*ndim + face]: Doppler rebin of uniform bins across
 *   that face (new bin = j + m + [w >= thr]); face = 2a + (side > 0).
 * k_out (optional): k_ij.  rate_out (optional): the K leakage coefficients.
 * Returns 0, or -1 for an unsupported grid.
 */
int orc_build_table(const orc_grid* g, uint32_t* thr, uint32_t* flags, int32_t* rebin_m,
                    uint32_t* rebin_thr, double* k_out, double* rate_out, double* surv_out) {
    if (g->ndim != 1 && g->ndim != 3) return -1;
    if (g->dust_abs < 0.0 || g->dust_scat < 0.0 || (g->dust_abs > 0.0 && g->hybrid)) return -1;
    const int J = g->J, K = orc_nout(g), NT = orc_nthr(g), KT = NT + 1;
    const int64_t nc = orc_ncell(g);
    const double a = orc_damping(g->T);
    double* phi = (double*)malloc(sizeof(double) * J);
    for (int j = 0; j < J; ++j) phi[j] = orc_bin_mean_H(a, g->edges[j], g->edges[j + 1]);
    /* memo of the shifted bin means phi_j(delta) for the distinct face shifts
     * met so far (a pure function of delta; a Hubble flow has a single one) */
    enum { NMEMO = 16 };
    double memo_delta[NMEMO];
    double* memo_phi[NMEMO];
    int nmemo = 0;
    double dzmin = 1e300;
    for (int ax = 0; ax < g->ndim; ++ax) dzmin = fmin(dzmin, orc_dz(g, ax));

    for (int64_t c = 0; c < nc; ++c) {
        int idx[3];
        orc_idx_of(g, c, idx);
        const double k0c = orc_k0(g, c);
        /* grey dust per unit length: scattering adds to every k_ij, absorption
         * is its own process (Sec. 2.6) */
        const double nrel = g->n_rel ? g->n_rel[c] : 1.0;
        const double ksc = g->dust_scat / g->R * nrel, kac = g->dust_abs / g->R * nrel;
        int moving = 0;
        if (g->v)
            for (int ax = 0; ax < 3; ++ax) moving |= (g->v[3 * c + ax] != 0.0);
        /* Doppler rebin per face, uniform bins assumed (checked by the caller). */
        double dx0 = g->edges[1] - g->edges[0];
        for (int ax = 0; ax < g->ndim; ++ax)
            for (int sd = 0; sd < 2; ++sd) {
                int side = sd ? 1 : -1, nidx[3] = {idx[0], idx[1], idx[2]};
                nidx[ax] += side;
                double delta = 0.0;
                if (orc_in_medium(g, idx) && orc_in_medium(g, nidx))
                    delta = orc_face_shift(g, c, orc_cell_of(g, nidx), ax, side);
                double q = delta / dx0, m = floor(q), f = q - m;
                rebin_m[c * 2 * g->ndim + 2 * ax + sd] = (int32_t)m;
                rebin_thr[c * 2 * g->ndim + 2 * ax + sd] = orc_quantise(1.0 - f);
            }
        for (int j = 0; j < J; ++j) {
            const int64_t s = c * J + j;
            const double dxj = g->edges[j + 1] - g->edges[j];
            const double k = k0c * phi[j] + ksc;
            double rate[9] = {0};
            unsigned act[9] = {0};
            int thin = g->hybrid && (k * dzmin < g->tau_ddmc);
            /* frequency leakage, eq. x-leakage; no flux beyond the grid ends */
            for (int sd = 0; sd < 2; ++sd) {
                int jn = j + (sd ? 1 : -1);
                if (jn < 0 || jn >= J) { rate[sd] = 0.0; act[sd] = ORC_ACT_MOVE; continue; }
                double dxn = g->edges[jn + 1] - g->edges[jn];
                double kn = k0c * phi[jn] + ksc;
                rate[sd] = 1.0 / (dxj * (dxj / k + dxn / kn));
                act[sd] = (g->hybrid && kn * dzmin < g->tau_ddmc) ? ORC_ACT_TO_MC : ORC_ACT_MOVE;
            }
            /* spatial leakage, eq. z-leakage; exterior and thin neighbours use
             * the extrapolation-distance form of Sec. 5.1 */
            for (int ax = 0; ax < g->ndim; ++ax) {
                const double dz = orc_dz(g, ax);
                for (int sd = 0; sd < 2; ++sd) {
                    int side = sd ? 1 : -1, o = 2 + 2 * ax + sd, nidx[3] = {idx[0], idx[1], idx[2]};
                    nidx[ax] += side;
                    double r_bnd = 1.0 / (3.0 * dz) * 2.0 / (k * dz + 2.0 * g->lambda);
                    if (!orc_in_medium(g, nidx)) { rate[o] = r_bnd; act[o] = ORC_ACT_ESCAPE; continue; }
                    int64_t nb = orc_cell_of(g, nidx);
                    double delta = orc_face_shift(g, c, nb, ax, side);
                    double phin;
                    if (delta == 0.0) {
                        phin = phi[j];
                    } else {
                        int m = 0;
                        while (m < nmemo && memo_delta[m] != delta) ++m;
                        if (m == nmemo && nmemo < NMEMO) {
                            memo_delta[nmemo] = delta;
                            memo_phi[nmemo] = (double*)malloc(sizeof(double) * J);
                            for (int jj = 0; jj < J; ++jj)
                                memo_phi[nmemo][jj] = orc_bin_mean_H(a, g->edges[jj] + delta, g->edges[jj + 1] + delta);
                            ++nmemo;
                        }
                        phin = (m < nmemo) ? memo_phi[m][j]
                                           : orc_bin_mean_H(a, g->edges[j] + delta, g->edges[j + 1] + delta);
                    }
                    double knb = orc_k0(g, nb) * phin + g->dust_scat / g->R * (g->n_rel ? g->n_rel[nb] : 1.0);
                    double dznb = dz;
                    if (g->hybrid && knb * dznb < g->tau_ddmc) { rate[o] = r_bnd; act[o] = ORC_ACT_TO_MC; continue; }
                    rate[o] = 1.0 / (3.0 * dz) * 2.0 / (k * dz + knb * dznb);
                    act[o] = (delta != 0.0) ? ORC_ACT_REBIN : ORC_ACT_MOVE;
                }
            }
            if (orc_dusty(g)) rate[K] = kac;  /* absorption, the last outcome */
            double tot = 0.0;
            for (int o = 0; o < KT; ++o) tot += rate[o];
            /* continuous absorption: the expected weight kept over one dwell,
             * E[exp(-k_a dl)] = K_s / (K_s + k_a) for dl ~ Exp(K_s) */
            if (surv_out) surv_out[s] = g->dust_weights ? tot / (tot + kac) : 1.0;
            double C = 0.0;
            for (int o = 0; o < NT; ++o) {
                C += rate[o] / tot;
                thr[s * NT + o] = orc_quantise(C);
            }
            uint32_t fl = 0;
            for (int o = 0; o < K; ++o) fl |= (act[o] & 3u) << (2 * o);
            if (moving) fl |= ORC_FLAG_MOVING;
            if (thin) fl |= ORC_FLAG_THIN;
            flags[s] = fl;
            if (k_out) k_out[s] = k;
            if (rate_out)
                for (int o = 0; o < KT; ++o) rate_out[s * KT + o] = rate[o];
        }
    }
    free(phi);
    for (int m = 0; m < nmemo; ++m) free(memo_phi[m]);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Walk (Sec. 2.3)                                                           */
/* ------------------------------------------------------------------------- */

/* Tally layout (uint64): see ORC_T_* ; faces [ORC_T_FACE, +6); histogram of
 * escape frequency [ORC_T_HIST, +J+2) with 0 = below the grid, J+1 = above. */
#define ORC_T_EMITTED 0
#define ORC_T_ESCAPED 1
#define ORC_T_ABORTED 2
#define ORC_T_STEPS 3
#define ORC_T_MC_EVENTS 4
#define ORC_T_CONVERSIONS 5
#define ORC_T_CLAMPS 6
#define ORC_T_EVENT_DRAWS 7
#define ORC_T_ABSORBED 8
#define ORC_T_FACE 9
#define ORC_T_HIST 15
#define ORC_NSB 64          /* impact-parameter bins over b/R in [0, 1.28); larger b in the last bin */
#define ORC_SB_MAX 1.28

int orc_tally_len(int J) { return ORC_T_HIST + J + 2 + ORC_NSB; }

/* Source: the cell(s) at the domain centre and the bin(s) containing x0.  With
 * an even count the centre is a face/edge and both neighbours are used with
 * equal probability (the paper enforces odd counts instead). */
typedef struct orc_source {
    int ncand[3];
    int cand[3][2];
    int nbin;
    int bin[2];
} orc_source;

static int orc_make_source(const orc_grid* g, double x0, orc_source* src) {
    for (int ax = 0; ax < 3; ++ax) {
        int n = g->n[ax];
        if (n % 2) { src->ncand[ax] = 1; src->cand[ax][0] = src->cand[ax][1] = n / 2; }
        else { src->ncand[ax] = 2; src->cand[ax][0] = n / 2 - 1; src->cand[ax][1] = n / 2; }
    }
    src->nbin = 0;
    for (int j = 1; j < g->J; ++j)
        if (g->edges[j] == x0) { src->nbin = 2; src->bin[0] = j - 1; src->bin[1] = j; }
    if (!src->nbin) {
        for (int j = 0; j < g->J; ++j)
            if (g->edges[j] < x0 && x0 < g->edges[j + 1]) { src->nbin = 1; src->bin[0] = src->bin[1] = j; }
    }
    return src->nbin ? 0 : -1;
}

/* Draw 0: bit 31-a picks the cell along axis a (a = 0,1,2), bit 28 picks the bin. */
static void orc_emit(const orc_source* src, uint32_t w, int idx[3], int* j) {
    for (int ax = 0; ax < 3; ++ax) idx[ax] = src->cand[ax][src->ncand[ax] == 2 ? (w >> (31 - ax)) & 1u : 0];
    *j = src->bin[src->nbin == 2 ? (w >> 28) & 1u : 0];
}

typedef struct orc_walk_args {
    const orc_grid* g;
    const uint32_t* thr;
    const uint32_t* flags;
    const int32_t* rebin_m;
    const uint32_t* rebin_thr;
    const double* rate;  /* for the competing-exponentials form */
    const orc_source* src;
    uint64_t seed, p0, p1, max_steps;
    int literal;         /* 1: competing exponentials in FP64 (eq. l_min_1/2) */
    uint64_t limit;      /* transitions per packet, UINT64_MAX = until escape or abort */
    const double* k;     /* k_ij per state (hybrid walk) */
    const double* upar;  /* (u1, u0) rejection-envelope split points per |x| grid point (hybrid) */
    const double* surv;  /* continuous absorption: weight factor per state, NULL = none */
    double* wtally;      /* per-thread escaped weight: [0] total, [1 + b] per histogram bin b */
    uint64_t* tally;     /* per-thread */
    int status;
} orc_walk_args;

/* Escape through the face of outcome o from cell c at bin j.
 * Slab, static cell: tally the packet's bin.  Otherwise draw a point on the
 * face (uniform over the cell's face, two draws for the tangential axes), an
 * isotropic outward direction (mu uniform on (0,1], azimuth phi uniform) and x
 * uniform in the bin; tally x_obs = x + n.u_c (u = v/v_th) and, in 3D, the
 * impact parameter b = |r x n| of the escaping ray. */
static int orc_escape(const orc_walk_args* A, int64_t c, int j, int o, uint64_t pk, uint64_t* e, uint64_t* t) {
    const orc_grid* g = A->g;
    const int J = g->J;
    int face = o - 2;
    t[ORC_T_ESCAPED]++;
    t[ORC_T_FACE + face]++;
    if (g->ndim == 1 && !(A->flags[c * J + j] & ORC_FLAG_MOVING)) { t[ORC_T_HIST + 1 + j]++; return 1 + j; }
    int ax = face / 2, side = (face & 1) ? 1 : -1;
    int t1 = (ax + 1) % 3, t2 = (ax + 2) % 3;
    int idx[3];
    orc_idx_of(g, c, idx);
    double r[3];
    r[ax] = -g->R + (idx[ax] + (side > 0 ? 1 : 0)) * orc_dz(g, ax);
    double p1 = orc_unif(orc_word(A->seed, pk, ORC_EVENT, (*e)++));
    double p2 = orc_unif(orc_word(A->seed, pk, ORC_EVENT, (*e)++));
    r[t1] = (t1 < g->ndim) ? -g->R + (idx[t1] + p1) * orc_dz(g, t1) : 0.0;
    r[t2] = (t2 < g->ndim) ? -g->R + (idx[t2] + p2) * orc_dz(g, t2) : 0.0;
    double mu = 1.0 - orc_unif(orc_word(A->seed, pk, ORC_EVENT, (*e)++));
    double ph = 2.0 * ORC_PI * orc_unif(orc_word(A->seed, pk, ORC_EVENT, (*e)++));
    double xu = orc_unif(orc_word(A->seed, pk, ORC_EVENT, (*e)++));
    double x = g->edges[j] + xu * (g->edges[j + 1] - g->edges[j]);
    double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    double n[3];
    n[ax] = side * mu;
    n[t1] = st * cos(ph);
    n[t2] = st * sin(ph);
    double nu = 0.0;
    if (g->v) {
        double vth = orc_vth(g);
        nu = n[0] * (g->v[3 * c + 0] / vth) + n[1] * (g->v[3 * c + 1] / vth) + n[2] * (g->v[3 * c + 2] / vth);
    }
    double xo = x + nu;
    int b;
    if (xo < g->edges[0]) b = 0;
    else if (xo >= g->edges[J]) b = J + 1;
    else {
        b = 1;
        while (b < J && xo >= g->edges[b]) ++b;
    }
    t[ORC_T_HIST + b]++;
    if (g->ndim == 3) {
        double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        double rn = r[0] * n[0] + r[1] * n[1] + r[2] * n[2];
        double bb = sqrt(fmax(0.0, rr - rn * rn)) / g->R;
        int k = (int)(bb / ORC_SB_MAX * ORC_NSB);
        if (k > ORC_NSB - 1) k = ORC_NSB - 1;
        t[ORC_T_HIST + J + 2 + k]++;
    }
    return b;
}

/* ------------------------------------------------------------------------- */
/* Continuous MC in thin states (Sec. 5.1, Sec. 5.2)                          */
/* ------------------------------------------------------------------------- */

#define ORC_UPAR_STEP (1.0 / 16.0)  /* |x| grid of the envelope split points */
#define ORC_UPAR_N 1024

/* Mass of the three-part envelope of f(u) = e^{-u^2} / (a^2 + (x-u)^2) (x >= 0):
 * u < u1: e^{-u^2} g(u1);  u1 <= u <= u0: c2 g(u), c2 = max of e^{-u^2} there;
 * u > u0: e^{-u0^2} g(u), with g(u) = 1/(a^2 + (x-u)^2) and u1 <= u0 <= x,
 * 0 <= u0.  Every piece bounds f because g rises up to x and e^{-u^2} falls
 * away from 0. */
static double orc_env_mass(double a, double x, double u1, double u0) {
    double g1 = 1.0 / (a * a + (x - u1) * (x - u1));
    double w1 = g1 * 0.5 * ORC_SQRTPI * (1.0 + erf(u1));
    double th1 = atan((u1 - x) / a), th0 = atan((u0 - x) / a);
    double c2 = (u1 <= 0.0) ? 1.0 : exp(-u1 * u1);
    double w2 = c2 * (th0 - th1) / a;
    double w3 = exp(-u0 * u0) * (0.5 * ORC_PI - th0) / a;
    return w1 + w2 + w3;
}

/* Split points minimising the envelope mass on a grid of candidates, for each
 * |x| = i * ORC_UPAR_STEP.  Any valid pair samples the same distribution; the
 * choice only sets the acceptance rate. */
void orc_upar_table(double a, double* tab) {
    for (int i = 0; i < ORC_UPAR_N; ++i) {
        double x = i * ORC_UPAR_STEP, best = INFINITY, b1 = -40.0, b0 = 0.0;
        for (int p = 0; p <= 24; ++p) {
            double u0 = x * p / 24.0;
            for (int q = 0; q <= 25; ++q) {
                double u1 = (q == 25) ? -40.0 : -3.0 + (u0 + 3.0) * q / 24.0;
                double m = orc_env_mass(a, x, u1, u0);
                if (m < best) { best = m; b1 = u1; b0 = u0; }
            }
        }
        tab[2 * i] = b1;
        tab[2 * i + 1] = b0;
    }
}

static double orc_ev(const orc_walk_args* A, uint64_t pk, uint64_t* e) {
    return orc_unif(orc_word(A->seed, pk, ORC_EVENT, (*e)++));
}

/* Parallel atom velocity u (Doppler units) of a scattering at frequency x:
 * density e^{-u^2} / (a^2 + (x-u)^2) (Sec. 5.2; Maxwellian sign per the
 * standard Voigt convolution), by rejection from the three-part envelope. */
static double orc_sample_upar(const orc_walk_args* A, double a, double xin, uint64_t pk, uint64_t* e) {
    const double x = fabs(xin), sg = xin < 0.0 ? -1.0 : 1.0;
    int i = (int)(x / ORC_UPAR_STEP);
    if (i > ORC_UPAR_N - 1) i = ORC_UPAR_N - 1;
    const double u1 = A->upar[2 * i], u0 = A->upar[2 * i + 1];
    const double g1 = 1.0 / (a * a + (x - u1) * (x - u1));
    const double th1 = atan((u1 - x) / a), th0 = atan((u0 - x) / a);
    const double c2 = (u1 <= 0.0) ? 1.0 : exp(-u1 * u1);
    const double w1 = g1 * 0.5 * ORC_SQRTPI * (1.0 + erf(u1));
    const double w2 = c2 * (th0 - th1) / a;
    const double w3 = exp(-u0 * u0) * (0.5 * ORC_PI - th0) / a;
    const double sig = sqrt(0.5);
    for (int it = 0; it < 1000000; ++it) {
        double pick = orc_ev(A, pk, e) * (w1 + w2 + w3), u, acc;
        if (pick < w1) {
            /* Gaussian N(0, 1/2) below u1: rejection from the full Gaussian
             * when u1 >= 0, Marsaglia's tail method otherwise */
            if (u1 >= 0.0) {
                do {
                    double r1 = orc_ev(A, pk, e), r2 = orc_ev(A, pk, e);
                    u = sig * sqrt(-2.0 * log(r1)) * cos(2.0 * ORC_PI * r2);
                } while (u >= u1);
            } else {
                const double c = -u1 / sig;
                double X;
                for (;;) {
                    double r1 = orc_ev(A, pk, e), r2 = orc_ev(A, pk, e);
                    X = sqrt(c * c - 2.0 * log(r1));
                    if (r2 * X < c) break;
                }
                u = -sig * X;
            }
            acc = (1.0 / (a * a + (x - u) * (x - u))) / g1;
        } else if (pick < w1 + w2) {
            double th = th1 + orc_ev(A, pk, e) * (th0 - th1);
            u = x + a * tan(th);
            acc = exp(-u * u) / c2;
        } else {
            double th = th0 + orc_ev(A, pk, e) * (0.5 * ORC_PI - th0);
            u = x + a * tan(th);
            acc = exp(u0 * u0 - u * u);
        }
        if (orc_ev(A, pk, e) < acc) return sg * u;
    }
    return sg * x;
}

/* Isotropic direction: mu uniform on (-1,1), azimuth uniform. */
static void orc_iso_dir(const orc_walk_args* A, uint64_t pk, uint64_t* e, double n[3]) {
    double mu = 2.0 * orc_ev(A, pk, e) - 1.0, ph = 2.0 * ORC_PI * orc_ev(A, pk, e);
    double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    n[0] = st * cos(ph); n[1] = st * sin(ph); n[2] = mu;
}

/* Direction uniform over the half-space around +/- e_ax (mu uniform on (0,1]). */
static void orc_half_dir(const orc_walk_args* A, uint64_t pk, uint64_t* e, int ax, int side, double n[3]) {
    double mu = 1.0 - orc_ev(A, pk, e), ph = 2.0 * ORC_PI * orc_ev(A, pk, e);
    double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    n[ax] = side * mu; n[(ax + 1) % 3] = st * cos(ph); n[(ax + 2) % 3] = st * sin(ph);
}

/* Coherent scattering in the atom frame, isotropic phase function, no recoil:
 * x' = x + u_par (mu - 1) + u_perp sqrt(1 - mu^2), u_perp ~ N(0, 1/2),
 * mu = n.n' (Sec. 5.2). */
static double orc_scatter(const orc_walk_args* A, double a, double x, double n[3], uint64_t pk, uint64_t* e) {
    double up = orc_sample_upar(A, a, x, pk, e);
    double r1 = orc_ev(A, pk, e), r2 = orc_ev(A, pk, e);
    double uperp = sqrt(0.5) * sqrt(-2.0 * log(r1)) * cos(2.0 * ORC_PI * r2);
    double nn[3];
    orc_iso_dir(A, pk, e, nn);
    double mu = n[0] * nn[0] + n[1] * nn[1] + n[2] * nn[2];
    if (mu > 1.0) mu = 1.0;
    if (mu < -1.0) mu = -1.0;
    n[0] = nn[0]; n[1] = nn[1]; n[2] = nn[2];
    return x + up * (mu - 1.0) + uperp * sqrt(1.0 - mu * mu);
}

static int orc_bin_of(const orc_grid* g, double x) {
    if (x < g->edges[0]) return -1;
    if (x >= g->edges[g->J]) return g->J;
    int lo = 0, hi = g->J;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (x >= g->edges[mid]) lo = mid; else hi = mid;
    }
    return lo;
}

static int orc_is_thick(const orc_walk_args* A, int64_t c, int j) {
    if (j < 0 || j >= A->g->J) return 0;
    return !(A->flags[c * A->g->J + j] & ORC_FLAG_THIN);
}

static double orc_u(const orc_grid* g, int64_t c, int a) { return g->v ? g->v[3 * c + a] / orc_vth(g) : 0.0; }

typedef struct orc_mc {
    int idx[3];
    double r[3], n[3], x;
} orc_mc;

/* Tally an escape of an MC packet leaving cell c through face (ax, side). */
static void orc_mc_escape(const orc_walk_args* A, const orc_mc* m, int64_t c, int ax, int side, uint64_t* t) {
    const orc_grid* g = A->g;
    const int J = g->J;
    t[ORC_T_ESCAPED]++;
    t[ORC_T_FACE + 2 * ax + (side > 0 ? 1 : 0)]++;
    double xo = m->x + m->n[0] * orc_u(g, c, 0) + m->n[1] * orc_u(g, c, 1) + m->n[2] * orc_u(g, c, 2);
    int b = orc_bin_of(g, xo);
    t[ORC_T_HIST + (b < 0 ? 0 : (b >= J ? J + 1 : b + 1))]++;
    if (g->ndim == 3) {
        double rr = m->r[0] * m->r[0] + m->r[1] * m->r[1] + m->r[2] * m->r[2];
        double rn = m->r[0] * m->n[0] + m->r[1] * m->n[1] + m->r[2] * m->n[2];
        double bb = sqrt(fmax(0.0, rr - rn * rn)) / g->R;
        int k = (int)(bb / ORC_SB_MAX * ORC_NSB);
        if (k > ORC_NSB - 1) k = ORC_NSB - 1;
        t[ORC_T_HIST + J + 2 + k]++;
    }
}

/* Cross from the MC packet's cell through face (ax, side): escape, continue in
 * a thin neighbour, convert to DDMC in a thick neighbour with probability
 * 2/(tau + 2 lambda) (2/3 + mu) (Sec. 5.1), or reflect from it (random point on
 * the face, isotropic inward direction).  Returns 0 to continue MC, 1 escaped,
 * 2 converted to DDMC (state in *cell_out, *bin_out). */
static int orc_mc_cross(orc_walk_args* A, orc_mc* m, int ax, int side, uint64_t pk, uint64_t* e, uint64_t* t,
                        int64_t* cell_out, int* bin_out) {
    const orc_grid* g = A->g;
    int64_t c = orc_cell_of(g, m->idx);
    int nidx[3] = {m->idx[0], m->idx[1], m->idx[2]};
    nidx[ax] += side;
    if (!orc_in_medium(g, nidx)) { orc_mc_escape(A, m, c, ax, side, t); return 1; }
    int64_t nb = orc_cell_of(g, nidx);
    double xn = m->x + m->n[0] * (orc_u(g, c, 0) - orc_u(g, nb, 0)) + m->n[1] * (orc_u(g, c, 1) - orc_u(g, nb, 1)) +
                m->n[2] * (orc_u(g, c, 2) - orc_u(g, nb, 2));
    int jn = orc_bin_of(g, xn);
    if (!orc_is_thick(A, nb, jn)) {
        m->idx[ax] += side;
        m->x = xn;
        return 0;
    }
    double tau = A->k[nb * g->J + jn] * orc_dz(g, ax);
    double P = 2.0 / (tau + 2.0 * g->lambda) * (2.0 / 3.0 + fabs(m->n[ax]));
    if (orc_ev(A, pk, e) < P) {
        t[ORC_T_CONVERSIONS]++;
        *cell_out = nb;
        *bin_out = jn;
        return 2;
    }
    /* reflect: a random point on the same face, isotropic inward direction */
    int t1 = (ax + 1) % 3, t2 = (ax + 2) % 3;
    double p1 = orc_ev(A, pk, e), p2 = orc_ev(A, pk, e);
    if (t1 < g->ndim) m->r[t1] = -g->R + (m->idx[t1] + p1) * orc_dz(g, t1);
    if (t2 < g->ndim) m->r[t2] = -g->R + (m->idx[t2] + p2) * orc_dz(g, t2);
    orc_half_dir(A, pk, e, ax, -side, m->n);
    int j = orc_bin_of(g, m->x);
    if (orc_is_thick(A, c, j)) {
        t[ORC_T_CONVERSIONS]++;
        *cell_out = c;
        *bin_out = j;
        return 2;
    }
    return 0;
}

/* Run an MC packet until it converts to DDMC (returns 2, state in *cell_out,
 * *bin_out), escapes (1) or meets the event watchdog (3): at most
 * min(max_steps, 1e8) events per excursion. */
static int orc_mc_run(orc_walk_args* A, orc_mc* m, uint64_t pk, uint64_t* e, uint64_t* t, int64_t* cell_out,
                      int* bin_out) {
    const orc_grid* g = A->g;
    const double a = orc_damping(g->T);
    const uint64_t cap = A->max_steps < (uint64_t)100000000 ? A->max_steps : (uint64_t)100000000;
    for (uint64_t ev = 0;; ++ev) {
        if (ev >= cap) return 3;
        int64_t c = orc_cell_of(g, m->idx);
        /* frequency grouping (Sec. 5.3): the bin-mean opacity of the packet's bin */
        /* (a Doppler shift across a face may carry x past the grid ends: grouping
         * then uses the end bin, as the leakage has no flux beyond them) */
        int jb = orc_bin_of(g, m->x);
        jb = jb < 0 ? 0 : (jb > g->J - 1 ? g->J - 1 : jb);
        double k = g->redist ? A->k[c * g->J + jb] : orc_k0(g, c) * orc_voigt_H(a, m->x);
        double s = -log(orc_ev(A, pk, e)) / k;
        /* distance to the cell boundary along n */
        double dmin = INFINITY;
        int fax = -1, fside = 0;
        for (int ax = 0; ax < g->ndim; ++ax) {
            if (m->n[ax] == 0.0) continue;
            double lo = -g->R + m->idx[ax] * orc_dz(g, ax), hi = lo + orc_dz(g, ax);
            double d = m->n[ax] > 0.0 ? (hi - m->r[ax]) / m->n[ax] : (lo - m->r[ax]) / m->n[ax];
            if (d < 0.0) d = 0.0;
            if (d < dmin) { dmin = d; fax = ax; fside = m->n[ax] > 0.0 ? 1 : -1; }
        }
        t[ORC_T_MC_EVENTS]++;
        if (s < dmin) {
            for (int q = 0; q < 3; ++q) m->r[q] += s * m->n[q];
            if (g->redist) {
                /* frequency grouping: the new bin from the row of eq. R_discrete
                 * (categorical draw on its thresholds), x uniform in it, a new
                 * isotropic direction */
                const int jp = jb;
                const uint32_t w = orc_word(A->seed, pk, ORC_EVENT, (*e)++);
                int jn = 0;
                while (jn < g->J - 1 && w >= g->redist[(size_t)jp * (g->J - 1) + jn]) ++jn;
                m->x = g->edges[jn] + orc_ev(A, pk, e) * (g->edges[jn + 1] - g->edges[jn]);
                orc_iso_dir(A, pk, e, m->n);
            } else {
                m->x = orc_scatter(A, a, m->x, m->n, pk, e);
            }
            int j = orc_bin_of(g, m->x);
            if (orc_is_thick(A, c, j)) {
                t[ORC_T_CONVERSIONS]++;
                *cell_out = c;
                *bin_out = j;
                return 2;
            }
            continue;
        }
        for (int q = 0; q < 3; ++q) m->r[q] += dmin * m->n[q];
        m->r[fax] = -g->R + (m->idx[fax] + (fside > 0 ? 1 : 0)) * orc_dz(g, fax);
        int rc = orc_mc_cross(A, m, fax, fside, pk, e, t, cell_out, bin_out);
        if (rc) return rc;
    }
}

/* A DDMC packet at (c, j) hands off to MC.  Spatial outcome into a thin
 * neighbour: a random point on the face and an isotropic outward direction,
 * x uniform in the bin, then the crossing into the neighbour.  Frequency
 * outcome into a thin bin j_new (or a thin source state): a random point in
 * the cell, an isotropic direction, x uniform in bin j_new. */
static void orc_handoff(orc_walk_args* A, int64_t c, int j, int face, uint64_t pk, uint64_t* e, orc_mc* m) {
    const orc_grid* g = A->g;
    orc_idx_of(g, c, m->idx);
    for (int q = 0; q < 3; ++q) m->r[q] = 0.0;
    if (face >= 0) {
        int ax = face / 2, side = (face & 1) ? 1 : -1;
        int t1 = (ax + 1) % 3, t2 = (ax + 2) % 3;
        m->r[ax] = -g->R + (m->idx[ax] + (side > 0 ? 1 : 0)) * orc_dz(g, ax);
        double p1 = orc_ev(A, pk, e), p2 = orc_ev(A, pk, e);
        if (t1 < g->ndim) m->r[t1] = -g->R + (m->idx[t1] + p1) * orc_dz(g, t1);
        if (t2 < g->ndim) m->r[t2] = -g->R + (m->idx[t2] + p2) * orc_dz(g, t2);
        orc_half_dir(A, pk, e, ax, side, m->n);
    } else {
        double p[3] = {orc_ev(A, pk, e), orc_ev(A, pk, e), orc_ev(A, pk, e)};
        for (int ax = 0; ax < g->ndim; ++ax) m->r[ax] = -g->R + (m->idx[ax] + p[ax]) * orc_dz(g, ax);
        orc_iso_dir(A, pk, e, m->n);
    }
    m->x = g->edges[j] + orc_ev(A, pk, e) * (g->edges[j + 1] - g->edges[j]);
}

/* Per-packet state of the walk. */
typedef struct orc_pstate {
    int idx[3];
    int j;
    uint64_t steps, e;
    int done;      /* 0 in flight, 1 escaped, 2 aborted, 3 met an MC state, 4 absorbed by dust */
    double w;      /* packet weight (continuous absorption) */
} orc_pstate;

/* Advance packet pk by at most `limit` transitions (stopping at escape or at
 * the watchdog), accumulating tallies into t. */
static void orc_advance(orc_walk_args* A, uint64_t pk, orc_pstate* P, uint64_t limit, uint64_t* t) {
    const orc_grid* g = A->g;
    const int J = g->J, K = orc_nout(g), nf = 2 * g->ndim, NT = orc_nthr(g), KT = NT + 1;
    int64_t c = orc_cell_of(g, P->idx);
    if (A->flags[c * J + P->j] & ORC_FLAG_THIN) {
        /* only a source state can be thin: the packet starts as MC */
        if (!A->upar) { A->status = -2; t[ORC_T_ABORTED]++; P->done = 3; return; }
        orc_mc m;
        t[ORC_T_CONVERSIONS]++;
        orc_handoff(A, c, P->j, -1, pk, &P->e, &m);
        int64_t cn;
        int jn;
        int rc = orc_mc_run(A, &m, pk, &P->e, t, &cn, &jn);
        if (rc == 1) { P->done = 1; return; }
        if (rc == 3) { t[ORC_T_ABORTED]++; P->done = 2; return; }
        orc_idx_of(g, cn, P->idx);
        P->j = jn;
        c = cn;
    }
    for (uint64_t n = 0; n < limit; ++n) {
        if (P->steps >= A->max_steps) { t[ORC_T_ABORTED]++; P->done = 2; return; }
        const int64_t s = c * J + P->j;
        int o;
        if (!A->literal) {
            /* categorical draw: outcome o iff thr[o-1] <= w < thr[o] */
            uint32_t w = orc_word(A->seed, pk, ORC_TRANS, P->steps);
            o = 0;
            while (o < NT && w >= A->thr[s * NT + o]) ++o;
        } else {
            /* eq. l_min_2: dl_X = -ln(xi)/k_X for every process (absorption
             * included); eq. l_min_1: execute the smallest */
            double best = INFINITY;
            o = -1;
            for (int q = 0; q < KT; ++q) {
                double xi = orc_unif(orc_word(A->seed, pk, ORC_TRANS, 16 * P->steps + q));
                double kx = A->rate[s * KT + q];
                if (kx <= 0.0) continue;
                double dl = -log(xi) / kx;
                if (dl < best) { best = dl; o = q; }
            }
        }
        P->steps++;
        t[ORC_T_STEPS]++;
        if (o == K) { t[ORC_T_ABSORBED]++; P->done = 4; return; }  /* absorbed by dust (Sec. 2.6) */
        if (A->surv) P->w *= A->surv[s];  /* continuous absorption over the dwell in s */
        unsigned act = (A->flags[s] >> (2 * o)) & 3u;
        if (act == ORC_ACT_ESCAPE) {
            const int b = orc_escape(A, c, P->j, o, pk, &P->e, t);
            if (A->wtally) { A->wtally[0] += P->w; A->wtally[1 + b] += P->w; }  /* the escaped weight */
            P->done = 1;
            return;
        }
        if (A->surv && P->w < ORC_W_MIN) { t[ORC_T_ABSORBED]++; P->done = 4; return; }
        if (act == ORC_ACT_TO_MC) {
            if (!A->upar) { A->status = -2; t[ORC_T_ABORTED]++; P->done = 3; return; }
            orc_mc m;
            t[ORC_T_CONVERSIONS]++;
            int64_t cn; int jn, rc;
            if (o < 2) {
                orc_handoff(A, c, P->j + (o ? 1 : -1), -1, pk, &P->e, &m);
                rc = orc_mc_run(A, &m, pk, &P->e, t, &cn, &jn);
            } else {
                orc_handoff(A, c, P->j, o - 2, pk, &P->e, &m);
                int face = o - 2;
                rc = orc_mc_cross(A, &m, face / 2, (face & 1) ? 1 : -1, pk, &P->e, t, &cn, &jn);
                if (rc == 0) rc = orc_mc_run(A, &m, pk, &P->e, t, &cn, &jn);
            }
            if (rc == 1) { P->done = 1; return; }
            if (rc == 3) { t[ORC_T_ABORTED]++; P->done = 2; return; }
            orc_idx_of(g, cn, P->idx); P->j = jn; c = cn;
            continue;
        }
        if (o < 2) { P->j += o ? 1 : -1; continue; }
        int face = o - 2, ax = face / 2, side = (face & 1) ? 1 : -1;
        if (act == ORC_ACT_REBIN) {
            uint32_t w1 = orc_word(A->seed, pk, ORC_EVENT, P->e++);
            int jn = P->j + A->rebin_m[c * nf + face] + (w1 >= A->rebin_thr[c * nf + face] ? 1 : 0);
            if (jn < 0) { jn = 0; t[ORC_T_CLAMPS]++; }
            if (jn > J - 1) { jn = J - 1; t[ORC_T_CLAMPS]++; }
            P->j = jn;
        }
        P->idx[ax] += side;
        c = orc_cell_of(g, P->idx);
    }
}

static void orc_start(orc_walk_args* A, uint64_t pk, orc_pstate* P, uint64_t* t) {
    memset(P, 0, sizeof(*P));
    P->w = 1.0;
    orc_emit(A->src, orc_word(A->seed, pk, ORC_EVENT, P->e++), P->idx, &P->j);
    t[ORC_T_EMITTED]++;
}

static void* orc_walk_thread(void* vp) {
    orc_walk_args* A = (orc_walk_args*)vp;
    uint64_t* t = A->tally;
    for (uint64_t pk = A->p0; pk < A->p1; ++pk) {
        orc_pstate P;
        orc_start(A, pk, &P, t);
        if (A->limit == UINT64_MAX)
            while (!P.done) orc_advance(A, pk, &P, UINT64_MAX, t);
        else
            orc_advance(A, pk, &P, A->limit, t);
        t[ORC_T_EVENT_DRAWS] += P.e;
    }
    return NULL;
}

/*
 * Run packets [p0, p0+np) of the DDMC walk on a table built by orc_build_table.
 * literal = 0: categorical draw on the quantised thresholds (the stream contract);
 * literal = 1: competing exponentials on the FP64 rates (a different stream use,
 *              equal in distribution up to the quantisation of the thresholds).
 * tally must hold orc_tally_len(J) words; it is overwritten.
 * Returns 0, -1 on bad input, -2 if a packet met a thin (MC) state: the hybrid
 * walk is orc_hybrid_walk_slab.
 */
static int orc_walk_run(const orc_grid* g, const uint32_t* thr, const uint32_t* flags, const int32_t* rebin_m,
                        const uint32_t* rebin_thr, const double* rate, const double* k, double x0, uint64_t seed,
                        uint64_t p0, uint64_t np, uint64_t max_steps, int literal, uint64_t limit, int nthreads,
                        uint64_t* tally, const double* surv, double* wtally) {
    double* upar = NULL;
    if (g->hybrid) {
        if (!k) return -1;
        upar = (double*)malloc(sizeof(double) * 2 * ORC_UPAR_N);
        orc_upar_table(orc_damping(g->T), upar);
    }
    orc_source src;
    if (orc_make_source(g, x0, &src)) return -1;
    if (literal && !rate) return -1;
    if (nthreads < 1) nthreads = 1;
    if ((uint64_t)nthreads > np) nthreads = np ? (int)np : 1;
    const int L = orc_tally_len(g->J);
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
    orc_walk_args* args = (orc_walk_args*)calloc(nthreads, sizeof(orc_walk_args));
    uint64_t* tl = (uint64_t*)calloc((size_t)nthreads * L, sizeof(uint64_t));
    const int LW = g->J + 3;
    double* twl = wtally ? (double*)calloc((size_t)nthreads * LW, sizeof(double)) : NULL;
    for (int i = 0; i < nthreads; ++i) {
        orc_walk_args* A = &args[i];
        A->g = g; A->thr = thr; A->flags = flags; A->rebin_m = rebin_m; A->rebin_thr = rebin_thr;
        A->rate = rate; A->src = &src; A->seed = seed; A->max_steps = max_steps; A->literal = literal;
        A->limit = limit;
        A->k = k;
        A->upar = upar;
        A->surv = surv;
        A->wtally = twl ? twl + (size_t)i * LW : NULL;
        A->p0 = p0 + np * (uint64_t)i / nthreads;
        A->p1 = p0 + np * (uint64_t)(i + 1) / nthreads;
        A->tally = tl + (size_t)i * L;
        pthread_create(&th[i], NULL, orc_walk_thread, A);
    }
    int status = 0;
    memset(tally, 0, sizeof(uint64_t) * L);
    if (wtally) memset(wtally, 0, sizeof(double) * LW);
    for (int i = 0; i < nthreads; ++i) {
        pthread_join(th[i], NULL);
        for (int q = 0; q < L; ++q) tally[q] += tl[(size_t)i * L + q];
        if (twl)
            for (int q = 0; q < LW; ++q) wtally[q] += twl[(size_t)i * LW + q];
        if (args[i].status) status = args[i].status;
    }
    free(th); free(args); free(tl); free(upar); free(twl);
    return status;
}

int orc_walk_ddmc(const orc_grid* g, const uint32_t* thr, const uint32_t* flags, const int32_t* rebin_m,
                  const uint32_t* rebin_thr, const double* rate, const double* k, double x0, uint64_t seed,
                  uint64_t p0, uint64_t np, uint64_t max_steps, int literal, int nthreads, uint64_t* tally) {
    return orc_walk_run(g, thr, flags, rebin_m, rebin_thr, rate, k, x0, seed, p0, np, max_steps, literal,
                        UINT64_MAX, nthreads, tally, NULL, NULL);
}

/*
 * The DDMC walk with continuous absorption by dust (Sec. 2.6, the weight
 * method): a packet's weight is multiplied by surv[s] = K_s / (K_s + k_a) at
 * each transition out of state s (the expected attenuation exp(-k_a dl) over
 * its dwell dl ~ Exp(K_s); the categorical walk has no path length) and the
 * packet is eliminated (counted as absorbed) once it falls below 1e-10.
 * wtally (J + 3 doubles, overwritten): [0] total escaped weight, [1 + b] the
 * escaped weight in escape-histogram bin b.  The grid needs dust_weights = 1.
 */
int orc_walk_weights(const orc_grid* g, const uint32_t* thr, const uint32_t* flags, const int32_t* rebin_m,
                     const uint32_t* rebin_thr, const double* surv, double x0, uint64_t seed, uint64_t p0,
                     uint64_t np, uint64_t max_steps, int nthreads, uint64_t* tally, double* wtally) {
    if (!g || !surv || !wtally || !g->dust_weights || g->hybrid) return -1;
    return orc_walk_run(g, thr, flags, rebin_m, rebin_thr, NULL, NULL, x0, seed, p0, np, max_steps, 0, UINT64_MAX,
                        nthreads, tally, surv, wtally);
}

/* ------------------------------------------------------------------------- */
/* Time-dependent walk (Sec. 2.3: causality within a time step; eq.          */
/* E_estimator: bin and path estimates of the energy density)                */
/* ------------------------------------------------------------------------- */

typedef struct orc_time_args {
    orc_walk_args w;
    const double* t_edges;
    int nt;
    uint64_t* bins;   /* per thread: nt x S */
    double* path;     /* per thread: nt x S */
    uint64_t* esc;    /* per thread: nt */
    double* leak;     /* per thread: nt x ncell x 2 ndim x 2, or NULL */
    double* wbins;    /* dust weights, per thread: nt x S weights in each state at t_end, or NULL */
    double* wpath;    /* dust weights, per thread: nt x S weighted path per state, or NULL */
    uint64_t steps, dwells, aborted;
} orc_time_args;

/* One DDMC transition of packet P in its current state (categorical draw on
 * the transition stream, action of the outcome).  A spatial outcome is a leak
 * through a face of the cell: if `leak` is set, the optical depth k dl of the
 * dwell dl that ended in it is added for the cell it leaves (index 0 of its
 * face) and, unless it escapes, for the cell it enters with that cell's k at
 * the new bin (index 1 of the face it enters through; eq. a_estimator).
 * Returns 1 if the packet escaped, 2 if dust absorbed it, -1 if it met an MC
 * state, 0 otherwise. */
static int orc_time_transition(orc_walk_args* A, uint64_t pk, orc_pstate* P, uint64_t* t, double dl,
                               double* leak) {
    const orc_grid* g = A->g;
    const int J = g->J, K = orc_nout(g), nf = 2 * g->ndim, NT = orc_nthr(g);
    int64_t c = orc_cell_of(g, P->idx);
    const int64_t s = c * J + P->j;
    uint32_t w = orc_word(A->seed, pk, ORC_TRANS, P->steps);
    int o = 0;
    while (o < NT && w >= A->thr[s * NT + o]) ++o;
    P->steps++;
    t[ORC_T_STEPS]++;
    if (o == K) { t[ORC_T_ABSORBED]++; return 2; }  /* absorbed by dust (Sec. 2.6) */
    unsigned act = (A->flags[s] >> (2 * o)) & 3u;
    if (act == ORC_ACT_TO_MC) return -1;
    if (o >= 2 && leak) leak[(c * nf + (o - 2)) * 2 + 0] += A->k[s] * dl;
    if (act == ORC_ACT_ESCAPE) { orc_escape(A, c, P->j, o, pk, &P->e, t); return 1; }
    if (o < 2) { P->j += o ? 1 : -1; return 0; }
    int face = o - 2, ax = face / 2, side = (face & 1) ? 1 : -1;
    if (act == ORC_ACT_REBIN) {
        uint32_t w1 = orc_word(A->seed, pk, ORC_EVENT, P->e++);
        int jn = P->j + A->rebin_m[c * nf + face] + (w1 >= A->rebin_thr[c * nf + face] ? 1 : 0);
        if (jn < 0) { jn = 0; t[ORC_T_CLAMPS]++; }
        if (jn > J - 1) { jn = J - 1; t[ORC_T_CLAMPS]++; }
        P->j = jn;
    }
    P->idx[ax] += side;
    if (leak) {
        const int64_t cn = orc_cell_of(g, P->idx);
        leak[(cn * nf + (face ^ 1)) * 2 + 1] += A->k[cn * J + P->j] * dl;
    }
    return 0;
}

static void* orc_time_thread(void* vp) {
    orc_time_args* T = (orc_time_args*)vp;
    orc_walk_args* A = &T->w;
    const orc_grid* g = A->g;
    const int J = g->J, KT = orc_nthr(g) + 1;
    const int64_t S = (int64_t)orc_ncell(g) * J;
    const size_t L = (size_t)orc_ncell(g) * 2 * g->ndim * 2;
    for (uint64_t pk = A->p0; pk < A->p1; ++pk) {
        orc_pstate P;
        orc_start(A, pk, &P, A->tally);
        double tau = T->t_edges[0];
        uint64_t d = 0;  /* dwell draws */
        int done = 0;
        double wgt = 1.0;  /* dust weights: the packet weight */
        for (int n = 0; n < T->nt && !done; ++n) {
            const double t_end = T->t_edges[n + 1];
            for (;;) {
                if (P.steps >= A->max_steps) { T->aborted++; done = 2; break; }
                const int64_t s = orc_cell_of(g, P.idx) * J + P.j;
                double ksum = 0.0;
                for (int q = 0; q < KT; ++q) ksum += A->rate[s * KT + q];  /* absorption included */
                /* eq. l_min_2: the smallest of the exponential leakage lengths is Exp(sum k) */
                const double dl = -log(orc_unif(orc_word(A->seed, pk, ORC_TIME, d++))) / ksum;
                T->dwells++;
                /* dust by weights (Sec. 2.6): over a path l the weight falls by
                 * exp(-k_a l); the path estimate takes the weight averaged along
                 * it, w (1 - e^{-k_a l}) / (k_a l) */
                const double ka = g->dust_weights ? g->dust_abs / g->R * (g->n_rel ? g->n_rel[s / J] : 1.0) : 0.0;
                if (tau + dl > t_end) {          /* causality: stay in the state until t_end */
                    const double l = t_end - tau;
                    T->path[(size_t)n * S + s] += l;
                    if (T->wpath) {
                        T->wpath[(size_t)n * S + s] += ka > 0.0 ? wgt * -expm1(-ka * l) / ka : wgt * l;
                        wgt *= exp(-ka * l);
                        T->wbins[(size_t)n * S + s] += wgt;
                    }
                    tau = t_end;
                    T->bins[(size_t)n * S + s]++;
                    break;
                }
                T->path[(size_t)n * S + s] += dl;
                if (T->wpath) {
                    T->wpath[(size_t)n * S + s] += ka > 0.0 ? wgt * -expm1(-ka * dl) / ka : wgt * dl;
                    wgt *= exp(-ka * dl);
                }
                tau += dl;
                int r = orc_time_transition(A, pk, &P, A->tally, dl, T->leak ? T->leak + (size_t)n * L : NULL);
                if (r == 1) { T->esc[n]++; done = 1; break; }
                if (r == 2) { done = 4; break; }
                if (T->wpath && wgt < ORC_W_MIN) { A->tally[ORC_T_ABSORBED]++; done = 4; break; }
                if (r == -1) { A->status = -2; done = 3; break; }
            }
        }
        A->tally[ORC_T_EVENT_DRAWS] += P.e;
    }
    return NULL;
}

/*
 * Time-dependent DDMC walk of packets [p0, p0+np), all emitted at the source at
 * t_edges[0] (a flash), through the steps [t_edges[n], t_edges[n+1]], n < nt.
 * Path lengths and times share one unit (c = 1), the unit of the grid's R.
 * In state s a packet draws a dwell path dl = -ln(xi) / K_s, K_s the sum of the
 * state's leakage coefficients (rate[s*K..]): by eq. l_min_1/2 the smallest of
 * the competing exponential lengths is Exp(K_s), independent of the process
 * that wins, which the categorical draw picks.  xi is word d of the packet's
 * time stream (lane d&3 of Philox4x32-10(ctr = (d>>2, p_lo, p_hi | 2^30))).
 * If the dwell would pass the step's end, the packet stays in its state until
 * t_end without leaking (Sec. 2.3) and draws a new dwell in the next step (the
 * exponential is memoryless).  Outputs, accumulated (+=):
 *   bins[n*S + s]: packets in state s at t_edges[n+1] (the bin estimate)
 *   path[n*S + s]: path length spent in state s during step n (the path estimate)
 *   esc[n]: packets escaped during step n;  tally: the walk's counters
 *   leak[((n*ncell + c)*2ndim + f)*2 + io] (if leak and k are given): the
 *       optical depths k dl of the leaks of eq. a_estimator through face f of
 *       cell c during step n, io = 0 leaving the cell (k of the cell at the
 *       bin it leaves), io = 1 entering it (k of the cell at the bin it
 *       enters); dl is the dwell that ended in the leak.  The acceleration of
 *       cell c is proportional to sum_f (leak[out] - leak[in]) n_f.
 *   wbins, wpath (required with dust weights, else NULL; nt x S): the bin and
 *       path estimates weighted by packet weight (Sec. 2.6: the weight falls by
 *       exp(-k_a l) over a path l; the path estimate takes the weight averaged
 *       along the path); packets below weight 1e-10 are eliminated.
 * with S = ncell * J.  DDMC tables only.  stats[3] = {transitions, dwell draws,
 * aborted}.  Returns 0, -1 on bad input, -2 if a packet met an MC state.
 */
int orc_walk_time(const orc_grid* g, const uint32_t* thr, const uint32_t* flags, const int32_t* rebin_m,
                  const uint32_t* rebin_thr, const double* rate, double x0, uint64_t seed, uint64_t p0, uint64_t np,
                  const double* t_edges, int nt, uint64_t max_steps, int nthreads, uint64_t* bins, double* path,
                  uint64_t* esc, uint64_t* tally, uint64_t* stats, const double* k, double* leak, double* wbins,
                  double* wpath) {
    if (!g || !thr || !flags || !rate || !t_edges || nt < 1 || !bins || !path || !esc || !tally || !stats) return -1;
    if (leak && !k) return -1;
    if ((!wbins) != (!wpath) || ((wbins != NULL) != (g->dust_weights != 0))) return -1;
    if (p0 + np > ((uint64_t)1 << 62)) return -1;
    for (int n = 0; n < nt; ++n)
        if (!(t_edges[n + 1] > t_edges[n])) return -1;
    orc_source src;
    if (orc_make_source(g, x0, &src)) return -1;
    if (nthreads < 1) nthreads = 1;
    if ((uint64_t)nthreads > np) nthreads = np ? (int)np : 1;
    const int L = orc_tally_len(g->J);
    const size_t S = (size_t)orc_ncell(g) * g->J;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
    orc_time_args* args = (orc_time_args*)calloc(nthreads, sizeof(orc_time_args));
    uint64_t* tl = (uint64_t*)calloc((size_t)nthreads * L, sizeof(uint64_t));
    uint64_t* tb = (uint64_t*)calloc((size_t)nthreads * nt * S, sizeof(uint64_t));
    double* tp = (double*)calloc((size_t)nthreads * nt * S, sizeof(double));
    uint64_t* te = (uint64_t*)calloc((size_t)nthreads * nt, sizeof(uint64_t));
    const size_t LN = (size_t)nt * orc_ncell(g) * 2 * g->ndim * 2;
    double* tlk = leak ? (double*)calloc((size_t)nthreads * LN, sizeof(double)) : NULL;
    double* twb = wbins ? (double*)calloc((size_t)nthreads * nt * S, sizeof(double)) : NULL;
    double* twp = wpath ? (double*)calloc((size_t)nthreads * nt * S, sizeof(double)) : NULL;
    for (int i = 0; i < nthreads; ++i) {
        orc_time_args* T = &args[i];
        orc_walk_args* A = &T->w;
        A->g = g; A->thr = thr; A->flags = flags; A->rebin_m = rebin_m; A->rebin_thr = rebin_thr;
        A->rate = rate; A->src = &src; A->seed = seed; A->max_steps = max_steps; A->k = k;
        A->p0 = p0 + np * (uint64_t)i / nthreads;
        A->p1 = p0 + np * (uint64_t)(i + 1) / nthreads;
        A->tally = tl + (size_t)i * L;
        T->t_edges = t_edges; T->nt = nt;
        T->leak = tlk ? tlk + (size_t)i * LN : NULL;
        T->wbins = twb ? twb + (size_t)i * nt * S : NULL;
        T->wpath = twp ? twp + (size_t)i * nt * S : NULL;
        T->bins = tb + (size_t)i * nt * S;
        T->path = tp + (size_t)i * nt * S;
        T->esc = te + (size_t)i * nt;
        pthread_create(&th[i], NULL, orc_time_thread, T);
    }
    int status = 0;
    memset(tally, 0, sizeof(uint64_t) * L);
    stats[0] = stats[1] = stats[2] = 0;
    for (int i = 0; i < nthreads; ++i) {
        pthread_join(th[i], NULL);
        for (int q = 0; q < L; ++q) tally[q] += tl[(size_t)i * L + q];
        for (size_t q = 0; q < (size_t)nt * S; ++q) {
            bins[q] += tb[(size_t)i * nt * S + q];
            path[q] += tp[(size_t)i * nt * S + q];
        }
        for (int n = 0; n < nt; ++n) esc[n] += te[(size_t)i * nt + n];
        if (tlk)
            for (size_t q = 0; q < LN; ++q) leak[q] += tlk[(size_t)i * LN + q];
        if (twb)
            for (size_t q = 0; q < (size_t)nt * S; ++q) {
                wbins[q] += twb[(size_t)i * nt * S + q];
                wpath[q] += twp[(size_t)i * nt * S + q];
            }
        stats[0] += args[i].w.tally[ORC_T_STEPS];
        stats[1] += args[i].dwells;
        stats[2] += args[i].aborted;
        if (args[i].w.status) status = args[i].w.status;
    }
    free(th); free(args); free(tl); free(tb); free(tp); free(te); free(tlk); free(twb); free(twp);
    return status;
}

/* Start packets [p0, p0+np) at the source and advance each by at most
 * n_trans transitions (a bounded slice of the walk, as one time slice of the
 * GPU walk does); the tallies count what happened within the slice. */
int orc_walk_slice(const orc_grid* g, const uint32_t* thr, const uint32_t* flags, const int32_t* rebin_m,
                   const uint32_t* rebin_thr, const double* k, double x0, uint64_t seed, uint64_t p0, uint64_t np,
                   uint64_t n_trans, int nthreads, uint64_t* tally) {
    return orc_walk_run(g, thr, flags, rebin_m, rebin_thr, NULL, k, x0, seed, p0, np, (uint64_t)1 << 62, 0, n_trans,
                        nthreads, tally, NULL, NULL);
}

/*
 * Replay packet `pk` for at most n_trans transitions; writes its state
 * (cell index, bin, transitions, event draws, done flag) to out[5] and its
 * tallies to tally (orc_tally_len(J) words, overwritten).
 */
int orc_replay_packet(const orc_grid* g, const uint32_t* thr, const uint32_t* flags, const int32_t* rebin_m,
                      const uint32_t* rebin_thr, const double* k, double x0, uint64_t seed, uint64_t pk,
                      uint64_t n_trans, uint64_t max_steps, uint64_t* out, uint64_t* tally) {
    orc_source src;
    if (orc_make_source(g, x0, &src)) return -1;
    orc_walk_args A;
    memset(&A, 0, sizeof(A));
    A.g = g; A.thr = thr; A.flags = flags; A.rebin_m = rebin_m; A.rebin_thr = rebin_thr; A.src = &src;
    A.seed = seed; A.max_steps = max_steps; A.k = k;
    double* upar = NULL;
    if (g->hybrid) {
        if (!k) return -1;
        upar = (double*)malloc(sizeof(double) * 2 * ORC_UPAR_N);
        orc_upar_table(orc_damping(g->T), upar);
    }
    A.upar = upar;
    memset(tally, 0, sizeof(uint64_t) * orc_tally_len(g->J));
    orc_pstate P;
    orc_start(&A, pk, &P, tally);
    orc_advance(&A, pk, &P, n_trans, tally);
    tally[ORC_T_EVENT_DRAWS] += P.e;
    out[0] = (uint64_t)orc_cell_of(g, P.idx);
    out[1] = (uint64_t)P.j;
    out[2] = P.steps;
    out[3] = P.e;
    out[4] = (uint64_t)P.done;
    free(upar);
    return A.status;
}

/* Outgoing frequencies of n independent scatterings of a photon at x_in with
 * incoming direction +e_z (isotropic phase function, no recoil); sample i uses
 * the event stream of packet i.  Their density is R_II-A(x_out, x_in). */
void orc_scatter_samples(double T, double x_in, uint64_t seed, uint64_t n, double* out) {
    orc_walk_args A;
    memset(&A, 0, sizeof(A));
    A.seed = seed;
    double* upar = (double*)malloc(sizeof(double) * 2 * ORC_UPAR_N);
    const double a = orc_damping(T);
    orc_upar_table(a, upar);
    A.upar = upar;
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t e = 0;
        double d[3] = {0.0, 0.0, 1.0};
        out[i] = orc_scatter(&A, a, x_in, d, i, &e);
    }
    free(upar);
}

/* ------------------------------------------------------------------------- */
/* First passage through a uniform brick (training data of the learned exit  */
/* proposal)                                                                 */
/* ------------------------------------------------------------------------- */

/*
 * Sample i (packet id p0+i under `seed`) reads event words 0..2 of its event
 * stream: w0 picks a density level l = floor(w0 L / 2^32), w1 a start bin
 * j0 = jlo[l] + floor(w1 n / 2^32) with n = jhi[l] - jlo[l] + 1, and w2 a
 * cell of the b^3 brick, m = floor(w2 b^3 / 2^32) = i0 + b i1 + b^2 i2.  The
 * cell is folded into the fundamental domain of the cube's symmetry group:
 * each coordinate i becomes min(i, b-1-i), then the three are sorted
 * ascending, (c0 <= c1 <= c2).  A uniform static brick is invariant under
 * these reflections and axis permutations, so the first passage from any cell
 * is the image of one from its folded cell.  From (c, j0) the sample takes
 * DDMC transitions with the rows of an interior cell of a uniform medium at
 * that level (3D rows: 7 cumulative thresholds, then the flag word, per bin)
 * until its first spatial move leaves the brick, or `cap` transitions.
 * out[8*i..]: {l, j0, folded start cell c0 + b c1 + b^2 c2, exit face (0..5 =
 * -x,+x,-y,+y,-z,+z; 6 = step cap reached), exit bin, exit position (the
 * coordinates of the last cell inside the brick along the two axes other than
 * the exit face's, lower axis first: q1 + b q2; -1 on a cap), 0, 0};
 * steps[i]: transitions.
 */
void orc_fp_samples(const uint32_t* rows, int L, int J, int b, const int32_t* jlo, const int32_t* jhi,
                    uint64_t seed, uint64_t p0, uint64_t n, uint64_t cap, int32_t* out, uint64_t* steps) {
    for (uint64_t i = 0; i < n; ++i) {
        const uint64_t pk = p0 + i;
        const uint32_t w0 = orc_word(seed, pk, ORC_EVENT, 0);
        const uint32_t w1 = orc_word(seed, pk, ORC_EVENT, 1);
        const uint32_t w2 = orc_word(seed, pk, ORC_EVENT, 2);
        const int l = (int)(((uint64_t)w0 * (uint64_t)L) >> 32);
        const int nb = jhi[l] - jlo[l] + 1;
        int j = jlo[l] + (int)(((uint64_t)w1 * (uint64_t)nb) >> 32);
        const int m = (int)(((uint64_t)w2 * (uint64_t)(b * b * b)) >> 32);
        int idx[3] = {m % b, (m / b) % b, m / (b * b)};
        /* fold: reflect each axis into its lower half, then sort */
        for (int a = 0; a < 3; ++a)
            if (b - 1 - idx[a] < idx[a]) idx[a] = b - 1 - idx[a];
        for (int pass = 0; pass < 2; ++pass)
            for (int a = 0; a < 2; ++a)
                if (idx[a + 1] < idx[a]) { int tmp = idx[a]; idx[a] = idx[a + 1]; idx[a + 1] = tmp; }
        out[8 * i + 0] = l;
        out[8 * i + 1] = j;
        out[8 * i + 2] = idx[0] + b * idx[1] + b * b * idx[2];
        int face = 6, pos = -1;
        uint64_t t = 0;
        while (t < cap) {
            const uint32_t* r = rows + ((size_t)l * J + j) * 8;
            uint32_t wt = orc_word(seed, pk, ORC_TRANS, t);
            ++t;
            int o = 0;
            while (o < 7 && wt >= r[o]) ++o;
            if (o < 2) { j += o ? 1 : -1; continue; }
            int f = o - 2, ax = f / 2, side = (f & 1) ? 1 : -1;
            if (idx[ax] + side < 0 || idx[ax] + side >= b) {
                face = f;
                const int u = ax == 0 ? 1 : 0, v = ax == 2 ? 1 : 2;  /* the other two axes, lower first */
                pos = idx[u] + b * idx[v];
                break;
            }
            idx[ax] += side;
        }
        out[8 * i + 3] = face;
        out[8 * i + 4] = j;
        out[8 * i + 5] = pos;
        out[8 * i + 6] = 0;
        out[8 * i + 7] = 0;
        steps[i] = t;
    }
}

/* First passages out of non-uniform regions of a grid's own medium (training
 * data of the learned proposal for media that vary from cell to cell).  The
 * grid is cut into bricks of bl^3 cells, brick coordinate (i + sh) / bl of cell
 * index i on every axis (brick index axis 0 fastest, nbx bricks per axis); a
 * brick's region is its inner cube of side r = bl - 2 m.  Sample i uses packet
 * pk = p0 + i: event draw 0 picks the brick bricks[k], k = (w0 nel) >> 32;
 * draw 1 the start cell of the region, (w1 r^3) >> 32 (axis 0 fastest); draw 2
 * the start bin among that brick's listed bins bins[off[k] ..  off[k+1]).  The
 * packet then takes the walk's own transitions on the grid's table (Sec. 2.3;
 * Doppler rebins take the next event draws) until an outcome would carry it
 * out of the region: that crossing is not made, and the sample records the
 * face, the bin and the cell on the face it leaves from.  Out, per sample (8
 * ints): brick, start bin, start cell (region-local index), exit face (6: none
 * within cap transitions), exit bin, exit cell on the face (the other two axes,
 * lower axis first, u + r v), event draws taken by rebins, 0; steps: the
 * transitions taken, the crossing one included. */
void orc_fp_region_samples(const orc_grid* g, const uint32_t* thr, const uint32_t* flags, const int32_t* rebin_m,
                           const uint32_t* rebin_thr, int bl, int sh, int m, int nbx, const int32_t* bricks,
                           int nel, const int32_t* off, const int32_t* bins, uint64_t seed, uint64_t p0, uint64_t n,
                           uint64_t cap, int32_t* out, uint64_t* steps) {
    const int J = g->J, NT = orc_nthr(g), nf = 2 * g->ndim, r = bl - 2 * m;
    for (uint64_t i = 0; i < n; ++i) {
        const uint64_t pk = p0 + i;
        const uint32_t w0 = orc_word(seed, pk, ORC_EVENT, 0);
        const uint32_t w1 = orc_word(seed, pk, ORC_EVENT, 1);
        const uint32_t w2 = orc_word(seed, pk, ORC_EVENT, 2);
        const int k = (int)(((uint64_t)w0 * (uint64_t)nel) >> 32);
        const int br = bricks[k];
        const int bc[3] = {br % nbx, (br / nbx) % nbx, br / (nbx * nbx)};
        const int mc = (int)(((uint64_t)w1 * (uint64_t)(r * r * r)) >> 32);
        int l[3] = {mc % r, (mc / r) % r, mc / (r * r)};
        int base[3];
        for (int a = 0; a < 3; ++a) base[a] = bc[a] * bl - sh + m;
        const int cnt = off[k + 1] - off[k];
        int j = bins[off[k] + (int)(((uint64_t)w2 * (uint64_t)cnt) >> 32)];
        out[8 * i + 0] = br;
        out[8 * i + 1] = j;
        out[8 * i + 2] = mc;
        uint64_t e = 3, t = 0;
        int face = 6, pos = -1;
        while (t < cap) {
            int idx[3] = {base[0] + l[0], base[1] + l[1], base[2] + l[2]};
            const int64_t c = orc_cell_of(g, idx);
            const int64_t st = c * J + j;
            const uint32_t wt = orc_word(seed, pk, ORC_TRANS, t);
            ++t;
            int o = 0;
            while (o < NT && wt >= thr[st * NT + o]) ++o;
            const unsigned act = (flags[st] >> (2 * o)) & 3u;
            if (o < 2) { j += o ? 1 : -1; continue; }
            const int f = o - 2, ax = f / 2, side = (f & 1) ? 1 : -1;
            if (l[ax] + side < 0 || l[ax] + side >= r) {
                face = f;
                const int u = ax == 0 ? 1 : 0, v = ax == 2 ? 1 : 2;
                pos = l[u] + r * l[v];
                break;
            }
            if (act == ORC_ACT_ESCAPE || act == ORC_ACT_TO_MC) break;  /* not inside a region: no sample */
            if (act == ORC_ACT_REBIN) {
                const uint32_t wr = orc_word(seed, pk, ORC_EVENT, e++);
                int jn = j + rebin_m[c * nf + f] + (wr >= rebin_thr[c * nf + f] ? 1 : 0);
                j = jn < 0 ? 0 : (jn > J - 1 ? J - 1 : jn);
            }
            l[ax] += side;
        }
        out[8 * i + 3] = face;
        out[8 * i + 4] = j;
        out[8 * i + 5] = pos;
        out[8 * i + 6] = (int32_t)(e - 3);
        out[8 * i + 7] = 0;
        steps[i] = t;
    }
}
