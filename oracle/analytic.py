"""Closed forms and exact solves that pin the oracle and judge the method.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* Neufeld / Harrington slab escape profile (Sec. 3.2, eq. Neufeld):
  J(x, a tau0) = x^2 / (4 sqrt(6 pi) a tau0) sech(sqrt(pi^3/54) x^3 / (a tau0)),
  normalised to 1/(4 pi).  Its bin masses have a closed form through the
  Gudermannian gd(y) = 2 atan(tanh(y/2)): with c = sqrt(pi^3/54)/(a tau0) the
  normalised CDF is 1/2 + gd(c x^3)/pi.
* The DDMC walk with a fixed (quantised) table is an absorbing Markov chain
  over states (cell, bin).  Expected visits v solve (I - P)^T v = s for the
  source distribution s; expected escapes per state/outcome are v_s q_so; the
  mean and second moment of the number of transitions solve (I - P) t = 1 and
  (I - P) m2 = 2 t - 1.  This is exact for the walk, up to linear-algebra
  rounding, with no Monte Carlo noise.
* Quadrature references for the Dawson integral, the Voigt function of eq. H
  (also through the Faddeeva function, H(a,x) = Re w(x + i a)) and bin means.
"""
from __future__ import annotations

import numpy as np
import scipy.integrate as si
import scipy.linalg as sla
import scipy.optimize as so
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import scipy.special as ss

TWO32 = 4294967296.0
ACT_MOVE, ACT_ESCAPE, ACT_TO_MC, ACT_REBIN = 0, 1, 2, 3
FLAG_MOVING = 1 << 30
FLAG_THIN = 1 << 31


# --------------------------------------------------------------------------- Neufeld profile
def neufeld_J(x, atau0):
    """Angle-averaged escaping intensity of a static slab, eq. Neufeld."""
    x = np.asarray(x, dtype=np.float64)
    c = np.sqrt(np.pi ** 3 / 54.0) / atau0
    return x * x / (4.0 * np.sqrt(6.0 * np.pi) * atau0) / np.cosh(c * x ** 3)


def neufeld_cdf(x, atau0):
    """Normalised CDF of 4 pi J(x): 1/2 + gd(c x^3)/pi = (2/pi) atan(exp(c x^3))."""
    c = np.sqrt(np.pi ** 3 / 54.0) / atau0
    y = c * np.asarray(x, dtype=np.float64) ** 3
    return 2.0 / np.pi * np.arctan(np.exp(y))


def neufeld_bin_mass(edges, atau0):
    """Probability that an escaping photon falls in each bin of ``edges``.

    Differences are taken of the lower tail (2/pi) atan(e^y) left of line centre
    and of the upper tail (2/pi) atan(e^-y) right of it, so far-wing bins keep
    full relative precision."""
    c = np.sqrt(np.pi ** 3 / 54.0) / atau0
    y = c * np.asarray(edges, dtype=np.float64) ** 3
    lo = 2.0 / np.pi * np.arctan(np.exp(np.minimum(y, 0.0)))      # F(x) for x <= 0
    up = 2.0 / np.pi * np.arctan(np.exp(-np.maximum(y, 0.0)))     # 1 - F(x) for x >= 0
    F = np.where(y <= 0.0, lo, 1.0 - up)
    mass = np.diff(F)
    right = y[:-1] >= 0.0
    left = y[1:] <= 0.0
    mass[right] = up[:-1][right] - up[1:][right]
    mass[left] = lo[1:][left] - lo[:-1][left]
    return mass


def neufeld_peak(atau0):
    """Peak location and height: xbar tanh xbar = 2/3 with xbar = sqrt(pi^3/54) x^3 / (a tau0).

    Returns (xbar, x_p, J(x_p))."""
    xbar = so.brentq(lambda v: v * np.tanh(v) - 2.0 / 3.0, 0.1, 5.0, xtol=1e-15)
    x_p = (xbar * atau0 / np.sqrt(np.pi ** 3 / 54.0)) ** (1.0 / 3.0)
    return xbar, x_p, float(neufeld_J(x_p, atau0))


# --------------------------------------------------------------------------- quadrature references
def dawson_quad(x):
    """F(x) = int_0^x exp(y^2 - x^2) dy by adaptive quadrature of the definition."""
    x = float(x)
    if x == 0.0:
        return 0.0
    val, _ = si.quad(lambda y: np.exp((y - x) * (y + x)), 0.0, x, epsabs=0.0, epsrel=1e-13, limit=400)
    return val


def voigt_faddeeva(a, x):
    """H(a,x) = Re w(x + i a): the exact Voigt-Hjerting function of eq. H."""
    return np.real(ss.wofz(np.asarray(x, dtype=np.float64) + 1j * a))


def voigt_quad(a, x):
    """H(a,x) = (a/pi) int exp(-y^2) / (a^2 + (y-x)^2) dy by quadrature (eq. H)."""
    f = lambda y: np.exp(-y * y) / (a * a + (y - x) ** 2)
    pts = sorted({-6.0, x - 50 * a, x, x + 50 * a, 6.0})
    pts = [p for p in pts if -8.0 <= p <= 8.0]
    val, _ = si.quad(f, -8.0, 8.0, points=pts, epsabs=0.0, epsrel=1e-12, limit=800)
    return a / np.pi * val


def bin_mean_quad(Hfun, a, xlo, xhi):
    val, _ = si.quad(lambda y: Hfun(a, y), xlo, xhi, epsabs=0.0, epsrel=1e-12, limit=400)
    return val / (xhi - xlo)


# --------------------------------------------------------------------------- exact absorbing chain
def quantised_probs(thr: np.ndarray) -> np.ndarray:
    """Per-state outcome probabilities implied by the cumulative thresholds: shape (S, K)."""
    S, Km1 = thr.shape
    c = np.concatenate([np.zeros((S, 1)), thr.astype(np.float64), np.full((S, 1), TWO32)], axis=1)
    return np.diff(c, axis=1) / TWO32


def source_states(w, edges=None):
    """States and probabilities of the centre source: the centre cell(s) (both
    neighbours of the midplane for even counts) and the bin(s) containing x0."""
    cells = []
    for a in range(3):
        m = w.n[a]
        cells.append([m // 2] if m % 2 else [m // 2 - 1, m // 2])
    e = w.edges() if edges is None else np.asarray(edges)
    bins = [j for j in range(1, w.J) if e[j] == w.x0]
    bins = [bins[0] - 1, bins[0]] if bins else [j for j in range(w.J) if e[j] < w.x0 < e[j + 1]]
    states, probs = [], []
    n0, n1 = w.n[0], w.n[1]
    for i2 in cells[2]:
        for i1 in cells[1]:
            for i0 in cells[0]:
                c = i0 + n0 * (i1 + n1 * i2)
                for j in bins:
                    states.append(c * w.J + j)
                    probs.append(1.0 / (len(cells[0]) * len(cells[1]) * len(cells[2]) * len(bins)))
    return np.array(states, dtype=np.int64), np.array(probs)


def _neighbour(w, c, axis, side):
    n = w.n
    idx = [c % n[0], (c // n[0]) % n[1], c // (n[0] * n[1])]
    idx[axis] += side
    if idx[axis] < 0 or idx[axis] >= n[axis]:
        return -1
    return idx[0] + n[0] * (idx[1] + n[1] * idx[2])


def chain_matrix(w, table):
    """Transition matrix of the DDMC walk between its states (sparse, S x S;
    each row sums to one minus the state's escape probability) and the
    escape probability per (state, outcome), from the quantised thresholds."""
    J, K = w.J, 2 + 2 * w.ndim
    thr, flags = table["thr"], table["flags"]
    S = thr.shape[0]
    q = quantised_probs(thr)
    nf = 2 * w.ndim
    rows, cols, vals = [], [], []
    esc = np.zeros((S, K))
    for s in range(S):
        c, j = divmod(s, J)
        fl = int(flags[s])
        for o in range(K):
            p = q[s, o]
            if p == 0.0:
                continue
            act = (fl >> (2 * o)) & 3
            if act == ACT_ESCAPE:
                esc[s, o] = p
                continue
            if act == ACT_TO_MC:
                raise ValueError("chain_solve handles DDMC-only tables")
            if o < 2:
                rows.append(s); cols.append(s + (1 if o else -1)); vals.append(p)
                continue
            face = o - 2
            nb = _neighbour(w, c, face // 2, 1 if face & 1 else -1)
            if act == ACT_MOVE:
                rows.append(s); cols.append(nb * J + j); vals.append(p)
            else:
                m = int(table["rebin_m"][c * nf + face])
                pr = float(table["rebin_thr"][c * nf + face]) / TWO32
                for jn, pj in ((j + m, pr), (j + m + 1, 1.0 - pr)):
                    jn = min(max(jn, 0), J - 1)
                    if pj > 0:
                        rows.append(s); cols.append(nb * J + jn); vals.append(p * pj)
    return sp.csr_matrix((vals, (rows, cols)), shape=(S, S)), esc


def chain_solve(w, table, edges=None):
    """Exact expectations of the DDMC walk on a quantised table.

    Returns a dict with the expected escape histogram per emitted packet (J+2
    bins, static cells only), expected escapes per face, escapes per
    (state, outcome), the mean and variance of the number of transitions."""
    J, K = w.J, 2 + 2 * w.ndim
    flags = table["flags"]
    P, esc = chain_matrix(w, table)
    S = P.shape[0]
    A = (sp.identity(S, format="csr") - P).tocsc()
    lu = spla.splu(A)
    src_s, src_p = source_states(w, edges)
    src = np.zeros(S)
    src[src_s] = src_p
    v = lu.solve(src, trans="T")
    t = lu.solve(np.ones(S))
    m2 = lu.solve(2.0 * t - 1.0)
    mean = float(src @ t)
    var = float(src @ m2) - mean * mean
    esc_so = v[:, None] * esc
    hist = np.zeros(J + 2)
    faces = np.zeros(6)
    for o in range(2, K):
        faces[o - 2] = esc_so[:, o].sum()
        per_state = esc_so[:, o].reshape(-1, J)
        moving = (flags.reshape(-1, J) & FLAG_MOVING) != 0
        hist[1:J + 1] += np.where(moving, 0.0, per_state).sum(axis=0)
    return dict(hist=hist, faces=faces, esc_so=esc_so, visits=v, steps_mean=mean, steps_var=var,
                escape_total=float(esc_so.sum()))


def leak_matrices(w, table):
    """For the leaks of eq. a_estimator: Lout[s, c*2ndim + f] = k_s P(f | s)
    (the cell c of s leaves through face f), Lin[s, c'*2ndim + f'] = P(f | s)
    times the expected k of the entered state of c' (f' the face c' is entered
    through; Doppler rebins averaged), and Pf[s, f] = P(f | s), from the
    quantised thresholds."""
    J, nf = w.J, 2 * w.ndim
    thr, flags, k = table["thr"], table["flags"], np.asarray(table["k"], dtype=np.float64)
    S = thr.shape[0]
    q = quantised_probs(thr)
    Lout = np.zeros((S, w.ncell * nf))
    Lin = np.zeros((S, w.ncell * nf))
    for s in range(S):
        c, j = divmod(s, J)
        fl = int(flags[s])
        for f in range(nf):
            p = q[s, 2 + f]
            if p == 0.0:
                continue
            Lout[s, c * nf + f] += k[s] * p
            act = (fl >> (2 * (2 + f))) & 3
            if act == ACT_ESCAPE:
                continue
            if act == ACT_TO_MC:
                raise ValueError("leak_matrices handles DDMC-only tables")
            nb = _neighbour(w, c, f // 2, 1 if f & 1 else -1)
            if act == ACT_MOVE:
                Lin[s, nb * nf + (f ^ 1)] += p * k[nb * J + j]
            else:
                m = int(table["rebin_m"][c * nf + f])
                pr = float(table["rebin_thr"][c * nf + f]) / TWO32
                for jn, pj in ((j + m, pr), (j + m + 1, 1.0 - pr)):
                    jn = min(max(jn, 0), J - 1)
                    Lin[s, nb * nf + (f ^ 1)] += p * pj * k[nb * J + jn]
    return Lout, Lin, q[:, 2:2 + nf]


def chain_time(w, table, t_edges, edges=None, leaks=False):
    """Exact expectations of the time-dependent DDMC walk (Sec. 2.3): the walk
    is a continuous-time Markov chain whose state s is left at the total
    leakage rate K_s (per unit path length; c = 1) for the outcomes of the
    quantised thresholds, so the occupancy is p(t) = p(0) exp(Q t) with
    Q = diag(K) (P - I).  For time steps [t_edges[n], t_edges[n+1]] returns
    the occupancy at each step's end (nt x S), the expected path length spent
    in each state during each step (nt x S), both per emitted packet, and the
    escape probability per step (nt).  Dense: for small grids.

    leaks=True also returns the expected optical depths of the leaks of eq.
    a_estimator (nt x ncell x 2ndim x 2, leaving / entering each face) and the
    expected number of leaks (same shape).  A leak out of s at time u ends a
    dwell that began at the later of the previous jump and the step's start
    (every step draws a fresh dwell), so by the memoryless property its
    expected length sum over the step is P(f|s) times the completed-dwell mass
    C_s = int p_s du - r_s(t_end), where r_s(t) = int p_s(u) exp(-K_s (t - u)) du
    (the expected length of the dwell cut off at t_end) solves r' = p - K r.
    [p, path, r] evolve together under one augmented matrix exponential."""
    P, esc = chain_matrix(w, table)
    S = P.shape[0]
    K = np.asarray(table["rate"], dtype=np.float64).sum(axis=1)
    Q = K[:, None] * (P.toarray() - np.eye(S))
    src_s, src_p = source_states(w, edges)
    p = np.zeros(S)
    p[src_s] = src_p
    if leaks:
        Lout, Lin, Pf = leak_matrices(w, table)
        nf = 2 * w.ndim
    occ, path, esc_t, lk, cnt = [], [], [], [], []
    for n in range(len(t_edges) - 1):
        h = float(t_edges[n + 1] - t_edges[n])
        if not leaks:
            M = np.zeros((2 * S, 2 * S))
            M[:S, :S] = Q * h
            M[:S, S:] = np.eye(S) * h
            E = sla.expm(M)  # top-left exp(Q h), top-right int_0^h exp(Q u) du
            pn = p @ E[:S, :S]
            path.append(p @ E[:S, S:])
        else:
            M = np.zeros((3 * S, 3 * S))
            M[:S, :S] = Q * h
            M[:S, S:2 * S] = np.eye(S) * h
            M[:S, 2 * S:] = np.eye(S) * h
            M[2 * S:, 2 * S:] = -np.diag(K) * h
            E = sla.expm(M)
            pn = p @ E[:S, :S]
            ps = p @ E[:S, S:2 * S]
            r = p @ E[:S, 2 * S:]
            path.append(ps)
            C = ps - r
            lk.append(np.stack([(C @ Lout).reshape(w.ncell, nf), (C @ Lin).reshape(w.ncell, nf)], axis=-1))
            ncount = (ps * K)[:, None] * Pf  # expected leaks per (state, face)
            out_c = np.zeros((w.ncell, nf))
            for f in range(nf):
                np.add.at(out_c[:, f], np.arange(S) // w.J, ncount[:, f])
            cnt.append(out_c)
        occ.append(pn)
        esc_t.append(p.sum() - pn.sum())
        p = pn
    if leaks:
        return np.array(occ), np.array(path), np.array(esc_t), np.array(lk), np.array(cnt)
    return np.array(occ), np.array(path), np.array(esc_t)


# --------------------------------------------------------------------------- comparisons
def l1_distance(p, q):
    p = np.asarray(p, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    return float(np.abs(p / p.sum() - q / q.sum()).sum())


def compare_counts_to_probs(counts, probs, n, min_expected=20.0):
    """Bin-wise z-scores of multinomial counts against exact probabilities.

    Returns (max |z|, fraction of bins with |z| > 3, chi2 p-value) over bins with
    expected count >= min_expected (G12 reading of 'within 3 sigma')."""
    counts = np.asarray(counts, dtype=np.float64)
    probs = np.asarray(probs, dtype=np.float64)
    e = n * probs
    sel = e >= min_expected
    z = (counts[sel] - e[sel]) / np.sqrt(e[sel] * (1.0 - probs[sel]))
    chi2 = float(((counts[sel] - e[sel]) ** 2 / e[sel]).sum())
    dof = max(int(sel.sum()) - 1, 1)
    pval = float(ss.chdtrc(dof, chi2))
    return float(np.abs(z).max()) if z.size else 0.0, float((np.abs(z) > 3).mean()) if z.size else 0.0, pval


def compare_two_samples(c1, n1, c2, n2, min_expected=20.0):
    """Bin-wise z-scores between two independent multinomial samples."""
    c1 = np.asarray(c1, dtype=np.float64)
    c2 = np.asarray(c2, dtype=np.float64)
    p1, p2 = c1 / n1, c2 / n2
    sel = (c1 + c2) * min(n1, n2) / (n1 + n2) >= min_expected
    var = p1[sel] * (1 - p1[sel]) / n1 + p2[sel] * (1 - p2[sel]) / n2
    z = (p1[sel] - p2[sel]) / np.sqrt(np.maximum(var, 1e-300))
    return float(np.abs(z).max()) if z.size else 0.0, float((np.abs(z) > 3).mean()) if z.size else 0.0


# --------------------------------------------------------------------------- redistribution (Appendix A)
def R_IIA(x, xp, a):
    """Angle-averaged redistribution for isotropic coherent scattering without
    recoil (Appendix A): R(x, x') = 1/(pi H(x',a)) int_zeta^inf e^{-u^2}
    [atan((xmin + u)/a) - atan((xmax - u)/a)] du, zeta = |x - x'|/2; the
    density of the outgoing x given the incoming x'."""
    xmax, xmin = max(x, xp), min(x, xp)
    zeta = 0.5 * abs(x - xp)
    f = lambda u: np.exp(-u * u) * (np.arctan((xmin + u) / a) - np.arctan((xmax - u) / a))
    pts = [p for p in (zeta, 0.5 * (xmax - xmin) + 0.0, xmax, abs(xmax)) if p >= zeta]
    val, _ = si.quad(f, zeta, zeta + 12.0, points=sorted(set(pts))[1:] or None, epsabs=1e-14, epsrel=1e-10,
                     limit=400)
    return val / (np.pi * voigt_faddeeva(a, xp))


def R_IA_core(x, xp):
    """Core (a -> 0) limit printed in Appendix A: (sqrt(pi)/2) e^{x'^2} erfc(max(|x|,|x'|))."""
    return 0.5 * np.sqrt(np.pi) * np.exp(xp * xp) * ss.erfc(max(abs(x), abs(xp)))


def R_IIA_wing(x, xp):
    """Wing limit printed in Appendix A: (2x'/(x+x'))^2 [e^{-zeta^2}/sqrt(pi) - zeta erfc(zeta)]."""
    zeta = 0.5 * abs(x - xp)
    return (2.0 * xp / (x + xp)) ** 2 * (np.exp(-zeta * zeta) / np.sqrt(np.pi) - zeta * ss.erfc(zeta))


def redistribution_cdf_at(edges, xp, a, span=14.0):
    """F(e | x') = int_{-inf}^{e} R_II-A(x, x') dx at every edge e (normalised by
    the total, which is 1 up to the quadrature error), by adaptive
    quadrature of R_II-A over the pieces between the edges, x' and -x' (the
    kinks of R in x) and at the integers, within x' +- span (R is below
    e^{-(span/2)^2} beyond)."""
    lo, hi = xp - span, xp + span
    unit = list(np.arange(np.ceil(lo), hi))  # unit pieces keep the adaptive rule local
    cuts = sorted(set([lo, hi] + unit + [e for e in edges if lo < e < hi] + [p for p in (xp, -xp) if lo < p < hi]))
    cum = [0.0]
    for u, v in zip(cuts[:-1], cuts[1:]):
        val, _ = si.quad(lambda x: R_IIA(x, xp, a), u, v, epsabs=1e-11, epsrel=1e-8, limit=100)
        cum.append(cum[-1] + val)
    cuts, cum = np.array(cuts), np.array(cum)
    # normalised by the total mass (1 up to the quadrature error)
    return np.interp(np.asarray(edges, dtype=np.float64), cuts, cum, left=0.0, right=cum[-1]) / cum[-1]


def redistribution_cdf(edges, a, n_sub=3):
    """Eq. R_discrete as cumulative probabilities: row j' holds, for the J-1
    interior edges e_1..e_{J-1}, the average over x' in bin j' of F(e | x'), the
    x' integral taken with n_sub Gauss-Legendre nodes (uniform weight in the
    bin, as the equation's 1/dx_j' average).  Outgoing frequencies beyond the
    grid ends fall in the end bins (no flux beyond the grid, as for the
    leakage).  Returns (J, J-1)."""
    e = np.asarray(edges, dtype=np.float64)
    J = len(e) - 1
    gx, gw = np.polynomial.legendre.leggauss(n_sub)
    C = np.zeros((J, J - 1))
    for jp in range(J):
        for xg, wg in zip(gx, gw):
            xp = 0.5 * (e[jp + 1] - e[jp]) * xg + 0.5 * (e[jp + 1] + e[jp])
            F = redistribution_cdf_at(e, xp, a)
            C[jp] += 0.5 * wg * F[1:J]
    return C


def redistribution_thresholds(C):
    """32-bit thresholds of cumulative probabilities: round half to even of
    C 2^32, saturated at 2^32 - 1 (the rule of the leakage thresholds)."""
    return np.minimum(np.rint(np.asarray(C) * TWO32), TWO32 - 1).astype(np.uint32)


def R_IIA_bin_probs(edges, xp, a, n_sub=8):
    """Probability of each outgoing-frequency bin, integrating R_II-A over the bin
    with Gauss-Legendre nodes."""
    gx, gw = np.polynomial.legendre.leggauss(n_sub)
    out = np.zeros(len(edges) - 1)
    for i in range(len(edges) - 1):
        lo, hi = edges[i], edges[i + 1]
        xs = 0.5 * (hi - lo) * gx + 0.5 * (hi + lo)
        out[i] = 0.5 * (hi - lo) * sum(w * R_IIA(x, xp, a) for x, w in zip(xs, gw))
    return out
