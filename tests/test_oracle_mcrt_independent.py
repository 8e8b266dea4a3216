"""The oracle's continuous MC (Sec. 5.2, Appendix A) against an independent
Monte Carlo radiative transfer of the same problem.

The oracle's MC alone (every state thin) is the brute-force MCRT of the
method: flights with k = k0 H(a, x), coherent isotropic scattering in the
atom frame, escape through the faces.  Its other pins check single pieces:
one flight (the first-flight escape fraction), one scattering (the law of x'
against R_II-A) and the all-thick limit.  This file checks the whole chain of
flights and scatterings in a medium against a second implementation that
shares no step with it:

* the profile is the exact Voigt function Re w(x + i a) (Faddeeva), not the
  second-order expansion eq. H_approx;
* the atom velocity along the photon is drawn from its density
  f(u) ~ exp(-u^2) / ((x - u)^2 + a^2) by rejection from a two-part envelope
  split at |u - x| = 1/2: a Gaussian bounded by 1 / (1/4 + a^2) away from
  the resonance and a Lorentzian bounded by the largest exp(-u^2) near it;
* the frequency change is written with vectors, x' = x - u.n + u.n' for the
  atom velocity u = u_par n + u_perp1 e1 + u_perp2 e2 and directions n, n',
  not with the scattering-angle form the oracle uses;
* photons are followed in numpy, all at once, with numpy's generator.

Only the problem is shared: a one-cell static slab of half-thickness R and
line-centre optical depth tau0, photons started uniformly in the cell with an
isotropic direction and x uniform in the source bins, escape spectrum
tallied in the grid's bins (under- and overflow included)."""
import numpy as np
import pytest
import scipy.special as ss

from oracle import coracle as C
from paper_1709_10187_gb300 import workloads as W

N = 40_000
SLAB = W.Workload("thin_slab_tau10_1x60", 1, (1, 1, 1), 60, -6.0, 6.0, 10.0, 1.0e4, N, 0x5EED0411)


def _voigt(a, x):
    return ss.wofz(x + 1j * a).real


def _atom_velocity(rng, a, x, d=0.5):
    """u_par given x (arrays), exact: a mixture of two envelopes of
    g(u) = exp(-u^2) / ((x - u)^2 + a^2).
      away (|u - x| > d): g <= exp(-u^2) / (d^2 + a^2): a Gaussian proposal
        (variance 1/2), accepted with (d^2 + a^2) / ((x - u)^2 + a^2);
      near (|u - x| <= d): g <= exp(-m^2) / ((x - u)^2 + a^2), m the smallest
        |u| on the interval: a Lorentzian proposal x + a tan(phi), accepted
        with exp(m^2 - u^2).
    The envelope masses pick the part."""
    x = np.asarray(x, dtype=np.float64)
    lo, hi = x - d, x + d
    m = np.where((lo <= 0.0) & (hi >= 0.0), 0.0, np.minimum(np.abs(lo), np.abs(hi)))
    mass_away = np.sqrt(np.pi) * (1.0 - 0.5 * (ss.erf(hi) - ss.erf(lo))) / (d * d + a * a)
    mass_near = np.exp(-m * m) * 2.0 / a * np.arctan(d / a)
    p_away = mass_away / (mass_away + mass_near)
    u = np.empty_like(x)
    todo = np.arange(x.size)
    while todo.size:
        xs, ms, pa = x[todo], m[todo], p_away[todo]
        away = rng.random(todo.size) < pa
        cand = np.empty(todo.size)
        ok = np.zeros(todo.size, dtype=bool)
        # away from the resonance
        na = int(away.sum())
        if na:
            ua = rng.normal(0.0, np.sqrt(0.5), na)
            xa = xs[away]
            inside = np.abs(ua - xa) <= d
            acc = (~inside) & (rng.random(na) < (d * d + a * a) / ((xa - ua) ** 2 + a * a))
            cand[away] = ua
            ok[away] = acc
        # near the resonance
        nn = todo.size - na
        if nn:
            phi = (2.0 * rng.random(nn) - 1.0) * np.arctan(d / a)
            un = xs[~away] + a * np.tan(phi)
            acc = rng.random(nn) < np.exp(ms[~away] ** 2 - un * un)
            cand[~away] = un
            ok[~away] = acc
        u[todo[ok]] = cand[ok]
        todo = todo[~ok]
    return u


def _isotropic(rng, n):
    mu = 2.0 * rng.random(n) - 1.0
    ph = 2.0 * np.pi * rng.random(n)
    s = np.sqrt(1.0 - mu * mu)
    return np.stack([s * np.cos(ph), s * np.sin(ph), mu], axis=1)


def _perp_basis(nv):
    """Two unit vectors orthogonal to each row of nv and to each other."""
    t = np.where(np.abs(nv[:, :1]) < 0.9, np.array([[1.0, 0.0, 0.0]]), np.array([[0.0, 1.0, 0.0]]))
    e1 = np.cross(nv, t)
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(nv, e1)
    return e1, e2


def independent_mcrt(w, n, seed):
    """Escape histogram (J + 2 bins), scatterings per photon and crossings of
    the cell faces per photon (the escape included) of the uniform static slab
    w, by straightforward MCRT (the slab normal is the z component of the
    direction).  Photons start uniformly in the source cells (the centre cell,
    or the two that meet at the midplane)."""
    rng = np.random.default_rng(seed)
    a = C.damping(w.T)
    k0 = w.tau0 / w.R
    edges = w.edges()
    src = [j for j in range(w.J) if edges[j] < 0.0 < edges[j + 1]]
    if src:
        xlo, xhi = edges[src[0]], edges[src[0] + 1]
    else:  # x0 = 0 on an edge: the two bins that meet there, equally likely
        j = int(np.searchsorted(edges, 0.0))
        xlo, xhi = edges[j - 1], edges[j + 1]
    nz = w.n[0]
    dz = 2.0 * w.R / nz
    half = dz / 2.0 if nz % 2 else dz
    z = half * (2.0 * rng.random(n) - 1.0)
    faces = -w.R + dz * np.arange(1, nz)  # interior faces
    ncross = np.zeros(n, dtype=np.int64)
    nv = _isotropic(rng, n)
    x = xlo + (xhi - xlo) * rng.random(n)
    nscat = np.zeros(n, dtype=np.int64)
    x_esc = np.empty(n)
    alive = np.arange(n)
    while alive.size:
        s = rng.exponential(1.0, alive.size) / (k0 * _voigt(a, x[alive]))
        zn = z[alive] + s * nv[alive, 2]
        out = np.abs(zn) > w.R
        zc = np.clip(zn, -w.R, w.R)
        lo, hi = np.minimum(z[alive], zc), np.maximum(z[alive], zc)
        ncross[alive] += ((faces[None, :] > lo[:, None]) & (faces[None, :] < hi[:, None])).sum(axis=1) + out
        x_esc[alive[out]] = x[alive[out]]
        sc = alive[~out]
        z[sc] = zn[~out]
        # coherent scattering in the frame of an atom of velocity u (units of v_th)
        n_in = nv[sc]
        e1, e2 = _perp_basis(n_in)
        upar = _atom_velocity(rng, a, x[sc])
        u1 = rng.normal(0.0, np.sqrt(0.5), sc.size)
        u2 = rng.normal(0.0, np.sqrt(0.5), sc.size)
        uvec = upar[:, None] * n_in + u1[:, None] * e1 + u2[:, None] * e2
        n_out = _isotropic(rng, sc.size)
        x[sc] = x[sc] - np.einsum("ij,ij->i", uvec, n_in) + np.einsum("ij,ij->i", uvec, n_out)
        nv[sc] = n_out
        nscat[sc] += 1
        alive = sc
    j = np.searchsorted(edges, x_esc, side="right")  # 0 below the grid, J + 1 above
    hist = np.bincount(np.clip(j, 0, w.J + 1), minlength=w.J + 2)
    return hist, nscat, ncross


def _oracle_mcrt(w, n):
    g = C.Grid(w, hybrid=True, tau_ddmc=1e30)  # every state thin: the oracle's MC alone
    t = g.table()
    r = C.walk(g, t, w.seed, 0, n)
    assert r["escaped"] == n and r["aborted"] == 0 and r["steps"] == 0
    return r


def _two_sample(h1, h2, n_min=40):
    h1, h2 = np.asarray(h1, float), np.asarray(h2, float)
    sel = h1 + h2 >= n_min
    z = (h1[sel] - h2[sel]) / np.sqrt(h1[sel] + h2[sel])
    chi2 = float((z * z).sum())
    return float(np.abs(z).max()), float(ss.chdtrc(int(sel.sum()) - 1, chi2))


def test_independent_mcrt_samples_the_atom_velocity_density():
    # the independent sampler against its own target density, so that the
    # comparison below rests on two checked samplers
    rng = np.random.default_rng(7)
    a = C.damping(1.0e4)
    for x in (0.0, 1.2, 2.6, 4.0):
        u = _atom_velocity(rng, a, np.full(200_000, x))
        edges = np.linspace(-3.0, 3.0 + x, 61)
        cnt, _ = np.histogram(u, bins=edges)
        grid = np.linspace(edges[0], edges[-1], 600_001)
        f = np.exp(-grid ** 2) / ((x - grid) ** 2 + a * a)
        cdf = np.concatenate([[0.0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(grid))])
        tot = np.pi / a * _voigt(a, x)  # int f du over the line = pi H(a, x) / a
        cdf_e = np.interp(edges, grid, cdf)
        p = np.diff(cdf_e) / tot
        inside = cnt.sum() / u.size
        assert inside == pytest.approx(p.sum(), abs=5e-3)
        e = u.size * p
        sel = e > 30
        zz = (cnt[sel] - e[sel]) / np.sqrt(e[sel])
        assert np.abs(zz).max() < 5.0, (x, np.abs(zz).max())


def test_oracle_mcrt_matches_an_independent_mcrt():
    w = SLAB
    r = _oracle_mcrt(w, N)
    hist_i, nscat, _ = independent_mcrt(w, N, 0x1DE9)
    zmax, pval = _two_sample(r["hist"], hist_i)
    assert zmax < 5.0 and pval > 1e-3, (zmax, pval)
    # the oracle counts every flight: the scatterings plus the escaping one
    m_o = r["mc_events"] / N - 1.0
    m_i = nscat.mean()
    zs = (m_o - m_i) / np.sqrt(2.0 * nscat.var() / N)
    assert abs(zs) < 4.0, (m_o, m_i)
    # a test with power: photons scatter many times and most leave the source
    # bins' neighbourhood (|x| < 0.6) before escaping
    assert m_i > 20.0 and r["hist"][w.J // 2 - 3: w.J // 2 + 3].sum() < 0.3 * N


def test_oracle_mcrt_crosses_thin_cells_like_an_independent_mcrt():
    # four thin cells: flights cross interior faces into thin neighbours, which
    # the oracle's MC continues (a new flight from the face, memoryless) and
    # counts as events; photons start in the two central cells
    w = SLAB.with_(name="thin_slab_tau10_4x60", n=(4, 1, 1), seed=0x5EED0412)
    r = _oracle_mcrt(w, N)
    hist_i, nscat, ncross = independent_mcrt(w, N, 0x1DEA)
    zmax, pval = _two_sample(r["hist"], hist_i)
    assert zmax < 5.0 and pval > 1e-3, (zmax, pval)
    ev = nscat + ncross
    zs = (r["mc_events"] / N - ev.mean()) / np.sqrt(2.0 * ev.var() / N)
    assert abs(zs) < 4.0, (r["mc_events"] / N, ev.mean())
    assert ncross.mean() > 2.0  # interior crossings happen


def independent_grouped_mcrt(w, probs, kbin, n, seed):
    """Frequency-grouped MCRT (Sec. 5.3) of the uniform static slab w: flights
    with the bin-mean opacity kbin[j] of the photon's bin, every scattering
    draws the new bin from row j of `probs` (eq. R_discrete) and a new
    isotropic direction.  Returns the escape histogram over the bins (J + 2,
    no photon leaves the grid) and the events per photon (scatterings plus
    crossings of interior faces plus the escape)."""
    rng = np.random.default_rng(seed)
    nz = w.n[0]
    dz = 2.0 * w.R / nz
    half = dz / 2.0 if nz % 2 else dz
    faces = -w.R + dz * np.arange(1, nz)
    edges = w.edges()
    j = np.full(n, int(np.searchsorted(edges, 0.0, side="right") - 1))
    z = half * (2.0 * rng.random(n) - 1.0)
    mu = 2.0 * rng.random(n) - 1.0
    events = np.zeros(n, dtype=np.int64)
    j_esc = np.empty(n, dtype=np.int64)
    cum = np.cumsum(probs, axis=1)
    alive = np.arange(n)
    while alive.size:
        s = rng.exponential(1.0, alive.size) / kbin[j[alive]]
        zn = z[alive] + s * mu[alive]
        out = np.abs(zn) > w.R
        zc = np.clip(zn, -w.R, w.R)
        lo, hi = np.minimum(z[alive], zc), np.maximum(z[alive], zc)
        events[alive] += ((faces[None, :] > lo[:, None]) & (faces[None, :] < hi[:, None])).sum(axis=1) + 1
        j_esc[alive[out]] = j[alive[out]]
        sc = alive[~out]
        z[sc] = zn[~out]
        u = rng.random(sc.size)
        j[sc] = np.minimum((u[:, None] >= cum[j[sc]]).sum(axis=1), w.J - 1)
        mu[sc] = 2.0 * rng.random(sc.size) - 1.0
        alive = sc
    return np.bincount(j_esc + 1, minlength=w.J + 2), events


def test_oracle_grouped_mc_matches_an_independent_grouped_mcrt():
    # Sec. 5.3: the bin-mean opacity (here from adaptive quadrature of the exact
    # Voigt profile over each bin) and the rows of eq. R_discrete (pinned by
    # the scattering sampler in their own tests) drive a three-cell thin slab
    import scipy.integrate as si
    from oracle import analytic as A
    w = W.Workload("grouped_slab_tau8_3x9", 1, (3, 1, 1), 9, -6.0, 6.0, 8.0, 1.0e4, N, 0x5EED0413)
    a = C.damping(w.T)
    edges = w.edges()
    thr = A.redistribution_thresholds(A.redistribution_cdf(edges, a, 3))
    g = C.Grid(w, hybrid=True, tau_ddmc=1e30, redist=thr)
    r = _oracle_mcrt(w, N)  # without grouping: a different law
    t = g.table()
    rg = C.walk(g, t, w.seed, 0, N)
    assert rg["escaped"] == N and rg["aborted"] == 0 and rg["steps"] == 0
    kbin = np.array([w.tau0 / w.R * si.quad(lambda x: _voigt(a, x), lo, hi, epsabs=1e-13, limit=200)[0] / (hi - lo)
                     for lo, hi in zip(edges[:-1], edges[1:])])
    c = np.concatenate([np.zeros((w.J, 1)), thr.astype(np.float64) / 2.0 ** 32, np.ones((w.J, 1))], axis=1)
    probs = np.diff(c, axis=1)
    hist_i, ev = independent_grouped_mcrt(w, probs, kbin, N, 0x1DEB)
    zmax, pval = _two_sample(rg["hist"], hist_i)
    assert zmax < 5.0 and pval > 1e-3, (zmax, pval)
    zs = (rg["mc_events"] / N - ev.mean()) / np.sqrt(2.0 * ev.var() / N)
    assert abs(zs) < 4.0, (rg["mc_events"] / N, ev.mean())
    # grouping changes the law: the continuous MC of the same slab differs
    zmax_c, pval_c = _two_sample(r["hist"], hist_i)
    assert pval_c < 1e-3 or ev.mean() > 1.05 * (r["mc_events"] / N) or ev.mean() < 0.95 * (r["mc_events"] / N)
