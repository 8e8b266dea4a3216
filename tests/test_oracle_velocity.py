"""Pins of the oracle's moving-medium and 3D escape arithmetic.

Three oracle functions are checked here against results that do not come from
the oracle's own formulas:

* the comoving Doppler shift across a face (eq. velocity-shift, Sec. 2.5) and
  its quantised rebin: a homologous (Hubble-like) flow v = V r / R shifts every
  crossing by the same delta = -f_mu V dz / (R v_th), whatever the face or
  direction, and a uniform translation shifts no crossing at all;
* the observer-frame escape frequency x_obs = x + n.u: for a slab in uniform
  translation the escape histogram is the exact absorbing chain's comoving
  escapes per face, each convolved with the face's outward mu u (mu uniform on
  (0, 1]) and with x uniform in the bin, in closed form;
* the impact parameter b = |r x n| of an escaping ray: for a one-cell cube
  every escape starts uniformly on a face with an isotropic outward direction,
  so its histogram is an integral over face points and directions, evaluated
  here by quasi-Monte Carlo with numpy.
"""
import numpy as np
import pytest

from oracle import analytic as A
from oracle import coracle as C
from paper_1709_10187_gb300 import workloads as W

TWO32 = 4294967296.0
F_MU = 0.5  # the isotropic-flux angle factor of eq. velocity-shift


def _faces(w, t):
    """(cell, axis, side, rebin_m, P(m+1), both cells in the medium) per face."""
    nf = 2 * w.ndim
    mask = w.mask()
    inside = np.ones(w.ncell, dtype=bool) if mask is None else mask.astype(bool)
    out = []
    for c in range(w.ncell):
        idx = [c % w.n[0], (c // w.n[0]) % w.n[1], c // (w.n[0] * w.n[1])]
        for ax in range(w.ndim):
            for sd, side in enumerate((-1, 1)):
                nidx = list(idx)
                nidx[ax] += side
                ok = 0 <= nidx[ax] < w.n[ax]
                nb = nidx[0] + w.n[0] * (nidx[1] + w.n[1] * nidx[2]) if ok else -1
                both = bool(inside[c]) and ok and bool(inside[nb])
                f = c * nf + 2 * ax + sd
                out.append((c, ax, side, int(t["rebin_m"][f]), 1.0 - float(t["rebin_thr"][f]) / TWO32, both))
    return out


@pytest.mark.parametrize("w", [
    W.SPHERE8_V,
    W.SPHERE9_V,
    W.C3.with_(name="sphere_16c_32b_v200", n=(16, 16, 16), J=32, vmax_kms=200.0),
    W.C3.with_(name="sphere_12c_24b_v20", n=(12, 12, 12), J=24, vmax_kms=20.0),
    # |delta| several bins wide: m = -4
    W.SPHERE8.with_(name="sphere_8c_64b_v200", J=64, vmax_kms=200.0),
])
def test_hubble_flow_shifts_every_crossing_by_the_same_delta(w):
    # v = V r / R: along the axis of a crossing the neighbour moves V dz / R
    # faster in the direction of motion, so the comoving frequency drops by
    # f_mu V dz / (R v_th) on every crossing, outward or inward.
    t = C.Grid(w).table()
    vth = 12.85 * np.sqrt(w.T / 1.0e4)  # km/s (Sec. 2.1)
    dx = (w.x_max - w.x_min) / w.J
    n_in = 0
    for c, ax, side, m, p_up, both in _faces(w, t):
        if not both:  # no crossing into vacuum or out of the grid: no shift
            assert m == 0 and p_up <= 1.0 / TWO32, (c, ax, side, m, p_up)
            continue
        n_in += 1
        dz = 2.0 * w.R / w.n[ax]
        q = -F_MU * w.vmax_kms * dz / (w.R * vth) / dx
        assert m == int(np.floor(q)), (c, ax, side, m, q)
        # a uniform x in the bin lands in bin j + m + 1 with probability frac(q)
        assert abs(p_up - (q - np.floor(q))) <= 1.0 / TWO32, (c, ax, side, p_up, q)
    assert n_in > 0


def test_uniform_translation_shifts_no_crossing():
    # the same velocity in every cell: no relative motion across any face, so
    # the leakage rows are those of the static medium and nothing is rebinned
    w = W.SPHERE8.with_(name="cube_5c_16b", n=(5, 5, 5), sphere=False)
    gs = C.Grid(w)
    gm = C.Grid(w)
    gm.v = np.ascontiguousarray(np.tile([30.0, -20.0, 10.0], (w.ncell, 1)), dtype=np.float64)
    gm.g.v = C._ptr(gm.v)
    ts, tm = gs.table(), gm.table()
    assert np.array_equal(ts["thr"], tm["thr"])
    assert np.array_equal(ts["flags"] | np.uint32(A.FLAG_MOVING), tm["flags"])
    assert np.all(tm["rebin_m"] == 0)
    for o in range(2, 8):  # no spatial outcome is a rebin
        assert np.all(((tm["flags"] >> np.uint32(2 * o)) & np.uint32(3)) != A.ACT_REBIN)


def _sum_uniform_cdf(y, a, h, c):
    """P(X + Y <= y) for independent X ~ U(a, a + h), Y ~ U(0, c)."""
    r = lambda z: 0.5 * np.maximum(z, 0.0) ** 2
    return (r(y - a) - r(y - a - h) - r(y - a - c) + r(y - a - h - c)) / (h * c)


def _observer_bin_probs(edges, j, s_u):
    """Histogram (J + 2 bins, under/overflow at the ends) of x + s_u mu with x
    uniform in bin j and mu uniform on (0, 1]."""
    a, h = edges[j], edges[j + 1] - edges[j]
    if s_u < 0.0:  # x - |u| mu = -((-x) + |u| mu)
        lo, hi = -edges[j + 1], -edges[j]
        F = lambda y: 1.0 - _sum_uniform_cdf(-y, lo, hi - lo, -s_u)
    else:
        F = lambda y: _sum_uniform_cdf(y, a, h, s_u)
    cdf = np.array([F(e) for e in edges])
    p = np.empty(len(edges) + 1)
    p[0] = cdf[0]
    p[1:-1] = np.diff(cdf)
    p[-1] = 1.0 - cdf[-1]
    return p


def _moving_slab(u_kms, n_rel):
    w = W.Workload("slab_moving_7x21", 1, (7, 1, 1), 21, -10.5, 10.5, 200.0, 1.0e4, 40_000, 0x5EED0701)
    gs = C.Grid(w, n_rel=n_rel)
    gm = C.Grid(w, n_rel=n_rel)
    gm.v = np.ascontiguousarray(np.tile([u_kms, 0.0, 0.0], (w.ncell, 1)), dtype=np.float64)
    gm.g.v = C._ptr(gm.v)
    return w, gs, gm


def test_observer_frame_escape_of_a_translating_slab():
    # A slab whose density rises from one face to the other, moving as a whole
    # at u = 1.5 v_th along its axis.  The walk inside is the static one (no
    # relative motion); each escape then leaves with mu uniform on (0, 1]
    # through its face and is seen at x + (+-mu) u.  The denser side lets fewer
    # packets out, so the two faces' shifts do not cancel in the histogram.
    vth = 12.85
    u = 1.5
    n_rel = np.linspace(0.4, 2.0, 7)
    w, gs, gm = _moving_slab(u * vth, n_rel)
    ts, tm = gs.table(), gm.table()
    assert np.array_equal(ts["thr"], tm["thr"])
    ch = A.chain_solve(w, ts)
    assert ch["escape_total"] == pytest.approx(1.0, abs=1e-9)
    assert abs(ch["faces"][0] - ch["faces"][1]) > 0.2  # the faces differ enough to see a sign error
    edges = w.edges()
    J = w.J
    expect = np.zeros(J + 2)
    for o, s_u in ((2, -u), (3, u)):  # face -z: n_z = -mu; face +z: n_z = +mu
        per_bin = ch["esc_so"][:, o].reshape(w.ncell, J).sum(axis=0)
        for j in range(J):
            if per_bin[j] > 0.0:
                expect += per_bin[j] * _observer_bin_probs(edges, j, s_u)
    assert expect.sum() == pytest.approx(1.0, abs=1e-9)
    N = w.packets
    r = C.walk(gm, tm, w.seed, 0, N)
    assert r["escaped"] == N and r["aborted"] == 0
    # five event draws per escape from a moving cell (face point x2, mu, phi, x)
    assert r["event_draws"] == N * 6
    zmax, frac, pval = A.compare_counts_to_probs(r["hist"], expect, N)
    assert zmax < 5.0 and frac <= 0.02 and pval > 1e-3, (zmax, frac, pval)
    # the comoving spectrum (static twin, same stream up to the escape) differs
    # from the observer one: the shift is really applied
    rs = C.walk(gs, ts, w.seed, 0, N)
    assert np.array_equal(rs["faces"], r["faces"])
    xc = np.concatenate([[edges[0] - 1.0], 0.5 * (edges[1:] + edges[:-1]), [edges[-1] + 1.0]])
    m_obs = float((r["hist"] * xc).sum()) / N
    m_com = float((rs["hist"] * xc).sum()) / N
    m_exp = float((ch["faces"][1] - ch["faces"][0]) * 0.5 * u)  # E[x_obs - x] = (P+ - P-) u E[mu]
    assert abs((m_obs - m_com) - m_exp) < 0.03, (m_obs - m_com, m_exp)


def _impact_parameter_probs(n_pts=1 << 21, seed=20170930):
    """Histogram of b/R = |r x n| / R over the ORC 64 bins in [0, 1.28) (the
    last bin takes everything above) for r uniform on the face x = R of the
    cube [-R, R]^3 and n isotropic outward (mu = n_x uniform on (0, 1], azimuth
    uniform): scrambled Sobol points over (y, z, mu, phi)."""
    from scipy.stats import qmc
    pts = qmc.Sobol(d=4, scramble=True, seed=seed).random(n_pts)
    y, z = 2.0 * pts[:, 0] - 1.0, 2.0 * pts[:, 1] - 1.0
    mu = 1.0 - pts[:, 2]
    ph = 2.0 * np.pi * pts[:, 3]
    st = np.sqrt(1.0 - mu * mu)
    n = np.stack([mu, st * np.cos(ph), st * np.sin(ph)], axis=1)
    r = np.stack([np.ones_like(y), y, z], axis=1)
    b = np.linalg.norm(np.cross(r, n), axis=1)
    k = np.minimum((b / 1.28 * 64).astype(np.int64), 63)
    return np.bincount(k, minlength=64) / n_pts


def test_impact_parameter_histogram_of_a_one_cell_cube():
    w = W.Workload("cube_1c_8b", 3, (1, 1, 1), 8, -4.0, 4.0, 20.0, 1.0e4, 200_000, 0x5EED0702)
    g = C.Grid(w)
    t = g.table()
    N = w.packets
    r = C.walk(g, t, w.seed, 0, N)
    assert r["escaped"] == N
    assert int(r["sb"].sum()) == N
    p = _impact_parameter_probs()
    zmax, frac, pval = A.compare_counts_to_probs(r["sb"], p, N)
    assert zmax < 5.0 and frac <= 0.02 and pval > 1e-3, (zmax, frac, pval)
    # the six faces of the cube are equally likely
    fz = (r["faces"] - N / 6.0) / np.sqrt(N * (1.0 / 6.0) * (5.0 / 6.0))
    assert np.all(np.abs(fz) < 4.0), r["faces"]
