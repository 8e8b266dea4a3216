"""Pins of the oracle's dust absorption (Sec. 2.6, the probabilistic method).

Grey dust adds a scattering coefficient k_s to every k_ij of the leakage
coefficients and an absorption process of coefficient k_a that competes with
the leakage processes (one more exponential in eq. l_min_1/2, so one more
outcome of the categorical draw, taken last).

* A grey slab (one frequency bin) is a symmetric random walk on n cells with
  killing: interior cells move left or right with probability p = r/(2r+k_a)
  each (r = 1/(3 k dz^2), eq. z-leakage), boundary cells escape with the rate
  r_b = 2/(3 dz (k dz + 2 lambda)).  The escape probability from the centre has
  the closed form f = e_1 / (cosh(m theta) - p_1 cosh((m-1) theta)), cosh theta
  = 1/(2p), m = (n-1)/2, with e_1, p_1 the boundary cell's escape and inward
  probabilities (the two-term solution f_i = A cosh(theta (i - c)) of
  f_i = p (f_{i-1} + f_{i+1}) with the boundary equation).
* With frequency diffusion the walk is pinned to the exact absorbing chain:
  escapes per bin, the absorbed fraction and the mean transition count.
"""
import numpy as np
import pytest

from oracle import analytic as A
from oracle import coracle as C
from paper_1709_10187_gb300 import workloads as W

GREY21 = W.Workload("grey_slab_21x1", 1, (21, 1, 1), 1, -5.0, 5.0, 200.0, 1.0e4, 200_000, 0x5EED0D01)


def _closed_form_escape(w, k, ka, lam=0.7104):
    dz = 2.0 * w.R / w.n[0]
    r = 1.0 / (3.0 * k * dz * dz)
    rb = 2.0 / (3.0 * dz * (k * dz + 2.0 * lam))
    p = r / (2.0 * r + ka)
    e1 = rb / (rb + r + ka)
    p1 = r / (rb + r + ka)
    th = np.arccosh(1.0 / (2.0 * p))
    m = (w.n[0] - 1) // 2
    return e1 / (np.cosh(m * th) - p1 * np.cosh((m - 1) * th))


def test_dust_scattering_adds_to_every_opacity():
    w = W.SMALL
    t0 = C.Grid(w).table()
    n_rel = np.linspace(0.5, 2.0, w.ncell)
    t1 = C.Grid(w, dust_scat=30.0, n_rel=n_rel).table()
    t2 = C.Grid(w, n_rel=n_rel).table()
    ks = np.repeat(30.0 / w.R * n_rel, w.J)
    assert np.allclose(t1["k"] - t2["k"], ks, rtol=1e-12, atol=1e-12)
    assert not np.array_equal(t0["thr"], t1["thr"])
    # no absorption: no extra outcome
    assert t1["thr"].shape == t0["thr"].shape and t1["rate"].shape == t0["rate"].shape


@pytest.mark.parametrize("tau_a", [0.05, 0.5, 3.0])
def test_grey_slab_escape_fraction_has_the_closed_form(tau_a):
    w = GREY21
    g = C.Grid(w, dust_abs=tau_a, dust_scat=5.0)
    t = g.table()
    k = float(t["k"][w.n[0] // 2])
    assert k == pytest.approx(float(C.Grid(w).table()["k"][w.n[0] // 2]) + 5.0 / w.R, rel=1e-12)
    f = _closed_form_escape(w, k, tau_a / w.R)
    ch = A.chain_solve(w, t)
    assert ch["escape_total"] == pytest.approx(f, rel=1e-6, abs=1e-9)
    n = w.packets
    r = C.walk(g, t, w.seed, 0, n)
    assert r["emitted"] == n and r["escaped"] + r["absorbed"] == n and r["aborted"] == 0
    z = (r["escaped"] - n * f) / np.sqrt(n * f * (1.0 - f))
    assert abs(z) < 5.0, (r["escaped"], n * f)
    # mean transitions (absorption is a transition) against the chain
    assert abs(r["steps"] / n - ch["steps_mean"]) <= 5.0 * np.sqrt(ch["steps_var"] / n)


@pytest.mark.parametrize("w,ka", [(W.SMALL.with_(packets=100_000), 0.3), (W.SPHERE8.with_(packets=40_000), 0.5)],
                         ids=["slab", "sphere"])
def test_dusty_walk_follows_the_absorbing_chain(w, ka):
    g = C.Grid(w, dust_abs=ka, dust_scat=2.0)
    t = g.table()
    K = 2 + 2 * w.ndim
    assert t["thr"].shape[1] == K and t["rate"].shape[1] == K + 1
    ch = A.chain_solve(w, t)
    n = w.packets
    r = C.walk(g, t, w.seed, 0, n)
    pa = 1.0 - ch["escape_total"]
    assert 0.05 < pa < 0.95
    za = (r["absorbed"] - n * pa) / np.sqrt(n * pa * (1.0 - pa))
    assert abs(za) < 5.0, (r["absorbed"], n * pa)
    zmax, frac, pval = A.compare_counts_to_probs(r["hist"], ch["hist"], n)
    assert zmax < 5.0 and frac <= 0.02 and pval > 1e-3, (zmax, frac, pval)
    assert abs(r["steps"] / n - ch["steps_mean"]) <= 5.0 * np.sqrt(ch["steps_var"] / n)
    # the literal competing exponentials (absorption one of them) agree in law
    rl = C.walk(g, t, w.seed + 1, 0, n, literal=True)
    zl = (rl["absorbed"] - n * pa) / np.sqrt(n * pa * (1.0 - pa))
    assert abs(zl) < 5.0, (rl["absorbed"], n * pa)


def test_dusty_time_walk_follows_the_chain():
    """With dust the dwell rate K_s includes k_a (absorption competes in time
    as well); occupancies per step against the chain."""
    w = W.TINY
    # k_a = 10 per R, comparable to the wing states' leakage rates (K_s from 9
    # to 1e4), so that the dwell rate's absorption term matters
    g = C.Grid(w, dust_abs=10.0)
    t = g.table()
    te = np.array([0.0, 0.05, 0.15, 0.4])
    n = 40_000
    r = C.walk_time(g, t, w.seed, 0, n, te)
    occ, path, lost = A.chain_time(w, t, te)
    for k in range(len(te) - 1):
        e = occ[k] * n
        sel = e >= 20.0
        z = (r["bins"][k][sel] - e[sel]) / np.sqrt(e[sel] * (1.0 - occ[k][sel]))
        assert np.abs(z).max() < 5.0, (k, np.abs(z).max())
    # absorption happens at rate k_a while in a state: its expected count is the
    # step-integrated occupancy times k_a; the chain's loss per step is escapes
    # plus absorptions
    absorbed_exp = float((path.sum(axis=0) * t["rate"][:, -1]).sum())
    assert abs(r["absorbed"] / n - absorbed_exp) <= 5.0 * np.sqrt(absorbed_exp * (1 - absorbed_exp) / n)
    done = (r["esc"].sum() + r["absorbed"]) / n
    assert abs(done - lost.sum()) <= 5.0 * np.sqrt(lost.sum() * (1 - lost.sum()) / n)


@pytest.mark.parametrize("w,tau_a", [(W.SMALL.with_(packets=40_000), 0.3), (W.SMALL.with_(packets=40_000), 20.0),
                                     (W.SPHERE8.with_(packets=20_000), 0.5)], ids=["slab_0.3", "slab_20", "sphere_0.5"])
def test_weight_method_has_the_probabilistic_escape_in_expectation(w, tau_a):
    """The continuous method of Sec. 2.6: weights multiplied by K_s/(K_s+k_a)
    per transition (the expected exp(-k_a dl) over a dwell) give an escaped
    weight whose expectation, in total and per escape bin, is the escape
    probability of the probabilistic method (the absorbing chain); weights lie
    in [0, 1], so the standard error is at most sqrt(p/n).  At tau_a = 20 many
    packets fall below the 1e-10 elimination weight."""
    n = w.packets
    g = C.Grid(w, dust_abs=tau_a, dust_scat=2.0, dust_weights=True)
    t = g.table()
    assert t["thr"].shape[1] == 1 + 2 * w.ndim  # no absorption outcome in the weight method
    r = C.walk_weights(g, t, w.seed, 0, n)
    ch = A.chain_solve(w, C.Grid(w, dust_abs=tau_a, dust_scat=2.0).table())
    p = ch["escape_total"]
    assert r["escaped"] + r["absorbed"] == n
    assert abs(r["escaped_weight"] / n - p) <= 5.0 * np.sqrt(p / n) + 1e-10, (r["escaped_weight"] / n, p)
    h = ch["hist"]
    sel = h * n >= 20.0
    assert np.all(np.abs(r["weight_hist"][sel] / n - h[sel]) <= 5.0 * np.sqrt(h[sel] / n))
    if tau_a > 1.0:
        assert r["absorbed"] > 0
    # the weight method tallies every escape: at most as noisy as counting the
    # probabilistic walk's escapes
    assert r["escaped"] >= C.walk(C.Grid(w, dust_abs=tau_a, dust_scat=2.0),
                                  C.Grid(w, dust_abs=tau_a, dust_scat=2.0).table(), w.seed, 0, n)["escaped"]


@pytest.mark.parametrize("tau_a", [0.5, 3.0])
def test_weight_method_on_the_grey_slab_has_the_closed_form(tau_a):
    """The mean escaped weight of the grey slab equals the closed-form escape
    probability of the random walk with killing; batch means of 20 packet sets
    give the (small) standard error of the weights."""
    w = GREY21
    g = C.Grid(w, dust_abs=tau_a, dust_scat=5.0, dust_weights=True)
    t = g.table()
    f = _closed_form_escape(w, float(t["k"][w.n[0] // 2]), tau_a / w.R)
    B, m = 20, 10_000
    means = np.array([C.walk_weights(g, t, w.seed, b * m, m)["escaped_weight"] / m for b in range(B)])
    se = means.std(ddof=1) / np.sqrt(B)
    assert abs(means.mean() - f) <= 5.0 * se, (means.mean(), f, se)
    # far tighter than counting the escapes of as many probabilistic packets
    assert se < 0.5 * np.sqrt(f * (1.0 - f) / (B * m)), (se, np.sqrt(f * (1.0 - f) / (B * m)))


def test_weighted_time_estimates_follow_the_absorbing_chain():
    """Dust by packet weights in the time-dependent walk (Sec. 2.6): over a path
    l the weight falls by exp(-k_a l), the path estimate takes the weight
    averaged along the path.  In expectation the weighted bin and path
    estimates are the occupancy and step-integrated occupancy of the chain
    with absorption as a competing process.  A density gradient makes k_a, and
    so the weights, differ between packets; weights lie in [0, 1], so a state's
    weighted count varies at most as its count."""
    w = W.TINY
    te = np.array([0.0, 0.05, 0.15, 0.4])
    n = 60_000
    n_rel = np.linspace(0.5, 2.0, w.ncell)
    g = C.Grid(w, dust_abs=10.0, dust_weights=True, n_rel=n_rel)
    r = C.walk_time(g, g.table(), w.seed, 0, n, te)
    occ, path, _ = A.chain_time(w, C.Grid(w, dust_abs=10.0, n_rel=n_rel).table(), te)
    for k in range(len(te) - 1):
        e = occ[k] * n
        sel = e >= 20.0
        assert np.all(np.abs(r["wbins"][k][sel] - e[sel]) <= 5.0 * np.sqrt(e[sel])), k
        dt = te[k + 1] - te[k]
        ep = path[k] * n
        assert np.all(np.abs(r["wpath"][k] - ep) <= 5.0 * np.sqrt(dt * ep) + 1e-9), k
        # the weights do fall: the weighted estimates lie below the unweighted ones
        assert r["wbins"][k].sum() < r["bins"][k].sum() and r["wpath"][k].sum() < r["path"][k].sum()
