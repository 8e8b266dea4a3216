"""Pins of the oracle's continuous-MC part of the hybrid scheme (Sec. 5.1,
Sec. 5.2, Appendix A): the redistribution function, the scattering sampler,
the flight geometry, and the reductions of the hybrid walk."""
import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as ss

from oracle import analytic as A
from oracle import coracle as C
from paper_1709_10187_gb300 import workloads as W


@pytest.mark.parametrize("xp", [0.0, 1.5, 3.0, 8.0])
def test_R_IIA_is_a_normalised_density(xp):
    a = C.damping(1.0e4)
    tot, _ = si.quad(lambda x: A.R_IIA(x, xp, a), xp - 12, xp + 12, limit=400, points=[xp])
    assert tot == pytest.approx(1.0, abs=1e-8)


def test_R_IIA_limits_printed_in_the_appendix():
    # core (a -> 0) and wing (|x + x'| -> inf) approximations of Appendix A
    for x, xp in ((0.3, 0.5), (1.7, -0.4), (-1.1, 0.2)):
        assert A.R_IIA(x, xp, 1e-7) == pytest.approx(A.R_IA_core(x, xp), rel=1e-4)
    a = C.damping(1.0e4)
    for x, xp in ((30.5, 30.0), (29.0, 30.0), (61.0, 60.0)):
        assert A.R_IIA(x, xp, a) == pytest.approx(A.R_IIA_wing(x, xp), rel=3e-3)


def test_R_IIA_detailed_balance():
    # H(x') R(x, x') is symmetric in (x, x') for coherent isotropic scattering
    a = C.damping(1.0e4)
    for x, xp in ((0.4, 1.9), (2.5, 3.7), (-0.8, 1.2)):
        lhs = A.voigt_faddeeva(a, xp) * A.R_IIA(x, xp, a)
        rhs = A.voigt_faddeeva(a, x) * A.R_IIA(xp, x, a)
        assert lhs == pytest.approx(rhs, rel=1e-7)


@pytest.mark.parametrize("xp,T", [(0.0, 1.0e4), (1.5, 1.0e4), (3.0, 1.0e4), (8.0, 1.0e4), (2.2, 10.0)])
def test_scattering_sampler_follows_R_IIA(xp, T):
    # u_par by rejection from a three-part envelope, u_perp ~ N(0, 1/2), isotropic
    # new direction, x' = x + u_par (mu - 1) + u_perp sqrt(1 - mu^2) (Sec. 5.2):
    # the outgoing frequency must have density R_II-A(x', x) (Appendix A).
    a = C.damping(T)
    n = 200_000
    s = C.scatter_samples(T, xp, 0x5CA77E2 + int(10 * xp), n)
    lo, hi = min(-4.0, xp - 6.0), max(4.0, xp + 6.0)
    edges = np.linspace(lo, hi, 41)
    counts, _ = np.histogram(s, bins=edges)
    probs = A.R_IIA_bin_probs(edges, xp, a)
    zmax, frac, pval = A.compare_counts_to_probs(counts, probs, n)
    assert zmax < 5.0 and frac <= 0.05 and pval > 1e-3, (zmax, frac, pval)


def test_wing_scattering_drift_and_rms():
    # Sec. 4.2: a wing photon drifts back toward the core by <dx> ~ -1/x with RMS ~ 1
    for x in (8.0, 15.0):
        s = C.scatter_samples(1.0e4, x, 17, 400_000) - x
        assert s.mean() == pytest.approx(-1.0 / x, abs=0.02)
        assert np.sqrt((s * s).mean()) == pytest.approx(1.0, abs=0.05)


def test_first_flight_escape_fraction_is_exact():
    # One-cell, all-thin slab (pure MC) with the event watchdog at one event: a
    # packet escapes iff its first flight leaves the slab.  Position uniform in
    # |z| <= R, mu uniform on (-1,1), x uniform in the source bin: the escape
    # probability is (1/(2 tau)) (1/2 - E_3(2 tau)), tau = k0 R H(a, x).
    w = W.Workload("thin_cell", 1, (1, 1, 1), 1, -0.5, 0.5, 0.3, 1.0e4, 200_000, 0x5EED0401)
    g = C.Grid(w, hybrid=True, tau_ddmc=1e30)
    t = g.table()
    r = C.walk(g, t, w.seed, 0, w.packets, max_steps=1)
    a = C.damping(w.T)
    p_esc = lambda x: (0.5 - ss.expn(3, 2 * w.tau0 * A.voigt_faddeeva(a, x))) / (2 * w.tau0 * A.voigt_faddeeva(a, x))
    pe, _ = si.quad(p_esc, -0.5, 0.5, epsabs=1e-12)
    N = w.packets
    assert r["escaped"] + r["aborted"] == N
    z = (r["escaped"] - N * pe) / np.sqrt(N * pe * (1 - pe))
    assert abs(z) < 4.0, (r["escaped"] / N, pe)
    assert r["mc_events"] == N


def test_hybrid_with_every_state_thick_is_the_ddmc_walk():
    w = W.SMALL
    g0 = C.Grid(w)
    g1 = C.Grid(w, hybrid=True, tau_ddmc=1e-30)
    t0, t1 = g0.table(), g1.table()
    assert np.array_equal(t0["thr"], t1["thr"]) and np.array_equal(t0["flags"], t1["flags"])
    a = C.walk(g0, t0, w.seed, 0, 4000)
    b = C.walk(g1, t1, w.seed, 0, 4000)
    for k in ("escaped", "steps", "mc_events", "conversions"):
        assert a[k] == b[k]
    assert np.array_equal(a["hist"], b["hist"])


@pytest.mark.parametrize("w", [W.C1.with_(packets=800), W.SPHERE8.with_(packets=3000)], ids=lambda w: w.name)
def test_hybrid_walk_conserves_packets_and_is_symmetric(w):
    g = C.Grid(w, hybrid=True)
    t = g.table()
    r = C.walk(g, t, w.seed, 0, w.packets)
    r2 = C.walk(g, t, w.seed, 0, w.packets, nthreads=3)
    assert r["emitted"] == r["escaped"] == w.packets
    assert r["mc_events"] > 0 and r["conversions"] > 0
    for k in ("escaped", "steps", "mc_events", "conversions", "event_draws"):
        assert r[k] == r2[k]
    assert np.array_equal(r["hist"], r2["hist"])
    f = r["faces"][: 2 * w.ndim].astype(float)
    z = (f - w.packets / len(f)) / np.sqrt(w.packets / len(f))
    assert np.all(np.abs(z) < 4.5)


def test_optically_thin_limit_escapes_with_the_source_spectrum():
    # tau0 -> 0: the hybrid oracle's packets leave without scattering, in the
    # source bins (x0 = 0 is the edge between the two central bins, each
    # chosen with probability 1/2)
    w = W.Workload("slab_thin", 1, (16, 1, 1), 32, -8.0, 8.0, 1.0e-3, 1.0e4, 200_000, 0x5EED0811)
    g = C.Grid(w, hybrid=True)
    r = C.walk(g, g.table(), w.seed, 0, w.packets)
    h = r["hist"][1:-1].astype(np.float64)
    assert r["escaped"] == w.packets and r["steps"] == 0
    src = h[w.J // 2 - 1] + h[w.J // 2]
    assert src / h.sum() >= 0.995, src / h.sum()
    z = (h[w.J // 2] - src / 2) / np.sqrt(src / 4)
    assert abs(z) < 4.0, z
