"""Pins of the oracle's discrete frequency redistribution (Sec. 5.3, eq.
R_discrete): the bin-averaged R_II-A, kept as cumulative probabilities at the
interior bin edges.

* At fixed incoming x' the edge CDF (adaptive quadrature of R_II-A) matches
  the histogram of the continuous scattering sampler (the atom-velocity
  rejection sampler of Sec. 5.2 / Appendix A, an independent route), outgoing
  frequencies beyond the grid counted in the end bins.
* A row, the average over the incoming bin, matches the sampler fed with the
  same incoming nodes.
* R(x, x') = R(-x, -x'): row j' mirrors row J-1-j'.
"""
import numpy as np
import pytest

from oracle import analytic as A
from oracle import coracle as C

T = 1.0e4
EDGES = np.linspace(-6.0, 6.0, 10)


@pytest.fixture(scope="module")
def cdf():
    a = C.damping(T)
    return A.redistribution_cdf(EDGES, a, 3)


def _clamped_bins(x, edges):
    return np.clip(np.searchsorted(edges, x, side="right") - 1, 0, len(edges) - 2)


@pytest.mark.parametrize("xp", [0.3, 1.7, 3.4, 5.9])
def test_edge_cdf_matches_the_scattering_sampler(xp):
    a = C.damping(T)
    F = A.redistribution_cdf_at(EDGES, xp, a)
    J = len(EDGES) - 1
    probs = np.diff(np.concatenate([[0.0], F[1:J], [1.0]]))
    n = 400_000
    x = C.scatter_samples(T, xp, 0xD15C + int(10 * xp), n)
    counts = np.bincount(_clamped_bins(x, EDGES), minlength=J)
    zmax, frac, pval = A.compare_counts_to_probs(counts, probs, n)
    assert zmax < 5.0 and frac <= 0.02 and pval > 1e-3, (xp, zmax, frac, pval)


def test_rows_average_the_incoming_bin(cdf):
    a = C.damping(T)
    J = len(EDGES) - 1
    gx, gw = np.polynomial.legendre.leggauss(3)
    for jp in (4, 6):
        probs = np.diff(np.concatenate([[0.0], cdf[jp], [1.0]]))
        counts = np.zeros(J)
        n_tot = 0
        for k, (xg, wg) in enumerate(zip(gx, gw)):
            xp = 0.5 * (EDGES[jp + 1] - EDGES[jp]) * xg + 0.5 * (EDGES[jp + 1] + EDGES[jp])
            m = int(round(300_000 * wg / 2.0))
            x = C.scatter_samples(T, xp, 0xD15D + 17 * jp + k, m)
            counts += np.bincount(_clamped_bins(x, EDGES), minlength=J)
            n_tot += m
        zmax, frac, pval = A.compare_counts_to_probs(counts, probs, n_tot)
        assert zmax < 5.0 and frac <= 0.02 and pval > 1e-3, (jp, zmax, frac, pval)
    assert a > 0


def test_rows_are_cumulative_and_mirror_symmetric(cdf):
    J = len(EDGES) - 1
    assert np.all(np.diff(cdf, axis=1) >= -1e-12) and cdf.min() >= 0.0 and cdf.max() <= 1.0 + 1e-12
    for jp in range(J):
        assert np.allclose(cdf[J - 1 - jp], 1.0 - cdf[jp][::-1], atol=1e-7), jp
    thr = A.redistribution_thresholds(cdf)
    assert thr.dtype == np.uint32 and np.all(np.diff(thr.astype(np.int64), axis=1) >= 0)


def test_grouped_first_flight_uses_the_bin_mean_opacity():
    """Frequency-grouped MC (Sec. 5.3) flies with the bin-mean opacity k_j: a
    one-cell, all-thin slab with one event per packet escapes with the exact
    first-flight probability (1/(2 tau)) (1/2 - E_3(2 tau)), tau = k_j R, for
    position uniform in |z| <= R and mu uniform on (-1, 1)."""
    import scipy.special as ss
    from paper_1709_10187_gb300 import workloads as W
    w = W.Workload("thin_cell", 1, (1, 1, 1), 1, -0.5, 0.5, 0.3, 1.0e4, 200_000, 0x5EED0402)
    g = C.Grid(w, hybrid=True, tau_ddmc=1e30, redist=np.zeros((1, 1), dtype=np.uint32))
    t = g.table()
    tau = float(t["k"][0]) * w.R
    pe = (0.5 - ss.expn(3, 2.0 * tau)) / (2.0 * tau)
    r = C.walk(g, t, w.seed, 0, w.packets, max_steps=1)
    n = w.packets
    assert r["escaped"] + r["aborted"] == n and r["mc_events"] == n
    z = (r["escaped"] - n * pe) / np.sqrt(n * pe * (1 - pe))
    assert abs(z) < 4.0, (r["escaped"] / n, pe)
