"""Pins of the oracle's random stream and DDMC walk (Sec. 2.3): Philox
known-answer vectors, the exact absorbing chain, the literal competing
exponentials, conservation and the step watchdog."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import analytic as A
from oracle import coracle as C
from paper_1709_10187_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    assert list(C.philox(ctr, key)) == out


def test_chain_solver_gamblers_ruin():
    # Pin of the linear algebra itself: a symmetric walk on 1..n-1 absorbed at 0 and n
    # has E[T | start k] = k (n - k).
    n = 23
    S = n - 1
    P = sp.lil_matrix((S, S))
    for i in range(S):
        if i > 0:
            P[i, i - 1] = 0.5
        if i < S - 1:
            P[i, i + 1] = 0.5
    lu = sp.linalg.splu((sp.identity(S) - P.tocsr()).tocsc())
    t = lu.solve(np.ones(S))
    k = np.arange(1, n)
    assert np.allclose(t, k * (n - k), rtol=1e-12)


@pytest.mark.parametrize("w", [W.TINY, W.SMALL, W.GREY_LIKE])
def test_walk_matches_exact_chain(w):
    g = C.Grid(w)
    t = g.table()
    ch = A.chain_solve(w, t)
    assert ch["escape_total"] == pytest.approx(1.0, abs=1e-9)
    r = C.walk(g, t, w.seed, 0, w.packets)
    N = w.packets
    assert r["emitted"] == N and r["escaped"] == N and r["aborted"] == 0
    zmax, frac, pval = A.compare_counts_to_probs(r["hist"], ch["hist"], N)
    assert zmax < 5.0 and frac <= 0.02 and pval > 1e-3, (zmax, frac, pval)
    fz = (r["faces"][:2] - N * ch["faces"][:2]) / np.sqrt(N * ch["faces"][:2] * (1 - ch["faces"][:2]))
    assert np.all(np.abs(fz) < 4.0)
    zs = (r["steps"] / N - ch["steps_mean"]) / np.sqrt(ch["steps_var"] / N)
    assert abs(zs) < 4.0, zs
    # symmetric slab: the exact spectrum is mirror symmetric in x up to the 32-bit
    # quantisation of the thresholds (which is not mirror symmetric)
    h = ch["hist"][1:-1]
    assert np.abs(h - h[::-1]).sum() < 1e-6
    assert ch["faces"][0] == pytest.approx(0.5, abs=1e-7)


@pytest.mark.parametrize("w", [W.SPHERE8, W.SPHERE9_V], ids=lambda w: w.name)
def test_3d_walk_matches_exact_chain(w):
    # three axes, the class of every entered cell, the vacuum around a sphere
    # and (moving) Doppler rebins across faces: the exact chain's escapes per
    # face and mean transitions; for static cells also the spectrum
    g = C.Grid(w)
    t = g.table()
    ch = A.chain_solve(w, t)
    assert ch["escape_total"] == pytest.approx(1.0, abs=1e-9)
    r = C.walk(g, t, w.seed, 0, w.packets)
    N = w.packets
    assert r["emitted"] == N and r["escaped"] == N and r["aborted"] == 0
    pf = ch["faces"][:6]
    fz = (r["faces"][:6] - N * pf) / np.sqrt(N * pf * (1 - pf))
    assert np.all(np.abs(fz) < 4.0), fz
    assert np.allclose(pf, 1.0 / 6.0, atol=2e-3)  # a centred sphere: every face direction alike
    zs = (r["steps"] / N - ch["steps_mean"]) / np.sqrt(ch["steps_var"] / N)
    assert abs(zs) < 4.0, zs
    if w.vmax_kms == 0.0:
        zmax, frac, pval = A.compare_counts_to_probs(r["hist"], ch["hist"], N)
        assert zmax < 5.0 and frac <= 0.02 and pval > 1e-3, (zmax, frac, pval)
    else:
        _rebins_match_chain(w, g, t, ch)


def _rebins_match_chain(w, g, t, ch, batches=10):
    # Faces and transitions are blind to the frequency (the sphere is symmetric
    # under x -> -x); the rebins are not.  From the chain's expected visits v_s:
    # rebins per packet sum_s v_s sum_{rebin faces f} p_sf, and clamped rebins
    # per packet, where j + m_f + B leaves [0, J-1] with B = 1 at probability
    # 1 - thr_f / 2^32 (eq. velocity-shift, reading R6).  Observed: the event
    # draws less the source draw and the five of each 3D escape, and the clamp
    # count; batch means over independent packet ranges for the error.
    J, nf = w.J, 6
    q = A.quantised_probs(t["thr"])
    v = ch["visits"]
    reb = np.zeros(q.shape[0])
    clamp = np.zeros(q.shape[0])
    for f in range(nf):
        o = 2 + f
        is_reb = ((t["flags"].astype(np.int64) >> (2 * o)) & 3) == A.ACT_REBIN
        s = np.nonzero(is_reb & (q[:, o] > 0))[0]
        c, j = np.divmod(s, J)
        m = t["rebin_m"][c * nf + f].astype(np.int64)
        p1 = 1.0 - t["rebin_thr"][c * nf + f].astype(np.float64) / 2.0 ** 32
        out0 = ((j + m) < 0) | ((j + m) > J - 1)
        out1 = ((j + m + 1) < 0) | ((j + m + 1) > J - 1)
        reb[s] += q[s, o]
        clamp[s] += q[s, o] * ((1.0 - p1) * out0 + p1 * out1)
    e_reb, e_clamp = float(v @ reb), float(v @ clamp)
    nb = w.packets // batches
    obs_reb, obs_clamp = [], []
    for b in range(batches):
        rb = C.walk(g, t, w.seed, b * nb, nb)
        obs_reb.append((rb["event_draws"] - 6 * nb) / nb)
        obs_clamp.append(rb["clamps"] / nb)
    for name, o, e in (("rebins", obs_reb, e_reb), ("clamps", obs_clamp, e_clamp)):
        o = np.asarray(o)
        z = (o.mean() - e) / (o.std(ddof=1) / np.sqrt(batches))
        assert abs(z) < 4.0, (name, o.mean(), e, z)
    assert e_reb > 100.0 and e_clamp > 10.0  # both are common enough to be tested


def test_competing_exponentials_match_categorical_form():
    # eq. l_min_1/2 executed literally in FP64 (one exponential per process) must
    # agree in distribution with the categorical draw on quantised probabilities.
    w = W.SMALL
    g = C.Grid(w)
    t = g.table()
    ch = A.chain_solve(w, t)
    r = C.walk(g, t, w.seed + 1, 0, w.packets, literal=True)
    zmax, frac, pval = A.compare_counts_to_probs(r["hist"], ch["hist"], w.packets)
    assert zmax < 5.0 and frac <= 0.02 and pval > 1e-3, (zmax, frac, pval)
    zs = (r["steps"] / w.packets - ch["steps_mean"]) / np.sqrt(ch["steps_var"] / w.packets)
    assert abs(zs) < 4.0
    assert r["event_draws"] == w.packets   # the source draw; transitions use their own stream


def test_tallies_independent_of_thread_count_and_split():
    w = W.TINY
    g = C.Grid(w)
    t = g.table()
    a = C.walk(g, t, w.seed, 0, 4000, nthreads=1)
    b = C.walk(g, t, w.seed, 0, 4000, nthreads=7)
    c1 = C.walk(g, t, w.seed, 0, 1500, nthreads=3)
    c2 = C.walk(g, t, w.seed, 1500, 2500, nthreads=2)
    for k in ("escaped", "steps", "event_draws"):
        assert a[k] == b[k] == c1[k] + c2[k]
    assert np.array_equal(a["hist"], b["hist"]) and np.array_equal(a["hist"], c1["hist"] + c2["hist"])
    # conservation: every emitted packet escapes or is aborted; a static medium
    # takes one event draw per packet (the source)
    assert a["emitted"] == a["escaped"] + a["aborted"] == 4000
    assert a["event_draws"] == a["emitted"]


def test_step_watchdog_matches_chain_survival():
    # A packet is aborted when it would take transition max_steps+1, i.e. iff its
    # absorption time exceeds max_steps.  The chain gives P(T > m) = s P^m 1.
    w = W.SMALL
    g = C.Grid(w)
    t = g.table()
    m = 2000
    r = C.walk(g, t, w.seed, 0, w.packets, max_steps=m)
    assert r["emitted"] == r["escaped"] + r["aborted"]
    # survival from the chain
    q = A.quantised_probs(t["thr"])
    S, J = q.shape[0], w.J
    rows, cols, vals = [], [], []
    for s in range(S):
        c, j = divmod(s, J)
        for o in range(4):
            if q[s, o] == 0 or ((int(t["flags"][s]) >> (2 * o)) & 3) == A.ACT_ESCAPE:
                continue
            d = {0: -1, 1: 1, 2: -J, 3: J}[o]
            rows.append(s); cols.append(s + d); vals.append(q[s, o])
    P = sp.csr_matrix((vals, (rows, cols)), shape=(S, S))
    ss, sp_ = A.source_states(w)
    x = np.zeros(S)
    x[ss] = sp_
    for _ in range(m):
        x = P.T @ x
    p_alive = x.sum()
    N = w.packets
    z = (r["aborted"] - N * p_alive) / np.sqrt(N * p_alive * (1 - p_alive))
    assert abs(z) < 4.0, (r["aborted"], N * p_alive)
    assert r["steps"] <= N * m
