"""Dust absorption on the GPU (Sec. 2.6, the probabilistic method) against the
FP64 oracle: the FP64 device precompute gives the same thresholds (absorption
threshold included) and the integer walk the same tallies, absorbed packets
included; the grey slab's escape fraction follows its closed form at 1e6
packets; the time-dependent walk absorbs in time as the oracle does."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import coracle as C  # noqa: E402
from paper_1709_10187_gb300 import build as B  # noqa: E402
from paper_1709_10187_gb300 import rddmc as R  # noqa: E402
from paper_1709_10187_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

GREY21 = W.Workload("grey_slab_21x1", 1, (21, 1, 1), 1, -5.0, 5.0, 200.0, 1.0e4, 1_000_000, 0x5EED0D01)

CASES = [  # workload, dust_abs, dust_scat, density gradient (probabilistic method)
    (W.TINY, 0.5, 0.0, False),
    (W.SMALL, 0.3, 2.0, True),
    (W.SPHERE8_V, 0.2, 1.0, False),
]


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def _pair(w, da, ds, grad):
    n_rel = np.linspace(0.5, 2.0, w.ncell) if grad else None
    p = R.Problem(w, n_rel=n_rel, dust_abs=da, dust_scat=ds)
    og = C.Grid(w, n_rel=n_rel, dust_abs=da, dust_scat=ds)
    return p, og, og.table()


@pytest.mark.parametrize("w,da,ds,grad", CASES, ids=lambda v: getattr(v, "name", str(v)))
def test_dusty_table_matches_the_oracle(w, da, ds, grad):
    p, og, t = _pair(w, da, ds, grad)
    thr, flags = p.rows()
    assert thr.shape == t["thr"].shape and thr.shape[1] == 2 * w.ndim + 2  # absorption adds one threshold
    m = w.mask()
    sel = np.ones(w.ncell * w.J, bool) if m is None else np.repeat(m.astype(bool), w.J)
    d = thr[sel].astype(np.int64) - t["thr"][sel].astype(np.int64)
    assert np.abs(d).max() <= 1 and (d != 0).mean() <= 1e-3
    assert np.array_equal(flags[sel], t["flags"][sel])
    p.close()


@pytest.mark.parametrize("w,da,ds,grad", CASES, ids=lambda v: getattr(v, "name", str(v)))
def test_dusty_walk_is_bit_exact(w, da, ds, grad):
    n = 20_000
    p, og, t = _pair(w, da, ds, grad)
    thr, _ = p.rows()
    m = w.mask()
    sel = np.ones(w.ncell * w.J, bool) if m is None else np.repeat(m.astype(bool), w.J)
    # the oracle walks the device's own thresholds (they may differ by one count
    # of 2^32 in the last bits of the FP64 evaluation order)
    t = dict(t)
    t["thr"] = np.where(sel[:, None], thr, t["thr"]).astype(np.uint32)
    g = p.run(n, w.seed)
    o = C.walk(og, t, w.seed, 0, n)
    assert g["absorbed"] > 0.02 * n
    for k in ("emitted", "escaped", "absorbed", "aborted", "steps", "event_draws", "clamps"):
        assert g[k] == o[k], (k, g[k], o[k])
    assert g["escaped"] + g["absorbed"] == n
    assert np.array_equal(g["hist"], o["hist"]) and np.array_equal(g["faces"], o["faces"][: 2 * w.ndim])
    p.close()


def test_grey_slab_escape_fraction_at_a_million_packets():
    w = GREY21
    tau_a = 0.5
    p = R.Problem(w, dust_abs=tau_a, dust_scat=5.0)
    t = C.Grid(w, dust_abs=tau_a, dust_scat=5.0).table()
    k = float(t["k"][w.n[0] // 2])
    dz = 2.0 * w.R / w.n[0]
    r, rb, ka = 1.0 / (3.0 * k * dz * dz), 2.0 / (3.0 * dz * (k * dz + 2.0 * 0.7104)), tau_a / w.R
    pm = r / (2.0 * r + ka)
    e1, p1 = rb / (rb + r + ka), r / (rb + r + ka)
    th = np.arccosh(1.0 / (2.0 * pm))
    mm = (w.n[0] - 1) // 2
    f = e1 / (np.cosh(mm * th) - p1 * np.cosh((mm - 1) * th))
    n = w.packets
    g = p.run(n, w.seed)
    z = (g["escaped"] - n * f) / np.sqrt(n * f * (1.0 - f))
    assert abs(z) < 5.0, (g["escaped"], n * f)
    p.close()


def test_dusty_time_walk_tracks_the_oracle():
    w = W.TINY
    te = [0.0, 0.05, 0.15, 0.4]
    n = 20_000
    p = R.Problem(w, dust_abs=10.0)
    g = p.time_run(n, w.seed, te)
    og = C.Grid(w, dust_abs=10.0)
    o = C.walk_time(og, og.table(), w.seed, 0, n, te)
    allow = 8 + int(np.ceil(4e-7 * o["transitions"]))
    assert abs(int(g["tallies"]["absorbed"]) - o["absorbed"]) <= allow
    assert int(g["absorbed"].sum()) == int(g["tallies"]["absorbed"])
    for k in range(len(te) - 1):
        db = int(np.abs(g["bins"][k].astype(np.int64) - o["bins"][k].astype(np.int64)).sum())
        assert db <= 2 * allow, (k, db)
    alive_start = np.concatenate([[n], g["alive"][:-1].astype(np.int64)])
    assert np.array_equal(alive_start - g["esc"].astype(np.int64) - g["absorbed"].astype(np.int64),
                          g["alive"].astype(np.int64))
    p.close()


def test_dust_is_refused_where_the_method_has_no_absorption():
    # the batched walk and the learned proposal assume no absorption
    w = W.TINY
    p = R.Problem(w, dust_abs=0.5)
    with pytest.raises(R.RDDMCError) as ei:
        R.Batch([p], [100])
    assert ei.value.status == R.ERR_UNSUPPORTED
    p.close()


@pytest.mark.parametrize("w,tau_a", [(W.TINY, 0.5), (W.SMALL, 0.3), (W.SMALL, 20.0), (W.SPHERE8_V, 0.5)],
                         ids=["tiny", "small", "small_strong", "sphere_moving"])
def test_weight_method_tracks_the_oracle(w, tau_a):
    """The weight method (Sec. 2.6): the device sums -ln of the per-dwell weight
    factors exactly in 2^-40 units and forms each escaped weight once; the
    oracle multiplies FP64 factors.  Integer tallies agree count for count (a
    packet whose weight lands within rounding of the 1e-10 elimination weight
    could differ: none does here), the escaped weight to 1e-6."""
    n = 20_000
    p = R.Problem(w, dust_abs=tau_a, dust_scat=1.0, dust_weights=True)
    og = C.Grid(w, dust_abs=tau_a, dust_scat=1.0, dust_weights=True)
    t = og.table()
    thr, _ = p.rows()
    m = w.mask()
    sel = np.ones(w.ncell * w.J, bool) if m is None else np.repeat(m.astype(bool), w.J)
    t = dict(t)
    t["thr"] = np.where(sel[:, None], thr, t["thr"]).astype(np.uint32)
    g = p.run(n, w.seed)
    o = C.walk_weights(og, t, w.seed, 0, n)
    for k in ("emitted", "escaped", "absorbed", "steps", "event_draws"):
        assert g[k] == o[k], (k, g[k], o[k])
    assert np.array_equal(g["hist"], o["hist"])
    assert abs(g["escaped_weight"] - o["escaped_weight"]) <= 1e-6 * o["escaped_weight"]
    assert np.abs(g["weight_hist"] - o["weight_hist"]).max() <= 1e-6 * o["escaped_weight"]
    if tau_a > 1.0:
        assert g["absorbed"] > 0
    p.close()


def test_weight_method_and_probabilistic_method_agree_in_expectation():
    w = W.SMALL
    n = 200_000
    pw = R.Problem(w, dust_abs=0.3, dust_scat=1.0, dust_weights=True)
    pp = R.Problem(w, dust_abs=0.3, dust_scat=1.0)
    a = pw.run(n, w.seed)
    b = pp.run(n, w.seed + 1)
    f = b["escaped"] / n
    assert abs(a["escaped_weight"] / n - f) <= 5.0 * np.sqrt(f * (1 - f) / n), (a["escaped_weight"] / n, f)
    pw.close()
    pp.close()


def test_weight_method_does_not_depend_on_slicing():
    """The log-weight is saved with the packet state between slices: sliced
    launches give the same integer tallies and escaped weight bit for bit."""
    w = W.SMALL
    n = 20_000
    p = R.Problem(w, dust_abs=20.0, dust_scat=1.0, dust_weights=True)
    a = p.run(n, w.seed)
    p.reset()
    p.launch(n, w.seed, steps_per_launch=256)
    for _ in range(100_000):
        r = p.read()
        if r["escaped"] + r["absorbed"] + r["aborted"] == n:
            break
        p.launch(n, w.seed, steps_per_launch=256, resume=1)
    for k in ("escaped", "absorbed", "steps", "event_draws"):
        assert r[k] == a[k], k
    assert r["escaped_weight"] == a["escaped_weight"] and np.array_equal(r["weight_hist"], a["weight_hist"])
    p.close()


def test_weighted_time_estimates_track_the_oracle():
    """Dust by weights in the time-dependent walk: the device attenuates each
    path l by exp(-k_a l) in FP32 and sums weighted estimates in FP64; the
    oracle in FP64.  Same state sequences, so the weighted bin and path
    estimates agree to the FP32 rounding and the clock's step-end flips."""
    w = W.TINY
    te = [0.0, 0.05, 0.15, 0.4]
    n = 20_000
    n_rel = np.linspace(0.5, 2.0, w.ncell)
    p = R.Problem(w, n_rel=n_rel, dust_abs=10.0, dust_weights=True)
    g = p.time_run(n, w.seed, te)
    og = C.Grid(w, n_rel=n_rel, dust_abs=10.0, dust_weights=True)
    o = C.walk_time(og, og.table(), w.seed, 0, n, te)
    for k in range(len(te) - 1):
        rb = float(np.abs(g["wbins"][k] - o["wbins"][k]).sum() / o["wbins"][k].sum())
        rp = float(np.abs(g["wpath"][k] - o["wpath"][k]).sum() / o["wpath"][k].sum())
        assert rb <= 2e-3 and rp <= 2e-3, (k, rb, rp)
    assert abs(int(g["tallies"]["absorbed"]) - int(o["absorbed"])) <= 8
    # the leak tally does not combine with weights
    with pytest.raises(R.RDDMCError) as ei:
        p.time_run(100, w.seed, te, leaks=True)
    assert ei.value.status == R.ERR_UNSUPPORTED
    p.close()
