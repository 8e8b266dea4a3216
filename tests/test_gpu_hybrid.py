"""GPU parity of the hybrid scheme (Sec. 5.1, Sec. 5.2): the FP32 continuous-MC
part is compared with the FP64 oracle statistically (its trajectories are not
bit-exact by design), its exact reductions bit-exactly."""
import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as ss

torch = pytest.importorskip("torch")

from oracle import analytic as A  # noqa: E402
from oracle import coracle as C  # noqa: E402
from paper_1709_10187_gb300 import build as B  # noqa: E402
from paper_1709_10187_gb300 import rddmc as R  # noqa: E402
from paper_1709_10187_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def test_hybrid_with_every_state_thick_is_the_ddmc_walk_bit_exactly():
    w = W.SMALL
    a = R.Problem(w).run(w.packets, w.seed)
    b = R.Problem(w, mode=R.MODE_HYBRID, tau_ddmc=1e-30).run(w.packets, w.seed)
    for k in ("escaped", "steps", "event_draws", "mc_events", "conversions"):
        assert a[k] == b[k], k
    assert np.array_equal(a["hist"], b["hist"])


@pytest.mark.parametrize("xp,T", [(0.0, 1.0e4), (1.5, 1.0e4), (3.0, 1.0e4), (8.0, 1.0e4), (2.2, 10.0)])
def test_device_scattering_sampler_follows_R_IIA(xp, T):
    w = W.TINY.with_(T=T)
    p = R.Problem(w, mode=R.MODE_HYBRID)
    n = 400_000
    s = p.scatter(xp, 0xD5CA77E + int(10 * xp), n)
    lo, hi = min(-4.0, xp - 6.0), max(4.0, xp + 6.0)
    edges = np.linspace(lo, hi, 41)
    counts, _ = np.histogram(s, bins=edges)
    probs = A.R_IIA_bin_probs(edges, xp, C.damping(T))
    zmax, frac, pval = A.compare_counts_to_probs(counts, probs, n)
    assert zmax < 5.0 and frac <= 0.05 and pval > 1e-3, (zmax, frac, pval)


def test_device_first_flight_escape_fraction_is_exact():
    w = W.Workload("thin_cell", 1, (1, 1, 1), 1, -0.5, 0.5, 0.3, 1.0e4, 1_000_000, 0x5EED0402)
    r = R.Problem(w, mode=R.MODE_HYBRID, tau_ddmc=1e30).run(w.packets, w.seed, max_steps=1)
    a = C.damping(w.T)
    p_esc = lambda x: (0.5 - ss.expn(3, 2 * w.tau0 * A.voigt_faddeeva(a, x))) / (2 * w.tau0 * A.voigt_faddeeva(a, x))
    pe, _ = si.quad(p_esc, -0.5, 0.5, epsabs=1e-12)
    N = w.packets
    assert r["escaped"] + r["aborted"] == N and r["mc_events"] == N
    z = (r["escaped"] - N * pe) / np.sqrt(N * pe * (1 - pe))
    assert abs(z) < 4.0, (r["escaped"] / N, pe)


@pytest.mark.parametrize("w,n", [(W.TINY, 40_000), (W.SMALL, 20_000), (W.SPHERE8, 40_000), (W.SPHERE8_V, 20_000),
                                 (W.C1, 1000)], ids=lambda v: getattr(v, "name", str(v)))
def test_hybrid_spectrum_matches_oracle(w, n):
    og = C.Grid(w, hybrid=True)
    ot = og.table()
    orc = C.walk(og, ot, w.seed + 11, 0, n)
    gpu = R.Problem(w, mode=R.MODE_HYBRID).run(n, w.seed)
    assert gpu["emitted"] == gpu["escaped"] == n and gpu["status"] == R.OK
    zmax, frac = A.compare_two_samples(gpu["hist"], n, orc["hist"], n)
    assert zmax < 5.0 and frac <= 0.05, (zmax, frac)
    if w.ndim == 3:
        zmax, frac = A.compare_two_samples(gpu["sb"], n, orc["sb"], n)
        assert zmax < 5.0 and frac <= 0.05, (zmax, frac)
    # per-packet means of MC events, conversions and DDMC transitions agree
    for k in ("mc_events", "conversions", "steps"):
        g, o = gpu[k] / n, orc[k] / n
        assert abs(g - o) <= 0.1 * max(g, o) + 1.0, (k, g, o)


def test_hybrid_time_slices_equal_one_launch():
    w = W.SMALL
    p = R.Problem(w, mode=R.MODE_HYBRID)
    one = p.run(w.packets, w.seed)
    p.reset()
    n = 0
    while True:
        p.launch(w.packets, w.seed, steps_per_launch=64, resume=1 if n else 0)
        n += 1
        t = p.read()
        if t["escaped"] + t["aborted"] == w.packets:
            break
        assert n < 10_000
    for k in ("escaped", "steps", "event_draws", "mc_events", "conversions"):
        assert t[k] == one[k], k
    assert np.array_equal(t["hist"], one["hist"])
