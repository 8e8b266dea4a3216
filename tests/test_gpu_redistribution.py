"""Frequency-grouped MC on the GPU (Sec. 5.3, eq. R_discrete): the FP64 device
thresholds of the bin-averaged redistribution against the oracle's adaptive
quadrature; the grouped MC's first flight against its closed form; the grouped
hybrid walk against the oracle's grouped hybrid walk (statistically: the MC
runs in FP32 on the device)."""
import numpy as np
import pytest
import scipy.special as ss

torch = pytest.importorskip("torch")

from oracle import analytic as A  # noqa: E402
from oracle import coracle as C  # noqa: E402
from paper_1709_10187_gb300 import build as B  # noqa: E402
from paper_1709_10187_gb300 import rddmc as R  # noqa: E402
from paper_1709_10187_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

GRID9 = W.Workload("redist_9bins", 1, (3, 1, 1), 9, -6.0, 6.0, 100.0, 1.0e4, 1000, 0x5EED0E01)


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def _device_thresholds(p, n_sub=3):
    buf = p.redistribution(n_sub)
    torch.cuda.synchronize()
    J = p.J
    return buf.cpu().numpy().view(np.uint32)[: J * (J - 1)].reshape(J, J - 1)


def test_device_redistribution_matches_the_oracle_quadrature():
    w = GRID9
    p = R.Problem(w, mode=R.MODE_HYBRID)
    thr = _device_thresholds(p)
    cdf = A.redistribution_cdf(w.edges(), C.damping(w.T), 3)
    d = np.abs(thr.astype(np.float64) / 2.0 ** 32 - cdf)
    print(f"\nmax |device - oracle| = {d.max():.2e} of probability")
    assert d.max() <= 2e-6, d.max()
    J = w.J
    # the x -> -x mirror of R holds on the device too
    for jp in range(J):
        assert np.abs(thr[J - 1 - jp].astype(np.int64) - (2 ** 32 - thr[jp][::-1].astype(np.int64))).max() <= 2e-6 * 2 ** 32
    p.close()


def test_device_grouped_first_flight_uses_the_bin_mean_opacity():
    # one thin cell, two bins split at the source frequency (R4: the source
    # takes either bin): escape on the first flight with tau = k_j R
    w = W.Workload("thin_cell_2b", 1, (1, 1, 1), 2, -0.5, 0.5, 0.3, 1.0e4, 1_000_000, 0x5EED0403)
    p = R.Problem(w, mode=R.MODE_HYBRID, tau_ddmc=1e30)
    red = p.redistribution()
    r = p.run(w.packets, w.seed, max_steps=1, redist=red)
    t = C.Grid(w, hybrid=True, tau_ddmc=1e30).table()
    pe = np.mean([(0.5 - ss.expn(3, 2.0 * k * w.R)) / (2.0 * k * w.R) for k in t["k"][:2]])
    n = w.packets
    assert r["escaped"] + r["aborted"] == n and r["mc_events"] == n
    z = (r["escaped"] - n * pe) / np.sqrt(n * pe * (1 - pe))
    assert abs(z) < 4.0, (r["escaped"] / n, pe)
    p.close()


@pytest.mark.parametrize("w,n", [(W.TINY, 40_000), (W.SPHERE8_V, 20_000)], ids=lambda v: getattr(v, "name", str(v)))
def test_grouped_hybrid_walk_follows_the_oracle(w, n):
    p = R.Problem(w, mode=R.MODE_HYBRID)
    red = p.redistribution()
    thr = _device_thresholds(p)
    g = p.run(n, w.seed, redist=red)
    c = p.run(n, w.seed)
    og = C.Grid(w, hybrid=True, redist=thr)
    o = C.walk(og, og.table(), w.seed + 1, 0, n)
    assert g["aborted"] == 0 and o["aborted"] == 0
    assert g["escaped"] == n and o["escaped"] == n
    assert g["conversions"] > 0 and g["mc_events"] > 0
    zmax, frac = A.compare_two_samples(g["hist"], n, o["hist"], n)
    assert zmax < 5.0 and frac <= 0.05, (zmax, frac)
    # MC events and hand-offs per packet agree in mean
    for k in ("mc_events", "conversions"):
        assert abs(g[k] / o[k] - 1.0) <= 0.05, (k, g[k], o[k])
    # the option acts: the continuous MC takes other draws
    assert g["event_draws"] != c["event_draws"]
    p.close()
