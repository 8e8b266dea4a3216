"""Each result's error against the FP64 oracle: the FP64
device precompute agrees to one count of 2^32 and the integer walk is exact; the
FP32 continuous MC of the
hybrid scheme differs only statistically, as much as two independent FP64 runs
differ from each other.  Prints the table the design notes quote."""
import numpy as np
import pytest

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


def _l1(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.abs(a / a.sum() - b / b.sum()).sum())


def test_precision_report():
    lines = ["| result | precision | error against the FP64 oracle |", "|---|---|---|"]
    # FP64 device precompute: thresholds within one count of 2^32 (the two sides
    # evaluate the same formulas in different orders), flags equal
    for w in (W.C1, W.GREY_LIKE, W.SPHERE9_V):
        thr, flags = R.Problem(w).rows()
        t = C.Grid(w).table()
        m = w.mask()
        sel = np.ones(w.ncell * w.J, bool) if m is None else np.repeat(m.astype(bool), w.J)
        d = thr[sel].astype(np.int64) - t["thr"][sel].astype(np.int64)
        d_flags = int(np.count_nonzero(flags[sel] != t["flags"][sel]))
        assert np.abs(d).max() <= 1 and (d != 0).mean() <= 1e-4 and d_flags == 0, (w.name, d_flags)
        lines.append(f"| leakage table {w.name} ({d.size} thresholds) | FP64 | {int((d != 0).sum())} thresholds "
                     f"differ, by at most {int(np.abs(d).max())} count of 2^32; 0 differing flags |")
    # integer DDMC walk: tallies equal, count for count
    for w, n in ((W.TINY, 20_000), (W.SPHERE8_V, 20_000)):
        g = R.Problem(w).run(n, w.seed)
        og = C.Grid(w)
        o = C.walk(og, og.table(), w.seed, 0, n)
        diff = int(np.abs(g["hist"].astype(np.int64) - o["hist"].astype(np.int64)).sum())
        diff += sum(abs(int(g[k]) - int(o[k])) for k in ("escaped", "steps", "event_draws", "clamps"))
        assert diff == 0, (w.name, diff)
        lines.append(f"| DDMC walk {w.name}, {n} packets | integer (escape geometry FP64) | 0 differing counts "
                     f"({g['steps']} transitions) |")
    # hybrid: FP32 MC against FP64 MC, beside the spread of two FP64 runs
    for w, n in ((W.TINY, 40_000), (W.SPHERE8_V, 20_000)):
        og = C.Grid(w, hybrid=True)
        ot = og.table()
        o1 = C.walk(og, ot, w.seed + 11, 0, n)
        o2 = C.walk(og, ot, w.seed + 12, 0, n)
        g = R.Problem(w, mode=R.MODE_HYBRID).run(n, w.seed)
        l1_g, l1_o = _l1(g["hist"], o1["hist"]), _l1(o2["hist"], o1["hist"])
        zmax, frac = A.compare_two_samples(g["hist"], n, o1["hist"], n)
        assert zmax < 5.0 and frac <= 0.05, (w.name, zmax, frac)
        assert l1_g <= 2.0 * l1_o + 0.01, (w.name, l1_g, l1_o)
        ev = abs(g["mc_events"] / n - o1["mc_events"] / n) / (o1["mc_events"] / n)
        lines.append(f"| hybrid spectrum {w.name}, {n} packets | FP32 MC, FP64 table | L1 {l1_g:.4f} (two FP64 "
                     f"runs: {l1_o:.4f}); max bin z {zmax:.2f}; MC events/packet rel. diff {ev:.3f} |")
    print("\n" + "\n".join(lines))
