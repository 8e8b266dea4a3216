"""GPU checks of the learned proposal on a medium that varies from cell to cell
(region mode): first passages out of the medium's own regions bit-exact against
the oracle, and a walk with region proposals that conserves packets and does
not depend on how it is sliced.  How close its spectrum comes to the plain
walk's is measured, not asserted: the region proposal is an approximation."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import coracle as C  # noqa: E402
from paper_1709_10187_gb300 import build as B  # noqa: E402
from paper_1709_10187_gb300 import learned as Lr  # noqa: E402
from paper_1709_10187_gb300 import rddmc as R  # noqa: E402
from paper_1709_10187_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

BRICK, MARGIN = 8, 1


@pytest.fixture(scope="module")
def medium():
    B.build()
    # 24^3 cells with a cell-resolution lognormal density and turbulent
    # velocity, 32 bins over [-32, 32], tau0 = 3e4 at the mean density
    return W.clumpy_medium(n=24, J=32, x_max=32.0, tau0=3.0e4, brick=1, sigma_v_kms=20.0, packets=1,
                           seed=0x5EED0720)


def test_region_first_passages_are_bit_exact_against_the_oracle(medium):
    med = medium
    w = med.workload
    prob = R.Problem.clumpy(med)
    prop = Lr.RegionProposal(prob, med.n_rel, med.v_kms, BRICK, MARGIN, tau_lo=3.0, tau_hi=1.0e12)
    assert int(prop.bricks.numel()) == 27  # every brick of the 3^3 lattice is whole
    n = 6000
    d = prop.generate(n, seed=0xA11CE, p0=77)
    thr, flags = prob.rows()
    og = C.Grid(w, n_rel=med.n_rel)
    og.v = np.ascontiguousarray(med.v_kms, dtype=np.float64)
    og.g.v = C._ptr(og.v)
    ot = og.table()
    assert np.abs(thr.astype(np.int64) - ot["thr"].astype(np.int64)).max() <= 1
    assert np.array_equal(flags, ot["flags"])
    out, steps = C.fp_region_samples(og, dict(ot, thr=thr, flags=flags), BRICK, 0, MARGIN, 3,
                                     prop.bricks.cpu().numpy(), prop.bin_off.cpu().numpy(), prop.bins.cpu().numpy(),
                                     0xA11CE, 77, n, 10_000_000)
    rec = d["rec"].cpu().numpy()
    assert np.array_equal(rec, out)
    assert np.array_equal(d["steps"].cpu().numpy().astype(np.uint64), steps)
    assert (out[:, 3] < 6).all() and out[:, 6].sum() > 0  # every sample left its region; some crossings rebinned
    # the targets follow the records
    tA, tC = d["tA"].cpu().numpy(), d["tC"].cpu().numpy()
    assert np.array_equal(tA, out[:, 3] * w.J + out[:, 4])
    assert np.array_equal(tC, out[:, 3] * prop.S + out[:, 5])


def test_walk_with_region_proposals_conserves_packets_and_ignores_slicing(medium):
    med = medium
    prob = R.Problem.clumpy(med)
    prop = Lr.RegionProposal(prob, med.n_rel, med.v_kms, BRICK, MARGIN, tau_lo=3.0, tau_hi=1.0e12)
    data = prop.generate(200_000, seed=5)
    prop.train(data, iters=400, batch=4096, lr=2e-3)
    n = 20_000
    a = prop.run(n_packets=n, seed=0xBEE, time_slice_us=150)
    b = prop.run(n_packets=n, seed=0xBEE, time_slice_us=0, steps_per_launch=1 << 40)
    assert a["escaped"] + a["aborted"] == n and a["aborted"] == 0
    assert a["proposals"] > 0 and a["launches"] > b["launches"]
    for k in ("emitted", "escaped", "aborted", "steps", "clamps", "event_draws", "proposals", "proposed_steps"):
        assert a[k] == b[k], (k, a[k], b[k])
    for k in ("hist", "faces", "sb"):
        assert np.array_equal(a[k], b[k]), k
    pl = prob.run(n, 0xBEE + 1)
    print(f"\nregion proposals: {a['proposals'] / n:.3g} per packet, {a['steps'] / n:.4g} transitions/packet "
          f"against {pl['steps'] / n:.4g} plain")
