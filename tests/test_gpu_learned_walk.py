"""GPU checks of the walk with the learned exit proposal on a clumpy 3D medium:
results independent of how the walk is sliced, escape spectra that agree bin
by bin with the plain walk within the combined Monte Carlo error, and fewer
DDMC transitions than the plain walk (the gain the trained network brings)."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1709_10187_gb300 import build as B  # noqa: E402
from paper_1709_10187_gb300 import learned as Lr  # noqa: E402
from paper_1709_10187_gb300 import rddmc as R  # noqa: E402
from paper_1709_10187_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

BRICK, MARGIN = 8, 1
SEED = 0x1EA2


@pytest.fixture(scope="module")
def setup():
    B.build()
    # 32^3 cells in 4^3 bricks of lognormal density and turbulent velocity,
    # 64 bins over [-64, 64], tau0 = 1e6 at the mean density
    med = W.clumpy_medium(n=32, J=64, x_max=64.0, tau0=1.0e6, brick=BRICK, packets=1)
    prob = R.Problem.clumpy(med)
    rho = med.brick_rho
    levels = np.logspace(np.log10(rho.min()) - 0.05, np.log10(rho.max()) + 0.05, 12)
    prop = Lr.ExitProposal(med.workload, BRICK - 2 * MARGIN, levels, tau_lo=5.0, tau_hi=1.0e12)
    data = prop.generate(600_000, seed=3, cap=20_000_000)
    prop.train(data, iters=1500, batch=8192, lr=2e-3)
    torch.cuda.synchronize()
    return med, prob, prop


def _run(setup, n, seed, **kw):
    med, prob, prop = setup
    return prop.run(prob, med.brick_rho, n, seed, margin=MARGIN, tau_lo=5.0, tau_hi=1.0e12, **kw)


def test_walk_with_proposal_does_not_depend_on_slicing(setup):
    a = _run(setup, 20_000, SEED, time_slice_us=150)
    b = _run(setup, 20_000, SEED, time_slice_us=0, steps_per_launch=1 << 40)
    assert a["launches"] > b["launches"]
    for k in ("emitted", "escaped", "aborted", "steps", "clamps", "event_draws", "proposals", "proposed_steps"):
        assert a[k] == b[k], (k, a[k], b[k])
    for k in ("hist", "faces", "sb"):
        assert np.array_equal(a[k], b[k]), k


def test_walk_with_proposal_matches_plain_and_saves_transitions(setup):
    med, prob, prop = setup
    n, n_ref = 300_000, 1_200_000
    torch.cuda.synchronize()
    t0 = time.time()
    lr = _run(setup, n, SEED)
    torch.cuda.synchronize()
    t_learned = time.time() - t0
    t0 = time.time()
    pl = prob.run(n, SEED)
    torch.cuda.synchronize()
    t_plain = time.time() - t0
    ref = prob.run(n_ref, SEED + 1)
    assert lr["escaped"] == n and lr["aborted"] == 0 and lr["emitted"] == n
    assert lr["proposals"] > n // 4
    # bin by bin within the combined multinomial error (4 sigma; 64 bins)
    h, r = lr["hist"].astype(np.float64), ref["hist"].astype(np.float64)
    p, q = h / h.sum(), r / r.sum()
    ok = (h >= 20) & (r >= 20)
    z = (p - q)[ok] / np.sqrt(p[ok] * (1 - p[ok]) / h.sum() + q[ok] * (1 - q[ok]) / r.sum())
    assert np.max(np.abs(z)) <= 4.0, np.max(np.abs(z))
    hp = pl["hist"].astype(np.float64)
    l1_learned = float(np.abs(p - q).sum())
    l1_plain = float(np.abs(hp / hp.sum() - q).sum())
    assert l1_learned <= 1.5 * l1_plain + 0.004, (l1_learned, l1_plain)
    # the gain: DDMC transitions the walk still takes, against the plain walk
    ratio = lr["steps"] / pl["steps"]
    print(f"\nlearned: {t_learned:.3f} s, {lr['steps'] / n:.4g} transitions/packet, "
          f"{lr['proposals'] / n:.3g} proposals/packet, L1 {l1_learned:.4f}; "
          f"plain: {t_plain:.3f} s, {pl['steps'] / n:.4g} transitions/packet, L1 {l1_plain:.4f}; "
          f"transition ratio {ratio:.3f}")
    assert ratio <= 0.9, ratio
