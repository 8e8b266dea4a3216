"""Why the leakage precompute runs in FP64: what an FP32
precompute would lose on the tau0 = 1e7 slab, measured against the FP64 oracle.

* Wing bin means (Sec. 2.2): k_j / k0 = (calH(x+) - calH(x-)) / dx is a
  difference of two numbers near sqrt(pi) whose gap in the far wing
  (~ a dx / (sqrt(pi) x^2) ~ 1.7e-8 at x = 60) is below FP32 resolution.
* Thick cells: the spatial leakage of a near-core state is a tiny share of
  its total rate, so its probability 1 - p(frequency moves) lives in the last
  bits of a cumulative sum; FP32 cumulative thresholds misplace it.  (Shares
  below 2^-32 are beyond any 32-bit threshold; see the quantisation rule.)
"""
import numpy as np

from oracle import coracle as C
from paper_1709_10187_gb300 import workloads as W


def test_fp32_bin_means_lose_the_far_wing():
    w = W.C2
    a = C.damping(w.T)
    e = w.edges()
    H = np.array([C.voigt_Hint(a, x) for x in e])
    dx = np.diff(e)
    k64 = np.diff(H) / dx
    k32 = (np.diff(H.astype(np.float32)).astype(np.float64)) / dx
    ref = np.array([C.bin_mean_H(a, lo, hi) for lo, hi in zip(e[:-1], e[1:])])
    wing = np.abs(0.5 * (e[:-1] + e[1:])) > 40.0
    rel64 = np.abs(k64 - ref) / ref
    rel32 = np.abs(k32 - ref) / ref
    print(f"\nwing bins |x| > 40: FP64 max rel err {rel64[wing].max():.2e}, FP32 median rel err "
          f"{np.median(rel32[wing]):.2f}, max {rel32[wing].max():.2f}")
    # the oracle's own bin mean uses the same closed form: FP64 differences agree closely
    assert rel64[wing].max() < 1e-6
    assert np.median(rel32[wing]) > 0.3


def test_fp32_thresholds_misplace_thick_cell_spatial_leakage():
    w = W.C2
    t = C.Grid(w).table()
    rate = t["rate"]                     # [states x 4]: bin-1, bin+1, -z, +z
    thr64 = t["thr"].astype(np.int64)    # [states x 3]
    r32 = rate.astype(np.float32)
    c32 = np.cumsum(r32, axis=1, dtype=np.float32) / r32.sum(axis=1, dtype=np.float32)[:, None]
    thr32 = np.minimum(np.rint(c32[:, :3].astype(np.float64) * 2.0 ** 32), 2.0 ** 32 - 1).astype(np.int64)
    ps64 = (2 ** 32 - thr64[:, 1]).astype(np.float64)   # spatial share (counts)
    ps32 = (2 ** 32 - thr32[:, 1]).astype(np.float64)
    share = (rate[:, 2] + rate[:, 3]) / rate.sum(axis=1)
    # states whose spatial share FP64 thresholds resolve with >= 100 counts but
    # which sit in the last 1e-5 of the cumulative sum
    sel = (share > 100 * 2.0 ** -32) & (share < 1e-5)
    rel32 = np.abs(ps32 - ps64)[sel] / ps64[sel]
    rel64 = np.abs(ps64 - share * 2.0 ** 32)[sel] / (share[sel] * 2.0 ** 32)
    print(f"\nstates with spatial share in (2.3e-8, 1e-5): {sel.sum()}; FP64 thresholds: rel err max "
          f"{rel64.max():.2e}; FP32 thresholds: median {np.median(rel32):.2e}, max {rel32.max():.2f}; "
          f"FP32 thresholds differ in {np.mean(np.any(thr32 != thr64, axis=1)):.3f} of all rows")
    assert sel.sum() > 1000
    assert rel64.max() <= 0.01          # FP64: within half a count of at least 100
    assert rel32.max() > 0.1            # FP32: up to tens of per cent off
