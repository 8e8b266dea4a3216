"""The cost of a pure DDMC run, as the paper states it (Sec. 4, the slab timing
suite at a tau0 = 1e6, T = 10 K over |z| <= R and |x| <= 2.5 (a tau0)^(1/3)):

* it scales as dz^-2 where spatial diffusion dominates and as dx^-3 where
  frequency diffusion dominates (leakage events stand in for scatterings; the
  frequency cost carries the diffusive dx^2 and a drift factor dx);
* it does not depend on the optical depth, only on the discretisation.

The cost of a run is its number of transitions, whose expectation per packet
the exact absorbing chain of the oracle's table gives without sampling noise
(analytic.chain_solve).  The scalings are asymptotic, so the exponents are
compared where one diffusion clearly dominates (coarse bins for the spatial
one, few cells for the frequency one, bins wider than the core, dx > 2 x_cw)."""
import numpy as np

from oracle import analytic as A
from oracle import coracle as C
from paper_1709_10187_gb300 import workloads as W

T = 10.0


def _mean_transitions(atau, nz, nx):
    a = C.damping(T)
    xm = 2.5 * atau ** (1.0 / 3.0)
    w = W.Workload(f"slab_atau{atau:.0e}_{nz}x{nx}", 1, (nz, 1, 1), nx, -xm, xm, atau / a, T, 1, 1)
    g = C.Grid(w)
    return A.chain_solve(w, g.table())["steps_mean"], w


def _local_slopes(costs, sizes):
    return np.diff(np.log(costs)) / np.diff(np.log(sizes))


def test_spatial_diffusion_cost_scales_as_dz_to_the_minus_two():
    nzs = [41, 81, 161]
    c = [_mean_transitions(1.0e6, nz, 11)[0] for nz in nzs]
    s = _local_slopes(c, [2.0 / nz for nz in nzs])
    assert np.all(s < -1.85) and np.all(s > -2.1), s


def test_frequency_diffusion_cost_scales_as_dx_to_the_minus_three():
    nxs = [21, 31, 41]
    c, ws = zip(*[_mean_transitions(1.0e6, 5, nx) for nx in nxs])
    dx = [w.edges()[1] - w.edges()[0] for w in ws]
    assert min(dx) > 5.0  # wider than the line core (2 x_cw ~ 5 at 10 K)
    s = _local_slopes(c, dx)
    assert np.all(s < -2.85) and np.all(s > -3.2), s


def test_cost_does_not_depend_on_the_optical_depth():
    for nz, nx in ((21, 21), (41, 11)):
        c = np.array([_mean_transitions(at, nz, nx)[0] for at in (1.0e5, 1.0e6, 1.0e7, 1.0e8)])
        assert c.max() / c.min() < 1.1, (nz, nx, c)
