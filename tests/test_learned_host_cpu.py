"""Host-side description of a medium for region-mode proposals
(learned.region_summaries): each brick's inner cube summarised by its mean
log density, spread, density slopes and Doppler shifts per crossing, checked on
media whose summaries are known in closed form."""
import numpy as np
import pytest

pytest.importorskip("torch")  # the learned module binds the CUDA library lazily; no GPU is used here

from paper_1709_10187_gb300 import learned as Lr  # noqa: E402
from paper_1709_10187_gb300 import workloads as W  # noqa: E402

N, BRICK, MARGIN = 16, 8, 1
R_IN = BRICK - 2 * MARGIN


def _w(tau0=1.0e6, T=1.0e4):
    return W.Workload("cube_16", 3, (N, N, N), 8, -8.0, 8.0, tau0, T, 1, 1)


def _coords():
    c = (np.arange(N) + 0.5) * (2.0 / N) - 1.0
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return x.ravel(), y.ravel(), z.ravel()


def test_uniform_medium_has_flat_summaries():
    w = _w()
    s, full = Lr.region_summaries(w, np.full(w.ncell, 2.0), None, BRICK, MARGIN)
    assert full.all() and s.shape == (8, 8)
    dz = 2.0 * w.R / N
    assert np.allclose(s[:, 0], np.log10(w.tau0 / w.R * dz) + np.log10(2.0), atol=1e-6)
    assert np.allclose(s[:, 1:], 0.0, atol=1e-6)


def test_exponential_density_gives_its_slope():
    # log10 n = g x: across a region of r cells the positions (2l+1)/r - 1 span
    # 2 (r - 1)/r, i.e. (r - 1) dz in x; the slope against them is g r dz / 2
    w = _w()
    x, y, z = _coords()
    g = 0.7
    s, _ = Lr.region_summaries(w, 10.0 ** (g * x), None, BRICK, MARGIN)
    dz = 2.0 / N
    assert np.allclose(s[:, 2], g * R_IN * dz / 2.0, rtol=1e-5)
    assert np.allclose(s[:, 3:5], 0.0, atol=1e-6)
    # spread of a linear profile over r equally spaced cells
    lx = g * dz * (np.arange(R_IN) - (R_IN - 1) / 2.0)
    assert np.allclose(s[:, 1], lx.std(), rtol=1e-5)


def test_hubble_flow_shifts_by_its_closed_form():
    # v = V r / R: every interior face of a region shifts by -f_mu V dz / (R v_th)
    T = 1.0e4
    w = _w(T=T)
    x, y, z = _coords()
    V = 40.0
    v = V * np.stack([x, y, z], axis=1)
    s, _ = Lr.region_summaries(w, np.ones(w.ncell), v, BRICK, MARGIN)
    vth = 12.85 * np.sqrt(T / 1.0e4)
    delta = -0.5 * V * (2.0 / N) / vth
    assert np.allclose(s[:, 5], delta, rtol=1e-5)
    assert np.allclose(s[:, 6], abs(delta), rtol=1e-5)


def test_partial_bricks_are_marked():
    w = _w()
    s, full = Lr.region_summaries(w, np.ones(w.ncell), None, BRICK, MARGIN, offset=3)
    assert s.shape[0] == 27 and full.sum() == 1  # lattice 3^3 with one whole brick
    assert np.all(s[~full] == 0.0)
