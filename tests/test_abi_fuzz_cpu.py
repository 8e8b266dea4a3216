"""Property test of rddmc_build_grid's validation (host-only, no GPU): over
random grid descriptions the library accepts exactly the valid ones and
refuses the others with the status its header documents, in its order:

* RDDMC_ERR_ARG for non-finite or non-positive R and T, a negative or
  non-finite tau0, frequency edges that are not finite and strictly
  increasing, a negative or non-finite density, a non-finite velocity;
* then RDDMC_ERR_UNSUPPORTED for a moving medium on non-uniform bins;
* then RDDMC_ERR_ARG when x0 = 0 lies in no bin, or a source cell (the centre
  cell, or the two that straddle the centre on an axis of even count) is
  outside the medium mask."""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

from paper_1709_10187_gb300 import rddmc as R  # noqa: E402


def _centre(m):
    return [m // 2] if m % 2 else [m // 2 - 1, m // 2]


def _expected(ndim, n, edges, Rv, tau0, T, n_rel, v, mask):
    fin = np.all(np.isfinite(edges)) and np.all(np.diff(edges) > 0.0)
    if not (Rv > 0 and np.isfinite(Rv) and T > 0 and np.isfinite(T) and tau0 >= 0 and np.isfinite(tau0) and fin):
        return R.ERR_ARG
    if n_rel is not None and not np.all((n_rel >= 0.0) & np.isfinite(n_rel)):
        return R.ERR_ARG
    if v is not None and not np.all(np.isfinite(v)):
        return R.ERR_ARG
    dx = np.diff(edges)
    uniform = bool(np.all(np.abs(dx - dx[0]) <= 1e-9 * abs(dx[0])))
    if v is not None and np.any(v != 0.0) and not uniform:
        return R.ERR_UNSUPPORTED
    J = len(edges) - 1
    has_src = any(edges[j] == 0.0 for j in range(1, J)) or any(edges[j] < 0.0 < edges[j + 1] for j in range(J))
    if not has_src:
        return R.ERR_ARG
    if mask is not None:
        for i2 in _centre(n[2]):
            for i1 in _centre(n[1]):
                for i0 in _centre(n[0]):
                    if not mask[i0 + n[0] * (i1 + n[1] * i2)]:
                        return R.ERR_ARG
    return R.OK


DEFECTS = ["none", "none", "none", "R", "tau0", "T", "edges_repeat", "edges_nan", "edges_one_side", "density",
           "velocity_nan", "moving_nonuniform", "mask_source"]


@settings(max_examples=500, deadline=None, derandomize=True, database=None)
@given(st.data())
def test_build_grid_accepts_exactly_the_valid_descriptions(data):
    # a valid description with at most one defect; the expected status is
    # computed from the description itself, not from the defect's name
    ndim = data.draw(st.sampled_from([1, 3]))
    if ndim == 1:
        n = (data.draw(st.integers(1, 7)), 1, 1)
    else:
        n = tuple(data.draw(st.integers(1, 4)) for _ in range(3))
    ncell = n[0] * n[1] * n[2]
    J = data.draw(st.integers(1, 10))
    rng = np.random.default_rng(data.draw(st.integers(0, 2 ** 32 - 1)))
    xm = float(data.draw(st.sampled_from([1.0, 7.5, 60.0])))
    defect = data.draw(st.sampled_from(DEFECTS))
    uniform = data.draw(st.booleans())
    edges = np.linspace(-xm, xm, J + 1)
    if not uniform and J >= 2:
        inner = np.sort(rng.uniform(-xm, xm, J - 1))
        inner[np.argmin(np.abs(inner))] = 0.0 if rng.random() < 0.5 else inner[np.argmin(np.abs(inner))]
        edges = np.concatenate([[-xm], inner, [xm]])
    Rv, tau0, T = 1.0, float(data.draw(st.sampled_from([0.0, 10.0, 1.0e7]))), float(data.draw(st.sampled_from([10.0, 1.0e4])))
    n_rel = rng.uniform(0.1, 3.0, ncell) if data.draw(st.booleans()) else None
    v = None
    vel = data.draw(st.sampled_from(["none", "static", "moving"]))
    if vel != "none":
        v = np.zeros((ncell, 3)) if vel == "static" else rng.normal(0.0, 20.0, (ncell, 3))
    mask = None
    if ndim == 3 and data.draw(st.booleans()):
        mask = (rng.random(ncell) < 0.5).astype(np.uint8)
        for i2 in _centre(n[2]):
            for i1 in _centre(n[1]):
                for i0 in _centre(n[0]):
                    mask[i0 + n[0] * (i1 + n[1] * i2)] = 1
    if defect == "R":
        Rv = float(data.draw(st.sampled_from([0.0, -1.0, float("inf")])))
    elif defect == "tau0":
        tau0 = float(data.draw(st.sampled_from([-1.0, float("nan"), float("inf")])))
    elif defect == "T":
        T = float(data.draw(st.sampled_from([0.0, -3.0])))
    elif defect == "edges_repeat" and J >= 2:
        edges[1] = edges[0]
    elif defect == "edges_nan":
        edges[rng.integers(0, J + 1)] = np.nan
    elif defect == "edges_one_side":
        edges = edges - edges[0] + 1.0  # x0 = 0 below the grid
    elif defect == "density":
        n_rel = rng.uniform(0.1, 3.0, ncell)
        n_rel[rng.integers(0, ncell)] = -0.5 if rng.random() < 0.5 else np.nan
    elif defect == "velocity_nan":
        v = np.zeros((ncell, 3))
        v[rng.integers(0, ncell), rng.integers(0, 3)] = np.nan
    elif defect == "moving_nonuniform" and J >= 3:
        v = rng.normal(0.0, 20.0, (ncell, 3))
        edges = np.concatenate([[-xm], np.sort(rng.uniform(-xm, xm, J - 1)), [xm]])
    elif defect == "mask_source" and ndim == 3:
        mask = np.ones(ncell, dtype=np.uint8)
        mask[_centre(n[0])[0] + n[0] * (_centre(n[1])[0] + n[1] * _centre(n[2])[0])] = 0
    want = _expected(ndim, n, edges, Rv, tau0, T, n_rel, v, mask)
    hyp.event(f"status {want}")
    geom = R.GEOM_SLAB_1D if ndim == 1 else R.GEOM_CART_3D
    try:
        g = R.build_grid(geom, n, edges, Rv, tau0, T, n_rel=n_rel, v_kms=v, mask=mask)
    except R.RDDMCError as e:
        assert e.status == want, (e.status, want, defect, edges, Rv, tau0, T)
        return
    assert want == R.OK, (want, defect, edges, Rv, tau0, T)
    s = R.grid_sizes(g, 10)
    assert s.n_class >= 1 and s.table_bytes > 0 and s.state_bytes > 0
    R.destroy_grid(g)
