"""C-ABI checks that need no GPU: the library loads, exports every function
declared in include/rddmc.h, and its host-only calls (grid validation, class
deduplication, buffer sizes) behave as documented."""
import os
import re

import numpy as np
import pytest

from paper_1709_10187_gb300 import build as B
from paper_1709_10187_gb300 import rddmc as R
from paper_1709_10187_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def _declared():
    txt = open(os.path.join(ROOT, "include", "rddmc.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|uint64_t|const char\*)\s+(rddmc_\w+)\s*\(", txt, re.M)))


def test_library_exports_every_declared_symbol():
    names = _declared()
    assert len(names) >= 10
    L = R.lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(R.EXPORTED)
    assert R.lib().rddmc_version() >= 100
    assert R.status_string(R.ERR_SIZE) == "buffer too small"


def _grid(w, **kw):
    return R.build_grid(R.GEOM_SLAB_1D if w.ndim == 1 else R.GEOM_CART_3D, w.n, w.edges(), w.R, w.tau0, w.T,
                        v_kms=w.velocity_kms(), mask=w.mask(), **kw)


def test_dedup_classes_and_sizes():
    g = _grid(W.C2)
    s = R.grid_sizes(g, 10_000_000)
    # uniform static slab: left boundary cell, interior cells, right boundary cell
    assert s.n_class == 3 and s.row_bytes == 16 and s.n_outcomes == 4
    assert s.table_bytes >= 3 * 512 * 16
    assert s.tally_bytes == (22 + 512 + 2 + 64 + 512 + 3) * 8
    assert s.state_bytes >= 10_000_000 * 33
    R.destroy_grid(g)
    g = _grid(W.C2, layout=R.LAYOUT_DENSE)
    assert R.grid_sizes(g, 1).n_class == 256
    R.destroy_grid(g)
    # a density gradient leaves every cell its own class
    w = W.SMALL
    g = R.build_grid(R.GEOM_SLAB_1D, w.n, w.edges(), w.R, w.tau0, w.T, n_rel=np.linspace(0.5, 2.0, w.ncell))
    assert R.grid_sizes(g, 1).n_class == w.ncell
    R.destroy_grid(g)


@pytest.mark.parametrize("bad", ["nbins", "edges", "tau0", "slab_n", "density", "source"])
def test_grid_validation_rejects_bad_input(bad):
    w = W.SMALL
    e = w.edges()
    kw = dict(geometry=R.GEOM_SLAB_1D, n=w.n, edges=e, R=w.R, tau0=w.tau0, T=w.T)
    if bad == "nbins":
        kw["edges"] = e[:1]
    elif bad == "edges":
        e2 = e.copy(); e2[3] = e2[2]; kw["edges"] = e2
    elif bad == "tau0":
        kw["tau0"] = -1.0
    elif bad == "slab_n":
        kw["n"] = (w.n[0], 2, 1)
    elif bad == "density":
        kw["n_rel"] = np.full(w.ncell, -1.0)
    elif bad == "source":
        kw["edges"] = np.linspace(1.0, 5.0, w.J + 1)   # x0 = 0 outside the grid
    with pytest.raises(R.RDDMCError) as ei:
        R.build_grid(**kw)
    assert ei.value.status == R.ERR_ARG


def test_moving_medium_requires_uniform_bins():
    w = W.Workload("m", 3, (4, 4, 4), 8, -8.0, 8.0, 1e3, 1e4, 1, 1, sphere=True, vmax_kms=20.0)
    e = np.concatenate([[-8.0], np.sort(np.random.default_rng(1).uniform(-8, 8, 7)), [8.0]])
    with pytest.raises(R.RDDMCError) as ei:
        R.build_grid(R.GEOM_CART_3D, w.n, e, w.R, w.tau0, w.T, v_kms=w.velocity_kms(), mask=w.mask())
    assert ei.value.status == R.ERR_UNSUPPORTED


def test_hubble_sphere_has_few_classes():
    # Homologous flow: every interior face sees the same velocity difference, so
    # the sphere's cells fall into classes by their exterior-face pattern only.
    w = W.C3.with_(vmax_kms=200.0)
    g = _grid(w)
    n_class = R.grid_sizes(g, 1).n_class
    R.destroy_grid(g)
    assert 1 < n_class <= 64, n_class


def test_time_step_validation_without_a_gpu():
    """rddmc_time_step_launch checks its arguments before touching any buffer:
    the pointers below are never dereferenced."""
    g = _grid(W.TINY)
    assert R.time_state_bytes(1000) >= R.grid_sizes(g, 1000).state_bytes + 8 * 1000
    assert R.time_state_bytes(1 << 62) == 0
    fake = 1 << 20  # 256-byte aligned, never dereferenced

    def call(**kw):
        st = R.TimeStep(1, 1000, 0, 0.0, 1.0, 1, 0, 0, 0)
        for k, v in kw.items():
            setattr(st, k, v)
        return R.lib().rddmc_time_step_launch(g, fake, st, fake, 1 << 30, fake, 1 << 20, fake, fake, fake, None,
                                              None, None, None)

    assert call() == R.ERR_TABLE          # no precompute on this grid
    st = R.TimeStep(1, 1000, 0, 0.0, 1.0, 1, 0, 0, 0)
    assert R.lib().rddmc_time_step_launch(g, fake, st, None, 1 << 30, fake, 1 << 20, fake, fake, fake, None,
                                          None, None, None) == R.ERR_ARG
    assert R.lib().rddmc_time_step_launch(g, fake, st, fake, 1 << 30, fake, 1 << 20, fake, fake, fake, fake + 4,
                                          None, None, None) == R.ERR_ARG   # misaligned leak buffer
    R.destroy_grid(g)


def test_dust_parameters_are_validated_without_a_gpu():
    """rddmc_precompute_leakage rejects negative or non-finite dust and dust
    absorption with the hybrid scheme before touching the table buffer."""
    w = W.TINY
    g = _grid(w)
    s = R.grid_sizes(g, 1)
    fake = 1 << 20  # 256-byte aligned, never dereferenced
    bad = [(R.MODE_DDMC, -1.0, 0.0, R.ERR_ARG), (R.MODE_DDMC, 0.0, -2.0, R.ERR_ARG),
           (R.MODE_DDMC, float("inf"), 0.0, R.ERR_ARG), (R.MODE_HYBRID, 0.5, 0.0, R.ERR_UNSUPPORTED)]
    for mode, da, ds, want in bad:
        p = R.LeakParams(5.0, 0.7104, 0.5, mode, 0, da, ds)
        rc = R.lib().rddmc_precompute_leakage(g, p, fake, int(s.table_bytes), None)
        assert rc == want, (mode, da, ds, rc)
    # the outcome count grows by one only once a dusty table is precomputed
    assert s.n_outcomes == 4
    R.destroy_grid(g)


def test_redistribution_sizes_and_validation_without_a_gpu():
    g = _grid(W.SMALL)
    J = W.SMALL.J
    assert R.redistribution_bytes(g) == (J * (J - 1) * 4 + 255) // 256 * 256
    fake = 1 << 20
    nb = R.redistribution_bytes(g)
    L = R.lib()
    assert L.rddmc_precompute_redistribution(g, fake, 0, fake, nb, None) == R.ERR_ARG      # n_sub < 1
    assert L.rddmc_precompute_redistribution(g, fake, 9, fake, nb, None) == R.ERR_ARG      # n_sub > 8
    assert L.rddmc_precompute_redistribution(g, fake, 3, fake, nb - 256, None) == R.ERR_SIZE
    assert L.rddmc_precompute_redistribution(g, fake, 3, fake, nb, None) == R.ERR_TABLE    # no precompute yet
    R.destroy_grid(g)
    g1 = _grid(W.Workload("one_bin", 1, (3, 1, 1), 1, -1.0, 1.0, 10.0, 1.0e4, 1, 1))
    assert R.redistribution_bytes(g1) == 0
    R.destroy_grid(g1)


def test_noalloc_launch_checks_its_arguments_like_launch_packets():
    """rddmc_launch_packets_noalloc runs the checks of rddmc_launch_packets
    (one shared routine), so both return the same status for the same bad
    arguments; here on a grid without a table, where no pointer is touched."""
    import ctypes
    g = _grid(W.TINY)
    fake = 1 << 20  # 256-byte aligned, never dereferenced
    L = R.lib()
    tb = int(R.grid_sizes(g, 1).tally_bytes)

    def both(table, opts, tally):
        a = L.rddmc_launch_packets(g, table, ctypes.byref(opts), fake, 1 << 30, tally, tb, None)
        b = L.rddmc_launch_packets_noalloc(g, table, ctypes.byref(opts), tally, tb, None)
        return a, b

    o = R.RunOpts(1, 1000, 0, 0, 0, 0, 0, 0, 0, 0)
    assert both(None, o, fake) == (R.ERR_ARG, R.ERR_ARG)      # no table
    assert both(fake, o, None) == (R.ERR_ARG, R.ERR_ARG)      # no tallies
    assert both(fake, o, fake) == (R.ERR_TABLE, R.ERR_TABLE)  # table not precomputed
    bad = R.RunOpts(1, 0, 0, 0, 0, 0, 0, 0, 0, 0)             # no packets: still the table first
    assert both(fake, bad, fake) == (R.ERR_TABLE, R.ERR_TABLE)
    assert L.rddmc_launch_packets_noalloc(None, fake, ctypes.byref(o), fake, tb, None) == R.ERR_ARG
    # a learned proposal needs a caller-owned state buffer
    pr = R.Proposal()
    op = R.RunOpts(1, 1000, 0, 64, 0, 0, 0, 0, 0, 0, ctypes.addressof(pr), None)
    assert L.rddmc_launch_packets_noalloc(g, fake, ctypes.byref(op), fake, tb, None) == R.ERR_UNSUPPORTED
    R.destroy_grid(g)


def test_propose_checks_its_arguments_without_a_gpu():
    """rddmc_propose refuses a grid without a table, null buffers (the
    proposal's device buffers included) and misaligned ones before it touches
    any of them; here with fake device addresses that are never dereferenced."""
    import ctypes
    L = R.lib()
    fake = 1 << 20  # 256-byte aligned, never dereferenced
    g = _grid(W.SPHERE8)
    J = W.SPHERE8.J
    served = ctypes.c_uint64(0)

    def call(pr, table=fake, state=fake, tally=fake, work=fake, n=1000, grid=g):
        return L.rddmc_propose(grid, table, ctypes.byref(pr), 1, n, state, tally, 6 * J + 16, 6 * J, 8, 0,
                               fake, fake, 64, work, ctypes.byref(served), None)

    full = R.Proposal(8, 0, fake, fake, fake, 0.0, 12.0, fake, fake, 1, 0, None)
    assert call(full) == R.ERR_TABLE                       # table not precomputed
    assert call(full, table=None) == R.ERR_ARG
    assert call(full, state=None) == R.ERR_ARG
    assert call(full, work=None) == R.ERR_ARG
    assert call(full, grid=None) == R.ERR_ARG
    R.destroy_grid(g)


def test_gather_probe_checks_its_arguments_without_a_gpu():
    """rddmc_gather_probe rejects bad sizes before any launch."""
    import ctypes
    L = R.lib()
    fake = 1 << 20
    n = ctypes.c_uint64(0)

    def call(nbytes, rb, smem=0, chain=16, ctas=0, threads=256, table=fake, sink=fake):
        return L.rddmc_gather_probe(table, nbytes, rb, smem, chain, ctas, threads, 1, 0, sink, ctypes.byref(n), None)

    assert call(4096, 12) == R.ERR_ARG            # row size
    assert call(3000 * 8, 8) == R.ERR_ARG         # not a power of two
    assert call(32 * 8, 8) == R.ERR_ARG           # fewer than 64 rows
    assert call(4096, 8, chain=0) == R.ERR_ARG
    assert call(4096, 8, threads=100) == R.ERR_ARG
    assert call(4096, 8, table=fake + 16) == R.ERR_ARG
    assert call(4096, 8, sink=None) == R.ERR_ARG
    assert call(256 << 10, 8, smem=1) == R.ERR_SIZE
