"""rddmc_launch_packets_noalloc against rddmc_launch_packets.

The no-allocation entry point serves callers that cannot call cudaMalloc (for
example a plug-in whose host application owns all device memory): it keeps the
packet cursor and saved packet states in a fixed array inside the library
instead of a caller buffer.  Its results must equal the ordinary entry point's
exactly (the tallies are integers), on two calls in a row, since every call
reuses the array the previous call left behind.  This file is collected last,
so a stopping run has already run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1709_10187_gb300 import build as B  # noqa: E402
from paper_1709_10187_gb300 import rddmc as R  # noqa: E402
from paper_1709_10187_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


def _same(a, b):
    for k in ("emitted", "escaped", "aborted", "steps", "clamps", "event_draws", "status"):
        assert a[k] == b[k], (k, a[k], b[k])
    for k in ("hist", "faces", "sb"):
        assert np.array_equal(a[k], b[k]), k


def _noalloc_run(p, opts):
    p.reset()
    R.launch_packets_noalloc(p.grid, p.table.data_ptr(), opts, p.tally.data_ptr(), p.tally.numel() * 8, p.stream())
    return p.read()


def test_noalloc_matches_launch_packets_on_two_calls():
    B.build()
    w = W.SMALL
    p = R.Problem(w)
    ref = p.run(w.packets, w.seed)
    opts = R.RunOpts(w.seed, w.packets, 0, 0, 0, 0, 0, 0, 1, 0)
    for _ in range(2):
        _same(_noalloc_run(p, opts), ref)


def test_noalloc_time_sliced_run_matches_on_two_calls():
    B.build()
    w = W.SPHERE8
    p = R.Problem(w)
    ref = p.run(w.packets, w.seed)
    for _ in range(2):
        p.reset()
        n = 0
        while True:
            o = R.RunOpts(w.seed, w.packets, 0, 64, 1 if n else 0, 0, 0, 0, 1, 0)
            R.launch_packets_noalloc(p.grid, p.table.data_ptr(), o, p.tally.data_ptr(), p.tally.numel() * 8,
                                     p.stream())
            n += 1
            t = p.read()
            if t["escaped"] + t["aborted"] == w.packets:
                break
            assert n < 10_000
        _same(t, ref)


def test_noalloc_rejects_sliced_runs_beyond_its_array():
    B.build()
    w = W.TINY
    p = R.Problem(w)
    o = R.RunOpts(w.seed, 5_000_000, 0, 64, 0, 0, 0, 0, 1, 0)
    with pytest.raises(R.RDDMCError) as ei:
        R.launch_packets_noalloc(p.grid, p.table.data_ptr(), o, p.tally.data_ptr(), p.tally.numel() * 8, p.stream())
    assert ei.value.status == R.ERR_SIZE


def _sliced(p, n, seed, step, launch_fn, done):
    p.reset()
    r = None
    for i in range(100_000):
        launch_fn(R.RunOpts(seed, n, 0, step, 1 if i else 0, 0, 0, 0, 0, 0, None, None))
        r = p.read()
        if done(r):
            return r
    raise AssertionError("sliced run did not finish")


def test_noalloc_weighted_dust_sliced_run_matches():
    # dust by packet weights keeps each packet's -ln(weight) in the last slot
    # of the state, which only a time-sliced run saves and reloads
    B.build()
    w = W.SMALL
    n = 20_000
    p = R.Problem(w, dust_abs=20.0, dust_scat=1.0, dust_weights=True)
    done = lambda r: r["escaped"] + r["absorbed"] + r["aborted"] == n
    p.ensure_state(n)
    ref = _sliced(p, n, w.seed, 256, lambda o: R.launch_packets(
        p.grid, p.table.data_ptr(), o, p.state.data_ptr(), p.state.numel(), p.tally.data_ptr(),
        p.tally.numel() * 8, p.stream()), done)
    for _ in range(2):
        got = _sliced(p, n, w.seed, 256, lambda o: R.launch_packets_noalloc(
            p.grid, p.table.data_ptr(), o, p.tally.data_ptr(), p.tally.numel() * 8, p.stream()), done)
        for k in ("escaped", "absorbed", "aborted", "steps", "event_draws"):
            assert got[k] == ref[k], (k, got[k], ref[k])
        assert got["escaped_weight"] == ref["escaped_weight"]
        assert np.array_equal(got["weight_hist"], ref["weight_hist"]) and np.array_equal(got["hist"], ref["hist"])


def test_noalloc_grouped_hybrid_run_matches():
    # a hybrid table with frequency-grouped MC (the redist option)
    B.build()
    w = W.SPHERE8_V
    n = 20_000
    p = R.Problem(w, mode=R.MODE_HYBRID)
    red = p.redistribution()
    ref = p.run(n, w.seed, redist=red)
    assert ref["mc_events"] > 0
    o = R.RunOpts(w.seed, n, 0, 0, 0, 0, 0, 0, 0, 0, None, red.data_ptr())
    for _ in range(2):
        got = _noalloc_run(p, o)
        _same(got, ref)
        for k in ("mc_events", "conversions"):
            assert got[k] == ref[k], k


def test_noalloc_refuses_the_redistribution_options_launch_packets_refuses():
    # frequency grouping needs a hybrid table and a 4-byte aligned buffer; both
    # entry points check before launching, so the pointers are never read
    B.build()
    L = R.lib()
    w = W.TINY
    pd = R.Problem(w)
    ph = R.Problem(w, mode=R.MODE_HYBRID)
    red = ph.redistribution()
    pd.ensure_state(1000)
    ph.ensure_state(1000)
    for p, ptr in ((pd, red.data_ptr()), (ph, red.data_ptr() + 2)):
        o = R.RunOpts(w.seed, 1000, 0, 0, 0, 0, 0, 0, 0, 0, None, ptr)
        a = L.rddmc_launch_packets(p.grid, p.table.data_ptr(), ctypes.byref(o), p.state.data_ptr(),
                                   p.state.numel(), p.tally.data_ptr(), p.tally.numel() * 8, p.stream())
        b = L.rddmc_launch_packets_noalloc(p.grid, p.table.data_ptr(), ctypes.byref(o), p.tally.data_ptr(),
                                           p.tally.numel() * 8, p.stream())
        assert a == b == R.ERR_ARG, (a, b)
