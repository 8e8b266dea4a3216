"""rddmc_launch_packets_noalloc against rddmc_launch_packets.

The no-allocation entry point serves callers that cannot call cudaMalloc (for
example a plug-in whose host application owns all device memory): it keeps the
packet cursor and saved packet states in a fixed array inside the library
instead of a caller buffer.  Its results must equal the ordinary entry point's
exactly (the tallies are integers), on two calls in a row, since every call
reuses the array the previous call left behind.  This file is collected last,
so a stopping run has already run every other test.
"""
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
