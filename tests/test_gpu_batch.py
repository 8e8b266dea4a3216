"""Batched instances in one persistent launch (C-ABI rddmc_batch_*): every
instance's integer tallies equal the oracle's for the same global packet ids;
CUDA-graph replays and autotuned schedules change nothing."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import coracle as C  # noqa: E402
from paper_1709_10187_gb300 import build as B  # noqa: E402
from paper_1709_10187_gb300 import rddmc as R  # noqa: E402
from paper_1709_10187_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

MIX = [W.TINY, W.SMALL, W.GREY_LIKE, W.SPHERE8, W.SPHERE8_V,
       W.Workload("slab_one_cell_1x21", 1, (1, 1, 1), 21, -10.0, 10.0, 30.0, 1.0e4, 4000, 0x5EED0202)]
NPK = [3000, 1000, 2000, 1500, 700, 2500]
SEED = 0xBA7C4


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def _same(a, b):
    for k in ("emitted", "escaped", "aborted", "steps", "clamps", "event_draws"):
        assert a[k] == b[k], (k, a[k], b[k])
    assert np.array_equal(a["hist"], b["hist"])
    assert np.array_equal(a["faces"], b["faces"][: len(a["faces"])])
    assert np.array_equal(a["sb"], b["sb"])


def _opts(**kw):
    o = R.RunOpts(SEED, 0, 0, 0, 0, 0, 0, 0, 0, 0)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def test_batch_instances_match_oracle_bit_exactly():
    probs = [R.Problem(w) for w in MIX]
    b = R.Batch(probs, NPK)
    b.launch(_opts())
    off = np.concatenate([[0], np.cumsum(NPK)])
    for i, w in enumerate(MIX):
        og = C.Grid(w)
        ot = og.table()
        orc = C.walk(og, ot, SEED, int(off[i]), NPK[i])
        _same(b.read(i), orc)


def test_graph_replay_and_autotuned_schedule_change_nothing():
    probs = [R.Problem(w) for w in MIX]
    b = R.Batch(probs, NPK, trial_fraction=0.2)
    b.launch(_opts())
    ref = [b.read(i) for i in range(len(MIX))]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # graphs are captured on a non-default stream
        ge = b.graph(_opts(chunk=64))
        try:
            for _ in range(2):
                b.graph_launch(ge)
                for i in range(len(MIX)):
                    _same(b.read(i), ref[i])
        finally:
            R.Batch.graph_destroy(ge)
    torch.cuda.current_stream().wait_stream(side)
    best, rate = b.autotune(_opts())
    assert rate > 0 and best.threads_per_cta in (128, 256) and best.chunk in (64, 256, 1024)
    b.launch(best)
    for i in range(len(MIX)):
        _same(b.read(i), ref[i])


def test_batched_workload_subset_conserves_and_matches_oracle():
    # 48 instances of the batched workload (tau0 1e4-1e8, T 1e2-1e5 K, slabs and
    # spheres, 128-512 bins) at 1/200 of their packets
    ws = W.batched_instances(512, packet_scale=0.005)[:48]
    npk = [w.packets for w in ws]
    probs = [R.Problem(w) for w in ws]
    b = R.Batch(probs, npk)
    b.launch(_opts(max_steps=2_000_000))
    off = np.concatenate([[0], np.cumsum(npk)])
    checked = 0
    for i, w in enumerate(ws):
        t = b.read(i)
        assert t["emitted"] == npk[i] and t["emitted"] == t["escaped"] + t["aborted"]
        if w.ndim == 1 and w.ncell * w.J <= 60_000 and w.tau0 < 1.0e5 and checked < 3:
            og = C.Grid(w)
            ot = og.table()
            thr, _ = probs[i].rows()
            if np.array_equal(thr, ot["thr"]):
                _same(t, C.walk(og, ot, SEED, int(off[i]), npk[i], max_steps=2_000_000))
                checked += 1
    assert checked >= 1


def test_batch_buffers_checked_before_any_write():
    # the autotuner zeroes and reads the whole tally buffer in every trial, and a
    # graph captures the launch: both check the buffers first, as a launch does
    import ctypes
    probs = [R.Problem(w) for w in MIX[:2]]
    b = R.Batch(probs, NPK[:2])
    L = R.lib()
    nb = b.tally.numel() * 8
    b.tally.fill_(0x5A5A)
    torch.cuda.synchronize()
    best = R.RunOpts()
    rate = ctypes.c_double(0.0)
    o = _opts()
    rc = L.rddmc_batch_autotune(b.h, b.desc.data_ptr(), ctypes.byref(o), b.scratch.data_ptr(),
                                b.scratch.numel() * 8, b.tally.data_ptr(), nb - 8, b.stream(), ctypes.byref(best),
                                ctypes.byref(rate))
    assert rc == R.ERR_SIZE
    torch.cuda.synchronize()
    assert bool((b.tally == 0x5A5A).all()), "a refused autotune wrote to the tally buffer"
    side = torch.cuda.Stream()
    ge = ctypes.c_void_p(0)
    for scratch, tally in ((b.scratch.data_ptr() + 4, b.tally.data_ptr()), (b.scratch.data_ptr(), b.tally.data_ptr() + 4)):
        rc = L.rddmc_batch_graph_create(b.h, b.desc.data_ptr(), ctypes.byref(o), scratch, 248, tally, nb - 8,
                                        side.cuda_stream, ctypes.byref(ge))
        assert rc in (R.ERR_ARG, R.ERR_SIZE) and not ge.value, rc
    rc = L.rddmc_batch_launch(b.h, b.desc.data_ptr() + 8, ctypes.byref(o), 0, b.scratch.data_ptr(),
                              b.scratch.numel() * 8, b.tally.data_ptr(), nb, b.stream())
    assert rc == R.ERR_ARG
