"""GPU parity of the leakage table and the DDMC walk against the FP64 oracle.

Integer results are compared bit-exactly (thresholds to one count where CUDA's
and the C library's erf/exp may round differently), spectra statistically
against the exact absorbing chain and the Neufeld profile.  All calls go
through the C-ABI (paper_1709_10187_gb300.rddmc)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import analytic as A  # noqa: E402
from oracle import coracle as C  # noqa: E402
from paper_1709_10187_gb300 import build as B  # noqa: E402
from paper_1709_10187_gb300 import rddmc as R  # noqa: E402
from paper_1709_10187_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

# Edge cases: a single grey bin, a single cell (both faces exterior), a wide
# histogram that does not fit shared memory, odd cell/bin counts.
ONE_BIN = W.Workload("slab_one_bin_9x1", 1, (9, 1, 1), 1, -5.0, 5.0, 50.0, 1.0e4, 4000, 0x5EED0201)
ONE_CELL = W.Workload("slab_one_cell_1x21", 1, (1, 1, 1), 21, -10.0, 10.0, 30.0, 1.0e4, 4000, 0x5EED0202)
WIDE_J = W.Workload("slab_wide_hist_5x9001", 1, (5, 1, 1), 9001, -450.0, 450.0, 2.0e3, 1.0e4, 1000, 0x5EED0203)
BIT_EXACT = [W.TINY, W.SMALL, W.GREY_LIKE, ONE_BIN, ONE_CELL, WIDE_J, W.SPHERE8, W.SPHERE8_V, W.SPHERE9_V]


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    assert torch.cuda.is_available()


def _oracle(w, hybrid=False):
    g = C.Grid(w, hybrid=hybrid)
    return g, g.table()


def _same_tallies(gpu, orc, check_draws=True):
    for k in ("emitted", "escaped", "aborted", "steps", "clamps"):
        assert gpu[k] == orc[k], (k, gpu[k], orc[k])
    if check_draws:
        assert gpu["event_draws"] == orc["event_draws"]
    assert np.array_equal(gpu["hist"], orc["hist"])
    assert np.array_equal(gpu["faces"], orc["faces"][: len(gpu["faces"])])
    assert np.array_equal(gpu["sb"], orc["sb"])


@pytest.mark.parametrize("w", BIT_EXACT + [W.C1, W.C2, W.P1, W.P2, W.C3, W.C3_V200], ids=lambda w: w.name)
@pytest.mark.parametrize("hybrid", [False, True], ids=["ddmc", "hybrid"])
def test_table_matches_oracle(w, hybrid):
    og, ot = _oracle(w, hybrid)
    p = R.Problem(w, mode=R.MODE_HYBRID if hybrid else R.MODE_DDMC)
    thr, flags = p.rows()
    # vacuum cells (outside a sphere) hold no rows on the GPU; compare the medium
    m = w.mask()
    sel = np.ones(w.ncell * w.J, bool) if m is None else np.repeat(m.astype(bool), w.J)
    assert np.array_equal(flags[sel], ot["flags"][sel])
    thr, ot = thr[sel], dict(ot, thr=ot["thr"][sel])
    d = thr.astype(np.int64) - ot["thr"].astype(np.int64)
    assert np.abs(d).max() <= 1
    assert (d != 0).mean() <= 1e-4, (d != 0).sum()


@pytest.mark.parametrize("w", BIT_EXACT, ids=lambda w: w.name)
def test_walk_bit_exact_vs_oracle(w):
    og, ot = _oracle(w)
    p = R.Problem(w)
    thr, flags = p.rows()
    assert _medium_rows_equal(w, thr, ot), "tables differ: bit-exact walk needs identical thresholds"
    gpu = p.run(w.packets, w.seed)
    orc = C.walk(og, ot, w.seed, 0, w.packets)
    _same_tallies(gpu, orc)
    assert gpu["status"] == R.OK
    assert gpu["emitted"] == gpu["escaped"] == w.packets


def test_walk_bit_exact_c1_subset_and_p2():
    for w, npk in ((W.C1, 200), (W.P2, 20000)):
        og, ot = _oracle(w)
        p = R.Problem(w)
        thr, _ = p.rows()
        assert np.array_equal(thr, ot["thr"])
        _same_tallies(p.run(npk, w.seed), C.walk(og, ot, w.seed, 0, npk))


def test_time_sliced_launches_equal_one_launch():
    w = W.SMALL
    p = R.Problem(w)
    one = p.run(w.packets, w.seed)
    p.reset()
    n = 0
    while True:
        p.launch(w.packets, w.seed, steps_per_launch=64, resume=1 if n else 0)
        n += 1
        t = p.read()
        if t["escaped"] + t["aborted"] == w.packets:
            break
        assert n < 10_000
    _same_tallies(t, one)
    assert n > 10


def test_watchdog_aborts_match_oracle():
    w = W.SMALL
    og, ot = _oracle(w)
    p = R.Problem(w)
    gpu = p.run(w.packets, w.seed, max_steps=1001)
    orc = C.walk(og, ot, w.seed, 0, w.packets, max_steps=1001)
    _same_tallies(gpu, orc)
    assert gpu["aborted"] > 0 and gpu["status"] == R.ERR_STEP_LIMIT


@pytest.mark.parametrize("sched", [dict(ctas_per_sm=1, threads_per_cta=64, chunk=4, table_in_smem=0),
                                   dict(ctas_per_sm=2, threads_per_cta=256, chunk=256, table_in_smem=1),
                                   dict(threads_per_cta=96, chunk=12)])
def test_schedule_does_not_change_results(sched):
    w = W.SMALL
    p = R.Problem(w)
    ref = p.run(w.packets, w.seed)
    _same_tallies(p.run(w.packets, w.seed, **sched), ref)


def test_dense_layout_equals_dedup_layout():
    w = W.GREY_LIKE
    a = R.Problem(w).run(w.packets, w.seed)
    b = R.Problem(w, layout=R.LAYOUT_DENSE).run(w.packets, w.seed)
    _same_tallies(a, b)


@pytest.mark.parametrize("npk", [1, 31, 33, 1000])
def test_ragged_packet_counts(npk):
    w = W.TINY
    og, ot = _oracle(w)
    _same_tallies(R.Problem(w).run(npk, w.seed + npk), C.walk(og, ot, w.seed + npk, 0, npk))


def test_spectrum_p1_matches_chain_and_neufeld():
    # Fig. 2 setup, 1e6 packets: 3 sigma against the exact chain; L1 <= 2% vs eq. Neufeld.
    w = W.P1
    og, ot = _oracle(w)
    ch = A.chain_solve(w, ot)
    gpu = R.Problem(w).run(w.packets, w.seed)
    N = w.packets
    assert gpu["escaped"] == N
    zmax, frac, pval = A.compare_counts_to_probs(gpu["hist"], ch["hist"], N)
    assert zmax < 5.0 and frac <= 0.02 and pval > 1e-3, (zmax, frac, pval)
    zs = (gpu["steps"] / N - ch["steps_mean"]) / np.sqrt(ch["steps_var"] / N)
    assert abs(zs) < 4.0
    l1 = A.l1_distance(gpu["hist"][1:-1], A.neufeld_bin_mass(w.edges(), C.damping(w.T) * w.tau0))
    assert l1 <= 0.02, l1


def test_spectrum_c1_matches_chain():
    w = W.C1
    og, ot = _oracle(w)
    ch = A.chain_solve(w, ot)
    gpu = R.Problem(w).run(w.packets, w.seed)
    zmax, frac, pval = A.compare_counts_to_probs(gpu["hist"], ch["hist"], w.packets)
    assert zmax < 5.0 and frac <= 0.02 and pval > 1e-3, (zmax, frac, pval)
    zs = (gpu["steps"] / w.packets - ch["steps_mean"]) / np.sqrt(ch["steps_var"] / w.packets)
    assert abs(zs) < 4.0


def test_wide_core_grid_walk_is_bit_exact():
    # non-uniform bins (one wide core bin, unit wing bins) on the tau0 = 1e5 slab
    w = W.C1_WIDECORE
    og, ot = _oracle(w)
    thr, flags = R.Problem(w).rows()
    d = thr.astype(np.int64) - ot["thr"].astype(np.int64)
    assert np.abs(d).max() <= 1 and np.array_equal(flags, ot["flags"])
    # the oracle walks the table the device exported, so one-count differences
    # cannot make the trajectories part
    n = 20_000
    _same_tallies(R.Problem(w).run(n, w.seed), C.walk(og, dict(ot, thr=thr, flags=flags), w.seed, 0, n))


def test_c2_completed_subset_matches_the_exact_chain():
    # 1e5 packets of the tau0 = 1e7 slab (256 cells x 512 uniform bins) walked
    # to escape in step slices of 2^24 transitions: ~3e13 transitions, the
    # slowest packet ~3e9.  The spectrum, the face counts and the mean number
    # of transitions against the exact absorbing chain of the oracle's table
    # (the device table is bit-identical on this grid).
    w = W.C2
    og, ot = _oracle(w)
    ch = A.chain_solve(w, ot)
    n = 100_000
    p = R.Problem(w)
    thr, flags = p.rows()
    assert np.array_equal(thr, ot["thr"]) and np.array_equal(flags, ot["flags"])
    p.reset()
    launches = 0
    while True:
        p.launch(n, w.seed, steps_per_launch=1 << 24, resume=1 if launches else 0)
        launches += 1
        t = p.read()
        if t["escaped"] + t["aborted"] == n:
            break
        assert launches < 2000
    assert t["escaped"] == n and t["aborted"] == 0
    zmax, frac, pval = A.compare_counts_to_probs(t["hist"], ch["hist"], n)
    assert zmax < 5.0 and frac <= 0.02 and pval > 1e-3, (zmax, frac, pval)
    fz = (t["faces"][:2] - n * ch["faces"][:2]) / np.sqrt(n * ch["faces"][:2] * (1 - ch["faces"][:2]))
    assert np.all(np.abs(fz) < 4.0), fz
    zs = (t["steps"] / n - ch["steps_mean"]) / np.sqrt(ch["steps_var"] / n)
    assert abs(zs) < 4.0, (t["steps"] / n, ch["steps_mean"])


def test_c2_wide_core_run_to_completion_matches_chain():
    # every one of 1e6 packets of the tau0 = 1e7 slab on the wide-core grid walked
    # to escape (~2e4 transitions each), against the exact chain's spectrum and
    # mean transition count
    w = W.C2_WIDECORE
    og, ot = _oracle(w)
    ch = A.chain_solve(w, ot)
    n = 1_000_000
    gpu = R.Problem(w).run(n, w.seed)
    assert gpu["escaped"] == n and gpu["aborted"] == 0
    zmax, frac, pval = A.compare_counts_to_probs(gpu["hist"], ch["hist"], n)
    assert zmax < 5.0 and frac <= 0.02 and pval > 1e-3, (zmax, frac, pval)
    zs = (gpu["steps"] / n - ch["steps_mean"]) / np.sqrt(ch["steps_var"] / n)
    assert abs(zs) < 4.0, zs


def test_c2_full_size_sampled_packets_replay_exactly():
    # tau0 = 1e7 slab, 256 x 512, all 1e7 packets, one time slice of 4096
    # transitions as the benchmark launches it; sampled packets are replayed one
    # by one by the oracle and must end in the same state.
    w = W.C2
    S = 4096
    og, ot = _oracle(w)
    p = R.Problem(w)
    thr, _ = p.rows()
    assert np.array_equal(thr, ot["thr"])
    p.reset()
    p.launch(w.packets, w.seed, steps_per_launch=S)
    t = p.read()
    assert t["emitted"] == w.packets
    ids = np.unique(np.concatenate([np.arange(8), np.linspace(8, w.packets - 1, 40).astype(np.int64)]))
    for pid in ids:
        st = p.packet_states(w.packets, int(pid), 1)
        ref = C.replay_packet(og, ot, w.seed, int(pid), S)
        assert st["status"][0] == (2 if ref["done"] else 1)
        if not ref["done"]:
            assert (st["cell"][0], st["bin"][0], st["steps"][0], st["event_draws"][0]) == \
                (ref["cell"], ref["bin"], ref["steps"], ref["event_draws"])
    # every packet advanced S transitions unless it escaped first
    assert t["steps"] <= w.packets * S
    assert t["steps"] + t["escaped"] * S >= w.packets * S


def _medium_rows_equal(w, thr, ot):
    m = w.mask()
    sel = np.ones(w.ncell * w.J, bool) if m is None else np.repeat(m.astype(bool), w.J)
    return np.array_equal(thr[sel], ot["thr"][sel])


def _sampled_replay(w, S, n_ids=40):
    og, ot = _oracle(w)
    p = R.Problem(w)
    thr, flags = p.rows()
    assert _medium_rows_equal(w, thr, ot)
    p.reset()
    p.launch(w.packets, w.seed, steps_per_launch=S)
    t = p.read()
    assert t["emitted"] == w.packets
    ids = np.unique(np.concatenate([np.arange(8), np.linspace(8, w.packets - 1, n_ids).astype(np.int64)]))
    for pid in ids:
        st = p.packet_states(w.packets, int(pid), 1)
        ref = C.replay_packet(og, ot, w.seed, int(pid), S)
        assert st["status"][0] == (2 if ref["done"] else 1)
        if not ref["done"]:
            assert (st["cell"][0], st["bin"][0], st["steps"][0], st["event_draws"][0]) == \
                (ref["cell"], ref["bin"], ref["steps"], ref["event_draws"])
    return t


@pytest.mark.parametrize("w", [W.C3, W.C3_V200], ids=lambda w: w.name)
def test_c3_full_size_sampled_packets_replay_exactly(w):
    # 64^3 sphere x 128 bins, all 1e7 packets, one slice of 2048 transitions;
    # sampled packets replayed one by one by the oracle end in the same state.
    t = _sampled_replay(w, 2048)
    assert t["steps"] <= w.packets * 2048


@pytest.mark.parametrize("w", [W.SPHERE8, W.SPHERE9_V.with_(vmax_kms=0.0, name="sphere_small_static")],
                         ids=lambda w: w.name)
def test_static_sphere_matches_chain_and_is_isotropic(w):
    og, ot = _oracle(w)
    ch = A.chain_solve(w, ot)
    N = 200_000
    gpu = R.Problem(w).run(N, w.seed + 7)
    assert gpu["escaped"] == N
    zmax, frac, pval = A.compare_counts_to_probs(gpu["hist"], ch["hist"], N)
    assert zmax < 5.0 and frac <= 0.02 and pval > 1e-3, (zmax, frac, pval)
    # six faces equally likely; escape points lie at b <= ~R (sphere of radius R)
    f = gpu["faces"].astype(float)
    z = (f - N / 6) / np.sqrt(N / 6 * 5 / 6)
    assert np.all(np.abs(z) < 4.0), f
    sb = gpu["sb"].astype(float)
    assert sb.sum() == N and sb[int(1.25 / 1.28 * 64):].sum() == 0


def test_outflow_shifts_escape_spectrum_red():
    # Hubble-like outflow: photons are redshifted relative to the static sphere
    # (qualitative, Sec. 5.4 discusses the red/blue asymmetry).
    w0 = W.SPHERE9_V.with_(vmax_kms=0.0, name="s0")
    w1 = W.SPHERE9_V.with_(vmax_kms=200.0, name="s1")
    N = 100_000
    e = w0.edges()
    xc = 0.5 * (e[1:] + e[:-1])
    m = []
    for w in (w0, w1):
        h = R.Problem(w).run(N, w.seed)["hist"][1:-1].astype(float)
        m.append((h * xc).sum() / h.sum())
    assert m[1] < m[0] - 0.5, m
