"""Host logic of the benchmark's learned-against-plain protocol, on synthetic
multinomial spectra whose bias and noise are known."""
import numpy as np

import bench


def _spectra(p, npk, runs, rng, sec):
    return [(sec, rng.multinomial(npk, p).astype(np.float64)) for _ in range(runs)]


def test_equal_l1_recovers_bias_floor_and_time_ratio():
    rng = np.random.default_rng(1)
    x = np.linspace(-6, 6, 60)
    p = np.exp(-0.5 * x * x)
    p /= p.sum()
    npk, n_ref = 20_000, 4_000_000
    ref = rng.multinomial(n_ref, p)
    # unbiased arms: the "learned" one is twice as fast per packet
    runs_p = _spectra(p, npk, 8, rng, 2.0)
    runs_l = _spectra(p, npk, 8, rng, 1.0)
    r = bench._equal_l1(runs_l, runs_p, ref, n_ref, npk, n_boot=50)
    assert r["bias_floor_plain"]["value"] < 0.01 and r["bias_floor_learned"]["value"] < 0.01
    assert 1.3 < r["speedup_at_0.02"]["value"] < 3.2, r["speedup_at_0.02"]
    assert len(r["curve_learned"]["l1"]) == 8 and r["curve_learned"]["l1"][-1] < r["curve_learned"]["l1"][0]
    # a biased learned arm: L1 distance 0.03 from the truth; the floor shows, and
    # the 1 % target is out of its reach
    q = p * (1.0 + 0.3 * np.sin(x))
    q /= q.sum()
    b = float(np.abs(q - p).sum())
    runs_b = _spectra(q, npk, 8, rng, 1.0)
    r = bench._equal_l1(runs_b, runs_p, ref, n_ref, npk, n_boot=50)
    assert abs(r["bias_floor_learned"]["value"] - b) < 0.35 * b, (r["bias_floor_learned"], b)
    assert r["speedup_at_0.01"]["value"] == 0.0 or b < 0.01


def test_reference_arm_prints_one_contract_line():
    # the reference arm (the FP64 oracle on the host cores) needs no GPU: one
    # JSON line with the contract's keys, its own e2e block and no host copies
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "dtype",
              "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]


def test_walk_counters_describe_the_current_walk_source():
    # the bench states the walk's issue fraction and DRAM traffic from a committed
    # ncu capture only while the walk's sources hash to the captured ones; a
    # change to them needs a new capture (or, for a host-only change, evidence
    # that the device code is unchanged, recorded beside the hash)
    import json
    import os
    p = os.path.join(os.path.dirname(bench.__file__), "profiles", "walk_kernel_traffic.json")
    d = json.load(open(p))
    assert d["kernel_hash"] == bench._kernel_hash()
    assert d["packets"] == 10_000_000 and d["slice_transitions"] == 4096
