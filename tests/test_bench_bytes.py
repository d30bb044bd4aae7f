"""The algorithmic byte counts behind bench.py's roofline figure (host logic, no GPU): every
array a launch must touch is read once and every output written once."""
import bench


def test_algorithmic_bytes_of_the_cylinder_batch():
    n = 16 * 257 * 512
    es = ms = 4
    # Y0: phi and s_1 in, D_1 and s_1 d4_1 out
    assert bench.algorithmic_bytes("deriv", n, 2, es, ms, True) == n * 4 * es
    # direction-0 pass: phi, D_1, s_1 d4_1, s_0 and 4 metric arrays in; D_0, Lap_0, G_0 (and
    # kappa_0 with the curvature correction) out
    assert bench.algorithmic_bytes("line0", n, 2, es, ms, True) == n * (3 * es + 5 * ms + 4 * es)
    assert bench.algorithmic_bytes("line0", n, 2, es, ms, False) == n * (3 * es + 5 * ms + 3 * es)
    # direction-1 pass averaged over the 4 stages: 11 state-size fields, 1.5 of dt / acc, 0.5 of
    # the time-step metric sums, 0.75 of s_1 in, 3.5 out, the flags
    assert bench.algorithmic_bytes("line1", n, 2, es, ms, True) == n * 70
    assert bench.algorithmic_bytes("filter", n, 2, es, ms, True) == n * 2 * es
    assert bench.algorithmic_bytes("norm", n, 2, es, ms, True) == n * (3 * es + 1)
    assert bench.algorithmic_bytes("gauss", n, 2, es, ms, True) is None


def test_reference_arm_contract():
    """`bench.py --impl reference` (the oracle on the host cores) prints one JSON line with
    the contract's keys: the same metric and unit as the native arm, its own e2e block and a
    cpu_baseline describing the run."""
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3 and d["higher_is_better"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
