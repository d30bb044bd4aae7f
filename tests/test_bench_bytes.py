"""The algorithmic byte counts behind bench.py's roofline figure (host logic, no GPU): every
array a launch must touch is read once and every output written once."""
import bench


def test_algorithmic_bytes_of_the_cylinder_batch():
    n = 16 * 257 * 512
    es = ms = 4
    # direction derivative: phi in, D_l out; LAD on average s_l in plus 1.5 state fields
    assert bench.algorithmic_bytes("deriv", n, 2, es, ms, True) == int(n * (2 * es + 1.5 * es + ms))
    # both directions' divergence passes in one launch: D_0, D_1 and the 4 metric arrays in
    # once; Lap_0, Lap_1 (and kappa_0, kappa_1 with the curvature correction) out
    assert bench.algorithmic_bytes("div", n, 2, es, ms, True) == n * (2 * es + 4 * ms + 4 * es)
    assert bench.algorithmic_bytes("div", n, 2, es, ms, False) == n * (2 * es + 4 * ms + 2 * es)
    assert bench.algorithmic_bytes("div", n, 2, es, ms, True) == 84213760
    # the stage: 11 state-size fields and 4 metric arrays in, the stage value and acc out, flags
    assert bench.algorithmic_bytes("point", n, 2, es, ms, True) == n * (13 * es + 4 * ms + 1)
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
