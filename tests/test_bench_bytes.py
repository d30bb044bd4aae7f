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
