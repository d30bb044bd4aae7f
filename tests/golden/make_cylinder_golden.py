"""Writes tests/golden/cylinder257x512_c6_lad_curv.json: the FP64 oracle's converged wall
distance on the sixteen full-size cylinder O-grids of the batched benchmark workload
(257 radial x 512 periodic nodes, wall radius 0.5 (1 + k/100), outer radius 10, radial
ratio 1.03), C6 + LAD + the curvature correction of Eq. 25, alpha_f 0.495, solved to an
RMS change of 1e-12.

Calls only the oracle (oracle/) and the input generator (workloads.py); no value comes from
the CUDA path.  Each grid is rotationally symmetric: rotating by one angular step maps node
(i, j) onto node (i + 1, j) exactly in exact arithmetic, and every operator of the method
(the HJ terms, the LAD diffusivity, the curvature correction, the filter along the periodic
direction, the local time step) is invariant under that map.  So the discrete solution
depends on j alone, up to rounding.  The file stores, per grid, the oracle's field averaged
over i for each j, and the largest spread over i of the full field (max - min at one j),
which bounds what the average leaves out.

    python tests/golden/make_cylinder_golden.py [--members K] [--workers W]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "cylinder257x512_c6_lad_curv.json")

NR, NT, RATIO = 257, 512, 1.03
PARAMS = dict(equation=1, scheme=4, curvature=1, eps=0.2, C_lad=0.1, lad_exp=3.0, alpha_f=0.495,
              filter=1, cfl=0.6, eps0=1e-8, tol_l2=1e-12, tol_linf=0.0, max_iters=60000,
              check_every=10, init=1, poisson_tol=0.0, poisson_max_iters=100)


def r_wall(k):
    return 0.5 * (1 + 0.01 * k)


def solve_member(k):
    sys.path.insert(0, ROOT)
    import numpy as np

    import oracle as O
    from paper_2111_09859_gb300 import workloads as W

    sp = W.cylinder(NR, NT, RATIO, r_wall=r_wall(k))
    og = O.Grid(sp.shape, sp.xyz, sp.bc_lo, sp.bc_hi, scheme=O.C6, period=sp.period, L_ref=sp.L_ref)
    t0 = time.time()
    phi, st = og.solve(**PARAMS)
    a = phi.reshape(NR, NT)
    spread = float((a.max(axis=1) - a.min(axis=1)).max())
    exact = np.hypot(*sp.xyz) - r_wall(k)
    return dict(k=k, r_wall=r_wall(k), iters=st["iters"], poisson_iters=st["poisson_iters"],
                res_l2=st["res_l2"], converged=st["converged"], spread_over_i=spread,
                max_err_vs_exact=float(np.abs(phi - exact).max()), seconds=round(time.time() - t0, 1),
                d=[float(v) for v in a.mean(axis=1)])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--members", type=int, default=16)
    ap.add_argument("--workers", type=int, default=min(8, os.cpu_count() or 1))
    args = ap.parse_args()
    sys.path.insert(0, ROOT)
    import oracle as O

    O.build()
    with mp.get_context("spawn").Pool(args.workers) as pool:
        rows = pool.map(solve_member, range(args.members))
    for r in rows:
        assert r["converged"], r
        assert r["spread_over_i"] <= 1e-9, r["spread_over_i"]
    doc = {
        "what": "FP64 oracle wall distance d(j) on the 257 x 512 cylinder O-grids of the batched workload; "
                "d depends on the radial index j only (rotational symmetry), spread_over_i bounds the rest",
        "grid": {"nr": NR, "nt": NT, "ratio": RATIO, "r_out": 10.0, "r_wall": "0.5 (1 + k/100)"},
        "params": PARAMS,
        "writer": "tests/golden/make_cylinder_golden.py (oracle/ only)",
        "members": rows,
    }
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=0)
    print(OUT, [(r["k"], r["iters"], r["seconds"]) for r in rows])


if __name__ == "__main__":
    main()
