"""Runs pseudo steps of a named workload on the GPU, for profilers (ncu) and quick per-class
kernel timings; prints one line per run.

    python -m paper_2111_09859_gb300.profile_case CASE [--steps K] [--warmup W] [--timer]

CASE:
  cyl16     16 stacked cylinder O-grids 257 x 512, C6 + LAD + curvature, alpha_f 0.495,
            FP32 state (metrics computed in FP64)
  cyl16-64  the same 16 cylinders in FP64
  duct256   square duct 256^3, E6 + LAD, FP32
  duct128   square duct 128 x 128 x 128 (a small case of the same kernels)
  star1025  star port 1025^2, E4 + LAD, FP32
  star1025-ls  the same star, level-set steps (F = 0.3, dt = 0.5 h / F) instead of pseudo
            steps, from the exact signed distance
  chan-uw   channel 1024 x 513, baseline upwind scheme, standard HJ, FP64 (generic path)
  ell2048   one ellipse O-grid 1025 x 2048, C6 + LAD, FP32

The field starts from the exact distance where one exists (random smooth field
otherwise), so the steps exercise the converged regime.  --timer turns on the library's
per-class kernel timer (CUDA events around every launch) and prints the class totals.
"""
from __future__ import annotations

import argparse
import time

import numpy as np


def build_case(name):
    from paper_2111_09859_gb300 import workloads as W, wd

    if name.startswith("cyl16"):
        spec = W.stack([W.cylinder(257, 512, 1.03, r_wall=0.5 * (1 + 0.01 * k)) for k in range(16)])
        prec = wd.FP64 if name == "cyl16-64" else wd.FP32_METRIC64
        p = wd.default_params(wd.C6, equation=wd.HJ_LAD, curvature=1, alpha_f=0.495)
        x, y = spec.xyz
        r0 = np.repeat([0.5 * (1 + 0.01 * k) for k in range(16)], 257 * 512)
        return spec, prec, wd.C6, p, np.hypot(x, y) - r0
    if name.startswith("duct"):
        n = int(name[4:])
        spec = W.duct(n)
        p = wd.default_params(wd.E6, equation=wd.HJ_LAD)
        x, y, z = spec.xyz
        return spec, wd.FP32_METRIC64, wd.E6, p, np.minimum.reduce([y, 1 - y, z, 1 - z])
    if name == "chan-uw":
        spec = W.channel(1024, 513)
        p = wd.default_params(wd.UW, equation=wd.HJ_STD)
        y = spec.xyz[1]
        return spec, wd.FP64, wd.UW, p, np.minimum(y, 1.0 - y)
    if name.startswith("star1025"):
        spec = W.star(1025)
        p = wd.default_params(wd.E4, equation=wd.HJ_LAD, eps=0.15, alpha_f=0.45, lad_exp=4.0)
        sd = spec.meta["signed_distance"]
        return spec, wd.FP32_METRIC64, wd.E4, p, np.where(spec.mask == 1, spec.dval, sd)
    if name == "ell2048":
        spec = W.ellipse(1025, 2048, 2.0)
        p = wd.default_params(wd.C6, equation=wd.HJ_LAD)
        return spec, wd.FP32_METRIC64, wd.C6, p, 0.3 * W.random_field(spec, 1) + np.hypot(*spec.xyz)
    raise SystemExit(f"unknown case {name}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case")
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--timer", action="store_true")
    args = ap.parse_args()
    import torch

    from paper_2111_09859_gb300 import build, wd

    build.build()
    spec, prec, scheme, p, phi0 = build_case(args.case)
    g = wd.Grid(spec, prec, scheme)
    if args.case.endswith("-ls"):
        phi = g.as_field(spec.meta["signed_distance"])
        F = 0.3
        ls_dt = 0.5 * spec.meta["h"] / F

        def run(n):
            g.levelset(phi, F, ls_dt, n)
    else:
        phi = g.as_field(phi0)

        def run(n):
            g.steps(p, phi, n)
    run(args.warmup)
    torch.cuda.synchronize()
    if args.timer:
        g.profile(True)
    t = time.time()
    run(args.steps)
    torch.cuda.synchronize()
    dt = time.time() - t
    line = f"{args.case}: {spec.N} nodes, {args.steps} steps, {dt / max(args.steps, 1) * 1e3:.3f} ms/step"
    if args.timer:
        prof = g.profile_read()
        g.profile(False)
        line += " | " + ", ".join(f"{k} {v[0] / max(v[1], 1) * 1e3:.1f} us x{v[1]}" for k, v in prof.items() if v[1])
    print(line, flush=True)
    g.close()


if __name__ == "__main__":
    main()
