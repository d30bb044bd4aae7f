#!/usr/bin/env python
"""Benchmark of the GB300 wall-distance solver (HJ / LAD pseudo-HJ, arXiv 2111.09859).

A step = one complete wall-distance solve of the workload: Poisson initial guess, HJ
pseudo-time marching (RK4, local time steps, filter, change norms) until the tolerance.
Workload (the cylinder case): O-grids around circular cylinders, 257 radial x 512 periodic
circumferential nodes, outer radius 10, radial ratio 1.03, compact C6 scheme, LAD
pseudo-HJ with the curvature correction, alpha_f = 0.495.  The timed form is FP32 state
with FP64 metrics, BATCH cylinders stacked in one grid object (wall radii 0.5 (1 + k/100)),
tolerance RMS(dphi) <= 1e-6 per cylinder; the FP64 plain form (one cylinder, tolerance
1e-10) is timed once beside it.  Metric: Mcell-iter/s = cylinders x nodes x pseudo steps /
device time.  Ranks solve their own batches (weak scaling, no collective on the data path);
rank 0 prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
    python bench.py --case NAME [--steps K] [--warmup W] [--timer]   (profiling cases)
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mcell-iter/s & time-to-converged d (FP32 batched vs FP64 plain), p99 latency"
UNIT = "Mcell-iter/s"


BATCH = 16


def workload_spec(batch=1):
    from paper_2111_09859_gb300 import workloads as W

    members = [W.cylinder(257, 512, 1.03, r_wall=0.5 * (1 + 0.01 * k)) for k in range(batch)]
    return W.stack(members) if batch > 1 else members[0]


def solve_params(wd, tol):
    return wd.default_params(wd.C6, equation=wd.HJ_LAD, curvature=1, alpha_f=0.495,
                             tol_l2=tol, max_iters=20000, check_every=10, poisson_max_iters=100)


class ClockSampler:
    """nvidia-smi SM clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def flush_l2(buf):
    buf.add_(1)      # writes 256 MB, more than the 129 MB L2


def peak_hbm():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# DRAM bytes (read + write) per launch of the dominant kernel class, from one ncu capture of
# the current kernel on this workload (profiles/k_l2_passes_cylinder_batch16.md): k_l2_y, the
# direction-1 pass of an RK stage, stage 2 (120.2 MB read + 14.2 MB written).
PROFILED_TRAFFIC = {"line1": 131.3e6}


def algorithmic_bytes(cls, nodes, nd, es, ms, curv, lad=True):
    """Algorithmic DRAM bytes of one launch of a kernel class of the line-resident 2-D step
    (every array a launch must touch read once, every output written once), averaged over
    the four RK stages where they differ:
      deriv  Y0: phi and s_1 in; D_1 and s_1 d4_1(phi) out
      line0  direction-0 pass: phi, D_1, s_1 d4_1, s_0 and the 4 metric arrays of U in; D_0,
             the direction-0 Laplacian part, the smoothed C|LAD| (and the direction-0
             curvature part) out
      line1  direction-1 pass: D_0, D_1, the 4 metric arrays, smoothed C|LAD|, Laplacian (and
             curvature) part, phi_s, phi^n, the Dirichlet flags in; stage 0 the two metric
             sums of the time step, stages 1-3 dt and acc; stages 0-2 s_1.  Out: the stage
             value; acc (stages 0-2), dt (stage 0), D_1 and s_1 d4_1 (stages 0-2)
      filter FX: the field in and out
      norm   FY: the field, phi^n and the flags in; phi^n out"""
    lad_f = 1 if lad else 0
    kap = 1 if curv else 0
    if cls == "deriv":
        return int(nodes * (es + lad_f * ms + es + lad_f * es))
    if cls == "line0":
        return int(nodes * ((2 + lad_f) * es + (lad_f + 4) * ms + (2 + lad_f + kap) * es))
    if cls == "line1":
        reads = (2 + 4 + lad_f + 1 + kap + 2) * es + 0.25 * 2 * ms + 0.75 * 2 * es + 0.75 * lad_f * ms
        writes = (1 + 0.75 + 0.25 + 0.75 * (1 + lad_f)) * es
        return int(nodes * (reads + writes + 1))
    if cls == "filter":
        return nodes * 2 * es
    if cls == "norm":
        return nodes * (3 * es + 1)
    return None


def reduce_over_ranks(ms, cells, world, device):
    """Replicas: the job's time is the slowest rank's, its work the sum of all ranks' (one
    all-reduce each; no collective touches the data path)."""
    if world == 1:
        return ms, cells
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    c = torch.tensor([float(cells)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), float(c.item())


def square_report(wd):
    """Unit square 65^2, four walls, E4, standard HJ, FP64, tolerance 1e-10: time to the
    converged distance (latency-bound: 4 225 nodes) and the error against min(x,1-x,y,1-y)."""
    import numpy as np
    import torch

    from paper_2111_09859_gb300 import workloads as W

    sp = W.square(65)
    g = wd.Grid(sp, wd.FP64, wd.E4)
    p = wd.default_params(wd.E4, equation=wd.HJ_STD, tol_l2=1e-10)
    g.solve(p)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    phi, st = g.solve(p)
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    x, y = sp.xyz
    err = float(np.abs(phi.cpu().numpy() - np.minimum.reduce([x, 1 - x, y, 1 - y])).max())
    g.close()
    return {"nodes": sp.N, "time_to_converged_s": round(ts, 4), "iters": st["iters"] + st["poisson_iters"],
            "max_err_vs_exact": float("%.3g" % err)}


def run_native(args, rank, world):
    import torch

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_2111_09859_gb300 import build as B

    B.build()
    from paper_2111_09859_gb300 import wd

    spec = workload_spec(BATCH)
    single = workload_spec(1)
    prec = wd.FP32_METRIC64
    tol = 1e-6
    p = solve_params(wd, tol)
    stream = torch.cuda.current_stream()
    g = wd.Grid(spec, prec, wd.C6, stream=stream)
    phi = g.empty()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    for _ in range(args.warmup):
        g.solve(p, phi)
    torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    g.profile(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total_ms, iters, piters = 0.0, 0, 0
    stats = []
    for _ in range(args.steps):
        flush_l2(flush)
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        _, st = g.solve(p, phi)
        ev1.record(stream)
        torch.cuda.synchronize()
        total_ms += ev0.elapsed_time(ev1)
        iters += st["iters"]
        piters += st["poisson_iters"]
        stats.append(st)
    prof = g.profile_read()
    g.profile(False)
    clk = clocks.stop()
    # the kernel timer adds gaps between launches: time the same steps again without it
    total_ms_plain = 0.0
    for _ in range(args.steps):
        flush_l2(flush)
        torch.cuda.synchronize()
        ev0.record(stream)
        g.solve(p, phi)
        ev1.record(stream)
        torch.cuda.synchronize()
        total_ms_plain += ev0.elapsed_time(ev1)
    nodes = spec.N
    ms, cell_iters = reduce_over_ranks(total_ms_plain, nodes * (iters + piters), world, "cuda")
    value = cell_iters / (ms * 1e-3) / 1e6

    # accuracy of the timed result against the FP64 oracle (the stored oracle solutions of the
    # 16 cylinders, tests/golden, written by the oracle alone) and the exact r - r_wall
    import numpy as np

    n1 = single.N
    rw = np.repeat([0.5 * (1 + 0.01 * k) for k in range(BATCH)], n1)
    exact = np.hypot(*spec.xyz) - rw
    phi_np = phi.double().cpu().numpy()
    err32 = float(np.abs(phi_np - exact).max())
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "cylinder257x512_c6_lad_curv.json")))["members"]
    d_oracle = np.concatenate([np.repeat(np.asarray(m["d"]), 512) for m in gold[:BATCH]])
    err32_oracle = float(np.abs(phi_np - d_oracle).max())

    # FP64 plain form on one cylinder (r_wall 0.5): time-to-converged at tolerance 1e-10
    g64 = wd.Grid(single, wd.FP64, wd.C6, stream=stream)
    phi64 = g64.empty()
    p64 = solve_params(wd, 1e-10)
    g64.solve(p64, phi64)
    torch.cuda.synchronize()
    flush_l2(flush)
    ev0.record(stream)
    _, st64 = g64.solve(p64, phi64)
    ev1.record(stream)
    torch.cuda.synchronize()
    t64 = ev0.elapsed_time(ev1) * 1e-3
    err64 = float(np.abs(phi64.cpu().numpy() - exact[:n1]).max())
    err64_oracle = float(np.abs(phi64.cpu().numpy() - d_oracle[:n1]).max())
    diff = float(np.abs(phi64.cpu().numpy() - phi_np[:n1]).max())
    del g64

    # end to end through the public API with host buffers: grid creation from host
    # coordinates (H2D), solve, result copied to pinned host memory (D2H)
    host_phi = torch.empty(nodes, dtype=torch.float32).pin_memory()   # whole batch
    e2e_ms = 0.0
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ge = wd.Grid(spec, prec, wd.C6, stream=stream)
        ge.solve(p, host_phi)
        ge.close()
        torch.cuda.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
    e2e_value = cell_iters / (e2e_ms * 1e-3) / 1e6 if e2e_ms > 0 else None

    # roofline of the dominant kernel class
    es, msz = 4, 4      # FP32 state, metrics used in FP32 (computed in FP64)
    best = max((k for k in prof if prof[k][1] > 0), key=lambda k: prof[k][0])
    kms, kn = prof[best]
    ab = algorithmic_bytes(best, nodes, spec.ndim, es, msz, True)
    peak, src = peak_hbm()
    roof = None
    if ab is not None and kn > 0:
        ach = ab / (kms / kn * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": best, "achieved": round(ach, 1), "peak": peak,
                "peak_source": src + " (of " + src + ")", "unit": "GB/s", "frac": round(ach / peak, 4),
                "traffic": PROFILED_TRAFFIC.get(best), "algorithmic_bytes_per_launch": ab,
                "avg_launch_us": round(kms / kn * 1e3, 3),
                "frac_of_nominal_7900": round(ach / 7900.0, 4),
                "share_of_timed": round(kms / max(1e-9, sum(v[0] for v in prof.values())), 3)}
    # launches of the timed solves: the profiled solves run the batch as one part; the timed
    # ones split the line-resident passes into the autotuned number of parts
    parts = max(1, g.tuning()[2])
    split = ("deriv", "line0", "line1", "filter", "norm")
    launches = sum(v[1] * (parts if k in split else 1) for k, v in prof.items())

    out = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (metric Jacobians computed in f64)",
        "data": "synthetic",
        "config": {"workload": f"{BATCH} stacked cylinder O-grids 257x512 (r_wall 0.5(1+k/100), "
                               "r_out 10, ratio 1.03), C6 + LAD + curvature, alpha_f 0.495, "
                               "FP32 state and loop, metric Jacobians computed in FP64, tol RMS 1e-6 per cylinder, Poisson 100",
                   "batch": BATCH, "nodes": nodes, "pseudo_steps_per_solve": (iters + piters) / args.steps,
                   "l2_between_steps": "flushed (256 MB write)",
                   "parallelism": f"replicas x{world}", "batch_parts": parts},
        "roofline": roof,
        "kernel_ms": {k: round(v[0], 3) for k, v in prof.items()},
        "gpu_launches": int(launches),
        "clocks": clk,
        "e2e": {"value": round(e2e_value, 2) if e2e_value else None, "unit": UNIT,
                "h2d_bytes_per_step": int(spec.xyz.nbytes), "d2h_bytes_per_step": int(nodes * 4),
                "what": "wd_create_grid from host coordinates + wd_solve into pinned host memory + destroy"},
    }
    tail = {
        "time_to_converged_s": {"fp32_batch_of_%d" % BATCH: round(ms / args.steps * 1e-3, 4),
                                "fp32_batched_per_cylinder": round(ms / args.steps * 1e-3 / BATCH, 4),
                                "fp64_plain_one_cylinder": round(t64, 4), "fp64_iters": st64["iters"],
                                "fp32_iters": round((iters + piters) / args.steps, 1)},
        "accuracy": {"max_abs_vs_fp64_oracle": {"fp32_batch": float("%.3g" % err32_oracle),
                                                "fp64_plain": float("%.3g" % err64_oracle),
                                                "bar": {"fp32": 2e-4, "fp64": 1e-6}},
                     "max_abs_vs_exact": {"fp32_batch": float("%.3g" % err32), "fp64_plain": float("%.3g" % err64)},
                     "max_fp32_minus_fp64": float("%.3g" % diff),
                     "oracle": "FP64 CPU oracle solved to RMS 1e-12 (tests/golden/cylinder257x512_c6_lad_curv.json)"},
    }
    if rank == 0:
        if not args.no_extras:
            out["serving"] = serving_report(wd, args.full)
            out["star_burn"] = star_report(wd, args.full)
            d = duct_report(wd)
            peak_hbm_gbs = peak_hbm()[0]
            d["frac_of_112B_roofline"] = round(d["mcell_iter_s"] * 1e6 * 112 / (peak_hbm_gbs * 1e9), 4)
            out["duct"] = d
            out["square65"] = square_report(wd)
            out["upwind_vs_central"] = upwind_report(wd)
            out["levelset_regression"] = levelset_report(wd)
        out["cpu_baseline"] = cpu_baseline()
        out.update(tail)
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def serving_report(wd, full):
    """Ellipse stream through the request loop (wd_server_*): the closed-loop saturation rate
    of the request mix, then Poisson arrivals at 0.7 x that rate; p50 / p99 latency from
    submission to completion, throughput.  Default: 48 requests (full: 1000)."""
    import numpy as np
    import torch

    from paper_2111_09859_gb300 import workloads as W

    n = 1000 if full else 48
    shapes = W.ellipse_stream(n)
    specs = [W.ellipse(*sh) for sh in shapes]
    p = wd.default_params(wd.C6, equation=wd.HJ_LAD, tol_l2=1e-6, max_iters=20000)

    def run(arrivals):
        srv = wd.Server(max_active=32)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tickets = []
        for k, sp in enumerate(specs):
            if arrivals is not None:
                dt = arrivals[k] - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
            tickets.append((srv.submit(sp, p)[0], sp))
        lat, cells = [], 0
        for t, sp in tickets:
            s_, st, l = srv.wait(t, 3600)
            lat.append(l)
            cells += sp.N * (st["iters"] + st["poisson_iters"])
        span = time.perf_counter() - t0
        info = srv.info()
        srv.close()
        return span, np.array(lat), cells, info

    span, lat, cells, info = run(None)
    rate_sat = n / span
    rate = 0.7 * rate_sat
    arr = W.poisson_arrivals(n, rate, seed=2111)
    span2, lat2, cells2, info2 = run(arr)
    return {"requests": n, "sizes": "ellipse 65x128..1025x2048, AR U[1,4]", "fp": "FP32 (FP64 metrics), C6+LAD, tol 1e-6",
            "sat_req_s": round(rate_sat, 3), "rate_req_s": round(rate, 3),
            "p50_s": round(float(np.percentile(lat2, 50)), 3), "p99_s": round(float(np.percentile(lat2, 99)), 3),
            "req_s": round(n / span2, 3), "mcell_iter_s": round(cells2 / span2 / 1e6, 1),
            "peak_concurrent": info2["peak_running"]}


def star_report(wd, full):
    """Receding star grain: 1025^2 box, E4 + LAD (Delta x^4 scale), eps 0.15, alpha_f 0.45,
    FP32; the surface recedes by 0.002 per step, each step a warm re-solve on a session grid
    through the request loop, 200 steps (the configuration's full burn).  The burning perimeter of the
    computed zero level against the marching-squares length of the exact offset field."""
    import numpy as np
    import torch

    from paper_2111_09859_gb300 import workloads as W

    steps = 200
    sp = W.star(1025)
    h, sd = sp.meta["h"], sp.meta["signed_distance"]
    g = wd.Grid(sp, wd.FP32_METRIC64, wd.E4)
    p = wd.default_params(wd.E4, equation=wd.HJ_LAD, eps=0.15, alpha_f=0.45, lad_exp=4.0, tol_l2=1e-7,
                          max_iters=40000)
    srv = wd.Server()
    phi = g.empty()
    t0 = time.perf_counter()
    _, st0, lat0 = srv.wait(srv.submit_grid(g, p, phi), 3600)
    lats, its = [], []
    for k in range(1, steps + 1):
        m, d = g.recede(phi, 0.002, -3 * h)
        _, st, lat = srv.wait(srv.submit_grid(g, p, phi, warm=True, mask=m, dval=d), 3600)
        lats.append(lat)
        its.append(st["iters"])
    torch.cuda.synchronize()
    total = time.perf_counter() - t0
    ex = sd - steps * 0.002
    L = g.level_length(phi, 0.0)
    Lx = g.level_length(g.as_field(ex), 0.0)
    a = phi.double().cpu().numpy()
    sel = (m.cpu().numpy() == 0) & (ex < 0.3)
    err = float(np.abs(a - ex)[sel].max())
    srv.close()
    g.close()
    return {"steps": steps, "grid": "1025^2", "first_solve_s": round(lat0, 3), "first_iters": st0["iters"],
            "step_p50_s": round(float(np.percentile(lats, 50)), 4), "step_p99_s": round(float(np.percentile(lats, 99)), 4),
            "warm_iters_median": int(np.median(its)), "total_s": round(total, 2),
            "perimeter_rel_err": round((L - Lx) / Lx, 5), "max_err_near_port_h": round(err / h, 3)}


def _ms_per_steps(wd, g, p, phi, n):
    import torch

    g.steps(p, phi, 3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    g.steps(p, phi, n)
    ev1.record()
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1)


def upwind_report(wd):
    """The baseline upwind scheme (UW, Sec. 3.2.1) against the central schemes, as in the
    paper's timing comparison (time per 100 pseudo steps on the channel): channel 1024 x 513
    nodes, FP64.  For UW with the standard HJ, E2 and E4 with the standard HJ, E4 and C6 with
    LAD: ms per 100 pseudo steps (from the exact distance min(y, 1 - y)) on the generic
    per-operator path (the only path of UW) and on the scheme's own fast path."""
    import os

    import numpy as np

    from paper_2111_09859_gb300 import workloads as W

    sp = W.channel(1024, 513)
    y = sp.xyz[1]
    ex = np.minimum(y, 1.0 - y)
    cases = [("UW_std", wd.UW, wd.HJ_STD), ("E2_std", wd.E2, wd.HJ_STD), ("E4_std", wd.E4, wd.HJ_STD),
             ("E4_lad", wd.E4, wd.HJ_LAD), ("C6_lad", wd.C6, wd.HJ_LAD)]
    out = {"grid": "channel 1024 x 513 (periodic x, walls y = 0, 1), FP64"}
    for name, sch, eq in cases:
        p = wd.default_params(sch, equation=eq)
        row = {}
        for path in ("generic", "fast"):
            if path == "fast" and sch == wd.UW:
                continue
            if path == "generic":
                os.environ["WD_FORCE_GENERIC"] = "1"
            try:
                g = wd.Grid(sp, wd.FP64, sch)
            finally:
                os.environ.pop("WD_FORCE_GENERIC", None)
            phi = g.as_field(ex)
            row["ms_per_100_steps_" + path] = round(_ms_per_steps(wd, g, p, phi, 100), 3)
            g.close()
        out[name] = row
    uw = out["UW_std"]["ms_per_100_steps_generic"]
    compact = {"grid": "channel 1024x513 FP64", "ms_per_100": {}}
    for k in ("UW_std", "E2_std", "E4_std", "E4_lad", "C6_lad"):
        compact["ms_per_100"][k] = [out[k]["ms_per_100_steps_generic"], out[k].get("ms_per_100_steps_fast")]
    compact["uw_over_fast"] = {k: round(uw / out[k]["ms_per_100_steps_fast"], 2)
                               for k in ("E2_std", "E4_std", "E4_lad", "C6_lad")}
    return compact


def levelset_report(wd):
    """Grain regression (Sec. 5.5): the 1025^2 star, FP32.  The HJ-LAD field of the star (its
    first solve) starts the level-set march d(phi)/dt + F |grad phi| = 0 at F = 0.3 to t = 1
    (RK4, dt = 0.5 h / F, upwind slopes of Eqs. UW3-UW5).  Reports ms per step, node updates
    per second, the stage kernel's algorithmic HBM bytes and its fraction of the measured
    copy bandwidth, and the burning perimeter at t = 0.25 .. 1 against the exact front
    {d_0 = F t} (marching squares on the exact field); the same march started from the exact
    d_0 separates the march's own error from the initialization's."""
    import numpy as np
    import torch

    from paper_2111_09859_gb300 import workloads as W

    sp = W.star(1025)
    h, d0 = sp.meta["h"], sp.meta["signed_distance"]
    g = wd.Grid(sp, wd.FP32_METRIC64, wd.E4)
    p = wd.default_params(wd.E4, equation=wd.HJ_LAD, eps=0.15, alpha_f=0.45, lad_exp=4.0, tol_l2=1e-6,
                          max_iters=20000)
    phi, st = g.solve(p)
    F, T, parts = 0.3, 1.0, 4
    ns_ = int(np.ceil(T / (0.5 * h / F) / parts)) * parts
    exm = g.as_field(d0)
    g.levelset(exm, F, T / ns_, ns_)
    L_exact_start = g.level_length(exm, 0.0)
    ns = int(np.ceil(T / (0.5 * h / F) / parts)) * parts
    dt = T / ns
    g.levelset(phi.clone(), F, dt, 4)                        # warm-up: graph capture
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(parts + 1)]
    per = []
    torch.cuda.synchronize()
    ms = 0.0
    for k in range(parts):
        ev[k].record()
        g.levelset(phi, F, dt, ns // parts)
        ev[k + 1].record()
        torch.cuda.synchronize()
        ms += ev[k].elapsed_time(ev[k + 1])
        t = (k + 1) * T / parts
        L = g.level_length(phi, 0.0)
        Lx = g.level_length(g.as_field(d0), F * t)
        per.append({"t": t, "perimeter": round(L, 5), "exact": round(Lx, 5), "rel_err": round(L / Lx - 1, 5)})
    nodes = sp.N
    ms_step = ms / ns
    # per stage and node: src, phin and dst once, acc read-modify-write on two of the four
    # stages (4.5 floats); the uniform grid's metrics are constants
    bytes_stage = nodes * 4 * 4.5
    stage_us = ms_step * 1e3 / 4
    g.close()
    return {"grid": "star 1025^2", "F": F, "t_end": T, "steps": ns, "ms_per_step": round(ms_step, 4),
            "stage_us": round(stage_us, 2), "stage_gbs_from_l2": round(bytes_stage / (stage_us * 1e-6) / 1e9, 1),
            "perimeter_rel_err_t_end": per[-1]["rel_err"],
            "perimeter_rel_err_from_exact_d0": round(L_exact_start / per[-1]["exact"] - 1, 5)}


def duct_report(wd):
    """Square duct 256^3, E6 + LAD, FP32: Mcell-iter/s of the pseudo steps and the solve."""
    import numpy as np
    import torch

    from paper_2111_09859_gb300 import workloads as W

    sp = W.duct(256)
    g = wd.Grid(sp, wd.FP32_METRIC64, wd.E6)
    p = wd.default_params(wd.E6, equation=wd.HJ_LAD, tol_l2=1e-6, max_iters=5000)
    x, y, z = sp.xyz
    ex = np.minimum.reduce([y, 1 - y, z, 1 - z])
    phi = g.as_field(ex)
    g.steps(p, phi, 3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    g.steps(p, phi, 20)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / 20
    # per-pass device time (the library's CUDA-event timer around each launch) against the
    # pass's algorithmic bytes per node (every array it must touch read once, every output
    # written once; stage: LAD, averaged over the four RK stages)
    g.profile(True)
    g.steps(p, phi, 4)
    prof = g.profile_read()
    g.profile(False)
    peak = peak_hbm()[0]
    per_node = {"deriv": ("U: phi in; U_0..2 and C|LAD| out", 20),
                "gauss": ("Gaussian of C|LAD| along x and y", 8),
                "point": ("RK stage: U_0..2, G, phi, phi^n, flags, dt and acc in; stage, acc (dt) out", 39),
                "filter": ("filters along x and y (one timed scope): field in and out, twice", 16),
                "norm": ("filter along z + commit: field, phi^n, flags in; phi^n out", 13)}
    kernels = {}
    for cls, (what, b) in per_node.items():
        tot, n = prof.get(cls, (0.0, 0))
        if not n:
            continue
        launches = n   # timed scopes
        us = tot / launches * 1e3
        gbs = b * sp.N / (us * 1e-6) / 1e9
        kernels[cls] = {"what": what, "us_per_launch": round(us, 1), "launches_per_step": round(launches / 4, 2),
                        "bytes_per_node": b, "GBps": round(gbs, 1), "frac_of_measured_hbm": round(gbs / peak, 3)}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out, st = g.solve(p)
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    err = float(np.abs(out.double().cpu().numpy() - ex).max())
    g.close()
    return {"nodes": sp.N, "ms_per_step": round(ms, 3), "mcell_iter_s": round(sp.N / (ms * 1e-3) / 1e6, 1),
            "solve_s": round(ts, 3), "solve_iters": st["iters"] + st["poisson_iters"],
            "max_err_vs_exact": float("%.3g" % err), "kernels": kernels}


def cpu_baseline(n_steps=12):
    """The FP64 oracle (one thread) on a bounded sample of the same workload: a Poisson
    step and n HJ pseudo steps of the full cylinder grid from its Poisson guess."""
    import numpy as np

    import oracle as O

    spec = workload_spec(1)
    og = O.Grid(spec.shape, spec.xyz, spec.bc_lo, spec.bc_hi, scheme=O.C6, period=spec.period)
    kw = dict(equation=O.HJ_LAD, scheme=O.C6, curvature=1, alpha_f=0.495, cfl=0.6)
    phi0 = og.apply_bc(np.hypot(*spec.xyz) - 0.5)
    t0 = time.perf_counter()
    og.hj_steps(phi0, n_steps, **kw)
    dt = time.perf_counter() - t0
    return {"value": round(spec.N * n_steps / dt / 1e6, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n_steps} HJ pseudo steps of the 257x512 cylinder grid (FP64, one thread)",
            "seconds": round(dt, 2)}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import numpy as np

    import oracle as O

    O.build()
    spec = workload_spec(1)
    og = O.Grid(spec.shape, spec.xyz, spec.bc_lo, spec.bc_hi, scheme=O.C6, period=spec.period)
    kw = dict(equation=O.HJ_LAD, scheme=O.C6, curvature=1, alpha_f=0.495, cfl=0.6)
    phi = og.apply_bc(np.hypot(*spec.xyz) - 0.5)
    n = 4
    for _ in range(args.warmup):
        phi, _ = og.hj_steps(phi, 1, **kw)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        phi, _ = og.hj_steps(phi, n, **kw)
    dt = time.perf_counter() - t0
    v = spec.N * n * args.steps / dt / 1e6
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "cylinder O-grid 257x512, C6 + LAD + curvature, alpha_f 0.495",
                   "sample": f"each step = {n} HJ pseudo steps of the full grid"},
        "cpu_baseline": {"value": round(v, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{n} HJ pseudo steps per step, FP64, one thread"},
        "e2e": {"value": round(v, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


CASES = """
  cylK      K stacked cylinder O-grids 257 x 512 (cyl16: the headline batch), C6 + LAD +
            curvature, alpha_f 0.495, FP32 state (metrics computed in FP64)
  cylK-64   the same K cylinders in FP64
  duct256   square duct 256^3, E6 + LAD, FP32
  duct128   square duct 128^3 (a small case of the same kernels)
  star1025  star port 1025^2, E4 + LAD, FP32
  star1025-ls  the same star, level-set steps (F = 0.3, dt = 0.5 h / F) instead of pseudo
            steps, from the exact signed distance
  chan-uw   channel 1024 x 513, baseline upwind scheme, standard HJ, FP64 (generic path)
  ell2048   one ellipse O-grid 1025 x 2048, C6 + LAD, FP32"""


def build_case(name):
    """(spec, precision, scheme, params, initial field) of a --case workload: the exact
    distance where one exists, a smooth random field otherwise, so that the steps run in the
    converged regime."""
    import numpy as np

    from paper_2111_09859_gb300 import workloads as W, wd

    if name.startswith("cyl"):
        nb = int(name[3:].split("-")[0])
        members = [W.cylinder(257, 512, 1.03, r_wall=0.5 * (1 + 0.01 * k)) for k in range(nb)]
        spec = W.stack(members) if nb > 1 else members[0]
        prec = wd.FP64 if name.endswith("-64") else wd.FP32_METRIC64
        p = wd.default_params(wd.C6, equation=wd.HJ_LAD, curvature=1, alpha_f=0.495)
        x, y = spec.xyz
        r0 = np.repeat([0.5 * (1 + 0.01 * k) for k in range(nb)], 257 * 512)
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



def run_case(args):
    """--case NAME: W pseudo steps (or level-set steps), then K timed ones, of a named
    workload; one line per run.  For profilers (ncu) and quick per-class kernel timings
    (--timer: the library's CUDA-event timer around every launch).  Not a bench line."""
    import torch

    from paper_2111_09859_gb300 import build as B

    B.build()
    from paper_2111_09859_gb300 import wd

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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--full", action="store_true", help="serving: 1000 requests; star: 200 steps")
    ap.add_argument("--no-extras", action="store_true", help="only the headline cylinder workload")
    ap.add_argument("--case", default=None, help="run pseudo steps of a named workload (profiling):" + CASES)
    ap.add_argument("--timer", action="store_true", help="--case: per-class kernel timer")
    args = ap.parse_args()
    if args.case:
        run_case(args)
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_native(args, rank, world)


if __name__ == "__main__":
    main()
