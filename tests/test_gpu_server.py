"""Request loop (wd_server_*): continuous batching of independent solves of the ellipse
stream.  A request gives the same result in the mix as alone (the same kernels, slices and
convergence checks; all reductions have a fixed order, so the results are bit-identical),
admission respects the device-memory cap, caller-owned grids run warm-started requests, a
grid re-used through the geometry reset equals a fresh one, and a served ellipse matches
the brute-force distance to points sampled on the ellipse."""
import numpy as np
import pytest

from paper_2111_09859_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SMALL = ((65, 128), (129, 256))


@pytest.fixture(scope="module")
def wd():
    import torch

    assert torch.cuda.is_available()
    from paper_2111_09859_gb300 import build, wd as _wd

    build.build()
    return _wd


def params(wd, **kw):
    kw.setdefault("tol_l2", 1e-6)
    kw.setdefault("max_iters", 8000)
    return wd.default_params(wd.C6, equation=wd.HJ_LAD, **kw)


def mix(n, seed=9859):
    return [W.ellipse(nr, nt, ar) for nr, nt, ar in W.ellipse_stream(n, seed, SMALL)]


def alone(wd, specs, p):
    out = []
    for sp in specs:
        g = wd.Grid(sp, wd.FP32_METRIC64, wd.C6)
        phi, st = g.solve(p)
        out.append((phi.cpu().numpy().copy(), st))
        g.close()
    return out


def test_alone_vs_mix(wd):
    specs = mix(10)
    p = params(wd)
    ref = alone(wd, specs, p)
    srv = wd.Server(max_active=16)
    try:
        sub = [srv.submit(sp, p) for sp in specs]
        for (t, out), (a, st) in zip(sub, ref):
            s, d, lat = srv.wait(t, 300)
            assert s == wd.OK and d["converged"] == 1
            assert d["iters"] == st["iters"] and d["poisson_iters"] == st["poisson_iters"]
            np.testing.assert_array_equal(out.cpu().numpy(), a)
            assert lat > 0
        info = srv.info()
        assert info["done"] == len(specs) and info["running"] == 0 and info["queued"] == 0
        assert info["peak_running"] > 1          # the requests really ran side by side
    finally:
        srv.close()


def test_staggered_arrivals_and_pool_reuse(wd):
    """Requests submitted while others run; same-shape requests re-use pooled grids."""
    import time

    specs = mix(8, seed=77)
    p = params(wd)
    ref = alone(wd, specs, p)
    srv = wd.Server(max_active=4, pool_per_shape=1)
    try:
        sub = []
        for sp in specs:
            sub.append(srv.submit(sp, p))
            time.sleep(0.01)
        for (t, out), (a, st) in zip(sub, ref):
            s, d, _ = srv.wait(t, 300)
            assert d["iters"] == st["iters"]
            np.testing.assert_array_equal(out.cpu().numpy(), a)
        assert srv.info()["peak_running"] <= 4
    finally:
        srv.close()


def test_admission_by_footprint(wd):
    specs = [W.ellipse(129, 256, ar) for ar in (1.5, 2.0, 3.0)]
    p = params(wd)
    ref = alone(wd, specs, p)
    fp = wd.footprint(specs[0], wd.FP32_METRIC64, wd.C6)
    srv = wd.Server(max_device_bytes=int(1.5 * fp), max_active=8)
    try:
        sub = [srv.submit(sp, p) for sp in specs]
        for (t, out), (a, st) in zip(sub, ref):
            s, d, _ = srv.wait(t, 300)
            np.testing.assert_array_equal(out.cpu().numpy(), a)
        assert srv.info()["peak_running"] == 1    # a second request never fitted the cap
    finally:
        srv.close()


def test_oversize_request_rejected(wd):
    sp = W.ellipse(129, 256, 2.0)
    fp = wd.footprint(sp, wd.FP32_METRIC64, wd.C6)
    srv = wd.Server(max_device_bytes=fp // 2)
    try:
        with pytest.raises(wd.WDError) as e:
            srv.submit(sp, params(wd))
        assert e.value.status == wd.ERR_OOM
    finally:
        srv.close()


def test_wait_timeout_then_result(wd):
    sp = W.ellipse(129, 256, 2.0)
    srv = wd.Server()
    try:
        t, out = srv.submit(sp, params(wd))
        s, d, lat = srv.wait(t, 0.0)
        assert s in (wd.ERR_TIMEOUT, wd.OK)
        s, d, lat = srv.wait(t, 300)
        assert s == wd.OK and d["converged"] == 1
        with pytest.raises(wd.WDError):
            srv.wait(t, 1.0)                     # the ticket was released
    finally:
        srv.close()


def test_caller_grid_warm_start(wd):
    """A session grid owned by the caller: the re-solve warm-started from the converged
    field stops at its first convergence check."""
    import torch

    sp = W.ellipse(65, 128, 2.0)
    p = params(wd)
    g = wd.Grid(sp, wd.FP32_METRIC64, wd.C6)
    phi, st = g.solve(p)
    srv = wd.Server()
    try:
        phi2 = phi.clone()
        t = srv.submit_grid(g, p, phi2, warm=True)
        s, d, _ = srv.wait(t, 300)
        assert s == wd.OK and d["converged"] == 1
        assert d["iters"] == p.check_every and d["poisson_iters"] == 0
        assert float((phi2 - phi).abs().max()) <= 2e-4 * float(phi.abs().max())
    finally:
        srv.close()
        g.close()
    torch.cuda.synchronize()


def test_reset_geometry_equals_fresh_grid(wd):
    a, b = W.ellipse(129, 256, 1.2), W.ellipse(129, 256, 3.7)
    p = params(wd)
    g = wd.Grid(a, wd.FP32_METRIC64, wd.C6)
    g.solve(p)
    g.reset_geometry(b)
    phi, st = g.solve(p)
    (ref, rst), = alone(wd, [b], p)
    assert st["iters"] == rst["iters"]
    np.testing.assert_array_equal(phi.cpu().numpy(), ref)
    g.close()


def test_served_ellipse_vs_sampled_distance(wd):
    """Ellipse pin: brute-force distance to 16384 points sampled on the ellipse (the
    sampling error is below half the largest chord, about 1e-4 here)."""
    from scipy.spatial import cKDTree

    sp = W.ellipse(129, 256, 2.5)
    srv = wd.Server()
    try:
        t, out = srv.submit(sp, params(wd))
        s, d, _ = srv.wait(t, 300)
    finally:
        srv.close()
    a, b = sp.meta["a"], sp.meta["b"]
    th = 2 * np.pi * np.arange(16384) / 16384
    tree = cKDTree(np.stack([a * np.cos(th), b * np.sin(th)], 1))
    exact, _ = tree.query(sp.xyz.T)
    err = np.abs(out.double().cpu().numpy() - exact)
    print("ellipse 129x256 AR 2.5: max err %.3e, rms %.3e" % (err.max(), np.sqrt((err ** 2).mean())))
    assert err.max() <= 2e-2 and np.sqrt((err ** 2).mean()) <= 5e-3
