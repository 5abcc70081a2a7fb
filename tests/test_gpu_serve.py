"""Serving (continuous batching of flow requests): results in the mix equal
the results alone, match the single-flow mixed path and the oracle, and the
scheduler admits by HBM budget, rejects, cancels and reports latency."""
import math
import time

import numpy as np
import pytest

import ffrg_inputs as fi
import oracle
from gpu_common import gpu_context

pytestmark = pytest.mark.gpu

ENDPOINT_TOL = 1e-8     # served mixed endpoints vs the oracle's truth, element-wise
SERVE_RTOL = 2e-11      # step tolerance at which the served flows meet it (also the bench's)


def _stream(n, seed=11):
    return fi.serving_stream(seed=seed, n_requests=n, ext_range=(9, 27), rad_range=(8, 24), ang_range=(4, 12),
                             pts_range=(16, 40), t_max=0.5, n_cap=6)


def _submit(ctx, wl, rtol=1e-10, atol=1e-13):
    t1 = math.log(wl.Lambda / wl.k_end)
    return ctx.serve_submit(wl.problem, wl.tables, wl.y0, wl.Lambda, t1, rtol=rtol, atol=atol)


def _wait(ctx, tickets, sizes, timeout=120.0):
    import paper_2412_13043_gb300 as ffrg
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for tk, n in zip(tickets, sizes):
            if tk in out:
                continue
            st, res, stats, lat = ctx.serve_poll(tk, n)
            if st != ffrg.EPENDING:
                out[tk] = (st, res, stats, lat)
        assert time.time() - t0 < timeout, "serving did not finish"
        time.sleep(0.002)
    return out


def test_mix_equals_alone_and_single_flow_path():
    import paper_2412_13043_gb300 as ffrg
    reqs = _stream(12)
    # alone: one request at a time through its own server
    alone = []
    for rq in reqs:
        ctx = gpu_context()
        ctx.serve_start(max_slots=1)
        tk = _submit(ctx, rq.workload)
        alone.append(_wait(ctx, [tk], [rq.workload.problem.n_ext()])[tk])
        assert ctx.serve_stop() == ffrg.OK
        ctx.close()
    # in the mix: all at once, fewer slots than requests so that some queue
    ctx = gpu_context()
    ctx.serve_start(max_slots=5)
    tks = [_submit(ctx, rq.workload) for rq in reqs]
    mix = _wait(ctx, tks, [rq.workload.problem.n_ext() for rq in reqs])
    stats = ctx.serve_stats()
    assert ctx.serve_stop() == ffrg.OK
    assert stats["completed"] == len(reqs) and stats["peak_resident"] <= 5
    for rq, tk, al in zip(reqs, tks, alone):
        st, res, fst, lat = mix[tk]
        assert st == ffrg.OK and al[0] == ffrg.OK
        assert np.array_equal(res, al[1]), rq.rid          # bitwise, independent of batch composition
        assert fst["steps"] == al[2]["steps"] and lat > 0
    # single-flow mixed path (ffrg_flow) on two of them
    for rq, tk in list(zip(reqs, tks))[:2]:
        wl = rq.workload
        import torch
        tabs = ctx.tables(wl.problem, wl.tables)
        y = torch.tensor(wl.y0, dtype=torch.float64, device="cuda")
        ctx.flow(wl.problem, tabs, y, wl.Lambda, math.log(wl.Lambda / wl.k_end), precision=ffrg.MIXED,
                 rtol=1e-10, atol=1e-13)
        tabs.free()
        ref = y.cpu().numpy()
        res = mix[tk][1]
        assert np.max(np.abs(res - ref) / np.abs(ref)) < 1e-9
    ctx.close()


def test_served_results_match_oracle():
    import paper_2412_13043_gb300 as ffrg
    reqs = _stream(4, seed=17)
    ctx = gpu_context()
    ctx.serve_start(max_slots=4)
    tks = [_submit(ctx, rq.workload, rtol=SERVE_RTOL) for rq in reqs]
    res = _wait(ctx, tks, [rq.workload.problem.n_ext() for rq in reqs])
    ctx.serve_stop()
    ctx.close()
    for rq, tk in zip(reqs, tks):
        wl = rq.workload
        truth, _ = oracle.flow(wl.problem, wl.tables, wl.y0, wl.Lambda, math.log(wl.Lambda / wl.k_end),
                               rtol=1e-13, atol=1e-16)
        st, y, _, _ = res[tk]
        assert st == ffrg.OK
        assert np.max(np.abs(y - truth) / np.abs(truth)) < ENDPOINT_TOL, rq.rid


def _bench_sized_requests():
    """Requests of the serving mix that reach its largest sizes, one dimension
    at a time (the oracle's truth of one request with all of them at once
    would take minutes): d=3 with 256 external points and 128 radial nodes,
    d=3 with 64 angular nodes, finite T with N = 64 and 256-point tables (the
    FP64 stack exceeds shared memory), finite T with 252 external points;
    masses across w = m^2/k^2 in [-0.2, 1]."""
    out = []
    wl = fi.make_d3(seed=81, n_pts=200, n_ext_p=256, n_rad=128, n_ang=16, m2_over_k2=-0.15)
    out.append(wl)
    out.append(fi.make_d3(seed=82, n_pts=64, n_ext_p=48, n_rad=32, n_ang=64, m2_over_k2=0.9))
    for seed, N, T, pts, n_p, nr, na, w in ((83, 64, 0.02, 256, 3, 32, 16, -0.1),
                                            (84, 2, 0.8, 64, 28, 32, 16, 0.3)):
        wl = fi.make_finite_t(seed=seed, N=N, T=T, n_pts=pts, n_ext_p=n_p, n_rad=nr, n_ang=na)
        wl.problem.m2_over_k2 = w
        wl.y0 = wl.y0 - 0.5 * wl.Lambda ** 2 + w * wl.Lambda ** 2
        out.append(wl)
    return out


def test_served_endpoints_within_1e8_of_oracle_truth_at_bench_sizes():
    """The served mixed-precision flows (FP32 integrand) reach the FP64
    endpoint accuracy: within 1e-8 of the oracle's rtol-1e-12 truth on every
    component, at the serving mix's largest sizes."""
    import paper_2412_13043_gb300 as ffrg
    wls = _bench_sized_requests()
    ctx = gpu_context()
    ctx.serve_start(max_slots=8, hbm_budget_bytes=1 << 30)
    tks = [_submit(ctx, wl, rtol=SERVE_RTOL) for wl in wls]
    res = _wait(ctx, tks, [wl.problem.n_ext() for wl in wls], timeout=300.0)
    ctx.serve_stop()
    ctx.close()
    for wl, tk in zip(wls, tks):
        truth, _ = oracle.flow(wl.problem, wl.tables, wl.y0, wl.Lambda, math.log(wl.Lambda / wl.k_end),
                               rtol=1e-12, atol=1e-16)
        st, y, _, _ = res[tk]
        assert st == ffrg.OK
        err = float(np.max(np.abs(y - truth) / np.abs(truth)))
        print(f"model {wl.problem.model} n_ext {wl.problem.n_ext()} N {wl.problem.n_matsubara}: {err:.2e}")
        assert err < ENDPOINT_TOL, (wl.problem.model, err)


def test_admission_by_hbm_budget_and_rejection():
    import paper_2412_13043_gb300 as ffrg
    reqs = _stream(6, seed=23)
    ctx = gpu_context()
    # budget for about two of these requests at a time
    ctx.serve_start(max_slots=8, max_queue=16, hbm_budget_bytes=150_000)
    sizes = [rq.workload.problem.n_ext() for rq in reqs]
    tks = []
    for rq in reqs:
        try:
            tks.append(_submit(ctx, rq.workload))
        except ffrg.FfrgError as e:
            assert e.code == ffrg.ENOMEM            # larger than the whole budget
            tks.append(None)
    live = [(t, n) for t, n in zip(tks, sizes) if t is not None]
    out = _wait(ctx, [t for t, _ in live], [n for _, n in live])
    stats = ctx.serve_stats()
    ctx.serve_stop()
    assert all(v[0] == ffrg.OK for v in out.values())
    assert stats["completed"] == len(live) and stats["peak_resident"] <= 8
    assert stats["hbm_in_use"] <= 150_000
    # queue limit
    ctx.serve_start(max_slots=1, max_queue=1)
    wl = reqs[0].workload
    first = _submit(ctx, wl)
    with pytest.raises(ffrg.FfrgError) as ei:
        for _ in range(50):
            _submit(ctx, wl)
    assert ei.value.code == ffrg.EBUSY
    ctx.serve_stop()
    assert ctx.serve_poll(first, 1)[0] == ffrg.EINVAL      # the server is gone
    ctx.close()


def test_cancel_and_unknown_ticket():
    import paper_2412_13043_gb300 as ffrg
    reqs = _stream(3, seed=29)
    ctx = gpu_context()
    ctx.serve_start(max_slots=1)
    tks = [_submit(ctx, rq.workload, rtol=1e-12) for rq in reqs]
    assert ctx.serve_cancel(tks[2]) == ffrg.OK            # still queued
    out = _wait(ctx, tks, [rq.workload.problem.n_ext() for rq in reqs])
    assert out[tks[2]][0] == ffrg.ECANCELED
    assert out[tks[0]][0] == ffrg.OK
    assert ctx.serve_poll(12345678, 1)[0] == ffrg.ENOTFOUND
    assert ctx.serve_cancel(12345678) == ffrg.ENOTFOUND
    ctx.serve_stop()
    ctx.close()


def test_cancel_resident_flow_and_reuse_its_slot():
    """A flow cancelled while resident (ticks in flight behind it) finishes
    with FFRG_ECANCELED; its slot cools down and then serves the next requests,
    whose results equal their results alone, bitwise."""
    import paper_2412_13043_gb300 as ffrg
    reqs = _stream(4, seed=41)
    alone = []
    for rq in reqs:
        ctx = gpu_context()
        ctx.serve_start(max_slots=1)
        tk = _submit(ctx, rq.workload)
        alone.append(_wait(ctx, [tk], [rq.workload.problem.n_ext()])[tk])
        assert ctx.serve_stop() == ffrg.OK
        ctx.close()
    long_wl = fi.make_d3(seed=5, n_pts=32, n_ext_p=16, n_rad=24, n_ang=12)
    ctx = gpu_context()
    ctx.serve_start(max_slots=1)
    long_tk = _submit(ctx, long_wl, rtol=1e-12, atol=1e-15)
    t0 = time.time()
    while ctx.serve_stats()["ticks"] < 2:   # admitted and stepping
        assert time.time() - t0 < 60.0
        time.sleep(0.0005)
    assert ctx.serve_cancel(long_tk) == ffrg.OK
    tks = [_submit(ctx, rq.workload) for rq in reqs]
    out = _wait(ctx, [long_tk] + tks, [long_wl.problem.n_ext()] + [rq.workload.problem.n_ext() for rq in reqs])
    stats = ctx.serve_stats()
    assert ctx.serve_stop() == ffrg.OK
    ctx.close()
    assert out[long_tk][0] == ffrg.ECANCELED
    for a, tk in zip(alone, tks):
        st, y, fs, _ = out[tk]
        assert st == ffrg.OK and a[0] == ffrg.OK
        assert np.array_equal(y, a[1])
        assert fs["steps"] == a[2]["steps"]
    assert stats["cancelled"] == 1 and stats["completed"] == len(reqs)


def test_served_fermionic_flows_match_oracle():
    """Finite-T flows with a fermionic loop through the server."""
    import paper_2412_13043_gb300 as ffrg
    wls = [fi.make_finite_t(seed=70 + i, N=n, T=t, n_pts=24, n_ext_p=3, n_ext_m=3, n_rad=12, n_ang=6,
                            fermionic=True) for i, (n, t) in enumerate(((2, 0.3), (4, 0.15), (1, 0.5)))]
    ctx = gpu_context()
    ctx.serve_start(max_slots=3)
    tks = [_submit(ctx, wl, rtol=SERVE_RTOL) for wl in wls]
    res = _wait(ctx, tks, [wl.problem.n_ext() for wl in wls])
    ctx.serve_stop()
    ctx.close()
    for wl, tk in zip(wls, tks):
        truth, _ = oracle.flow(wl.problem, wl.tables, wl.y0, wl.Lambda, math.log(wl.Lambda / wl.k_end),
                               rtol=1e-13, atol=1e-16)
        st, y, _, _ = res[tk]
        assert st == ffrg.OK
        assert np.max(np.abs(y - truth) / np.abs(truth)) < ENDPOINT_TOL
