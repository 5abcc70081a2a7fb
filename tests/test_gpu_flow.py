"""GPU parity of ffrg_flow (device Dormand-Prince 5(4), t_+ = ln(Lambda/k),
d_t y = -Flow; Sec. 2.1, Sec. 5.2.2 Eqs. assVar/flowVar, Sec. 5.2.1 RK45,
App. C step parameters) against the CPU oracle's flow.

Endpoint bar (FP64 RHS): 1e-8 relative to the oracle's "truth" run at
rtol = 1e-13.  The GPU and the oracle may accept/reject differently near the
tolerance, so each is compared with the truth, not with the other's steps.
"""
import math

import numpy as np
import pytest

import ffrg_inputs as fi
import oracle
from gpu_common import gpu_context

pytestmark = pytest.mark.gpu
ENDPOINT_TOL = 1e-8
MIXED_ENDPOINT_TOL = 1e-8
# d=4 feedback: d_t Z_i = -(D2(p_i) - D2(0))/p_i^2 amplifies the FP32 integrand
# error (~3e-7 per RHS value) by |D2|/|D2(p_i) - D2(0)| ~ (k/p_i)^2 for p_i << k;
# the stated bound of the mixed path on this flow is 5e-6.
MIXED_FEEDBACK_ENDPOINT_TOL = 5e-6


@pytest.fixture(scope="module")
def ctx():
    c = gpu_context()
    yield c
    c.close()


def _gpu_flow(ctx, wl, precision, t1=None, **kw):
    import torch
    t1 = math.log(wl.Lambda / wl.k_end) if t1 is None else t1
    tabs = ctx.tables(wl.problem, wl.tables)
    y = torch.tensor(wl.y0, dtype=torch.float64, device="cuda")
    st = ctx.flow(wl.problem, tabs, y, wl.Lambda, t1, feedback=wl.feedback, precision=precision, **kw)
    out = y.cpu().numpy()
    tabs.free()
    return out, st


def _truth(wl, t1=None):
    t1 = math.log(wl.Lambda / wl.k_end) if t1 is None else t1
    y, _ = oracle.flow(wl.problem, wl.tables, wl.y0, wl.Lambda, t1, feedback=wl.feedback, rtol=1e-13,
                       atol=1e-16)
    return y


def _rel(a, b, floor=0.0):
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), floor))


def test_d3_frozen_full_size_fp64_and_mixed(ctx):
    import paper_2412_13043_gb300 as ffrg
    wl = fi.make_d3(seed=1)                       # 64 ext, 64 x 32 nodes, k: 10 -> 0.01
    truth = _truth(wl)
    y64, st = _gpu_flow(ctx, wl, ffrg.FP64)
    assert st["status"] == 0 and abs(st["t_reached"] - math.log(1000.0)) < 1e-12
    assert _rel(y64, truth) < ENDPOINT_TOL
    yo, sto = oracle.flow(wl.problem, wl.tables, wl.y0, wl.Lambda, math.log(1000.0), rtol=1e-11, atol=1e-14)
    assert abs(st["steps"] - sto["steps"]) <= 2
    y32, st32 = _gpu_flow(ctx, wl, ffrg.MIXED)
    err32 = _rel(y32, truth)
    print(f"d3 frozen: fp64 endpoint {_rel(y64, truth):.2e} ({st['steps']} steps), mixed {err32:.2e}")
    assert err32 < MIXED_ENDPOINT_TOL


def test_d3_feedback_flow(ctx):
    import paper_2412_13043_gb300 as ffrg
    wl = fi.make_d3(seed=4, n_pts=32, n_ext_p=32, n_rad=32, n_ang=16, feedback=1, x_min=0.01)
    truth = _truth(wl)
    y, st = _gpu_flow(ctx, wl, ffrg.FP64)
    assert st["status"] == 0
    assert _rel(y, truth, floor=1e-3) < ENDPOINT_TOL


def test_d4_feedback_flow_small(ctx):
    import paper_2412_13043_gb300 as ffrg
    wl = fi.make_d4(seed=6, n_pts=16, n_ext_ang=2, n_rad=16, n_ang1=8, n_ang2=4)
    wl.problem.p_min = wl.problem.x_min = 0.01
    truth = _truth(wl)
    y, st = _gpu_flow(ctx, wl, ffrg.FP64)
    assert st["status"] == 0 and st["steps"] > 3
    assert _rel(y, truth, floor=1e-3) < ENDPOINT_TOL
    y32, _ = _gpu_flow(ctx, wl, ffrg.MIXED)
    print(f"d4 feedback: fp64 endpoint {_rel(y, truth, 1e-3):.2e}, mixed {_rel(y32, truth, 1e-3):.2e}")
    assert _rel(y32, truth, floor=1e-3) < MIXED_FEEDBACK_ENDPOINT_TOL


def test_finite_t_frozen_flow_small(ctx):
    import paper_2412_13043_gb300 as ffrg
    wl = fi.make_finite_t(seed=7, N=3, T=0.05, n_pts=16, n_ext_p=6, n_ext_m=3, n_rad=16, n_ang=8)
    truth = _truth(wl)
    y, st = _gpu_flow(ctx, wl, ffrg.FP64)
    assert st["status"] == 0
    assert _rel(y, truth) < ENDPOINT_TOL
    y32, st32 = _gpu_flow(ctx, wl, ffrg.MIXED)
    assert st32["status"] == 0
    assert _rel(y32, truth) < MIXED_ENDPOINT_TOL


def test_zero_length_flow_is_identity(ctx):
    import paper_2412_13043_gb300 as ffrg
    wl = fi.make_d3(seed=1, n_ext_p=8, n_rad=8, n_ang=4)
    y, st = _gpu_flow(ctx, wl, ffrg.FP64, t1=0.0)
    assert np.array_equal(y, wl.y0) and st["steps"] == 0


def test_step_underflow_status(ctx):
    import paper_2412_13043_gb300 as ffrg
    wl = fi.make_d3(seed=1, n_ext_p=4, n_rad=8, n_ang=4)
    _, st = _gpu_flow(ctx, wl, ffrg.FP64, dt0=0.5, dt_min=0.5, dt_max=0.5, rtol=1e-16, atol=1e-300,
                      raise_on_error=False)
    assert st["status"] == ffrg.ESTEP_UNDERFLOW
    _, so = oracle.flow(wl.problem, wl.tables, wl.y0, wl.Lambda, math.log(1000.0), dt0=0.5, dt_min=0.5,
                        dt_max=0.5, rtol=1e-16, atol=1e-300, raise_on_error=False)
    assert so["status"] == oracle.ESTEP_UNDERFLOW


def test_max_steps_status(ctx):
    import paper_2412_13043_gb300 as ffrg
    wl = fi.make_d3(seed=1, n_ext_p=4, n_rad=8, n_ang=4)
    _, st = _gpu_flow(ctx, wl, ffrg.FP64, max_steps=3, raise_on_error=False)
    assert st["status"] == ffrg.EMAXSTEPS and st["steps"] + st["rejects"] == 3


def test_nonfinite_state_status(ctx):
    import paper_2412_13043_gb300 as ffrg
    wl = fi.make_d3(seed=1, n_ext_p=4, n_rad=8, n_ang=4)
    wl.y0 = wl.y0.copy()
    wl.y0[2] = float("nan")
    _, st = _gpu_flow(ctx, wl, ffrg.FP64, raise_on_error=False)
    assert st["status"] == ffrg.ENONFINITE
    ctx.status_read()


def test_flow_rejects_bad_options(ctx):
    import paper_2412_13043_gb300 as ffrg
    wl = fi.make_d3(seed=1, n_ext_p=4, n_rad=8, n_ang=4)
    with pytest.raises(ffrg.FfrgError):
        _gpu_flow(ctx, wl, ffrg.FP64, t1=-1.0)
    wl3 = fi.make_finite_t(seed=1, N=2, n_pts=8, n_ext_p=8, n_ext_m=2, n_rad=4, n_ang=4)
    wl3.feedback = 1
    with pytest.raises(ffrg.FfrgError):
        _gpu_flow(ctx, wl3, ffrg.FP64)


# ----------------------------------------------------------------------------- Adams-Bashforth-Moulton
def _gpu_abm(ctx, wl, n, order, precision, t1):
    import torch
    tabs = ctx.tables(wl.problem, wl.tables)
    y = torch.tensor(wl.y0, dtype=torch.float64, device="cuda")
    st = ctx.abm_flow(wl.problem, tabs, y, wl.Lambda, t1, n, order=order, feedback=wl.feedback, precision=precision)
    tabs.free()
    return y.cpu().numpy(), st


ABM_CASES = {
    "d3_frozen": (lambda: fi.make_d3(seed=21, n_pts=16, n_ext_p=9, n_rad=12, n_ang=6), None),
    "d3_feedback": (lambda: fi.make_d3(seed=22, n_pts=12, n_ext_p=12, n_rad=10, n_ang=6, feedback=1, x_min=0.05), 3.0),
    "d4_feedback": (lambda: fi.make_d4(seed=23, n_pts=8, n_ext_ang=2, n_rad=8, n_ang1=4, n_ang2=3), 2.0),
    "ft_fermionic": (lambda: fi.make_finite_t(seed=24, N=2, T=0.3, n_pts=12, n_ext_p=3, n_ext_m=3, n_rad=8, n_ang=4,
                                              fermionic=True), None),
}


@pytest.mark.parametrize("name", list(ABM_CASES))
@pytest.mark.parametrize("order", [2, 4, 5])
def test_abm_flow_matches_oracle_abm(ctx, name, order):
    """Same fixed-step PECE method on both sides: the endpoints differ only by
    RHS rounding (FP64), and by the stated mixed bound (mixed)."""
    import paper_2412_13043_gb300 as ffrg
    make, t1 = ABM_CASES[name]
    wl = make()
    if name == "d4_feedback":
        wl.problem.p_min = wl.problem.x_min = 0.05
    t1 = math.log(wl.Lambda / wl.k_end) if t1 is None else t1
    n = 60
    ref, so = oracle.abm_flow(wl.problem, wl.tables, wl.y0, wl.Lambda, t1, n, order=order, feedback=wl.feedback)
    y, st = _gpu_abm(ctx, wl, n, order, ffrg.FP64, t1)
    assert st["status"] == ffrg.OK and st["rhs_evals"] == so["rhs_evals"]
    assert abs(st["t_reached"] - t1) < 1e-12 * max(1.0, t1)
    assert np.max(np.abs(y - ref) / np.abs(ref)) < 1e-10
    if order == 4:
        ym, _ = _gpu_abm(ctx, wl, n, order, ffrg.MIXED, t1)
        tol = MIXED_FEEDBACK_ENDPOINT_TOL if name == "d4_feedback" else MIXED_ENDPOINT_TOL
        assert np.max(np.abs(ym - ref) / np.abs(ref)) < tol


def test_abm_flow_fourth_order_against_dp45_truth(ctx):
    import paper_2412_13043_gb300 as ffrg
    wl = ABM_CASES["d3_frozen"][0]()
    t1 = math.log(wl.Lambda / wl.k_end)
    truth, _ = oracle.flow(wl.problem, wl.tables, wl.y0, wl.Lambda, t1, rtol=1e-13, atol=1e-16)
    errs = []
    for n in (60, 120, 240):
        y, _ = _gpu_abm(ctx, wl, n, 4, ffrg.FP64, t1)
        errs.append(np.max(np.abs(y - truth) / np.abs(truth)))
    assert errs[0] / errs[1] > 10 and errs[1] / errs[2] > 12, errs
    assert errs[2] < 1e-8


def test_abm_flow_rejects_bad_arguments(ctx):
    import torch

    import paper_2412_13043_gb300 as ffrg
    wl = ABM_CASES["d3_frozen"][0]()
    tabs = ctx.tables(wl.problem, wl.tables)
    y = torch.tensor(wl.y0, dtype=torch.float64, device="cuda")
    for order, n in ((1, 10), (6, 10), (4, 0)):
        with pytest.raises(ffrg.FfrgError):
            ctx.abm_flow(wl.problem, tabs, y, wl.Lambda, 1.0, n, order=order)
    tabs.free()
