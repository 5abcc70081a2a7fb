"""GPU adjoint (ffrg_rhs_adjoint, reverse mode) against the oracle's
forward-mode Jacobian (dual numbers, the paper's approach in Sec. 5.2.2),
a dot-product identity and central finite differences (h = 1e-6, FP64)."""
import numpy as np
import pytest

import ffrg_inputs as fi
import oracle
from gpu_common import gpu_context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gpu_context()
    yield c
    c.close()


def _vjp(ctx, wl, k, gbar):
    import torch
    tabs = ctx.tables(wl.problem, wl.tables)
    g = torch.tensor(gbar, dtype=torch.float64, device="cuda")
    tb = ctx.rhs_adjoint(wl.problem, tabs, k, g).cpu().numpy()
    assert ctx.status_read() == 0
    tabs.free()
    return tb


CASES = {
    "d3": lambda: fi.make_d3(seed=8, n_pts=16, n_ext_p=11, n_rad=19, n_ang=9),
    "d3p0": lambda: fi.make_d3(seed=9, n_pts=12, n_ext_p=12, n_rad=13, n_ang=7, feedback=1),
    "d4": lambda: fi.make_d4(seed=8, n_pts=12, n_ext_ang=3, n_rad=11, n_ang1=7, n_ang2=5),
}


@pytest.mark.parametrize("name", list(CASES))
def test_vjp_matches_oracle_jacobian(ctx, name):
    wl = CASES[name]()
    k = 1.3
    rng = np.random.default_rng(5)
    gbar = rng.normal(size=wl.problem.n_ext())
    J = oracle.rhs_jacobian(wl.problem, wl.tables, k)
    ref = J.T @ gbar
    got = _vjp(ctx, wl, k, gbar)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)) / scale < 1e-12, np.max(np.abs(got - ref)) / scale


def test_dot_product_identity_and_fd(ctx):
    import torch

    import paper_2412_13043_gb300 as ffrg
    wl = CASES["d4"]()
    k = 0.8
    rng = np.random.default_rng(11)
    gbar = rng.normal(size=wl.problem.n_ext())
    dT = rng.normal(size=wl.tables.shape)
    tbar = _vjp(ctx, wl, k, gbar)
    _, jv = oracle.rhs_jvp(wl.problem, wl.tables, dT, k)
    lhs, rhs = float(gbar @ jv), float(tbar @ dT.ravel())
    assert abs(lhs - rhs) / abs(lhs) < 1e-12
    # central differences of the GPU forward (FP64), h = 1e-6
    h = 1e-6
    tp = ctx.tables(wl.problem, wl.tables + h * dT)
    tm = ctx.tables(wl.problem, wl.tables - h * dT)
    fp = ctx.rhs(wl.problem, tp, k, precision=ffrg.FP64).cpu().numpy()
    fm = ctx.rhs(wl.problem, tm, k, precision=ffrg.FP64).cpu().numpy()
    tp.free()
    tm.free()
    fd = float(gbar @ ((fp - fm) / (2 * h)))
    assert abs(fd - rhs) / abs(rhs) < 1e-7


def test_vjp_is_reproducible(ctx):
    wl = CASES["d4"]()
    gbar = np.random.default_rng(3).normal(size=wl.problem.n_ext())
    a = _vjp(ctx, wl, 1.1, gbar)
    b = _vjp(ctx, wl, 1.1, gbar)
    assert np.array_equal(a, b)


def test_autograd_function(ctx):
    import torch

    from paper_2412_13043_gb300.autograd import rhs as drhs
    wl = CASES["d3"]()
    k = 0.9
    T = torch.tensor(wl.tables, dtype=torch.float64, device="cuda", requires_grad=True)
    out = drhs(T, ctx, wl.problem, k)
    gbar = torch.linspace(-1.0, 2.0, out.numel(), dtype=torch.float64, device="cuda")
    (out * gbar).sum().backward()
    J = oracle.rhs_jacobian(wl.problem, wl.tables, k)
    ref = J.T @ gbar.cpu().numpy()
    got = T.grad.cpu().numpy().ravel()
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-12
    ref_out = oracle.rhs(wl.problem, wl.tables, k)
    assert np.max(np.abs(out.detach().cpu().numpy() - ref_out) / np.abs(ref_out)) < 1e-12


def test_adjoint_rejects_unsupported(ctx):
    import torch

    import paper_2412_13043_gb300 as ffrg
    wl = fi.make_finite_t(seed=1, N=2, n_pts=8, n_ext_p=4, n_ext_m=2, n_rad=4, n_ang=4)
    tabs = ctx.tables(wl.problem, wl.tables)
    g = torch.ones(wl.problem.n_ext(), dtype=torch.float64, device="cuda")
    with pytest.raises(ffrg.FfrgError):
        ctx.rhs_adjoint(wl.problem, tabs, 1.0, g)
    wl1 = CASES["d3"]()
    t1 = ctx.tables(wl1.problem, wl1.tables)
    g1 = torch.ones(wl1.problem.n_ext(), dtype=torch.float64, device="cuda")
    with pytest.raises(ffrg.FfrgError):
        ctx.rhs_adjoint(wl1.problem, t1, 1.0, g1, precision=ffrg.MIXED)
    tabs.free()
    t1.free()


@pytest.mark.parametrize("name", list(CASES))
def test_full_jacobian_matches_oracle(ctx, name):
    wl = CASES[name]()
    k = 0.9
    tabs = ctx.tables(wl.problem, wl.tables)
    J = ctx.rhs_jacobian(wl.problem, tabs, k).cpu().numpy()
    tabs.free()
    ref = oracle.rhs_jacobian(wl.problem, wl.tables, k)
    assert np.max(np.abs(J - ref)) / np.max(np.abs(ref)) < 1e-12


def test_jacobian_and_vjp_at_the_d4_bench_size(ctx):
    """The full d=4 workload (128-point tables, 1281 external points x 128 x
    64 x 16 nodes): the 1281 x 384 Jacobian applied to random table directions
    against the oracle's forward-mode JVPs, and the VJP against J^T g."""
    import torch
    wl = fi.make_d4(seed=2)
    k = 0.5
    tabs = ctx.tables(wl.problem, wl.tables)
    J = ctx.rhs_jacobian(wl.problem, tabs, k).cpu().numpy()
    rng = np.random.default_rng(13)
    for _ in range(2):
        dT = rng.normal(size=wl.tables.shape)
        _, jv = oracle.rhs_jvp(wl.problem, wl.tables, dT, k)
        got = J @ dT.ravel()
        assert np.max(np.abs(got - jv)) / np.max(np.abs(jv)) < 1e-12
    gbar = rng.normal(size=wl.problem.n_ext())
    tb = ctx.rhs_adjoint(wl.problem, tabs, k, torch.tensor(gbar, dtype=torch.float64, device="cuda")).cpu().numpy()
    tabs.free()
    ref = J.T @ gbar
    assert np.max(np.abs(tb - ref)) / np.max(np.abs(ref)) < 1e-12


def test_rosenbrock_flow_matches_oracle_ros2_and_dp45():
    """ROS2 on the device (Jacobian from the reverse-mode kernels, LU on the
    device) against the oracle's ROS2 and a tight DP5(4) reference."""
    import math

    import torch

    import paper_2412_13043_gb300 as ffrg
    c = gpu_context()
    wl = fi.make_d4(seed=6, n_pts=8, n_ext_ang=2, n_rad=8, n_ang1=4, n_ang2=3)
    pb = wl.problem
    pb.p_min = pb.x_min = 0.05
    t1 = 2.0
    ref, _ = oracle.flow(pb, wl.tables, wl.y0, wl.Lambda, t1, feedback=1, rtol=1e-12, atol=1e-14)
    yo, so = oracle.ros2_flow(pb, wl.y0, wl.Lambda, t1, rtol=1e-8, atol=1e-12)
    tabs = c.tables(pb, wl.tables)
    y = torch.tensor(wl.y0, dtype=torch.float64, device="cuda")
    st = c.rosenbrock_flow(pb, tabs, y, wl.Lambda, t1, rtol=1e-8, atol=1e-12)
    tabs.free()
    c.close()
    yg = y.cpu().numpy()
    assert st["status"] == ffrg.OK and st["jac_evals"] >= st["steps"]
    assert abs(st["steps"] - so["steps"]) <= 2
    assert np.max(np.abs(yg - yo) / np.abs(yo)) < 1e-9      # same method, same decisions
    assert np.max(np.abs(yg - ref) / np.abs(ref)) < 2e-6     # second-order accuracy at rtol 1e-8
