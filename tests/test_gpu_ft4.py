"""GPU parity of the finite-T model with a 4D regulator on a k-scaled
frequency domain (Sec. 5.3.2 "Quadraturex0"; App. G fermion legs at p0f)
against the oracle, through the C ABI: FP64 1e-12 per output, mixed 1e-6;
both branches of the frequency integral (Matsubara sum while at most
2N+1 (+1) loop frequencies lie in |q0| <= qmax k, Gauss-Legendre beyond),
both loop statistics, the bench workload on every output, and a frozen flow
from k = 10 to 0.01 that crosses the branch switch."""
import math

import numpy as np
import pytest

import ffrg_inputs as fi
import oracle
from gpu_common import gpu_context, rel_err

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 1e-6


@pytest.fixture(scope="module")
def ctx():
    c = gpu_context()
    yield c
    c.close()


def _run(ctx, wl, k, precision):
    import paper_2412_13043_gb300 as ffrg
    tabs = ctx.tables(wl.problem, wl.tables)
    out = ctx.rhs(wl.problem, tabs, k, precision=precision).cpu().numpy()
    st = ctx.status_read()
    tabs.free()
    assert st == ffrg.OK, ffrg.strerror(st)
    return out


def _check(ctx, wl, k):
    import paper_2412_13043_gb300 as ffrg
    ref = oracle.rhs(wl.problem, wl.tables, k)
    e64 = rel_err(_run(ctx, wl, k, ffrg.FP64), ref)
    e32 = rel_err(_run(ctx, wl, k, ffrg.MIXED), ref)
    nf = oracle.ft4_frequencies(wl.problem, k)[0].size
    print(f"ft4 k={k} frequencies {nf}: fp64 {np.max(e64):.2e}, mixed {np.max(e32):.2e}")
    assert np.max(e64) < FP64_TOL, (k, np.max(e64))
    assert np.max(e32) < MIXED_TOL, (k, np.max(e32))


@pytest.mark.parametrize("fermionic", [False, True])
def test_small_ragged_both_branches(ctx, fermionic):
    """k = 0.3 and 0.5: Matsubara sums (bosonic 7 and 13 frequencies, the
    second at the cap 13; fermionic 8 and 12 of cap 14); k = 8: more than the
    cap lie in the domain, the 21-node quadrature."""
    wl = fi.make_finite_t_4d(seed=51, N=6, T=0.05, n_pts=24, n_ext_p=7, n_ext_m=3, n_rad=13, n_ang=9, n_x0=21,
                             fermionic=fermionic)
    counts = [oracle.ft4_frequencies(wl.problem, k)[0].size for k in (0.3, 0.5, 8.0)]
    assert counts == ([8, 12, 21] if fermionic else [7, 13, 21])
    for k in (0.3, 0.5, 8.0):
        _check(ctx, wl, k)


def test_no_frequency_in_the_domain_gives_zero(ctx):
    """Fermionic loop with qmax k < pi T: no loop frequency, the integral is 0."""
    import paper_2412_13043_gb300 as ffrg
    wl = fi.make_finite_t_4d(seed=52, N=4, T=0.5, n_pts=16, n_ext_p=3, n_rad=8, n_ang=4, n_x0=8, fermionic=True)
    k = 0.3            # 4k = 1.2 < pi T = 1.57
    assert oracle.ft4_frequencies(wl.problem, k)[0].size == 0
    assert np.all(_run(ctx, wl, k, ffrg.FP64) == 0.0)


def test_bench_workload_every_output(ctx):
    """64 |p| x 9 external frequencies, 96 x 48 nodes, cap N = 16, T = 0.05:
    the Matsubara sum at k = 1 (25 frequencies) and the 64-node quadrature at
    k = 10."""
    wl = fi.make_finite_t_4d()
    for k in (1.0, 10.0):
        _check(ctx, wl, k)


def test_frozen_flow_across_the_branch_switch(ctx):
    """k: 10 -> 0.01 passes from the quadrature through Matsubara sums of
    decreasing length to a single frequency; FP64 endpoint against the
    oracle's truth (rtol 1e-13)."""
    import torch

    import paper_2412_13043_gb300 as ffrg
    wl = fi.make_finite_t_4d(seed=53, N=5, T=0.05, n_pts=16, n_ext_p=4, n_ext_m=2, n_rad=12, n_ang=6, n_x0=16)
    t1 = math.log(wl.Lambda / wl.k_end)
    truth, _ = oracle.flow(wl.problem, wl.tables, wl.y0, wl.Lambda, t1, rtol=1e-13, atol=1e-16)
    tabs = ctx.tables(wl.problem, wl.tables)
    y = torch.tensor(wl.y0, dtype=torch.float64, device="cuda")
    st = ctx.flow(wl.problem, tabs, y, wl.Lambda, t1, precision=ffrg.FP64, rtol=1e-11, atol=1e-14)
    tabs.free()
    assert st["status"] == ffrg.OK
    got = y.cpu().numpy()
    assert np.max(np.abs(got - truth) / np.abs(truth)) < 1e-8
