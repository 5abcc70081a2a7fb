"""GPU parity of ffrg_ft_states (finite-T sums of many loop-side states against
one angle-integrated kernel K(p, q), Sec. 5.3.2; the contraction runs on the
tensor cores with an FP64-faithful slice split) against the oracle's plain
definition, through the C ABI.

Bars: FP64 K: 1e-12 per output (relative to the sum of the terms' magnitudes
where the states change sign); mixed K (FP32 angular sums): the mixed bound
1e-6.  Covers several output tiles with ragged edges in both directions,
more K-elements than one exact pass holds (two K ranges per slice pair), the
model's own loop factor (= the RHS), both loop statistics and repeatability.
"""
import numpy as np
import pytest

import ffrg_inputs as fi
import oracle
from gpu_common import gpu_context

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 1e-6


@pytest.fixture(scope="module")
def ctx():
    c = gpu_context()
    yield c
    c.close()


def _gpu(ctx, wl, k, F, precision):
    import torch

    import paper_2412_13043_gb300 as ffrg
    tabs = ctx.tables(wl.problem, wl.tables)
    Fd = torch.tensor(np.ascontiguousarray(F), dtype=torch.float64, device="cuda")
    out = ctx.ft_states(wl.problem, tabs, k, Fd, precision=precision).cpu().numpy()
    st = ctx.status_read()
    tabs.free()
    assert st == ffrg.OK, ffrg.strerror(st)
    return out


@pytest.mark.parametrize("fermionic", [False, True])
def test_model_loop_factor_reproduces_the_rhs(ctx, fermionic):
    import paper_2412_13043_gb300 as ffrg
    wl = fi.make_finite_t(seed=101, N=4, T=0.05, n_pts=16, n_ext_p=7, n_ext_m=4, n_rad=13, n_ang=9,
                          fermionic=fermionic)
    for k in (1.3, 0.2):
        F = oracle.ft_loop_factors(wl.problem, wl.tables, k)[None]
        ref = oracle.rhs(wl.problem, wl.tables, k)
        got = _gpu(ctx, wl, k, F, ffrg.FP64)[0]
        assert np.max(np.abs(got - ref) / np.abs(ref)) < FP64_TOL
        got32 = _gpu(ctx, wl, k, F, ffrg.MIXED)[0]
        assert np.max(np.abs(got32 - ref) / np.abs(ref)) < MIXED_TOL


def test_many_states_span_tiles_with_ragged_edges(ctx):
    """300 states (two column tiles, the second ragged) x 140 external points
    (two row tiles, the second ragged), positive and mixed-sign states."""
    import paper_2412_13043_gb300 as ffrg
    wl = fi.make_finite_t(seed=102, N=3, T=0.08, n_pts=16, n_ext_p=35, n_ext_m=4, n_rad=11, n_ang=6)
    pb = wl.problem
    k = 0.9
    rng = np.random.default_rng(21)
    base = oracle.ft_loop_factors(pb, wl.tables, k)
    F = base[None] * rng.uniform(0.2, 3.0, size=(300,) + base.shape)
    ref = oracle.ft_states(pb, wl.tables, k, F)
    got = _gpu(ctx, wl, k, F, ffrg.FP64)
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref) / np.abs(ref)) < FP64_TOL
    Fs = base[None] * rng.normal(size=(37,) + base.shape)          # sign changes
    ref = oracle.ft_states(pb, wl.tables, k, Fs)
    scale = oracle.ft_states(pb, wl.tables, k, np.abs(Fs))         # sum of |terms| (K > 0)
    got = _gpu(ctx, wl, k, Fs, ffrg.FP64)
    assert np.max(np.abs(got - ref) / scale) < FP64_TOL


def test_more_terms_than_one_exact_pass(ctx):
    """nfreq x n_rad = 130 x 160 = 20800 > 16384 terms: every slice pair takes
    two K ranges; fermionic loop at N = 64."""
    import paper_2412_13043_gb300 as ffrg
    wl = fi.make_finite_t(seed=103, N=64, T=0.003, n_pts=32, n_ext_p=2, n_ext_m=3, n_rad=160, n_ang=3,
                          fermionic=True)
    pb = wl.problem
    k = 0.6
    rng = np.random.default_rng(22)
    base = oracle.ft_loop_factors(pb, wl.tables, k)
    assert base.size > 16384
    F = base[None] * rng.uniform(0.5, 2.0, size=(5,) + base.shape)
    ref = oracle.ft_states(pb, wl.tables, k, F)
    got = _gpu(ctx, wl, k, F, ffrg.FP64)
    assert np.max(np.abs(got - ref) / np.abs(ref)) < FP64_TOL


def test_bench_workload_sampled_states(ctx):
    """The finite-T bench workload (576 external points, 96 x 48 nodes, N = 16)
    with 512 states; every output of 4 states against the oracle."""
    import paper_2412_13043_gb300 as ffrg
    wl = fi.make_finite_t(seed=3, N=16, T=0.0005)
    pb = wl.problem
    k = 1.0
    rng = np.random.default_rng(23)
    base = oracle.ft_loop_factors(pb, wl.tables, k)
    F = base[None] * rng.uniform(0.5, 2.0, size=(512,) + base.shape)
    got = _gpu(ctx, wl, k, F, ffrg.FP64)
    sel = [0, 137, 300, 511]
    ref = oracle.ft_states(pb, wl.tables, k, F[sel])
    assert np.max(np.abs(got[sel] - ref) / np.abs(ref)) < FP64_TOL


def test_repeatable_and_rejects_other_models(ctx):
    import torch

    import paper_2412_13043_gb300 as ffrg
    wl = fi.make_finite_t(seed=104, N=2, T=0.1, n_pts=8, n_ext_p=3, n_ext_m=2, n_rad=5, n_ang=3)
    F = np.random.default_rng(1).uniform(size=(3, oracle.ft_nfreq(wl.problem), wl.problem.n_rad))
    a = _gpu(ctx, wl, 0.7, F, ffrg.FP64)
    b = _gpu(ctx, wl, 0.7, F, ffrg.FP64)
    assert np.array_equal(a, b)
    w3 = fi.make_d3(seed=1, n_pts=8, n_ext_p=4, n_rad=4, n_ang=2)
    tabs = ctx.tables(w3.problem, w3.tables)
    Fd = torch.ones(2, 1, 4, dtype=torch.float64, device="cuda")
    with pytest.raises(ffrg.FfrgError):
        ctx.ft_states(w3.problem, tabs, 1.0, Fd)
    tabs.free()
