"""GPU parity of ffrg_rhs (through the C ABI) against the FP64 CPU oracle.

FP64 path: 1e-12 relative per output (Sec. 5.3.2 quadrature, computed by the
same discrete sums; the two sides differ only in summation order and libm vs
CUDA rounding).  Mixed path (FP32 integrand, FP64 per-radial factors and
cross-node accumulation): the stated bound MIXED_TOL per output.
Small cases span several work items with ragged tails; the full-size
workloads (d=4 1281 x 128 x 64 x 16, the 96 x 8 x 7 full vertex, finite T at
N = 16/32/64 with both loop statistics) are compared on every output.  The
d=4 Z block D2 = int dR G^2 [-lam4/2 + lam3^2 G] is a difference of two
single-signed parts that can cancel; there the error is taken relative to
the sum of the parts' magnitudes (both computed by the oracle), and the
condition number |parts| / |D2| is printed beside it.
"""
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


def _run(ctx, wl, k, precision, out=None):
    import paper_2412_13043_gb300 as ffrg
    tabs = ctx.tables(wl.problem, wl.tables)
    o = ctx.rhs(wl.problem, tabs, k, out=out, precision=precision)
    st = ctx.status_read()
    res = o.cpu().numpy()
    tabs.free()
    assert st == ffrg.OK, ffrg.strerror(st)
    return res


def _oracle_scale(wl, k, ref, sel=None):
    """Per output, the magnitude the error is measured against: |ref|, except
    in the Z block of the d=4 models, where it is |D2 at lam4 = 0| + |D2 at
    lam3 = 0| (the two single-signed parts of D2), from the oracle."""
    pb = wl.problem
    scale = np.abs(ref).copy()
    if pb.model not in (fi.MODEL_D4_VERTEX, fi.MODEL_D4_FULL):
        return scale
    nz = pb.n_ext_p + 1
    idx = np.arange(pb.n_ext()) if sel is None else np.asarray(sel)
    zpos = np.nonzero(idx < nz)[0]
    if zpos.size == 0:
        return scale
    parts = np.zeros(zpos.size)
    for zero in (2, 1):
        t = wl.tables.copy()
        t[zero] = 0.0
        parts += np.abs(oracle.rhs_subset(pb, t, k, idx[zpos]))
    scale[zpos] = parts
    return scale


def _check(ctx, wl, k, sel=None, mixed=True):
    import paper_2412_13043_gb300 as ffrg
    if sel is None:
        ref = oracle.rhs(wl.problem, wl.tables, k)
    else:
        ref = oracle.rhs_subset(wl.problem, wl.tables, k, sel)
    scale = _oracle_scale(wl, k, ref, sel)
    cond = float(np.max(scale / np.maximum(np.abs(ref), 1e-300)))
    g64 = _run(ctx, wl, k, ffrg.FP64)
    g64 = g64 if sel is None else g64[sel]
    e64 = np.abs(g64 - ref) / scale
    assert np.max(e64) < FP64_TOL, (np.max(e64), int(np.argmax(e64)))
    msg = f"model {wl.problem.model} k={k} n={ref.size}: fp64 max {np.max(e64):.2e}"
    if mixed:
        g32 = _run(ctx, wl, k, ffrg.MIXED)
        g32 = g32 if sel is None else g32[sel]
        e32 = np.abs(g32 - ref) / scale
        msg += f", mixed max {np.max(e32):.2e}"
        assert np.max(e32) < MIXED_TOL, (np.max(e32), int(np.argmax(e32)))
    print(msg + f", max condition {cond:.1f}")
    return e64


# ----------------------------------------------------------------------------- d=3
@pytest.mark.parametrize("k", [10.0, 1.3, 0.05, 0.01])
def test_d3_small_ragged(ctx, k):
    wl = fi.make_d3(seed=31, n_pts=23, n_ext_p=29, n_rad=37, n_ang=13)
    wl.problem.include_p0 = 1
    _check(ctx, wl, k)


def test_d3_full_size(ctx):
    wl = fi.make_d3(seed=1)       # 64 ext x (64 radial x 32 angular)
    for k in (10.0, 0.3, 0.01):
        _check(ctx, wl, k)


@pytest.mark.parametrize("n_ext_p,n_rad,n_ang", [(1, 1, 1), (1, 3, 2), (2, 1, 5), (5, 600, 3), (300, 7, 1)])
def test_d3_degenerate_shapes(ctx, n_ext_p, n_rad, n_ang):
    wl = fi.make_d3(seed=3, n_pts=8, n_ext_p=n_ext_p, n_rad=n_rad, n_ang=n_ang)
    _check(ctx, wl, 2.0)


def test_d3_momenta_outside_table_clamp(ctx):
    wl = fi.make_d3(seed=5, n_pts=16, n_ext_p=12)
    wl.problem.p_min, wl.problem.p_max = 1e-6, 80.0   # beyond [x_min, x_max] on both sides
    _check(ctx, wl, 3.0)


def test_d3_litim_closed_form_on_gpu(ctx):
    import paper_2412_13043_gb300 as ffrg
    pb = fi.Problem(model=fi.MODEL_D3, n_rad=16, n_ang1=4, n_ext_p=1, include_p0=1, regulator=fi.REG_LITIM,
                    m2_over_k2=0.5, qmax_over_k=1.0)
    wl = fi.Workload(pb, fi.constant_tables(pb, [1.0]))
    k = 1.7
    exact = k ** -1 / (3 * math.pi ** 2 * 1.5 ** 3)
    g = _run(ctx, wl, k, ffrg.FP64)
    assert abs(g[-1] - exact) / exact < 1e-13


def test_d3_near_pole_mixed_uses_fp64_propagator(ctx):
    """w = m^2/k^2 -> -0.999: Z s^2 + R >= k^2, so the denominator cancels to
    ~1e-3 k^2; the mixed path must recompute those propagators in FP64."""
    wl = fi.make_d3(seed=9, n_pts=32, n_ext_p=16, n_rad=32, n_ang=16)
    wl.tables[:] = 1.0                     # Z = 1 makes the pole reachable at x -> 0
    wl.problem.m2_over_k2 = -0.999
    _check(ctx, wl, 1.0)


# ----------------------------------------------------------------------------- d=4
def test_d4_small_ragged(ctx):
    wl = fi.make_d4(seed=41, n_pts=24, n_ext_ang=3, n_rad=19, n_ang1=11, n_ang2=5)
    for k in (10.0, 0.7, 0.01):
        _check(ctx, wl, k)


def test_d4_full_size_every_output(ctx):
    """The d=4 vertex workload at full size, (128 + 1 + 1024 + 128) external
    points x (128 x 64 x 16) nodes, every output against the oracle."""
    wl = fi.make_d4(seed=2)
    for k in (10.0, 0.5):
        _check(ctx, wl, k)


@pytest.mark.parametrize("full", [False, True])
def test_d4_near_pole_mixed_uses_fp64_propagator(ctx, full):
    """m^2 = -0.999 k^2 with Z = 1: every propagator denominator Z k^2 h(x) + m^2
    cancels to ~1e-3 k^2 at small momenta, so the mixed d=4 kernels run their
    near-pole variant (scalar second-angle loop, FP64 recompute)."""
    if full:
        wl = fi.make_d4_full(seed=13, n_pts=16, n_va=3, n_vb=2, n_ext_ang=2, n_rad=12, n_ang1=6, n_ang2=5)
    else:
        wl = fi.make_d4(seed=12, n_pts=24, n_ext_ang=3, n_rad=16, n_ang1=8, n_ang2=5)
    import paper_2412_13043_gb300 as ffrg
    wl.tables[0][:] = 1.0
    wl.problem.m2_over_k2 = -0.999
    wl.problem.m2_shift = 0.0
    for k in (1.0, 0.05):
        ref = oracle.rhs(wl.problem, wl.tables, k)
        scale = _oracle_scale(wl, k, ref)   # the Z block can cross zero
        g64 = _run(ctx, wl, k, ffrg.FP64)
        g32 = _run(ctx, wl, k, ffrg.MIXED)
        assert np.max(np.abs(g64 - ref) / scale) < FP64_TOL
        assert np.max(np.abs(g32 - ref) / scale) < MIXED_TOL, (k, np.max(np.abs(g32 - ref) / scale))


def test_d4_litim_closed_forms_on_gpu(ctx):
    import paper_2412_13043_gb300 as ffrg
    k, M2 = 2.0, 1.0
    pb = fi.Problem(model=fi.MODEL_D4_VERTEX, n_rad=8, n_ang1=4, n_ang2=3, n_ext_p=2, n_ext_ang=3,
                    regulator=fi.REG_LITIM, m2_over_k2=0.5, m2_shift=M2, qmax_over_k=1.0, n_tables=3, n_pts=16,
                    p_min=1e-200, p_max=2e-200)
    wl = fi.Workload(pb, fi.constant_tables(pb, [1.0, 0.8, 1.3]))
    w = 0.5 + M2 / k ** 2
    v4 = 1.0 / (32 * math.pi ** 2)
    ex3 = 4 * v4 * k ** 0 * 0.5 / (1 + w) ** 3
    ex4 = 4 * v4 * k ** -2 * 0.5 / (1 + w) ** 4
    g = _run(ctx, wl, k, ffrg.FP64)
    np_ = pb.n_ext_p
    blk3 = g[np_ + 1: np_ + 1 + np_ * 3]
    blk4 = g[np_ + 1 + np_ * 3:]
    assert np.max(np.abs(blk3 - 3 * 0.8 ** 3 * ex4)) / ex4 < 1e-13
    assert np.max(np.abs(blk4 - 1.5 * 1.3 ** 2 * ex3)) / ex3 < 1e-13


# ----------------------------------------------------------------------------- d=4, full vertex
def test_d4_full_small_ragged(ctx):
    """lambda3 on (S0, a, b) (trilinear), compact tables staged per CTA."""
    for seed, na, nb in ((41, 3, 4), (42, 1, 5), (43, 4, 1)):
        wl = fi.make_d4_full(seed=seed, n_pts=12, n_va=na, n_vb=nb, n_ext_ang=3, n_rad=9, n_ang1=5, n_ang2=4)
        for k in (1.3, 0.4):
            _check(ctx, wl, k)


def test_d4_full_line_rows_when_cells_exceed_shared_memory(ctx):
    """A 96 x 12 x 12 vertex grid: its FP32 cell polynomials (32 bytes per
    (S0, a, b) node, 444 KB) exceed shared memory, so the mixed kernel reads
    lambda3 from line rows (8 bytes per node, 112 KB), four rows per lookup;
    the 96 x 8 x 7 grids of the other tests use the cells."""
    wl = fi.make_d4_full(seed=46, n_pts=96, n_va=12, n_vb=12, n_ext_ang=2, n_rad=9, n_ang1=5, n_ang2=4)
    for k in (1.3, 0.2):
        _check(ctx, wl, k)


def test_d4_full_full_size_every_output(ctx):
    """96-point log grid x 8 x 7 vertex grid, 961 external points x
    (128 x 64 x 16) nodes, every output against the oracle."""
    wl = fi.make_d4_full()
    for k in (1.0, 0.1):
        _check(ctx, wl, k)


def test_d4_full_reduces_to_d4_vertex_on_gpu(ctx):
    import dataclasses

    import paper_2412_13043_gb300 as ffrg
    wl = fi.make_d4(seed=44, n_pts=16, n_ext_ang=3, n_rad=11, n_ang1=7, n_ang2=5)
    na, nb = 3, 2
    pf = dataclasses.replace(wl.problem, model=fi.MODEL_D4_FULL, n_stack=na * nb, n_va=na, n_vb=nb)
    tf = np.zeros((3, na * nb, pf.n_pts))
    tf[0, 0], tf[2, 0] = wl.tables[0, 0], wl.tables[2, 0]
    tf[1, :] = wl.tables[1, 0]
    wf = fi.Workload(pf, tf, None)
    for prec, tol in ((ffrg.FP64, 1e-13), (ffrg.MIXED, 1e-6)):
        a = _run(ctx, wl, 0.9, prec)
        b = _run(ctx, wf, 0.9, prec)
        assert np.max(np.abs(a - b) / np.abs(a)) < tol, prec


def test_d4_full_rejects_adjoint_and_feedback(ctx):
    import torch

    import paper_2412_13043_gb300 as ffrg
    wl = fi.make_d4_full(seed=45, n_pts=8, n_va=2, n_vb=2, n_ext_ang=2, n_rad=4, n_ang1=3, n_ang2=2)
    tabs = ctx.tables(wl.problem, wl.tables)
    g = torch.ones(wl.problem.n_ext(), dtype=torch.float64, device="cuda")
    with pytest.raises(ffrg.FfrgError):
        ctx.rhs_adjoint(wl.problem, tabs, 1.0, g)
    y = torch.ones(3 * wl.problem.n_pts, dtype=torch.float64, device="cuda")
    with pytest.raises(ffrg.FfrgError):
        ctx.flow(wl.problem, tabs, y, 10.0, 1.0, feedback=1)
    tabs.free()


# ----------------------------------------------------------------------------- finite T
def test_finite_t_small_ragged(ctx):
    wl = fi.make_finite_t(seed=51, N=3, T=0.05, n_pts=16, n_ext_p=7, n_ext_m=4, n_rad=13, n_ang=9)
    for k in (10.0, 0.4):
        _check(ctx, wl, k)


@pytest.mark.parametrize("N,T_over_kend", [(16, 0.05), (32, 0.2), (64, 1.0)])
def test_finite_t_full_size_every_output(ctx, N, T_over_kend):
    """64 |p| x 9 p0 external points x 96 x 48 x (2N+1) nodes, every output."""
    wl = fi.make_finite_t(seed=3, N=N, T=T_over_kend * 0.01)
    _check(ctx, wl, 1.0)


# ----------------------------------------------------------------------------- fermionic loop
def test_finite_t_fermionic_small_ragged(ctx):
    """nu_n = (2n+1) pi T, n = -N-1..N, fermionic stacks (App. F)."""
    for N, T in ((0, 0.3), (3, 0.05), (5, 0.5)):
        wl = fi.make_finite_t(seed=61 + N, N=N, T=T, n_pts=16, n_ext_p=7, n_ext_m=4, n_rad=13, n_ang=9,
                              fermionic=True)
        for k in (10.0, 0.4):
            _check(ctx, wl, k)


@pytest.mark.parametrize("N,T_over_kend", [(16, 0.05), (32, 0.2), (64, 1.0)])
def test_finite_t_fermionic_full_size_every_output(ctx, N, T_over_kend):
    """Fermionic loop, 96 x 48 x (2N+2) nodes, every output."""
    wl = fi.make_finite_t(seed=4, N=N, T=T_over_kend * 0.01, fermionic=True)
    _check(ctx, wl, 1.0)


def test_finite_t_fermionic_litim_closed_form_on_gpu(ctx):
    """Flat regulator, Z = lam = 1, p -> 0: k^5/(3 pi^2) T sum_n (nu_n^2+E^2)^-3
    summed over the 2N+2 fermionic frequencies (rational sum in mpmath)."""
    import mpmath

    import paper_2412_13043_gb300 as ffrg
    k, w, T, N = 1.3, 0.5, 0.3, 16
    pb = fi.Problem(model=fi.MODEL_FINITE_T, n_rad=8, n_ang1=3, n_ext_p=1, n_ext_ang=1, n_matsubara=N,
                    regulator=fi.REG_LITIM, m2_over_k2=w, T=T, qmax_over_k=1.0, n_tables=2, n_pts=8,
                    n_stack=N + 2, p_min=1e-200, p_max=1e-200, statistics=fi.STAT_FERMI)
    wl = fi.Workload(pb, fi.constant_tables(pb, [1.0, 1.0]), None, 10.0, 0.01, 0, 0, {})
    E2 = mpmath.mpf(k * k * (1 + w))
    s = sum(1 / (((2 * n + 1) * mpmath.pi * T) ** 2 + E2) ** 3 for n in range(-N - 1, N + 1))
    exact = float(k ** 3 / (6 * mpmath.pi ** 2) * 2 * k * k * T * s)
    g = _run(ctx, wl, k, ffrg.FP64)[0]
    assert abs(g - exact) / exact < 1e-12


def test_fermionic_flag_rejected_outside_finite_t(ctx):
    import paper_2412_13043_gb300 as ffrg
    wl = fi.make_d3(seed=1, n_pts=16, n_ext_p=8, n_rad=8, n_ang=4)
    wl.problem.statistics = fi.STAT_FERMI
    tabs = ctx.tables(wl.problem, wl.tables)
    with pytest.raises(ffrg.FfrgError):
        ctx.rhs(wl.problem, tabs, 1.0)
    tabs.free()


# ----------------------------------------------------------------------------- errors
# ----------------------------------------------------------------------------- maximum sizes
def test_d3_maximum_table_and_rule_sizes(ctx):
    """4096-point tables (the largest table), 4096 radial and 1024 angle nodes
    (the largest rules) in one RHS."""
    wl = fi.make_d3(seed=21, n_pts=4096, n_ext_p=4, n_rad=4096, n_ang=1024)
    _check(ctx, wl, 0.7)


def test_d4_maximum_angle_rules(ctx):
    """1024 x 1024 angle nodes per radial node (512 packed pairs in the FP32
    three-point loop)."""
    wl = fi.make_d4(seed=22, n_pts=16, n_ext_ang=1, n_rad=2, n_ang1=1024, n_ang2=1024)
    wl.problem.n_ext_p = 1
    _check(ctx, wl, 1.1)


def test_finite_t_maximum_matsubara_count(ctx):
    """N = 4096 (8193 loop frequencies, 4097 stack rows) with the smallest tables."""
    wl = fi.make_finite_t(seed=23, N=4096, T=0.002, n_pts=2, n_ext_p=1, n_ext_m=1, n_rad=2, n_ang=2)
    _check(ctx, wl, 0.5)


def test_fp64_tables_beyond_shared_memory_read_from_l2(ctx):
    """A stack larger than shared memory (4097 rows x 8 points: 524 KB in
    FP64) runs in the FP64 kernels with the tables read in place from global
    memory (L2) and matches the oracle; the mixed kernels, whose FP32 rows are
    addressed in shared memory (262 KB here), refuse it before any launch."""
    import torch

    import paper_2412_13043_gb300 as ffrg
    wl = fi.make_finite_t(seed=24, N=4096, T=0.002, n_pts=8, n_ext_p=1, n_ext_m=1, n_rad=2, n_ang=2)
    ref = oracle.rhs(wl.problem, wl.tables, 0.5)
    got = _run(ctx, wl, 0.5, ffrg.FP64)
    assert np.max(rel_err(got, ref)) < FP64_TOL
    tabs = ctx.tables(wl.problem, wl.tables)
    out = torch.empty(wl.problem.n_ext(), dtype=torch.float64, device="cuda")
    with pytest.raises(ffrg.FfrgError):
        ctx.rhs(wl.problem, tabs, 0.5, out=out, precision=ffrg.MIXED)
    assert ctx.status_read() == ffrg.OK
    tabs.free()


@pytest.mark.parametrize("fermionic", [False, True])
def test_finite_t_fp64_stack_of_the_serving_mix_beyond_shared_memory(ctx, fermionic):
    """N = 64 with 256-point tables (a request of the serving mix): 73 rows x
    256 points x 2 tables = 299 KB in FP64, read from L2 by the FP64 kernels;
    the mixed kernels stage it (150 KB of FP32 pairs)."""
    wl = fi.make_finite_t(seed=25, N=64, T=0.0002, n_pts=256, n_ext_p=3, n_ext_m=9, n_rad=16, n_ang=8,
                          fermionic=fermionic)
    for k in (1.0, 0.05):
        _check(ctx, wl, k)


def test_nonfinite_table_sets_status(ctx):
    import paper_2412_13043_gb300 as ffrg
    wl = fi.make_d3(seed=1, n_pts=16, n_ext_p=8, n_rad=8, n_ang=4)
    wl.tables[0, 0, 12] = float("nan")       # node near 1.7: reached by q in [0, 4k] at k = 1
    tabs = ctx.tables(wl.problem, wl.tables)
    ctx.rhs(wl.problem, tabs, 1.0)
    assert ctx.status_read() == ffrg.ENONFINITE
    assert ctx.status_read() == ffrg.OK           # cleared after reading
    tabs.free()


def test_invalid_arguments_rejected(ctx):
    import paper_2412_13043_gb300 as ffrg
    wl = fi.make_d3(seed=1, n_pts=16, n_ext_p=8, n_rad=8, n_ang=4)
    tabs = ctx.tables(wl.problem, wl.tables)
    with pytest.raises(ffrg.FfrgError) as ei:
        ctx.rhs(wl.problem, tabs, -1.0)
    assert ei.value.code == ffrg.EINVAL
    bad = fi.make_d4(n_pts=16).problem          # needs 3 tables, the upload has 1
    with pytest.raises((ffrg.FfrgError, ValueError)):
        ctx.rhs(bad, tabs, 1.0)
    tabs.free()


def test_repeat_is_bitwise_deterministic(ctx):
    import paper_2412_13043_gb300 as ffrg
    wl = fi.make_d4(seed=4, n_pts=32, n_ext_ang=4, n_rad=24, n_ang1=16, n_ang2=8)
    a = _run(ctx, wl, 0.9, ffrg.MIXED)
    b = _run(ctx, wl, 0.9, ffrg.MIXED)
    assert np.array_equal(a, b)


def test_finite_t_single_launch_near_pole(ctx):
    """The single-launch finite-T RHS (1248 K-row items) at w = m^2/k^2 =
    -0.999 with Z = 1: the n = 0 denominators cancel to ~1e-3 k^2, so the
    mixed K rows recompute those propagators in FP64 from the block's own
    q and p; every output against the oracle."""
    wl = fi.make_finite_t(seed=64, N=8, T=0.05, n_pts=16, n_ext_p=52, n_ext_m=4, n_rad=64, n_ang=4)
    wl.tables[0] = 1.0
    wl.problem.m2_over_k2 = -0.999
    for k in (1.0, 0.3):
        _check(ctx, wl, k)


def test_finite_t_single_launch_falls_back_when_momenta_exceed_shared_memory(ctx):
    """60000 external momenta (240 KB of FP32 p_i per block) with 1.2e5 K-row
    items: too large for the single launch's shared memory, so the three
    launches run; sampled outputs against the oracle."""
    wl = fi.make_finite_t(seed=65, N=1, T=0.05, n_pts=8, n_ext_p=60000, n_ext_m=1, n_rad=2, n_ang=2)
    sel = [0, 1, 7, 12345, 29999, 45678, 59998, 59999]
    _check(ctx, wl, 0.8, sel=sel)


def test_rhs_host_outputs_equal_device_outputs(ctx):
    """ffrg_rhs_host: the same kernels; into pinned memory (also a view that
    starts inside a pinned block) the kernels write the outputs directly,
    into pageable memory through the context's device buffer and a copy.
    Both bitwise equal to ffrg_rhs, for every kernel that writes outputs (d=3,
    d=4, the finite-T contraction of the three-launch and single-launch forms,
    the 4D-regulator kernel); a larger problem after a smaller one grows the
    context's device buffer."""
    import torch

    import paper_2412_13043_gb300 as ffrg
    for wl, k in ((fi.make_d3(seed=5, n_pts=16, n_ext_p=7, n_rad=8, n_ang=6), 0.8),
                  (fi.make_d4(seed=6, n_pts=32, n_ext_ang=3, n_rad=16, n_ang1=8, n_ang2=4), 0.6),
                  (fi.make_finite_t(seed=7, N=3, T=0.05, n_pts=16, n_ext_p=9, n_ext_m=2, n_rad=16, n_ang=6), 0.9),
                  (fi.make_finite_t(seed=61, N=8, T=0.05, n_pts=16, n_ext_p=52, n_ext_m=4, n_rad=64, n_ang=4), 1.1),
                  (fi.make_finite_t_4d(seed=8, N=3, T=0.05, n_pts=16, n_ext_p=6, n_ext_m=2, n_rad=16, n_ang=8,
                                       n_x0=8), 1.2)):
        tabs = ctx.tables(wl.problem, wl.tables)
        n = wl.problem.n_ext()
        for prec in (ffrg.FP64, ffrg.MIXED):
            dev = ctx.rhs(wl.problem, tabs, k, precision=prec).cpu().numpy()
            pinned = torch.empty(n, dtype=torch.float64).pin_memory()
            ctx.rhs_host(wl.problem, tabs, k, out=pinned, precision=prec)
            block = torch.full((n + 5,), -1.0, dtype=torch.float64).pin_memory()
            ctx.rhs_host(wl.problem, tabs, k, out=block[5:], precision=prec)
            torch.cuda.synchronize()
            pageable = ctx.rhs_host(wl.problem, tabs, k, precision=prec)
            assert np.array_equal(pinned.numpy(), dev) and np.array_equal(pageable, dev)
            assert np.array_equal(block[5:].numpy(), dev) and np.all(block[:5].numpy() == -1.0)
        tabs.free()
    with pytest.raises(ValueError):
        ctx.rhs_host(wl.problem, tabs, 0.5, out=np.empty(3))


def test_finite_t_single_launch_counters_across_calls_and_shapes(ctx):
    """With at least 1216 K-row items (here 1248 and 1260: (N + M) n_p x two
    radial chunks) the mixed finite-T RHS runs as one cooperative launch whose
    grid counters persist in the plan: many calls in a row, alternating
    between two plans and two scales, give bitwise the same outputs each time,
    equal to the oracle within the mixed bound."""
    import paper_2412_13043_gb300 as ffrg
    w1 = fi.make_finite_t(seed=61, N=8, T=0.05, n_pts=16, n_ext_p=52, n_ext_m=4, n_rad=64, n_ang=4)
    w2 = fi.make_finite_t(seed=62, N=6, T=0.1, n_pts=12, n_ext_p=70, n_ext_m=3, n_rad=40, n_ang=3, fermionic=True)
    first = {}
    for it in range(6):
        for name, wl in (("b", w1), ("f", w2)):
            for k in (1.1, 0.3):
                got = _run(ctx, wl, k, ffrg.MIXED)
                key = (name, k)
                if key not in first:
                    first[key] = got
                    ref = oracle.rhs(wl.problem, wl.tables, k)
                    assert np.max(np.abs(got - ref) / np.abs(ref)) < MIXED_TOL, key
                else:
                    assert np.array_equal(got, first[key]), (it, key)


@pytest.mark.parametrize("case", ["d3", "d4", "d4_full", "finite_t_three_launches", "finite_t_single_launch",
                                  "finite_t_4d"])
def test_back_to_back_calls_equal_synchronised_calls(ctx, case):
    """The main kernel is launched as the precompute kernel's programmatic
    dependent: its CTAs start while the precompute kernel runs and wait for
    its writes.  RHS calls at alternating scales and precisions issued back to
    back on one stream, with no synchronisation between them, give bitwise the
    outputs of the same calls made one at a time; so do they with profiling
    events between the two kernels (which keep the main kernel from starting
    early)."""
    import torch

    import paper_2412_13043_gb300 as ffrg
    wl = {"d3": lambda: fi.make_d3(seed=71, n_pts=24, n_ext_p=40, n_rad=37, n_ang=9),
          "d4": lambda: fi.make_d4(seed=72, n_pts=20, n_ext_ang=3, n_rad=19, n_ang1=9, n_ang2=5),
          "d4_full": lambda: fi.make_d4_full(seed=73, n_pts=12, n_va=3, n_vb=4, n_ext_ang=2, n_rad=9, n_ang1=7,
                                             n_ang2=3),
          "finite_t_three_launches": lambda: fi.make_finite_t(seed=74, N=4, T=0.05, n_pts=16, n_ext_p=20, n_ext_m=3,
                                                              n_rad=24, n_ang=8),
          "finite_t_single_launch": lambda: fi.make_finite_t(seed=61, N=8, T=0.05, n_pts=16, n_ext_p=52, n_ext_m=4,
                                                             n_rad=64, n_ang=4),
          "finite_t_4d": lambda: fi.make_finite_t_4d(seed=75, N=4, T=0.05, n_pts=16, n_ext_p=12)}[case]()
    pb = wl.problem
    tabs = ctx.tables(pb, wl.tables)
    calls = [(k, prec) for k in (1.3, 0.4, 2.0) for prec in (ffrg.MIXED, ffrg.FP64)]
    ref = {}
    for key in calls:
        o = ctx.rhs(pb, tabs, key[0], precision=key[1])
        torch.cuda.synchronize()
        ref[key] = o.cpu().numpy()
    for prof in (False, True):
        ctx.set_profiling(prof)
        outs = [(key, ctx.rhs(pb, tabs, key[0], precision=key[1])) for _ in range(3) for key in calls]
        torch.cuda.synchronize()
        if prof:
            ctx.profile_read()
            ctx.set_profiling(False)
        for key, o in outs:
            assert np.array_equal(o.cpu().numpy(), ref[key]), (case, prof, key)
    assert ctx.status_read() == ffrg.OK
    tabs.free()
