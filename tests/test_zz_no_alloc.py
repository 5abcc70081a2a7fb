"""ffrg_rhs_noalloc: the RHS entry point for callers that cannot allocate
device memory (for example when another allocator owns the HBM, or when
cudaMalloc's implicit synchronisation is not acceptable).  Called through the
C ABI and checked against ffrg_rhs, the allocating entry point, on two calls
in a row with different shapes (the shared scratch array must not leak state
from one call into the next).  Both run the same kernels with the same work
items and a fixed reduction order, so their outputs must agree bit for bit;
no output may carry the NaN that marks a bounded device wait that gave up.
Kept in its own file, collected last."""
import ctypes

import numpy as np
import pytest

import ffrg_inputs as fi

pytestmark = pytest.mark.gpu

def _noalloc(lib, ffrg, wl, k, precision):
    import torch
    pb = ffrg.to_problem(wl.problem)
    desc = ffrg.to_desc(wl.problem)
    tab = torch.tensor(wl.tables, dtype=torch.float64, device="cuda").contiguous()
    out = torch.full((wl.problem.n_ext(),), float("nan"), dtype=torch.float64, device="cuda")
    code = lib.ffrg_rhs_noalloc(ctypes.byref(pb), ctypes.byref(desc), tab.data_ptr(), float(k), out.data_ptr(),
                                int(precision), torch.cuda.current_stream().cuda_stream)
    assert code == ffrg.OK, ffrg.strerror(code)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _allocating(ffrg, ctx, wl, k, precision):
    tabs = ctx.tables(wl.problem, wl.tables)
    out = ctx.rhs(wl.problem, tabs, k, precision=precision).cpu().numpy()
    tabs.free()
    return out


def test_noalloc_matches_rhs_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_13043_gb300 as ffrg
    lib = ffrg.load()
    ctx = ffrg.Context(0)
    try:
        first = fi.make_d4(seed=21, n_pts=32, n_ext_ang=3, n_rad=24, n_ang1=16, n_ang2=8)
        second = fi.make_finite_t(seed=22, N=4, T=0.05, n_pts=16, n_ext_p=9, n_ext_m=3, n_rad=20, n_ang=12)
        for precision in (ffrg.FP64, ffrg.MIXED):
            for wl, k in ((first, 0.7), (second, 1.3)):       # two calls in a row, different shapes
                got = _noalloc(lib, ffrg, wl, k, precision)
                ref = _allocating(ffrg, ctx, wl, k, precision)
                assert np.all(np.isfinite(got)), (wl.problem.model, precision)
                assert np.array_equal(got, ref), (wl.problem.model, precision,
                                                  float(np.max(np.abs(got - ref) / np.abs(ref))))
    finally:
        ctx.close()


def test_noalloc_matches_the_single_launch_rhs():
    """A finite-T problem with 1248 K-row items: ffrg_rhs takes its mixed RHS
    in one cooperative launch, ffrg_rhs_noalloc in the three launches
    (precompute, K rows, contraction); the arithmetic is the same, so the
    outputs agree bit for bit."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_13043_gb300 as ffrg
    lib = ffrg.load()
    ctx = ffrg.Context(0)
    try:
        wl = fi.make_finite_t(seed=63, N=8, T=0.05, n_pts=16, n_ext_p=52, n_ext_m=4, n_rad=64, n_ang=6)
        pole = fi.make_finite_t(seed=63, N=8, T=0.05, n_pts=16, n_ext_p=52, n_ext_m=4, n_rad=64, n_ang=6)
        pole.tables[0] = 1.0                     # near the pole: FP64 recompute in the K rows
        pole.problem.m2_over_k2 = -0.999
        for w in (wl, pole):
            for k in (1.3, 0.2):
                got = _noalloc(lib, ffrg, w, k, ffrg.MIXED)
                ref = _allocating(ffrg, ctx, w, k, ffrg.MIXED)
                assert np.all(np.isfinite(got))
                assert np.array_equal(got, ref), float(np.max(np.abs(got - ref) / np.abs(ref)))
    finally:
        ctx.close()


def test_noalloc_rejects_problems_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_13043_gb300 as ffrg
    lib = ffrg.load()
    # (2N+1) x n_rad per-radial factors = 1201 x 512 doubles = 4.9 MB > 4 MiB
    wl = fi.make_finite_t(seed=23, N=600, T=0.05, n_pts=8, n_ext_p=2, n_ext_m=2, n_rad=512, n_ang=2)
    pb = ffrg.to_problem(wl.problem)
    desc = ffrg.to_desc(wl.problem)
    tab = torch.tensor(wl.tables, dtype=torch.float64, device="cuda")
    out = torch.empty(wl.problem.n_ext(), dtype=torch.float64, device="cuda")
    code = lib.ffrg_rhs_noalloc(ctypes.byref(pb), ctypes.byref(desc), tab.data_ptr(), 1.0, out.data_ptr(),
                                ffrg.FP64, torch.cuda.current_stream().cuda_stream)
    assert code == ffrg.EINVAL
