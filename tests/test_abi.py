"""C-ABI checks that need no GPU: the library loads, exports every symbol the
header declares, and its host-side logic (quadrature rules, sizes, argument
validation) behaves as documented."""
import os
import re

import numpy as np
import pytest

import ffrg_inputs as fi
import paper_2412_13043_gb300 as ffrg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    syms = []
    for name in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if name.endswith(".h"):
            text = open(os.path.join(ROOT, "include", name)).read()
            syms += re.findall(r"^FFRG_API\s+[\w\s\*]*?\b(ffrg_\w+)\s*\(", text, flags=re.M)
    return syms


def test_library_exports_every_declared_symbol():
    lib = ffrg.load()
    declared = _declared_symbols()
    assert len(declared) >= 15
    missing = [s for s in declared if not hasattr(lib, s)]
    assert not missing, missing
    # and the binding knows the signature of each one
    assert not [s for s in declared if s not in ffrg._SIGS]


@pytest.mark.parametrize("n", [1, 2, 5, 32, 64, 127, 512])
def test_host_gauss_legendre(n):
    """Library rule (long-double Newton) against the oracle's rule, which the
    pin tests tie to 40-digit Gauss-Legendre nodes and weights."""
    import oracle
    x, w = ffrg.quad_nodes(ffrg.RULE_GL, n, 0.0, 4.0)
    xr, wr = oracle.gauss_legendre(n, 0.0, 4.0)
    assert np.max(np.abs(x - xr)) < 2e-14
    assert np.max(np.abs(w - wr) / wr) < 1e-12
    assert abs(w.sum() - 4.0) < 1e-13


@pytest.mark.parametrize("n", [1, 3, 64])
def test_host_gauss_chebyshev2(n):
    from scipy.special import roots_chebyu
    x, w = ffrg.quad_nodes(ffrg.RULE_GC2, n)
    xr, wr = roots_chebyu(n)
    o = np.argsort(x)
    assert np.max(np.abs(x[o] - xr)) < 1e-14 and np.max(np.abs(w[o] - wr)) < 1e-14


def test_quad_nodes_rejects_bad_arguments():
    lib = ffrg.load()
    x = np.empty(4)
    w = np.empty(4)
    assert lib.ffrg_quad_nodes(ffrg.RULE_GL, 0, 0.0, 1.0, x.ctypes.data, w.ctypes.data) == ffrg.EINVAL
    assert lib.ffrg_quad_nodes(7, 4, 0.0, 1.0, x.ctypes.data, w.ctypes.data) == ffrg.EINVAL
    assert lib.ffrg_quad_nodes(ffrg.RULE_GL, 4, 0.0, 1.0, None, w.ctypes.data) == ffrg.EINVAL


@pytest.mark.parametrize("make", [lambda: fi.make_d3(), lambda: fi.make_d4(), lambda: fi.make_finite_t(N=32),
                                  lambda: fi.make_d3(feedback=1)])
def test_sizes_match_problem_description(make):
    wl = make()
    assert ffrg.n_ext(wl.problem) == wl.problem.n_ext()
    assert ffrg.evals(wl.problem) == float(wl.problem.evals())


def test_sizes_reject_bad_problem():
    pb = fi.make_d3().problem
    pb.model = 9
    assert ffrg.n_ext(pb) == -1
    assert ffrg.evals(pb) < 0


def test_flow_state_size():
    wl = fi.make_d3(feedback=1)
    assert ffrg.flow_state_size(wl.problem, 1) == 65
    wl = fi.make_d4(n_pts=16)
    assert ffrg.flow_state_size(wl.problem, 1) == 48
    assert ffrg.flow_state_size(wl.problem, 0) == wl.problem.n_ext()
    wl = fi.make_finite_t(N=4)
    assert ffrg.flow_state_size(wl.problem, 0) == wl.problem.n_ext()
    assert ffrg.flow_state_size(wl.problem, 1) == -1


def test_strerror_covers_codes():
    for c in range(12):
        assert ffrg.strerror(c)
    assert "unknown" in ffrg.strerror(99)


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(ffrg.FfrgError):
        ffrg.Context(0)


def test_ctypes_structs_match_the_c_header(tmp_path):
    """Every field of the binding's ctypes structures has the offset and size
    that the C compiler gives the header's struct (a mismatch would corrupt
    the arguments of every call silently)."""
    import ctypes
    import shutil
    import subprocess
    gcc = shutil.which("gcc") or shutil.which("cc")
    if not gcc:
        pytest.skip("no C compiler")
    pairs = [("ffrg_problem", ffrg.Problem), ("ffrg_table_desc", ffrg.TableDesc), ("ffrg_step_opts", ffrg.StepOpts),
             ("ffrg_flow_stats", ffrg.FlowStats), ("ffrg_serve_opts", ffrg.ServeOpts),
             ("ffrg_serve_stats", ffrg.ServeStats)]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "ffrg.h"', "int main(void) {"]
    for cname, cls in pairs:
        lines.append(f'  printf("{cname} - %zu %zu\\n", (size_t)0, sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu %zu\\n", offsetof({cname}, {fname}), '
                         f'sizeof((({cname} *)0)->{fname}));')
    lines += ["  return 0;", "}"]
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    c = {(out[i], out[i + 1]): (int(out[i + 2]), int(out[i + 3])) for i in range(0, len(out), 4)}
    for cname, cls in pairs:
        assert c[(cname, "-")][1] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            f = getattr(cls, fname)
            assert c[(cname, fname)] == (f.offset, f.size), (cname, fname)
