"""Stored FP64 oracle values (tests/golden/oracle_rhs_small.txt, written by
tests/golden/make_golden.py from the oracle alone): the oracle still computes
them (any change of its arithmetic shows here), and the GPU path matches them
in FP64 and in mixed precision."""
import importlib.util
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "oracle_rhs_small.txt")


def _generator():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _stored():
    """{(workload, k): values by external point}"""
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, k, e, v = line.split()
            out.setdefault((name, float(k)), {})[int(e)] = float(v)
    return {key: np.array([d[i] for i in range(len(d))]) for key, d in out.items()}


def test_golden_file_covers_every_model_and_scale():
    gen = _generator()
    stored = _stored()
    names = [n for n, _ in gen.workloads()]
    assert sorted(stored) == sorted((n, k) for n in names for k in gen.SCALES)
    for (name, _), vals in stored.items():
        wl = dict(gen.workloads())[name]
        assert len(vals) == wl.problem.n_ext() and np.all(np.isfinite(vals))


def test_oracle_reproduces_stored_values():
    import oracle
    gen = _generator()
    stored = _stored()
    for name, wl in gen.workloads():
        for k in gen.SCALES:
            got = oracle.rhs(wl.problem, wl.tables, k)
            ref = stored[(name, k)]
            # libm of another host may differ in the last bits
            assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-13, (name, k)


@pytest.mark.gpu
def test_gpu_matches_stored_values():
    import paper_2412_13043_gb300 as ffrg
    from gpu_common import gpu_context
    gen = _generator()
    stored = _stored()
    ctx = gpu_context()
    try:
        for name, wl in gen.workloads():
            tabs = ctx.tables(wl.problem, wl.tables)
            for k in gen.SCALES:
                ref = stored[(name, k)]
                for prec, tol in ((ffrg.FP64, 1e-12), (ffrg.MIXED, 1e-6)):
                    got = ctx.rhs(wl.problem, tabs, k, precision=prec).cpu().numpy()
                    assert ctx.status_read() == ffrg.OK
                    err = np.max(np.abs(got - ref) / np.abs(ref))
                    assert err < tol, (name, k, prec, err)
            tabs.free()
    finally:
        ctx.close()
