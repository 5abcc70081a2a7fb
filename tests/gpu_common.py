"""Helpers shared by the GPU parity tests (comparison metrics, contexts)."""
import numpy as np
import pytest


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)


def gpu_context():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_13043_gb300 as ffrg
    return ffrg.Context(0)
