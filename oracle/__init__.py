"""CPU FP64 oracle for the momentum-loop RHS and its RK flow -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product library never loads it.  The C
source ``ffrg_oracle.c`` shares no code with the CUDA path; this wrapper only
marshals arguments (ctypes) and compiles the C file with gcc on first use.

Pins: every model reduces to a closed form in a special case, and with
non-constant tables away from p = 0 every RHS summand matches an independent
route to the same integral (angle substitution and adaptive quadrature, or
summands written from the model definitions over explicit 4-vectors; see
tests/test_oracle_pins.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ffrg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ENONFINITE, ESTEP_UNDERFLOW, EMAXSTEPS = range(6)


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


class _Problem(ctypes.Structure):
    _fields_ = [
        ("model", ctypes.c_int), ("regulator", ctypes.c_int),
        ("n_rad", ctypes.c_int), ("n_ang1", ctypes.c_int), ("n_ang2", ctypes.c_int),
        ("n_ext_p", ctypes.c_int), ("n_ext_ang", ctypes.c_int), ("n_matsubara", ctypes.c_int),
        ("include_p0", ctypes.c_int),
        ("n_tables", ctypes.c_int), ("n_pts", ctypes.c_int), ("n_stack", ctypes.c_int),
        ("statistics", ctypes.c_int), ("n_va", ctypes.c_int), ("n_vb", ctypes.c_int), ("n_x0", ctypes.c_int),
        ("m2_over_k2", ctypes.c_double), ("m2_shift", ctypes.c_double), ("lam", ctypes.c_double),
        ("T", ctypes.c_double), ("p_min", ctypes.c_double), ("p_max", ctypes.c_double),
        ("qmax_over_k", ctypes.c_double), ("prefactor", ctypes.c_double),
        ("x_min", ctypes.c_double), ("x_max", ctypes.c_double),
    ]


class _StepOpts(ctypes.Structure):
    _fields_ = [("t0", ctypes.c_double), ("t1", ctypes.c_double), ("dt0", ctypes.c_double),
                ("dt_min", ctypes.c_double), ("dt_max", ctypes.c_double), ("atol", ctypes.c_double),
                ("rtol", ctypes.c_double), ("max_steps", ctypes.c_long)]


class _Stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_long), ("rejects", ctypes.c_long), ("rhs_evals", ctypes.c_long)]


def build(force: bool = False) -> str:
    """Compile ffrg_oracle.c with gcc (OpenMP when available).  Returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:2] + ["-fopenmp"] + base[2:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        D, I, P = ctypes.c_double, ctypes.c_int, ctypes.POINTER
        dp = P(D)
        lib.orc_gauss_legendre.argtypes = [I, D, D, dp, dp]
        lib.orc_gauss_chebyshev2.argtypes = [I, dp, dp]
        lib.orc_reg_r.argtypes = [I, D]
        lib.orc_reg_r.restype = D
        lib.orc_reg_rdot.argtypes = [I, D]
        lib.orc_reg_rdot.restype = D
        lib.orc_lerp_log.argtypes = [dp, I, D, D, D]
        lib.orc_lerp_log.restype = D
        pp = P(_Problem)
        lib.orc_n_ext.argtypes = [pp]
        lib.orc_rhs.argtypes = [pp, dp, D, dp]
        lib.orc_rhs_subset.argtypes = [pp, dp, D, P(I), I, dp]
        lib.orc_rhs_jvp.argtypes = [pp, dp, dp, D, dp, dp]
        lib.orc_rhs_jacobian.argtypes = [pp, dp, D, dp]
        lib.orc_flow.argtypes = [pp, dp, I, D, dp, P(_StepOpts), P(_Stats)]
        lib.orc_flow_deriv.argtypes = [pp, dp, I, D, D, dp, dp]
        lib.orc_dp45_textbook.argtypes = [I, dp, P(_StepOpts), P(_Stats)]
        lib.orc_ros2_textbook.argtypes = [I, dp, P(_StepOpts), P(_Stats)]
        lib.orc_ros2_flow.argtypes = [pp, D, dp, P(_StepOpts), P(_Stats)]
        lib.orc_d4_state_jacobian.argtypes = [pp, D, D, dp, dp]
        lib.orc_ft_loop_factors.argtypes = [pp, dp, D, dp]
        lib.orc_ft_states.argtypes = [pp, dp, D, I, dp, dp]
        lib.orc_ft4_frequencies.argtypes = [pp, D, dp, dp]
        lib.orc_ft4_external_frequency.argtypes = [pp, D, I]
        lib.orc_ft4_external_frequency.restype = D
        lib.orc_abm_textbook.argtypes = [I, I, D, D, ctypes.c_long, dp, P(ctypes.c_long)]
        lib.orc_lam3_full.argtypes = [pp, dp, D, D, D]
        lib.orc_lam3_full.restype = D
        lib.orc_d4_shape.argtypes = [D, D, D, I]
        lib.orc_d4_shape.restype = D
        lib.orc_abm_flow.argtypes = [pp, dp, I, D, dp, D, D, ctypes.c_long, I, P(_Stats)]
        lib.orc_flow_state_size.argtypes = [pp, I]
        lib.orc_d3_summand.argtypes = [pp, dp, D, D, D]
        lib.orc_d3_summand.restype = D
        lib.orc_d4_summand_z.argtypes = [pp, dp, D, D, D, D]
        lib.orc_d4_summand_z.restype = D
        lib.orc_d4_summand_3.argtypes = [pp, dp, D, D, D, D, D, D]
        lib.orc_d4_summand_3.restype = D
        lib.orc_d4_summand_4.argtypes = [pp, dp, D, D, D, D]
        lib.orc_d4_summand_4.restype = D
        lib.orc_ft_summand.argtypes = [pp, dp, D, I, I, D, D]
        lib.orc_ft_summand.restype = D
        L = ctypes.c_long
        lib.orc_d3_summand_batch.argtypes = [pp, dp, D, L, dp, dp, dp]
        lib.orc_d4_summand_batch.argtypes = [I, pp, dp, D, L, dp, D, dp, dp, D, dp]
        lib.orc_num_threads.restype = I
        lib.orc_set_threads.argtypes = [I]
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _problem(pb) -> _Problem:
    c = _Problem()
    for name, _ in _Problem._fields_:
        setattr(c, name, getattr(pb, name))
    return c


def _check(code, what):
    if code != OK:
        raise OracleError(code, what)


def num_threads() -> int:
    return _load().orc_num_threads()


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def gauss_legendre(n: int, a: float = -1.0, b: float = 1.0):
    x = np.empty(n)
    w = np.empty(n)
    _check(_load().orc_gauss_legendre(n, a, b, _ptr(x), _ptr(w)), "gauss_legendre")
    return x, w


def gauss_chebyshev2(n: int):
    x = np.empty(n)
    w = np.empty(n)
    _check(_load().orc_gauss_chebyshev2(n, _ptr(x), _ptr(w)), "gauss_chebyshev2")
    return x, w


def reg_r(reg: int, x: float) -> float:
    return _load().orc_reg_r(reg, x)


def reg_rdot(reg: int, x: float) -> float:
    return _load().orc_reg_rdot(reg, x)


def lerp_log(table, xmin: float, xmax: float, s: float) -> float:
    t = _f64(table)
    return _load().orc_lerp_log(_ptr(t), t.size, xmin, xmax, s)


def rhs(pb, tables, k: float) -> np.ndarray:
    """Raw loop integrals, one per external point (layout as in the problem)."""
    lib = _load()
    c = _problem(pb)
    t = _f64(tables)
    out = np.empty(pb.n_ext())
    _check(lib.orc_rhs(ctypes.byref(c), _ptr(t), k, _ptr(out)), "rhs")
    return out


def rhs_subset(pb, tables, k: float, sel) -> np.ndarray:
    """The RHS at the external points listed in sel only."""
    lib = _load()
    c = _problem(pb)
    t = _f64(tables)
    idx = np.ascontiguousarray(np.asarray(sel, dtype=np.int32))
    out = np.empty(idx.size)
    _check(lib.orc_rhs_subset(ctypes.byref(c), _ptr(t), k, idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                              idx.size, _ptr(out)), "rhs_subset")
    return out


def rhs_jvp(pb, tables, dtables, k: float):
    lib = _load()
    c = _problem(pb)
    t, dt = _f64(tables), _f64(dtables)
    out = np.empty(pb.n_ext())
    dout = np.empty(pb.n_ext())
    _check(lib.orc_rhs_jvp(ctypes.byref(c), _ptr(t), _ptr(dt), k, _ptr(out), _ptr(dout)), "rhs_jvp")
    return out, dout


def rhs_jacobian(pb, tables, k: float) -> np.ndarray:
    lib = _load()
    c = _problem(pb)
    t = _f64(tables)
    J = np.empty((pb.n_ext(), t.size))
    _check(lib.orc_rhs_jacobian(ctypes.byref(c), _ptr(t), k, _ptr(J)), "rhs_jacobian")
    return J


def flow_state_size(pb, feedback: int) -> int:
    return _load().orc_flow_state_size(ctypes.byref(_problem(pb)), int(feedback))


def flow_deriv(pb, tables, feedback: int, Lambda: float, t: float, y) -> np.ndarray:
    lib = _load()
    c = _problem(pb)
    tab = _f64(tables)
    yy = _f64(y).copy()
    dy = np.empty_like(yy)
    _check(lib.orc_flow_deriv(ctypes.byref(c), _ptr(tab), int(feedback), Lambda, t, _ptr(yy), _ptr(dy)),
           "flow_deriv")
    return dy


def flow(pb, tables, y0, Lambda: float, t1: float, feedback: int = 0, dt0: float = 1e-3,
         dt_min: float = 1e-10, dt_max: float = 0.5, atol: float = 1e-14, rtol: float = 1e-11,
         max_steps: int = 1_000_000, t0: float = 0.0, raise_on_error: bool = True):
    """Integrate the flow state from t_+ = t0 to t1 with the oracle's DP5(4)."""
    lib = _load()
    c = _problem(pb)
    tab = _f64(tables)
    y = _f64(y0).copy()
    o = _StepOpts(t0, t1, dt0, dt_min, dt_max, atol, rtol, max_steps)
    st = _Stats()
    code = lib.orc_flow(ctypes.byref(c), _ptr(tab), int(feedback), Lambda, _ptr(y), ctypes.byref(o),
                        ctypes.byref(st))
    if raise_on_error:
        _check(code, "flow")
    return y, dict(steps=st.steps, rejects=st.rejects, rhs_evals=st.rhs_evals, status=code)


def dp45_textbook(which: int, y0, t1: float, dt0: float = 0.1, dt_min: float = 1e-12, dt_max: float = 1.0,
                  atol: float = 1e-14, rtol: float = 1e-12, max_steps: int = 1_000_000, t0: float = 0.0):
    """The oracle's DP5(4) driver on a textbook ODE (0: y'=y cos t, 1: y'=-2ty^2,
    2: harmonic oscillator)."""
    y = _f64(y0).copy()
    o = _StepOpts(t0, t1, dt0, dt_min, dt_max, atol, rtol, max_steps)
    st = _Stats()
    code = _load().orc_dp45_textbook(int(which), _ptr(y), ctypes.byref(o), ctypes.byref(st))
    return y, dict(steps=st.steps, rejects=st.rejects, rhs_evals=st.rhs_evals, status=code)


def ros2_textbook(which: int, y0, t1: float, dt0: float = 0.1, dt_min: float = 1e-12, dt_max: float = 1.0,
                  atol: float = 1e-12, rtol: float = 1e-9, max_steps: int = 1_000_000, t0: float = 0.0):
    """The oracle's ROS2 driver on a textbook ODE (see orc_ros2_textbook)."""
    y = _f64(y0).copy()
    o = _StepOpts(t0, t1, dt0, dt_min, dt_max, atol, rtol, max_steps)
    st = _Stats()
    code = _load().orc_ros2_textbook(int(which), _ptr(y), ctypes.byref(o), ctypes.byref(st))
    return y, dict(steps=st.steps, rejects=st.rejects, jacobians=st.rhs_evals, status=code)


def lam3_full(pb, tables, s1: float, s2: float, s3: float) -> float:
    """lambda3 of the D4_FULL model at a vertex with squared leg magnitudes s1, s2, s3."""
    return _load().orc_lam3_full(ctypes.byref(_problem(pb)), _ptr(_f64(tables)), s1, s2, s3)


def d4_shape(s1: float, s2: float, s3: float):
    """(a, b) shape variables of a vertex with squared leg magnitudes s1, s2, s3."""
    lib = _load()
    return lib.orc_d4_shape(s1, s2, s3, 0), lib.orc_d4_shape(s1, s2, s3, 1)


def abm_textbook(which: int, order: int, y0, t1: float, n: int, t0: float = 0.0):
    """Adams-Bashforth-Moulton (PECE, order 2..5, RK4 start) in n fixed steps on a
    textbook ODE (0-2 as dp45_textbook, 3: y' = 4 t^3)."""
    y = _f64(y0).copy()
    ev = ctypes.c_long()
    _check(_load().orc_abm_textbook(int(which), int(order), t0, t1, int(n), _ptr(y), ctypes.byref(ev)),
           "abm_textbook")
    return y, ev.value


def abm_flow(pb, tables, y0, Lambda: float, t1: float, n: int, order: int = 4, feedback: int = 0,
             t0: float = 0.0):
    """ABM flow of the state from t_+ = t0 to t1 in n fixed steps."""
    y = _f64(y0).copy()
    st = _Stats()
    _check(_load().orc_abm_flow(ctypes.byref(_problem(pb)), _ptr(_f64(tables)), int(feedback), Lambda, _ptr(y),
                                t0, t1, int(n), int(order), ctypes.byref(st)), "abm_flow")
    return y, dict(steps=st.steps, rhs_evals=st.rhs_evals)


def ft_nfreq(pb) -> int:
    """Loop frequencies of the finite-T model: 2N+1 bosonic, 2N+2 fermionic."""
    return 2 * pb.n_matsubara + 1 + (1 if pb.statistics else 0)


def ft4_frequencies(pb, k: float):
    """Loop frequencies and their weights of the 4D-regulator finite-T model at scale k."""
    n = 2 * pb.n_matsubara + 2 + pb.n_x0
    w, wt = np.empty(n), np.empty(n)
    nf = _load().orc_ft4_frequencies(ctypes.byref(_problem(pb)), k, _ptr(w), _ptr(wt))
    return w[:nf], wt[:nf]


def ft4_external_frequency(pb, k: float, m: int) -> float:
    return _load().orc_ft4_external_frequency(ctypes.byref(_problem(pb)), k, int(m))


def ft_loop_factors(pb, tables, k: float) -> np.ndarray:
    """The model's loop-side factor dR G^2 L at (loop frequency, radial node): [nfreq][n_rad]."""
    F = np.empty((ft_nfreq(pb), pb.n_rad))
    _check(_load().orc_ft_loop_factors(ctypes.byref(_problem(pb)), _ptr(_f64(tables)), k, _ptr(F)),
           "ft_loop_factors")
    return F


def ft_states(pb, tables, k: float, F) -> np.ndarray:
    """Finite-T sums of many loop-side states F[s][n - n_lo][i] with the shifted line: [S][n_ext]."""
    Fa = _f64(F).reshape(-1, ft_nfreq(pb), pb.n_rad)
    out = np.empty((Fa.shape[0], pb.n_ext()))
    _check(_load().orc_ft_states(ctypes.byref(_problem(pb)), _ptr(_f64(tables)), k, Fa.shape[0], _ptr(Fa),
                                 _ptr(out)), "ft_states")
    return out


def d4_state_jacobian(pb, Lambda: float, t: float, y) -> np.ndarray:
    """d(d_t y)/dy of the d=4 feedback state (the tables) at RG time t."""
    yy = _f64(y).copy()
    J = np.empty((yy.size, yy.size))
    _check(_load().orc_d4_state_jacobian(ctypes.byref(_problem(pb)), Lambda, t, _ptr(yy), _ptr(J)),
           "d4_state_jacobian")
    return J


def ros2_flow(pb, y0, Lambda: float, t1: float, dt0: float = 1e-2, dt_min: float = 1e-10, dt_max: float = 0.5,
              atol: float = 1e-12, rtol: float = 1e-8, max_steps: int = 1_000_000, t0: float = 0.0):
    """ROS2 flow of the d=4 feedback state (the tables) with the exact state Jacobian."""
    y = _f64(y0).copy()
    o = _StepOpts(t0, t1, dt0, dt_min, dt_max, atol, rtol, max_steps)
    st = _Stats()
    code = _load().orc_ros2_flow(ctypes.byref(_problem(pb)), Lambda, _ptr(y), ctypes.byref(o), ctypes.byref(st))
    _check(code, "ros2_flow")
    return y, dict(steps=st.steps, rejects=st.rejects, rhs_evals=st.rhs_evals)


def d3_summand(pb, tables, k, q2, s2) -> float:
    t = _f64(tables)
    return _load().orc_d3_summand(ctypes.byref(_problem(pb)), _ptr(t), k, q2, s2)


def d4_summand(block: int, pb, tables, k, q2, p2, A2, B2=0.0, C2=0.0) -> float:
    lib = _load()
    t = _f64(tables)
    c = ctypes.byref(_problem(pb))
    if block == 0:
        return lib.orc_d4_summand_z(c, _ptr(t), k, q2, p2, A2)
    if block == 1:
        return lib.orc_d4_summand_3(c, _ptr(t), k, q2, p2, A2, B2, C2)
    return lib.orc_d4_summand_4(c, _ptr(t), k, q2, p2, A2)


def ft_summand(pb, tables, k, n, m, q2, s2) -> float:
    t = _f64(tables)
    return _load().orc_ft_summand(ctypes.byref(_problem(pb)), _ptr(t), k, n, m, q2, s2)


def d3_summand_batch(pb, tables, k, q2, s2) -> np.ndarray:
    t = _f64(tables)
    q2, s2 = _f64(q2), _f64(s2)
    out = np.empty(q2.size)
    _load().orc_d3_summand_batch(ctypes.byref(_problem(pb)), _ptr(t), k, q2.size, _ptr(q2), _ptr(s2), _ptr(out))
    return out


def d4_summand_batch(block: int, pb, tables, k, q2, p2, A2, B2, C2) -> np.ndarray:
    t = _f64(tables)
    q2, A2, B2 = _f64(q2), _f64(A2), _f64(B2)
    out = np.empty(q2.size)
    _load().orc_d4_summand_batch(block, ctypes.byref(_problem(pb)), _ptr(t), k, q2.size, _ptr(q2), p2,
                                 _ptr(A2), _ptr(B2), C2, _ptr(out))
    return out
