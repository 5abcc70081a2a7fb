"""Thin Python binding of libffrg.so (the C ABI in include/ffrg.h).

Only argument marshalling lives here: every step of the momentum-loop RHS,
the adjoint, the flow and serving runs in the library's CUDA kernels.  PyTorch
supplies device memory (tensors) and streams.  There is no CPU fallback: if
the shared library is missing or cannot be loaded, importing the binding's
compute entry points raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libffrg.so")

(OK, EINVAL, ENOMEM, ENONFINITE, ESTEP_UNDERFLOW, EMAXSTEPS, ETIMEOUT, EPENDING, EBUSY, ECUDA, ENOTFOUND,
 ECANCELED) = range(12)
FP64, MIXED = 0, 1
RULE_GL, RULE_GC2 = 0, 1
REG_EXP, REG_LITIM = 0, 1
MODEL_D3, MODEL_D4_VERTEX, MODEL_FINITE_T, MODEL_D4_FULL, MODEL_FINITE_T_4D = 1, 2, 3, 4, 5
STAT_BOSE, STAT_FERMI = 0, 1


class FfrgError(RuntimeError):
    def __init__(self, code: int, what: str, detail: str = ""):
        msg = f"{what}: {strerror(code) if _lib else code} (status {code})"
        if detail:
            msg += f" [{detail}]"
        super().__init__(msg)
        self.code = code


class Problem(ctypes.Structure):
    _fields_ = [
        ("model", ctypes.c_int), ("regulator", ctypes.c_int),
        ("n_rad", ctypes.c_int), ("n_ang1", ctypes.c_int), ("n_ang2", ctypes.c_int),
        ("n_ext_p", ctypes.c_int), ("n_ext_ang", ctypes.c_int), ("n_matsubara", ctypes.c_int),
        ("include_p0", ctypes.c_int), ("statistics", ctypes.c_int),
        ("m2_over_k2", ctypes.c_double), ("m2_shift", ctypes.c_double), ("lam", ctypes.c_double),
        ("T", ctypes.c_double), ("p_min", ctypes.c_double), ("p_max", ctypes.c_double),
        ("qmax_over_k", ctypes.c_double), ("prefactor", ctypes.c_double),
        ("n_va", ctypes.c_int), ("n_vb", ctypes.c_int), ("n_x0", ctypes.c_int),
    ]


class TableDesc(ctypes.Structure):
    _fields_ = [("n_tables", ctypes.c_int), ("n_stack", ctypes.c_int), ("n_pts", ctypes.c_int),
                ("reserved0", ctypes.c_int), ("x_min", ctypes.c_double), ("x_max", ctypes.c_double)]


class StepOpts(ctypes.Structure):
    _fields_ = [("t0", ctypes.c_double), ("t1", ctypes.c_double), ("dt0", ctypes.c_double),
                ("dt_min", ctypes.c_double), ("dt_max", ctypes.c_double), ("atol", ctypes.c_double),
                ("rtol", ctypes.c_double), ("max_steps", ctypes.c_longlong)]


class FlowStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_longlong), ("rejects", ctypes.c_longlong), ("rhs_evals", ctypes.c_longlong),
                ("integrand_evals", ctypes.c_double), ("t_reached", ctypes.c_double),
                ("jac_evals", ctypes.c_longlong)]


class ServeOpts(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int), ("max_queue", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_size_t)]


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("admitted", ctypes.c_longlong),
                ("completed", ctypes.c_longlong), ("cancelled", ctypes.c_longlong),
                ("rejected", ctypes.c_longlong), ("ticks", ctypes.c_longlong),
                ("resident", ctypes.c_int), ("queued", ctypes.c_int), ("peak_resident", ctypes.c_int),
                ("reserved0", ctypes.c_int), ("hbm_in_use", ctypes.c_size_t)]


_lib = None

# name -> (restype, argtypes)
_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_SIGS = {
    "ffrg_create": (_I, [ctypes.POINTER(_P), _I, ctypes.c_size_t]),
    "ffrg_destroy": (_I, [_P]),
    "ffrg_quad_nodes": (_I, [_I, _I, _D, _D, _P, _P]),
    "ffrg_tables_upload": (_I, [_P, ctypes.POINTER(TableDesc), _P, _I, ctypes.POINTER(_P), _P]),
    "ffrg_tables_update": (_I, [_P, _P, _P, _I, _P]),
    "ffrg_tables_free": (_I, [_P, _P]),
    "ffrg_tables_device_ptr": (_I, [_P, ctypes.POINTER(_P)]),
    "ffrg_n_ext": (_I, [ctypes.POINTER(Problem)]),
    "ffrg_evals": (_D, [ctypes.POINTER(Problem)]),
    "ffrg_rhs": (_I, [_P, ctypes.POINTER(Problem), _P, _D, _P, _I, _P]),
    "ffrg_rhs_host": (_I, [_P, ctypes.POINTER(Problem), _P, _D, _P, _I, _P]),
    "ffrg_rhs_noalloc": (_I, [ctypes.POINTER(Problem), ctypes.POINTER(TableDesc), _P, _D, _P, _I, _P]),
    "ffrg_rhs_adjoint": (_I, [_P, ctypes.POINTER(Problem), _P, _D, _P, _P, _I, _P]),
    "ffrg_ft_states": (_I, [_P, ctypes.POINTER(Problem), _P, _D, _I, _P, _P, _I, _P]),
    "ffrg_flow": (_I, [_P, ctypes.POINTER(Problem), _P, _I, _D, _P, ctypes.POINTER(StepOpts), _I,
                       ctypes.POINTER(FlowStats), _P]),
    "ffrg_rhs_jacobian": (_I, [_P, ctypes.POINTER(Problem), _P, _D, _P, _P]),
    "ffrg_abm_flow": (_I, [_P, ctypes.POINTER(Problem), _P, _I, _D, _P, _D, _D, ctypes.c_longlong, _I, _I,
                           ctypes.POINTER(FlowStats), _P]),
    "ffrg_rosenbrock_flow": (_I, [_P, ctypes.POINTER(Problem), _P, _D, _P, ctypes.POINTER(StepOpts),
                                  ctypes.POINTER(FlowStats), _P]),
    "ffrg_flow_state_size": (_I, [ctypes.POINTER(Problem), ctypes.POINTER(TableDesc), _I]),
    "ffrg_status_read": (_I, [_P, _P]),
    "ffrg_set_profiling": (_I, [_P, _I]),
    "ffrg_profile_read": (_I, [_P, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_longlong)]),
    "ffrg_serve_start": (_I, [_P, ctypes.POINTER(ServeOpts)]),
    "ffrg_serve_submit": (_I, [_P, ctypes.POINTER(Problem), ctypes.POINTER(TableDesc), _P, _P, _D,
                               ctypes.POINTER(StepOpts), ctypes.POINTER(ctypes.c_ulonglong)]),
    "ffrg_serve_poll": (_I, [_P, ctypes.c_ulonglong, _P, ctypes.POINTER(FlowStats), ctypes.POINTER(_D)]),
    "ffrg_serve_cancel": (_I, [_P, ctypes.c_ulonglong]),
    "ffrg_serve_get_stats": (_I, [_P, ctypes.POINTER(ServeStats)]),
    "ffrg_serve_stop": (_I, [_P]),
    "ffrg_strerror": (ctypes.c_char_p, [_I]),
    "ffrg_last_error": (ctypes.c_char_p, [_P]),
}


def load(path: Optional[str] = None):
    """Load libffrg.so (building it in-tree first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _build
    p = path or LIB_PATH
    if path is None and not _build.up_to_date():
        _build.build()
    if not os.path.exists(p):
        raise RuntimeError(f"libffrg.so not found at {p}; the CUDA library is required (no CPU fallback)")
    lib = ctypes.CDLL(p)
    for name, (res, args) in _SIGS.items():
        if hasattr(lib, name):
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    lib = load()
    return [n for n in _SIGS if hasattr(lib, n)]


def strerror(code: int) -> str:
    return load().ffrg_strerror(int(code)).decode()


def _check(ctx_handle, code: int, what: str):
    if code != OK:
        detail = ""
        if ctx_handle:
            try:
                detail = load().ffrg_last_error(ctx_handle).decode()
            except Exception:  # pragma: no cover - best effort detail
                detail = ""
        raise FfrgError(code, what, detail)


def to_problem(pb) -> Problem:
    """Build the C struct from any object with the problem's attribute names."""
    c = Problem()
    for name, _ in Problem._fields_:
        default = {"statistics": 0, "n_va": 1, "n_vb": 1, "n_x0": 0}
        setattr(c, name, getattr(pb, name, default[name]) if name in default else getattr(pb, name))
    return c


def to_desc(pb) -> TableDesc:
    return TableDesc(pb.n_tables, pb.n_stack, pb.n_pts, 0, pb.x_min, pb.x_max)


def n_ext(pb) -> int:
    return load().ffrg_n_ext(ctypes.byref(to_problem(pb)))


def evals(pb) -> float:
    return load().ffrg_evals(ctypes.byref(to_problem(pb)))


def quad_nodes(rule: int, n: int, a: float = -1.0, b: float = 1.0):
    x = np.empty(n)
    w = np.empty(n)
    code = load().ffrg_quad_nodes(rule, n, a, b, x.ctypes.data, w.ctypes.data)
    _check(None, code, "ffrg_quad_nodes")
    return x, w


def _stream_handle(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _dev_ptr(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    return t.data_ptr()


class Tables:
    """Device dressing tables owned by the library."""

    def __init__(self, ctx: "Context", handle: int, desc: TableDesc, shape):
        self.ctx = ctx
        self.handle = handle
        self.desc = desc
        self.shape = shape

    def update(self, values, stream=None):
        """Overwrite the values: CUDA tensor (device copy), pinned CPU tensor
        (asynchronous host-to-device copy; keep it alive until the stream has
        passed), or any other host array (copied, then the stream is synchronised)."""
        lib = load()
        sh = _stream_handle(stream)
        if hasattr(values, "is_cuda") and values.is_cuda:
            code = lib.ffrg_tables_update(self.ctx.handle, self.handle, _dev_ptr(values, "values"), 1, sh)
        elif hasattr(values, "is_pinned") and values.is_pinned() and values.is_contiguous():
            import torch
            if values.dtype != torch.float64:
                raise ValueError("values must be float64")
            code = lib.ffrg_tables_update(self.ctx.handle, self.handle, values.data_ptr(), 0, sh)
        else:
            v = np.ascontiguousarray(np.asarray(values.cpu() if hasattr(values, "cpu") else values,
                                                dtype=np.float64))
            code = lib.ffrg_tables_update(self.ctx.handle, self.handle, v.ctypes.data, 0, sh)
            if code == OK:
                import torch
                torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        _check(self.ctx.handle, code, "ffrg_tables_update")

    def device_ptr(self) -> int:
        p = _P()
        _check(None, load().ffrg_tables_device_ptr(self.handle, ctypes.byref(p)), "ffrg_tables_device_ptr")
        return p.value

    def free(self):
        if self.handle:
            load().ffrg_tables_free(self.ctx.handle, self.handle)
            self.handle = None


class Context:
    """One library context on one CUDA device (use one per concurrent stream)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        lib = load()
        h = _P()
        code = lib.ffrg_create(ctypes.byref(h), device, hbm_budget_bytes)
        _check(None, code, "ffrg_create")
        self.handle = h.value
        self.device = device

    def close(self):
        if self.handle:
            load().ffrg_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tables(self, pb, values, stream=None) -> Tables:
        """Upload tables (host numpy array or CUDA float64 tensor)."""
        lib = load()
        desc = to_desc(pb)
        h = _P()
        if hasattr(values, "is_cuda") and values.is_cuda:
            code = lib.ffrg_tables_upload(self.handle, ctypes.byref(desc), _dev_ptr(values, "values"), 1,
                                          ctypes.byref(h), _stream_handle(stream))
            shape = tuple(values.shape)
        else:
            v = np.ascontiguousarray(np.asarray(values, dtype=np.float64))
            code = lib.ffrg_tables_upload(self.handle, ctypes.byref(desc), v.ctypes.data, 0, ctypes.byref(h),
                                          _stream_handle(stream))
            shape = v.shape
            if code == OK:
                import torch
                (torch.cuda.current_stream() if stream is None else stream).synchronize()
        _check(self.handle, code, "ffrg_tables_upload")
        return Tables(self, h.value, desc, shape)

    def rhs(self, pb, tables: Tables, k: float, out=None, precision: int = FP64, stream=None):
        """One RHS into a CUDA float64 tensor (allocated when out is None)."""
        import torch
        c = to_problem(pb)
        ne = load().ffrg_n_ext(ctypes.byref(c))
        if ne < 0:
            raise ValueError("bad problem")
        if out is None:
            out = torch.empty(ne, dtype=torch.float64, device=f"cuda:{self.device}")
        code = load().ffrg_rhs(self.handle, ctypes.byref(c), tables.handle, float(k), _dev_ptr(out, "out"),
                               int(precision), _stream_handle(stream))
        _check(self.handle, code, "ffrg_rhs")
        return out

    def rhs_host(self, pb, tables: Tables, k: float, out=None, precision: int = FP64, stream=None):
        """One RHS with the outputs in host memory (ffrg_rhs_host): `out` a
        contiguous float64 CPU tensor (pinned: the kernels write into it
        asynchronously, synchronise the stream before reading) or numpy array;
        allocated as a numpy array (pageable: the call returns after the copy)
        when None."""
        c = to_problem(pb)
        ne = load().ffrg_n_ext(ctypes.byref(c))
        if ne < 0:
            raise ValueError("bad problem")
        if out is None:
            out = np.empty(ne, dtype=np.float64)
        if hasattr(out, "is_cuda"):
            import torch
            if out.is_cuda or out.dtype != torch.float64 or not out.is_contiguous() or out.numel() != ne:
                raise ValueError("out must be a contiguous float64 CPU tensor of n_ext values")
            ptr = out.data_ptr()
        else:
            if out.dtype != np.float64 or not out.flags["C_CONTIGUOUS"] or out.size != ne:
                raise ValueError("out must be a contiguous float64 array of n_ext values")
            ptr = out.ctypes.data
        code = load().ffrg_rhs_host(self.handle, ctypes.byref(c), tables.handle, float(k), ptr, int(precision),
                                    _stream_handle(stream))
        _check(self.handle, code, "ffrg_rhs_host")
        return out

    def rhs_adjoint(self, pb, tables: Tables, k: float, gbar, tbar=None, precision: int = FP64, stream=None):
        import torch
        c = to_problem(pb)
        if tbar is None:
            n = tables.desc.n_tables * tables.desc.n_stack * tables.desc.n_pts
            tbar = torch.empty(n, dtype=torch.float64, device=f"cuda:{self.device}")
        code = load().ffrg_rhs_adjoint(self.handle, ctypes.byref(c), tables.handle, float(k),
                                       _dev_ptr(gbar, "gbar"), _dev_ptr(tbar, "tbar"), int(precision),
                                       _stream_handle(stream))
        _check(self.handle, code, "ffrg_rhs_adjoint")
        return tbar

    def ft_states(self, pb, tables: Tables, k: float, F, out=None, precision: int = FP64, stream=None):
        """Finite-T sums of the loop-side states F (CUDA float64 [S, nfreq, n_rad]) against the
        angle-integrated kernel of `tables`: a CUDA float64 tensor [S, n_ext]."""
        import torch
        c = to_problem(pb)
        n_states = int(F.shape[0])
        if out is None:
            out = torch.empty(n_states, load().ffrg_n_ext(ctypes.byref(c)), dtype=torch.float64,
                              device=f"cuda:{self.device}")
        code = load().ffrg_ft_states(self.handle, ctypes.byref(c), tables.handle, float(k), n_states,
                                     _dev_ptr(F, "F"), _dev_ptr(out, "out"), int(precision), _stream_handle(stream))
        _check(self.handle, code, "ffrg_ft_states")
        return out

    def flow(self, pb, tables: Tables, state, Lambda: float, t1: float, feedback: int = 0, precision: int = FP64,
             t0: float = 0.0, dt0: float = 1e-3, dt_min: float = 1e-10, dt_max: float = 0.5, atol: float = 1e-14,
             rtol: float = 1e-11, max_steps: int = 1_000_000, stream=None, raise_on_error: bool = True):
        """Integrate `state` (CUDA float64 tensor, overwritten) from t0 to t1."""
        c = to_problem(pb)
        o = StepOpts(t0, t1, dt0, dt_min, dt_max, atol, rtol, max_steps)
        st = FlowStats()
        code = load().ffrg_flow(self.handle, ctypes.byref(c), tables.handle, int(feedback), float(Lambda),
                                _dev_ptr(state, "state"), ctypes.byref(o), int(precision), ctypes.byref(st),
                                _stream_handle(stream))
        if raise_on_error:
            _check(self.handle, code, "ffrg_flow")
        return dict(steps=st.steps, rejects=st.rejects, rhs_evals=st.rhs_evals, jac_evals=st.jac_evals,
                    integrand_evals=st.integrand_evals, t_reached=st.t_reached, status=code)

    # ---- serving (continuous batching of flow requests) ----
    def serve_start(self, max_slots: int = 64, max_queue: int = 4096, hbm_budget_bytes: int = 0):
        o = ServeOpts(max_slots, max_queue, hbm_budget_bytes)
        _check(self.handle, load().ffrg_serve_start(self.handle, ctypes.byref(o)), "ffrg_serve_start")

    def serve_submit(self, pb, tables, y0, Lambda: float, t1: float, t0: float = 0.0, dt0: float = 1e-3,
                     dt_min: float = 1e-10, dt_max: float = 0.5, atol: float = 1e-14, rtol: float = 1e-11,
                     max_steps: int = 1_000_000) -> int:
        """Queue a frozen-background flow request; returns its ticket (inputs are copied)."""
        t = np.ascontiguousarray(np.asarray(tables, dtype=np.float64))
        y = np.ascontiguousarray(np.asarray(y0, dtype=np.float64))
        c, d = to_problem(pb), to_desc(pb)
        o = StepOpts(t0, t1, dt0, dt_min, dt_max, atol, rtol, max_steps)
        tk = ctypes.c_ulonglong()
        code = load().ffrg_serve_submit(self.handle, ctypes.byref(c), ctypes.byref(d), t.ctypes.data, y.ctypes.data,
                                        float(Lambda), ctypes.byref(o), ctypes.byref(tk))
        _check(self.handle, code, "ffrg_serve_submit")
        return tk.value

    def serve_poll(self, ticket: int, n_out: int):
        """(status, result or None, stats dict, latency_s); status EPENDING while running."""
        out = np.empty(n_out)
        st = FlowStats()
        lat = _D()
        code = load().ffrg_serve_poll(self.handle, ticket, out.ctypes.data, ctypes.byref(st), ctypes.byref(lat))
        if code == EPENDING:
            return code, None, None, None
        stats = dict(steps=st.steps, rejects=st.rejects, rhs_evals=st.rhs_evals,
                     integrand_evals=st.integrand_evals, t_reached=st.t_reached)
        return code, (out if code in (OK,) else None), stats, lat.value

    def serve_cancel(self, ticket: int) -> int:
        return load().ffrg_serve_cancel(self.handle, ticket)

    def serve_stats(self) -> dict:
        s = ServeStats()
        _check(self.handle, load().ffrg_serve_get_stats(self.handle, ctypes.byref(s)), "ffrg_serve_get_stats")
        return {name: getattr(s, name) for name, _ in ServeStats._fields_ if name != "reserved0"}

    def serve_stop(self) -> int:
        return load().ffrg_serve_stop(self.handle)

    def set_profiling(self, enable: bool) -> None:
        _check(self.handle, load().ffrg_set_profiling(self.handle, int(bool(enable))), "ffrg_set_profiling")

    def profile_read(self):
        """(summed main-kernel milliseconds, launches) since profiling was enabled or last read."""
        ms = _D()
        n = ctypes.c_longlong()
        _check(self.handle, load().ffrg_profile_read(self.handle, ctypes.byref(ms), ctypes.byref(n)),
               "ffrg_profile_read")
        return ms.value, n.value

    def rhs_jacobian(self, pb, tables: Tables, k: float, J=None, stream=None):
        """d out_e / d T_j as a CUDA float64 tensor [n_ext, table values]."""
        import torch
        c = to_problem(pb)
        n = tables.desc.n_tables * tables.desc.n_stack * tables.desc.n_pts
        if J is None:
            J = torch.empty(load().ffrg_n_ext(ctypes.byref(c)), n, dtype=torch.float64, device=f"cuda:{self.device}")
        code = load().ffrg_rhs_jacobian(self.handle, ctypes.byref(c), tables.handle, float(k), _dev_ptr(J, "J"),
                                        _stream_handle(stream))
        _check(self.handle, code, "ffrg_rhs_jacobian")
        return J

    def rosenbrock_flow(self, pb, tables: Tables, state, Lambda: float, t1: float, t0: float = 0.0,
                        dt0: float = 1e-2, dt_min: float = 1e-10, dt_max: float = 0.5, atol: float = 1e-12,
                        rtol: float = 1e-8, max_steps: int = 1_000_000, stream=None, raise_on_error: bool = True):
        """ROS2 flow of the d=4 feedback state (CUDA float64 tensor, overwritten)."""
        c = to_problem(pb)
        o = StepOpts(t0, t1, dt0, dt_min, dt_max, atol, rtol, max_steps)
        st = FlowStats()
        code = load().ffrg_rosenbrock_flow(self.handle, ctypes.byref(c), tables.handle, float(Lambda),
                                           _dev_ptr(state, "state"), ctypes.byref(o), ctypes.byref(st),
                                           _stream_handle(stream))
        if raise_on_error:
            _check(self.handle, code, "ffrg_rosenbrock_flow")
        return dict(steps=st.steps, rejects=st.rejects, rhs_evals=st.rhs_evals, jac_evals=st.jac_evals,
                    integrand_evals=st.integrand_evals, t_reached=st.t_reached, status=code)

    def abm_flow(self, pb, tables: Tables, state, Lambda: float, t1: float, n_steps: int, order: int = 4,
                 feedback: int = 0, precision: int = FP64, t0: float = 0.0, stream=None, raise_on_error: bool = True):
        """Adams-Bashforth-Moulton flow in n_steps fixed steps (state: CUDA float64 tensor, overwritten)."""
        c = to_problem(pb)
        st = FlowStats()
        code = load().ffrg_abm_flow(self.handle, ctypes.byref(c), tables.handle, int(feedback), float(Lambda),
                                    _dev_ptr(state, "state"), float(t0), float(t1), int(n_steps), int(order),
                                    int(precision), ctypes.byref(st), _stream_handle(stream))
        if raise_on_error:
            _check(self.handle, code, "ffrg_abm_flow")
        return dict(steps=st.steps, rejects=st.rejects, rhs_evals=st.rhs_evals,
                    integrand_evals=st.integrand_evals, t_reached=st.t_reached, status=code)

    def status_read(self, stream=None) -> int:
        return load().ffrg_status_read(self.handle, _stream_handle(stream))


def flow_state_size(pb, feedback: int) -> int:
    return load().ffrg_flow_state_size(ctypes.byref(to_problem(pb)), ctypes.byref(to_desc(pb)), int(feedback))
