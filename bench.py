"""Benchmark of the momentum-loop RHS engine on one GB300 (or N replicas).

Workload (one "step"): one full right-hand side of the d=4 vertex-expansion
model -- 3 dressing tables on 128-point log grids, 1281 external points
(128 |p| for the propagator flow + p = 0, 128 |p| x 8 angles for the
three-point flow, 128 |p| for the four-point flow) x 131072 quadrature nodes
(128 radial x 64 Gauss-Chebyshev-II x 16 Gauss-Legendre) = 1.68e8 integrand
evaluations, in the mixed-precision path.  Inputs stay resident; L2 is
flushed between timed steps.  Extra keys: the plain FP64 path on the same
workload, the end-to-end call with host buffers, full RG flows (d=3 two-point
flow k: 10 -> 0.01, FP64 vs mixed, endpoint error), the roofline of the
dominant kernel, clocks, and the CPU oracle on the host cores.

Multi-GPU: replicas only (every rank evaluates its own RHS; no collective on
the data path); value = all ranks' evaluations / max-over-ranks time.
`--impl reference` times the CPU oracle on the same workload (a bounded
sample of external points per step).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "integrand evals/s & flows/s vs plain FP64 GPU at 1e-8 endpoint err; p50/p99 latency"
WORKLOAD = "d4 vertex-expansion RHS: 3 tables x 128 pts, 1281 ext x (128 rad x 64 GC-II x 16 GL) nodes"

# Special-function work per integrand term of the mixed d=4 kernel, from the
# integrand's formula (not from the compiled code), in units of one log2 or
# reciprocal (16 results per clock per SM); the exponential runs at twice that
# rate on this GPU (a throughput loop measured 15.1 lg2, 15.1 rcp and 29.9 ex2
# results per SM per clock), so it counts one half.  Inner term of the
# three-point diagram: 3 table coordinates (log) + 1 regulator exponential +
# 1 reciprocal (propagator N / (Z k^2 x + m^2 N)).  Per (radial, c1) row: the
# |q+p1| leg (1 log + 1 exponential + 1 reciprocal) and the row's vertex
# lookups (Z block 2, three-point block 1, lambda4 block 1 log).
SFU_INNER = 4.5
SFU_LEG = 2.5
SFU_PER_CLK_SM = 16      # log2 / reciprocal results per clock per SM
# DRAM bytes (read + write) of one rhs_main<2, float> launch on the default
# d=4 workload, from an ncu capture of the current kernel
# (dram__bytes_read.sum + dram__bytes_write.sum: 83.5 KB + 0 B)
D4_MAIN_DRAM_BYTES = 83456
FP32_PER_CLK_SM = 128    # FP32 FMA lanes per SM
# FP64-pipe thread instructions per integrand term of rhs_main<2, double> (the
# plain FP64 path), from an ncu capture of the d=4 workload with 16 external
# momenta: pipe_fp64 86.1 % of 1.077e7 active cycles x 2 per cycle x 152 SMs
# over 2.11e7 terms
FP64_OPS_PER_TERM_D4 = 134
FP64_PER_CLK_SM = 2      # FP64 (DFMA) results per clock per SM on this part


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ffrg", choices=["ffrg", "reference"])
    ap.add_argument("--no-flows", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-models", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=1024)
    ap.add_argument("--model-filter", default="",
                    help="run only the model rows whose workload name contains this text")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x of all ranks (x itself without a process group): every
    timed region is charged at its slowest rank."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: float, t_max: float) -> float:
    """Units of all ranks per second of the slowest rank (replicas: every rank
    processes units_per_rank)."""
    return world * units_per_rank / t_max


def sfu_ops_per_launch(pb):
    """Algorithmic special-function work of one d=4 RHS launch (log2 units)."""
    n_p, n_psi = pb.n_ext_p, pb.n_ext_ang
    rows = pb.n_rad * pb.n_ang1
    inner = n_p * n_psi * rows * pb.n_ang2               # three-point diagram terms
    row_units = rows * ((n_p + 1) * (SFU_LEG + 2) + n_p * n_psi * (SFU_LEG + 1) + n_p * (SFU_LEG + 1))
    return inner * SFU_INNER + row_units


class ClockSampler:
    def __init__(self, device_index: int):
        self.proc = None
        self.path = None
        self.dev = device_index

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        busy = sorted(sm)[len(sm) // 2:] if sm else []
        return {"sm_mhz": statistics.median(busy) if busy else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p))
        except ValueError:
            return {}
    return {}


def cpu_baseline(wl, stride: int, stride_1t: int = 32):
    """The CPU oracle, as it stands, on every `stride`-th external point with
    all host threads (OpenMP over external points), and on every
    `stride_1t`-th point with one thread."""
    import oracle
    pb = wl.problem

    def timed(step):
        sel = list(range(0, pb.n_ext(), step))
        t = time.perf_counter()
        oracle.rhs_subset(pb, wl.tables, 1.0, sel)
        dt = time.perf_counter() - t
        ev = len(sel) * pb.n_nodes()
        return ev / dt, f"{len(sel)} of {pb.n_ext()} external points (every {step}th) of the d4 RHS at k=1, " \
                        f"{ev:.3g} evals, {dt:.2f} s wall"

    cores = oracle.num_threads()
    v, sample = timed(stride)
    oracle.set_threads(1)
    try:
        v1, sample1 = timed(stride_1t)
    finally:
        oracle.set_threads(cores)
    return {"value": v, "unit": "integrand evals/s", "cores": cores, "kind": "oracle", "sample": sample,
            "single_thread": {"value": v1, "unit": "integrand evals/s", "cores": 1, "sample": sample1}}


def serving_bench(ctx, n_req: int, seconds_cap: float = 120.0):
    """Served mixed-precision flows (continuous batching) against the plain
    path, one flow at a time through ffrg_flow in FP64 and in mixed precision,
    on the same requests.  The launch plans of every request shape are built
    before any timing; each one-at-a-time flow is timed from its table upload
    to its result on the host, like a served request from submit to poll.
    Every served endpoint is compared with its FP64 counterpart; p50/p99
    latency under Poisson arrivals at 0.8x the measured served capacity."""
    import numpy as np
    import torch

    import ffrg_inputs as fi
    import paper_2412_13043_gb300 as ffrg
    reqs = fi.serving_stream(seed=5, n_requests=n_req)
    rtol, atol = 1e-10, 1e-13

    def t1_of(wl):
        return math.log(wl.Lambda / wl.k_end)

    for rq in reqs:                       # plans (device scratch, rules, launch geometry) per shape
        wl = rq.workload
        tabs = ctx.tables(wl.problem, wl.tables)
        for prec in (ffrg.FP64, ffrg.MIXED):
            ctx.rhs(wl.problem, tabs, wl.Lambda, precision=prec)
        torch.cuda.synchronize()
        tabs.free()

    single = {}
    for name, prec in (("fp64", ffrg.FP64), ("mixed", ffrg.MIXED)):
        outs, times, ev = [], [], 0.0
        for rq in reqs:
            wl = rq.workload
            torch.cuda.synchronize()
            t = time.perf_counter()
            tabs = ctx.tables(wl.problem, wl.tables)
            y = torch.tensor(wl.y0, dtype=torch.float64, device="cuda")
            fs = ctx.flow(wl.problem, tabs, y, wl.Lambda, t1_of(wl), precision=prec, rtol=rtol, atol=atol)
            outs.append(y.cpu().numpy())
            times.append(time.perf_counter() - t)
            tabs.free()
            ev += fs["integrand_evals"]
        single[name] = {"flows_per_s": len(outs) / sum(times), "evals_per_s": ev / sum(times), "outs": outs,
                        "p50_s": sorted(times)[len(times) // 2]}

    def run(arrivals):
        ctx.serve_start(max_slots=64, max_queue=len(reqs) + 8, hbm_budget_bytes=8 << 30)
        tick, lat, res, ev = {}, {}, {}, [0.0]
        t0 = time.perf_counter()
        i = 0
        while len(lat) < len(reqs):
            now = time.perf_counter() - t0
            while i < len(reqs) and arrivals[i] <= now:
                wl = reqs[i].workload
                tick[ctx.serve_submit(wl.problem, wl.tables, wl.y0, wl.Lambda, t1_of(wl), rtol=rtol,
                                      atol=atol)] = i
                i += 1
            for tk, j in list(tick.items()):
                st, out, fst, l = ctx.serve_poll(tk, reqs[j].workload.problem.n_ext())
                if st != ffrg.EPENDING:
                    assert st == ffrg.OK, ffrg.strerror(st)
                    ev[0] += fst["integrand_evals"]
                    lat[j] = l
                    res[j] = out
                    del tick[tk]
            if now > seconds_cap:
                raise RuntimeError("serving benchmark exceeded its time cap")
            time.sleep(0.0005)
        wall = time.perf_counter() - t0
        stats = ctx.serve_stats()
        ctx.serve_stop()
        return wall, lat, res, stats, ev[0]

    wall, lat_sat, res, stats, ev_sat = run([0.0] * len(reqs))
    capacity = len(reqs) / wall

    # Endpoint errors of a flow y(t1) = y0 - int I dt against a reference r:
    #   norm: max_i |y_i - r_i| / max_i |r_i|  (the endpoint accuracy compared)
    #   cancel: max_i |y_i - r_i| / (|y0_i| + |r_i - y0_i|), each component
    #     against the magnitudes of the two parts that can cancel (components
    #     that end near zero: y0 and the integrated flow nearly equal)
    #   elem: max_i |y_i - r_i| / |r_i|
    def endpoint_errs(y, r, y0):
        d = np.abs(y - r)
        return (float(np.max(d) / np.max(np.abs(r))), float(np.max(d / (np.abs(y0) + np.abs(r - y0)))),
                float(np.max(d / np.abs(r))))

    def errs(other):
        return np.array([endpoint_errs(res[j], single[other]["outs"][j], reqs[j].workload.y0)
                         for j in range(len(reqs))])
    e64 = errs("fp64")
    emx = errs("mixed")
    # truth (FP64 at rtol 1e-13) on a seeded sample: every path's endpoint error
    sample = sorted(np.random.default_rng(11).choice(len(reqs), min(64, len(reqs)), replace=False).tolist())
    vs_truth = {"served": np.zeros(3), "fp64": np.zeros(3), "mixed": np.zeros(3)}
    for j in sample:
        wl = reqs[j].workload
        tabs = ctx.tables(wl.problem, wl.tables)
        y = torch.tensor(wl.y0, dtype=torch.float64, device="cuda")
        ctx.flow(wl.problem, tabs, y, wl.Lambda, t1_of(wl), precision=ffrg.FP64, rtol=1e-13, atol=1e-16)
        tr = y.cpu().numpy()
        tabs.free()
        for name, v in (("served", res[j]), ("fp64", single["fp64"]["outs"][j]),
                        ("mixed", single["mixed"]["outs"][j])):
            vs_truth[name] = np.maximum(vs_truth[name], endpoint_errs(v, tr, wl.y0))
    keys = ("norm", "cancel", "elem")
    rate = 0.8 * capacity
    arrivals = [rq.arrival_s * (200.0 / rate) for rq in reqs]   # the stream was drawn at 200 Hz
    wall_p, lat, _, stats_p, _ = run(arrivals)
    lv = sorted(lat.values())
    return {"requests": len(reqs), "families": "T=0 d3 frozen flows and finite-T frozen flows, "
                                              "ext 32-256, radial 32-128, angular 16-64, tables 64-256 pts",
            "served_flows_per_s": capacity, "served_integrand_evals_per_s": ev_sat / wall,
            "fp64_one_at_a_time_flows_per_s": single["fp64"]["flows_per_s"],
            "mixed_one_at_a_time_flows_per_s": single["mixed"]["flows_per_s"],
            "fp64_one_at_a_time_evals_per_s": single["fp64"]["evals_per_s"],
            "mixed_one_at_a_time_evals_per_s": single["mixed"]["evals_per_s"],
            "one_at_a_time_timing": "every request, plans built beforehand, upload + flow + result copy",
            "speedup_served_over_fp64": capacity / single["fp64"]["flows_per_s"],
            "speedup_served_over_mixed_one_at_a_time": capacity / single["mixed"]["flows_per_s"],
            "peak_resident": stats["peak_resident"], "ticks": stats["ticks"],
            "endpoint_error_measures": "norm = max|y - r| / max|r|; cancel = max |y_i - r_i| / (|y0_i| + "
                                       "|r_i - y0_i|); elem = max |y_i - r_i| / |r_i|",
            "served_vs_fp64_endpoint_max": dict(zip(keys, e64.max(axis=0).tolist())),
            "served_vs_fp64_endpoint_p99": dict(zip(keys, np.quantile(e64, 0.99, axis=0).tolist())),
            "served_vs_mixed_one_at_a_time_max": dict(zip(keys, emx.max(axis=0).tolist())),
            "endpoint_max_vs_truth": {**{nm: dict(zip(keys, v.tolist())) for nm, v in vs_truth.items()},
                                      "sample": len(sample), "truth": "FP64 ffrg_flow at rtol 1e-13, atol 1e-16"},
            "endpoints_compared": len(reqs), "rtol": rtol,
            "poisson_rate_hz": rate, "poisson_flows_per_s": len(reqs) / wall_p,
            "latency_p50_s": lv[len(lv) // 2], "latency_p99_s": lv[min(len(lv) - 1, int(0.99 * len(lv)))],
            "saturation_latency_p50_s": sorted(lat_sat.values())[len(lat_sat) // 2],
            "fp64_one_at_a_time_p50_s": single["fp64"]["p50_s"]}


def stepper_bench(ctx):
    """Steppers on d=4 feedback flows at matched endpoint error against a tight
    DP5(4) reference, all FP64: adaptive DP5(4) (6 RHS per step), fixed-step
    Adams-Bashforth-Moulton (PECE, 2 RHS per step) and the linearly implicit
    ROS2 (Jacobian from the adjoint kernels).  Two flows: M^2 = 1 (not stiff
    on k in [0.01, 10]) and the massless M^2 = 0 flow, whose state Jacobian
    reaches eigenvalues near -92 at k = 0.01 (DP5(4) then rejects about half
    of its steps)."""
    import numpy as np
    import torch

    import ffrg_inputs as fi
    import paper_2412_13043_gb300 as ffrg
    cases = []
    wl = fi.make_d4(seed=6, n_pts=32, n_ext_ang=4, n_rad=32, n_ang1=16, n_ang2=8)
    wl.problem.p_min = wl.problem.x_min = 0.01
    cases.append(("d4 feedback flow, M^2 = 1, 32-pt tables, 4 ext angles, 32 x 16 x 8 nodes, k: 10 -> 0.01, FP64", wl,
                  (("dp45", 1e-6), ("dp45", 1e-8), ("abm4", 50), ("abm4", 100), ("abm4", 200), ("abm4", 400),
                   ("ros2", 1e-5), ("ros2", 1e-6), ("ros2", 1e-7))))
    wl0 = fi.make_d4(seed=2, n_pts=16, n_ext_ang=2, n_rad=16, n_ang1=8, n_ang2=4, M2=0.0)
    cases.append(("massless d4 feedback flow, M^2 = 0, 16-pt tables, 2 ext angles, 16 x 8 x 4 nodes, "
                  "k: 10 -> 0.01, FP64", wl0,
                  (("dp45", 1e-6), ("dp45", 1e-7), ("abm4", 400), ("abm4", 1600), ("ros2", 1e-4), ("ros2", 1e-5),
                   ("ros2", 1e-6))))
    out = []
    for name, wl, runs in cases:
        pb = wl.problem
        t1 = math.log(wl.Lambda / wl.k_end)
        tabs = ctx.tables(pb, wl.tables)

        def run(kind, par):
            y = torch.tensor(wl.y0, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            t = time.perf_counter()
            if kind == "dp45":
                st = ctx.flow(pb, tabs, y, wl.Lambda, t1, feedback=1, precision=ffrg.FP64, rtol=par, atol=1e-14,
                              raise_on_error=False)
            elif kind == "abm4":   # fixed steps: may leave its stability region on the stiff flow
                st = ctx.abm_flow(pb, tabs, y, wl.Lambda, t1, par, order=4, feedback=1, precision=ffrg.FP64,
                                  raise_on_error=False)
            else:
                st = ctx.rosenbrock_flow(pb, tabs, y, wl.Lambda, t1, rtol=par, atol=1e-14, raise_on_error=False)
            torch.cuda.synchronize()
            ctx.status_read()   # a flow that left its stability region set the non-finite bit
            return y.cpu().numpy(), time.perf_counter() - t, st

        ref, _, _ = run("dp45", 1e-12)
        rows = []
        for kind, par in runs:
            y, dt, st = run(kind, par)
            ok = st["status"] == ffrg.OK and bool(np.all(np.isfinite(y)))
            rows.append({"method": kind, ("steps_requested" if kind == "abm4" else "rtol"): par,
                         "status": ffrg.strerror(st["status"]) if st["status"] else "ok",
                         "endpoint_rel_err": float(np.max(np.abs(y - ref) / np.abs(ref))) if ok else None,
                         "steps": st["steps"], "rejects": st["rejects"], "rhs_evals": st["rhs_evals"],
                         "jacobians": st.get("jac_evals", 0), "seconds": dt})
        tabs.free()
        out.append({"workload": name, "runs": rows})
    return out


def adjoint_bench(ctx, wl, tabs, reps: int = 3):
    """Reverse-mode derivatives of the d=4 RHS with respect to the 3 x 128
    table values at the full workload size (FP64): one VJP
    (ffrg_rhs_adjoint) and the full 1281 x 384 Jacobian (ffrg_rhs_jacobian),
    each against the FP64 RHS of the same workload."""
    import torch
    pb = wl.problem
    g = torch.ones(pb.n_ext(), dtype=torch.float64, device="cuda")
    J = ctx.rhs_jacobian(pb, tabs, 1.0)
    ctx.rhs_adjoint(pb, tabs, 1.0, g)
    torch.cuda.synchronize()
    res = {"workload": "d4 vertex RHS, 3 x 128-pt tables, 1281 ext x (128 x 64 x 16) nodes, FP64",
           "table_values": int(wl.tables.size)}
    for name, fn in (("vjp", lambda: ctx.rhs_adjoint(pb, tabs, 1.0, g)),
                     ("jacobian", lambda: ctx.rhs_jacobian(pb, tabs, 1.0, J=J))):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        res[name + "_ms"] = e0.elapsed_time(e1) / reps
    return res


STATES_SLICE_PAIRS = 55   # slice pairs of the FP64-faithful split (ten 5-bit slices, levels 0..9)


def states_bench(ctx, peaks, n_states: int = 1024, reps: int = 5, check: bool = True):
    """Finite-T sums of many loop-side states against one angle-integrated
    kernel (ffrg_ft_states) on the finite-T workloads (576 external points, 96
    radial x 48 angle nodes, N = 16 and 64), FP64 K: one call per step (K
    build, slicing, the tensor-core slice-pair kernel, combination).  The
    roofline is that of the tensor-core kernel: its algorithmic work is the
    slice products, 55 x 2 n_ext n_states (nfreq n_rad) BF16 FLOPs, against
    the measured BF16 peak.  Compared with n_states separate FP64 RHS calls
    (what the RHS path alone would take), and 2 states checked against the
    oracle (N = 16); the same calls with mixed-precision K rows beside them."""
    import numpy as np
    import torch

    import ffrg_inputs as fi
    import paper_2412_13043_gb300 as ffrg
    rows = []
    bf16 = peaks.get("bf16_tflops", 1853.1)
    for N, T in ((16, 0.0005), (64, 0.01)):
        wl = fi.make_finite_t(seed=3, N=N, T=T)
        pb = wl.problem
        tabs = ctx.tables(pb, wl.tables)
        nfreq = 2 * N + 1
        gen = torch.Generator(device="cuda").manual_seed(N)
        F = torch.rand(n_states, nfreq, pb.n_rad, dtype=torch.float64, device="cuda", generator=gen) + 0.5
        out = ctx.ft_states(pb, tabs, 1.0, F)
        torch.cuda.synchronize()
        # call time without profiling events, then the tensor-core kernel's time with them
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            ctx.ft_states(pb, tabs, 1.0, F, out=out)
        e1.record()
        torch.cuda.synchronize()
        total_ms = e0.elapsed_time(e1) / reps
        ctx.set_profiling(True)
        for _ in range(reps):
            ctx.ft_states(pb, tabs, 1.0, F, out=out)
        torch.cuda.synchronize()
        gemm_ms, cnt = ctx.profile_read()
        ctx.set_profiling(False)
        gemm_ms /= max(cnt, 1)
        r64 = torch.empty(pb.n_ext(), dtype=torch.float64, device="cuda")
        ctx.rhs(pb, tabs, 1.0, out=r64, precision=ffrg.FP64)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(3):
            ctx.rhs(pb, tabs, 1.0, out=r64, precision=ffrg.FP64)
        e1.record()
        torch.cuda.synchronize()
        rhs64_ms = e0.elapsed_time(e1) / 3
        kdim = nfreq * pb.n_rad
        slice_flops = STATES_SLICE_PAIRS * 2.0 * pb.n_ext() * n_states * kdim
        achieved = slice_flops / (gemm_ms * 1e-3) / 1e12
        row = {"workload": f"finite T N={N}: {pb.n_ext()} ext x {nfreq} freq x {pb.n_rad} radial, "
                           f"{n_states} states, FP64 K", "n_states": n_states, "terms_per_state": kdim,
               "call_ms": total_ms, "tensor_kernel_ms": gemm_ms,
               "fp64_equivalent_tflops": 2.0 * pb.n_ext() * n_states * kdim / (total_ms * 1e-3) / 1e12,
               "roofline": {"bound": "tensor", "kernel": "slice_pair_gemm (tcgen05 kind::f16, BF16 slices, "
                                                          "FP32 accumulators in tensor memory)",
                            "achieved": achieved, "peak": bf16, "unit": "TFLOP/s", "frac": achieved / bf16,
                            "work": "55 slice pairs x 2 n_ext n_states nfreq n_rad",
                            "peak_source": "bf16_tflops of measured (burst)"},
               "one_state_at_a_time_fp64_rhs_ms": rhs64_ms * n_states,
               "speedup_over_fp64_rhs_per_state": rhs64_ms * n_states / total_ms}
        # the same call with the K rows in mixed precision (FP32 angular sums):
        # the slicing, tensor-core passes and combination are unchanged
        outm = ctx.ft_states(pb, tabs, 1.0, F, precision=ffrg.MIXED)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            ctx.ft_states(pb, tabs, 1.0, F, out=outm, precision=ffrg.MIXED)
        e1.record()
        torch.cuda.synchronize()
        o64, om = out.cpu().numpy(), outm.cpu().numpy()
        row["mixed_K"] = {"call_ms": e0.elapsed_time(e1) / reps,
                          "max_rel_err_vs_fp64_K": float(np.max(np.abs(om - o64) / np.abs(o64)))}
        if check and N == 16:
            import oracle
            sel = [0, n_states - 1]
            ref = oracle.ft_states(pb, wl.tables, 1.0, F[sel].cpu().numpy())
            got = out[sel].cpu().numpy()
            row["max_rel_err_vs_oracle_2_states"] = float(np.max(np.abs(got - ref) / np.abs(ref)))
        rows.append(row)
        tabs.free()
    return rows


def ft4_rows(ctx, name, wl, steps):
    """The 4D-regulator finite-T model at k = 1 (Matsubara sum) and k = 10
    (frequency quadrature): terms = external points x frequencies in use x
    radial x angle nodes."""
    import numpy as np
    import torch

    import oracle
    import paper_2412_13043_gb300 as ffrg
    pb = wl.problem
    tabs = ctx.tables(pb, wl.tables)
    rows = []
    for k in (1.0, 10.0):
        nf = oracle.ft4_frequencies(pb, k)[0].size
        terms = pb.n_ext() * nf * pb.n_rad * pb.n_ang1
        row = {"workload": f"{name}, k = {k:g} ({'Matsubara sum' if nf <= 2 * pb.n_matsubara + 1 else 'quadrature'}"
                           f", {nf} frequencies)", "evals_per_rhs": terms}
        outs = {}
        for pname, prec in (("mixed", ffrg.MIXED), ("fp64", ffrg.FP64)):
            out = torch.empty(pb.n_ext(), dtype=torch.float64, device="cuda")
            for _ in range(2):
                ctx.rhs(pb, tabs, k, out=out, precision=prec)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                ctx.rhs(pb, tabs, k, out=out, precision=prec)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            row[pname] = {"step_ms": ms, "evals_per_s": terms / (ms * 1e-3)}
            outs[pname] = out.cpu().numpy()
        row["mixed_vs_fp64_max_rel_err"] = float(np.max(np.abs(outs["mixed"] - outs["fp64"]) / np.abs(outs["fp64"])))
        row["speedup_mixed_over_fp64"] = row["fp64"]["step_ms"] / row["mixed"]["step_ms"]
        rows.append(row)
    tabs.free()
    return rows


def model_bench(ctx, steps: int = 5, name_filter: str = ""):
    """Single-RHS throughput of the other model workloads, mixed and FP64:
    d=3 (64 ext x 64 x 32 nodes), finite T (64 |p| x 9 p0, 96 x 48 x (2N+1))
    at N = 16/32/64 with T/k_end = 0.05/0.2/1, the d=4 model with the
    three-point vertex on a 96 x 8 x 7 (S0, a, b) grid, and the fermionic
    loop at N = 16 (2N+2 frequencies).  step_ms: one ffrg_rhs (precompute + main);
    kernel_ms: the main kernel (profiling events; mixed finite T: the single
    cooperative launch of the whole RHS); k = 1."""
    import numpy as np
    import torch

    import ffrg_inputs as fi
    import paper_2412_13043_gb300 as ffrg
    cases = [("d3, 64 ext x (64 x 32)", fi.make_d3(seed=1))]
    for N, tk in ((16, 0.05), (32, 0.2), (64, 1.0)):
        cases.append((f"finite T bosonic N={N}, T/k_end={tk}", fi.make_finite_t(seed=3, N=N, T=tk * 0.01)))
    cases.append(("d4 full vertex: lambda3 on 96 x 8 x 7 (S0, a, b), 1281 ext x (128 x 64 x 16)",
                  fi.make_d4_full()))
    cases.append(("finite T fermionic N=16, T/k_end=0.05",
                  fi.make_finite_t(seed=3, N=16, T=0.05 * 0.01, fermionic=True)))
    # 4D regulator, k-scaled frequency domain: the Matsubara sum (25 frequencies) at k = 1
    # and the 64-node frequency quadrature at k = 10
    cases.append(("finite T, 4D regulator (Quadraturex0), 64 |p| x 9 p0, 96 x 48 nodes, T = 0.05",
                  fi.make_finite_t_4d()))
    rows = []
    for name, wl in cases:
        if name_filter and name_filter not in name:
            continue
        pb = wl.problem
        if pb.model == fi.MODEL_FINITE_T_4D:
            rows.extend(ft4_rows(ctx, name, wl, steps))
            continue
        tabs = ctx.tables(pb, wl.tables)
        # finite T evaluates the angular sums once per (stack row, |p|, radial node)
        # through K(p, q): the terms of the discrete sum (evals_per_rhs, the metric's
        # unit) are computed from (N + M) instead of (2N + 1) M angular sums
        computed = (pb.n_matsubara + pb.n_ext_ang) * pb.n_ext_p * pb.n_rad * pb.n_ang1 \
            if pb.model == fi.MODEL_FINITE_T else pb.evals()
        row = {"workload": name, "evals_per_rhs": pb.evals(), "integrands_computed_per_rhs": computed}
        outs = {}
        for pname, prec in (("mixed", ffrg.MIXED), ("fp64", ffrg.FP64)):
            out = torch.empty(pb.n_ext(), dtype=torch.float64, device="cuda")
            for _ in range(3):
                ctx.rhs(pb, tabs, 1.0, out=out, precision=prec)
            torch.cuda.synchronize()
            # RHS time without profiling events (they would hold the main
            # kernel back from starting early), then the kernel time with them
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                ctx.rhs(pb, tabs, 1.0, out=out, precision=prec)
            e1.record()
            torch.cuda.synchronize()
            step_ms = e0.elapsed_time(e1) / steps
            ctx.set_profiling(True)
            for _ in range(steps):
                ctx.rhs(pb, tabs, 1.0, out=out, precision=prec)
            torch.cuda.synchronize()
            kms, cnt = ctx.profile_read()
            ctx.set_profiling(False)
            row[pname] = {"step_ms": step_ms, "kernel_ms": kms / max(cnt, 1),
                          "evals_per_s": pb.evals() / (step_ms * 1e-3),
                          "integrands_computed_per_s": computed / (step_ms * 1e-3)}
            outs[pname] = out.cpu().numpy()
        row["mixed_vs_fp64_max_rel_err"] = float(np.max(np.abs(outs["mixed"] - outs["fp64"]) / np.abs(outs["fp64"])))
        # d=4 models: the Z block (D2 = int dR G^2 [-lam4/2 + lam3^2 G]) can cross
        # zero; its error is also given against |lam4 = 0 part| + |lam3 = 0 part|
        if pb.model in (fi.MODEL_D4_VERTEX, fi.MODEL_D4_FULL):
            n = pb.n_ext_p + 1
            scale = np.abs(outs["fp64"]).copy()
            scale[:n] = 0.0
            for zero in (2, 1):
                t = ctx.tables(pb, np.where(np.arange(3)[:, None, None] == zero, 0.0, wl.tables))
                scale[:n] += np.abs(ctx.rhs(pb, t, 1.0, precision=ffrg.FP64).cpu().numpy()[:n])
                t.free()
            row["mixed_vs_fp64_max_err_termwise"] = float(np.max(np.abs(outs["mixed"] - outs["fp64"]) / scale))

        row["speedup_mixed_over_fp64"] = row["fp64"]["step_ms"] / row["mixed"]["step_ms"]
        rows.append(row)
        tabs.free()
    return rows


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import ffrg_inputs as fi
    import oracle
    wl = fi.make_d4(seed=2)
    pb = wl.problem
    stride = 16
    sel = list(range(0, pb.n_ext(), stride))
    for _ in range(args.warmup):
        oracle.rhs_subset(pb, wl.tables, 1.0, sel[:8])
    times = []
    for s in range(args.steps):
        sub = [e for e in range((s % stride), pb.n_ext(), stride)]
        t = time.perf_counter()
        oracle.rhs_subset(pb, wl.tables, 1.0, sub)
        times.append((time.perf_counter() - t, len(sub) * pb.n_nodes()))
    tot_t = sum(t for t, _ in times)
    tot_ev = sum(e for _, e in times)
    val = tot_ev / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "integrand evals/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (CPU oracle, 1/16 of the external points per step)",
                       "l2": "n/a (host)"},
            "cpu_baseline": {"value": val, "unit": "integrand evals/s", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": f"each step: every 16th external point, offset by step"},
            "e2e": {"value": val, "unit": "integrand evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    rank, world, local = dist_env()
    import numpy as np
    import torch

    import ffrg_inputs as fi
    import paper_2412_13043_gb300 as ffrg

    if not torch.cuda.is_available():
        print(json.dumps({"metric": METRIC, "error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    ctx = ffrg.Context(local)
    wl = fi.make_d4(seed=2 + rank)
    pb = wl.problem
    evals = float(pb.evals())
    tabs = ctx.tables(pb, wl.tables)
    out = torch.empty(pb.n_ext(), dtype=torch.float64, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 512 MB > 129 MB L2
    stream = torch.cuda.current_stream()

    def step(prec, k=1.0):
        ctx.rhs(pb, tabs, k, out=out, precision=prec)

    # warm-up (also builds the launch plan)
    for _ in range(max(3, args.warmup)):
        step(ffrg.MIXED)
        step(ffrg.FP64)
    torch.cuda.synchronize()
    assert ctx.status_read() == ffrg.OK

    # ---------------- main timed region: mixed-precision RHS ----------------
    K = args.steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    sampler = ClockSampler(local)
    sampler.start()
    # untimed pre-roll under load (~0.5 s) so that the clock samples cover a
    # sustained window around the timed region
    t_pre = time.perf_counter()
    while time.perf_counter() - t_pre < 0.5:
        for _ in range(20):
            step(ffrg.MIXED)
        torch.cuda.synchronize()
    barrier()
    wall0 = time.perf_counter()
    for i in range(K):
        flush.zero_()
        starts[i].record(stream)
        step(ffrg.MIXED)
        stops[i].record(stream)
    barrier()
    wall = time.perf_counter() - wall0
    # the main kernel's own duration: CUDA events around its launch over K
    # more steps, identical but for those events.  They stay out of the timed
    # steps: an event between the precompute and the main kernel makes the
    # main kernel wait for it, so it can no longer start early as the
    # precompute's programmatic dependent (about 4 us more per step)
    ctx.set_profiling(True)
    prof_starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    prof_stops = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    for i in range(K):
        flush.zero_()
        prof_starts[i].record(stream)
        step(ffrg.MIXED)
        prof_stops[i].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    main_ms, launches = ctx.profile_read()
    ctx.set_profiling(False)
    prof_step_ms = [s.elapsed_time(e) for s, e in zip(prof_starts, prof_stops)]
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, stops)]
    t_max = max_over_ranks(sum(step_ms) / 1e3, dist, "cuda")
    value = whole_job_rate(world, evals * K, t_max)
    assert ctx.status_read() == ffrg.OK

    # ---------------- FP64 path on the same workload ----------------
    K64 = max(2, K // 5)
    s64 = [torch.cuda.Event(enable_timing=True) for _ in range(K64)]
    e64 = [torch.cuda.Event(enable_timing=True) for _ in range(K64)]
    barrier()
    for i in range(K64):
        flush.zero_()
        s64[i].record(stream)
        step(ffrg.FP64)
        e64[i].record(stream)
    barrier()
    fp64_ms = sum(s.elapsed_time(e) for s, e in zip(s64, e64)) / K64
    ref64 = out.cpu().numpy().copy()
    step(ffrg.MIXED)
    mixed_out = out.cpu().numpy()
    mixed_err = float(np.max(np.abs(mixed_out - ref64) / np.abs(ref64)))

    # ---------------- end to end: public API with host buffers ----------------
    # tables in by ffrg_tables_update, outputs out by ffrg_rhs_host: both C-ABI
    # calls with pinned host memory; the table copy and the kernels' writes of
    # the outputs into host memory are inside the timed region
    host_tab = torch.tensor(wl.tables, dtype=torch.float64).pin_memory()
    host_out = torch.empty(pb.n_ext(), dtype=torch.float64).pin_memory()
    ctx.rhs_host(pb, tabs, 1.0, out=host_out, precision=ffrg.MIXED)   # warm (allocates its buffer)
    torch.cuda.synchronize()
    es = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ee = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    barrier()
    for i in range(K):
        flush.zero_()
        es[i].record(stream)
        tabs.update(host_tab)            # pinned host -> device, stream-ordered
        ctx.rhs_host(pb, tabs, 1.0, out=host_out, precision=ffrg.MIXED)   # RHS, device -> pinned host
        ee[i].record(stream)
    barrier()
    torch.cuda.synchronize()
    assert np.array_equal(host_out.numpy(), mixed_out), "ffrg_rhs_host differs from ffrg_rhs"
    e2e_t = max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(es, ee)) / 1e3, dist, "cuda")
    e2e_val = whole_job_rate(world, evals * K, e2e_t)

    # ---------------- roofline of the dominant kernel ----------------
    peaks = measured_peaks()
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    sfu_peak = SFU_PER_CLK_SM * n_sm * sm_mhz * 1e6
    kern_s = (main_ms / 1e3) / max(1, launches)
    sfu_ops = sfu_ops_per_launch(pb)
    achieved = sfu_ops / kern_s
    roofline = {"bound": "alu", "pipe": "MUFU (special-function unit, log2-equivalent results)",
                "achieved": achieved / 1e12,
                "peak": sfu_peak / 1e12, "unit": "Tops/s", "frac": achieved / sfu_peak, "traffic": D4_MAIN_DRAM_BYTES,
                "peak_source": f"{SFU_PER_CLK_SM}/clk/SM x {n_sm} SMs x {sm_mhz:.0f} MHz (max SM clock of measured)",
                "kernel": "rhs_main<2, float>", "kernel_ms": kern_s * 1e3, "ops_per_launch": sfu_ops,
                "kernel_share_of_step": (main_ms / max(1, launches)) / (sum(prof_step_ms) / K),
                "kernel_timing": "CUDA events around each main-kernel launch over K steps run right after "
                                 "the timed ones (same inputs, L2 flush, stream)"}

    # ---------------- full flows (d=3 two-point flow k: 10 -> 0.01) ----------------
    flows = None
    if not args.no_flows:
        wf = fi.make_d3(seed=1)
        tf = ctx.tables(wf.problem, wf.tables)
        t1 = math.log(wf.Lambda / wf.k_end)

        def run_flow(prec, rtol, atol):
            y = torch.tensor(wf.y0, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            t = time.perf_counter()
            st = ctx.flow(wf.problem, tf, y, wf.Lambda, t1, precision=prec, rtol=rtol, atol=atol)
            torch.cuda.synchronize()
            return y.cpu().numpy(), time.perf_counter() - t, st
        truth, _, _ = run_flow(ffrg.FP64, 1e-13, 1e-16)
        res = {}
        for name, prec in (("fp64", ffrg.FP64), ("mixed", ffrg.MIXED)):
            y, dt, st = run_flow(prec, 1e-10, 1e-13)
            res[name] = {"flows_per_s": 1.0 / dt, "s_per_flow": dt, "steps": st["steps"],
                         "rhs_evals": st["rhs_evals"],
                         "endpoint_rel_err": float(np.max(np.abs(y - truth) / np.abs(truth)))}
        flows = {"workload": "d3 two-point flow, 64 ext x (64 x 32) nodes, k: 10 -> 0.01, rtol 1e-10",
                 **res}
        tf.free()

    adjoint = adjoint_bench(ctx, wl, tabs)
    adjoint["fp64_rhs_ms"] = fp64_ms
    states = None
    if not args.no_models:
        states = states_bench(ctx, measured_peaks(), check=(rank == 0 and not args.no_cpu))

    serving = None
    if not args.no_serve:
        serving = serving_bench(ctx, args.serve_requests)

    steppers = None
    if not args.no_flows:
        steppers = stepper_bench(ctx)

    models = None
    if not args.no_models:
        models = model_bench(ctx, name_filter=args.model_filter)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(wl, stride=1)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "integrand evals/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": sum(step_ms) / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 integrand + f64 accumulation", "data": "synthetic",
            "config": {"workload": WORKLOAD, "evals_per_step": evals, "precision": "mixed",
                       "l2": "flushed between steps (512 MB write)", "parallelism": f"replicas x{world}"},
            "wall_s_timed_region": wall,
            "fp64_path": {"value": evals / (fp64_ms / 1e3), "unit": "integrand evals/s", "ms_per_step": fp64_ms,
                          "speedup_mixed_over_fp64": (value / world) / (evals / (fp64_ms / 1e3)),
                          "fp64_pipe_frac": evals / (fp64_ms / 1e3) * FP64_OPS_PER_TERM_D4
                          / (FP64_PER_CLK_SM * n_sm * sm_mhz * 1e6),
                          "fp64_pipe_frac_basis": f"{FP64_OPS_PER_TERM_D4} FP64-pipe ops per term (ncu) x terms/s "
                                                  f"/ ({FP64_PER_CLK_SM}/clk/SM x {n_sm} SMs x {sm_mhz:.0f} MHz)"},
            "mixed_vs_fp64_max_rel_err": mixed_err,
            "e2e": {"value": e2e_val, "unit": "integrand evals/s",
                    "h2d_bytes_per_step": int(wl.tables.size * 8), "d2h_bytes_per_step": int(pb.n_ext() * 8),
                    "path": "tables: pinned host -> device copy (ffrg_tables_update); outputs: written by the "
                            "kernels into the pinned host buffer (ffrg_rhs_host), read on the host after the step"},
            # per timed step and rank: precompute_kernel and rhs_main (the d=4 main
            # kernel writes the outputs itself); the L2 flush is torch's fill kernel
            "gpu_launches": 2 * K * world,
            "roofline": roofline,
            "clocks": clocks,
            "flows": flows,
            "serving": serving,
            "steppers": steppers,
            "adjoint": adjoint,
            "states": states,
            "models": models,
            "cpu_baseline": cpu,
        }
        # last key of the line, so that a truncated tail of the output still shows it
        summ = {"fp64_d4_evals_per_s": line["fp64_path"]["value"],
                "fp64_d4_pipe_frac": line["fp64_path"]["fp64_pipe_frac"],
                "mixed_over_fp64_d4": line["fp64_path"]["speedup_mixed_over_fp64"]}
        if states:
            summ["states_tensor_frac"] = {r["workload"].split(":")[0]: r["roofline"]["frac"] for r in states}
        if serving:
            summ.update({k: serving[k] for k in (
                "served_flows_per_s", "fp64_one_at_a_time_flows_per_s", "speedup_served_over_fp64",
                "mixed_one_at_a_time_flows_per_s", "latency_p50_s", "latency_p99_s",
                "endpoints_compared")})
            summ["served_vs_fp64_endpoint_norm_max"] = serving["served_vs_fp64_endpoint_max"]["norm"]
            vt = serving["endpoint_max_vs_truth"]
            summ["endpoint_vs_truth_norm_max"] = {"served": vt["served"]["norm"], "fp64": vt["fp64"]["norm"]}
            summ["endpoint_vs_truth_cancel_max"] = {"served": vt["served"]["cancel"], "fp64": vt["fp64"]["cancel"]}
        if models:
            # mixed single-RHS time of every model workload (ms per ffrg_rhs call)
            mm = {}
            for r in models:
                key = r["workload"][:40]
                if "k = " in r["workload"]:   # the two scales of one workload
                    key += " " + r["workload"][r["workload"].index("k = "):].split(" (")[0]
                mm[key] = round(r["mixed"]["step_ms"], 4)
            summ["models_mixed_ms"] = mm
        line["summary"] = summ
        print(json.dumps(line))
    tabs.free()
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
