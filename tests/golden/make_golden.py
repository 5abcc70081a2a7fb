"""Writes oracle_rhs_small.txt: FP64 oracle RHS values of small seeded
workloads of every model (d=3, the d=4 vertex model, the full three-point
vertex, finite T with bosonic and fermionic loops) at two scales.

It calls only the oracle (oracle/) and the seeded input generators
(ffrg_inputs.py).  Run from the repository root:

    python tests/golden/make_golden.py

The stored values let a CPU test notice any change of the oracle's
arithmetic; regenerate them only together with such a change.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import ffrg_inputs as fi  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(HERE, "oracle_rhs_small.txt")


def workloads():
    """(name, workload) pairs; names are parsed by the test."""
    return [
        ("d3", fi.make_d3(seed=101, n_pts=16, n_ext_p=8, n_rad=12, n_ang=6)),
        ("d4", fi.make_d4(seed=102, n_pts=12, n_ext_ang=2, n_rad=8, n_ang1=4, n_ang2=3)),
        ("d4_full", fi.make_d4_full(seed=103, n_pts=10, n_va=3, n_vb=2, n_ext_ang=2, n_rad=6, n_ang1=4, n_ang2=3)),
        ("finite_t_bose", fi.make_finite_t(seed=104, N=3, T=0.05, n_pts=12, n_ext_p=3, n_ext_m=2, n_rad=8, n_ang=4)),
        ("finite_t_fermi", fi.make_finite_t(seed=105, N=3, T=0.05, n_pts=12, n_ext_p=3, n_ext_m=2, n_rad=8, n_ang=4,
                                            fermionic=True)),
    ]


SCALES = (1.0, 0.3)


def main():
    lines = ["# FP64 oracle RHS (k d_k of the target per external point) of small seeded",
             "# workloads; written by tests/golden/make_golden.py (oracle/ only).",
             "# columns: workload  k  external_point  value"]
    for name, wl in workloads():
        for k in SCALES:
            out = oracle.rhs(wl.problem, wl.tables, k)
            for e, v in enumerate(out):
                lines.append(f"{name} {k!r} {e} {float(v)!r}")
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(f"wrote {OUT} ({len(lines) - 3} values)")


if __name__ == "__main__":
    main()
