"""Times one hot kernel of the step on a workload's own data (CUDA events on
the problem's stream) and prints one JSON line: mean duration, algorithmic
bytes per launch and the resulting GB/s.

    python -m paper_2605_25403_gb300.profile_kernel --workload cube --kernel cheb --reps 20

The kernel runs exactly `3 + reps` times after the problem's set-up and one
assembly, so a profiler can select its first launches by name.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--workload", default="cube", choices=["channel", "cube", "unit_square"])
    p.add_argument("--kernel", default="cheb",
                   choices=["cheb", "spmv", "spmv_fp64", "assemble", "precond", "cgs",
                            "cgs_dot", "cgs_upd", "cgs_fin"])
    p.add_argument("--cold", action="store_true",
                   help="time each launch after the L2 was filled with other data")
    p.add_argument("--precision", default="fp32_refine", choices=["fp32_refine", "fp64"])
    p.add_argument("--reps", type=int, default=20)
    p.add_argument("--n", type=int, default=0,
                   help="cells per axis instead of the workload's own (cube and channel x)")
    a = p.parse_args(argv)
    import fs_workloads as W
    from paper_2605_25403_gb300 import build
    build.build()
    from paper_2605_25403_gb300 import fs
    wl = {"channel": W.C2, "cube": W.C3, "unit_square": W.C1}[a.workload]
    if a.n > 0:
        wl = W.cube(a.n, jitter=0.05, seed=W.C3.seed) if a.workload == "cube" else \
            W.channel(a.n, max(2, a.n * 96 // 512)) if a.workload == "channel" else W.unit_square(a.n)
    prec = fs.FS_PREC_FP32_REFINE if a.precision == "fp32_refine" else fs.FS_PREC_FP64
    kid = {"cheb": fs.FS_KERNEL_CHEB, "spmv": fs.FS_KERNEL_SPMV,
           "spmv_fp64": fs.FS_KERNEL_SPMV_FP64, "assemble": fs.FS_KERNEL_ASSEMBLE_CONV,
           "precond": fs.FS_KERNEL_PRECOND, "cgs": fs.FS_KERNEL_CGS,
           "cgs_dot": fs.FS_KERNEL_CGS_DOT, "cgs_upd": fs.FS_KERNEL_CGS_UPD,
           "cgs_fin": fs.FS_KERNEL_CGS_FIN}[a.kernel]
    S = fs.Stepper.from_workload(wl, precision=prec)
    try:
        ms, by = fs.fs_profile_kernel(S.prob, kid, reps=a.reps, cold=a.cold)
    finally:
        S.close()
    print(json.dumps({"workload": wl.name, "kernel": a.kernel, "precision": a.precision,
                      "cold": a.cold,
                      "ms": ms, "alg_bytes": by, "gbs": by / ms / 1e6 if by else None}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
