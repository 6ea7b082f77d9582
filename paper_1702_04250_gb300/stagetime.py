"""Per-stage device times of the PPPM step on one of the synthetic workloads.

    python -m paper_1702_04250_gb300.stagetime c3 ad fp32c [steps] [--graph] [--variant V]

Runs `steps` steps (the first two untimed), each after a 64 MiB L2 flush,
with CUDA events at every stage boundary, and prints the last step's stage
times and the mean step time.  The same command line serves as the launch
list for profilers (one kernel per stage per step).
"""
import argparse
import os
import sys

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=["c1", "c2", "c3", "c5"])
    ap.add_argument("mode", choices=["ik", "ad"])
    ap.add_argument("precision", choices=["fp64", "fp32c", "fp32"])
    ap.add_argument("steps", type=int, nargs="?", default=6)
    ap.add_argument("--graph", action="store_true")
    ap.add_argument("--variant", type=int, default=None)
    a = ap.parse_args(argv)

    import torch

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_1702_04250_gb300 import build, pppm
    from paper_1702_04250_gb300.workloads import config

    build.build()
    w = config(a.workload)
    g = pppm.estimate_g(w.rel_acc, w.r_cut, w.n, float(np.sum(w.q ** 2)), w.box)
    dt = torch.float64 if a.precision == "fp64" else torch.float32
    plan = pppm.PPPM(w.box, w.n, w.order, w.mesh, g, mode=a.mode, precision=a.precision, qqrd2e=w.qqrd2e,
                     graph=a.graph)
    if a.variant is not None:
        plan.set_variant(a.variant)
    x = torch.tensor(w.x, dtype=dt, device="cuda")
    q = torch.tensor(w.q, dtype=dt, device="cuda")
    f = torch.empty((w.n, 3), dtype=dt, device="cuda")
    ev = torch.zeros(8, dtype=torch.float64, device="cuda")
    flush = torch.empty(16 << 20, dtype=torch.float32, device="cuda")
    plan.set_profiling(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    tot, st = 0.0, {}
    for i in range(a.steps):
        with torch.cuda.stream(plan.stream):
            flush.zero_()
        e0.record(plan.stream)
        plan.compute(x, q, f, ev)
        e1.record(plan.stream)
        plan.sync()
        st = plan.stage_times()
        if i >= 2:
            tot += e0.elapsed_time(e1)
    print(f"{a.workload} {a.mode} {a.precision} n={w.n} mesh={w.mesh} P={w.order}: "
          + ", ".join(f"{k} {v * 1000:.1f} us" for k, v in st.items())
          + f"; step {1000 * tot / max(a.steps - 2, 1):.1f} us (events at every stage boundary); "
          + f"energy {float(ev[0]):.6g}")


if __name__ == "__main__":
    main()
