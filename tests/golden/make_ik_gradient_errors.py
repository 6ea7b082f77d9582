"""Writes ik_gradient_errors.txt: how far the two forces an ik PPPM plan
offers lie from the exact Ewald reciprocal force, and from each other.

An ik plan gives two forces: F_ik, the mesh field E = -i k G rho_hat
interpolated to the particles, and -dE/dx, the exact gradient of the PPPM
energy of the same plan (what the autograd energy's backward returns).  Both
approximate the Ewald reciprocal force of Sec. 2.1; neither is the other.
For each workload below this script computes, with the FP64 oracle only,
  e_ik   = |F_ik - F_ewald| / |F_ewald|      (relative RMS over all charges)
  e_grad = |-dE/dx - F_ewald| / |F_ewald|
  d      = |-dE/dx - F_ik| / |F_ik|
where F_ewald is the direct reciprocal sum (oracle/ewald.py, k-vectors to
exp(-k^2/4g^2) >= 1e-16).  By the triangle inequality d <= (e_ik + e_grad)
|F_ewald| / |F_ik|, so e_ik + e_grad (times that norm ratio) bounds the
difference the GPU test may see on the same workload.

Workloads: c5 (99,999 water-like charges, 100 A cube, 96^3, P = 5) -- the
autograd workload, about 2.6e5 k-vectors, several minutes on one core;
c2 (32,001 charges, 64^3); and c1 (4096 +-1 charges, 24 A cube) on meshes
16^3 .. 48^3, where the difference must fall as the mesh is refined.

    python tests/golden/make_ik_gradient_errors.py [--skip-c5]
"""
from __future__ import annotations

import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import OraclePPPM, estimate_g_ewald  # noqa: E402
from oracle.ewald import ewald_kspace  # noqa: E402
from paper_1702_04250_gb300.workloads import config  # noqa: E402


def rel_rms(a, b):
    return math.sqrt(float(np.sum((a - b) ** 2)) / float(np.sum(b ** 2)))


def errors(w, mesh):
    g = estimate_g_ewald(w.rel_acc, w.r_cut, w.n, float(np.sum(w.q ** 2)), w.box)
    o = OraclePPPM(w.box, mesh, w.order, g, "ik", w.qqrd2e)
    f_ik = o.compute(w.x, w.q)["f"]
    dEdx, _ = o.energy_gradients(w.x, w.q)
    _, f_ew, _ = ewald_kspace(w.x, w.q, w.box, g, w.qqrd2e)
    return {"e_ik": rel_rms(f_ik, f_ew), "e_grad": rel_rms(-dEdx, f_ew), "d": rel_rms(-dEdx, f_ik),
            "norm_ratio": math.sqrt(float(np.sum(f_ew ** 2)) / float(np.sum(f_ik ** 2)))}


def main():
    rows = []
    names = [("c1", m) for m in (16, 24, 32, 48)] + [("c2", 64)]
    if "--skip-c5" not in sys.argv:
        names.append(("c5", 96))
    for name, m in names:
        w = config(name)
        t0 = time.time()
        r = errors(w, (m, m, m))
        rows.append((name, m, w.order, r))
        print(name, m, {k: f"{v:.4e}" for k, v in r.items()}, f"{time.time() - t0:.0f} s", flush=True)
    out = os.path.join(HERE, "ik_gradient_errors.txt")
    with open(out, "w") as fh:
        fh.write("# ik PPPM: F_ik and -dE/dx against the exact Ewald reciprocal force (Sec. 2.1), FP64 oracle.\n")
        fh.write("# Written by tests/golden/make_ik_gradient_errors.py (oracle/ only); relative RMS over all charges.\n")
        fh.write("# workload mesh order e_ik e_grad d norm_ratio(|F_ewald|/|F_ik|)\n")
        for name, m, P, r in rows:
            fh.write(f"{name} {m} {P} {r['e_ik']:.6e} {r['e_grad']:.6e} {r['d']:.6e} {r['norm_ratio']:.9f}\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
