"""The ik energy gradient against the ik force, pinned by the exact Ewald sum.

An ik plan offers two forces: the interpolated ik field F_ik and -dE/dx, the
exact gradient of the same plan's energy (what the autograd backward gives).
Both approximate the Ewald reciprocal force of Sec. 2.1; the bound on their
difference comes from measuring each against the direct Ewald sum
(tests/golden/ik_gradient_errors.txt, written from oracle/ only): by the
triangle inequality |dE/dx + F_ik| <= |F_ik - F_ewald| + |-dE/dx - F_ewald|.
These tests re-derive the small rows live and check the table's structure.
"""
import math
import os

import numpy as np
import pytest

from oracle import OraclePPPM, estimate_g_ewald
from oracle.ewald import ewald_kspace
from paper_1702_04250_gb300.workloads import config

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ik_gradient_errors.txt")


def table():
    rows = {}
    for ln in open(GOLDEN):
        if ln.startswith("#") or not ln.strip():
            continue
        name, m, P, e_ik, e_grad, d, ratio = ln.split()
        rows[(name, int(m))] = dict(order=int(P), e_ik=float(e_ik), e_grad=float(e_grad), d=float(d),
                                    ratio=float(ratio))
    return rows


def rel_rms(a, b):
    return math.sqrt(float(np.sum((a - b) ** 2)) / float(np.sum(b ** 2)))


def test_table_obeys_the_triangle_inequality():
    for key, r in table().items():
        assert r["d"] <= (r["e_ik"] + r["e_grad"]) * r["ratio"] * (1 + 1e-9), key
        assert r["d"] >= abs(r["e_ik"] - r["e_grad"]) * r["ratio"] * (1 - 1e-9), key


def test_difference_falls_as_the_mesh_is_refined():
    t = table()
    meshes = sorted(m for (name, m) in t if name == "c1")
    assert meshes == [16, 24, 32, 48]
    d = [t[("c1", m)]["d"] for m in meshes]
    e_ik = [t[("c1", m)]["e_ik"] for m in meshes]
    e_grad = [t[("c1", m)]["e_grad"] for m in meshes]
    for seq in (d, e_ik, e_grad):
        assert all(b < a for a, b in zip(seq, seq[1:])), seq
    assert d[-1] < d[0] / 100  # two orders of magnitude from 16^3 to 48^3


@pytest.mark.parametrize("m", [16, 24])
def test_c1_rows_rederived(m):
    """The stored c1 rows equal a fresh oracle computation."""
    w = config("c1")
    g = estimate_g_ewald(w.rel_acc, w.r_cut, w.n, float(np.sum(w.q ** 2)), w.box)
    o = OraclePPPM(w.box, (m,) * 3, w.order, g, "ik", w.qqrd2e)
    f_ik = o.compute(w.x, w.q)["f"]
    dEdx, _ = o.energy_gradients(w.x, w.q)
    _, f_ew, _ = ewald_kspace(w.x, w.q, w.box, g, w.qqrd2e)
    r = table()[("c1", m)]
    assert abs(rel_rms(f_ik, f_ew) - r["e_ik"]) <= 1e-6 * r["e_ik"]
    assert abs(rel_rms(-dEdx, f_ew) - r["e_grad"]) <= 1e-6 * r["e_grad"]
    assert abs(rel_rms(-dEdx, f_ik) - r["d"]) <= 1e-6 * r["d"]


def test_c5_bound_is_what_the_gpu_test_uses():
    r = table()[("c5", 96)]
    bound = (r["e_ik"] + r["e_grad"]) * r["ratio"]
    assert 1e-4 < r["d"] < bound < 3e-4
