"""Pins of the oracle's lookup-table coefficients (R17; Sec. 3.1 "precompute",
Table 1's LUT-500 / LUT-5000): the rounded offset stays in its bin, a fine
table reproduces the exact coefficients, the table's error falls as 1/K, and
against the exact Ewald sum LUT-500 is clearly worse than exact while
LUT-5000 stays close (Table 1's trend)."""
import math

import numpy as np
import pytest

from oracle import OraclePPPM, ewald_kspace, estimate_g_ewald, lut_offset
from paper_1702_04250_gb300.workloads import config


def rel_rms(a, b):
    return math.sqrt(float(np.sum((a - b) ** 2)) / float(np.sum(b ** 2)))


@pytest.mark.parametrize("P", [4, 5])
@pytest.mark.parametrize("K", [7, 500])
def test_rounded_offset_is_its_bin_centre(P, K):
    lo = -0.5 if P % 2 else -1.0
    d = np.random.default_rng(1).uniform(lo, lo + 1.0, 20000)
    dq = lut_offset(d, P, K)
    assert np.all(np.abs(dq - d) <= 0.5 / K + 1e-15)
    b = (dq - lo) * K - 0.5                    # bin index of the centre
    assert np.allclose(b, np.round(b), atol=1e-9)
    assert np.array_equal(np.round(b), np.floor((d - lo) * K))
    # the range end maps into the last bin
    assert lut_offset(np.array([lo + 1.0 - 1e-17]), P, K)[0] == lo + (K - 0.5) / K


@pytest.fixture(scope="module")
def c1():
    w = config("c1")
    g = estimate_g_ewald(w.rel_acc, w.r_cut, w.n, float(np.sum(w.q ** 2)), w.box)
    return w, g


def test_fine_table_is_exact(c1):
    w, g = c1
    ref = OraclePPPM(w.box, w.mesh, 5, g, "ad", 1.0).compute(w.x, w.q)
    fine = OraclePPPM(w.box, w.mesh, 5, g, "ad", 1.0, lut=1 << 26).compute(w.x, w.q)
    assert rel_rms(fine["f"], ref["f"]) < 1e-6
    assert abs(fine["energy"] - ref["energy"]) < 1e-6 * abs(ref["energy"])


def test_table_error_falls_as_one_over_entries(c1):
    w, g = c1
    exact = OraclePPPM(w.box, (24, 24, 24), 7, g, "ik", 1.0).compute(w.x, w.q)["f"]
    err = {K: rel_rms(OraclePPPM(w.box, (24, 24, 24), 7, g, "ik", 1.0, lut=K).compute(w.x, w.q)["f"], exact)
           for K in (50, 500, 5000)}
    assert 6.0 < err[500] / err[5000] < 14.0
    assert 6.0 < err[50] / err[500] < 14.0


def test_table1_trend_against_ewald(c1):
    """P = 7, ik, 16^3 against the exact reciprocal sum: the oracle measures
    exact 2.5e-5, LUT-5000 6.1e-5, LUT-500 5.7e-4 (the paper's Table 1:
    0.0186, 0.0188, 0.0313 in its units, where the PPPM error is larger)."""
    w, g = c1
    _, Fk, _ = ewald_kspace(w.x, w.q, w.box, g, 1.0)
    err = {K: rel_rms(OraclePPPM(w.box, w.mesh, 7, g, "ik", 1.0, lut=K).compute(w.x, w.q)["f"], Fk)
           for K in (0, 500, 5000)}
    assert err[500] > 5.0 * err[0]
    assert err[5000] < 3.0 * err[0]
    assert err[500] > 5.0 * err[5000]
