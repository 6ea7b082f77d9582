"""Plausible mistakes planted in the oracle (on the CPU) must trip its pins.

Each test patches one step of the oracle the way a slip would change it and
checks that the comparison used by the pin tests fails by a wide margin.
"""
import math

import numpy as np
import pytest

import oracle.pppm_oracle as po
from oracle import background_energy, estimate_g_ewald, ewald_kspace, self_energy
from paper_1702_04250_gb300.workloads import config


@pytest.fixture(scope="module")
def ref():
    w = config("c1")
    g = estimate_g_ewald(w.rel_acc, w.r_cut, w.n, float(np.sum(w.q ** 2)), w.box)
    Ek, Fk, _ = ewald_kspace(w.x, w.q, w.box, g, w.qqrd2e)
    E = Ek + self_energy(w.q, g, w.qqrd2e) + background_energy(w.q, g, w.qqrd2e, w.box)
    return w, g, E, Fk


def _errors(w, g, E, Fk, mode="ik"):
    r = po.OraclePPPM(w.box, w.mesh, w.order, g, mode, w.qqrd2e).compute(w.x, w.q)
    ferr = math.sqrt(float(np.sum((r["f"] - Fk) ** 2) / np.sum(Fk ** 2)))
    return ferr, abs(r["energy"] - E) / abs(E)


def test_unplanted_baseline(ref):
    ferr, eerr = _errors(*ref)
    assert ferr < 5e-4 and eerr < 5e-5


def test_planted_half_spectrum_weight(ref, monkeypatch):
    monkeypatch.setattr(po, "half_spectrum_weights", lambda Mz: np.ones(Mz // 2 + 1))
    _, eerr = _errors(*ref)
    assert eerr > 1e-2


def test_planted_odd_anchor_floor(ref, monkeypatch):
    real = po.stencil

    def bad(u, P, M, lut=0):
        u = np.asarray(u, dtype=np.float64)
        n = np.floor(u)  # should round to the nearest point for odd P
        pts = n[:, None] - (P - 1) // 2 + np.arange(P)[None, :]
        return np.mod(pts, M).astype(np.int64), pts - u[:, None]

    monkeypatch.setattr(po, "stencil", bad)
    ferr, _ = _errors(*ref)
    # the Ewald comparison (tolerance 5e-4) and charge conservation both fail
    assert ferr > 5e-4
    r = np.random.default_rng(3)
    x = r.uniform(0, 10, (300, 3))
    qq = r.normal(size=300)
    rho = po.make_rho(x, qq, (10.0,) * 3, (10,) * 3, 5)
    assert abs(rho.sum() - qq.sum()) > 1e-6 * np.abs(qq).sum()
    monkeypatch.setattr(po, "stencil", real)


def test_planted_field_sign(ref, monkeypatch):
    real = po.poisson_ik

    def bad(rho, G, box):
        rh, f = real(rho, G, box)
        return rh, [-e for e in f]

    monkeypatch.setattr(po, "poisson_ik", bad)
    ferr, _ = _errors(*ref)
    assert ferr > 1.0


def test_planted_unsquared_denominator(ref, monkeypatch):
    real = po.alias_sum_u2
    monkeypatch.setattr(po, "alias_sum_u2", lambda k, h, P, mmax=2000: np.sqrt(real(k, h, P, mmax)))
    ferr, eerr = _errors(*ref)
    assert ferr > 1e-3 or eerr > 1e-4


def test_planted_selfforce_sign():
    box, mesh, P, g = (10.0, 11.0, 12.0), (10, 12, 8), 5, 0.6
    o = po.OraclePPPM(box, mesh, P, g, "ad", 1.0)
    h = np.array(box) / np.array(mesh)
    x = (np.array([3.2, 4.0, 2.0]) * h)[None, :]
    q = np.array([1.0])
    good = o.compute(x, q)["f"]
    o.sf = -o.sf
    bad = o.compute(x, q)["f"]
    assert abs(bad[0, 0]) > 10 * abs(good[0, 0])
