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


def test_planted_virial_dropped_gaussian_term(ref, monkeypatch):
    """W_ab without the (1 + k^2/4g^2) factor's k^2/4g^2 part: the PPPM virial
    no longer matches the direct Ewald virial (4e-4 unplanted)."""
    w, g, _, _ = ref
    Wk = ewald_kspace(w.x, w.q, w.box, g, w.qqrd2e)[2]
    real = po.energy_virial_mesh

    def bad(rho_hat, G, box, mesh, g_, C):
        box_a = np.asarray(box, dtype=np.float64)
        mesh_a = np.asarray(mesh, dtype=np.int64)
        vcell = float(np.prod(box_a / mesh_a))
        pref = 0.5 * C * vcell * vcell / float(np.prod(box_a))
        s = po.half_spectrum_weights(int(mesh_a[2]))[None, None, :] * G * np.abs(rho_hat) ** 2
        kx, ky, kz = po._half_k(box_a, mesh_a)
        K = [kx[:, None, None], ky[None, :, None], kz[None, None, :]]
        k2 = K[0] ** 2 + K[1] ** 2 + K[2] ** 2
        with np.errstate(divide="ignore", invalid="ignore"):
            fac = 2.0 / k2  # dropped: the k^2 / 4g^2 term
        fac[0, 0, 0] = 0.0
        vir = np.array([pref * float(np.sum(s * ((1.0 if a == b else 0.0) - fac * K[a] * K[b])))
                        for a, b in ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))])
        return real(rho_hat, G, box, mesh, g_, C)[0], vir

    r0 = po.OraclePPPM(w.box, w.mesh, w.order, g, "ik", w.qqrd2e).compute(w.x, w.q)
    assert np.linalg.norm(r0["virial"] - Wk) / np.linalg.norm(Wk) < 1e-3
    monkeypatch.setattr(po, "energy_virial_mesh", bad)
    r1 = po.OraclePPPM(w.box, w.mesh, w.order, g, "ik", w.qqrd2e).compute(w.x, w.q)
    assert np.linalg.norm(r1["virial"] - Wk) / np.linalg.norm(Wk) > 1e-1


def test_planted_derivative_sign(ref, monkeypatch):
    """A sign slip in the assignment polynomial's derivative flips the ad
    field: the ad forces leave the Ewald forces (5e-4 unplanted) by ~2."""
    w, g, _, Fk = ref
    real = po.bspline_deriv
    monkeypatch.setattr(po, "bspline_deriv", lambda P, s: -real(P, s))
    ferr, _ = _errors(w, g, 1.0, Fk, mode="ad")
    assert ferr > 0.5


def test_planted_transposed_field_components(ref, monkeypatch):
    """Interpolating E_y into F_x (and E_x into F_y) in the ik path."""
    real = po.fieldforce_ik
    monkeypatch.setattr(po, "fieldforce_ik",
                        lambda x, q, f, *a, **k: real(x, q, [f[1], f[0], f[2]], *a, **k))
    ferr, _ = _errors(*ref)
    assert ferr > 0.5


def test_planted_background_sign(monkeypatch):
    """The neutralising-background energy with the wrong sign, on a strongly
    non-neutral system (200 positive charges), against the direct Ewald sum."""
    r = np.random.default_rng(5)
    box, mesh, P, g = (12.0, 12.0, 12.0), (16, 16, 16), 5, 0.35
    x = r.uniform(0, 12, (200, 3))
    q = np.abs(r.normal(size=200)) + 0.2
    E = ewald_kspace(x, q, box, g, 1.0)[0] + self_energy(q, g, 1.0) + background_energy(q, g, 1.0, box)

    def err():
        return abs(po.OraclePPPM(box, mesh, P, g, "ik", 1.0).compute(x, q)["energy"] - E) / abs(E)

    assert err() < 1e-6
    real = po.background_energy
    monkeypatch.setattr(po, "background_energy", lambda q_, g_, C, b: -real(q_, g_, C, b))
    assert err() > 0.5
