"""Pins of the oracle's reciprocal-space pieces (readings R4-R7).

The FFT conventions are checked against a brute-force DFT; the aliased
denominator against Hockney & Eastwood's closed forms and against its
Poisson-summed finite form; the influence functions against their small-k
limit (the bare Ewald kernel) and against k -> -k symmetry.
"""
import math

import numpy as np
import pytest

from oracle import (alias_sum_u2, bspline, influence_ad, influence_ik, poisson_ad,
                    poisson_ik, wavenumbers)

GOLDEN = __file__.rsplit("/", 1)[0] + "/golden/alias_sums.txt"


def _brute_dft(a):
    Mx, My, Mz = a.shape
    out = np.zeros((Mx, My, Mz // 2 + 1), dtype=complex)
    n = np.stack(np.meshgrid(np.arange(Mx), np.arange(My), np.arange(Mz), indexing="ij"), -1)
    for i in range(Mx):
        for j in range(My):
            for k in range(Mz // 2 + 1):
                ph = 2 * np.pi * (i * n[..., 0] / Mx + j * n[..., 1] / My + k * n[..., 2] / Mz)
                out[i, j, k] = np.sum(a * np.exp(-1j * ph))
    return out


@pytest.mark.parametrize("shape", [(4, 6, 5), (3, 5, 6)])
def test_fft_convention_matches_brute_force_dft(shape):
    a = np.random.default_rng(1).normal(size=shape)
    np.testing.assert_allclose(np.fft.rfftn(a), _brute_dft(a), atol=1e-12)
    # irfftn is (1/M) times the unnormalised inverse
    back = np.fft.irfftn(np.fft.rfftn(a), s=shape)
    np.testing.assert_allclose(back, a, atol=1e-13)


def test_wavenumbers_nyquist_is_negative():
    k = wavenumbers(8, 4.0)
    np.testing.assert_allclose(k * 4.0 / (2 * np.pi), [0, 1, 2, 3, -4, -3, -2, -1])
    k = wavenumbers(7, 7.0)
    np.testing.assert_allclose(k * 7.0 / (2 * np.pi), [0, 1, 2, 3, -3, -2, -1])


def _golden():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        v = line.split()
        out[int(v[0])] = [float(c) for c in v[1:]]
    return out


@pytest.mark.parametrize("P", [1, 2, 3])
def test_alias_sum_closed_forms(P):
    coeffs = _golden()[P]
    h = 0.7
    k = np.linspace(-np.pi / h, np.pi / h, 41)
    s2 = np.sin(k * h / 2) ** 2
    ref = sum(c * s2 ** j for j, c in enumerate(coeffs))
    # P = 1 converges only like 1/mmax; the path uses P >= 2
    tol = 1e-3 if P == 1 else 1e-12
    np.testing.assert_allclose(alias_sum_u2(k, h, P), ref, atol=tol)


@pytest.mark.parametrize("P", [2, 3, 4, 5, 6, 7])
def test_alias_sum_equals_poisson_summed_spline(P):
    """sum_m sinc^{2P}(kh/2 + pi m) = sum_g M_{2P}(g) cos(k h g): the
    discrete-time Fourier transform of the order-2P spline at the integers."""
    h = 1.3
    k = np.linspace(-np.pi / h, np.pi / h, 33)
    g = np.arange(-P, P + 1)
    ref = np.sum(bspline(2 * P, g)[None, :] * np.cos(k[:, None] * h * g[None, :]), axis=1)
    np.testing.assert_allclose(alias_sum_u2(k, h, P), ref, atol=1e-12)


@pytest.mark.parametrize("mode", ["ik", "ad"])
def test_influence_small_k_limit(mode):
    """For k h -> 0 the aliases vanish and U -> 1, so G -> 4 pi e^{-k^2/4g^2}/k^2."""
    box, mesh, P, g = (40.0, 40.0, 40.0), (128, 128, 128), 5, 0.3
    f = influence_ik if mode == "ik" else influence_ad
    G = f(box, (16, 16, 16), P, g)  # coarse call only to exercise shapes
    assert G.shape == (16, 16, 9)
    # fine mesh along z only is enough for the smallest k; use a thin mesh
    G = f(box, (4, 4, 128), P, g)
    kz = 2 * np.pi / 40.0
    ref = 4 * np.pi * np.exp(-kz * kz / (4 * g * g)) / (kz * kz)
    h = 40.0 / 128
    # relative deviation is O((k h)^2): sinc^{2P} and the denominator differ at that order
    assert abs(G[0, 0, 1] / ref - 1) < (kz * h) ** 2
    assert G[0, 0, 0] == 0.0


@pytest.mark.parametrize("mode", ["ik", "ad"])
def test_influence_symmetry(mode):
    f = influence_ik if mode == "ik" else influence_ad
    G = f((10.0, 12.0, 14.0), (10, 12, 8), 4, 0.5)
    # k -> -k within the kz = 0 plane: (mx, my) -> (-mx, -my)
    plane = G[:, :, 0]
    flipped = np.roll(plane[::-1, ::-1], shift=(1, 1), axis=(0, 1))
    np.testing.assert_allclose(plane, flipped, rtol=1e-13, atol=0)
    # ik's Nyquist entries cancel to ~0 (k.k_m of the m=0 and m=1 aliases are
    # opposite), so allow round-off below zero
    assert np.all(G >= -1e-12 * G.max())


def test_poisson_ik_is_minus_gradient_of_phi():
    """E = -grad phi: with the Nyquist planes zeroed, each ik field component
    equals the spectral derivative of the ad-style potential phi."""
    r = np.random.default_rng(2)
    rho = r.normal(size=(8, 10, 12))
    rho -= rho.mean()
    G = influence_ad((8.0, 10.0, 12.0), rho.shape, 4, 0.8)
    _, phi = poisson_ad(rho, G)
    _, E = poisson_ik(rho, G, (8.0, 10.0, 12.0))
    for a, L in enumerate((8.0, 10.0, 12.0)):
        M = rho.shape[a]
        k = wavenumbers(M, L)
        k[M // 2] = 0.0  # drop the Nyquist mode
        shape = [1, 1, 1]
        shape[a] = M
        dphi = np.real(np.fft.ifftn(1j * k.reshape(shape) * np.fft.fftn(phi)))
        np.testing.assert_allclose(E[a], -dphi, atol=1e-12 * np.abs(E[a]).max())
