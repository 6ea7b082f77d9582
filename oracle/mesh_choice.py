"""Mesh and g_ewald choice for a target accuracy -- TEST INFRASTRUCTURE.

The paper leaves the choice of mesh, order and splitting parameter to LAMMPS,
which derives the mesh from a requested accuracy (Sec. 4 "tunable
parameters": r_C, the relative accuracy, the stencil size; a larger stencil
allows a coarser mesh), and it fixes mesh sizes that upset its FFT library
(Sec. 5, "adjust grid sizes").  Readings used here (the paper prints no
formula):

* FFT-friendly sizes: a mesh edge is rounded up to the next number whose
  prime factors are 2, 3, 5, 7 (kind 1, what cuFFT handles in its fast
  kernels), or to the next power of two (kind 2, what the hand-written FFT
  handles); kind 0 leaves it as it is.
* k-space error of an ik mesh: the Hockney-Eastwood functional of the optimal
  influence function (Deserno & Holm, J. Chem. Phys. 109, 7694 (1998)):
      Q = (1/V) sum_{k in mesh, k != 0} { sum_m |R(k_m)|^2
            - [sum_m U^2(k_m) (k . k_m) phi(k_m)]^2 / (k^2 [sum_m U^2(k_m)]^2) }
  with phi(k) = 4 pi exp(-k^2/4g^2)/k^2, R(k) = -i k phi(k) (the reciprocal
  Ewald force between unit charges), U(k) = prod_d sinc^P(k_d h_d / 2),
  k_m = k + 2 pi m / h, the alias sums over |m_d| <= 2 except the full
  denominator sum.  For N charges placed at random,
      dF_rms = (sum q^2) sqrt(Q / (N V))   (force in units of C e^2 / A^2).
* k-space error of an ad mesh (reading R20): the same functional for forces
  taken as the gradient of the interpolated potential.  Averaging the squared
  difference between the mesh force and R over source and target positions,
  a target alias k_m now carries its own derivative i k_m (ik carries i k for
  every alias), so per k
      Q_k(G) = G^2 [sum_m U^2(k_m)] [sum_m U^2(k_m) k_m^2]
               - 2 G sum_m U^2(k_m) k_m^2 phi(k_m) + sum_m |R(k_m)|^2,
  evaluated at the plan's own ad influence function G (R6, influence_ad);
  the two plain alias sums run to |m_d| <= 2000 (the second one separates
  over dimensions), the others to |m_d| <= 2.  Same dF_rms.
* Choice: g from the real-space estimate (``estimate_g_ewald``); then, with
  c = P, P + 1, ... points along the longest edge, mesh_d =
  fft_size(ceil(L_d c / L_max)) until dF_rms <= rel_acc (the same reading
  of rel_acc as the real-space estimate), skipping repeated meshes.
"""
from __future__ import annotations

import math

import numpy as np

from .pppm_oracle import _half_k, alias_sum_u2, estimate_g_ewald, half_spectrum_weights, influence_ad

__all__ = ["fft_size", "kspace_error_ik", "kspace_error_ad", "kspace_error", "choose_mesh"]

ALIAS_FULL = 2000

TWO_PI = 2.0 * math.pi


def _prime_factors_ok(m: int, primes) -> bool:
    for p in primes:
        while m % p == 0:
            m //= p
    return m == 1


def fft_size(n: int, kind: int) -> int:
    """Smallest m >= n that is FFT-friendly of the given kind (brute force)."""
    if n < 1 or kind not in (0, 1, 2):
        raise ValueError((n, kind))
    if kind == 0:
        return n
    primes = (2, 3, 5, 7) if kind == 1 else (2,)
    m = n
    while not _prime_factors_ok(m, primes):
        m += 1
    return m


def kspace_error_ik(box, mesh, P: int, g: float, n: int, q2: float, mmax: int = 2) -> float:
    """RMS k-space force error of an ik mesh for n random charges (see module doc)."""
    box = np.asarray(box, dtype=np.float64)
    mesh = np.asarray(mesh, dtype=np.int64)
    h = box / mesh
    V = float(np.prod(box))
    kx, ky, kz = _half_k(box, mesh)
    K2 = kx[:, None, None] ** 2 + ky[None, :, None] ** 2 + kz[None, None, :] ** 2
    inv4g2 = 1.0 / (4.0 * g * g)
    s1 = np.zeros(K2.shape)
    num = np.zeros(K2.shape)
    with np.errstate(divide="ignore", invalid="ignore"):
        for mx in range(-mmax, mmax + 1):
            kmx = kx + TWO_PI * mx / h[0]
            ux = np.sinc(kx * h[0] / TWO_PI + mx) ** (2 * P)
            for my in range(-mmax, mmax + 1):
                kmy = ky + TWO_PI * my / h[1]
                uy = np.sinc(ky * h[1] / TWO_PI + my) ** (2 * P)
                for mz in range(-mmax, mmax + 1):
                    kmz = kz + TWO_PI * mz / h[2]
                    uz = np.sinc(kz * h[2] / TWO_PI + mz) ** (2 * P)
                    km2 = kmx[:, None, None] ** 2 + kmy[None, :, None] ** 2 + kmz[None, None, :] ** 2
                    phi = 4.0 * math.pi * np.exp(-km2 * inv4g2) / km2
                    r2 = km2 * phi * phi  # |R(k_m)|^2
                    dot = (kx[:, None, None] * kmx[:, None, None] + ky[None, :, None] * kmy[None, :, None]
                           + kz[None, None, :] * kmz[None, None, :])
                    u2 = ux[:, None, None] * uy[None, :, None] * uz[None, None, :]
                    t = u2 * dot * phi
                    r2[~np.isfinite(r2)] = 0.0  # k = 0, m = 0 only
                    t[~np.isfinite(t)] = 0.0
                    s1 += r2
                    num += t
        den = alias_sum_u2(kx, h[0], P)[:, None, None] * alias_sum_u2(ky, h[1], P)[None, :, None] \
            * alias_sum_u2(kz, h[2], P)[None, None, :]
        term = s1 - num * num / (K2 * den * den)
    term[0, 0, 0] = 0.0
    w = half_spectrum_weights(int(mesh[2]))[None, None, :]
    Q = float(np.sum(w * term)) / V
    return float(q2) * math.sqrt(Q / (n * V))


def _alias_sums_1d(k, h: float, P: int, mmax: int = ALIAS_FULL):
    """sum_m U1^2(k_m) and sum_m U1^2(k_m) k_m^2 over |m| <= mmax (one dimension)."""
    k = np.asarray(k, dtype=np.float64)
    m = np.arange(-mmax, mmax + 1)
    u = np.sinc(k[:, None] * h / TWO_PI + m[None, :]) ** (2 * P)
    km = k[:, None] + TWO_PI * m[None, :] / h
    return np.sum(u, axis=1), np.sum(u * km * km, axis=1)


def kspace_error_ad(box, mesh, P: int, g: float, n: int, q2: float, mmax: int = 2, conditioning: bool = False):
    """RMS k-space force error of an ad mesh for n random charges (see module doc).

    With conditioning=True, returns (error, kappa), kappa = the sum of the
    three terms' magnitudes over their signed sum: on accurate meshes the
    terms cancel (the Cauchy-Schwarz gap between sum |R|^2 and T^2/(S0 S2)),
    and FP64 rounding of the alias sums is amplified by kappa."""
    box = np.asarray(box, dtype=np.float64)
    mesh = np.asarray(mesh, dtype=np.int64)
    h = box / mesh
    V = float(np.prod(box))
    kx, ky, kz = _half_k(box, mesh)
    G = influence_ad(box, mesh, P, g)
    inv4g2 = 1.0 / (4.0 * g * g)
    r2s = np.zeros(G.shape)
    T = np.zeros(G.shape)
    with np.errstate(divide="ignore", invalid="ignore"):
        for mx in range(-mmax, mmax + 1):
            kmx = kx + TWO_PI * mx / h[0]
            ux = np.sinc(kx * h[0] / TWO_PI + mx) ** (2 * P)
            for my in range(-mmax, mmax + 1):
                kmy = ky + TWO_PI * my / h[1]
                uy = np.sinc(ky * h[1] / TWO_PI + my) ** (2 * P)
                for mz in range(-mmax, mmax + 1):
                    kmz = kz + TWO_PI * mz / h[2]
                    uz = np.sinc(kz * h[2] / TWO_PI + mz) ** (2 * P)
                    km2 = kmx[:, None, None] ** 2 + kmy[None, :, None] ** 2 + kmz[None, None, :] ** 2
                    phi = 4.0 * math.pi * np.exp(-km2 * inv4g2) / km2
                    u2 = ux[:, None, None] * uy[None, :, None] * uz[None, None, :]
                    r2 = km2 * phi * phi  # |R(k_m)|^2
                    t = u2 * km2 * phi    # U^2 (k_m . k_m) phi: the alias's own derivative against R(k_m)
                    r2[~np.isfinite(r2)] = 0.0  # k = 0, m = 0 only
                    t[~np.isfinite(t)] = 0.0
                    r2s += r2
                    T += t
    s0x, s2x = _alias_sums_1d(kx, h[0], P)
    s0y, s2y = _alias_sums_1d(ky, h[1], P)
    s0z, s2z = _alias_sums_1d(kz, h[2], P)
    S0 = s0x[:, None, None] * s0y[None, :, None] * s0z[None, None, :]
    S2 = (s2x[:, None, None] * s0y[None, :, None] * s0z[None, None, :]
          + s0x[:, None, None] * s2y[None, :, None] * s0z[None, None, :]
          + s0x[:, None, None] * s0y[None, :, None] * s2z[None, None, :])
    a, b, c = G * G * S0 * S2, 2.0 * G * T, r2s
    term = a - b + c
    term[0, 0, 0] = 0.0
    w = half_spectrum_weights(int(mesh[2]))[None, None, :]
    Q = float(np.sum(w * term)) / V
    err = float(q2) * math.sqrt(max(Q, 0.0) / (n * V))
    if not conditioning:
        return err
    mag = np.abs(a) + np.abs(b) + np.abs(c)
    mag[0, 0, 0] = 0.0
    return err, float(np.sum(w * mag)) / V / Q


def kspace_error(box, mesh, P: int, g: float, n: int, q2: float, mode: str = "ik") -> float:
    if mode == "ik":
        return kspace_error_ik(box, mesh, P, g, n, q2)
    if mode == "ad":
        return kspace_error_ad(box, mesh, P, g, n, q2)
    raise ValueError(mode)


def choose_mesh(box, n: int, q2: float, P: int, r_cut: float, rel_acc: float, kind: int = 1,
                max_mesh: int = 1024, mode: str = "ik"):
    """(mesh, g, estimated error): the first mesh of the scan that meets rel_acc."""
    box = [float(b) for b in box]
    g = estimate_g_ewald(rel_acc, r_cut, n, q2, box)
    lmax = max(box)
    prev = None
    c = P
    while True:
        mesh = tuple(max(P, fft_size(int(math.ceil(L * c / lmax)), kind)) for L in box)
        if max(mesh) > max_mesh:
            raise ValueError("no mesh up to the size limit meets the accuracy")
        if mesh != prev:
            err = kspace_error(box, mesh, P, g, n, q2, mode)
            if err <= rel_acc:
                return mesh, g, err
            prev = mesh
        c += 1
