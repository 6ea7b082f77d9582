"""Direct Ewald sums in FP64 -- TEST INFRASTRUCTURE.

PPPM approximates the reciprocal-space half of Ewald's split of the Coulomb
interaction (Sec. 2.1 of McDoniel et al., arXiv:1702.04250: a short-ranged
screened part summed directly within r_C and a smooth long-ranged part solved
on a grid).  These routines compute the exact reciprocal sum and a brute-force
real-space sum so the oracle itself can be checked against the quantity it
approximates and against the NaCl Madelung constant.

Reciprocal part, over k = 2 pi n / L, n integer, k != 0:
  E_k  = (C / 2V) sum_k A(k) |S(k)|^2,  A(k) = 4 pi exp(-k^2/4g^2)/k^2,
  S(k) = sum_j q_j exp(-i k.r_j),
  F_i  = (C q_i / V) sum_k A(k) k Im(S(k) exp(i k.r_i)),
  W_ab = (C / 2V) sum_k A(k)|S(k)|^2 [delta_ab - 2(1 + k^2/4g^2) k_a k_b / k^2].
Real part: E_r = C sum_{i<j} q_i q_j erfc(g r)/r over minimum images
(r_C < L/2), forces and virial sum_{pairs} r_a F_b.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc

__all__ = ["ewald_kspace", "ewald_real", "ewald_kvectors"]


def ewald_kvectors(box, g, tol=1e-16):
    """Half-space integer vectors n (first nonzero component > 0) with
    exp(-k^2/4g^2) >= tol, and their k = 2 pi n / L."""
    box = np.asarray(box, dtype=np.float64)
    kmax = 2.0 * g * math.sqrt(math.log(1.0 / tol))
    nmax = [int(math.floor(kmax * L / (2 * math.pi))) for L in box]
    rng = [np.arange(-m, m + 1) for m in nmax]
    n = np.stack(np.meshgrid(*rng, indexing="ij"), axis=-1).reshape(-1, 3)
    k = 2 * math.pi * n / box[None, :]
    k2 = np.sum(k * k, axis=1)
    first = np.where(n[:, 0] != 0, n[:, 0], np.where(n[:, 1] != 0, n[:, 1], n[:, 2]))
    keep = (first > 0) & (k2 <= kmax * kmax)
    return n[keep], k[keep]


def ewald_kspace(x, q, box, g, C, tol=1e-16, chunk=512):
    """Exact reciprocal-space energy (without self/background terms), forces
    and virial [xx, yy, zz, xy, xz, yz].  Each half-space k stands for +-k."""
    x = np.asarray(x, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    V = float(np.prod(box))
    _, k = ewald_kvectors(box, g, tol)
    E = 0.0
    F = np.zeros_like(x)
    vir = np.zeros(6)
    pairs = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))
    for s in range(0, k.shape[0], chunk):
        kc = k[s:s + chunk]
        k2 = np.sum(kc * kc, axis=1)
        A = 4 * math.pi * np.exp(-k2 / (4 * g * g)) / k2
        phase = x @ kc.T                      # [N, nk]
        c, sn = np.cos(phase), np.sin(phase)
        Sre = q @ c                           # S = sum q e^{-ik.r}
        Sim = -(q @ sn)
        S2 = Sre * Sre + Sim * Sim
        E += 2.0 * float(np.sum(A * S2))
        # Im(S e^{ik.r_i}) = Sre sin(k.r_i) + Sim cos(k.r_i)
        im = sn * Sre[None, :] + c * Sim[None, :]
        F += 2.0 * (q[:, None] * ((A[None, :] * im) @ kc))
        for n, (a, b) in enumerate(pairs):
            d = 1.0 if a == b else 0.0
            vir[n] += 2.0 * float(np.sum(A * S2 * (d - 2.0 * (1.0 + k2 / (4 * g * g)) * kc[:, a] * kc[:, b] / k2)))
    return C / (2 * V) * E, C / V * F, C / (2 * V) * vir


def ewald_real(x, q, box, g, r_cut, C, chunk=256):
    """Brute-force real-space energy, forces and virial over minimum images
    within r_cut (requires r_cut < L/2)."""
    x = np.asarray(x, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    if r_cut >= 0.5 * float(np.min(box)):
        raise ValueError("minimum image needs r_cut < L/2")
    N = x.shape[0]
    E = 0.0
    F = np.zeros_like(x)
    vir = np.zeros(6)
    pairs = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))
    for s in range(0, N, chunk):
        d = x[s:s + chunk, None, :] - x[None, :, :]       # r_i - r_j
        d -= box * np.round(d / box)
        r2 = np.sum(d * d, axis=2)
        ii = np.arange(s, min(s + chunk, N))[:, None]
        jj = np.arange(N)[None, :]
        mask = (r2 < r_cut * r_cut) & (jj != ii)
        r = np.sqrt(np.where(mask, r2, 1.0))
        qq = q[s:s + chunk, None] * q[None, :]
        e = np.where(mask, qq * erfc(g * r) / r, 0.0)
        E += 0.5 * float(np.sum(e))
        # |F| / r along (r_i - r_j): q q [erfc(gr)/r + 2g/sqrt(pi) e^{-g^2 r^2}] / r^2
        fr = np.where(mask, qq * (erfc(g * r) / r + 2 * g / math.sqrt(math.pi) * np.exp(-g * g * r * r)) / (r * r), 0.0)
        F[s:s + chunk] += np.sum(fr[:, :, None] * d, axis=1)
        for n, (a, b) in enumerate(pairs):
            vir[n] += 0.5 * float(np.sum(fr * d[:, :, a] * d[:, :, b]))
    return C * E, C * F, C * vir
