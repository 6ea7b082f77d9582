"""Plain FP64 CPU PPPM k-space solver (the oracle) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
arm of ``bench.py`` may use this module.  The CUDA library shares no code with
it: different language, its own coefficient and Green's-function code, and no
tables or constants passed between the two.

What it follows (McDoniel, Hoehnerbach, Canales, Ismail, Bientinesi, "LAMMPS'
PPPM Long-Range Solver for the Second Generation Xeon Phi", arXiv:1702.04250):

* Sec. 2.1, the three PPPM steps: (1) map particle charges onto a grid with a
  stencil, (2) solve Poisson's equation (Eq. "poisson") in reciprocal space:
  forward 3-D FFT, then three inverse FFTs for ik differentiation or one for
  ad, (3) map the result back to the particles with the same stencil, the
  force being F_j = -q_j grad Phi (Eq. "fpot").
* Sec. 3.1, the mapping functions: a loop over atoms, stencil coefficients
  that are the product of three 1-D polynomials of order S (= P here), and a
  triple loop over the S^3 stencil points.  ik multiplies three field values
  per point by the coefficient and sums three totals scaled by the charge
  afterwards; ad multiplies the scalar potential by three derivative
  coefficient sets and does extra per-atom work after the loop.

The paper prints none of the formulas below; it defers to Hockney & Eastwood.
Each is the standard P3M form, taken as the reading of the paper:

R1  Assignment function: the order-P charge-assignment function is the
    centred cardinal B-spline M_P of degree P-1 (P-fold convolution of the
    unit top-hat), evaluated with the Cox-de Boor recursion.
R2  Stencil placement: u = x/h on the wrapped position.  Odd P: anchor
    n = floor(u + 1/2); even P: n = floor(u).  The P stencil points are
    n - (P-1)//2 + k, k = 0..P-1 (mod M), with weights M_P(point - u).
R3  Mesh density rho(p) = (1/h^3) sum_i q_i W_x W_y W_z.
R4  Forward transform is the unnormalised DFT; k = 2 pi m'/L with m' = m for
    m < M/2 and m - M otherwise (an even mesh's Nyquist index is -M/2).
R5  ik influence function (Hockney-Eastwood optimal):
      G(k) = sum_m (k.k_m) R(k_m) U^2(k_m) / (|k|^2 [sum_m U^2(k_m)]^2),
      R(k) = 4 pi exp(-k^2/4g^2)/k^2, U(k) = prod_d sinc^P(k_d h_d/2),
      k_m = k + 2 pi m/h; numerator |m_d| <= 2, denominator per dimension
      summed to |m_d| <= 2000; G(0) = 0.
R6  ad influence function: sum_m R(k_m) U^2(k_m) / [sum_m U^2(k_m)]^2, same
    alias ranges.
R7  phi = (1/M) IDFT(G rho_hat); ik field E_a = (1/M) IDFT(-i k_a G rho_hat)
    with the Nyquist components along a set to zero.
R8  Energy E = (C/2)(h^3)^2/V sum_{k != 0} G |rho_hat|^2 over the full
    spectrum, minus the self term C g/sqrt(pi) sum q^2 and the neutralising
    background C pi Q^2/(2 g^2 V).
R9  Virial W_ab = (C/2)(h^3)^2/V sum G |rho_hat|^2 [delta_ab - 2(1 + k^2/4g^2)
    k_a k_b/k^2]; no background term.
R10 ik force F_i = C q_i sum_p W(p) E(p).
R11 ad force F_i,a = C q_i sum_p (M_P'(p_a - u_a)/h_a) W_b W_c phi(p) minus the
    self force q_i^2 sum_{n=1,2} c_{a,n} sin(2 pi n u_a), where c_{a,n} are the
    axis-aligned Fourier coefficients of the exact self force of a lone charge
    (derived from the Poisson-summed self energy; see ``ad_selfforce_coeffs``).
R12 g_ewald from the real-space force-error estimate
    2 q2 exp(-g^2 rc^2)/sqrt(N rc V) = rel_acc (q2 = sum q^2, in units where
    the force between two unit charges 1 A apart is 1).
R17 Lookup-table coefficients (Sec. 3.1 "precompute"; Table 1's LUT-500 and
    LUT-5000): the coefficients are tabulated at K equally spaced offsets and
    a particle takes the nearest entry.  A nearest-entry table of the exact
    polynomials is the polynomials evaluated at the offset rounded to the
    centre of its bin: delta_q = lo + (floor((delta - lo) K) + 1/2)/K over the
    offset range [lo, lo + 1) (lo = -1/2 for odd P, -1 for even P).  Every
    per-particle use of the offset takes delta_q, the ad self-force sines
    included.  K = 0 means exact coefficients.

Every function works in float64 and is written for reading, not speed.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "bspline", "bspline_deriv", "wrap_positions", "stencil", "make_rho",
    "wavenumbers", "alias_sum_u2", "influence_ik", "influence_ad",
    "half_spectrum_weights", "poisson_ik", "poisson_ad", "energy_virial_mesh",
    "fieldforce_ik", "fieldforce_ad", "fieldforce_ad_uncorrected", "interpolate_potential",
    "ad_selfforce_coeffs",
    "ad_selfforce", "estimate_g_ewald", "OraclePPPM", "self_energy", "lut_offset",
    "background_energy",
]

TWO_PI = 2.0 * math.pi
ALIAS_NUMERATOR = 2
ALIAS_DENOMINATOR = 2000
ALIAS_SELFFORCE = 50


# ----------------------------------------------------------------------------
# R1: assignment function (Sec. 3.1: "the stencil coefficients are the product
# of three polynomials of order equal to the stencil size")
# ----------------------------------------------------------------------------
def bspline(P: int, s) -> np.ndarray:
    """Centred cardinal B-spline M_P(s), support [-P/2, P/2].

    M_1 is the unit top-hat on [-1/2, 1/2); for p > 1
        M_p(s) = [(p/2 + s) M_{p-1}(s + 1/2) + (p/2 - s) M_{p-1}(s - 1/2)] / (p - 1),
    which is the P-fold self-convolution of the top-hat.
    """
    s = np.asarray(s, dtype=np.float64)
    memo = {}

    def f(p, t):  # M_p(s + t/2)
        key = (p, t)
        if key not in memo:
            y = s + 0.5 * t
            if p == 1:
                v = ((y >= -0.5) & (y < 0.5)).astype(np.float64)
            else:
                v = ((0.5 * p + y) * f(p - 1, t + 1) + (0.5 * p - y) * f(p - 1, t - 1)) / (p - 1)
            memo[key] = v
        return memo[key]

    return f(P, 0)


def bspline_deriv(P: int, s) -> np.ndarray:
    """dM_P/ds = M_{P-1}(s + 1/2) - M_{P-1}(s - 1/2)  (P >= 2)."""
    if P < 2:
        raise ValueError("derivative needs P >= 2")
    s = np.asarray(s, dtype=np.float64)
    return bspline(P - 1, s + 0.5) - bspline(P - 1, s - 0.5)


# ----------------------------------------------------------------------------
# R2: particle -> stencil (Sec. 3.1: loop over atoms, compute the coefficients)
# ----------------------------------------------------------------------------
def wrap_positions(x, box) -> np.ndarray:
    """Periodic wrap into [0, L) per dimension (x = L maps to 0)."""
    box = np.asarray(box, dtype=np.float64)
    xw = np.mod(np.asarray(x, dtype=np.float64), box)
    return np.where(xw >= box, 0.0, xw)


def lut_offset(delta, P: int, lut: int):
    """R17: the offset delta = n - u rounded to the centre of its table bin."""
    lo = -0.5 if P % 2 == 1 else -1.0
    b = np.clip(np.floor((delta - lo) * lut), 0, lut - 1)
    return lo + (b + 0.5) / lut


def stencil(u, P: int, M: int, lut: int = 0):
    """Stencil of a particle at grid coordinate u (one dimension).

    Returns (points [N, P] wrapped mod M, offsets s = point - u [N, P]);
    with a table of lut entries (R17) the offsets are those of the rounded
    offset.
    """
    u = np.asarray(u, dtype=np.float64)
    n = np.floor(u + 0.5) if P % 2 == 1 else np.floor(u)
    if lut:
        u = n - lut_offset(n - u, P, lut)
    pts = n[:, None] - (P - 1) // 2 + np.arange(P)[None, :]
    s = pts - u[:, None]
    return np.mod(pts, M).astype(np.int64), s


def _grid_coords(x, box, mesh):
    box = np.asarray(box, dtype=np.float64)
    mesh = np.asarray(mesh, dtype=np.int64)
    h = box / mesh
    xw = wrap_positions(x, box)
    return xw / h[None, :], h


# ----------------------------------------------------------------------------
# R3: make_rho (Sec. 3.1 Map-Charge: charge times coefficient added to the grid)
# ----------------------------------------------------------------------------
def make_rho(x, q, box, mesh, P: int, lut: int = 0) -> np.ndarray:
    """Mesh charge density rho[Mx, My, Mz] = (1/h^3) sum_i q_i Wx Wy Wz."""
    q = np.asarray(q, dtype=np.float64)
    Mx, My, Mz = (int(m) for m in mesh)
    u, h = _grid_coords(x, box, mesh)
    ix, sx = stencil(u[:, 0], P, Mx, lut)
    iy, sy = stencil(u[:, 1], P, My, lut)
    iz, sz = stencil(u[:, 2], P, Mz, lut)
    wx, wy, wz = bspline(P, sx), bspline(P, sy), bspline(P, sz)
    rho = np.zeros(Mx * My * Mz)
    for kx in range(P):
        for ky in range(P):
            flat = (ix[:, kx] * My + iy[:, ky])[:, None] * Mz + iz
            vals = (q * wx[:, kx] * wy[:, ky])[:, None] * wz
            rho += np.bincount(flat.ravel(), vals.ravel(), minlength=rho.size)
    return rho.reshape(Mx, My, Mz) / (h[0] * h[1] * h[2])


# ----------------------------------------------------------------------------
# R4-R6: reciprocal space
# ----------------------------------------------------------------------------
def wavenumbers(M: int, L: float) -> np.ndarray:
    """k = 2 pi m'/L for m = 0..M-1, m' = m (m < M/2) else m - M."""
    m = np.arange(M)
    mp = np.where(m < M / 2.0, m, m - M)
    return TWO_PI * mp / L


def _half_k(box, mesh):
    Mx, My, Mz = (int(m) for m in mesh)
    kx = wavenumbers(Mx, box[0])
    ky = wavenumbers(My, box[1])
    kz = wavenumbers(Mz, box[2])[: Mz // 2 + 1]
    return kx, ky, kz


def alias_sum_u2(k, h: float, P: int, mmax: int = ALIAS_DENOMINATOR) -> np.ndarray:
    """sum_{|m| <= mmax} sinc^{2P}((k + 2 pi m/h) h/2) for each k (1-D)."""
    k = np.asarray(k, dtype=np.float64)
    m = np.arange(-mmax, mmax + 1)
    return np.sum(np.sinc(k[:, None] * h / TWO_PI + m[None, :]) ** (2 * P), axis=1)


def _influence(box, mesh, P, g, ik: bool, mmax=ALIAS_NUMERATOR):
    box = np.asarray(box, dtype=np.float64)
    mesh = np.asarray(mesh, dtype=np.int64)
    h = box / mesh
    kx, ky, kz = _half_k(box, mesh)
    Kx, Ky, Kz = kx[:, None, None], ky[None, :, None], kz[None, None, :]
    num = np.zeros((kx.size, ky.size, kz.size))
    inv4g2 = 1.0 / (4.0 * g * g)
    with np.errstate(divide="ignore", invalid="ignore"):
        for mx in range(-mmax, mmax + 1):
            kmx = kx + TWO_PI * mx / h[0]
            ax = np.exp(-kmx ** 2 * inv4g2) * np.sinc(kx * h[0] / TWO_PI + mx) ** (2 * P)
            for my in range(-mmax, mmax + 1):
                kmy = ky + TWO_PI * my / h[1]
                ay = np.exp(-kmy ** 2 * inv4g2) * np.sinc(ky * h[1] / TWO_PI + my) ** (2 * P)
                for mz in range(-mmax, mmax + 1):
                    kmz = kz + TWO_PI * mz / h[2]
                    az = np.exp(-kmz ** 2 * inv4g2) * np.sinc(kz * h[2] / TWO_PI + mz) ** (2 * P)
                    km2 = kmx[:, None, None] ** 2 + kmy[None, :, None] ** 2 + kmz[None, None, :] ** 2
                    term = (4.0 * math.pi / km2) * (ax[:, None, None] * ay[None, :, None] * az[None, None, :])
                    if ik:
                        dot = Kx * kmx[:, None, None] + Ky * kmy[None, :, None] + Kz * kmz[None, None, :]
                        term = term * dot
                    term[~np.isfinite(term)] = 0.0  # only the k = 0, m = 0 entry
                    num += term
        dx = alias_sum_u2(kx, h[0], P)
        dy = alias_sum_u2(ky, h[1], P)
        dz = alias_sum_u2(kz, h[2], P)
        den = (dx[:, None, None] * dy[None, :, None] * dz[None, None, :]) ** 2
        if ik:
            den = den * (Kx ** 2 + Ky ** 2 + Kz ** 2)
        G = num / den
    G[0, 0, 0] = 0.0
    return G


def influence_ik(box, mesh, P: int, g: float) -> np.ndarray:
    """R5, on the half spectrum [Mx, My, Mz//2+1]."""
    return _influence(box, mesh, P, g, ik=True)


def influence_ad(box, mesh, P: int, g: float) -> np.ndarray:
    """R6, on the half spectrum [Mx, My, Mz//2+1]."""
    return _influence(box, mesh, P, g, ik=False)


def half_spectrum_weights(Mz: int) -> np.ndarray:
    """How many full-spectrum points each kz index of the half spectrum stands
    for: 1 for kz = 0 and (even Mz) the Nyquist plane, 2 otherwise."""
    w = np.full(Mz // 2 + 1, 2.0)
    w[0] = 1.0
    if Mz % 2 == 0:
        w[-1] = 1.0
    return w


# ----------------------------------------------------------------------------
# R7: Poisson step (Sec. 2.1 step 2, Sec. 3.2: forward FFT, 3 (ik) / 1 (ad)
# inverse FFTs).  numpy's rfftn is the unnormalised forward DFT and irfftn
# includes the 1/M of the inverse.
# ----------------------------------------------------------------------------
def poisson_ik(rho, G, box):
    """Returns (rho_hat, [Ex, Ey, Ez]) on the mesh."""
    mesh = rho.shape
    rho_hat = np.fft.rfftn(rho)
    phi_hat = G * rho_hat
    ks = _half_k(np.asarray(box, dtype=np.float64), mesh)
    fields = []
    for a in range(3):
        shape = [1, 1, 1]
        shape[a] = ks[a].size
        Ehat = -1j * ks[a].reshape(shape) * phi_hat
        if mesh[a] % 2 == 0:
            sl = [slice(None)] * 3
            sl[a] = mesh[a] // 2
            Ehat[tuple(sl)] = 0.0
        fields.append(np.fft.irfftn(Ehat, s=mesh, axes=(0, 1, 2)))
    return rho_hat, fields


def poisson_ad(rho, G):
    """Returns (rho_hat, phi) on the mesh."""
    rho_hat = np.fft.rfftn(rho)
    return rho_hat, np.fft.irfftn(G * rho_hat, s=rho.shape, axes=(0, 1, 2))


# ----------------------------------------------------------------------------
# R8, R9: energy and virial
# ----------------------------------------------------------------------------
def self_energy(q, g, C):
    q = np.asarray(q, dtype=np.float64)
    return -C * g / math.sqrt(math.pi) * float(np.sum(q * q))


def background_energy(q, g, C, box):
    Q = float(np.sum(np.asarray(q, dtype=np.float64)))
    V = float(np.prod(np.asarray(box, dtype=np.float64)))
    return -C * math.pi * Q * Q / (2.0 * g * g * V)


def energy_virial_mesh(rho_hat, G, box, mesh, g, C):
    """E_mesh and W_ab summed over the full spectrum (half spectrum x weights)."""
    box = np.asarray(box, dtype=np.float64)
    mesh = np.asarray(mesh, dtype=np.int64)
    h = box / mesh
    vcell = float(np.prod(h))
    V = float(np.prod(box))
    pref = 0.5 * C * vcell * vcell / V
    s = half_spectrum_weights(int(mesh[2]))[None, None, :] * G * np.abs(rho_hat) ** 2
    E = pref * float(np.sum(s))
    kx, ky, kz = _half_k(box, mesh)
    K = [kx[:, None, None], ky[None, :, None], kz[None, None, :]]
    k2 = K[0] ** 2 + K[1] ** 2 + K[2] ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        fac = 2.0 * (1.0 + k2 / (4.0 * g * g)) / k2
    fac[0, 0, 0] = 0.0
    vir = np.empty(6)
    for n, (a, b) in enumerate(((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))):
        delta = 1.0 if a == b else 0.0
        vir[n] = pref * float(np.sum(s * (delta - fac * K[a] * K[b])))
    return E, vir


# ----------------------------------------------------------------------------
# R10, R11: Distribute-Force (Sec. 3.1)
# ----------------------------------------------------------------------------
def _weights(x, box, mesh, P, deriv=False, lut=0):
    u, h = _grid_coords(x, box, mesh)
    out = []
    for d in range(3):
        idx, s = stencil(u[:, d], P, int(mesh[d]), lut)
        w = bspline(P, s)
        dw = bspline_deriv(P, s) if deriv else None
        out.append((idx, w, dw))
    return out, u, h


def fieldforce_ik(x, q, fields, box, mesh, P, C, lut=0):
    """F_i = C q_i sum over the P^3 stencil of W * (Ex, Ey, Ez)."""
    q = np.asarray(q, dtype=np.float64)
    (ix, wx, _), (iy, wy, _), (iz, wz, _) = _weights(x, box, mesh, P, lut=lut)[0]
    acc = np.zeros((q.size, 3))
    for kx in range(P):
        for ky in range(P):
            wxy = wx[:, kx] * wy[:, ky]
            for a in range(3):
                E = fields[a]
                acc[:, a] += wxy * np.sum(wz * E[ix[:, kx][:, None], iy[:, ky][:, None], iz], axis=1)
    return C * q[:, None] * acc


def interpolate_potential(x, phi, box, mesh, P, lut=0):
    """phi(x_i) = sum over the stencil of W * phi (transpose of make_rho)."""
    (ix, wx, _), (iy, wy, _), (iz, wz, _) = _weights(x, box, mesh, P, lut=lut)[0]
    out = np.zeros(ix.shape[0])
    for kx in range(P):
        for ky in range(P):
            out += wx[:, kx] * wy[:, ky] * np.sum(wz * phi[ix[:, kx][:, None], iy[:, ky][:, None], iz], axis=1)
    return out


def fieldforce_ad_uncorrected(x, q, phi, box, mesh, P, C, lut=0):
    """C q_i E_a with E_a = sum (M_P'(p_a - u_a)/h_a) W_b W_c phi(p)."""
    q = np.asarray(q, dtype=np.float64)
    (ix, wx, dx), (iy, wy, dy), (iz, wz, dz) = _weights(x, box, mesh, P, deriv=True, lut=lut)[0]
    h = np.asarray(box, dtype=np.float64) / np.asarray(mesh, dtype=np.float64)
    e = np.zeros((q.size, 3))
    for kx in range(P):
        for ky in range(P):
            vals = phi[ix[:, kx][:, None], iy[:, ky][:, None], iz]
            e[:, 0] += dx[:, kx] * wy[:, ky] * np.sum(wz * vals, axis=1) / h[0]
            e[:, 1] += wx[:, kx] * dy[:, ky] * np.sum(wz * vals, axis=1) / h[1]
            e[:, 2] += wx[:, kx] * wy[:, ky] * np.sum(dz * vals, axis=1) / h[2]
    return C * q[:, None] * e


def _b_alias(kappa, n, P, mmax=ALIAS_SELFFORCE):
    """B(kappa, n) = sum_m U1(kappa + 2 pi m) U1(kappa + 2 pi (m - n)),
    U1(kappa) = sinc^P(kappa/2), for grid-unit wavenumbers kappa = k h."""
    m = np.arange(-mmax, mmax + 1)
    t = kappa[:, None] / TWO_PI
    return np.sum(np.sinc(t + m[None, :]) ** P * np.sinc(t + m[None, :] - n) ** P, axis=1)


def ad_selfforce_coeffs(G, box, mesh, P, C) -> np.ndarray:
    """c[a, n-1], n = 1, 2: axis-aligned sine coefficients of the self force.

    A lone charge q at grid coordinate u has PPPM energy
      E_self(u) = (C q^2 / 2V) sum_k G(k) prod_d A_d(k_d h_d, u_d),
      A(kappa, u) = |sum_m U1(kappa + 2 pi m) e^{-i(kappa + 2 pi m) u}|^2
                  = B(kappa, 0) + 2 sum_{n>=1} B(kappa, n) cos(2 pi n u)
    (Poisson summation of the stencil sum).  The ad force is the exact
    gradient of the PPPM energy, so the lone charge feels -dE_self/dx.  Its
    terms that vary along axis a alone are q^2 sum_n c_{a,n} sin(2 pi n u_a),
      c_{a,n} = (2 pi n C / (h_a V)) sum_k G(k) B_a(kappa_a, n) prod_{b!=a} B_b(kappa_b, 0).
    """
    box = np.asarray(box, dtype=np.float64)
    mesh = np.asarray(mesh, dtype=np.int64)
    h = box / mesh
    V = float(np.prod(box))
    ks = _half_k(box, mesh)
    wz = half_spectrum_weights(int(mesh[2]))
    GW = G * wz[None, None, :]
    c = np.zeros((3, 2))
    for a in range(3):
        for n in (1, 2):
            f = []
            for d in range(3):
                f.append(_b_alias(ks[d] * h[d], n if d == a else 0, P))
            s = float(np.sum(GW * f[0][:, None, None] * f[1][None, :, None] * f[2][None, None, :]))
            c[a, n - 1] = TWO_PI * n * C / (h[a] * V) * s
    return c


def ad_selfforce(x, q, coeffs, box, mesh, P=None, lut=0):
    """q_i^2 sum_n c_{a,n} sin(2 pi n u_a) for each particle and axis (with
    a coefficient table, u from the rounded offset, R17)."""
    q = np.asarray(q, dtype=np.float64)
    u, _ = _grid_coords(x, box, mesh)
    if lut:
        n = np.floor(u + 0.5) if P % 2 == 1 else np.floor(u)
        u = n - lut_offset(n - u, P, lut)
    sf = np.zeros_like(u)
    for a in range(3):
        for n in (1, 2):
            sf[:, a] += coeffs[a, n - 1] * np.sin(TWO_PI * n * u[:, a])
    return (q * q)[:, None] * sf


def fieldforce_ad(x, q, phi, box, mesh, P, C, coeffs=None, lut=0):
    F = fieldforce_ad_uncorrected(x, q, phi, box, mesh, P, C, lut)
    if coeffs is not None:
        F = F - ad_selfforce(x, q, coeffs, box, mesh, P, lut)
    return F


# ----------------------------------------------------------------------------
# R12: g_ewald
# ----------------------------------------------------------------------------
def estimate_g_ewald(rel_acc, r_cut, n, q2, box) -> float:
    """Solve 2 q2 exp(-g^2 rc^2)/sqrt(N rc V) = rel_acc for g."""
    V = float(np.prod(np.asarray(box, dtype=np.float64)))
    arg = rel_acc * math.sqrt(n * r_cut * V) / (2.0 * q2)
    if not (0.0 < arg < 1.0):
        raise ValueError("no positive g_ewald satisfies the estimate")
    return math.sqrt(-math.log(arg)) / r_cut


# ----------------------------------------------------------------------------
# The whole path (Sec. 2.1 steps 1-3)
# ----------------------------------------------------------------------------
class OraclePPPM:
    """Set up once per (box, mesh, P, g, mode); ``compute`` runs steps 1-3."""

    def __init__(self, box, mesh, order, g_ewald, mode="ik", qqrd2e=1.0, selfforce=True, lut=0):
        if mode not in ("ik", "ad"):
            raise ValueError(mode)
        if order < 2:
            raise ValueError("order >= 2")
        self.box = np.asarray(box, dtype=np.float64)
        self.mesh = tuple(int(m) for m in mesh)
        self.P = int(order)
        self.g = float(g_ewald)
        self.mode = mode
        self.C = float(qqrd2e)
        self.lut = int(lut)  # R17: coefficient table entries, 0 = exact
        if mode == "ik":
            self.G = influence_ik(self.box, self.mesh, self.P, self.g)
            self.sf = None
        else:
            self.G = influence_ad(self.box, self.mesh, self.P, self.g)
            self.sf = ad_selfforce_coeffs(self.G, self.box, self.mesh, self.P, self.C) if selfforce else None

    def compute(self, x, q, keep=False, subset=None):
        """Forces, energy and virial.  ``subset``: indices of the particles
        whose forces are wanted (all particles still build the mesh)."""
        x = np.asarray(x, dtype=np.float64)
        q = np.asarray(q, dtype=np.float64)
        rho = make_rho(x, q, self.box, self.mesh, self.P, self.lut)
        xs, qs = (x, q) if subset is None else (x[subset], q[subset])
        out = {}
        if self.mode == "ik":
            rho_hat, fields = poisson_ik(rho, self.G, self.box)
            f = fieldforce_ik(xs, qs, fields, self.box, self.mesh, self.P, self.C, self.lut)
            if keep:
                out["fields"] = fields
        else:
            rho_hat, phi = poisson_ad(rho, self.G)
            f = fieldforce_ad(xs, qs, phi, self.box, self.mesh, self.P, self.C, self.sf, self.lut)
            if keep:
                out["phi"] = phi
        E_mesh, vir = energy_virial_mesh(rho_hat, self.G, self.box, self.mesh, self.g, self.C)
        energy = E_mesh + self_energy(q, self.g, self.C) + background_energy(q, self.g, self.C, self.box)
        out.update(f=f, energy=energy, energy_mesh=E_mesh, virial=vir)
        if keep:
            out.update(rho=rho, rho_hat=rho_hat)
        return out

    def potential_mesh(self, x, q):
        """phi on the mesh from this plan's G (the ik plan's G for ik)."""
        rho = make_rho(x, q, self.box, self.mesh, self.P, self.lut)
        return np.fft.irfftn(self.G * np.fft.rfftn(rho), s=self.mesh, axes=(0, 1, 2))

    def energy_gradients(self, x, q):
        """Exact gradients of this plan's energy: dE/dx [N,3], dE/dq [N].

        dE/dx_i = C q_i sum_p dW/dx_i phi(p) = -(uncorrected ad force);
        dE/dq_i = C phi(x_i) - 2 C g q_i/sqrt(pi) - C pi Q/(g^2 V).
        """
        x = np.asarray(x, dtype=np.float64)
        q = np.asarray(q, dtype=np.float64)
        phi = self.potential_mesh(x, q)
        dEdx = -fieldforce_ad_uncorrected(x, q, phi, self.box, self.mesh, self.P, self.C, self.lut)
        V = float(np.prod(self.box))
        dEdq = (self.C * interpolate_potential(x, phi, self.box, self.mesh, self.P, self.lut)
                - 2.0 * self.C * self.g * q / math.sqrt(math.pi)
                - self.C * math.pi * float(np.sum(q)) / (self.g * self.g * V))
        return dEdx, dEdq
