"""Seeded synthetic inputs for the PPPM k-space path.

This module only draws particles: positions, charges and box/mesh parameters.
It holds none of the method's arithmetic (no assignment weights, no Green's
function, no Ewald parameter estimate), so that both the CUDA path and the
FP64 oracle can be fed the same arrays without sharing any PPPM code.

The paper benchmarks LAMMPS on SPC/E water (Sec. 2.4: 36,000 atoms in a cubic
box).  That input deck is not available here, so ``water_like`` stands in for
it using only its composition: rigid 3-site molecules with the SPC/E charges
(O -0.8476 e, H +0.4238 e), 1.0 A O-H bonds and a 109.47 degree H-O-H angle,
placed on a jittered cubic lattice with uniformly random orientations.

All generators use numpy's PCG64 with an explicit seed and return float64
arrays; callers cast to float32 for the FP32 path.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

Q_OXYGEN = -0.8476
Q_HYDROGEN = 0.4238
OH_BOND = 1.0
HOH_ANGLE_DEG = 109.47

#: Coulomb constant in LAMMPS "real" units, kcal*A/(mol*e^2).
QQRD2E_REAL = 332.06371


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_alternating(n: int, box, seed: int):
    """n point charges uniform in [0, L)^3, q = +1, -1, +1, ... by index."""
    box = np.asarray(box, dtype=np.float64)
    r = rng(seed)
    x = r.random((n, 3)) * box
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    return x, q


def _random_rotations(r: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random rotation matrices from uniform unit quaternions (Shoemake)."""
    u1, u2, u3 = r.random(n), r.random(n), r.random(n)
    a = np.sqrt(1.0 - u1)
    b = np.sqrt(u1)
    qw = a * np.sin(2 * np.pi * u2)
    qx = a * np.cos(2 * np.pi * u2)
    qy = b * np.sin(2 * np.pi * u3)
    qz = b * np.cos(2 * np.pi * u3)
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (qy * qy + qz * qz)
    R[:, 0, 1] = 2 * (qx * qy - qz * qw)
    R[:, 0, 2] = 2 * (qx * qz + qy * qw)
    R[:, 1, 0] = 2 * (qx * qy + qz * qw)
    R[:, 1, 1] = 1 - 2 * (qx * qx + qz * qz)
    R[:, 1, 2] = 2 * (qy * qz - qx * qw)
    R[:, 2, 0] = 2 * (qx * qz - qy * qw)
    R[:, 2, 1] = 2 * (qy * qz + qx * qw)
    R[:, 2, 2] = 1 - 2 * (qx * qx + qy * qy)
    return R


def water_like(n_mol: int, box_edge: float, seed: int, jitter: float = 0.25):
    """Rigid 3-site water-like molecules in a cubic periodic box.

    Oxygens sit on a cubic lattice of ceil(n_mol^(1/3)) sites per edge; the
    lattice is truncated to n_mol sites in seeded random order and every site
    is jittered uniformly by +-jitter * spacing.  Each molecule gets a
    uniformly random orientation.  Positions are wrapped into [0, L).
    Returns (x [3*n_mol, 3], q [3*n_mol]) ordered O, H, H per molecule.
    """
    r = rng(seed)
    side = int(math.ceil(n_mol ** (1.0 / 3.0) - 1e-9))
    while side ** 3 < n_mol:
        side += 1
    spacing = box_edge / side
    sites = np.stack(np.meshgrid(np.arange(side), np.arange(side), np.arange(side),
                                 indexing="ij"), axis=-1).reshape(-1, 3).astype(np.float64)
    pick = r.permutation(sites.shape[0])[:n_mol]
    o = (sites[pick] + 0.5) * spacing
    o += (r.random((n_mol, 3)) * 2.0 - 1.0) * jitter * spacing
    half = math.radians(HOH_ANGLE_DEG) / 2.0
    h_local = np.array([[math.sin(half), 0.0, math.cos(half)],
                        [-math.sin(half), 0.0, math.cos(half)]]) * OH_BOND
    R = _random_rotations(r, n_mol)
    h = o[:, None, :] + np.einsum("mij,kj->mki", R, h_local)
    x = np.empty((n_mol, 3, 3))
    x[:, 0] = o
    x[:, 1:] = h
    x = x.reshape(-1, 3)
    x = np.mod(x, box_edge)
    x[x >= box_edge] = 0.0
    q = np.tile(np.array([Q_OXYGEN, Q_HYDROGEN, Q_HYDROGEN]), n_mol)
    return x, q


def rock_salt(n_side: int, a: float):
    """NaCl-type lattice: n_side^3 sites (n_side even) with spacing a and
    charges +1/-1 alternating with the parity of i+j+k.  Box edge n_side*a."""
    assert n_side % 2 == 0
    idx = np.stack(np.meshgrid(np.arange(n_side), np.arange(n_side), np.arange(n_side),
                               indexing="ij"), axis=-1).reshape(-1, 3)
    x = idx.astype(np.float64) * a
    q = np.where(idx.sum(axis=1) % 2 == 0, 1.0, -1.0)
    return x, q


@dataclass
class Workload:
    """One PPPM problem: particles, box, mesh and solver parameters.

    g_ewald is not stored: it is derived by each side from (rel_acc, r_cut),
    which is the method's setup arithmetic and therefore not this module's.
    """
    name: str
    x: np.ndarray
    q: np.ndarray
    box: tuple
    mesh: tuple
    order: int
    modes: tuple
    rel_acc: float = 1e-4
    r_cut: float = 10.0
    qqrd2e: float = QQRD2E_REAL
    notes: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.q.shape[0])


SEED_BASE = 1702


def config(name: str) -> Workload:
    """The five synthetic workloads (seed = 1702 + config number).

    c1  4096 +-1 charges, 24 A cube, mesh 16^3, P=5, ik
    c2  10,667 water-like molecules (32,001 charges), 68 A cube, 64^3, P=5
    c3  682,667 molecules (2,048,001 charges), 272 A cube, 256^3, P=7, ad
    c5  33,333 molecules (99,999 charges), 100 A cube, 96^3, P=5, ik
    (c4, the batch of 256 systems, is built by ``batch_systems``.)
    """
    if name == "c1":
        x, q = uniform_alternating(4096, (24.0, 24.0, 24.0), SEED_BASE + 1)
        return Workload("c1", x, q, (24.0,) * 3, (16,) * 3, 5, ("ik",),
                        notes="4096 +-1 charges uniform in a 24 A cube")
    if name == "c2":
        x, q = water_like(10667, 68.0, SEED_BASE + 2)
        return Workload("c2", x, q, (68.0,) * 3, (64,) * 3, 5, ("ik", "ad"),
                        notes="10,667 water-like molecules, 68 A cube")
    if name == "c3":
        x, q = water_like(682667, 272.0, SEED_BASE + 3)
        return Workload("c3", x, q, (272.0,) * 3, (256,) * 3, 7, ("ad",),
                        notes="682,667 water-like molecules, 272 A cube")
    if name == "c5":
        x, q = water_like(33333, 100.0, SEED_BASE + 5)
        return Workload("c5", x, q, (100.0,) * 3, (96,) * 3, 5, ("ik",),
                        notes="33,333 water-like molecules, 100 A cube")
    raise KeyError(name)


def _smooth_mesh_size(target: float, lo: int = 16, hi: int = 64) -> int:
    """Smallest 2^a 3^b 5^c >= target, clamped to [lo, hi]."""
    n = max(lo, int(math.ceil(target - 1e-9)))
    while True:
        m = n
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        if m == 1:
            return min(n, hi)
        n += 1


def batch_systems(n_sys: int = 256, seed: int = SEED_BASE + 4, density: float = 0.1,
                  n_lo: int = 500, n_hi: int = 20000):
    """Independent neutral +-1 systems with N log-uniform in [n_lo, n_hi].

    Edge L_s = (N_s / density)^(1/3); mesh = smallest 2^a3^b5^c >= L_s / 1 A,
    clamped to [16, 64]; order drawn uniformly from {3, 5, 7}; r_cut =
    min(10, L_s / 2).  Returns a list of Workload.
    """
    r = rng(seed)
    out = []
    for s in range(n_sys):
        n = int(round(math.exp(r.uniform(math.log(n_lo), math.log(n_hi))) / 2.0)) * 2
        edge = (n / density) ** (1.0 / 3.0)
        m = _smooth_mesh_size(edge / 1.0)
        order = int(r.choice([3, 5, 7]))
        x = r.random((n, 3)) * edge
        q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
        out.append(Workload(f"c4_{s}", x, q, (edge,) * 3, (m,) * 3, order, ("ik",),
                            r_cut=min(10.0, edge / 2.0)))
    return out
