"""The seeded synthetic inputs against the recipe they implement (CPU only):
rigid water-like molecules with the SPC/E charges, 1.0 A O-H bonds and a
109.47 degree angle on a jittered cubic lattice with random orientations;
the uniform +-1 charges of c1; the 256-system batch; the rock-salt lattice;
the sizes, boxes, meshes and orders of the named workloads; determinism."""
import math

import numpy as np
import pytest

from paper_1702_04250_gb300 import workloads as wl


def _min_image(d, L):
    return d - L * np.round(d / L)


@pytest.fixture(scope="module")
def c2():
    return wl.config("c2")


def test_water_geometry_and_charges(c2):
    L = c2.box[0]
    x = c2.x.reshape(-1, 3, 3)
    assert x.shape[0] == 10_667 and c2.n == 32_001
    oh1 = _min_image(x[:, 1] - x[:, 0], L)
    oh2 = _min_image(x[:, 2] - x[:, 0], L)
    r1, r2 = np.linalg.norm(oh1, axis=1), np.linalg.norm(oh2, axis=1)
    np.testing.assert_allclose(r1, 1.0, atol=1e-12)
    np.testing.assert_allclose(r2, 1.0, atol=1e-12)
    ang = np.degrees(np.arccos(np.sum(oh1 * oh2, axis=1) / (r1 * r2)))
    np.testing.assert_allclose(ang, 109.47, atol=1e-9)
    q = c2.q.reshape(-1, 3)
    assert np.all(q[:, 0] == -0.8476) and np.all(q[:, 1:] == 0.4238)
    assert abs(float(np.sum(c2.q))) < 1e-9
    assert np.all((c2.x >= 0.0) & (c2.x < L))
    # the c2 recipe's density: 0.1018 charges per cubic angstrom
    assert c2.n / L ** 3 == pytest.approx(0.1018, abs=5e-5)


def test_water_oxygens_on_a_jittered_lattice(c2):
    n_mol, L = 10_667, c2.box[0]
    side = 23  # ceil(10,667^(1/3))
    spacing = L / side
    o = c2.x.reshape(-1, 3, 3)[:, 0]
    frac = o / spacing
    cell = np.floor(frac).astype(int)
    inner = frac - cell
    # each oxygen stays within +-0.25 spacing of its site centre, so inside its own cell
    assert np.all((inner >= 0.25 - 1e-9) & (inner <= 0.75 + 1e-9))
    keys = (cell[:, 0] * side + cell[:, 1]) * side + cell[:, 2]
    assert len(np.unique(keys)) == n_mol


def test_water_orientations_are_isotropic(c2):
    """Uniform random rotations: the bisector (dipole) direction has mean ~0
    and <cos^2> = 1/3 along each axis, within sampling error."""
    L = c2.box[0]
    x = c2.x.reshape(-1, 3, 3)
    bis = _min_image(x[:, 1] - x[:, 0], L) + _min_image(x[:, 2] - x[:, 0], L)
    u = bis / np.linalg.norm(bis, axis=1)[:, None]
    n = u.shape[0]
    assert np.all(np.abs(u.mean(axis=0)) < 4.0 / math.sqrt(n))
    np.testing.assert_allclose((u ** 2).mean(axis=0), 1.0 / 3.0, atol=4.0 * math.sqrt(4.0 / 45.0 / n))


def test_named_workloads():
    c1 = wl.config("c1")
    assert (c1.n, c1.box, c1.mesh, c1.order, c1.modes) == (4096, (24.0,) * 3, (16,) * 3, 5, ("ik",))
    assert np.all((c1.x >= 0) & (c1.x < 24.0))
    assert np.array_equal(c1.q, np.where(np.arange(4096) % 2 == 0, 1.0, -1.0))
    c5 = wl.config("c5")
    assert (c5.n, c5.box, c5.mesh, c5.order) == (99_999, (100.0,) * 3, (96,) * 3, 5)
    c3 = wl.config("c3")
    assert (c3.n, c3.box, c3.mesh, c3.order, c3.modes) == (2_048_001, (272.0,) * 3, (256,) * 3, 7, ("ad",))
    assert abs(float(np.sum(c3.q))) < 1e-6
    with pytest.raises(KeyError):
        wl.config("c9")


def test_generators_are_deterministic_per_seed():
    a = wl.water_like(50, 12.0, 7)
    b = wl.water_like(50, 12.0, 7)
    c = wl.water_like(50, 12.0, 8)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0])
    u1, u2 = wl.uniform_alternating(100, (5.0, 6.0, 7.0), 3), wl.uniform_alternating(100, (5.0, 6.0, 7.0), 3)
    assert np.array_equal(u1[0], u2[0])
    assert np.all(u1[0] < np.array([5.0, 6.0, 7.0])) and np.all(u1[0] >= 0)


def test_batch_systems_recipe():
    sys_ = wl.batch_systems()
    assert len(sys_) == 256
    ns = np.array([s.n for s in sys_])
    assert np.all(ns % 2 == 0) and ns.min() >= 500 and ns.max() <= 20_000
    # log-uniform sizes: the median sits near the geometric mean of the range
    assert 0.5 < np.median(ns) / math.sqrt(500 * 20_000) < 2.0
    assert {s.order for s in sys_} == {3, 5, 7}
    for s in sys_:
        L = s.box[0]
        assert L == pytest.approx((s.n / 0.1) ** (1.0 / 3.0), rel=1e-12)
        m = s.mesh[0]
        assert s.mesh == (m, m, m) and 16 <= m <= 64
        r = m
        for p in (2, 3, 5):
            while r % p == 0:
                r //= p
        assert r == 1
        assert m >= min(64, math.ceil(L - 1e-9))  # at least one point per angstrom unless clamped
        assert float(np.sum(s.q)) == 0.0
        assert np.all((s.x >= 0) & (s.x < L))
        assert s.r_cut == pytest.approx(min(10.0, L / 2.0))


def test_rock_salt_lattice():
    x, q = wl.rock_salt(4, 2.5)
    assert x.shape == (64, 3) and float(np.sum(q)) == 0.0
    # every nearest neighbour (distance a) has the opposite charge
    d = np.linalg.norm(_min_image(x[:, None, :] - x[None, :, :], 10.0), axis=2)
    nn = np.isclose(d, 2.5)
    assert np.all(nn.sum(axis=1) == 6)
    assert np.all((q[:, None] * q[None, :])[nn] == -1.0)
