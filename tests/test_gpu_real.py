"""Real-space part of the Ewald split on the GPU (cell list, erfc pairs)
against the oracle's brute-force minimum-image sum, and the total Coulomb
interaction (PPPM k-space + real space) against direct Ewald and the NaCl
Madelung constant."""
import math
import os

import numpy as np
import pytest

from oracle import OraclePPPM, ewald_kspace, ewald_real
from paper_1702_04250_gb300.workloads import rock_salt, uniform_alternating

pytestmark = pytest.mark.gpu

GOLDEN_M = float([l for l in open(os.path.join(os.path.dirname(__file__), "golden", "madelung_nacl.txt"))
                  if not l.startswith("#")][0])


@pytest.fixture(scope="module")
def torch():
    import torch as t

    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_04250_gb300 import build

    build.build()
    return t


def rel_rms(a, b):
    return math.sqrt(float(np.sum((a - b) ** 2)) / max(float(np.sum(b ** 2)), 1e-300))


def real_gpu(torch, box, x, q, r_cut, g, prec, C=1.0):
    from paper_1702_04250_gb300 import pppm

    dt = torch.float64 if prec == "fp64" else torch.float32
    rs = pppm.RealSpace(box, len(q), r_cut, g, precision=prec, qqrd2e=C)
    f, ev = rs.compute(torch.tensor(x, dtype=dt, device="cuda"), torch.tensor(q, dtype=dt, device="cuda"))
    rs.sync()
    return rs, f.double().cpu().numpy(), ev.cpu().numpy().copy()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_real_space_vs_brute_force(torch, prec, tol):
    """4096 +-1 charges in a 24 A cube, r_C = 4.8 A: cells of 2.4 A, 10 per
    edge, the 5^3 neighbourhood of every cell.  FP32 at the 1e-4 bar of the
    k-space path: uniform random charges include pairs ~0.1 A apart, where a
    float position's ~1e-6 A resolution is a 1e-5 relative distance error
    that 1/r^2 forces amplify (measured 4.8e-5 relative RMS)."""
    x, q = uniform_alternating(4096, (24.0, 24.0, 24.0), 11)
    box, rc, g, C = (24.0, 24.0, 24.0), 4.8, 0.6, 2.0
    rs, f, ev = real_gpu(torch, box, x, q, rc, g, prec, C)
    assert rs.info()["cells"] == (10, 10, 10)
    if prec == "fp32":
        x = x.astype(np.float32).astype(np.float64)
        q = q.astype(np.float32).astype(np.float64)
    E, F, W = ewald_real(x, q, box, g, rc, C)
    assert rel_rms(f, F) < tol
    assert abs(ev[0] - E) < tol * abs(E)
    assert np.linalg.norm(ev[1:] - W) < tol * np.linalg.norm(W)


def test_real_space_single_cell_dimensions(torch):
    """Edges of 12 and 13 A with r_C = 5.5 A have fewer than 5 cells: those
    dimensions become one cell (minimum image per pair); a non-neutral set,
    positions outside the box."""
    r = np.random.default_rng(5)
    box, rc, g = (12.0, 13.0, 30.0), 5.5, 0.6
    x = r.uniform(-3.0, 33.0, (700, 3))
    q = r.normal(size=700)
    rs, f, ev = real_gpu(torch, box, x, q, rc, g, "fp64")
    assert rs.info()["cells"] == (1, 1, 10)
    E, F, W = ewald_real(x, q, box, g, rc, 1.0)
    assert rel_rms(f, F) < 1e-10
    assert abs(ev[0] - E) < 1e-10 * abs(E)
    assert np.linalg.norm(ev[1:] - W) < 1e-10 * np.linalg.norm(W)


def test_total_coulomb_vs_direct_ewald(torch):
    """k-space (PPPM) forces accumulated with the real-space forces equal the
    direct Ewald sum within the PPPM discretisation error."""
    from paper_1702_04250_gb300 import pppm

    x, q = uniform_alternating(4096, (24.0, 24.0, 24.0), 11)
    box, rc, g, C = (24.0, 24.0, 24.0), 10.0, 0.2854, 1.0
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    qt = torch.tensor(q, dtype=torch.float64, device="cuda")
    plan = pppm.PPPM(box, len(q), 5, (32, 32, 32), g, mode="ik", precision="fp64", qqrd2e=C)
    f, evk = plan.compute(xt, qt)
    rs = pppm.RealSpace(box, len(q), rc, g, precision="fp64", qqrd2e=C)
    f, evr = rs.compute(xt, qt, f=f, accumulate=True)
    rs.sync()
    plan.sync()
    Ek, Fk, Wk = ewald_kspace(x, q, box, g, C)
    Er, Fr, Wr = ewald_real(x, q, box, g, rc, C)
    self_e = -C * g / math.sqrt(math.pi) * float(np.sum(q * q))
    Etot = Ek + Er + self_e
    ftot = f.cpu().numpy()
    err = rel_rms(ftot, Fk + Fr)
    print("total Coulomb force vs direct Ewald, rel RMS", err)
    assert err < 1e-3
    e_gpu = evk[0].item() + evr[0].item()
    assert abs(e_gpu - Etot) < 1e-4 * abs(Etot)
    # the real-space share alone is exact
    _, fr_only, evr_only = real_gpu(torch, box, x, q, rc, g, "fp64", C)
    assert rel_rms(fr_only, Fr) < 1e-10


@pytest.mark.parametrize("mode", ["ik", "ad"])
def test_nacl_madelung_on_gpu(torch, mode):
    """8^3 rock-salt ions, spacing 2 A: the GPU's k-space + real-space energy
    gives the Madelung constant, and the forces vanish on the lattice."""
    from paper_1702_04250_gb300 import pppm

    x, q = rock_salt(8, 2.0)  # ions on mesh points (spacing 0.5 A): no stencil ties
    L, a, g, rc, C = 16.0, 2.0, 0.5, 7.9, 1.0
    box = (L, L, L)
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    qt = torch.tensor(q, dtype=torch.float64, device="cuda")
    plan = pppm.PPPM(box, len(q), 7, (32, 32, 32), g, mode=mode, precision="fp64", qqrd2e=C)
    f, evk = plan.compute(xt, qt)
    rs = pppm.RealSpace(box, len(q), rc, g, precision="fp64", qqrd2e=C)
    f, evr = rs.compute(xt, qt, f=f, accumulate=True)
    rs.sync()
    plan.sync()
    E = evk[0].item() + evr[0].item()
    M = -E * 2 * a / (C * len(q))
    print(mode, "Madelung from GPU k-space + real space", M)
    assert abs(M - GOLDEN_M) < 1e-5 * GOLDEN_M
    # every ion is an inversion centre: zero net force (scale C / a^2 = 0.25)
    assert np.abs(f.cpu().numpy()).max() < 1e-5


def test_real_space_rejects_cutoff_beyond_half_box(torch):
    from paper_1702_04250_gb300 import pppm

    with pytest.raises(pppm.PPPMError):
        pppm.RealSpace((10.0, 10.0, 10.0), 10, 5.0, 0.5, precision="fp64")
