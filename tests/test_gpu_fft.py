"""The hand-written Poisson solve (variant bit 3: FP32 plans, power-of-two
mesh edges 16..128 or cubic 48^3 / 96^3 / 256^3) vs the oracle's FP64 Poisson solve on the GPU's own mesh
charge, vs the cuFFT path of the same plan, and end to end vs the oracle.

Mesh-level bar: the field (ik) or potential (ad) within 2e-6 of its largest
magnitude -- FP32 radix-2 transforms of length <= 128 carry ~log2(M^3) ulp
of relative error, below 1e-6 -- and the energy/virial within 1e-5.  End to end
the FP32/FP32C bar of the other parity tests (1e-4) applies.
"""
import math

import numpy as np
import pytest

from oracle import OraclePPPM, influence_ad, influence_ik, poisson_ad, poisson_ik

pytestmark = pytest.mark.gpu

OWN_FFT = 8  # variant bit of the hand-written Poisson solve


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


def e_scale(E, q, g, C):
    """The rounding scale of the energy: the mesh sum, of which the self term
    C g / sqrt(pi) sum q^2 cancels all but a few percent."""
    return abs(E) + C * g / math.sqrt(math.pi) * float(np.sum(np.asarray(q, np.float64) ** 2))


def system(mesh, box, n, seed):
    r = np.random.default_rng(seed)
    x = r.uniform(-1.0, max(box) + 1.0, (n, 3)).astype(np.float32)
    q = r.normal(size=n).astype(np.float32)
    q -= q.mean()
    return x, q


MESHES = [
    ((16, 16, 16), (10.0, 10.0, 10.0)),
    ((32, 16, 64), (20.0, 11.0, 37.0)),
    ((64, 64, 64), (40.0, 40.0, 40.0)),
    ((128, 32, 16), (70.0, 19.0, 9.0)),
    ((16, 128, 128), (9.0, 66.0, 70.0)),
    ((48, 48, 48), (30.0, 30.0, 30.0)),   # mixed radix: 12 points per lane
    ((96, 96, 96), (60.0, 60.0, 60.0)),   # mixed radix: 24 points per lane
    ((256, 256, 256), (160.0, 160.0, 160.0)),  # plane passes on clusters of four CTAs
]


@pytest.mark.parametrize("mesh,box", MESHES)
@pytest.mark.parametrize("mode", ["ik", "ad"])
def test_mesh_field_vs_oracle_poisson(torch, mesh, box, mode):
    """Field/potential on the mesh from the GPU's own rho, through both
    Poisson paths, vs the oracle's numpy FFT solve in FP64."""
    from paper_1702_04250_gb300 import pppm

    P, g, n = 5, 0.9, 3000
    x, q = system(mesh, box, n, 11 + mesh[0] + mesh[2])
    plan = pppm.PPPM(box, n, P, mesh, g, mode, "fp32c", 1.0)
    xt = torch.tensor(x, device="cuda")
    qt = torch.tensor(q, device="cuda")
    out = {}
    for v in (0, OWN_FFT):
        plan.set_variant(v)
        f, ev = plan.compute(xt, qt)
        plan.sync()
        rho = plan.get_array("rho").astype(np.float64)
        out[v] = (plan.get_array("field"), ev.cpu().numpy().copy(), f.double().cpu().numpy(), rho)
    # each run's own mesh charge (FP32C make_rho adds its cross-tile halos in
    # a run-dependent order, so two runs may differ in the last bit)
    if mode == "ik":
        G = influence_ik(box, mesh, P, g)
        for v in (0, OWN_FFT):
            _, fields = poisson_ik(out[v][3], G, box)
            E = out[v][0]
            for a in range(3):
                ref = fields[a]
                err = np.abs(E[..., a] - ref).max() / np.abs(ref).max()
                assert err < 2e-6, (v, a, err)
    else:
        G = influence_ad(box, mesh, P, g)
        for v in (0, OWN_FFT):
            _, phi = poisson_ad(out[v][3], G)
            err = np.abs(out[v][0] - phi).max() / np.abs(phi).max()
            assert err < 2e-6, (v, err)
    ev0, ev1 = out[0][1], out[OWN_FFT][1]
    assert abs(ev1[0] - ev0[0]) <= 1e-5 * e_scale(ev0[0], q, g, 1.0)
    assert np.linalg.norm(ev1[1:7] - ev0[1:7]) <= 1e-5 * np.linalg.norm(ev0[1:7])
    assert rel_rms(out[OWN_FFT][2], out[0][2]) < 1e-5


@pytest.mark.parametrize("mode", ["ik", "ad"])
@pytest.mark.parametrize("prec", ["fp32", "fp32c"])
def test_end_to_end_vs_oracle(torch, mode, prec):
    from paper_1702_04250_gb300 import pppm

    mesh, box = (32, 16, 64), (20.0, 11.0, 37.0)
    P, g, n = 5, 0.9, 4000
    x, q = system(mesh, box, n, 5)
    plan = pppm.PPPM(box, n, P, mesh, g, mode, prec, 2.5)
    plan.set_variant(OWN_FFT)
    f, ev = plan.compute(torch.tensor(x, device="cuda"), torch.tensor(q, device="cuda"))
    plan.sync()
    ref = OraclePPPM(box, mesh, P, g, mode, 2.5).compute(x.astype(np.float64), q.astype(np.float64))
    ev = ev.cpu().numpy()
    assert rel_rms(f.double().cpu().numpy(), ref["f"]) < 1e-4
    assert abs(ev[0] - ref["energy"]) < 1e-4 * e_scale(ref["energy"], q, g, 2.5)
    assert np.linalg.norm(ev[1:7] - ref["virial"]) < 1e-4 * np.linalg.norm(ref["virial"])


@pytest.mark.parametrize("mode", ["ik", "ad"])
def test_energy_grad_and_potential(torch, mode):
    """The scalar-potential solve (one inverse transform) behind dE/dx, dE/dq
    and the per-atom potential, hand-written vs cuFFT."""
    from paper_1702_04250_gb300 import pppm

    mesh, box = (16, 32, 32), (10.0, 19.0, 21.0)
    P, g, n = 4, 0.9, 2000
    x, q = system(mesh, box, n, 9)
    xt, qt = torch.tensor(x, device="cuda"), torch.tensor(q, device="cuda")
    plan = pppm.PPPM(box, n, P, mesh, g, mode, "fp32c", 1.7)
    res = {}
    for v in (0, OWN_FFT):
        plan.set_variant(v)
        dx, dq, ev = plan.energy_grad(xt, qt)
        phi = plan.potential(xt, qt)
        plan.sync()
        res[v] = (dx.double().cpu().numpy(), dq.double().cpu().numpy(), ev.cpu().numpy().copy(),
                  phi.double().cpu().numpy())
    a, b = res[0], res[OWN_FFT]
    assert rel_rms(b[0], a[0]) < 1e-5
    assert rel_rms(b[1], a[1]) < 1e-5
    assert abs(b[2][0] - a[2][0]) < 1e-5 * e_scale(a[2][0], q, g, 1.7)
    assert rel_rms(b[3], a[3]) < 1e-5
    o = OraclePPPM(box, mesh, P, g, mode, 1.7)
    rdx, rdq = o.energy_gradients(x.astype(np.float64), q.astype(np.float64))
    assert rel_rms(b[0], rdx) < 1e-4
    assert rel_rms(b[1], rdq) < 1e-4


def test_repeated_steps_graph_and_profiling(torch):
    """The energy follows the charges on every call (no stale partials or
    sums), eagerly, inside a graph and with stage events."""
    from paper_1702_04250_gb300 import pppm

    mesh, box = (64, 64, 64), (40.0, 40.0, 40.0)
    x, q = system(mesh, box, 5000, 21)
    xt, qt = torch.tensor(x, device="cuda"), torch.tensor(q, device="cuda")
    for graph in (False, True):
        plan = pppm.PPPM(box, 5000, 5, mesh, 0.9, "ik", "fp32c", 1.0, graph=graph)
        plan.set_variant(OWN_FFT | 1)
        energies = []
        for s in (1.0, 2.0, 3.0, 1.0):
            _, ev = plan.compute(xt, qt * s)
            plan.sync()
            energies.append(ev[0].item())
        e1 = energies[0]
        sc = e_scale(e1, q, 0.9, 1.0)
        assert abs(energies[1] - 4 * e1) < 4e-5 * sc
        assert abs(energies[2] - 9 * e1) < 9e-5 * sc
        assert abs(energies[3] - e1) < 1e-6 * sc
        plan.set_profiling(True)
        _, ev = plan.compute(xt, qt)
        plan.sync()
        assert abs(ev[0].item() - e1) < 1e-6 * sc
        t = plan.stage_times()
        assert all(v >= 0.0 for v in t.values()) and t["green"] > 0.0
        plan.close()


def test_variant_bit_refused_where_unsupported(torch):
    from paper_1702_04250_gb300 import pppm

    box = (20.0, 20.0, 20.0)
    for mesh, prec in (((24, 32, 32), "fp32c"), ((32, 32, 256), "fp32"), ((32, 32, 32), "fp64"),
                       ((96, 96, 48), "fp32c")):
        plan = pppm.PPPM(box, 10, 5, mesh, 0.9, "ik", prec, 1.0)
        with pytest.raises(pppm.PPPMError):
            plan.set_variant(OWN_FFT)
        plan.close()
