"""Mesh choice through the C ABI (the error estimate runs as an FP64 kernel)
vs the oracle: the estimate to 1e-6 (see the cancellation note below), the
chosen mesh exactly, g to the last bits, and the accuracy the chosen mesh
actually delivers on the GPU against the direct Ewald sum."""
import math

import numpy as np
import pytest

from oracle import ewald_kspace
from oracle.mesh_choice import choose_mesh, kspace_error_ad, kspace_error_ik

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pppm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_04250_gb300 import build

    build.build()
    from paper_1702_04250_gb300 import pppm as p

    return p


@pytest.mark.parametrize("box,mesh,P,g", [
    ((10.0, 10.0, 10.0), (8, 8, 8), 3, 0.35),
    ((12.0, 13.2, 10.8), (10, 12, 14), 4, 0.4),
    ((20.0, 20.0, 20.0), (32, 32, 32), 7, 0.7),
    ((30.0, 15.0, 22.0), (27, 16, 25), 5, 0.5),
])
def test_kspace_error_vs_oracle(pppm, box, mesh, P, g):
    n, q2 = 1234, 987.5
    gpu = pppm.kspace_error(box, mesh, P, g, n, q2)
    ref = kspace_error_ik(box, mesh, P, g, n, q2)
    # the functional is the difference of two alias sums that cancel to ~1e-5
    # of each other on accurate meshes: FP64 rounding of those sums (the
    # device's exact cosine series for sum U^2 against the oracle's 4001-term
    # sum) moves the difference by up to ~1e-6 of itself
    assert gpu == pytest.approx(ref, rel=1e-6)


def ad_tolerance(kappa):
    """Relative tolerance of an ad estimate: its three terms cancel by a factor
    kappa (the oracle's conditioning, 1e2 to 1e11 on these meshes), which
    amplifies FP64 rounding of the alias sums (2^-53 each, the device's exact
    cosine series against the oracle's 4001-term sums); the error is the
    square root of the functional, halving the relative spread; 8 for the
    sums' accumulated roundings."""
    return max(1e-6, 8 * 2.0 ** -53 * kappa / 2)


@pytest.mark.parametrize("box,mesh,P,g", [
    ((10.0, 10.0, 10.0), (8, 8, 8), 3, 0.35),
    ((12.0, 13.2, 10.8), (10, 12, 14), 4, 0.4),
    ((20.0, 20.0, 20.0), (32, 32, 32), 7, 0.7),
    ((30.0, 15.0, 22.0), (27, 16, 25), 5, 0.5),
    ((10.0, 10.0, 10.0), (10, 10, 10), 2, 0.3),
])
def test_ad_kspace_error_vs_oracle(pppm, box, mesh, P, g):
    """The ad functional: G^2 S0 S2 - 2 G T + sum |R|^2 per k, at the plan's
    ad influence function, within the tolerance its conditioning allows."""
    n, q2 = 1234, 987.5
    gpu = pppm.kspace_error(box, mesh, P, g, n, q2, mode="ad")
    ref, kappa = kspace_error_ad(box, mesh, P, g, n, q2, conditioning=True)
    assert gpu == pytest.approx(ref, rel=ad_tolerance(kappa))
    assert gpu > pppm.kspace_error(box, mesh, P, g, n, q2)  # ad is the less accurate form


@pytest.mark.parametrize("box,n,P,r_cut,acc,kind", [
    ((24.0, 24.0, 24.0), 4096, 5, 10.0, 1e-4, 1),   # the 4096-charge cube
    ((18.0, 21.0, 16.0), 2000, 5, 6.0, 1e-3, 0),
    ((18.0, 21.0, 16.0), 2000, 3, 6.0, 1e-3, 2),
    ((30.0, 30.0, 30.0), 9000, 7, 8.0, 1e-4, 1),
])
def test_choose_mesh_vs_oracle(pppm, box, n, P, r_cut, acc, kind):
    q2 = float(n)
    mesh, g, err = pppm.choose_mesh(box, n, q2, P, r_cut, acc, kind)
    rmesh, rg, rerr = choose_mesh(box, n, q2, P, r_cut, acc, kind)
    assert mesh == rmesh
    assert g == pytest.approx(rg, rel=1e-15)
    assert err == pytest.approx(rerr, rel=1e-6) and err <= acc


@pytest.mark.parametrize("box,n,P,r_cut,acc,kind", [
    ((18.0, 21.0, 16.0), 2000, 5, 6.0, 1e-3, 1),
    ((30.0, 30.0, 30.0), 9000, 7, 8.0, 1e-4, 2),
])
def test_choose_mesh_ad_vs_oracle(pppm, box, n, P, r_cut, acc, kind):
    q2 = float(n)
    mesh, g, err = pppm.choose_mesh(box, n, q2, P, r_cut, acc, kind, mode="ad")
    rmesh, rg, rerr = choose_mesh(box, n, q2, P, r_cut, acc, kind, mode="ad")
    assert mesh == rmesh
    _, kappa = kspace_error_ad(box, rmesh, P, rg, n, q2, conditioning=True)
    assert err == pytest.approx(rerr, rel=ad_tolerance(kappa)) and err <= acc
    ik_mesh, _, _ = pppm.choose_mesh(box, n, q2, P, r_cut, acc, kind)
    assert np.prod(mesh) >= np.prod(ik_mesh)  # ad needs at least the ik mesh


def test_chosen_mesh_delivers_the_accuracy(pppm):
    """600 random +-1 charges, target 1e-3: the FP64 GPU forces on the chosen
    mesh are within 1.5x the target of the direct Ewald reciprocal forces."""
    import torch

    r = np.random.default_rng(11)
    box, n, P, r_cut, acc = (14.0, 16.0, 12.0), 600, 5, 5.0, 1e-3
    x = r.uniform(0.0, 1.0, (n, 3)) * np.asarray(box)
    q = r.choice([-1.0, 1.0], n)
    mesh, g, err = pppm.choose_mesh(box, n, float(np.sum(q * q)), P, r_cut, acc)
    plan = pppm.PPPM(box, n, P, mesh, g, "ik", "fp64", 1.0)
    f, _ = plan.compute(torch.tensor(x, device="cuda"), torch.tensor(q, device="cuda"))
    plan.sync()
    fe = ewald_kspace(x, q, box, g, 1.0)[1]
    meas = math.sqrt(float(np.mean(np.sum((f.cpu().numpy() - fe) ** 2, axis=1))))
    assert meas <= 1.5 * acc, (mesh, err, meas)
    plan.close()
    # ad: the mesh chosen for ad delivers the target with ad forces (FP32C)
    mesh, g, err = pppm.choose_mesh(box, n, float(np.sum(q * q)), P, r_cut, acc, mode="ad")
    plan = pppm.PPPM(box, n, P, mesh, g, "ad", "fp32c", 1.0)
    f, _ = plan.compute(torch.tensor(x, dtype=torch.float32, device="cuda"),
                        torch.tensor(q, dtype=torch.float32, device="cuda"))
    plan.sync()
    fe = ewald_kspace(x, q, box, g, 1.0)[1]
    meas = math.sqrt(float(np.mean(np.sum((f.double().cpu().numpy() - fe) ** 2, axis=1))))
    assert meas <= 1.5 * acc, (mesh, err, meas)
    plan.close()


def test_bad_arguments_are_refused(pppm):
    with pytest.raises(pppm.PPPMError):
        pppm.kspace_error((10.0,) * 3, (16,) * 3, 5, 0.5, 100, 100.0, mode="xy")
    with pytest.raises(pppm.PPPMError):
        pppm.kspace_error((10.0,) * 3, (4, 16, 16), 5, 0.5, 100, 100.0)  # edge below the order
    with pytest.raises(pppm.PPPMError):
        pppm.choose_mesh((10.0,) * 3, 100, 100.0, 5, 4.0, 10.0)  # no g meets it
