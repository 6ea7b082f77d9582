"""Pins of the oracle's mesh choice (FFT-friendly sizes, the k-space error
estimate of an ik mesh, the scan for a target accuracy) against what the
mathematics fixes: factorisations by brute force, and the estimate against
the measured RMS error of the oracle PPPM against the direct Ewald sum on
random charges (the estimate is the expectation of that error), plus the C
ABI's host-only size rule against the oracle's."""
import math

import numpy as np
import pytest

from oracle import OraclePPPM, ewald_kspace
from oracle.mesh_choice import choose_mesh, fft_size, kspace_error, kspace_error_ad, kspace_error_ik


def _factors_ok(m, primes):
    for p in primes:
        while m % p == 0:
            m //= p
    return m == 1


@pytest.mark.parametrize("kind,primes", [(1, (2, 3, 5, 7)), (2, (2,))])
def test_fft_size_is_the_smallest_friendly_size(kind, primes):
    for n in range(1, 700):
        m = fft_size(n, kind)
        assert m >= n and _factors_ok(m, primes)
        assert all(not _factors_ok(j, primes) for j in range(n, m))
    assert [fft_size(n, 1) for n in (61, 67, 97, 121, 127)] == [63, 70, 98, 125, 128]
    assert fft_size(65, 2) == 128 and fft_size(64, 2) == 64 and fft_size(37, 0) == 37


def _measured_error(box, mesh, P, g, n, seed, mode="ik"):
    r = np.random.default_rng(seed)
    x = r.uniform(0.0, 1.0, (n, 3)) * np.asarray(box)
    q = r.choice([-1.0, 1.0], n)
    f = OraclePPPM(box, mesh, P, g, mode, 1.0).compute(x, q)["f"]
    fe = ewald_kspace(x, q, box, g, 1.0)[1]
    return math.sqrt(float(np.mean(np.sum((f - fe) ** 2, axis=1)))), float(np.sum(q * q))


@pytest.mark.parametrize("box,mesh,P,g", [
    ((10.0, 10.0, 10.0), (8, 8, 8), 3, 0.35),
    ((10.0, 10.0, 10.0), (12, 12, 12), 5, 0.45),
    ((12.0, 13.2, 10.8), (10, 12, 14), 4, 0.4),
    ((10.0, 10.0, 10.0), (16, 16, 16), 7, 0.8),
])
def test_error_estimate_matches_measured_error(box, mesh, P, g):
    """400 random +-1 charges: the estimate is within 20 % of the RMS force
    error the oracle PPPM actually makes against the direct Ewald sum (errors
    from 5e-5 to 3e-3 across these cases; a dropped alias term, a wrong power
    of the denominator or of V moves the ratio by far more)."""
    n = 400
    meas, q2 = _measured_error(box, mesh, P, g, n, seed=3)
    est = kspace_error_ik(box, mesh, P, g, n, q2)
    assert 0.8 < est / meas < 1.25, (est, meas)


@pytest.mark.parametrize("box,mesh,P,g,lo,hi", [
    ((10.0, 10.0, 10.0), (8, 8, 8), 3, 0.35, 0.8, 1.25),
    ((10.0, 10.0, 10.0), (12, 12, 12), 5, 0.45, 0.8, 1.25),
    ((12.0, 13.2, 10.8), (10, 12, 14), 4, 0.4, 0.8, 1.25),
    ((10.0, 10.0, 10.0), (16, 16, 16), 7, 0.8, 0.8, 1.25),
    ((10.0, 10.0, 10.0), (10, 10, 10), 2, 0.3, 0.8, 1.4),
])
def test_ad_error_estimate_matches_measured_error(box, mesh, P, g, lo, hi):
    """The ad estimate (the same functional with each alias carrying its own
    derivative, at the plan's ad influence function) against the RMS force
    error the oracle's ad PPPM (self force removed) makes against the direct
    Ewald sum on 400 random charges; measured ratios 0.90-1.19, and 1.29 at
    P = 2, where the two-harmonic self-force correction leaves the most
    behind."""
    n = 400
    meas, q2 = _measured_error(box, mesh, P, g, n, seed=3, mode="ad")
    est = kspace_error_ad(box, mesh, P, g, n, q2)
    assert lo < est / meas < hi, (est, meas)
    # ad differentiation is the less accurate one at a fixed mesh
    assert est > kspace_error_ik(box, mesh, P, g, n, q2)


def test_ad_estimate_planted_slips_are_caught():
    """Plausible slips in the ad functional move the estimate away from the
    measured error by more than the tolerance above: dropping the aliases'
    own derivatives (using k^2 instead of k_m^2, i.e. the ik cross term with G
    in place of the optimum) or dropping the G^2 term."""
    box, mesh, P, g = (10.0, 10.0, 10.0), (12, 12, 12), 5, 0.45
    meas, q2 = _measured_error(box, mesh, P, g, 400, seed=3, mode="ad")
    good = kspace_error_ad(box, mesh, P, g, 400, q2)
    assert 0.8 < good / meas < 1.25
    import oracle.mesh_choice as mc

    orig = mc._alias_sums_1d

    def no_alias_derivative(k, h, P, mmax=mc.ALIAS_FULL):
        s0, _ = orig(k, h, P, mmax)
        return s0, s0 * np.asarray(k) ** 2  # k^2 for every alias
    mc._alias_sums_1d = no_alias_derivative
    try:
        slipped = mc.kspace_error_ad(box, mesh, P, g, 400, q2)
    finally:
        mc._alias_sums_1d = orig
    assert not (0.8 < slipped / meas < 1.25), slipped / meas


def test_error_estimate_falls_with_the_mesh_and_the_order():
    box, g, n, q2 = (20.0, 20.0, 20.0), 0.3, 1000, 1000.0
    errs = [kspace_error_ik(box, (m, m, m), 5, g, n, q2) for m in (12, 16, 20, 24)]
    assert all(a > b for a, b in zip(errs, errs[1:]))
    by_order = [kspace_error_ik(box, (16, 16, 16), P, g, n, q2) for P in (3, 5, 7)]
    assert by_order[0] > by_order[1] > by_order[2]
    # dF scales as q2 / sqrt(n) at a fixed mesh
    assert kspace_error_ik(box, (16,) * 3, 5, g, 4 * n, 2 * q2) == pytest.approx(errs[1], rel=1e-12)
    ad = [kspace_error_ad(box, (m, m, m), 5, g, n, q2) for m in (12, 16, 20, 24)]
    assert all(a > b for a, b in zip(ad, ad[1:]))
    ad_by_order = [kspace_error_ad(box, (16, 16, 16), P, g, n, q2) for P in (3, 5, 7)]
    assert ad_by_order[0] > ad_by_order[1] > ad_by_order[2]


@pytest.mark.parametrize("kind,mode", [(0, "ik"), (1, "ik"), (2, "ik"), (1, "ad"), (2, "ad")])
def test_choose_mesh_meets_the_target_with_the_first_mesh_that_does(kind, mode):
    box, n, q2, P, r_cut, acc = (18.0, 21.0, 16.0), 2000, 2000.0, 5, 6.0, 1e-3
    mesh, g, err = choose_mesh(box, n, q2, P, r_cut, acc, kind, mode=mode)
    assert err <= acc and err == pytest.approx(kspace_error(box, mesh, P, g, n, q2, mode), rel=1e-14)
    if kind:
        assert all(fft_size(m, kind) == m for m in mesh)
    # every distinct mesh the scan tried before it misses the target
    lmax = max(box)
    for c in range(P, 200):
        m2 = tuple(max(P, fft_size(int(math.ceil(L * c / lmax)), kind)) for L in box)
        if m2 == mesh:
            break
        assert kspace_error(box, m2, P, g, n, q2, mode) > acc


def test_abi_fft_size_matches_the_oracle():
    """The C ABI's size rule (host logic, no device work)."""
    from paper_1702_04250_gb300 import build, pppm

    build.build()
    for kind in (0, 1, 2):
        for n in range(1, 1100):
            assert pppm.fft_size(n, kind) == fft_size(n, kind), (n, kind)
    with pytest.raises(pppm.PPPMError):
        pppm.fft_size(0, 1)
    with pytest.raises(pppm.PPPMError):
        pppm.fft_size(10, 3)
