"""GPU path vs the FP64 oracle, through the C ABI.

Tolerances (relative RMS for forces, relative for energy, norm-relative for
the virial): FP64 1e-6, FP32 / FP32C 1e-4.  Integer outputs (stencil anchors,
the sort) are compared exactly; where several orders are valid (particles of
one tile) only validity is checked.  FP32 runs feed the oracle the same
float32-rounded inputs, so the comparison measures the arithmetic only.
"""
import math

import numpy as np
import pytest

from oracle import (OraclePPPM, estimate_g_ewald, influence_ad, influence_ik, make_rho, poisson_ad,
                    poisson_ik, stencil, wrap_positions)
from paper_1702_04250_gb300.workloads import batch_systems, config, uniform_alternating, water_like

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-6, "fp32c": 1e-4, "fp32": 1e-4}


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


def g_of(w):
    return estimate_g_ewald(w.rel_acc, w.r_cut, w.n, float(np.sum(w.q ** 2)), w.box)


def run(torch, box, mesh, order, g, mode, prec, x, q, C=1.0, **kw):
    from paper_1702_04250_gb300 import pppm

    dt = torch.float64 if prec == "fp64" else torch.float32
    plan = pppm.PPPM(box, max(len(q), 1), order, mesh, g, mode=mode, precision=prec, qqrd2e=C, **kw)
    xt = torch.tensor(np.asarray(x), dtype=dt, device="cuda")
    qt = torch.tensor(np.asarray(q), dtype=dt, device="cuda")
    f, ev = plan.compute(xt, qt)
    plan.sync()
    return plan, f.double().cpu().numpy(), ev.cpu().numpy().copy()


def oracle_inputs(x, q, prec):
    if prec == "fp64":
        return np.asarray(x, np.float64), np.asarray(q, np.float64)
    return np.asarray(x, np.float32).astype(np.float64), np.asarray(q, np.float32).astype(np.float64)


def check_all(f, ev, ref, prec, label=""):
    tol = TOL[prec]
    ferr = rel_rms(f, ref["f"])
    eerr = abs(ev[0] - ref["energy"]) / abs(ref["energy"])
    verr = np.linalg.norm(ev[1:7] - ref["virial"]) / np.linalg.norm(ref["virial"])
    print(f"{label} {prec}: force {ferr:.2e} energy {eerr:.2e} virial {verr:.2e}")
    assert ferr <= tol, ferr
    assert eerr <= tol, eerr
    assert verr <= tol, verr
    return ferr, eerr, verr


# ---------------------------------------------------------------------------
# stage by stage, FP64, c1 (16^3 mesh = 2x2x2 tiles)
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def c1_fp64_ik(torch):
    w = config("c1")
    g = g_of(w)
    plan, f, ev = run(torch, w.box, w.mesh, w.order, g, "ik", "fp64", w.x, w.q, w.qqrd2e)
    o = OraclePPPM(w.box, w.mesh, w.order, g, "ik", w.qqrd2e)
    ref = o.compute(w.x, w.q, keep=True)
    return w, g, plan, f, ev, o, ref


def test_anchor_and_sort(c1_fp64_ik):
    w, g, plan, *_ = c1_fp64_ik
    h = np.array(w.box) / np.array(w.mesh)
    u = wrap_positions(w.x, w.box) / h
    ref = np.stack([stencil(u[:, d], w.order, w.mesh[d])[0][:, (w.order - 1) // 2] for d in range(3)], axis=1)
    got = plan.get_array("anchor")
    np.testing.assert_array_equal(got, ref)
    perm = plan.get_array("perm")
    assert np.array_equal(np.sort(perm), np.arange(w.n))
    ts = plan.get_array("tilestart")
    assert ts[0] == 0 and ts[-1] == w.n and np.all(np.diff(ts) >= 0)
    inf = plan.info()
    T = [(m + inf["tile"] - 1) // inf["tile"] for m in w.mesh]
    tile = lambda a, d: ((a + 1) * T[d] - 1) // w.mesh[d]
    tid = (tile(ref[:, 0], 0) * T[1] + tile(ref[:, 1], 1)) * T[2] + tile(ref[:, 2], 2)
    sorted_tiles = tid[perm]
    owner = np.repeat(np.arange(len(ts) - 1), np.diff(ts))
    np.testing.assert_array_equal(sorted_tiles, owner)


@pytest.mark.parametrize("box,mesh,ntiles,n", [((40.0, 40.0, 42.0), (136, 136, 144), 5202, 60_001),
                                              ((78.0, 78.0, 80.0), (264, 264, 272), 37026, 150_001)])
def test_sort_many_tiles_ragged_scan(torch, box, mesh, ntiles, n):
    """More tiles than the per-block shared-memory scan holds: the one-CTA
    scan kernel.  5,202 tiles (17 x 17 x 18): 1,300 whole int4 groups over 21
    warps, two tail tiles; 37,026 tiles (33 x 33 x 34): segments of 320
    groups, more than the registers hold (a second load pass), one tail
    tile.  Exact anchors (FP64), a permutation, tile offsets equal to the
    exclusive scan of the brute-force tile counts, every particle in its tile."""
    P = 5
    x, q = uniform_alternating(n, box, seed=29)
    plan, *_ = run(torch, box, mesh, P, 0.6, "ik", "fp64", x, q)
    h = np.array(box) / np.array(mesh)
    u = wrap_positions(x, box) / h
    ref = np.stack([stencil(u[:, d], P, mesh[d])[0][:, (P - 1) // 2] for d in range(3)], axis=1)
    np.testing.assert_array_equal(plan.get_array("anchor"), ref)
    perm = plan.get_array("perm")
    assert np.array_equal(np.sort(perm), np.arange(len(q)))
    inf = plan.info()
    T = [(m + inf["tile"] - 1) // inf["tile"] for m in mesh]
    assert T[0] * T[1] * T[2] == ntiles
    tile = lambda a, d: ((a + 1) * T[d] - 1) // mesh[d]
    tid = (tile(ref[:, 0], 0) * T[1] + tile(ref[:, 1], 1)) * T[2] + tile(ref[:, 2], 2)
    counts = np.bincount(tid, minlength=T[0] * T[1] * T[2])
    ts = plan.get_array("tilestart")
    np.testing.assert_array_equal(ts, np.concatenate([[0], np.cumsum(counts)]))
    np.testing.assert_array_equal(tid[perm], np.repeat(np.arange(len(counts)), counts))
    plan.close()


def test_rho_green_field(c1_fp64_ik):
    w, g, plan, f, ev, o, ref = c1_fp64_ik
    rho = plan.get_array("rho")
    assert np.abs(rho - ref["rho"]).max() <= 1e-12 * np.abs(ref["rho"]).max()
    G = plan.get_array("green")
    assert np.abs(G - o.G).max() <= 1e-12 * np.abs(o.G).max()
    E = plan.get_array("field")
    for a in range(3):
        assert np.abs(E[..., a] - ref["fields"][a]).max() <= 1e-10 * np.abs(ref["fields"][a]).max()


def test_c1_fp64_ik_end_to_end(c1_fp64_ik):
    w, g, plan, f, ev, o, ref = c1_fp64_ik
    ferr, eerr, verr = check_all(f, ev, ref, "fp64", "c1 ik")
    assert ferr < 1e-10  # FP64 should agree to round-off


def test_c1_fp64_ad_stages(torch):
    w = config("c1")
    g = g_of(w)
    plan, f, ev = run(torch, w.box, w.mesh, w.order, g, "ad", "fp64", w.x, w.q, w.qqrd2e)
    o = OraclePPPM(w.box, w.mesh, w.order, g, "ad", w.qqrd2e)
    ref = o.compute(w.x, w.q, keep=True)
    G = plan.get_array("green")
    assert np.abs(G - o.G).max() <= 1e-12 * np.abs(o.G).max()
    sf = plan.get_array("selfforce")
    np.testing.assert_allclose(sf, o.sf, rtol=1e-9, atol=1e-12 * np.abs(o.sf).max())
    phi = plan.get_array("phi")
    assert np.abs(phi - ref["phi"]).max() <= 1e-10 * np.abs(ref["phi"]).max()
    ferr, *_ = check_all(f, ev, ref, "fp64", "c1 ad")
    assert ferr < 1e-10


# ---------------------------------------------------------------------------
# the water-like 64^3 system (512 tiles), both modes, all precisions
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def c2_refs():
    w = config("c2")
    g = g_of(w)
    refs = {}
    for mode in ("ik", "ad"):
        o = OraclePPPM(w.box, w.mesh, w.order, g, mode, w.qqrd2e)
        refs[(mode, "fp64")] = o.compute(w.x, w.q)
        x32, q32 = oracle_inputs(w.x, w.q, "fp32")
        refs[(mode, "fp32")] = o.compute(x32, q32)
    return w, g, refs


@pytest.mark.parametrize("mode", ["ik", "ad"])
@pytest.mark.parametrize("prec", ["fp64", "fp32c", "fp32"])
def test_c2_parity(torch, c2_refs, mode, prec):
    w, g, refs = c2_refs
    plan, f, ev = run(torch, w.box, w.mesh, w.order, g, mode, prec, w.x, w.q, w.qqrd2e)
    ref = refs[(mode, "fp64" if prec == "fp64" else "fp32")]
    check_all(f, ev, ref, prec, f"c2 {mode}")


def test_fp32c_is_not_worse_than_fp32(torch, c2_refs):
    w, g, refs = c2_refs
    ref = refs[("ik", "fp32")]
    errs = {}
    for prec in ("fp32", "fp32c"):
        plan, f, ev = run(torch, w.box, w.mesh, w.order, g, "ik", prec, w.x, w.q, w.qqrd2e)
        plan.compute(torch.tensor(w.x, dtype=torch.float32, device="cuda"),
                     torch.tensor(w.q, dtype=torch.float32, device="cuda"))
        rho = plan.get_array("rho").astype(np.float64)
        rref = make_rho(*oracle_inputs(w.x, w.q, "fp32"), w.box, w.mesh, w.order)
        errs[prec] = np.sqrt(np.mean((rho - rref) ** 2)) / np.sqrt(np.mean(rref ** 2))
    print("mesh rho rel RMS", errs)
    assert errs["fp32c"] <= errs["fp32"] * 1.05


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("P", [2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("mode", ["ik", "ad"])
@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_orders_on_ragged_mesh(torch, P, mode, prec):
    """Non-cubic box, mesh 20 x 17 x 12 (uneven tiles, odd Mz/2+1 handling),
    positions partly outside the box, a non-neutral charge set."""
    r = np.random.default_rng(100 + P)
    box = (13.0, 11.5, 9.0)
    mesh = (20, 17, 12)
    n = 700
    x = r.uniform(-5.0, 20.0, (n, 3))
    q = r.normal(size=n)
    g = 0.55
    plan, f, ev = run(torch, box, mesh, P, g, mode, prec, x, q, 2.0)  # default: 4^3 tiles (18 of 8^3)
    xo, qo = oracle_inputs(x, q, prec)
    ref = OraclePPPM(box, mesh, P, g, mode, 2.0).compute(xo, qo)
    check_all(f, ev, ref, prec, f"P={P} {mode}")
    plan.set_variant(32 if prec == "fp32c" else 0)  # 8^3 tiles (uneven: 7/7/6, 6/6/5, 6/6)
    dt = torch.float64 if prec == "fp64" else torch.float32
    f0, ev0 = plan.compute(torch.tensor(x, dtype=dt, device="cuda"), torch.tensor(q, dtype=dt, device="cuda"))
    plan.sync()
    check_all(f0.double().cpu().numpy(), ev0.cpu().numpy(), ref, prec, f"P={P} {mode} 8^3 tiles")
    if prec == "fp32c":
        # the persistent fieldforce on uneven tiles (element-wise brick copies,
        # every brick edge wrapping), 8^3 and 4^3 tiles
        for v in (96, 80):
            plan.set_variant(v)
            f0, ev0 = plan.compute(torch.tensor(x, dtype=dt, device="cuda"), torch.tensor(q, dtype=dt, device="cuda"))
            plan.sync()
            check_all(f0.double().cpu().numpy(), ev0.cpu().numpy(), ref, prec, f"P={P} {mode} variant {v}")


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_tiny_and_degenerate(torch, prec):
    box, mesh, P, g = (10.0, 10.0, 10.0), (8, 8, 8), 7, 0.6
    # mesh 8 with P=7: the stencil nearly wraps onto itself; single tile
    for n in (1, 2, 5):
        r = np.random.default_rng(n)
        x = r.uniform(0, 10, (n, 3))
        q = np.ones(n) if n == 1 else r.normal(size=n)
        for mode in ("ik", "ad"):
            plan, f, ev = run(torch, box, mesh, P, g, mode, prec, x, q)
            xo, qo = oracle_inputs(x, q, prec)
            ref = OraclePPPM(box, mesh, P, g, mode, 1.0).compute(xo, qo)
            tol = TOL[prec]
            # a lone charge in ik feels no force: compare absolutely
            scale = max(np.abs(ref["f"]).max(), 1e-3)
            assert np.abs(f - ref["f"]).max() <= tol * scale * 10
            assert abs(ev[0] - ref["energy"]) <= tol * abs(ref["energy"])


@pytest.mark.parametrize("prec,P", [("fp32c", 5), ("fp32c", 7), ("fp32", 5), ("fp64", 5)])
def test_dense_tile(torch, prec, P):
    """70,000 charges packed into one mesh tile: the FP32C fixed-point brick
    folds its low words twice (every 32,768 particles), and every precision
    must still match the oracle's mesh and forces."""
    r = np.random.default_rng(31)
    box, mesh, g = (20.0, 20.0, 20.0), (20, 20, 20), 0.5
    n = 70000
    x = 3.0 + r.uniform(0.0, 1.5, (n, 3))
    q = r.normal(size=n)
    plan, f, ev = run(torch, box, mesh, P, g, "ik", prec, x, q)
    xo, qo = oracle_inputs(x, q, prec)
    o = OraclePPPM(box, mesh, P, g, "ik", 1.0)
    ref = o.compute(xo, qo, keep=True)
    rho = plan.get_array("rho").astype(np.float64)
    rerr = np.sqrt(np.mean((rho - ref["rho"]) ** 2)) / np.sqrt(np.mean(ref["rho"] ** 2))
    print(prec, "dense tile rho rel RMS", rerr)
    assert rerr < (1e-12 if prec == "fp64" else 1e-5)
    check_all(f, ev, ref, prec, "dense tile")
    if prec != "fp64":
        # the persistent fieldforce: 70,000 charges in one tile is 274 sub-chunks of 256
        from paper_1702_04250_gb300 import pppm

        for mode in ("ik", "ad"):
            ref_m = ref if mode == "ik" else OraclePPPM(box, mesh, P, g, "ad", 1.0).compute(xo, qo)
            pm = pppm.PPPM(box, n, P, mesh, g, mode=mode, precision=prec)
            pm.set_variant(96)
            fm, evm = pm.compute(torch.tensor(x, dtype=torch.float32, device="cuda"),
                                 torch.tensor(q, dtype=torch.float32, device="cuda"))
            pm.sync()
            check_all(fm.double().cpu().numpy(), evm.cpu().numpy(), ref_m, prec, f"dense tile persistent {mode}")
            pm.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32c", "fp32"])
@pytest.mark.parametrize("P", [2, 5, 7])
def test_make_rho_tile_pairs(torch, prec, P):
    """make_rho on z-pairs of 8^3 tiles (variant bit 7): the mesh and forces
    match the oracle on a 32 x 24 x 48 mesh (6 z tiles, every pair's brick
    wrapping in z at the ends), on 40 z points (5 tiles: each row's last
    tile alone in its CTA), and on ragged tilings (45 = 6 tiles of 7-8
    points, 36 = 5 tiles of 7-8 points, 27 = 4 tiles of 6-7 points).  Then
    40,000 charges packed into one tile pair (two low-word folds in FP32C)."""
    from paper_1702_04250_gb300 import pppm

    r = np.random.default_rng(300 + P)
    box, g = (30.0, 22.0, 45.0), 0.5
    n = 9000
    x = r.uniform(-2.0, 50.0, (n, 3)) * np.array(box) / 48.0
    q = r.normal(size=n)
    dt = torch.float64 if prec == "fp64" else torch.float32
    xo, qo = oracle_inputs(x, q, prec)
    for mesh in ((32, 24, 48), (32, 24, 40), (27, 20, 45), (20, 18, 36), (24, 30, 27)):
        ref = OraclePPPM(box, mesh, P, g, "ik", 1.0).compute(xo, qo, keep=True)
        plan = pppm.PPPM(box, n, P, mesh, g, mode="ik", precision=prec)
        base = plan.variant()
        plan.set_variant((base & ~(4 | 16)) | 128)
        f, ev = plan.compute(torch.tensor(x, dtype=dt, device="cuda"), torch.tensor(q, dtype=dt, device="cuda"))
        plan.sync()
        rho = plan.get_array("rho").astype(np.float64)
        rerr = np.sqrt(np.mean((rho - ref["rho"]) ** 2)) / np.sqrt(np.mean(ref["rho"] ** 2))
        assert rerr < (1e-12 if prec == "fp64" else 1e-5), (mesh, rerr)
        check_all(f.double().cpu().numpy(), ev.cpu().numpy(), ref, prec, f"tile pairs P={P} mesh={mesh}")
        plan.close()
    if prec != "fp32c" or P != 7:
        return
    m = 40000
    xd = 10.0 + r.uniform(0.0, 1.2, (m, 3)) * np.array([1.0, 1.0, 2.0])
    qd = r.normal(size=m)
    xo, qo = oracle_inputs(xd, qd, prec)
    mesh = (32, 24, 48)
    refd = OraclePPPM(box, mesh, P, g, "ik", 1.0).compute(xo, qo, keep=True)
    pd = pppm.PPPM(box, m, P, mesh, g, mode="ik", precision=prec)
    pd.set_variant((pd.variant() & ~(4 | 16)) | 128)
    fd, evd = pd.compute(torch.tensor(xd, dtype=dt, device="cuda"), torch.tensor(qd, dtype=dt, device="cuda"))
    pd.sync()
    rd = pd.get_array("rho").astype(np.float64)
    assert np.sqrt(np.mean((rd - refd["rho"]) ** 2)) / np.sqrt(np.mean(refd["rho"] ** 2)) < 1e-5
    check_all(fd.double().cpu().numpy(), evd.cpu().numpy(), refd, prec, "dense tile pair")
    pd.close()


@pytest.mark.parametrize("prec,P,n,spread", [("fp32c", 5, 256, 1.5), ("fp32c", 7, 257, 1.5),
                                             ("fp32c", 5, 513, 0.2), ("fp64", 7, 257, 0.2)])
def test_subchunk_boundaries(torch, prec, P, n, spread):
    """make_rho orders each tile's particles in sub-chunks of 256 by the shared
    bank their stencil runs start on: one tile holding exactly 256, 257 or 513
    charges (a full sub-chunk, one plus a single particle, two plus one), and
    with spread 0.2 every charge on the same anchor (all in one bank bin)."""
    r = np.random.default_rng(37 + n)
    box, mesh, g = (20.0, 20.0, 20.0), (20, 20, 20), 0.5
    x = 3.3 + r.uniform(0.0, spread, (n, 3))
    q = r.normal(size=n)
    plan, f, ev = run(torch, box, mesh, P, g, "ik", prec, x, q)
    xo, qo = oracle_inputs(x, q, prec)
    ref = OraclePPPM(box, mesh, P, g, "ik", 1.0).compute(xo, qo, keep=True)
    rho = plan.get_array("rho").astype(np.float64)
    rerr = np.sqrt(np.mean((rho - ref["rho"]) ** 2)) / np.sqrt(np.mean(ref["rho"] ** 2))
    assert rerr < (1e-12 if prec == "fp64" else 1e-5), rerr
    check_all(f, ev, ref, prec, f"sub-chunk n={n}")
    plan.close()


def test_empty_input(torch):
    from paper_1702_04250_gb300 import pppm

    plan = pppm.PPPM((10.0, 10.0, 10.0), 16, 5, (16, 16, 16), 0.4, mode="ik", precision="fp64")
    x = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    q = torch.zeros((0,), dtype=torch.float64, device="cuda")
    f, ev = plan.compute(x, q)
    plan.sync()
    assert f.shape == (0, 3)
    assert np.all(ev.cpu().numpy() == 0.0)


def test_nonfinite_input_reports_status(torch):
    from paper_1702_04250_gb300 import pppm

    plan = pppm.PPPM((10.0, 10.0, 10.0), 16, 5, (16, 16, 16), 0.4, mode="ik", precision="fp32c")
    x = torch.rand((16, 3), device="cuda") * 10
    x[3, 1] = float("nan")
    q = torch.ones(16, device="cuda")
    plan.compute(x, q)
    assert plan.sync_status() == pppm.PPPM_ENONFINITE
    # the error word is cleared and the plan stays usable
    x[3, 1] = 1.0
    f, ev = plan.compute(x, q)
    assert plan.sync_status() == pppm.PPPM_OK
    assert torch.isfinite(f).all()


def test_n_above_plan_capacity_is_rejected(torch):
    from paper_1702_04250_gb300 import pppm

    plan = pppm.PPPM((10.0, 10.0, 10.0), 4, 5, (16, 16, 16), 0.4)
    x = torch.rand((8, 3), device="cuda")
    with pytest.raises(pppm.PPPMError):
        plan.compute(x, torch.ones(8, device="cuda"))


def test_graph_mode_and_host_path_match(torch, c2_refs):
    w, g, refs = c2_refs
    from paper_1702_04250_gb300 import pppm

    x = torch.tensor(w.x, dtype=torch.float32, device="cuda")
    q = torch.tensor(w.q, dtype=torch.float32, device="cuda")
    plain = pppm.PPPM(w.box, w.n, w.order, w.mesh, g, "ik", "fp32c", w.qqrd2e)
    f0, ev0 = plain.compute(x, q)
    plain.sync()
    graph = pppm.PPPM(w.box, w.n, w.order, w.mesh, g, "ik", "fp32c", w.qqrd2e, graph=True)
    for _ in range(3):
        f1, ev1 = graph.compute(x, q)
    graph.sync()
    assert rel_rms(f1.double().cpu().numpy(), f0.double().cpu().numpy()) < 1e-5
    fh, evh = plain.compute_host(w.x.astype(np.float32), w.q.astype(np.float32))
    assert rel_rms(fh.astype(np.float64), f0.double().cpu().numpy()) < 1e-5
    check_all(fh.astype(np.float64), evh, refs[("ik", "fp32")], "fp32c", "c2 host path")


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_host_call_with_pinned_buffers(torch, c2_refs, prec):
    """Pinned host buffers (read and written by the kernels over the link) and
    pageable ones (staged copies) give the device call's results, in graph
    mode too; a non-finite input still comes back as a status."""
    w, g, refs = c2_refs
    from paper_1702_04250_gb300 import pppm

    dt = torch.float64 if prec == "fp64" else torch.float32
    plan = pppm.PPPM(w.box, w.n, w.order, w.mesh, g, "ik", prec, w.qqrd2e, graph=True)
    f0, ev0 = plan.compute(torch.tensor(w.x, dtype=dt, device="cuda"), torch.tensor(w.q, dtype=dt, device="cuda"))
    plan.sync()
    f0 = f0.double().cpu().numpy()
    ev0 = ev0.cpu().numpy().copy()
    xh = torch.tensor(w.x, dtype=dt).pin_memory()
    qh = torch.tensor(w.q, dtype=dt).pin_memory()
    fh = torch.empty((w.n, 3), dtype=dt).pin_memory()
    evh = torch.zeros(8, dtype=torch.float64).pin_memory()
    for _ in range(3):
        fh.zero_()
        evh.zero_()
        plan.compute_host_into(w.n, xh.data_ptr(), qh.data_ptr(), fh.data_ptr(), evh.data_ptr())
        assert rel_rms(fh.double().numpy(), f0) < 1e-5
        assert abs(evh[0].item() - ev0[0]) <= 1e-6 * abs(ev0[0])
    npdt = np.float64 if prec == "fp64" else np.float32
    fp, _ = plan.compute_host(np.asarray(w.x, dtype=npdt), np.asarray(w.q, dtype=npdt))  # pageable: staged
    assert rel_rms(fp.astype(np.float64), f0) < 1e-5
    xh[5, 1] = float("nan")
    with pytest.raises(pppm.PPPMError):
        plan.compute_host_into(w.n, xh.data_ptr(), qh.data_ptr(), fh.data_ptr(), evh.data_ptr())
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_host_call_staged_through_particle_map(torch, prec):
    """From 262,144 charges on, pinned x and q are read over the link once by
    particle_map, which leaves device copies for the scatter: the host call
    matches the device call on 300,000 charges, three times in a row in graph
    mode and once without graphs, and a non-finite input still comes back as
    a status."""
    from paper_1702_04250_gb300 import pppm

    r = np.random.default_rng(2024)
    n, box, mesh, P, g = 300000, (60.0, 60.0, 60.0), (64, 64, 64), 5, 0.35
    x = r.uniform(0.0, 60.0, (n, 3))
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    dt = torch.float64 if prec == "fp64" else torch.float32
    for graph in (True, False):
        plan = pppm.PPPM(box, n, P, mesh, g, "ik", prec, 1.0, graph=graph)
        f0, ev0 = plan.compute(torch.tensor(x, dtype=dt, device="cuda"), torch.tensor(q, dtype=dt, device="cuda"))
        plan.sync()
        f0 = f0.double().cpu().numpy()
        ev0 = ev0.cpu().numpy().copy()
        xh = torch.tensor(x, dtype=dt).pin_memory()
        qh = torch.tensor(q, dtype=dt).pin_memory()
        fh = torch.empty((n, 3), dtype=dt).pin_memory()
        evh = torch.zeros(8, dtype=torch.float64).pin_memory()
        for _ in range(3 if graph else 1):
            fh.zero_()
            evh.zero_()
            plan.compute_host_into(n, xh.data_ptr(), qh.data_ptr(), fh.data_ptr(), evh.data_ptr())
            assert rel_rms(fh.double().numpy(), f0) < 1e-6
            assert abs(evh[0].item() - ev0[0]) <= 1e-6 * abs(ev0[0])
        xh[n - 7, 2] = float("nan")
        with pytest.raises(pppm.PPPMError):
            plan.compute_host_into(n, xh.data_ptr(), qh.data_ptr(), fh.data_ptr(), evh.data_ptr())
        plan.close()


@pytest.mark.parametrize("mode", ["ik", "ad"])
def test_fieldforce_variants_and_autotune(torch, c2_refs, mode):
    """Both fieldforce variants (per-particle through L1, tile-staged brick)
    match the oracle, and autotune keeps one of them with a valid result."""
    w, g, refs = c2_refs
    from paper_1702_04250_gb300 import pppm

    x = torch.tensor(w.x, dtype=torch.float32, device="cuda")
    q = torch.tensor(w.q, dtype=torch.float32, device="cuda")
    plan = pppm.PPPM(w.box, w.n, w.order, w.mesh, g, mode, "fp32c", w.qqrd2e)
    # fieldforce per particle / tile-staged x make_rho one / four brick copies
    # x cuFFT / hand-written Poisson solve x 8^3 / 4^3 tiles
    # ... x the persistent double-buffered fieldforce (bit 6)
    # ... x make_rho on z-pairs of tiles (bit 7)
    for v in (0, 1, 4, 5, 8, 9, 12, 13, 16, 17, 20, 25, 29, 32, 41, 57, 64, 68, 72, 80, 96, 104, 120,
              128, 129, 136, 160, 192, 200, 224):
        plan.set_variant(v)
        f, ev = plan.compute(x, q)
        plan.sync()
        check_all(f.double().cpu().numpy(), ev.cpu().numpy(), refs[(mode, "fp32")], "fp32c", f"variant {v} {mode}")
    plan.set_variant(41)
    assert plan.variant() == 41
    choice = plan.autotune(x, q)
    assert plan.variant() == choice
    assert choice & ~0xFD == 0 and not (choice & 4 and choice & 32)  # bits 0, 2, 3, 4, 5, 6, 7
    assert not (choice & 1 and choice & 64) and not (choice & 128 and choice & (4 | 16))
    f, ev = plan.compute(x, q)
    plan.sync()
    check_all(f.double().cpu().numpy(), ev.cpu().numpy(), refs[(mode, "fp32")], "fp32c", f"autotuned {choice}")
    for bad in (2, 3, 6, 7, 10, 18, 36, 65, 130, 132, 144, 256):  # long tiles are reserved; exclusive pairs; unknown bits
        with pytest.raises(pppm.PPPMError):
            plan.set_variant(bad)
    p64 = pppm.PPPM(w.box, w.n, w.order, w.mesh, g, mode, "fp64", w.qqrd2e)
    for bad in (4, 8, 64):  # the brick copies are the FP32C accumulator; the own FFT and the persistent
        # fieldforce are FP32
        with pytest.raises(pppm.PPPMError):
            p64.set_variant(bad)


@pytest.mark.parametrize("mode", ["ik", "ad"])
def test_order7_variants(torch, mode):
    """FP32C at P = 7 on the water-like 64^3 system: both fieldforce variants
    and both make_rho bricks match the oracle, long tiles (bit 1) are
    refused, autotune keeps a valid variant."""
    from paper_1702_04250_gb300 import pppm

    w = config("c2")
    g = g_of(w)
    xo, qo = oracle_inputs(w.x, w.q, "fp32")
    ref = OraclePPPM(w.box, w.mesh, 7, g, mode, w.qqrd2e).compute(xo, qo)
    x = torch.tensor(w.x, dtype=torch.float32, device="cuda")
    q = torch.tensor(w.q, dtype=torch.float32, device="cuda")
    plan = pppm.PPPM(w.box, w.n, 7, w.mesh, g, mode, "fp32c", w.qqrd2e)
    assert plan.info()["tile"] == 8 and plan.info()["ntiles"] == 512
    for v in (0, 1, 4, 5, 8, 13, 16, 29, 32, 41, 64, 96, 104, 112, 128, 192, 200):
        plan.set_variant(v)
        f, ev = plan.compute(x, q)
        plan.sync()
        check_all(f.double().cpu().numpy(), ev.cpu().numpy(), ref, "fp32c", f"P=7 variant {v} {mode}")
    for bad in (2, 3):
        with pytest.raises(pppm.PPPMError):
            plan.set_variant(bad)
    choice = plan.autotune(x, q)
    assert choice & ~0xFD == 0
    f, ev = plan.compute(x, q)
    plan.sync()
    check_all(f.double().cpu().numpy(), ev.cpu().numpy(), ref, "fp32c", f"P=7 autotuned {choice}")


@pytest.mark.parametrize("mode", ["ik", "ad"])
def test_lut_coefficients_vs_oracle(torch, mode):
    """Table coefficients (LUT-500 / LUT-5000) against the oracle's table,
    FP64 on c1 and FP32C on c2; entries = 0 restores the exact path."""
    from paper_1702_04250_gb300 import pppm

    w = config("c1")
    g = g_of(w)
    x = torch.tensor(w.x, dtype=torch.float64, device="cuda")
    q = torch.tensor(w.q, dtype=torch.float64, device="cuda")
    plan = pppm.PPPM(w.box, w.n, 7, w.mesh, g, mode, "fp64", w.qqrd2e)
    for K in (500, 5000):
        plan.set_lut(K)
        f, ev = plan.compute(x, q)
        plan.sync()
        ref = OraclePPPM(w.box, w.mesh, 7, g, mode, w.qqrd2e, lut=K).compute(w.x, w.q)
        check_all(f.cpu().numpy(), ev.cpu().numpy(), ref, "fp64", f"c1 LUT-{K} {mode}")
    plan.set_lut(0)
    f, ev = plan.compute(x, q)
    plan.sync()
    check_all(f.cpu().numpy(), ev.cpu().numpy(), OraclePPPM(w.box, w.mesh, 7, g, mode, w.qqrd2e).compute(w.x, w.q),
              "fp64", f"c1 exact {mode}")
    with pytest.raises(pppm.PPPMError):
        plan.set_lut(1)
    w2 = config("c2")
    g2 = g_of(w2)
    p32 = pppm.PPPM(w2.box, w2.n, w2.order, w2.mesh, g2, mode, "fp32c", w2.qqrd2e)
    p32.set_lut(5000)
    f, ev = p32.compute(torch.tensor(w2.x, dtype=torch.float32, device="cuda"),
                        torch.tensor(w2.q, dtype=torch.float32, device="cuda"))
    p32.sync()
    xo, qo = oracle_inputs(w2.x, w2.q, "fp32")
    ref = OraclePPPM(w2.box, w2.mesh, w2.order, g2, mode, w2.qqrd2e, lut=5000).compute(xo, qo)
    check_all(f.double().cpu().numpy(), ev.cpu().numpy(), ref, "fp32c", f"c2 LUT-5000 {mode}")


def test_fp64_repeatable(torch, c2_refs):
    w, g, refs = c2_refs
    outs = []
    for _ in range(3):
        _, f, ev = run(torch, w.box, w.mesh, w.order, g, "ad", "fp64", w.x, w.q, w.qqrd2e)
        outs.append((f, ev))
    for f, ev in outs[1:]:
        assert rel_rms(f, outs[0][0]) < 1e-12
        assert abs(ev[0] - outs[0][1][0]) < 1e-12 * abs(outs[0][1][0])


# ---------------------------------------------------------------------------
# energy gradients (the autograd backward)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mode", ["ik", "ad"])
def test_energy_gradients_match_oracle(torch, mode):
    r = np.random.default_rng(7)
    box, mesh, P, g = (12.0, 12.0, 12.0), (16, 16, 16), 5, 0.45
    n = 500
    x = r.uniform(0, 12, (n, 3))
    q = r.normal(size=n)
    from paper_1702_04250_gb300 import pppm

    plan = pppm.PPPM(box, n, P, mesh, g, mode=mode, precision="fp64", qqrd2e=3.0)
    dx, dq, ev = plan.energy_grad(torch.tensor(x, device="cuda"), torch.tensor(q, device="cuda"))
    plan.sync()
    o = OraclePPPM(box, mesh, P, g, mode, 3.0)
    rdx, rdq = o.energy_gradients(x, q)
    assert rel_rms(dx.cpu().numpy(), rdx) < 1e-10
    assert rel_rms(dq.cpu().numpy(), rdq) < 1e-10
    assert abs(ev[0].item() - o.compute(x, q)["energy"]) < 1e-10 * abs(ev[0].item())
    # the per-atom potential entry point is the same dE/dq
    phi = plan.potential(torch.tensor(x, device="cuda"), torch.tensor(q, device="cuda"))
    plan.sync()
    assert rel_rms(phi.cpu().numpy(), rdq) < 1e-10
