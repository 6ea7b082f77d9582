"""The allocation-free mesh builder against the plan-based path and the oracle.

pppm_make_rho_noalloc exists for callers that cannot allocate device memory
where they need a charge mesh (an engine that owns all GPU memory in its own
pool and budget, a step loop that must not pay cudaMalloc's device-wide
synchronisation).  It must produce the same mesh as pppm_compute does, call
after call, even though every call reuses one fixed scratch array that keeps
the previous call's contents; and that mesh must be the oracle's mesh.
This file is collected last so a stop-at-first-failure run has already run
every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from oracle import make_rho
from paper_1702_04250_gb300.workloads import config

pytestmark = pytest.mark.gpu

TOL = 1e-4      # FP32 / FP32C tolerance of the force parity tests (plan-path comparison)
RHO_TOL = 1e-5  # mesh relative RMS against the oracle, the plan path's bar for FP32 meshes


@pytest.fixture(scope="module")
def torch():
    import torch as t

    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_04250_gb300 import build

    build.build()
    return t


@pytest.fixture(scope="module")
def L(torch):
    from paper_1702_04250_gb300 import pppm

    lib = pppm.lib()
    lib.pppm_make_rho_noalloc.restype = ctypes.c_int
    lib.pppm_make_rho_noalloc_status.restype = ctypes.c_int
    lib.pppm_make_rho_noalloc_status.argtypes = [ctypes.c_void_p]
    return lib


def noalloc(L, box, mesh, order, prec, x, q, rho, stream):
    return L.pppm_make_rho_noalloc((ctypes.c_double * 3)(*box), (ctypes.c_int * 3)(*mesh), order, prec,
                                   x.shape[0], ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(q.data_ptr()),
                                   ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(stream))


def rel_rms(a, b):
    return float(np.sqrt(np.mean((a - b) ** 2)) / np.sqrt(np.mean(b ** 2)))


def run_noalloc(torch, L, box, mesh, order, prec, x, q):
    """One call on float32 inputs into a NaN-filled mesh; returns (mesh, status)."""
    from paper_1702_04250_gb300 import pppm

    stream = torch.cuda.current_stream().cuda_stream
    xd = torch.tensor(x, dtype=torch.float32, device="cuda").reshape(-1, 3)
    qd = torch.tensor(q, dtype=torch.float32, device="cuda").reshape(-1)
    rho = torch.full(tuple(mesh), float("nan"), dtype=torch.float32, device="cuda")
    rc = noalloc(L, box, mesh, order, pppm.PRECISIONS[prec], xd, qd, rho, stream)
    assert rc == pppm.PPPM_OK, pppm.strerror(rc)
    st = L.pppm_make_rho_noalloc_status(ctypes.c_void_p(stream))
    return rho.double().cpu().numpy(), st


def oracle_rho(x, q, box, mesh, order):
    """The oracle's mesh of the float32-rounded inputs (what the GPU sees)."""
    xo = np.asarray(x, dtype=np.float32).astype(np.float64).reshape(-1, 3)
    qo = np.asarray(q, dtype=np.float32).astype(np.float64).reshape(-1)
    return make_rho(xo, qo, box, mesh, order)


@pytest.mark.parametrize("prec", ["fp32c", "fp32"])
def test_noalloc_matches_plan_and_oracle_twice(torch, L, prec):
    from paper_1702_04250_gb300 import pppm

    w = config("c2")  # 32,001 charges, 64^3 mesh, order 5: 512 tiles
    g = pppm.estimate_g(w.rel_acc, w.r_cut, w.n, float(np.sum(w.q ** 2)), w.box)
    x = torch.tensor(w.x, dtype=torch.float32, device="cuda")
    q = torch.tensor(w.q, dtype=torch.float32, device="cuda")
    plan = pppm.PPPM(w.box, w.n, w.order, w.mesh, g, mode="ik", precision=prec, qqrd2e=w.qqrd2e)
    plan.compute(x, q)
    plan.sync()
    ref = plan.get_array("rho").astype(np.float64)
    plan.close()
    oref = oracle_rho(w.x, w.q, w.box, w.mesh, w.order)
    for _ in range(2):  # the second call reuses the scratch the first one left behind
        got, st = run_noalloc(torch, L, w.box, w.mesh, w.order, prec, w.x, w.q)
        assert st == pppm.PPPM_OK, pppm.strerror(st)
        assert np.isfinite(got).all()
        assert rel_rms(got, ref) <= TOL
        assert rel_rms(got, oref) <= RHO_TOL


def test_noalloc_empty_input_gives_a_zero_mesh(torch, L):
    from paper_1702_04250_gb300 import pppm

    # a full call first, so the scratch holds a previous call's histogram and records
    w = config("c1")
    got, st = run_noalloc(torch, L, w.box, w.mesh, w.order, "fp32c", w.x, w.q)
    assert st == pppm.PPPM_OK
    got, st = run_noalloc(torch, L, w.box, w.mesh, w.order, "fp32c", np.zeros((0, 3)), np.zeros(0))
    assert st == pppm.PPPM_OK
    assert (got == 0.0).all()


def test_noalloc_at_its_limits_then_a_small_call(torch, L):
    """65,536 charges on a 128^3 mesh (4,096 tiles, every slot of the scratch)
    at order 7, then 1,000 charges on a 16^3 mesh at order 2 and 600 on a
    ragged 20 x 17 x 12 mesh at order 4: the small calls must not see the large
    call's histogram, tile offsets or records."""
    from paper_1702_04250_gb300 import pppm

    r = np.random.default_rng(1702)
    box = (50.0, 50.0, 50.0)
    x = r.uniform(-10.0, 60.0, (65536, 3))
    q = r.normal(size=65536)
    got, st = run_noalloc(torch, L, box, (128, 128, 128), 7, "fp32c", x, q)
    assert st == pppm.PPPM_OK
    assert rel_rms(got, oracle_rho(x, q, box, (128, 128, 128), 7)) <= RHO_TOL
    cases = [((12.0, 12.0, 12.0), (16, 16, 16), 2, 1000), ((13.0, 11.5, 9.0), (20, 17, 12), 4, 600)]
    for bx, mesh, P, n in cases:
        xs = r.uniform(0.0, 1.0, (n, 3)) * np.asarray(bx)
        qs = r.normal(size=n)
        for prec in ("fp32c", "fp32"):
            got, st = run_noalloc(torch, L, bx, mesh, P, prec, xs, qs)
            assert st == pppm.PPPM_OK
            assert rel_rms(got, oracle_rho(xs, qs, bx, mesh, P)) <= RHO_TOL, (mesh, P, prec)


@pytest.mark.parametrize("P", [2, 3, 6, 7])
def test_noalloc_orders(torch, L, P):
    from paper_1702_04250_gb300 import pppm

    r = np.random.default_rng(40 + P)
    box, mesh = (24.0, 24.0, 24.0), (24, 24, 24)
    x = r.uniform(0.0, 24.0, (5000, 3))
    q = r.normal(size=5000)
    got, st = run_noalloc(torch, L, box, mesh, P, "fp32c", x, q)
    assert st == pppm.PPPM_OK
    assert rel_rms(got, oracle_rho(x, q, box, mesh, P)) <= RHO_TOL


def test_noalloc_reports_a_nonfinite_input(torch, L):
    """A NaN position is flagged on the device and reported by the status
    call; the next clean call reports OK again."""
    from paper_1702_04250_gb300 import pppm

    r = np.random.default_rng(7)
    box, mesh = (16.0, 16.0, 16.0), (16, 16, 16)
    x = r.uniform(0.0, 16.0, (300, 3))
    q = r.normal(size=300)
    xb = x.copy()
    xb[123, 1] = np.nan
    _, st = run_noalloc(torch, L, box, mesh, 5, "fp32c", xb, q)
    assert st == pppm.PPPM_ENONFINITE
    got, st = run_noalloc(torch, L, box, mesh, 5, "fp32c", x, q)
    assert st == pppm.PPPM_OK
    assert rel_rms(got, oracle_rho(x, q, box, mesh, 5)) <= RHO_TOL


def test_noalloc_rejects_sizes_beyond_its_limits(torch, L):
    from paper_1702_04250_gb300 import pppm

    stream = torch.cuda.current_stream().cuda_stream
    rho = torch.zeros((16, 16, 16), dtype=torch.float32, device="cuda")
    big = torch.zeros((65537, 3), dtype=torch.float32, device="cuda")
    qb = torch.zeros((65537,), dtype=torch.float32, device="cuda")
    assert noalloc(L, (10.0,) * 3, (16,) * 3, 5, 1, big, qb, rho, stream) == pppm.PPPM_EINVAL
    x = torch.zeros((8, 3), dtype=torch.float32, device="cuda")
    q = torch.zeros((8,), dtype=torch.float32, device="cuda")
    # 136^3 mesh = 17^3 tiles > 4096
    big_mesh = torch.zeros((1,), dtype=torch.float32, device="cuda")
    assert noalloc(L, (10.0,) * 3, (136,) * 3, 5, 1, x, q, big_mesh, stream) == pppm.PPPM_EINVAL
    assert noalloc(L, (10.0,) * 3, (16,) * 3, 5, 0, x, q, rho, stream) == pppm.PPPM_EINVAL  # FP64 not offered
    # boxes the float kernels cannot represent: infinite, NaN, below the smallest normal float
    # (and 16 / 1e-38 overflows), above the largest float
    for bad in ((float("inf"), 10.0, 10.0), (10.0, float("nan"), 10.0), (1e-38, 10.0, 10.0),
                (10.0, 10.0, 1e39)):
        assert noalloc(L, bad, (16,) * 3, 5, 1, x, q, rho, stream) == pppm.PPPM_EINVAL
