"""The allocation-free mesh builder against the plan-based path.

pppm_make_rho_noalloc exists for callers that cannot allocate device memory
where they need a charge mesh (an engine that owns all GPU memory in its own
pool, code under stream capture, a step loop that must not pay cudaMalloc's
device-wide synchronisation).  It must produce the same mesh as pppm_compute
does, call after call, even though every call reuses one fixed scratch array.
This file is collected last so a stop-at-first-failure run has already run
every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_1702_04250_gb300.workloads import config

pytestmark = pytest.mark.gpu

TOL = 1e-4  # FP32 / FP32C tolerance used by the parity tests


@pytest.fixture(scope="module")
def torch():
    import torch as t

    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_04250_gb300 import build

    build.build()
    return t


def noalloc(L, box, mesh, order, prec, x, q, rho, stream):
    return L.pppm_make_rho_noalloc((ctypes.c_double * 3)(*box), (ctypes.c_int * 3)(*mesh), order, prec,
                                   x.shape[0], ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(q.data_ptr()),
                                   ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(stream))


@pytest.mark.parametrize("prec", ["fp32c", "fp32"])
def test_noalloc_matches_plan_mesh_twice(torch, prec):
    from paper_1702_04250_gb300 import pppm

    L = pppm.lib()
    L.pppm_make_rho_noalloc.restype = ctypes.c_int
    w = config("c2")  # 32,001 charges, 64^3 mesh, order 5: 512 tiles
    g = pppm.estimate_g(w.rel_acc, w.r_cut, w.n, float(np.sum(w.q ** 2)), w.box)
    x = torch.tensor(w.x, dtype=torch.float32, device="cuda")
    q = torch.tensor(w.q, dtype=torch.float32, device="cuda")
    plan = pppm.PPPM(w.box, w.n, w.order, w.mesh, g, mode="ik", precision=prec, qqrd2e=w.qqrd2e)
    plan.compute(x, q)
    plan.sync()
    ref = plan.get_array("rho").astype(np.float64)
    stream = torch.cuda.current_stream().cuda_stream
    code = pppm.PRECISIONS[prec]
    for _ in range(2):  # the second call reuses the scratch the first one left behind
        rho = torch.full(w.mesh, float("nan"), dtype=torch.float32, device="cuda")
        rc = noalloc(L, w.box, w.mesh, w.order, code, x, q, rho, stream)
        assert rc == pppm.PPPM_OK, pppm.strerror(rc)
        torch.cuda.synchronize()
        got = rho.double().cpu().numpy()
        assert np.isfinite(got).all()
        err = np.sqrt(np.mean((got - ref) ** 2)) / np.sqrt(np.mean(ref ** 2))
        assert err <= TOL, err


def test_noalloc_rejects_sizes_beyond_its_limits(torch):
    from paper_1702_04250_gb300 import pppm

    L = pppm.lib()
    L.pppm_make_rho_noalloc.restype = ctypes.c_int
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
