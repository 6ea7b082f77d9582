"""The C-ABI library loads and exports every symbol include/pppm_gb300.h
declares; host-only entry points behave; nothing here touches a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pppm_gb300.h")


@pytest.fixture(scope="module")
def L():
    from paper_1702_04250_gb300 import build, pppm

    build.build()
    return pppm.lib()


def declared_symbols():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pppm_[a-z_0-9]+)\s*\(", txt)))


def test_exports_every_declared_symbol(L):
    syms = declared_symbols()
    assert len(syms) >= 12
    for s in syms:
        assert hasattr(L, s), s


def test_strerror(L):
    from paper_1702_04250_gb300 import pppm

    for s in range(8):
        assert len(pppm.strerror(s)) > 0
    assert pppm.strerror(99) == "unknown status"


def test_estimate_g_matches_oracle(L):
    from oracle import estimate_g_ewald
    from paper_1702_04250_gb300 import pppm
    from paper_1702_04250_gb300.workloads import config

    for name in ("c1", "c2"):
        w = config(name)
        q2 = float(np.sum(w.q ** 2))
        a = pppm.estimate_g(w.rel_acc, w.r_cut, w.n, q2, w.box)
        b = estimate_g_ewald(w.rel_acc, w.r_cut, w.n, q2, w.box)
        assert abs(a - b) < 1e-14 * b
    with pytest.raises(pppm.PPPMError):
        pppm.estimate_g(0.9, 1.0, 10, 1.0, (1.0, 1.0, 1.0))  # no positive root
    with pytest.raises(pppm.PPPMError):
        pppm.estimate_g(-1.0, 10.0, 10, 1.0, (10.0, 10.0, 10.0))


def test_setup_rejects_bad_arguments_before_touching_a_gpu(L):
    from paper_1702_04250_gb300 import pppm

    h = ctypes.c_void_p()
    box = (ctypes.c_double * 3)(10.0, 10.0, 10.0)
    good = (ctypes.c_int * 3)(16, 16, 16)
    small = (ctypes.c_int * 3)(16, 4, 16)
    cases = [
        (box, 10, 1, good, 0.3, 0, 0),      # order < 2
        (box, 10, 8, good, 0.3, 0, 0),      # order > 7
        (box, 10, 5, small, 0.3, 0, 0),     # mesh smaller than the stencil
        (box, 10, 5, good, -0.3, 0, 0),     # g <= 0
        (box, 10, 5, good, 0.3, 2, 0),      # bad mode
        (box, 10, 5, good, 0.3, 0, 9),      # bad precision
        (box, -1, 5, good, 0.3, 0, 0),      # negative n_max
    ]
    for b, n, P, m, g, mode, prec in cases:
        rc = L.pppm_setup(ctypes.byref(h), b, n, P, m, g, mode, prec, 1.0, None)
        assert rc == pppm.PPPM_EINVAL
        assert not h.value
    assert L.pppm_compute(None, 0, None, None, None, None) == pppm.PPPM_EINVAL
    assert L.pppm_destroy(None) == pppm.PPPM_EINVAL
