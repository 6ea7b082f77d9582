"""Python binding of the C ABI in include/pppm_gb300.h (argument marshalling only).

Every step of the k-space path runs in the CUDA library; this module passes
raw device pointers of torch tensors and the current CUDA stream.  It raises
if the library has not been built -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpppm_gb300.so")

(PPPM_OK, PPPM_EINVAL, PPPM_ENOMEM, PPPM_ECUDA, PPPM_ECUFFT, PPPM_ENONFINITE, PPPM_ETIMEOUT, PPPM_ENOTREADY,
 PPPM_EINTERNAL) = range(9)
MODES = {"ik": 0, "ad": 1}
PRECISIONS = {"fp64": 0, "fp32c": 1, "fp32": 2}
ARRAYS = {"rho": 0, "green": 1, "field": 2, "anchor": 3, "tilestart": 4, "perm": 5, "selfforce": 6, "energy": 7}

_lib = None


class PPPMError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = f"{what}: {strerror(status)} (status {status})"
        if status == PPPM_ECUDA:
            detail = lib().pppm_last_cuda_error().decode()
            if detail:
                msg += f" [{detail}]"
        super().__init__(msg)


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run python -m paper_1702_04250_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        dptr = ctypes.POINTER(ctypes.c_double)
        L.pppm_strerror.restype = ctypes.c_char_p
        L.pppm_strerror.argtypes = [i32]
        L.pppm_last_cuda_error.restype = ctypes.c_char_p
        L.pppm_last_cuda_error.argtypes = []
        L.pppm_estimate_g.argtypes = [dbl, dbl, i64, dbl, dptr, dptr]
        L.pppm_fft_size.argtypes = [i32, i32, ctypes.POINTER(i32)]
        L.pppm_kspace_error.argtypes = [dptr, ctypes.POINTER(i32), i32, dbl, i32, i64, dbl, dptr]
        L.pppm_choose_mesh.argtypes = [dptr, i64, dbl, i32, i32, dbl, dbl, i32, ctypes.POINTER(i32), dptr, dptr]
        L.pppm_setup.argtypes = [ctypes.POINTER(vp), dptr, i64, i32, ctypes.POINTER(i32), dbl, i32, i32, dbl, vp]
        L.pppm_destroy.argtypes = [vp]
        L.pppm_set_stream.argtypes = [vp, vp]
        L.pppm_set_graph.argtypes = [vp, i32]
        L.pppm_compute.argtypes = [vp, i64, vp, vp, vp, vp]
        L.pppm_compute_host.argtypes = [vp, i64, vp, vp, vp, vp]
        L.pppm_sync.argtypes = [vp]
        L.pppm_energy_grad.argtypes = [vp, i64, vp, vp, vp, vp, vp]
        L.pppm_potential.argtypes = [vp, i64, vp, vp, vp]
        L.pppm_get_array.argtypes = [vp, i32, vp, ctypes.c_size_t, i32]
        L.pppm_plan_info.argtypes = [vp, ctypes.POINTER(i64)]
        L.pppm_set_profiling.argtypes = [vp, i32]
        L.pppm_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
        L.pppm_set_variant.argtypes = [vp, i32]
        L.pppm_get_variant.argtypes = [vp, ctypes.POINTER(i32)]
        L.pppm_set_lut.argtypes = [vp, i32]
        L.pppm_autotune.argtypes = [vp, i64, vp, vp, vp, ctypes.POINTER(i32)]
        for name in ("pppm_estimate_g", "pppm_fft_size", "pppm_kspace_error", "pppm_choose_mesh", "pppm_setup", "pppm_destroy", "pppm_set_stream", "pppm_set_graph",
                     "pppm_compute", "pppm_compute_host", "pppm_sync", "pppm_energy_grad", "pppm_potential",
                     "pppm_get_array",
                     "pppm_plan_info", "pppm_set_profiling", "pppm_stage_times", "pppm_set_variant", "pppm_get_variant",
                     "pppm_set_lut",
                     "pppm_autotune"):
            getattr(L, name).restype = i32
        _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().pppm_strerror(int(status)).decode()


def _check(rc: int, what: str):
    if rc != PPPM_OK:
        raise PPPMError(rc, what)


def _d3(v):
    return (ctypes.c_double * 3)(*[float(a) for a in v])


def estimate_g(rel_acc: float, r_cut: float, n: int, q2: float, box) -> float:
    out = ctypes.c_double()
    _check(lib().pppm_estimate_g(float(rel_acc), float(r_cut), int(n), float(q2), _d3(box), ctypes.byref(out)),
           "pppm_estimate_g")
    return out.value


FFT_ANY, FFT_SMOOTH, FFT_POW2 = 0, 1, 2  # kinds of pppm_fft_size


def fft_size(n: int, kind: int = FFT_SMOOTH) -> int:
    """Smallest FFT-friendly mesh edge >= n (kind: 0 any, 1 primes <= 7, 2 powers of two)."""
    out = ctypes.c_int()
    _check(lib().pppm_fft_size(int(n), int(kind), ctypes.byref(out)), "pppm_fft_size")
    return out.value


def kspace_error(box, mesh, order: int, g_ewald: float, n: int, q2: float, mode: str = "ik") -> float:
    """Estimated RMS k-space force error of an ik or ad mesh (units of C e^2 / A^2)."""
    out = ctypes.c_double()
    m = (ctypes.c_int * 3)(*[int(v) for v in mesh])
    _check(lib().pppm_kspace_error(_d3(box), m, int(order), float(g_ewald), MODES.get(mode, -1), int(n), float(q2),
                                   ctypes.byref(out)), "pppm_kspace_error")
    return out.value


def choose_mesh(box, n: int, q2: float, order: int, r_cut: float, rel_acc: float, kind: int = FFT_SMOOTH,
                mode: str = "ik"):
    """(mesh, g_ewald, estimated error) meeting rel_acc with the coarsest FFT-friendly mesh of the scan."""
    mesh = (ctypes.c_int * 3)()
    g = ctypes.c_double()
    err = ctypes.c_double()
    _check(lib().pppm_choose_mesh(_d3(box), int(n), float(q2), int(order), MODES.get(mode, -1), float(r_cut),
                                  float(rel_acc), int(kind), mesh, ctypes.byref(g), ctypes.byref(err)),
           "pppm_choose_mesh")
    return tuple(mesh), g.value, err.value


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else int(t.data_ptr()))


class PPPM:
    """One plan: box, order, mesh, g_ewald, differentiation mode, precision."""

    def __init__(self, box, n_max, order, mesh, g_ewald, mode="ik", precision="fp32c", qqrd2e=1.0,
                 stream=None, graph=False, device=None):
        import torch

        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.box = tuple(float(b) for b in box)
        self.mesh = tuple(int(m) for m in mesh)
        self.order = int(order)
        self.g_ewald = float(g_ewald)
        self.mode = mode
        self.precision = precision
        self.qqrd2e = float(qqrd2e)
        self.n_max = int(n_max)
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        if stream is None:
            stream = torch.cuda.Stream(device=self.device) if graph else torch.cuda.current_stream(self.device)
        self.stream = stream
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().pppm_setup(ctypes.byref(h), _d3(box), self.n_max, self.order,
                                    (ctypes.c_int * 3)(*self.mesh), self.g_ewald, MODES[mode],
                                    PRECISIONS[precision], self.qqrd2e, ctypes.c_void_p(stream.cuda_stream)),
                   "pppm_setup")
        self._h = h
        self.ev = torch.zeros(8, dtype=torch.float64, device=self.device)
        if graph:
            _check(lib().pppm_set_graph(self._h, 1), "pppm_set_graph")

    # -- lifetime -------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().pppm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        a = (ctypes.c_int64 * 10)()
        _check(lib().pppm_plan_info(self._h, a), "pppm_plan_info")
        keys = ("Mx", "My", "Mz", "order", "ntiles", "tile", "mode", "precision", "n_max", "n_last")
        return dict(zip(keys, list(a)))

    # -- compute --------------------------------------------------------
    def _prep(self, x, q):
        torch = self.torch
        x = torch.as_tensor(x, device=self.device, dtype=self.dtype).contiguous()
        q = torch.as_tensor(q, device=self.device, dtype=self.dtype).contiguous()
        if x.dim() != 2 or x.shape[1] != 3 or q.shape != (x.shape[0],):
            raise ValueError("x must be [n, 3] and q [n]")
        return x, q

    def compute(self, x, q, f=None, ev=None):
        """Forces [n, 3] and the 7 energy/virial doubles (device tensors)."""
        x, q = self._prep(x, q)
        n = x.shape[0]
        if f is None:
            f = self.torch.empty((n, 3), dtype=self.dtype, device=self.device)
        if ev is None:
            ev = self.ev
        _check(lib().pppm_compute(self._h, n, _ptr(x), _ptr(q), _ptr(f), _ptr(ev)), "pppm_compute")
        return f, ev[:7]

    def compute_host(self, x, q):
        """Host arrays in, host arrays out (copies inside the call)."""
        npdt = np.float64 if self.precision == "fp64" else np.float32
        x = np.ascontiguousarray(x, dtype=npdt)
        q = np.ascontiguousarray(q, dtype=npdt)
        f = np.empty_like(x)
        ev = np.zeros(7, dtype=np.float64)
        rc = lib().pppm_compute_host(self._h, x.shape[0], x.ctypes.data_as(ctypes.c_void_p),
                                     q.ctypes.data_as(ctypes.c_void_p), f.ctypes.data_as(ctypes.c_void_p),
                                     ev.ctypes.data_as(ctypes.c_void_p))
        _check(rc, "pppm_compute_host")
        return f, ev

    def compute_host_into(self, n, x_ptr, q_ptr, f_ptr, ev_ptr):
        """pppm_compute_host on caller-provided host pointers (e.g. pinned tensors)."""
        rc = lib().pppm_compute_host(self._h, int(n), ctypes.c_void_p(x_ptr), ctypes.c_void_p(q_ptr),
                                     ctypes.c_void_p(f_ptr), ctypes.c_void_p(ev_ptr))
        _check(rc, "pppm_compute_host")

    def set_variant(self, variants: int):
        _check(lib().pppm_set_variant(self._h, int(variants)), "pppm_set_variant")

    def variant(self) -> int:
        """The plan's current kernel-variant bitmask."""
        v = ctypes.c_int()
        _check(lib().pppm_get_variant(self._h, ctypes.byref(v)), "pppm_get_variant")
        return v.value

    def set_lut(self, entries: int):
        """Tabulated stencil coefficients with `entries` samples (0: exact)."""
        _check(lib().pppm_set_lut(self._h, int(entries)), "pppm_set_lut")

    def autotune(self, x, q):
        """Time the kernel variants on these inputs, keep the fastest; returns its bitmask."""
        x, q = self._prep(x, q)
        f = self.torch.empty((x.shape[0], 3), dtype=self.dtype, device=self.device)
        choice = ctypes.c_int()
        _check(lib().pppm_autotune(self._h, x.shape[0], _ptr(x), _ptr(q), _ptr(f), ctypes.byref(choice)),
               "pppm_autotune")
        return choice.value

    def energy_grad(self, x, q):
        """(dE/dx [n, 3], dE/dq [n], energy/virial) of the PPPM energy."""
        x, q = self._prep(x, q)
        n = x.shape[0]
        dx = self.torch.empty((n, 3), dtype=self.dtype, device=self.device)
        dq = self.torch.empty((n,), dtype=self.dtype, device=self.device)
        _check(lib().pppm_energy_grad(self._h, n, _ptr(x), _ptr(q), _ptr(dx), _ptr(dq), _ptr(self.ev)),
               "pppm_energy_grad")
        return dx, dq, self.ev[:7]

    def potential(self, x, q):
        """phi_i = dE/dq_i, the k-space potential felt by each atom [n]."""
        x, q = self._prep(x, q)
        phi = self.torch.empty((x.shape[0],), dtype=self.dtype, device=self.device)
        _check(lib().pppm_potential(self._h, x.shape[0], _ptr(x), _ptr(q), _ptr(phi)), "pppm_potential")
        return phi

    STAGES = ("sort", "make_rho", "fft_fwd", "green", "fft_inv", "fieldforce")

    def set_profiling(self, stages=True):
        """True/False for all/no stages, or an iterable of stage names."""
        if stages is True:
            mask = 0x3F
        elif not stages:
            mask = 0
        else:
            mask = sum(1 << self.STAGES.index(s) for s in stages)
        _check(lib().pppm_set_profiling(self._h, mask), "pppm_set_profiling")

    def stage_times(self) -> dict:
        a = (ctypes.c_float * 6)()
        _check(lib().pppm_stage_times(self._h, a), "pppm_stage_times")
        return dict(zip(self.STAGES, [float(v) for v in a]))

    def sync(self):
        _check(lib().pppm_sync(self._h), "pppm_sync")

    def sync_status(self) -> int:
        return int(lib().pppm_sync(self._h))

    # -- inspection -----------------------------------------------------
    def get_array(self, name: str) -> np.ndarray:
        inf = self.info()
        Mx, My, Mz = inf["Mx"], inf["My"], inf["Mz"]
        rdt = np.float64 if self.precision == "fp64" else np.float32
        n = inf["n_last"]
        if name == "rho":
            out = np.empty((Mx, My, Mz), dtype=rdt)
        elif name == "green":
            out = np.empty((Mx, My, Mz // 2 + 1), dtype=np.float64)
        elif name == "field":
            out = np.empty((Mx, My, Mz, 4), dtype=rdt) if self.mode == "ik" else np.empty((Mx, My, Mz), dtype=rdt)
        elif name == "phi":
            out = np.empty((Mx, My, Mz), dtype=rdt)
            name = "field"
        elif name == "anchor":
            out = np.empty((max(n, 0), 3), dtype=np.int32)
        elif name == "tilestart":
            out = np.empty(inf["ntiles"] + 1, dtype=np.int32)
        elif name == "perm":
            out = np.empty(max(n, 0), dtype=np.int32)
        elif name == "selfforce":
            out = np.empty((3, 2), dtype=np.float64)
        elif name == "energy":
            out = np.empty(7, dtype=np.float64)
        else:
            raise KeyError(name)
        _check(lib().pppm_get_array(self._h, ARRAYS[name], out.ctypes.data_as(ctypes.c_void_p), out.nbytes, 1),
               f"pppm_get_array({name})")
        return out


class RealSpace:
    """Real-space (short-range erfc) part of the Ewald split within r_cut;
    with a PPPM plan of the same g_ewald and qqrd2e it completes the Coulomb
    interaction."""

    def __init__(self, box, n_max, r_cut, g_ewald, precision="fp32", qqrd2e=1.0, stream=None, device=None):
        import torch

        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.stream = torch.cuda.current_stream(self.device) if stream is None else stream
        L = lib()
        L.pppm_real_setup.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_double),
                                      ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_void_p]
        L.pppm_real_compute.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
        L.pppm_real_sync.argtypes = [ctypes.c_void_p]
        L.pppm_real_info.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]
        L.pppm_real_destroy.argtypes = [ctypes.c_void_p]
        for nm in ("pppm_real_setup", "pppm_real_compute", "pppm_real_sync", "pppm_real_info", "pppm_real_destroy"):
            getattr(L, nm).restype = ctypes.c_int
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(L.pppm_real_setup(ctypes.byref(h), _d3(box), int(n_max), float(r_cut), float(g_ewald),
                                     PRECISIONS[precision], float(qqrd2e), ctypes.c_void_p(self.stream.cuda_stream)),
                   "pppm_real_setup")
        self._h = h
        self.ev = torch.zeros(8, dtype=torch.float64, device=self.device)

    def close(self):
        if getattr(self, "_h", None):
            lib().pppm_real_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        a = (ctypes.c_int64 * 4)()
        _check(lib().pppm_real_info(self._h, a), "pppm_real_info")
        return {"cells": (a[0], a[1], a[2]), "n_max": a[3]}

    def compute(self, x, q, f=None, accumulate=False):
        """Forces [n, 3] (added onto f when accumulate) and energy/virial [7]."""
        torch = self.torch
        x = torch.as_tensor(x, device=self.device, dtype=self.dtype).contiguous()
        q = torch.as_tensor(q, device=self.device, dtype=self.dtype).contiguous()
        if f is None:
            if accumulate:
                raise ValueError("accumulate needs f")
            f = torch.empty((x.shape[0], 3), dtype=self.dtype, device=self.device)
        _check(lib().pppm_real_compute(self._h, x.shape[0], _ptr(x), _ptr(q), _ptr(f), int(bool(accumulate)),
                                       _ptr(self.ev)), "pppm_real_compute")
        return f, self.ev[:7]

    def sync(self):
        _check(lib().pppm_real_sync(self._h), "pppm_real_sync")


class PPPMBatch:
    """Many independent systems per call (one launch per stage, one graph)."""

    def __init__(self, systems, mode="ik", precision="fp32c", qqrd2e=1.0, stream=None, graph=False, device=None):
        """systems: list of dicts with keys box, n, order, mesh, g_ewald."""
        import torch

        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        ns = len(systems)
        self.nsys = ns
        self.n = [int(s["n"]) for s in systems]
        self.offsets = np.concatenate([[0], np.cumsum(self.n)]).astype(np.int64)
        box = (ctypes.c_double * (3 * ns))(*[float(v) for s in systems for v in s["box"]])
        nn = (ctypes.c_int64 * ns)(*self.n)
        order = (ctypes.c_int * ns)(*[int(s["order"]) for s in systems])
        mesh = (ctypes.c_int * (3 * ns))(*[int(v) for s in systems for v in s["mesh"]])
        gew = (ctypes.c_double * ns)(*[float(s["g_ewald"]) for s in systems])
        if stream is None:
            stream = torch.cuda.Stream(device=self.device) if graph else torch.cuda.current_stream(self.device)
        self.stream = stream
        L = lib()
        L.pppm_batch_setup.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_void_p]
        L.pppm_batch_compute.argtypes = [ctypes.c_void_p] * 5
        L.pppm_batch_set_graph.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.pppm_batch_sync.argtypes = [ctypes.c_void_p]
        L.pppm_batch_destroy.argtypes = [ctypes.c_void_p]
        L.pppm_batch_info.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]
        L.pppm_batch_set_variant.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.pppm_batch_autotune.argtypes = [ctypes.c_void_p] * 4 + [ctypes.POINTER(ctypes.c_int)]
        L.pppm_batch_get_variant.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]
        for nm in ("pppm_batch_setup", "pppm_batch_compute", "pppm_batch_set_graph", "pppm_batch_sync",
                   "pppm_batch_destroy", "pppm_batch_info", "pppm_batch_set_variant", "pppm_batch_autotune",
                   "pppm_batch_get_variant"):
            getattr(L, nm).restype = ctypes.c_int
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(L.pppm_batch_setup(ctypes.byref(h), ns, ctypes.cast(box, ctypes.c_void_p),
                                      ctypes.cast(nn, ctypes.c_void_p), ctypes.cast(order, ctypes.c_void_p),
                                      ctypes.cast(mesh, ctypes.c_void_p), ctypes.cast(gew, ctypes.c_void_p),
                                      MODES[mode], PRECISIONS[precision], float(qqrd2e),
                                      ctypes.c_void_p(stream.cuda_stream)), "pppm_batch_setup")
        self._h = h
        self.ev = torch.zeros((ns, 7), dtype=torch.float64, device=self.device)
        if graph:
            _check(L.pppm_batch_set_graph(self._h, 1), "pppm_batch_set_graph")

    def close(self):
        if getattr(self, "_h", None):
            lib().pppm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        a = (ctypes.c_int64 * 4)()
        _check(lib().pppm_batch_info(self._h, a), "pppm_batch_info")
        return dict(zip(("systems", "particles", "mesh_classes", "orders"), list(a)))

    def compute(self, x, q, f=None):
        """x [sum n, 3], q [sum n] concatenated in system order -> (f, ev [nsys, 7])."""
        torch = self.torch
        x = torch.as_tensor(x, device=self.device, dtype=self.dtype).contiguous()
        q = torch.as_tensor(q, device=self.device, dtype=self.dtype).contiguous()
        if f is None:
            f = torch.empty((x.shape[0], 3), dtype=self.dtype, device=self.device)
        _check(lib().pppm_batch_compute(self._h, _ptr(x), _ptr(q), _ptr(f), _ptr(self.ev)), "pppm_batch_compute")
        return f, self.ev

    def sync(self):
        _check(lib().pppm_batch_sync(self._h), "pppm_batch_sync")

    def set_variant(self, variants: int):
        _check(lib().pppm_batch_set_variant(self._h, int(variants)), "pppm_batch_set_variant")

    def variant(self) -> int:
        """The batch's current kernel-variant bitmask."""
        v = ctypes.c_int()
        _check(lib().pppm_batch_get_variant(self._h, ctypes.byref(v)), "pppm_batch_get_variant")
        return v.value

    def autotune(self, x, q):
        """Time the per-order make_rho and fieldforce variants on these inputs, keep the fastest; returns
        the mask."""
        torch = self.torch
        x = torch.as_tensor(x, device=self.device, dtype=self.dtype).contiguous()
        q = torch.as_tensor(q, device=self.device, dtype=self.dtype).contiguous()
        f = torch.empty((x.shape[0], 3), dtype=self.dtype, device=self.device)
        choice = ctypes.c_int()
        _check(lib().pppm_batch_autotune(self._h, _ptr(x), _ptr(q), _ptr(f), ctypes.byref(choice)),
               "pppm_batch_autotune")
        return choice.value
