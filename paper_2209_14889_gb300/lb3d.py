"""Python binding of the three-dimensional C ABI in include/lb3d.h (argument marshalling only).

Every step runs in the CUDA kernels of libvlb.so (lb3d.cu); there is no CPU fallback: loading
fails if the library has not been built.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import lb as _lb

FIELDS = {"drho": 0, "ux": 1, "uy": 2, "uz": 3, "sxx": 4, "syy": 5, "szz": 6, "syz": 7, "sxz": 8, "sxy": 9,
          "Px": 10, "Py": 11, "Pz": 12}
FIELD_POP0 = 13
SCALARS = tuple(FIELDS)


class lb3d_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("readout_every", ctypes.c_int32),
                ("tau", ctypes.c_double), ("rho0", ctypes.c_double),
                ("K1111", ctypes.c_double), ("K1122", ctypes.c_double), ("K2222", ctypes.c_double),
                ("K1212", ctypes.c_double), ("K2233", ctypes.c_double),
                ("eta_p", ctypes.c_double), ("Dp", ctypes.c_double),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("xi", ctypes.c_double),
                ("Gamma", ctypes.c_double), ("kappa", ctypes.c_double), ("P_cap", ctypes.c_double),
                ("fext", ctypes.c_double * 3), ("P_ref", ctypes.c_double * 3),
                ("ericksen", ctypes.c_int32), ("max_samples", ctypes.c_int32)]


_H = ctypes.c_void_p
_bound = False


def lib():
    """libvlb.so with the lb3d_* signatures declared."""
    global _bound
    L = _lb.lib()
    if not _bound:
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        sig = {
            "lb3d_create": (ctypes.c_int, [ctypes.POINTER(lb3d_params), ctypes.POINTER(_H)]),
            "lb3d_destroy": (None, [_H]),
            "lb3d_last_error": (ctypes.c_char_p, [_H]),
            "lb3d_init_fields": (ctypes.c_int, [_H, vp]),
            "lb3d_step": (ctypes.c_int, [_H, i64]),
            "lb3d_sync": (ctypes.c_int, [_H]),
            "lb3d_time": (i64, [_H]),
            "lb3d_readout": (ctypes.c_int, [_H, i32, vp, sz, i32]),
            "lb3d_series": (ctypes.c_int, [_H, vp, i32, ctypes.POINTER(i32)]),
            "lb3d_timing": (ctypes.c_int, [_H, i32]),
            "lb3d_kernel_time": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]),
            "lb3d_launches_per_step": (i32, [_H]),
            "lb3d_moment_table": (i32, [ctypes.c_double, vp, i32]),
            "lb3d_bytes_per_cell": (ctypes.c_double, [_H]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _bound = True
    return L


class LB3DError(_lb.LBError):
    pass


def _check(h, rc):
    if rc != _lb.LB_OK:
        raise LB3DError(rc, lib().lb3d_last_error(h).decode())


def reference_polarization(w: dict) -> np.ndarray:
    """P_eq d: the uniform state a workload's P fluctuates about (stored as the reference)."""
    Peq = np.sqrt(-w["alpha"] / w["beta"]) if (w["beta"] > 0 and w["alpha"] < 0) else 0.0
    return Peq * np.asarray(w["director"], dtype=np.float64)


def params_from_workload(w: dict, max_samples: int = 4096) -> lb3d_params:
    fe = w.get("fext") or (0.0, 0.0, 0.0)
    pr = reference_polarization(w)
    return lb3d_params(nx=w["nx"], ny=w["ny"], nz=w["nz"], readout_every=w.get("every", 10), tau=w["tau"],
                       rho0=w["rho0"], K1111=w["K"][0], K1122=w["K"][1], K2222=w["K"][2], K1212=w["K"][3],
                       K2233=w["K"][4], eta_p=w["eta_p"], Dp=w["Dp"], alpha=w["alpha"], beta=w["beta"],
                       xi=w["xi"], Gamma=w["Gamma"], kappa=w["kappa"], P_cap=w["P_cap"],
                       fext=(ctypes.c_double * 3)(*fe), P_ref=(ctypes.c_double * 3)(*pr),
                       ericksen=w["ericksen"], max_samples=max_samples)


def moment_table(P_cap: float) -> np.ndarray:
    """The (<mu^2>, <mu^4>) moments behind the kernels' table, [8193, 2] FP32 (host computation)."""
    L = lib()
    n = L.lb3d_moment_table(float(P_cap), None, 0)
    if n < 0:
        raise LB3DError(n, "bad P_cap")
    out = np.zeros(2 * n, dtype=np.float32)
    L.lb3d_moment_table(float(P_cap), out.ctypes.data, n)
    return out.reshape(n, 2)


class Solver3D:
    """A three-dimensional handle (periodic box) on the current CUDA device."""

    def __init__(self, params: lb3d_params):
        self.params = params
        self.shape = (params.nz, params.ny, params.nx)
        self.h = _H()
        rc = lib().lb3d_create(ctypes.byref(params), ctypes.byref(self.h))
        if rc != _lb.LB_OK:
            raise LB3DError(rc, "lb3d_create failed")

    @staticmethod
    def from_workload(w: dict, **kw) -> "Solver3D":
        """Fluid at rest, sigma = 0, P = P_eq d + the workload's seeded noise."""
        s = Solver3D(params_from_workload(w, **kw))
        pr = reference_polarization(w)
        P = np.broadcast_to(pr[:, None, None, None], (3,) + s.shape).copy()
        if w.get("noise") is not None:
            P += w["noise"]
        s.init_fields(P)
        return s

    def close(self):
        if self.h:
            lib().lb3d_destroy(self.h)
            self.h = _H()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_fields(self, P=None):
        Pv = None if P is None else np.ascontiguousarray(P, dtype=np.float64)
        _check(self.h, lib().lb3d_init_fields(self.h, None if Pv is None else Pv.ctypes.data))

    def step(self, n: int = 1):
        _check(self.h, lib().lb3d_step(self.h, int(n)))

    def sync(self):
        _check(self.h, lib().lb3d_sync(self.h))

    @property
    def t(self) -> int:
        return lib().lb3d_time(self.h)

    def readout(self, field) -> np.ndarray:
        idx = FIELDS[field] if isinstance(field, str) else int(field)
        out = np.zeros(self.shape, dtype=np.float32)
        _check(self.h, lib().lb3d_readout(self.h, idx, out.ctypes.data, out.size, 0))
        return out

    def readout_device(self, field, dst_ptr: int, count: int):
        idx = FIELDS[field] if isinstance(field, str) else int(field)
        _check(self.h, lib().lb3d_readout(self.h, idx, ctypes.c_void_p(dst_ptr), count, 1))

    def fields(self) -> dict:
        return {k: self.readout(k).astype(np.float64) for k in SCALARS}

    def populations(self) -> np.ndarray:
        return np.stack([self.readout(FIELD_POP0 + n) for n in range(19)])

    def series(self) -> np.ndarray:
        cap = self.params.max_samples
        buf = np.zeros((cap, 8))
        n = ctypes.c_int32(0)
        _check(self.h, lib().lb3d_series(self.h, buf.ctypes.data, cap, ctypes.byref(n)))
        return buf[:n.value].copy()

    def timing(self, enable: bool):
        _check(self.h, lib().lb3d_timing(self.h, 1 if enable else 0))

    def kernel_time(self):
        ms, n = ctypes.c_double(), ctypes.c_int64()
        _check(self.h, lib().lb3d_kernel_time(self.h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    @property
    def launches_per_step(self) -> int:
        return lib().lb3d_launches_per_step(self.h)

    @property
    def bytes_per_cell(self) -> float:
        return lib().lb3d_bytes_per_cell(self.h)
