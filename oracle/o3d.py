"""FP64 CPU oracle of the three-dimensional step (D3Q19; the orientation integral of Eq. CTens
over the unit sphere) -- the first extension of Sec. IV.

TEST INFRASTRUCTURE ONLY.  Only ``tests/`` and the CPU legs of ``bench.py`` may import this
module.  The arithmetic lives in ``vlb3d_oracle.c`` (plain C99, FP64); this module builds it and
marshals numpy arrays.

Layout: every field is a numpy array [component, z, y, x] (x fastest); populations are the
plain h_n (not shifted); sigma^p has the six components (xx, yy, zz, yz, xz, xy).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vlb3d_oracle.c")
_HDR = os.path.join(_HERE, "vlb3d_oracle.h")
# VLB_ORACLE_OPENMP=1 (read at import) loads the same source built with OpenMP: its per-cell
# loops write only their own cell and every sum stays serial, so the results are bitwise the
# serial ones
_OPENMP = os.environ.get("VLB_ORACLE_OPENMP", "") == "1"
_LIB = os.path.join(_HERE, "libvlb3d_oracle_omp.so" if _OPENMP else "libvlb3d_oracle.so")

SIGMA = ("sxx", "syy", "szz", "syz", "sxz", "sxy")


def build(force: bool = False) -> str:
    """Compile vlb3d_oracle.c into an in-tree shared library (gcc, -O2, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC),
                                                                          os.path.getmtime(_HDR)):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared"]
                              + (["-fopenmp"] if _OPENMP else []) + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("n_quad", ctypes.c_int32),
                ("tau", ctypes.c_double), ("rho0", ctypes.c_double),
                ("K1111", ctypes.c_double), ("K1122", ctypes.c_double),
                ("K2222", ctypes.c_double), ("K1212", ctypes.c_double), ("K2233", ctypes.c_double),
                ("eta_p", ctypes.c_double), ("Dp", ctypes.c_double),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("xi", ctypes.c_double),
                ("Gamma", ctypes.c_double), ("kappa", ctypes.c_double),
                ("P_cap", ctypes.c_double),
                ("ericksen", ctypes.c_int32), ("pad_", ctypes.c_int32)]


class _Diag(ctypes.Structure):
    _fields_ = [("mass_excess", ctypes.c_double), ("mom", ctypes.c_double * 3),
                ("force", ctypes.c_double * 3)]


_L = None


def lib():
    global _L
    if _L is None:
        L = ctypes.CDLL(build())
        d, vp, i32 = ctypes.c_double, ctypes.c_void_p, ctypes.c_int32
        P = ctypes.POINTER(_Params)
        sig = {
            "o3_lattice": (None, [vp, vp]),
            "o3_langevin": (d, [d]),
            "o3_k_of_P": (d, [d]),
            "o3_gauss_legendre": (None, [i32, vp, vp]),
            "o3_orientation_moments": (None, [d, i32, vp]),
            "o3_stiffness": (None, [P, vp, vp]),
            "o3_forces": (None, [P, vp, vp, vp, vp, vp, vp]),
            "o3_rhs": (None, [P, vp, vp, vp, vp, vp]),
            "o3_moments": (None, [P, vp, vp, vp, vp]),
            "o3_step": (ctypes.c_int, [P, vp, vp, vp, vp, ctypes.POINTER(_Diag)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _L = L
    return _L


@dataclass
class Params:
    nx: int
    ny: int
    nz: int
    tau: float = 0.8
    rho0: float = 1.0
    K: tuple = (2e-3, 1e-3, 1e-3, 1e-3, 5e-4)     # K1111, K1122, K2222, K1212, K2233
    eta_p: float = 0.05
    Dp: float = 0.05
    alpha: float = -0.9
    beta: float = 1.0
    xi: float = 1.1
    Gamma: float = 1.0
    kappa: float = 0.001
    P_cap: float = 0.99
    ericksen: int = 1
    n_quad: int = 24

    def c(self) -> _Params:
        return _Params(self.nx, self.ny, self.nz, self.n_quad, self.tau, self.rho0, *self.K, self.eta_p,
                       self.Dp, self.alpha, self.beta, self.xi, self.Gamma, self.kappa, self.P_cap,
                       self.ericksen, 0)


def params_from_workload(w: dict) -> Params:
    """The oracle's parameters of a three-dimensional workload (relaxation time lambda in steps:
    eta_p = lambda C~11(k = 0), the isotropic modulus of K^x, as in the two-dimensional recipe)."""
    return Params(nx=w["nx"], ny=w["ny"], nz=w["nz"], tau=w["tau"], rho0=w["rho0"], K=tuple(w["K"]),
                  eta_p=w["eta_p"], Dp=w["Dp"], alpha=w["alpha"], beta=w["beta"], xi=w["xi"],
                  Gamma=w["Gamma"], kappa=w["kappa"], P_cap=w["P_cap"], ericksen=w["ericksen"],
                  n_quad=w.get("n_quad", 24))


def lattice():
    c = np.zeros(57, dtype=np.int32)
    w = np.zeros(19)
    lib().o3_lattice(c.ctypes.data, w.ctypes.data)
    return c.reshape(19, 3), w


def langevin(k: float) -> float:
    return lib().o3_langevin(float(k))


def k_of_P(P: float) -> float:
    return lib().o3_k_of_P(float(P))


def gauss_legendre(n: int):
    x, w = np.zeros(n), np.zeros(n)
    lib().o3_gauss_legendre(n, x.ctypes.data, w.ctypes.data)
    return x, w


def orientation_moments(k: float, n_quad: int = 24) -> np.ndarray:
    m = np.zeros(5)
    lib().o3_orientation_moments(float(k), n_quad, m.ctypes.data)
    return m


def stiffness(p: Params, P) -> np.ndarray:
    """C_ijkl(P) as a [3, 3, 3, 3] array."""
    Pv = np.ascontiguousarray(P, dtype=np.float64)
    C = np.zeros(81)
    pc = p.c()
    lib().o3_stiffness(ctypes.byref(pc), Pv.ctypes.data, C.ctypes.data)
    return C.reshape(3, 3, 3, 3)


def forces(p: Params, sigma, P, fext=None):
    """(F, h, f^p), each [3, nz, ny, nx]."""
    shape = (3, p.nz, p.ny, p.nx)
    F, h, fp = np.zeros(shape), np.zeros(shape), np.zeros(shape)
    s = np.ascontiguousarray(sigma, dtype=np.float64)
    Pv = np.ascontiguousarray(P, dtype=np.float64)
    fe = None if fext is None else np.ascontiguousarray(fext, dtype=np.float64)
    pc = p.c()
    lib().o3_forces(ctypes.byref(pc), s.ctypes.data, Pv.ctypes.data, None if fe is None else fe.ctypes.data,
                    F.ctypes.data, h.ctypes.data, fp.ctypes.data)
    return F, h, fp


def rhs(p: Params, sigma, P, u):
    ds = np.zeros((6, p.nz, p.ny, p.nx))
    dP = np.zeros((3, p.nz, p.ny, p.nx))
    s = np.ascontiguousarray(sigma, dtype=np.float64)
    Pv = np.ascontiguousarray(P, dtype=np.float64)
    uv = np.ascontiguousarray(u, dtype=np.float64)
    pc = p.c()
    lib().o3_rhs(ctypes.byref(pc), s.ctypes.data, Pv.ctypes.data, uv.ctypes.data, ds.ctypes.data, dP.ctypes.data)
    return ds, dP


def moments(p: Params, h, F):
    rho = np.zeros((p.nz, p.ny, p.nx))
    u = np.zeros((3, p.nz, p.ny, p.nx))
    hv = np.ascontiguousarray(h, dtype=np.float64)
    Fv = np.ascontiguousarray(F, dtype=np.float64)
    pc = p.c()
    lib().o3_moments(ctypes.byref(pc), hv.ctypes.data, Fv.ctypes.data, rho.ctypes.data, u.ctypes.data)
    return rho, u


@dataclass
class Sim3:
    """A full oracle state: h[19,nz,ny,nx], sigma[6,nz,ny,nx], P[3,nz,ny,nx]."""
    p: Params
    h: np.ndarray
    sigma: np.ndarray
    P: np.ndarray
    t: int = 0
    fext: np.ndarray | None = None
    series: list = field(default_factory=list)

    @staticmethod
    def from_workload(w: dict) -> "Sim3":
        """Fluid at rest with rho0, sigma = 0, P = P_eq d + noise (d: the workload's director)."""
        p = params_from_workload(w)
        _, wts = lattice()
        h = np.broadcast_to(wts[:, None, None, None] * p.rho0, (19, p.nz, p.ny, p.nx)).copy()
        sigma = np.zeros((6, p.nz, p.ny, p.nx))
        Peq = np.sqrt(-p.alpha / p.beta) if (p.beta > 0 and p.alpha < 0) else 0.0
        d = np.asarray(w["director"], dtype=np.float64)
        P = np.broadcast_to((Peq * d)[:, None, None, None], (3, p.nz, p.ny, p.nx)).copy()
        if w.get("noise") is not None:
            P += w["noise"]
        fext = None if w.get("fext") is None else np.asarray(w["fext"], dtype=np.float64)
        return Sim3(p, h, sigma, P, fext=fext)

    def step(self, n: int = 1, every: int = 0):
        """Advance n steps; every `every` steps (t % every == 0) record the diagnostics of the
        state at t: (t, mass_excess, mom_x, mom_y, mom_z, F_x, F_y, F_z)."""
        L = lib()
        pc = self.p.c()
        fe = None if self.fext is None else np.ascontiguousarray(self.fext)
        for _ in range(n):
            rec = every > 0 and self.t % every == 0
            d = _Diag()
            rc = L.o3_step(ctypes.byref(pc), self.h.reshape(-1).ctypes.data, self.sigma.reshape(-1).ctypes.data,
                           self.P.reshape(-1).ctypes.data, None if fe is None else fe.ctypes.data,
                           ctypes.byref(d) if rec else None)
            if rc != 0:
                raise MemoryError("o3_step failed")
            if rec:
                self.series.append([self.t, d.mass_excess, *d.mom, *d.force])
            self.t += 1
        return self

    def fields(self):
        """rho - rho0, u (with the half-force correction) of the current state, sigma, P."""
        F, _, _ = forces(self.p, self.sigma, self.P, self.fext)
        rho, u = moments(self.p, self.h, F)
        out = {"drho": rho - self.p.rho0, "ux": u[0], "uy": u[1], "uz": u[2]}
        for c, k in enumerate(SIGMA):
            out[k] = self.sigma[c]
        for c, k in enumerate(("Px", "Py", "Pz")):
            out[k] = self.P[c]
        return out
