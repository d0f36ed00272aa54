"""FP64 CPU oracle for the fused IB-LB viscoelastic time step (arXiv 2209.14889).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` legs (serial, and OpenMP in a child process) and ``--impl reference`` leg of
``bench.py`` may import this package.
The product path (``paper_2209_14889_gb300``) never imports it, and it never imports
the product path.  The arithmetic lives in ``vlb_oracle.c`` (plain C99, FP64); this
module only builds it and marshals numpy arrays.

Layout: every field is a numpy array [component, y, x] (x fastest); populations are
the plain h_n (not shifted); node positions are unwrapped FP64 ``[n_nodes, 2]``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vlb_oracle.c")
# VLB_ORACLE_OPENMP=1 (read at import) loads the same source built with OpenMP: its per-cell loops
# write only their own cell and every sum stays serial, so the results are bitwise the serial ones
_OPENMP = os.environ.get("VLB_ORACLE_OPENMP", "") == "1"
_LIB = os.path.join(_HERE, "libvlb_oracle_omp.so" if _OPENMP else "libvlb_oracle.so")


def build(force: bool = False) -> str:
    """Compile vlb_oracle.c into an in-tree shared library (gcc, -O2, no FP contraction; with
    -fopenmp when VLB_ORACLE_OPENMP=1)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "vlb_oracle.h"))):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared"]
                              + (["-fopenmp"] if _OPENMP else []) + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("tau", ctypes.c_double), ("rho0", ctypes.c_double),
                ("K1111", ctypes.c_double), ("K1122", ctypes.c_double),
                ("K2222", ctypes.c_double), ("K1212", ctypes.c_double),
                ("eta_p", ctypes.c_double), ("Dp", ctypes.c_double),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("xi", ctypes.c_double),
                ("Gamma", ctypes.c_double), ("kappa", ctypes.c_double),
                ("P_cap", ctypes.c_double),
                ("ericksen", ctypes.c_int32), ("walls_y", ctypes.c_int32),
                ("diffusion_substeps", ctypes.c_int32), ("walls_x", ctypes.c_int32)]


class _Ring(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("k_spring", ctypes.c_double), ("eps_angle", ctypes.c_double),
                ("l_eq", ctypes.c_double), ("pull_x", ctypes.c_double), ("pull_y", ctypes.c_double),
                ("trap_k", ctypes.c_double), ("trap_x", ctypes.c_double), ("trap_y", ctypes.c_double)]


class _Diag(ctypes.Structure):
    _fields_ = [("mass_excess", ctypes.c_double), ("mom", ctypes.c_double * 2),
                ("force", ctypes.c_double * 2)]


_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.orc_bessel_i.restype = ctypes.c_double
        L.orc_bessel_i.argtypes = [ctypes.c_int, ctypes.c_double]
        L.orc_k_of_P.restype = ctypes.c_double
        L.orc_k_of_P.argtypes = [ctypes.c_double]
        L.orc_stiffness.argtypes = [ctypes.POINTER(_Params), ctypes.c_double, ctypes.c_double, _dp]
        L.orc_phi.restype = ctypes.c_double
        L.orc_phi.argtypes = [ctypes.c_double]
        L.orc_node_forces.argtypes = [ctypes.POINTER(_Ring), _dp, _dp]
        L.orc_ring_energy.restype = ctypes.c_double
        L.orc_ring_energy.argtypes = [ctypes.POINTER(_Ring), _dp]
        L.orc_spread.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, _dp, _dp, _dp]
        L.orc_interp.argtypes = [ctypes.POINTER(_Params), _dp, ctypes.c_int, _dp, _dp]
        L.orc_moments.argtypes = [ctypes.POINTER(_Params), _dp, _dp, _dp, _dp]
        L.orc_forces.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(_Ring), ctypes.c_int,
                                 _dp, _dp, _dp, ctypes.c_void_p, _dp, ctypes.c_void_p]
        L.orc_rhs.argtypes = [ctypes.POINTER(_Params), _dp, _dp, _dp, _dp, _dp, ctypes.c_int,
                              _dp, _dp]
        L.orc_step.restype = ctypes.c_int
        L.orc_step.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(_Ring), ctypes.c_int,
                               _dp, _dp, _dp, _dp, ctypes.c_void_p,
                               ctypes.POINTER(_Diag), ctypes.c_void_p, ctypes.c_void_p]
        _lib = L
    return _lib


# ---------------------------------------------------------------------------------------
# Parameters
# ---------------------------------------------------------------------------------------

@dataclass
class Params:
    """Method parameters in lattice units (names follow the paper)."""
    nx: int
    ny: int
    tau: float = 0.8
    rho0: float = 1.0
    K1111: float = 0.0
    K1122: float = 0.0
    K2222: float = 0.0
    K1212: float = 0.0
    eta_p: float = 1.0
    Dp: float = 0.0
    alpha: float = 0.0
    beta: float = 0.0
    xi: float = 0.0
    Gamma: float = 0.0
    kappa: float = 0.0
    P_cap: float = 0.99
    ericksen: int = 1
    walls_y: int = 0
    diffusion_substeps: int = 0
    walls_x: int = 0

    def c(self) -> _Params:
        return _Params(self.nx, self.ny, self.tau, self.rho0, self.K1111, self.K1122, self.K2222,
                       self.K1212, self.eta_p, self.Dp, self.alpha, self.beta, self.xi, self.Gamma,
                       self.kappa, self.P_cap, self.ericksen, self.walls_y,
                       self.diffusion_substeps, self.walls_x)


@dataclass
class Ring:
    n_nodes: int
    k_spring: float
    eps_angle: float
    l_eq: float
    pull_x: float = 0.0
    pull_y: float = 0.0
    trap_k: float = 0.0      # Eq. Utrap at the current step: k_trap(t) and R_ext(t)
    trap_x: float = 0.0
    trap_y: float = 0.0
    protocol: object = None  # TrapProtocol or None

    def c(self) -> _Ring:
        return _Ring(self.n_nodes, 0, self.k_spring, self.eps_angle, self.l_eq, self.pull_x,
                     self.pull_y, self.trap_k, self.trap_x, self.trap_y)


@dataclass
class TrapProtocol:
    """The pulling protocol of Eq. Utrap (App. C): the trap turns on over the equilibration, moves
    by d = (dx, dy) from the initial centre of mass R0 during `pull` steps, and turns off after.
    Every transition is a sigmoid of width `width` steps (the paper gives only the width and the
    equilibration time; this is the reading, taken from the transitions it names):
      s(t; c)  = 1 / (1 + exp(-8 (t - c) / width))           (2 % to 98 % within width steps)
      k(t)     = k_max s(t; width / 2) (1 - s(t; t_eq + pull + width / 2))
      g(t)     = (width / (8 pull)) [sp(8 (t - t_eq) / width) - sp(8 (t - t_eq - pull) / width)],
                 sp(z) = log(1 + e^z): the integral of s(t; t_eq) - s(t; t_eq + pull) over pull
                 (the trap's speed rises and falls by sigmoids), 0 before, 1 after
      R_ext(t) = R0 + d g(t)."""
    k_max: float
    dx: float
    dy: float
    t_eq: float = 30.0
    pull: float = 100.0
    width: float = 30.0
    x0: float = 0.0
    y0: float = 0.0

    def s(self, t, c):
        z = 8.0 * (t - c) / self.width
        if z >= 0:
            return 1.0 / (1.0 + math.exp(-z))
        e = math.exp(z)                  # the same value, without overflow far before c
        return e / (1.0 + e)

    @staticmethod
    def sp(z):
        return z + math.log1p(math.exp(-z)) if z > 0 else math.log1p(math.exp(z))

    def k(self, t):
        return self.k_max * self.s(t, self.width / 2) * (1.0 - self.s(t, self.t_eq + self.pull + self.width / 2))

    def g(self, t):
        a = 8.0 / self.width
        return (self.sp(a * (t - self.t_eq)) - self.sp(a * (t - self.t_eq - self.pull))) / (a * self.pull)

    def ext(self, t):
        g = self.g(t)
        return self.x0 + self.dx * g, self.y0 + self.dy * g


def params_from_workload(w: dict) -> Params:
    """Oracle parameters from a workload recipe.  The relaxation time lambda (in steps) is
    turned into eta_p = lambda * C~11 at k = 0 (reading of the scalar relation
    lambda = eta_p / C of Sec. II B applied to the isotropic modulus of Sec. II C 3)."""
    K = w["K"]
    eta_p = w.get("eta_p")
    if eta_p is None:
        eta_p = w["lambda_steps"] * (3 * K[0] + 2 * K[1] + 4 * K[3] + 3 * K[2]) / 8.0
    return Params(nx=w["nx"], ny=w["ny"], tau=w["tau"], rho0=w["rho0"], K1111=K[0], K1122=K[1],
                  K2222=K[2], K1212=K[3], eta_p=eta_p, Dp=w["Dp"], alpha=w["alpha"],
                  beta=w["beta"], xi=w["xi"], Gamma=w["Gamma"], kappa=w["kappa"],
                  P_cap=w.get("P_cap", 0.99), ericksen=w.get("ericksen", 1),
                  diffusion_substeps=w.get("diffusion_substeps", 0), walls_y=w.get("walls_y", 0),
                  walls_x=w.get("walls_x", 0))


# ---------------------------------------------------------------------------------------
# Thin wrappers of the C functions
# ---------------------------------------------------------------------------------------

def bessel_i(n: int, k: float) -> float:
    return lib().orc_bessel_i(n, k)


def k_of_P(P: float) -> float:
    return lib().orc_k_of_P(P)


def stiffness(p: Params, Px: float, Py: float) -> np.ndarray:
    C = np.zeros(9)
    lib().orc_stiffness(ctypes.byref(p.c()), Px, Py, C)
    return C.reshape(3, 3)


def phi(r: float) -> float:
    return lib().orc_phi(r)


def node_forces(ring: Ring, X: np.ndarray) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float64)
    f = np.zeros_like(X)
    lib().orc_node_forces(ctypes.byref(ring.c()), X.reshape(-1), f.reshape(-1))
    return f


def ring_energy(ring: Ring, X: np.ndarray) -> float:
    return lib().orc_ring_energy(ctypes.byref(ring.c()),
                                 np.ascontiguousarray(X, dtype=np.float64).reshape(-1))


def spread(p: Params, X: np.ndarray, f: np.ndarray) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros((2, p.ny, p.nx))
    lib().orc_spread(ctypes.byref(p.c()), X.shape[0], X.reshape(-1), f.reshape(-1), out.reshape(-1))
    return out


def interp(p: Params, u: np.ndarray, X: np.ndarray) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    V = np.zeros_like(X)
    lib().orc_interp(ctypes.byref(p.c()), u.reshape(-1), X.shape[0], X.reshape(-1), V.reshape(-1))
    return V


def moments(p: Params, h: np.ndarray, F: np.ndarray):
    rho = np.zeros((p.ny, p.nx))
    u = np.zeros((2, p.ny, p.nx))
    lib().orc_moments(ctypes.byref(p.c()), np.ascontiguousarray(h).reshape(-1),
                      np.ascontiguousarray(F).reshape(-1), rho.reshape(-1), u.reshape(-1))
    return rho, u


def _rings_c(rings):
    arr = (_Ring * max(1, len(rings)))()
    for i, r in enumerate(rings):
        arr[i] = r.c()
    return arr


def forces(p: Params, rings, sigma, P, X, fext=None):
    F = np.zeros((2, p.ny, p.nx))
    fp = np.zeros((2, p.ny, p.nx))
    Xc = np.ascontiguousarray(X, dtype=np.float64).reshape(-1) if len(rings) else np.zeros(2)
    fe = None if fext is None else np.ascontiguousarray(fext, dtype=np.float64)
    lib().orc_forces(ctypes.byref(p.c()), _rings_c(rings), len(rings),
                     np.ascontiguousarray(sigma).reshape(-1), np.ascontiguousarray(P).reshape(-1),
                     Xc, None if fe is None else fe.ctypes.data, F.reshape(-1), fp.ctypes.data)
    return F, fp


def rhs(p: Params, sigma, P, u, psi, omega, with_diffusion=True):
    ds = np.zeros((3, p.ny, p.nx))
    dP = np.zeros((2, p.ny, p.nx))
    lib().orc_rhs(ctypes.byref(p.c()), np.ascontiguousarray(sigma).reshape(-1),
                  np.ascontiguousarray(P).reshape(-1), np.ascontiguousarray(u).reshape(-1),
                  np.ascontiguousarray(psi).reshape(-1), np.ascontiguousarray(omega).reshape(-1),
                  int(with_diffusion), ds.reshape(-1), dP.reshape(-1))
    return ds, dP


W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
C9 = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]])


def equilibrium(rho, u):
    """Second-order D2Q9 equilibrium (the standard form the paper cites for Eq. BGK)."""
    cu = np.einsum("nc,cyx->nyx", C9.astype(float), u)
    uu = (u ** 2).sum(0)
    return W9[:, None, None] * rho[None] * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * uu[None])


# ---------------------------------------------------------------------------------------
# Simulation driver
# ---------------------------------------------------------------------------------------

@dataclass
class Sim:
    """A full oracle state: h[9,ny,nx], sigma[3,ny,nx] (xx,yy,xy), P[2,ny,nx], X[n,2]."""
    p: Params
    rings: list
    h: np.ndarray
    sigma: np.ndarray
    P: np.ndarray
    X: np.ndarray
    t: int = 0
    fext: np.ndarray | None = None
    series: list = field(default_factory=list)

    @staticmethod
    def from_workload(w: dict) -> "Sim":
        p = params_from_workload(w)
        ny, nx = p.ny, p.nx
        h = np.repeat(W9[:, None, None] * p.rho0, ny, axis=1).repeat(nx, axis=2).copy()
        sigma = np.zeros((3, ny, nx))
        Peq = np.sqrt(-p.alpha / p.beta) if (p.beta > 0 and p.alpha < 0) else 0.0
        th = w["director_angle"]
        P = np.zeros((2, ny, nx))
        P[0] = Peq * np.cos(th)
        P[1] = Peq * np.sin(th)
        if w.get("noise") is not None:
            P += w["noise"]
        rings, Xs = [], []
        for r in w["rings"]:
            Xr = np.asarray(r["X"], dtype=np.float64)
            tp = r.get("trap")
            prot = None
            if tp is not None:
                prot = TrapProtocol(k_max=tp["k"], dx=tp["dx"], dy=tp["dy"], t_eq=tp.get("t_eq", 30.0),
                                    pull=tp.get("pull", 100.0), width=tp.get("width", 30.0),
                                    x0=float(Xr[:, 0].mean()), y0=float(Xr[:, 1].mean()))
            rings.append(Ring(n_nodes=len(r["X"]), k_spring=r["k_spring"],
                              eps_angle=r["eps_angle"], l_eq=r["l_eq"],
                              pull_x=r["pull_force"] * np.cos(r["pull_angle"]),
                              pull_y=r["pull_force"] * np.sin(r["pull_angle"]), protocol=prot))
            Xs.append(Xr)
        X = np.concatenate(Xs) if Xs else np.zeros((0, 2))
        return Sim(p, rings, h, sigma, P, X)

    def step(self, n: int = 1, every: int = 0):
        """Advance n steps; every `every` steps (t % every == 0) record the diagnostics of
        the state at t: (t, mass_excess, mom_x, mom_y, F_x, F_y, [frest_x, frest_y, com_x,
        com_y] per ring)."""
        L = lib()
        pc = self.p.c()
        rc = _rings_c(self.rings)
        nr = len(self.rings)
        for _ in range(n):
            if self._set_trap():
                rc = _rings_c(self.rings)
            rec = every > 0 and self.t % every == 0
            d = _Diag()
            fr = np.zeros(2 * max(nr, 1))
            cm = np.zeros(2 * max(nr, 1))
            Xf = self.X.reshape(-1) if self.X.size else np.zeros(2)
            rc_ = L.orc_step(ctypes.byref(pc), rc, nr, self.h.reshape(-1), self.sigma.reshape(-1),
                             self.P.reshape(-1), Xf,
                             None if self.fext is None else self.fext.ctypes.data,
                             ctypes.byref(d) if rec else None,
                             fr.ctypes.data if rec else None, cm.ctypes.data if rec else None)
            if rc_ != 0:
                raise MemoryError("orc_step failed")
            if self.X.size:
                self.X = Xf.reshape(-1, 2)
            if rec:
                row = [self.t, d.mass_excess, d.mom[0], d.mom[1], d.force[0], d.force[1]]
                for r in range(nr):
                    row += [fr[2 * r], fr[2 * r + 1], cm[2 * r], cm[2 * r + 1]]
                self.series.append(row)
            self.t += 1
        return self

    def _set_trap(self) -> bool:
        """Eq. Utrap at the current step t on every trapped ring; False if there is none."""
        trapped = False
        for r in self.rings:
            if r.protocol is not None:
                r.trap_k = r.protocol.k(self.t)
                r.trap_x, r.trap_y = r.protocol.ext(self.t)
                trapped = True
        return trapped

    def fields(self):
        """rho - rho0, u (with the half-force correction) of the current state, sigma, P."""
        self._set_trap()          # the force of the state at t includes the trap at t
        F, fp = forces(self.p, self.rings, self.sigma, self.P, self.X, self.fext)
        rho, u = moments(self.p, self.h, F)
        return {"drho": rho - self.p.rho0, "ux": u[0], "uy": u[1], "sxx": self.sigma[0],
                "syy": self.sigma[1], "sxy": self.sigma[2], "Px": self.P[0], "Py": self.P[1]}
