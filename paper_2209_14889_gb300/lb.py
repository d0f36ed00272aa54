"""Python binding of the C ABI in include/lb.h (argument marshalling only).

Every step of the method runs in the CUDA kernels of libvlb.so; this module only converts
arguments, allocates readout tensors with torch and passes torch's current CUDA stream.  There
is no CPU fallback: importing the binding fails if the library has not been built.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import _build

LB_OK, LB_EINVAL, LB_ENOMEM, LB_ECUDA, LB_ENONFINITE, LB_EUNSTABLE, LB_EBODY, LB_ESTATE = \
    0, -1, -2, -3, -4, -5, -6, -7
LB_ETIMEOUT = -8
LB_FP32 = 0
LB_FP16_BF16 = 1
LB_KERNEL_AUTO, LB_KERNEL_TILE, LB_KERNEL_SWEEP, LB_KERNEL_PAIR, LB_KERNEL_STRIP = 0, 1, 2, 3, 4
FIELDS = {"drho": 0, "ux": 1, "uy": 2, "sxx": 3, "syy": 4, "sxy": 5, "Px": 6, "Py": 7}
LB_MODEL_TENSORIAL, LB_MODEL_SCALAR = 0, 1
LB_FIELD_POP0 = 8
LB_FIELD_NODES = 17


class LBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("lb error %d: %s" % (code, msg))
        self.code = code


class lb_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("tau", ctypes.c_double), ("rho0", ctypes.c_double),
                ("K1111", ctypes.c_double), ("K1122", ctypes.c_double),
                ("K2222", ctypes.c_double), ("K1212", ctypes.c_double),
                ("eta_p", ctypes.c_double), ("lambda_steps", ctypes.c_double),
                ("Dp", ctypes.c_double),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("xi", ctypes.c_double),
                ("Gamma", ctypes.c_double), ("kappa", ctypes.c_double),
                ("P_cap", ctypes.c_double), ("director_angle", ctypes.c_double),
                ("ericksen", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("readout_every", ctypes.c_int32), ("max_samples", ctypes.c_int32),
                ("diffusion_substeps", ctypes.c_int32), ("model", ctypes.c_int32),
                ("walls_y", ctypes.c_int32), ("walls_x", ctypes.c_int32)]


class lb_ring(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("k_spring", ctypes.c_double), ("eps_angle", ctypes.c_double),
                ("l_eq", ctypes.c_double), ("pull_force", ctypes.c_double),
                ("pull_angle", ctypes.c_double), ("trap_k", ctypes.c_double), ("trap_dx", ctypes.c_double),
                ("trap_dy", ctypes.c_double), ("trap_t_eq", ctypes.c_double), ("trap_pull", ctypes.c_double),
                ("trap_width", ctypes.c_double)]


_lib = None
_H = ctypes.c_void_p
_B = ctypes.c_void_p
_N = ctypes.c_void_p
_L = ctypes.c_void_p


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libvlb.so (raises if it was not built: there is no fallback)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise ImportError("libvlb.so not built: run __graft_entry__.build() (needs nvcc)")
        L = ctypes.CDLL(path)
        vp, i32, i64, sz, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, \
            ctypes.POINTER(ctypes.c_double)
        sig = {
            "lb_create": (ctypes.c_int, [ctypes.POINTER(lb_params), vp, ctypes.POINTER(_H)]),
            "lb_init_fields": (ctypes.c_int, [_H, vp]),
            "lb_set_body": (ctypes.c_int, [_H, i32, ctypes.POINTER(lb_ring), vp]),
            "lb_step": (ctypes.c_int, [_H, i64]),
            "lb_sync": (ctypes.c_int, [_H]),
            "lb_time": (i64, [_H]),
            "lb_readout": (ctypes.c_int, [_H, i32, vp, sz, i32]),
            "lb_write_field": (ctypes.c_int, [_H, i32, vp, sz, i32]),
            "lb_series": (ctypes.c_int, [_H, vp, i32, ctypes.POINTER(i32)]),
            "lb_series_row_len": (i32, [_H]),
            "lb_series_latest": (ctypes.c_int, [_H, vp, i32, ctypes.POINTER(i32)]),
            "lb_series_latest_async": (ctypes.c_int, [_H, vp, i32, ctypes.POINTER(i32)]),
            "lb_series_wait": (ctypes.c_int, [_H]),
            "lb_state_bytes": (i64, [_H]),
            "lb_read_state": (ctypes.c_int, [_H, vp, sz, i32]),
            "lb_write_state": (ctypes.c_int, [_H, vp, sz, i32]),
            "lb_stage_state": (ctypes.c_int, [_H, vp, sz, i32]),
            "lb_commit_state": (ctypes.c_int, [_H]),
            "lb_save": (ctypes.c_int, [_H, ctypes.c_char_p]),
            "lb_load": (ctypes.c_int, [_H, ctypes.c_char_p]),
            "lb_restoring_force": (ctypes.c_int, [_H, i32, vp, i32, ctypes.POINTER(i32)]),
            "lb_timing": (ctypes.c_int, [_H, i32]),
            "lb_kernel_time": (ctypes.c_int, [_H, dp, ctypes.POINTER(i64), dp,
                                              ctypes.POINTER(i64)]),
            "lb_launches_per_step": (i32, [_H]),
            "lb_set_kernel": (ctypes.c_int, [_H, i32]),
            "lb_set_node_tail": (ctypes.c_int, [_H, i32]),
            "lb_lattice_kernel": (i32, [_H]),
            "lb_stiffness_table": (i32, [ctypes.c_double, vp, i32]),
            "lb_bytes_per_cell": (ctypes.c_double, [_H]),
            "lb_last_error": (ctypes.c_char_p, [_H]),
            "lb_destroy": (None, [_H]),
            "lb_batch_create": (ctypes.c_int, [ctypes.POINTER(_H), i32, ctypes.POINTER(_B)]),
            "lb_batch_step": (ctypes.c_int, [_B, i64]),
            "lb_batch_sync": (ctypes.c_int, [_B]),
            "lb_batch_set_shape": (ctypes.c_int, [_B, i32, i32]),
            "lb_batch_shape": (i32, [_B, i32]),
            "lb_batch_autotune": (ctypes.c_int, [_B, ctypes.c_char_p, i32]),
            "lb_batch_set_persistent": (ctypes.c_int, [_B, i32]),
            "lb_batch_set_wait_limit": (ctypes.c_int, [_B, ctypes.c_double, i32]),
            "lb_batch_grid": (i32, [_B]),
            "lb_batch_uses_graph": (i32, [_B]),
            "lb_batch_last_error": (ctypes.c_char_p, [_B]),
            "lb_batch_destroy": (None, [_B]),
            "lb_net_create": (ctypes.c_int, [i32, i32, i32, ctypes.c_uint64, vp, ctypes.POINTER(_N)]),
            "lb_net_num_params": (i64, [_N]),
            "lb_net_set_params": (ctypes.c_int, [_N, vp, i64]),
            "lb_net_get_params": (ctypes.c_int, [_N, vp, i64]),
            "lb_net_get_grads": (ctypes.c_int, [_N, vp, i64]),
            "lb_net_forward": (ctypes.c_int, [_N, vp, vp]),
            "lb_net_output": (vp, [_N]),
            "lb_net_backward": (ctypes.c_int, [_N, vp]),
            "lb_net_mse": (ctypes.c_int, [_N, vp, vp, ctypes.POINTER(ctypes.c_double)]),
            "lb_net_loss_grad": (vp, [_N]),
            "lb_net_adam": (ctypes.c_int, [_N, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
            "lb_net_train_step": (ctypes.c_int, [_N, vp, vp, vp, ctypes.c_float,
                                                 ctypes.POINTER(ctypes.c_double)]),
            "lb_net_activation": (ctypes.c_int, [_N, i32, vp, i64]),
            "lb_net_last_error": (ctypes.c_char_p, [_N]),
            "lb_net_destroy": (None, [_N]),
            "lb_net_shape": (ctypes.c_int, [_N, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                            ctypes.POINTER(i32)]),
            "lb_learned_pack": (ctypes.c_int, [_H, vp, vp, vp]),
            "lb_learned_target": (ctypes.c_int, [vp, vp, vp, vp, i64, vp]),
            "lb_learned_normalize": (ctypes.c_int, [vp, vp, vp, i64, vp]),
            "lb_learned_create": (ctypes.c_int, [_H, _N, vp, ctypes.c_double, ctypes.c_double,
                                                 ctypes.POINTER(_L)]),
            "lb_learned_step": (ctypes.c_int, [_L, i64, ctypes.POINTER(i64)]),
            "lb_learned_stats": (ctypes.c_int, [_L, vp]),
            "lb_learned_last_error": (ctypes.c_char_p, [_L]),
            "lb_learned_destroy": (None, [_L]),
            "lb_conv_kernel": (ctypes.c_int, [i32]),
            "lb_conv_status": (ctypes.c_int, []),
            "lb_conv3x3": (ctypes.c_int, [vp, i64, i32, vp, vp, vp, vp, i64, i32, i32, i32, i32, i32, i32,
                                          i32, vp]),
            "lb_conv3x3_dgrad": (ctypes.c_int, [vp, vp, vp, i32, i32, i32, i32, i32, vp]),
            "lb_conv3x3_wgrad": (ctypes.c_int, [vp, vp, vp, vp, i32, i32, i32, i32, i32, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(h, rc):
    if rc != LB_OK:
        raise LBError(rc, lib().lb_last_error(h).decode())


def params_from_workload(w: dict, precision: int = LB_FP32, max_samples: int = 4096) -> lb_params:
    K = w["K"]
    return lb_params(nx=w["nx"], ny=w["ny"], tau=w["tau"], rho0=w["rho0"], K1111=K[0],
                     K1122=K[1], K2222=K[2], K1212=K[3], eta_p=w.get("eta_p", 0.0) or 0.0,
                     lambda_steps=w.get("lambda_steps", 0.0), Dp=w["Dp"], alpha=w["alpha"],
                     beta=w["beta"], xi=w["xi"], Gamma=w["Gamma"], kappa=w["kappa"],
                     P_cap=w.get("P_cap", 0.99), director_angle=w["director_angle"],
                     ericksen=w.get("ericksen", 1), precision=precision,
                     readout_every=w.get("every", 10), max_samples=max_samples,
                     diffusion_substeps=w.get("diffusion_substeps", 0), model=w.get("model", LB_MODEL_TENSORIAL),
                     walls_y=w.get("walls_y", 0), walls_x=w.get("walls_x", 0))


def stiffness_table(P_cap: float = 0.99) -> np.ndarray:
    """The host-built (a2, a4) table behind C~(P): FP32 [n, 2] (see lb_stiffness_table)."""
    L = lib()
    n = L.lb_stiffness_table(P_cap, None, 0)
    if n < 0:
        raise LBError(n, L.lb_last_error(None).decode())
    out = np.zeros((n, 2), dtype=np.float32)
    _check(None, 0 if L.lb_stiffness_table(P_cap, out.ctypes.data, n) == n else LB_EINVAL)
    return out


def return_metric(series: np.ndarray, ring: int, d_pull: float, nx: int, ny: int) -> float:
    """Return = 1 - d_rec / d_pull (Eq. Rec): d_rec is the distance (minimum image) between the
    ring's centre of mass in the first and the last row of a readout series."""
    com = series[:, 8 + 4 * ring: 10 + 4 * ring]
    d = com[-1] - com[0]
    d[0] -= nx * np.round(d[0] / nx)
    d[1] -= ny * np.round(d[1] / ny)
    return 1.0 - float(np.hypot(d[0], d[1])) / d_pull


class Solver:
    """One lattice with its rings, driven through the C ABI."""

    def __init__(self, params: lb_params, stream=None):
        import torch
        self._torch = torch
        L = lib()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.params = params
        self.h = _H()
        rc = L.lb_create(ctypes.byref(params), ctypes.c_void_p(stream.cuda_stream),
                         ctypes.byref(self.h))
        if rc != LB_OK:
            raise LBError(rc, L.lb_last_error(None).decode())
        self.nx, self.ny = params.nx, params.ny
        self.n_rings = 0
        self.n_total = 0

    @staticmethod
    def from_workload(w: dict, **kw) -> "Solver":
        s = Solver(params_from_workload(w, **kw))
        s.init_fields(w.get("noise"))
        if w["rings"]:
            s.set_body(w["rings"])
        return s

    def close(self):
        if self.h:
            lib().lb_destroy(self.h)
            self.h = _H()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_fields(self, noise=None):
        if noise is not None:
            noise = np.ascontiguousarray(noise, dtype=np.float64)
            assert noise.shape == (2, self.ny, self.nx)
        _check(self.h, lib().lb_init_fields(self.h, None if noise is None else noise.ctypes.data))

    def set_body(self, rings):
        arr = (lb_ring * max(1, len(rings)))()
        xy = []
        for i, r in enumerate(rings):
            tp = r.get("trap") or {}
            arr[i] = lb_ring(n_nodes=len(r["X"]), pad_=0, k_spring=r["k_spring"],
                             eps_angle=r["eps_angle"], l_eq=r["l_eq"],
                             pull_force=r["pull_force"], pull_angle=r["pull_angle"],
                             trap_k=tp.get("k", 0.0), trap_dx=tp.get("dx", 0.0), trap_dy=tp.get("dy", 0.0),
                             trap_t_eq=tp.get("t_eq", 30.0), trap_pull=tp.get("pull", 100.0),
                             trap_width=tp.get("width", 30.0))
            xy.append(np.asarray(r["X"], dtype=np.float64))
        X = np.ascontiguousarray(np.concatenate(xy) if xy else np.zeros((0, 2)))
        _check(self.h, lib().lb_set_body(self.h, len(rings), arr, X.ctypes.data if X.size else None))
        self.n_rings = len(rings)
        self.n_total = X.shape[0]

    def step(self, n: int = 1):
        _check(self.h, lib().lb_step(self.h, int(n)))

    def sync(self):
        _check(self.h, lib().lb_sync(self.h))

    @property
    def t(self) -> int:
        return lib().lb_time(self.h)

    def readout(self, name: str, device: bool = True):
        """A field of the current state: torch FP32 [ny, nx] on the GPU (device=True) or numpy."""
        torch = self._torch
        fid = FIELDS[name] if name in FIELDS else LB_FIELD_POP0 + int(name[3:])
        if device:
            out = torch.empty((self.ny, self.nx), dtype=torch.float32, device="cuda")
            _check(self.h, lib().lb_readout(self.h, fid, ctypes.c_void_p(out.data_ptr()),
                                            out.numel() * 4, 1))
            return out
        out = np.empty((self.ny, self.nx), dtype=np.float32)
        _check(self.h, lib().lb_readout(self.h, fid, out.ctypes.data, out.nbytes, 0))
        return out

    def fields(self) -> dict:
        return {k: self.readout(k, device=False).astype(np.float64) for k in FIELDS}

    def nodes(self) -> np.ndarray:
        out = np.empty((self.n_total, 2), dtype=np.float64)
        _check(self.h, lib().lb_readout(self.h, LB_FIELD_NODES, out.ctypes.data if out.size else
                                        ctypes.c_void_p(1), out.nbytes, 0))
        return out

    def write_field(self, name: str, data):
        fid = FIELDS[name] if name in FIELDS else LB_FIELD_POP0 + int(name[3:])
        torch = self._torch
        if isinstance(data, torch.Tensor):
            assert data.dtype == torch.float32 and data.is_contiguous()
            _check(self.h, lib().lb_write_field(self.h, fid, ctypes.c_void_p(data.data_ptr()),
                                                data.numel() * 4, 1 if data.is_cuda else 0))
        else:
            a = np.ascontiguousarray(data, dtype=np.float32)
            _check(self.h, lib().lb_write_field(self.h, fid, a.ctypes.data, a.nbytes, 0))

    def series_latest(self, n: int = 1) -> np.ndarray:
        """The most recent n readout rows (lb_series_latest)."""
        L = lib()
        buf = np.zeros((max(n, 1), L.lb_series_row_len(self.h)))
        k = ctypes.c_int32(0)
        _check(self.h, L.lb_series_latest(self.h, buf.ctypes.data, int(n), ctypes.byref(k)))
        return buf[:k.value].copy()

    def series_latest_async(self, out, n: int = 1) -> int:
        """Enqueue the copy of the most recent n readout rows into `out` (a pinned host torch
        tensor or a numpy array of FP64 [n][row length]) behind the steps enqueued so far and
        return the number of rows it will hold (lb_series_latest_async); series_wait() blocks
        until they are there."""
        k = ctypes.c_int32(0)
        ptr = out.ctypes.data if isinstance(out, np.ndarray) else ctypes.c_void_p(out.data_ptr())
        _check(self.h, lib().lb_series_latest_async(self.h, ptr, int(n), ctypes.byref(k)))
        return k.value

    def series_wait(self):
        _check(self.h, lib().lb_series_wait(self.h))

    @property
    def state_bytes(self) -> int:
        return lib().lb_state_bytes(self.h)

    def read_state(self, out=None):
        """The stored state in one copy (lb_read_state): into `out` (a torch tensor on the host or
        the device, or a numpy array) or a new numpy uint8 array."""
        n = self.state_bytes
        if out is None:
            out = np.zeros(n, dtype=np.uint8)
        if isinstance(out, np.ndarray):
            assert out.nbytes == n and out.flags.c_contiguous
            _check(self.h, lib().lb_read_state(self.h, out.ctypes.data, n, 0))
        else:
            assert out.is_contiguous() and out.numel() * out.element_size() == n
            _check(self.h, lib().lb_read_state(self.h, ctypes.c_void_p(out.data_ptr()), n, 1 if out.is_cuda else 0))
        return out

    def write_state(self, src):
        """Replace the stored state in one copy (lb_write_state) from a numpy array or a torch
        tensor (pinned host or device memory must stay unchanged until the next sync)."""
        n = self.state_bytes
        if isinstance(src, np.ndarray):
            assert src.nbytes == n and src.flags.c_contiguous
            _check(self.h, lib().lb_write_state(self.h, src.ctypes.data, n, 0))
        else:
            assert src.is_contiguous() and src.numel() * src.element_size() == n
            _check(self.h, lib().lb_write_state(self.h, ctypes.c_void_p(src.data_ptr()), n, 1 if src.is_cuda else 0))

    def stage_state(self, src):
        """Upload a whole stored state into the handle's staging buffer on its copy stream
        (lb_stage_state), overlapping the steps queued meanwhile; commit_state makes it current."""
        n = self.state_bytes
        if isinstance(src, np.ndarray):
            assert src.nbytes == n and src.flags.c_contiguous
            _check(self.h, lib().lb_stage_state(self.h, src.ctypes.data, n, 0))
        else:
            assert src.is_contiguous() and src.numel() * src.element_size() == n
            _check(self.h, lib().lb_stage_state(self.h, ctypes.c_void_p(src.data_ptr()), n, 1 if src.is_cuda else 0))

    def commit_state(self):
        """Make the staged state current, in stream order (lb_commit_state)."""
        _check(self.h, lib().lb_commit_state(self.h))

    def series(self) -> np.ndarray:
        L = lib()
        rl = L.lb_series_row_len(self.h)
        cap = self.params.max_samples
        buf = np.zeros((cap, rl))
        n = ctypes.c_int32(0)
        _check(self.h, L.lb_series(self.h, buf.ctypes.data, cap, ctypes.byref(n)))
        return buf[:n.value].copy()

    def set_kernel(self, kernel: int):
        """LB_KERNEL_AUTO (the fastest measured), LB_KERNEL_TILE, LB_KERNEL_PAIR, LB_KERNEL_SWEEP or
        LB_KERNEL_STRIP."""
        _check(self.h, lib().lb_set_kernel(self.h, int(kernel)))

    @property
    def lattice_kernel(self) -> str:
        """The lattice kernel lb_step launches ("tile", "sweep", "pair" or "strip")."""
        k = lib().lb_lattice_kernel(self.h)
        return {LB_KERNEL_TILE: "tile", LB_KERNEL_SWEEP: "sweep", LB_KERNEL_PAIR: "pair",
                LB_KERNEL_STRIP: "strip"}[k]

    def set_node_tail(self, enable: bool):
        """Node step in the tail of the tile kernels (True, default: one launch per step) or in a
        separate node kernel (False); the two compute the same values bit for bit."""
        _check(self.h, lib().lb_set_node_tail(self.h, 1 if enable else 0))

    def timing(self, enable: bool):
        _check(self.h, lib().lb_timing(self.h, 1 if enable else 0))

    def kernel_time(self):
        f, n = ctypes.c_double(), ctypes.c_int64()
        g, m = ctypes.c_double(), ctypes.c_int64()
        _check(self.h, lib().lb_kernel_time(self.h, ctypes.byref(f), ctypes.byref(n),
                                            ctypes.byref(g), ctypes.byref(m)))
        return {"fused_ms": f.value, "fused_launches": n.value, "node_ms": g.value,
                "node_launches": m.value}

    def save(self, path: str):
        """Checkpoint the whole state to a file (lb_save)."""
        _check(self.h, lib().lb_save(self.h, os.fsencode(path)))

    def load(self, path: str):
        """Resume from a checkpoint of a solver with equal parameters and ring layout (lb_load)."""
        _check(self.h, lib().lb_load(self.h, os.fsencode(path)))

    @property
    def bytes_per_cell(self) -> float:
        return lib().lb_bytes_per_cell(self.h)

    @property
    def launches_per_step(self) -> int:
        return lib().lb_launches_per_step(self.h)


TILE_SHAPES = {0: (32, 16), 1: (32, 8), 2: (64, 8), 3: (16, 16), 4: "strip"}


class Batch:
    """Independent lattices advanced together by the persistent batched kernel (lb_batch_*).

    The solvers stay usable for readouts; they must not be stepped on their own while the batch
    exists, and must outlive it (the batch keeps references to them)."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        L = lib()
        arr = (_H * len(self.solvers))(*[s.h for s in self.solvers])
        self.b = _B()
        rc = L.lb_batch_create(arr, len(self.solvers), ctypes.byref(self.b))
        if rc != LB_OK:
            raise LBError(rc, "lb_batch_create failed")

    def _check(self, rc):
        if rc != LB_OK:
            raise LBError(rc, lib().lb_batch_last_error(self.b).decode())

    def close(self):
        if self.b:
            lib().lb_batch_destroy(self.b)
            self.b = _B()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        self._check(lib().lb_batch_step(self.b, int(n)))

    def sync(self):
        self._check(lib().lb_batch_sync(self.b))

    def set_shape(self, shape: int, inst: int = -1):
        self._check(lib().lb_batch_set_shape(self.b, int(inst), int(shape)))

    def shape(self, inst: int) -> int:
        return lib().lb_batch_shape(self.b, int(inst))

    def autotune(self, cache_path=None, steps: int = 5):
        self._check(lib().lb_batch_autotune(self.b, None if cache_path is None else
                                            os.fsencode(cache_path), int(steps)))

    def set_persistent(self, enable: bool):
        """One persistent cooperative kernel per chunk (True) or phase launches (False, default)."""
        self._check(lib().lb_batch_set_persistent(self.b, 1 if enable else 0))

    def set_wait_limit(self, wait_ms: float, extra_arrivals: int = 0):
        self._check(lib().lb_batch_set_wait_limit(self.b, float(wait_ms), int(extra_arrivals)))

    @property
    def grid(self) -> int:
        return lib().lb_batch_grid(self.b)

    @property
    def uses_graph(self) -> bool:
        return bool(lib().lb_batch_uses_graph(self.b))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class Net:
    """The learned stepper's U-Net (lb_net_*): BF16 NHWC input [B, H, W, 16] on the GPU."""

    N_IN = N_OUT = 16

    def __init__(self, batch: int, height: int, width: int, seed: int = 0, stream=None):
        import torch
        self._torch = torch
        self.stream = torch.cuda.current_stream() if stream is None else stream
        self.B, self.H, self.W = batch, height, width
        self.n = _N()
        rc = lib().lb_net_create(batch, height, width, seed, ctypes.c_void_p(self.stream.cuda_stream),
                                 ctypes.byref(self.n))
        if rc != LB_OK:
            raise LBError(rc, "lb_net_create failed")
        self.n_params = lib().lb_net_num_params(self.n)

    def _check(self, rc):
        if rc != LB_OK:
            raise LBError(rc, lib().lb_net_last_error(self.n).decode())

    def close(self):
        if self.n:
            lib().lb_net_destroy(self.n)
            self.n = _N()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        self._check(lib().lb_net_get_params(self.n, out.ctypes.data, self.n_params))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.n_params
        self._check(lib().lb_net_set_params(self.n, p.ctypes.data, self.n_params))

    def grads(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        self._check(lib().lb_net_get_grads(self.n, out.ctypes.data, self.n_params))
        return out

    def forward(self, x, out=None):
        """x: torch bfloat16 [B, H, W, 16] on the GPU; returns the FP32 output [B, H, W, 16]."""
        torch = self._torch
        assert x.dtype == torch.bfloat16 and x.is_contiguous() and tuple(x.shape) == (self.B, self.H, self.W, 16)
        if out is None:
            out = torch.empty((self.B, self.H, self.W, 16), dtype=torch.float32, device="cuda")
        self._check(lib().lb_net_forward(self.n, _ptr(x), _ptr(out)))
        return out

    def backward(self, g):
        torch = self._torch
        assert g.dtype == torch.float32 and g.is_contiguous()
        self._check(lib().lb_net_backward(self.n, _ptr(g)))

    ACTIVATIONS = [("x", 0, 16), ("e0a", 0, 32), ("cat0", 0, 96), ("p1", 1, 32), ("e1a", 1, 64),
                   ("cat1", 1, 160), ("p2", 2, 64), ("e2a", 2, 96), ("cat2", 2, 224), ("p3", 3, 96),
                   ("bta", 3, 128), ("btb", 3, 128), ("d2a", 2, 96), ("d2b", 2, 96), ("d1a", 1, 64),
                   ("d1b", 1, 64), ("d0a", 0, 32), ("d0b", 0, 32)]

    def activation(self, name: str) -> np.ndarray:
        """A stored BF16 activation of the last forward, as FP32 numpy [B, H/2^l, W/2^l, C]."""
        k = [a[0] for a in self.ACTIVATIONS].index(name)
        _, lev, c = self.ACTIVATIONS[k]
        shape = (self.B, self.H >> lev, self.W >> lev, c)
        raw = np.empty(shape, dtype=np.uint16)
        self._check(lib().lb_net_activation(self.n, k, raw.ctypes.data, raw.nbytes))
        return (raw.astype(np.uint32) << 16).view(np.float32)

    def mse(self, target, mask16) -> float:
        m = np.ascontiguousarray(mask16, dtype=np.float32)
        loss = ctypes.c_double()
        self._check(lib().lb_net_mse(self.n, _ptr(target), m.ctypes.data, ctypes.byref(loss)))
        return loss.value

    def adam(self, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
        self._check(lib().lb_net_adam(self.n, lr, beta1, beta2, eps))

    def train_step(self, x, target, mask16, lr: float) -> float:
        m = np.ascontiguousarray(mask16, dtype=np.float32)
        loss = ctypes.c_double()
        self._check(lib().lb_net_train_step(self.n, _ptr(x), _ptr(target), m.ctypes.data, lr,
                                             ctypes.byref(loss)))
        return loss.value


def conv3x3(x, w, bias=None, act=False, out_f32=True, ldy=None, yoff=0, y=None):
    """The single-layer forward kernel: x bf16 [B, H, W, Ci], w bf16 [9, Co, Ci]."""
    import torch
    B, H, W, Ci = x.shape
    Co = w.shape[1]
    if y is None:
        y = torch.empty((B, H, W, Co), dtype=torch.float32 if out_f32 else torch.bfloat16, device="cuda")
    ldy = Co if ldy is None else ldy
    rc = lib().lb_conv3x3(_ptr(x), Ci, 0, _ptr(w), _ptr(bias), None if out_f32 else _ptr(y),
                          _ptr(y) if out_f32 else None, ldy, yoff, B, H, W, Ci, Co, 1 if act else 0,
                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _check(None, rc)
    return y


def conv3x3_dgrad(gz, w):
    import torch
    B, H, W, Co = gz.shape
    Ci = w.shape[2]
    gx = torch.empty((B, H, W, Ci), dtype=torch.bfloat16, device="cuda")
    rc = lib().lb_conv3x3_dgrad(_ptr(gz), _ptr(w), _ptr(gx), B, H, W, Ci, Co,
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _check(None, rc)
    return gx


def conv3x3_wgrad(x, gz):
    import torch
    B, H, W, Ci = x.shape
    Co = gz.shape[3]
    gw = torch.empty((9, Co, Ci), dtype=torch.float32, device="cuda")
    gb = torch.empty((Co,), dtype=torch.float32, device="cuda")
    rc = lib().lb_conv3x3_wgrad(_ptr(x), _ptr(gz), _ptr(gw), _ptr(gb), B, H, W, Ci, Co,
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _check(None, rc)
    return gw, gb


def conv_kernel(kernel: int):
    """Convolution kernel of the network: 0 mma.sync, 1 tcgen05 (tensor-memory accumulators)."""
    _check(None, lib().lb_conv_kernel(int(kernel)))


def conv_status():
    _check(None, lib().lb_conv_status())
