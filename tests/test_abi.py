"""The C-ABI library builds, loads without a GPU and exports every symbol include/lb.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def libvlb():
    from paper_2209_14889_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(libvlb):
    names = declared("lb.h")
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(libvlb, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2209_14889_gb300 import lb
    L = lb.lib()
    for n in declared("lb.h"):
        assert hasattr(L, n)


def test_struct_layout_matches_header():
    # lb_params: 2 int32, 16 doubles, 8 int32 ; lb_ring: 2 int32 + 11 doubles
    from paper_2209_14889_gb300 import lb
    assert ctypes.sizeof(lb.lb_params) == 8 + 16 * 8 + 32
    assert ctypes.sizeof(lb.lb_ring) == 8 + 11 * 8


def test_create_without_gpu_fails_cleanly():
    # No compute call is made: with no device, lb_create must return an error code, not crash.
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2209_14889_gb300 import lb
    L = lb.lib()
    p = lb.lb_params(nx=16, ny=16, tau=0.8, rho0=1.0, K1111=2e-3, K1122=1e-3, K2222=1e-3,
                     K1212=1e-3, eta_p=0.1, lambda_steps=0.0, Dp=0.05, alpha=-0.9, beta=1.0,
                     xi=1.1, Gamma=1.0, kappa=1e-3, P_cap=0.99, director_angle=0.0, ericksen=1,
                     precision=0, readout_every=10, max_samples=16)
    h = ctypes.c_void_p()
    rc = L.lb_create(ctypes.byref(p), None, ctypes.byref(h))
    assert rc in (lb.LB_ECUDA, lb.LB_ENOMEM)
    assert not h.value


def test_transfer_entry_points_reject_null_arguments_without_gpu():
    # The staged upload and the asynchronous readout rows check their arguments before touching
    # the device: a null handle or a null buffer is LB_EINVAL, with no CUDA call made.
    from paper_2209_14889_gb300 import lb
    L = lb.lib()
    buf = (ctypes.c_double * 64)()
    k = ctypes.c_int32(-1)
    assert L.lb_stage_state(None, buf, 8, 0) == lb.LB_EINVAL
    assert L.lb_commit_state(None) == lb.LB_EINVAL
    assert L.lb_series_latest_async(None, buf, 1, ctypes.byref(k)) == lb.LB_EINVAL
    assert L.lb_series_wait(None) == lb.LB_EINVAL
    assert k.value == -1


def test_parameter_validation_without_gpu():
    from paper_2209_14889_gb300 import lb
    L = lb.lib()
    base = dict(nx=16, ny=16, tau=0.8, rho0=1.0, K1111=2e-3, K1122=1e-3, K2222=1e-3,
                K1212=1e-3, eta_p=0.1, lambda_steps=0.0, Dp=0.05, alpha=-0.9, beta=1.0, xi=1.1,
                Gamma=1.0, kappa=1e-3, P_cap=0.99, director_angle=0.0, ericksen=1, precision=0,
                readout_every=10, max_samples=16)
    for bad, code in [(dict(nx=4), lb.LB_EINVAL), (dict(tau=0.5), lb.LB_EINVAL),
                      (dict(Dp=0.3), lb.LB_EUNSTABLE), (dict(alpha=-1.5), lb.LB_EUNSTABLE),
                      (dict(precision=7), lb.LB_EINVAL), (dict(eta_p=0.0), lb.LB_EINVAL)]:
        kw = dict(base)
        kw.update(bad)
        h = ctypes.c_void_p()
        rc = L.lb_create(ctypes.byref(lb.lb_params(**kw)), None, ctypes.byref(h))
        assert rc == code, (bad, rc)
        assert L.lb_last_error(None)


def test_library_stiffness_table_matches_oracle():
    """The table the kernels interpolate (host code of the library, no GPU) against the oracle's
    independent Bessel functions and k(P) inversion (Eq. Pk, App. B)."""
    import numpy as np
    import oracle as O
    from paper_2209_14889_gb300 import lb
    tab = lb.stiffness_table(0.99).astype(np.float64)
    n = tab.shape[0] - 1
    qcap = 0.99 ** 2
    assert abs(tab[0, 0] - 0.5) < 1e-7 and abs(tab[0, 1] - 1.0 / 24) < 1e-8
    for i in list(range(1, n + 1, 97)) + [n]:
        q = qcap * i / n
        k = O.k_of_P(np.sqrt(q))
        I0 = O.bessel_i(0, k)
        a2 = O.bessel_i(2, k) / I0 / q
        a4 = O.bessel_i(4, k) / I0 / q ** 2
        assert abs(tab[i, 0] - a2) < 2e-7 * a2, i
        assert abs(tab[i, 1] - a4) < 2e-7 * a4, i


def test_batch_entry_points_validate_without_gpu():
    # argument checks come before any CUDA call
    from paper_2209_14889_gb300 import lb
    L = lb.lib()
    b = ctypes.c_void_p()
    assert L.lb_batch_create(None, 0, ctypes.byref(b)) == lb.LB_EINVAL
    assert not b.value
    arr = (ctypes.c_void_p * 1)(None)
    assert L.lb_batch_create(arr, 1, ctypes.byref(b)) == lb.LB_ESTATE
    assert L.lb_batch_step(None, 1) == lb.LB_EINVAL
    assert L.lb_batch_sync(None) == lb.LB_EINVAL
    assert L.lb_batch_set_shape(None, 0, 0) == lb.LB_EINVAL
    assert L.lb_batch_shape(None, 0) == -1
    assert L.lb_batch_autotune(None, None, 1) == lb.LB_EINVAL
    assert L.lb_batch_set_wait_limit(None, 1.0, 0) == lb.LB_EINVAL
    assert L.lb_batch_grid(None) == 0
    L.lb_batch_destroy(None)


# ---- the three-dimensional entry points (include/lb3d.h) --------------------------------------

def _declared3d():
    src = open(os.path.join(ROOT, "include", "lb3d.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lb3d_\w+)\s*\(", src)))


def test_every_3d_symbol_is_exported_and_bound(libvlb):
    from paper_2209_14889_gb300 import lb3d
    names = _declared3d()
    assert len(names) >= 12
    assert not [n for n in names if not hasattr(libvlb, n)]
    L = lb3d.lib()
    for n in names:
        assert getattr(L, n).argtypes is not None, n


def _params3d(**kw):
    from paper_2209_14889_gb300 import lb3d
    base = dict(nx=8, ny=8, nz=8, readout_every=10, tau=0.8, rho0=1.0, K1111=2e-3, K1122=1e-3,
                K2222=1e-3, K1212=1e-3, K2233=5e-4, eta_p=0.05, Dp=0.05, alpha=-0.9, beta=1.0, xi=1.1,
                Gamma=1.0, kappa=1e-3, P_cap=0.99, ericksen=1, max_samples=16)
    base.update(kw)
    return lb3d.lb3d_params(**base)


def test_3d_struct_layout_and_validation_without_gpu():
    # lb3d_params: 4 int32, 15 doubles, 3 doubles of f_ext, 3 of P_ref, 2 int32
    from paper_2209_14889_gb300 import lb, lb3d
    assert ctypes.sizeof(lb3d.lb3d_params) == 16 + 15 * 8 + 24 + 24 + 8
    L = lb3d.lib()
    for bad, code in [(dict(nx=2), lb.LB_EINVAL), (dict(tau=0.5), lb.LB_EINVAL), (dict(eta_p=0.0), lb.LB_EINVAL),
                      (dict(P_cap=1.0), lb.LB_EINVAL), (dict(readout_every=0), lb.LB_EINVAL),
                      (dict(Dp=0.2), lb.LB_EUNSTABLE), (dict(alpha=-1.5), lb.LB_EUNSTABLE),
                      (dict(kappa=0.2), lb.LB_EUNSTABLE)]:
        h = ctypes.c_void_p()
        assert L.lb3d_create(ctypes.byref(_params3d(**bad)), ctypes.byref(h)) == code, bad
        assert not h.value


def test_3d_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2209_14889_gb300 import lb, lb3d
    h = ctypes.c_void_p()
    rc = lb3d.lib().lb3d_create(ctypes.byref(_params3d()), ctypes.byref(h))
    assert rc in (lb.LB_ECUDA, lb.LB_ENOMEM) and not h.value


def test_3d_moment_table_matches_oracle_quadrature():
    # the host table the kernels interpolate (series / recursion of the Fisher moments) against
    # the oracle's numerical sphere quadrature, to FP32 rounding
    import numpy as np
    import oracle.o3d as O3
    from paper_2209_14889_gb300 import lb3d
    for cap in (0.9, 0.99):
        t = lb3d.moment_table(cap)
        assert t.shape == (8193, 2)
        for i in (0, 1, 7, 100, 4095, 7200, 8191, 8192):
            m = O3.orientation_moments(O3.k_of_P(cap * i / 8192), 48)
            assert abs(t[i, 0] - m[2]) < 3e-8 and abs(t[i, 1] - m[4]) < 3e-8, (cap, i)
        assert np.all(np.diff(t[:, 0]) >= 0) and np.all(np.diff(t[:, 1]) >= 0)
