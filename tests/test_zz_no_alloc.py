"""lb_readout_noalloc gives the same fields as lb_readout without allocating device memory.

Callers whose device memory is owned by another allocator, or who must not allocate after
their set-up phase, read rho and u through lb_readout_noalloc: it keeps its intermediate planes
in a scratch array that is part of the library image instead of a buffer created with
cudaMalloc.  These tests call it through the C ABI and compare it with lb_readout: both run the
same moment launch on the same state, so the values agree bit for bit.  The file is named to
run last, so that a failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest

from paper_2209_14889_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = [("drho", 0), ("ux", 1), ("uy", 2), ("Px", 6), ("Py", 7)]


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_14889_gb300 import lb
    f = lb.lib().lb_readout_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32]
    return torch, lb, f


def test_noalloc_readout_matches_readout_twice():
    torch, lb, f = _setup()
    s = lb.Solver.from_workload(W.small(64, 48, steps=0))
    try:
        for call in range(2):                       # two calls in a row, state advanced between
            s.step(7)
            got = {}
            for name, fid in FIELDS:                # the no-allocation call first, on each state
                host = np.empty((48, 64), dtype=np.float32)
                assert f(s.h, fid, host.ctypes.data, host.nbytes, 0) == 0, lb.lib().lb_last_error(s.h)
                dev = torch.empty((48, 64), dtype=torch.float32, device="cuda")
                assert f(s.h, fid, dev.data_ptr(), dev.numel() * 4, 1) == 0, lb.lib().lb_last_error(s.h)
                got[name] = (host, dev.cpu().numpy())
            for name, _ in FIELDS:
                ref = s.readout(name, device=False)
                for g in got[name]:
                    assert np.array_equal(g, ref), (call, name)
    finally:
        s.close()


def test_noalloc_readout_allocates_nothing():
    # On a fresh 1024 x 1024 solver the first readout of u through lb_readout_noalloc leaves the
    # device's free memory unchanged, while lb_readout's first call takes its 12 MiB buffer.
    torch, lb, f = _setup()
    warm = lb.Solver.from_workload(W.make(32, 32, rings=[], noise_amp=0.0))   # the device's first call
    out = np.empty((32, 32), dtype=np.float32)
    assert f(warm.h, 1, out.ctypes.data, out.nbytes, 0) == 0
    warm.close()
    s = lb.Solver.from_workload(W.make(1024, 1024, rings=[], noise_amp=0.05))
    try:
        s.step(3)
        host = np.empty((1024, 1024), dtype=np.float32)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for fid in (0, 1, 2):
            assert f(s.h, fid, host.ctypes.data, host.nbytes, 0) == 0, lb.lib().lb_last_error(s.h)
        free1 = torch.cuda.mem_get_info()[0]
        assert free0 - free1 < (1 << 20), (free0, free1)
        uy = host.copy()
        ref = s.readout("uy", device=False)                      # lb_readout allocates here
        free2 = torch.cuda.mem_get_info()[0]
        assert free1 - free2 >= 12 << 20, (free1, free2)        # the measurement sees a buffer
        assert np.array_equal(uy, ref)
    finally:
        s.close()


def test_noalloc_rejects_oversized_lattice_and_other_fields():
    torch, lb, f = _setup()
    s = lb.Solver.from_workload(W.make(2048, 1024, rings=[], noise_amp=0.0))
    try:
        out = np.empty((1024, 2048), dtype=np.float32)
        rc = f(s.h, 1, out.ctypes.data, out.nbytes, 0)
        assert rc == lb.LB_EINVAL
        assert b"limit" in lb.lib().lb_last_error(s.h)
    finally:
        s.close()
    s = lb.Solver.from_workload(W.make(32, 32, rings=[], noise_amp=0.0))
    try:
        out = np.empty((32, 32), dtype=np.float32)
        assert f(s.h, 3, out.ctypes.data, out.nbytes, 0) == lb.LB_EINVAL      # SXX: no scratch
    finally:
        s.close()
