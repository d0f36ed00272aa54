"""The three-dimensional CUDA path (lb3d.cu, through the C ABI of include/lb3d.h) against the FP64
oracle (oracle/vlb3d_oracle.c).

Small lattices with ragged CTA tails run whole against the oracle (fields within 1e-5 relative L2,
as for the two-dimensional path: FP32 arithmetic over a few tens of steps); the measured 256^3 box
is checked on sampled patches, each advanced one step by the oracle from the GPU's own state (one
step reads at most four cells away, so the core of a 16^3 patch is exact under the patch's own
periodic wrap), and by its conservation laws.
"""
import numpy as np
import pytest

import oracle.o3d as O3
from paper_2209_14889_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ("drho", "ux", "uy", "uz", "sxx", "syy", "szz", "syz", "sxz", "sxy", "Px", "Py", "Pz")


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_14889_gb300 import lb3d
    return lb3d


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-9 * np.sqrt(b.size))


def _cases():
    return {
        "ragged": (W.make3d(40, 18, 11, seed=3), 24),
        "no_ericksen": (W.make3d(36, 12, 9, seed=4, ericksen=0), 24),
        "oblique_director": (W.make3d(24, 20, 10, seed=5, director=(0.48, 0.6, 0.64)), 24),
        "body_force": (W.make3d(33, 9, 7, seed=6, fext=(2e-5, -1e-5, 3e-5)), 24),
        "strong_anisotropy": (W.make3d(20, 16, 12, seed=8, K=(4e-3, 5e-4, 1e-3, 8e-4, 3e-4), alpha=-0.95,
                                       Dp=0.02), 24),
        "minimum_box": (W.make3d(3, 3, 3, seed=9), 12),
    }


@pytest.mark.parametrize("case", list(_cases()))
def test_3d_step_vs_oracle(case):
    lb3d = _gpu()
    w, steps = _cases()[case]
    s = lb3d.Solver3D.from_workload(w)
    s.step(steps)
    s.sync()
    got = s.fields()
    pops = s.populations()
    ser = s.series()
    assert s.t == steps and s.launches_per_step == (4 if w["ericksen"] else 3)
    s.close()
    sim = O3.Sim3.from_workload(w)
    sim.step(steps, every=w["every"])
    ref = sim.fields()
    for k in FIELDS:
        e = _rel(got[k], ref[k])
        assert e <= 1e-5, (case, k, e)
    _, wq = O3.lattice()
    hp = pops.astype(np.float64) + wq[:, None, None, None] * w["rho0"]
    assert np.abs(hp - sim.h).max() <= 1e-6 * (1 + np.abs(sim.h).max())
    rs = np.array(sim.series)
    assert ser.shape == rs.shape
    assert np.array_equal(ser[:, 0], rs[:, 0])
    N = w["nx"] * w["ny"] * w["nz"]
    # mass, momentum, force sums: FP32 per-cell values (rounding ~1e-7 of values below 0.1)
    # summed in FP64
    assert np.abs(ser[:, 1:] - rs[:, 1:]).max() <= 1e-6 * N


def test_3d_conserves_mass_and_adds_the_body_force():
    lb3d = _gpu()
    f = (1e-5, 2e-5, -3e-5)
    w = W.make3d(48, 40, 20, seed=11, fext=f, every=1)
    s = lb3d.Solver3D.from_workload(w)
    s.step(30)
    s.sync()
    ser = s.series()
    s.close()
    N = 48 * 40 * 20
    # mass: every collision conserves it up to FP32 rounding of the shifted populations
    assert np.abs(ser[:, 1]).max() < 1e-3
    # bare momentum grows by N f per step (div sigma^p and div sigma^E sum to zero)
    for t in range(1, 30):
        assert np.abs(ser[t, 2:5] - ser[0, 2:5] - t * N * np.array(f)).max() < 1e-3 * t * N * 3e-5
    assert np.abs(ser[:, 5:8] - N * np.array(f)).max() < 1e-2 * N * 3e-5


def _patch(a, c, r):
    """a[..., z, y, x] periodic patch of half-width r around c = (z, y, x)."""
    idx = [np.arange(ci - r, ci + r) % n for ci, n in zip(c, a.shape[-3:])]
    return a[..., idx[0][:, None, None], idx[1][None, :, None], idx[2][None, None, :]]


def test_3d_full_size_sampled_patches_vs_oracle():
    # the measured 256^3 box: after 20 GPU steps, three 16^3 patches of the GPU state are advanced
    # one step by the oracle; the 8^3 core of each equals the GPU's next state
    lb3d = _gpu()
    w = W.cube3d()
    s = lb3d.Solver3D.from_workload(w)
    s.step(20)
    s.sync()
    names = ["pop%d" % n for n in range(19)]
    state = {}
    for n in range(19):
        state[names[n]] = s.readout(lb3d.FIELD_POP0 + n)
    for k in ("sxx", "syy", "szz", "syz", "sxz", "sxy", "Px", "Py", "Pz"):
        state[k] = s.readout(k)
    s.step(1)
    s.sync()
    nxt = {k: s.readout(k) for k in ("sxx", "syy", "szz", "syz", "sxz", "sxy", "Px", "Py", "Pz")}
    nxt_pop = np.stack([s.readout(lb3d.FIELD_POP0 + n) for n in range(19)])
    ser = s.series()
    s.close()
    assert np.isfinite(ser).all()
    _, wq = O3.lattice()
    r = 8
    for c in ((0, 0, 0), (131, 77, 250), (255, 128, 3)):
        h = np.stack([_patch(state[names[n]], c, r) for n in range(19)]).astype(np.float64)
        h += wq[:, None, None, None] * w["rho0"]
        sig = np.stack([_patch(state[k], c, r) for k in ("sxx", "syy", "szz", "syz", "sxz", "sxy")]).astype(np.float64)
        P = np.stack([_patch(state[k], c, r) for k in ("Px", "Py", "Pz")]).astype(np.float64)
        p = O3.params_from_workload(dict(w, nx=2 * r, ny=2 * r, nz=2 * r))
        sim = O3.Sim3(p, np.ascontiguousarray(h), np.ascontiguousarray(sig), np.ascontiguousarray(P))
        sim.step(1)
        core = (slice(4, 12),) * 3
        for ci, k in enumerate(("sxx", "syy", "szz", "syz", "sxz", "sxy")):
            g = _patch(nxt[k], c, r)[core].astype(np.float64)
            o = sim.sigma[ci][core]
            assert np.abs(g - o).max() <= 1e-5 * np.abs(o).max() + 1e-9, (c, k)
        for ci, k in enumerate(("Px", "Py", "Pz")):
            g = _patch(nxt[k], c, r)[core].astype(np.float64)
            assert np.abs(g - sim.P[ci][core]).max() <= 2e-6, (c, k)
        hp = np.stack([_patch(nxt_pop[n], c, r)[core] for n in range(19)]).astype(np.float64)
        hp += wq[:, None, None, None] * w["rho0"]
        assert np.abs(hp - sim.h[(slice(None),) + core]).max() <= 2e-6, c


def test_3d_entry_points_device_readout_series_wrap_timing_and_zero_P():
    # lb3d_readout into device memory equals the host copy; the series keeps the last
    # max_samples rows in order; timing counts every step; P_init = NULL starts from P = 0
    lb3d = _gpu()
    import torch
    w = W.make3d(20, 12, 8, seed=21, every=2)
    p = lb3d.params_from_workload(w, max_samples=3)
    s = lb3d.Solver3D(p)
    Pref = lb3d.reference_polarization(w)
    P = np.broadcast_to(Pref[:, None, None, None], (3, 8, 12, 20)).copy() + w["noise"]
    s.init_fields(P)
    s.timing(True)
    s.step(11)
    ms, n = s.kernel_time()
    assert n == 11 and ms > 0
    s.timing(False)
    ser = s.series()
    assert ser.shape == (3, 8) and list(ser[:, 0]) == [6.0, 8.0, 10.0]
    for name in ("ux", "Pz", "sxy"):
        dev = torch.empty(8 * 12 * 20, dtype=torch.float32, device="cuda")
        s.readout_device(name, dev.data_ptr(), dev.numel())
        torch.cuda.synchronize()
        assert np.array_equal(dev.cpu().numpy().reshape(8, 12, 20), s.readout(name)), name
    # a restart without P: fluid at rest with P = 0 stays at rest (every force and source is zero)
    s.init_fields(None)
    s.step(5)
    s.sync()
    f = s.fields()
    for k in ("drho", "ux", "uy", "uz", "sxx", "sxy", "Px", "Py", "Pz"):
        assert np.abs(f[k]).max() == 0.0, k
    assert s.t == 5
    s.close()


def test_3d_nonfinite_state_is_reported_and_cleared():
    # a NaN in the initial P reaches the readout sums of step 0: lb3d_sync reports
    # LB_ENONFINITE once and clears the flag (nothing on the device faults: the table lookup
    # clamps a NaN |P|)
    lb3d = _gpu()
    from paper_2209_14889_gb300 import lb
    w = W.make3d(16, 8, 8, seed=22)
    s = lb3d.Solver3D(lb3d.params_from_workload(w))
    P = np.broadcast_to(lb3d.reference_polarization(w)[:, None, None, None], (3, 8, 8, 16)).copy()
    P[1, 4, 3, 7] = np.nan
    s.init_fields(P)
    s.step(2)
    with pytest.raises(lb3d.LB3DError) as e:
        s.sync()
    assert e.value.code == lb.LB_ENONFINITE
    s.sync()                     # cleared
    s.close()
