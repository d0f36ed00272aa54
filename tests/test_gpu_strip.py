"""The warp-strip lattice kernel against the tile kernel and the FP64 oracle, through the C ABI.

The strip kernel evaluates every per-cell expression of the step on the same operands as the
tile kernel (stencil neighbours from registers and warp shuffles instead of shared memory,
spreading scattered per strip in the gather's ring and node order), so the state (all 14
planes), the node positions and the ring columns of the readout series agree bit for bit; the
lattice sums of the series differ only in the order of their FP64 partial sums.  Cases cover
ragged strips and chunks, rings across the periodic seam, several rings and more than 32, the
trap, the precision form, the scalar model, diffusion sub-steps and a lattice with several
chunks and spreading sub-chunks per warp.
"""
import numpy as np
import pytest

import oracle as O
from paper_2209_14889_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STATE = ["drho", "ux", "uy", "sxx", "syy", "sxy", "Px", "Py"] + ["pop%d" % n for n in range(9)]


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_14889_gb300 import lb
    return lb


def _cases():
    trap = dict(k=0.02, dx=12.0, dy=3.0, t_eq=5, pull=20, width=6)
    return {
        "one_ring": (W.make(96, 64, rings=[W.ring(24, 5.0, (40.3, 30.7), pull_angle=0.5)], seed=2), 0),
        "ragged_seam": (W.make(100, 70, rings=[W.ring(30, 6.0, (1.2, 68.9), pull_angle=2.2)], seed=4), 0),
        "precision_form": (W.make(128, 96, rings=[W.ring(32, 6.0, (60.0, 40.0)),
                                                  W.ring(24, 5.0, (20.5, 80.2), pull_angle=1.0)], seed=5), 1),
        "scalar_model": (W.make(120, 64, rings=[W.ring(28, 5.5, (50.0, 33.0))], seed=6,
                                **W.scalar_physics()), 0),
        "trap": (W.make(96, 64, rings=[W.ring(24, 5.0, (48.0, 32.0), pull_force=0.0, trap=trap)], seed=8), 0),
        "substeps": (W.small(96, 80, n_nodes=40, radius=8.0, Dp=0.6, diffusion_substeps=3), 0),
        "forty_rings": (W.cfg3(seed=9, side=512, n_rings=40), 0),
        "tall_chunks": (W.make(512, 448, rings=[W.ring(160, 24.0, (250.0, 200.0), pull_angle=0.7),
                                                W.ring(64, 10.0, (20.0, 430.0))], seed=10), 0),
    }


def _run(lb, w, prec, kernel, steps):
    s = lb.Solver.from_workload(w, precision=prec)
    s.set_kernel(kernel)
    s.step(steps)
    s.sync()
    out = dict(state={k: s.readout(k, device=False) for k in STATE}, X=s.nodes(), series=s.series(),
               launches=s.launches_per_step, t=s.t)
    s.close()
    return out


@pytest.mark.parametrize("case", list(_cases()))
def test_strip_equals_tile_bitwise(case):
    lb = _gpu()
    w, prec = _cases()[case]
    steps = 23
    a = _run(lb, w, prec, lb.LB_KERNEL_STRIP, steps)
    b = _run(lb, w, prec, lb.LB_KERNEL_TILE, steps)
    for k in STATE:
        assert np.array_equal(a["state"][k], b["state"][k]), k
    assert np.array_equal(a["X"], b["X"])
    gs, rs = a["series"], b["series"]
    assert gs.shape == rs.shape and gs.shape[0] == 3
    assert np.array_equal(gs[:, 0], rs[:, 0])
    assert np.array_equal(gs[:, 6:], rs[:, 6:])         # ring columns: from the node kernel
    scale = np.abs(rs[:, 1:6]).max(axis=0) + 1e-30
    assert np.all(np.abs(gs[:, 1:6] - rs[:, 1:6]) <= 1e-11 * scale + 1e-13)
    dsub = w.get("diffusion_substeps", 0)
    assert a["launches"] == 2 + (dsub + (dsub & 1) if dsub else 0)
    assert a["t"] == steps


def test_strip_vs_oracle_cfg1_200_steps():
    # the 64^2 workload through the strip kernel against the FP64 oracle (fields <= 1e-5,
    # restoring force <= 1e-4, nodes <= 1e-5 cells)
    lb = _gpu()
    w = W.cfg1()
    steps = 200
    sim = O.Sim.from_workload(w)
    sim.step(steps, every=10)
    ref = sim.fields()
    s = lb.Solver.from_workload(w)
    s.set_kernel(lb.LB_KERNEL_STRIP)
    s.step(steps)
    s.sync()
    got = s.fields()
    X = s.nodes()
    ser = s.series()
    s.close()
    for k in ref:
        e = np.linalg.norm(got[k] - ref[k]) / max(np.linalg.norm(ref[k]), 1e-9 * np.sqrt(ref[k].size))
        assert e <= 1e-5, (k, e)
    rs = np.array(sim.series)
    fr_g, fr_r = ser[:, 6:8], rs[:, 6:8]
    assert np.linalg.norm(fr_g - fr_r) / np.linalg.norm(fr_r) <= 1e-4
    d = X - sim.X
    d -= 64 * np.round(d / 64)
    assert np.abs(d).max() < 1e-5


def test_strip_rejects_walls_and_small_lattices():
    lb = _gpu()
    for w in (W.make(96, 64, rings=[], walls_y=1), W.make(48, 64, rings=[]), W.make(96, 24, rings=[])):
        s = lb.Solver.from_workload(w)
        with pytest.raises(lb.LBError):
            s.set_kernel(lb.LB_KERNEL_STRIP)
        s.close()


def test_auto_takes_strip_where_it_is_faster():
    # LB_KERNEL_AUTO: the strip kernel from 4096^2 (four waves of its CTAs), the tile kernel below
    # and with walls
    lb = _gpu()
    for w, want in ((W.make(4096, 4096, rings=[], noise_amp=0.0), "strip"),
                    (W.make(1024, 1024, rings=[], noise_amp=0.0), "tile"),
                    (W.make(4096, 4096, rings=[], noise_amp=0.0, walls_y=1), "tile")):
        s = lb.Solver.from_workload(w)
        assert s.lattice_kernel == want, (w["nx"], w.get("walls_y"), s.lattice_kernel)
        s.set_kernel(lb.LB_KERNEL_TILE)
        assert s.lattice_kernel == "tile"
        s.close()
