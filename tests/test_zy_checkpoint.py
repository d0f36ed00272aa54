"""Checkpoint and resume through the C ABI (lb_save / lb_load): a run saved part-way, loaded into
another solver and continued is bitwise the uninterrupted run (fields, node positions, readout
series, step counter); a file of another parameter set or ring layout, a missing file and a
truncated one are refused and leave the solver as it was."""
import numpy as np
import pytest

from paper_2209_14889_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TRAP = dict(k=0.05, dx=4.0, dy=1.0, t_eq=30, pull=120, width=30)
FLUID_FIELDS = ["drho", "ux", "uy", "sxx", "syy", "sxy"]


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_14889_gb300 import lb
    return lb


def _case(name, lb):
    two_rings = [W.ring(20, 4.0, (20.3, 20.1), pull_force=1e-3, pull_angle=0.4),
                 W.ring(24, 5.0, (44.2, 30.5), pull_force=1e-3, pull_angle=2.0)]
    if name == "periodic_two_rings":
        return W.make(64, 48, rings=two_rings, seed=3), lb.LB_FP32
    if name == "closed_box_trap":
        return W.make(64, 48, rings=[W.ring(20, 4.0, (24.3, 23.9), pull_force=0.0, trap=TRAP)], seed=8,
                      walls_x=1, walls_y=1), lb.LB_FP32
    if name == "precision_form":
        return W.make(64, 64, rings=[W.ring(32, 6.0, (32.0, 32.0), pull_force=1e-3)], seed=1), lb.LB_FP16_BF16
    if name == "scalar_model":
        return W.make(64, 48, rings=two_rings, seed=5, **W.scalar_physics()), lb.LB_FP32
    raise KeyError(name)


def _state(s, fields):
    return {k: s.readout(k, device=False) for k in fields}, s.nodes(), s.series(), s.t


@pytest.mark.parametrize("name", ["periodic_two_rings", "closed_box_trap", "precision_form", "scalar_model"])
def test_resume_is_bitwise_the_uninterrupted_run(name, tmp_path):
    lb = _gpu()
    w, prec = _case(name, lb)
    fields = FLUID_FIELDS if name == "scalar_model" else FLUID_FIELDS + ["Px", "Py"]
    path = str(tmp_path / "run.ckpt")
    a = lb.Solver.from_workload(w, precision=prec)
    a.step(37)
    a.save(path)
    a.step(45)
    ref = _state(a, fields)
    a.close()
    b = lb.Solver.from_workload(w, precision=prec)
    b.step(5)                                   # another state, replaced by the load
    b.load(path)
    assert b.t == 37
    b.step(45)
    got = _state(b, fields)
    b.close()
    for k in fields:
        assert np.array_equal(got[0][k], ref[0][k]), k
    assert np.array_equal(got[1], ref[1])
    assert got[2].shape == ref[2].shape and np.array_equal(got[2], ref[2])
    assert got[3] == ref[3] == 82


def test_load_refuses_other_parameters_layout_and_bad_files(tmp_path):
    lb = _gpu()
    w, prec = _case("periodic_two_rings", lb)
    path = str(tmp_path / "run.ckpt")
    a = lb.Solver.from_workload(w)
    a.step(12)
    a.save(path)
    a.close()
    raw = open(path, "rb").read()
    short = str(tmp_path / "short.ckpt")
    open(short, "wb").write(raw[: len(raw) // 2])
    longer = str(tmp_path / "long.ckpt")
    open(longer, "wb").write(raw + b"x")
    r0, r1 = w["rings"][0], w["rings"][1]
    others = [dict(w, tau=0.9), dict(w, rings=w["rings"][:1]), dict(w, rings=w["rings"][::-1]),
              # the same layout (rings and node counts) with other ring physics
              dict(w, rings=[dict(r0, k_spring=2 * r0["k_spring"]), r1]),
              dict(w, rings=[r0, dict(r1, pull_force=2 * r1["pull_force"])]),
              dict(w, rings=[r0, dict(r1, eps_angle=0.5 * r1["eps_angle"])])]
    for o in others:
        s = lb.Solver.from_workload(o)
        with pytest.raises(lb.LBError):
            s.load(path)
        s.close()
    s = lb.Solver.from_workload(w)
    s.step(3)
    before = _state(s, FLUID_FIELDS)
    for bad in (short, longer, str(tmp_path / "missing.ckpt")):
        with pytest.raises(lb.LBError):
            s.load(bad)
    after = _state(s, FLUID_FIELDS)
    for k in FLUID_FIELDS:
        assert np.array_equal(before[0][k], after[0][k]), k
    assert np.array_equal(before[1], after[1]) and after[3] == 3
    s.load(path)                                # the good file still loads
    assert s.t == 12
    s.close()
