"""Batched persistent form (lb_batch_*) on the GPU.

Each instance of a batch must compute exactly what lb_step computes for its handle: fields and
node positions bitwise equal, for every tile shape, with and without diffusion sub-steps and
across chunk (graph replay) boundaries; and a small batch of the 256-instance recipe's kind
must match the FP64 oracle at the FP32 step's tolerance.  The grid barrier's bounded wait must
end in LB_ETIMEOUT when its arrival count cannot be met.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2209_14889_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-5
FREST_TOL = 1e-4


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_14889_gb300 import lb
    return lb


def rel_l2(a, b):
    nb = max(np.linalg.norm(b), 1e-9 * np.sqrt(b.size))
    return np.linalg.norm(a - b) / nb


def _mixed(seed=11):
    """Five small instances: uneven sizes, one ragged, one with diffusion sub-steps, one with
    no ring."""
    ws = [
        W.small(64, 64, seed=seed, n_nodes=32, radius=6.0),
        W.small(50, 37, seed=seed + 1, n_nodes=20, radius=4.5, centre=(2.3, 35.6)),
        W.small(96, 80, seed=seed + 2, n_nodes=40, radius=8.0, Dp=0.6, diffusion_substeps=3),
        W.small(40, 26, seed=seed + 3, n_nodes=0),
        W.small(128, 48, seed=seed + 4, n_nodes=48, radius=7.0, Dp=0.45, diffusion_substeps=2,
                lambda_steps=120.0),
    ]
    return ws


def _solvers(lb, ws):
    return [lb.Solver.from_workload(w) for w in ws]


def _state(s):
    return dict(fields=s.fields(), X=s.nodes(), series=s.series())


def _reference(lb, ws, steps):
    out = []
    for w in ws:
        s = lb.Solver.from_workload(w)
        s.step(steps)
        s.sync()
        out.append(_state(s))
        s.close()
    return out


def _assert_bitwise(got, ref, series_exact_cols=True):
    for k in ref["fields"]:
        assert np.array_equal(got["fields"][k], ref["fields"][k]), k
    assert np.array_equal(got["X"], ref["X"])
    gs, rs = got["series"], ref["series"]
    assert gs.shape == rs.shape
    assert np.array_equal(gs[:, 0], rs[:, 0])
    # ring columns come from the node kernel: bitwise; lattice sums: order of the tile partials
    assert np.array_equal(gs[:, 6:], rs[:, 6:])
    np.testing.assert_allclose(gs[:, 1:6], rs[:, 1:6], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("persistent", [False, True], ids=["phase_launches", "persistent"])
@pytest.mark.parametrize("shape", [0, 1, 2, 3])
def test_batch_matches_single_handles_bitwise(shape, persistent):
    lb = _gpu()
    ws = _mixed()
    steps = 37                                  # 3 graph chunks of 10 + 7 direct steps
    ref = _reference(lb, ws, steps)
    ss = _solvers(lb, ws)
    b = lb.Batch(ss)
    b.set_persistent(persistent)
    b.set_shape(shape)
    assert all(b.shape(i) == shape for i in range(len(ws)))
    b.step(steps)
    b.sync()
    for s, r in zip(ss, ref):
        assert s.t == steps
        _assert_bitwise(_state(s), r)
    b.close()
    for s in ss:
        s.close()


def test_batch_strip_shape_matches_single_handles_bitwise():
    # the warp-strip step as a batch shape (the instances it applies to; the others keep tiles):
    # fields and nodes bitwise equal to the single handles; the shape is refused where it does
    # not apply and in the persistent mode
    lb = _gpu()
    ws = _mixed(seed=13)
    steps = 37
    ref = _reference(lb, ws, steps)
    ss = _solvers(lb, ws)
    b = lb.Batch(ss)
    ok = [w["nx"] >= 64 and w["nx"] % 2 == 0 and w["ny"] >= 32 for w in ws]
    assert any(ok) and not all(ok)
    with pytest.raises(lb.LBError):
        b.set_shape(4)                          # some instances are too small
    for i, good in enumerate(ok):
        b.set_shape(4 if good else 0, inst=i)
    with pytest.raises(lb.LBError):
        b.set_persistent(True)
    b.step(steps)
    b.sync()
    for s, r in zip(ss, ref):
        assert s.t == steps
        _assert_bitwise(_state(s), r)
    b.close()
    for s in ss:
        s.close()


def test_batch_mixed_shapes_graph_and_resume():
    lb = _gpu()
    ws = _mixed(seed=21)
    ref = _reference(lb, ws, 45)
    ss = _solvers(lb, ws)
    b = lb.Batch(ss)
    for i in range(len(ws)):
        b.set_shape(i % 4, inst=i)
    b.step(20)
    b.sync()
    assert b.uses_graph
    # phase launches: one CTA per lattice tile of every instance (tile shape i % 4)
    dims = {0: (32, 16), 1: (32, 8), 2: (64, 8), 3: (16, 16)}
    tiles = sum(-(-w["nx"] // dims[i % 4][0]) * -(-w["ny"] // dims[i % 4][1]) for i, w in enumerate(ws))
    assert b.grid == tiles
    b.step(25)                                  # continues from the device-side parity
    b.sync()
    for s, r in zip(ss, ref):
        _assert_bitwise(_state(s), r)
    b.close()
    # the handles stay valid after the batch: one more plain step each
    for s, w in zip(ss, ws):
        s.step(1)
        s.sync()
        assert s.t == 46
        s.close()


def test_diffusion_substeps_vs_oracle():
    lb = _gpu()
    w = W.small(72, 56, seed=5, n_nodes=28, radius=6.0, Dp=0.6, diffusion_substeps=3)
    steps = 60
    sim = O.Sim.from_workload(w)
    sim.step(steps, every=w["every"])
    ref = sim.fields()
    s = lb.Solver.from_workload(w)
    s.step(steps)
    s.sync()
    got = s.fields()
    errs = {k: rel_l2(got[k], ref[k]) for k in ref}
    assert max(errs.values()) <= FIELD_TOL, errs
    rs = np.array(sim.series)
    gs = s.series()
    fr_g, fr_r = gs[:, 6:8], rs[:, 6:8]
    assert rel_l2(fr_g, fr_r) <= FREST_TOL
    s.close()


def test_diffusion_beyond_bound_without_substeps_is_rejected():
    lb = _gpu()
    w = W.small(32, 32, n_nodes=0, Dp=0.6)
    with pytest.raises(lb.LBError) as e:
        lb.Solver.from_workload(w)
    assert e.value.code == lb.LB_EUNSTABLE


def test_small_recipe_batch_vs_oracle():
    # the 256-instance recipe's kind of draws (sizes, radii, node counts, angles, D_p with
    # sub-steps, lambda), at sizes the oracle finishes in seconds
    lb = _gpu()
    ws = W.cfg4(seed=9, n_instances=6, sides=(48, 64, 80), steps=120)
    steps = 120
    ss = _solvers(lb, ws)
    b = lb.Batch(ss)
    b.step(steps)
    b.sync()
    for s, w in zip(ss, ws):
        sim = O.Sim.from_workload(w)
        sim.step(steps, every=w["every"])
        ref = sim.fields()
        got = s.fields()
        errs = {k: rel_l2(got[k], ref[k]) for k in ref}
        assert max(errs.values()) <= FIELD_TOL, (w["nx"], w["Dp"], errs)
        rs, gs = np.array(sim.series), s.series()
        assert rel_l2(gs[:, 6:8], rs[:, 6:8]) <= FREST_TOL
        d = s.nodes() - sim.X
        d -= w["nx"] * np.round(d / w["nx"])
        assert np.abs(d).max() < 1e-5
    b.close()
    for s in ss:
        s.close()


def test_autotune_restores_state_and_writes_cache(tmp_path):
    lb = _gpu()
    ws = _mixed(seed=31)
    ref = _reference(lb, ws, 15)
    ss = _solvers(lb, ws)
    for s in ss:
        s.step(5)                               # tune from a state that is not the initial one
    b = lb.Batch(ss)
    path = str(tmp_path / "tune.json")
    b.autotune(path, steps=3)
    shapes = [b.shape(i) for i in range(len(ws))]
    assert all(0 <= x < 4 for x in shapes)
    cache = json.load(open(path))
    assert len(cache) == len({(w["nx"], w["ny"]) for w in ws})
    for s in ss:
        assert s.t == 5
    b.step(10)
    b.sync()
    for s, r in zip(ss, ref):
        _assert_bitwise(_state(s), r)
    b.close()
    # a second batch reads the cache and takes the same shapes without timing
    ss2 = _solvers(lb, ws)
    b2 = lb.Batch(ss2)
    b2.autotune(path, steps=3)
    assert [b2.shape(i) for i in range(len(ws))] == shapes
    b2.close()
    for s in ss + ss2:
        s.close()


def test_barrier_wait_runs_out_with_timeout_status():
    # an arrival count that can never be met: every barrier wait gives up after its limit
    # (0.2 s), the kernel returns and the host reads LB_ETIMEOUT; the context stays usable
    lb = _gpu()
    ws = _mixed(seed=41)[:2]
    ss = _solvers(lb, ws)
    b = lb.Batch(ss)
    b.set_persistent(True)                      # the grid barrier is the persistent kernel's
    b.set_wait_limit(200.0, extra_arrivals=1)
    b.step(1)
    with pytest.raises(lb.LBError) as e:
        b.sync()
    assert e.value.code == lb.LB_ETIMEOUT
    b.close()
    for s in ss:
        s.close()
    # the device still runs work afterwards
    s = lb.Solver.from_workload(ws[0])
    s.step(3)
    s.sync()
    assert s.t == 3
    s.close()


def test_batch_rejects_bad_handles():
    lb = _gpu()
    w = W.small(32, 32, n_nodes=0)
    a = lb.Solver.from_workload(w)
    c = lb.Solver.from_workload(w)
    c.step(1)                                   # other buffer parity
    with pytest.raises(lb.LBError):
        lb.Batch([a, c])
    with pytest.raises(lb.LBError):
        lb.Batch([a, a])
    p = lb.params_from_workload(w, precision=lb.LB_FP16_BF16)
    d = lb.Solver(p)
    d.init_fields(w["noise"])
    with pytest.raises(lb.LBError):
        lb.Batch([a, d])
    for s in (a, c, d):
        s.close()


def test_batch_with_walls_and_traps_matches_single_handles_bitwise():
    # the paper's protocol in a batch: walls in y, trapped rings dragged at different D_p
    lb = _gpu()
    trap = dict(k=0.05, dx=3.0, dy=0.5, t_eq=30, pull=60, width=30)
    ws = [W.make(64 + 16 * i, 48, rings=[W.ring(20, 4.0, (20.3 + i, 23.7), pull_force=0.0, trap=trap)],
                 seed=50 + i, walls_y=1, walls_x=i % 2, Dp=dp, steps=0) for i, dp in enumerate((0.001, 0.02, 0.2))]
    ws.append(W.small(64, 64, seed=53, n_nodes=24, radius=5.0))          # a periodic one beside them
    steps = 45
    ref = _reference(lb, ws, steps)
    ss = _solvers(lb, ws)
    b = lb.Batch(ss)
    b.step(steps)
    b.sync()
    for s, r in zip(ss, ref):
        _assert_bitwise(_state(s), r)
    b.close()
    for s in ss:
        s.close()


def test_scalar_model_batch_matches_single_handles_bitwise():
    # the scalar model in the batched kernel (its own instantiation), closed boxes with traps
    lb = _gpu()
    trap = dict(k=0.05, dx=3.0, dy=0.5, t_eq=30, pull=60, width=30)
    ws = [W.make(48 + 16 * i, 48, rings=[W.ring(20, 4.0, (20.3 + i, 23.7), pull_force=0.0, trap=trap)],
                 seed=60 + i, walls_y=1, walls_x=1, Dp=dp, steps=0, **W.scalar_physics())
          for i, dp in enumerate((0.001, 0.05, 0.25))]
    steps = 35
    ref = _reference(lb, ws, steps)
    ss = _solvers(lb, ws)
    b = lb.Batch(ss)
    for i in range(len(ws)):
        b.set_shape(i % 4, inst=i)
    b.step(steps)
    b.sync()
    for s, r in zip(ss, ref):
        _assert_bitwise(_state(s), r)
    b.close()
    for s in ss:
        s.close()
