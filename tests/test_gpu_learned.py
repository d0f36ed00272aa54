"""The learned stepper (lb_learned_*): packing, the accept path, the fallback path, and what a
briefly trained network gains over the plain solver, measured against the plain FP32 step on the
same GPU."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_14889_gb300 import lb, learned as LR
    return torch, lb, LR


def _wl(LR, seed=5, side=64):
    return LR.learned_workloads(seed, 1, side=side)[0]


def test_pack_channels_and_body_indicator():
    torch, lb, LR = _gpu()
    w = _wl(LR)
    s = lb.Solver.from_workload(w)
    s.step(20)
    raw = torch.empty((w["ny"], w["nx"], 8), dtype=torch.float32, device="cuda")
    LR.pack(s, LR.IDENTITY_NORM, raw=raw)
    torch.cuda.synchronize()
    r = raw.cpu().numpy()
    f = s.fields()
    for c, name in [(0, "ux"), (1, "uy"), (2, "sxx"), (3, "sxy"), (4, "syy")]:
        assert np.array_equal(r[..., c], f[name].astype(np.float32)), name
    # dP = P - P_ref: a constant offset from the readout of P
    for c, name in [(5, "Px"), (6, "Py")]:
        off = f[name] - r[..., c]
        assert np.ptp(off) < 1e-6, name
    # the IB kernel is a partition of unity: the indicator sums to the node count
    n = len(w["rings"][0]["X"])
    assert abs(r[..., 7].sum() - n) < 1e-3 * n
    x = torch.empty((w["ny"], w["nx"], 16), dtype=torch.bfloat16, device="cuda")
    LR.pack(s, LR.IDENTITY_NORM, x=x)
    torch.cuda.synchronize()
    xv = x.float().cpu().numpy()
    assert np.all(xv[..., 8:] == 0)
    assert np.allclose(xv[..., 2], r[..., 2], rtol=2 ** -8, atol=0)
    s.close()


def test_fallback_reproduces_plain_solver_bitwise():
    # residual bounds no network meets: every call runs 16 plain steps
    torch, lb, LR = _gpu()
    w = _wl(LR, seed=6)
    plain = lb.Solver.from_workload(w)
    plain.step(5 * 16)
    plain.sync()
    s = lb.Solver.from_workload(w)
    net = lb.Net(1, w["ny"], w["nx"], seed=1)
    st = LR.Stepper(s, net, LR.IDENTITY_NORM, eps_momentum=1e-30, eps_tendency=1e-30)
    fb = st.step(5)
    s.sync()
    assert fb == 5 and st.stats()["accepted"] == 0
    assert s.t == plain.t == 80
    a, b = s.fields(), plain.fields()
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(s.nodes(), plain.nodes())
    assert np.array_equal(s.series(), plain.series())
    st.close()
    for o in (s, plain, net):
        o.close()


def test_untrained_network_trips_the_residual_check():
    torch, lb, LR = _gpu()
    w = _wl(LR, seed=7)
    s = lb.Solver.from_workload(w)
    s.step(16)
    net = lb.Net(1, w["ny"], w["nx"], seed=2)       # random weights: garbage output
    raw0 = torch.empty((w["ny"], w["nx"], 8), dtype=torch.float32, device="cuda")
    LR.pack(s, LR.IDENTITY_NORM, raw=raw0)
    norm = LR.fit_norm([raw0.cpu().numpy()], [raw0.cpu().numpy() * 1.01])
    st = LR.Stepper(s, net, norm, eps_momentum=0.25, eps_tendency=0.5)
    fb = st.step(4)
    s.sync()
    assert fb == 4
    stt = st.stats()
    assert stt["r_momentum"] > 0.25 or stt["r_tendency"] > 0.5
    st.close()
    s.close()
    net.close()


def test_accept_path_writes_the_network_state():
    # a network whose output is zero (all weights and biases zero) predicts "no change": with
    # bounds it meets (residuals are then exactly 1) the call is accepted, sigma and P return to
    # their values at t, the velocity to u(t) (moments of the rebuilt populations), rho to
    # rho(t+1), and the step counter and nodes advance by 16
    torch, lb, LR = _gpu()
    w = _wl(LR, seed=8)
    s = lb.Solver.from_workload(w)
    s.step(16)
    s.sync()
    f0 = s.fields()
    X0 = s.nodes()
    net = lb.Net(1, w["ny"], w["nx"], seed=3)
    net.set_params(np.zeros(net.n_params, dtype=np.float32))
    st = LR.Stepper(s, net, LR.IDENTITY_NORM, eps_momentum=1.5, eps_tendency=1.5)
    fb = st.step(1)
    s.sync()
    assert fb == 0 and st.stats()["accepted"] == 1
    assert s.t == 32
    f1 = s.fields()
    for k in ("sxx", "syy", "sxy"):
        assert np.array_equal(f1[k], f0[k]), k
    for k in ("Px", "Py"):
        assert np.abs(f1[k] - f0[k]).max() < 1e-6, k
    # readout u carries the Guo half force F / (2 rho) on top of the populations' momentum
    for k in ("ux", "uy"):
        assert np.abs(f1[k] - f0[k]).max() < 1e-5, k
    d = s.nodes() - X0
    assert np.abs(d).max() > 0 and np.abs(d).max() < 1.0
    st.close()
    s.close()
    net.close()


def test_trained_network_gain_against_plain_solver():
    """Train briefly on seeded trajectories of the batched recipe's physics (64^2, generated by the
    batched kernel, to keep the test short), then run 32 learned calls (512 steps) on a held-out
    seed against the plain FP32 run on the same GPU.  Asserted: the restoring force stays within
    1 % of the plain run (the bound the residual check is calibrated for), and the time is
    accounted for: with calls accepted the stepper must not be slower than the network passes
    it replaces plain steps with; with none accepted (every call falls back to the plain steps)
    it is slower than the plain run by at least the network passes it made, a measured loss."""
    torch, lb, LR = _gpu()
    side = 64
    data = LR.Dataset(LR.learned_workloads(11, 32, side=side), pairs_per_traj=3, batch=32)
    net = lb.Net(8, side, side, seed=1)
    held = list(range(0, data.n, 12))                 # a fixed subset of the pairs
    val0 = LR.evaluate(net, data, held)
    net, losses = LR.train(data, batch=8, seconds=25.0, lr=5e-4, seed=1, net=net)
    val1 = LR.evaluate(net, data, held)
    k = max(1, len(losses) // 10)
    print("training: %d steps, loss %.3f -> %.3f (running means), fixed subset %.3f -> %.3f"
          % (len(losses), np.mean(losses[:k]), np.mean(losses[-k:]), val0, val1))
    assert val1 < val0
    inf = LR.inference_net(net, side, side)
    # the time of one network pass at this size (the cost an accepted call pays instead of 16 steps)
    x = torch.zeros((1, side, side, 16), dtype=torch.bfloat16, device="cuda")
    for _ in range(3):
        inf.forward(x)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        inf.forward(x)
    e1.record()
    torch.cuda.synchronize()
    ms_net = e0.elapsed_time(e1) / 10
    # residual bounds fixed on a validation trajectory, then one held-out trajectory
    eps, acc_val, err_val = LR.calibrate(inf, data.norm, LR.learned_workloads(98, 1, side=side)[0], calls=32)
    w = LR.learned_workloads(99, 1, side=side)[0]
    fr_p, ms_p, _ = LR.run(w, calls=32)
    fr_l, ms_l, stt = LR.run(w, inf, data.norm, calls=32, eps=eps)
    err = float(np.linalg.norm(fr_l - fr_p) / np.linalg.norm(fr_p))
    acc = stt["accepted"]
    print("learned stepper: bounds %s (validation: %d accepted, error %.2e); held-out: accepted %d/32, "
          "restoring-force error vs plain %.3e, plain %.2f ms, learned %.2f ms (speed ratio %.3f), "
          "network pass %.3f ms" % (eps, acc_val, err_val, acc, err, ms_p, ms_l, ms_p / ms_l, ms_net))
    assert stt["calls"] == 32
    assert err <= 1e-2
    if acc == 0:
        # every call ran its network pass and then the 16 plain steps: a loss of at least the passes
        assert ms_l >= ms_p + 0.5 * 32 * ms_net, (ms_l, ms_p, ms_net)
    else:
        # accepted calls replaced 16 plain steps each by a network pass and a check step
        per_step = ms_p / (32 * 16)
        assert ms_l <= ms_p + 32 * ms_net - acc * 14 * per_step + 0.5 * ms_p, (ms_l, ms_p, ms_net, acc)
