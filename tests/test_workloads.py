"""The seeded workload recipes: reproducible, and within the solver's host-side rules."""
import math

import numpy as np

from paper_2209_14889_gb300 import workloads as W


def test_batched_recipe_draws():
    ws = W.cfg4()
    assert len(ws) == 256
    assert {w["nx"] for w in ws} == {128, 192, 256, 384, 512}
    cells = sum(w["nx"] * w["ny"] for w in ws)
    assert 20e6 < cells < 40e6
    for w in ws:
        (r,) = w["rings"]
        n = len(r["X"])
        assert 4.0 <= r["radius"] <= min(32.0, w["nx"] / 4 - 6)
        assert n == min(256, max(32, round(2 * math.pi * r["radius"] / 0.78)))
        assert 0.0 <= r["pull_angle"] <= math.pi / 2 and r["pull_force"] == 5e-4
        assert 1e-3 <= w["Dp"] <= 1.0 and 20.0 <= w["lambda_steps"] <= 500.0
        s = w["diffusion_substeps"]
        assert s == (math.ceil(w["Dp"] / 0.2) if w["Dp"] > 0.2 else 0)
        # Heun bound of the (sub-)stepped diffusion and the ring-fit rule of lb_set_body
        assert 8 * w["Dp"] / max(s, 1) <= 2.0
        ext = np.ptp(r["X"], axis=0)
        assert 2 * (math.ceil(ext.max()) + 8) <= w["nx"]
    # D_p spans the log-uniform range and some instances need sub-steps
    assert min(w["Dp"] for w in ws) < 3e-3 and max(w["Dp"] for w in ws) > 0.5
    assert sum(w["diffusion_substeps"] > 0 for w in ws) > 30


def test_recipes_are_reproducible():
    a, b = W.cfg4(n_instances=4), W.cfg4(n_instances=4)
    for x, y in zip(a, b):
        assert x["nx"] == y["nx"] and x["Dp"] == y["Dp"]
        assert np.array_equal(x["noise"], y["noise"])
        assert np.array_equal(x["rings"][0]["X"], y["rings"][0]["X"])
    c = W.cfg1()
    assert np.array_equal(c["noise"], W.cfg1()["noise"])


def test_return_metric_of_eq_rec():
    # Return = 1 - d_rec / d_pull from the first and last centre of mass of a readout series;
    # d_rec is taken as a minimum image on the periodic lattice
    from paper_2209_14889_gb300 import lb
    rows = np.zeros((3, 14))
    rows[:, 8:10] = [[10.0, 20.0], [30.0, 20.0], [13.0, 24.0]]     # ring 0: back to 5 cells off
    rows[:, 12:14] = [[1.0, 5.0], [50.0, 5.0], [63.0, 5.0]]        # ring 1: 2 cells across the seam
    assert abs(lb.return_metric(rows, 0, 20.0, 64, 64) - (1 - 5.0 / 20.0)) < 1e-15
    assert abs(lb.return_metric(rows, 1, 40.0, 64, 64) - (1 - 2.0 / 40.0)) < 1e-15


def test_scalar_physics_is_the_isotropic_stiffness():
    p = W.scalar_physics(2e-3)
    K1111, K1122, K2222, K1212 = p["K"]
    assert K2222 == K1111 and K1122 == 0.0 and K1212 == K1111 / 2
    assert p["ericksen"] == 0 and p["model"] == 1
    # Delta K = K1111 - K2222 and X = K1111 - 2 K1122 - 4 K1212 + K2222 vanish: C~ = C I (App. B)
    assert K1111 - K2222 == 0.0 and K1111 - 2 * K1122 - 4 * K1212 + K2222 == 0.0
