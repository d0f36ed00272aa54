"""The seeded workload recipes: reproducible, and within the solver's host-side rules."""
import json
import math
import os

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


# ------------------------------------------------------------------------------------------
# The paper's own setup (App. C, Tables I-IV) in lattice units
# ------------------------------------------------------------------------------------------

_GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_paper_si_values_are_the_printed_ones():
    # the recipe's SI constants, typed separately, against the tables as stored from the paper
    t1, t2, t4, si = _GOLD["table_I"], _GOLD["table_II"], _GOLD["table_IV"], W.PAPER_SI
    pairs = [(si["dx"], t1["dx_m"]), (si["dt"], t1["dt_s"]), (si["rho"], t1["rho_s_kg_m3"]),
             (si["eta_s"], t1["eta_s_Pa_s"]), (si["nx"], t1["nx"]), (si["ny"], t1["ny"]),
             (si["n_steps"], t1["n_steps"]), (si["l_eq"], t2["l_eq_m"]), (si["R"], t2["R_m"]),
             (si["k_spring"], t2["k_spring_N_m"]), (si["eps_angle"], t2["eps_angle_N_m"]),
             (si["k_trap"], t2["k_trap_N_m"]), (si["d_pull"], t2["d_pull_m"]), (si["T_pull"], t2["T_pull_s"]),
             (si["C"], t4["C_Pa"]), (si["eta_p"], t4["eta_p_Pa_s"]), (si["Dp"], t4["Dp_m2_s"]),
             (si["K"], (t4["K1111_Pa"], t4["K1122_Pa"], t4["K2222_Pa"], t4["K1212_Pa"]))]
    for a, b in pairs:
        assert a == b, (a, b)


def test_paper_setup_in_lattice_units():
    # Table I's tau follows from its own viscosity, density, dx and dt (c_s^2 = 1/3); the droplet of
    # Table II is a ring of radius 12.5 cells with ~157 nodes half a cell apart; the pull covers 100
    # cells in 25 000 steps, and Table I's 187 500 steps are 1.5 s
    lu = W.lattice_units()
    assert abs(lu["tau"] - _GOLD["table_I"]["tau"]) < 1e-12
    assert abs(lu["R"] - 12.5) < 1e-12 and abs(lu["l_eq"] - 0.5) < 1e-12
    assert abs(lu["d_pull"] - 100.0) < 1e-9 and abs(lu["T_pull"] - 25000.0) < 1e-6
    assert abs(lu["n_steps"] * W.PAPER_SI["dt"] - 1.5) < 1e-12
    # a modulus of 1 Pa is 2e-3 in these units (dt^2 / (rho dx^2)); viscosities and diffusivities
    # keep their ratios: the relaxation time eta_p / C is Table IV's 10 s in steps
    assert abs(lu["C"] - 2e-5) < 1e-18 and abs(lu["eta_p"] / lu["C"] - 10.0 / W.PAPER_SI["dt"]) < 1e-3
    assert abs(lu["Dp"] - 1e-13 * 8e-6 / 16e-16) < 1e-15
    w = W.paper_setup("scalar")
    r = w["rings"][0]
    assert len(r["X"]) == 157 and abs(r["l_eq"] - 0.5) < 1e-3
    assert r["centre"] == (74.5, 124.5)                         # x = -2 um, y = 0 in the paper's box
    assert r["trap"]["dx"] == 100.0 and r["trap"]["pull"] == 25000.0 and r["trap"]["t_eq"] == 30
    assert w["walls_x"] == 1 and w["walls_y"] == 1 and w["steps"] == 187500 and w["tau"] == lu["tau"]
    # the ring stays 5 cells from the walls over the whole pull
    assert r["centre"][0] - 12.5 > 5 and r["centre"][0] + 100 + 12.5 < 250 - 6
    t = W.paper_setup("tensorial", Dp=1e-15, R=3.2e-7)
    assert t["K"] == lu["K"] and len(t["rings"][0]["X"]) == round(2 * math.pi * 8.0 / 0.5)
    assert abs(t["Dp"] - 5e-6) < 1e-18
