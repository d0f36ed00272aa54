"""Seeded synthetic workloads (inputs only).

This module draws the random inputs and states the recipes of the benchmark workloads:
lattice size, physical parameters, the initial orientation noise and the positions of the
ring nodes.  It holds none of the method's arithmetic, so that the CUDA path and the FP64
oracle can both consume exactly the same arrays.  Every random number comes from numpy's
PCG64 generator seeded per workload.

Recipe of the default physics (lattice units, dx = dt = 1):
  * D2Q9 BGK, tau = 0.8, rho0 = 1, periodic in x and y, fluid at rest.
  * K^x = G0 (2, 1, 1, 1) for (K1111, K1122, K2222, K1212), G0 = 1e-3: the ratios of the
    paper's Table IV.
  * relaxation time lambda in steps (turned into eta_p by each consumer).
  * Beris-Edwards parameters of the paper's Table III: xi = 1.1, alpha = -0.9, beta = 1,
    kappa = 0.001, Gamma = 1.
  * P = P_eq (cos theta_d, sin theta_d) + noise, noise uniform in [-0.05, 0.05] per component.
  * sigma = 0.
  * rings: N nodes on a circle of radius r, node a at angle 2 pi a / N; l_eq = the initial
    chord; constant pull force split equally over the nodes.
"""
from __future__ import annotations

import math

import numpy as np

DEFAULT_PHYSICS = dict(tau=0.8, rho0=1.0, K=(2e-3, 1e-3, 1e-3, 1e-3), lambda_steps=50.0,
                       Dp=0.05, alpha=-0.9, beta=1.0, xi=1.1, Gamma=1.0, kappa=0.001,
                       P_cap=0.99, ericksen=1, director_angle=0.0)


def scalar_physics(C: float = 1.875e-3) -> dict:
    """Overrides for the scalar model (Eq. MaxDiff, Sec. II B): one modulus C written as the
    isotropic K^x (K1111 = K2222 = C, K1122 = 0, K1212 = C / 2; C defaults to C~11(k = 0) of the
    default K^x), no Ericksen force.  The oracle runs the same physics through the tensorial
    equations, whose C~ is then C times the identity."""
    return dict(K=(C, 0.0, C, C / 2), ericksen=0, model=1)


def ring(n_nodes: int, radius: float, centre, k_spring=0.1, eps_angle=0.01, pull_force=1e-3,
         pull_angle=0.0, phase=0.0, trap=None) -> dict:
    """A closed ring of n_nodes points on a circle (node a at angle phase + 2 pi a / N).
    trap: optional harmonic trap of Eq. Utrap, dict(k=k_max, dx=, dy=, t_eq=30, pull=100,
    width=30) (steps): it holds the ring at its initial centre of mass, drags it by (dx, dy)
    over `pull` steps after `t_eq` and lets go."""
    a = phase + 2.0 * np.pi * np.arange(n_nodes) / n_nodes
    X = np.stack([centre[0] + radius * np.cos(a), centre[1] + radius * np.sin(a)], axis=1)
    l_eq = float(np.hypot(*(X[1] - X[0])))
    return dict(X=X, k_spring=k_spring, eps_angle=eps_angle, l_eq=l_eq, pull_force=pull_force,
                pull_angle=pull_angle, radius=radius, centre=tuple(centre), trap=trap)


def make(nx: int, ny: int, rings=(), seed: int = 1, noise_amp: float = 0.05, steps: int = 100,
         every: int = 10, **physics) -> dict:
    """A workload: physics + seeded orientation noise [2, ny, nx] + rings."""
    w = dict(DEFAULT_PHYSICS)
    w.update(physics)
    w.update(nx=nx, ny=ny, seed=seed, steps=steps, every=every, rings=list(rings))
    rng = np.random.Generator(np.random.PCG64(seed))
    if noise_amp > 0:
        w["noise"] = rng.uniform(-noise_amp, noise_amp, size=(2, ny, nx))
    else:
        w["noise"] = None
    w["noise_amp"] = noise_amp
    return w


def cfg1(seed: int = 1) -> dict:
    """Plain method, 64x64 periodic; one ring of 32 nodes, radius 6, pulled along x with
    1e-3; relaxation 50 steps, D_p = 0.05; 2000 steps, restoring force every 10 steps."""
    return make(64, 64, rings=[ring(32, 6.0, (32.0, 32.0), pull_force=1e-3, pull_angle=0.0)],
                seed=seed, steps=2000, every=10, lambda_steps=50.0, Dp=0.05)


def cfg2(seed: int = 2) -> dict:
    """Plain method at scale, 1024x1024 periodic; one ring of 256 nodes, radius 24, pulled at
    30 degrees to the director (x) with 5e-4; relaxation 200 steps, D_p = 0.1; 20000 steps."""
    return make(1024, 1024,
                rings=[ring(256, 24.0, (512.0, 512.0), pull_force=5e-4, pull_angle=math.radians(30))],
                seed=seed, steps=20000, every=10, lambda_steps=200.0, Dp=0.1)


def cfg3(seed: int = 3, side: int = 4096, n_rings: int = 16) -> dict:
    """Precision-form workload: side x side periodic, n_rings rings of 128 nodes, radius 12,
    at seeded positions (centre separation >= 2r + 8, on the torus) with seeded pull angles in
    [0, 90] degrees, force 5e-4 each; relaxation 200 steps, D_p = 0.1; 10000 steps."""
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    r, sep = 12.0, 2 * 12.0 + 8.0
    centres = []
    while len(centres) < n_rings:
        c = rng.uniform(0, side, size=2)
        ok = True
        for d in centres:
            dx = abs(c[0] - d[0]); dx = min(dx, side - dx)
            dy = abs(c[1] - d[1]); dy = min(dy, side - dy)
            if math.hypot(dx, dy) < sep:
                ok = False
                break
        if ok:
            centres.append(c)
    angles = rng.uniform(0.0, math.pi / 2, size=n_rings)
    rings = [ring(128, r, tuple(c), pull_force=5e-4, pull_angle=float(a))
             for c, a in zip(centres, angles)]
    return make(side, side, rings=rings, seed=seed, steps=10000, every=10, lambda_steps=200.0,
                Dp=0.1)


def small(nx: int, ny: int, seed: int = 7, n_nodes: int = 24, radius: float = 5.0, centre=None,
          pull_angle: float = 0.3, steps: int = 50, **physics) -> dict:
    """Small parity case with an arbitrary (possibly ragged) lattice and one ring."""
    if centre is None:
        centre = (nx / 2 + 0.37, ny / 2 - 0.21)
    rings = [ring(n_nodes, radius, centre, pull_force=1e-3, pull_angle=pull_angle, phase=0.1)] \
        if n_nodes > 0 else []
    return make(nx, ny, rings=rings, seed=seed, steps=steps, every=10, **physics)


def cfg4(seed: int = 4, n_instances: int = 256, sides=(128, 192, 256, 384, 512),
         steps: int = 5000) -> list:
    """Batched workload: n_instances independent square periodic lattices, each with one ring.

    Per instance, drawn from one PCG64 stream: side uniform over `sides`; ring radius
    r ~ U[4, min(32, side/4 - 6)] (the upper bound keeps the ring with its supports within half
    the lattice); N = clamp(round(2 pi r / 0.78), 32, 256) nodes; pull 5e-4 at an angle
    U[0, 90] degrees; D_p log-uniform on [1e-3, 1], with ceil(D_p / 0.2) diffusion sub-steps
    when D_p > 0.2; relaxation time lambda ~ U[20, 500] steps; the ring centred at a uniform
    position; orientation noise from a per-instance seed.  The rest as in DEFAULT_PHYSICS.
    """
    rng = np.random.Generator(np.random.PCG64(seed + 4000))
    out = []
    for i in range(n_instances):
        side = int(sides[int(rng.integers(0, len(sides)))])
        r = float(rng.uniform(4.0, min(32.0, side / 4 - 6)))
        n_nodes = int(min(256, max(32, round(2 * math.pi * r / 0.78))))
        angle = float(rng.uniform(0.0, math.pi / 2))
        Dp = float(math.exp(rng.uniform(math.log(1e-3), math.log(1.0))))
        lam = float(rng.uniform(20.0, 500.0))
        centre = tuple(float(c) for c in rng.uniform(0.0, side, size=2))
        sub = int(math.ceil(Dp / 0.2)) if Dp > 0.2 else 0
        w = make(side, side, rings=[ring(n_nodes, r, centre, pull_force=5e-4, pull_angle=angle)],
                 seed=seed * 100000 + i, steps=steps, every=10, lambda_steps=lam, Dp=Dp,
                 diffusion_substeps=sub)
        out.append(w)
    return out


# ------------------------------------------------------------------------------------------
# The paper's own setup (App. C, Tables I-IV) in lattice units
# ------------------------------------------------------------------------------------------

# SI values of Tables I (lattice), II (droplet and protocol) and IV (viscoelastic stress; the
# Beris-Edwards parameters of Table III are already dimensionless and sit in DEFAULT_PHYSICS)
PAPER_SI = dict(dx=4e-8, dt=8e-6, rho=2e7, eta_s=1e-3, nx=250, ny=250, n_steps=187500,
                l_eq=2e-8, R=5e-7, k_spring=1e-5, eps_angle=1e-20, k_trap=1e-6, d_pull=4e-6, T_pull=0.2,
                C=0.01, eta_p=0.1, Dp=1e-13, K=(0.01, 0.005, 0.005, 0.005))


def lattice_units(si: dict = PAPER_SI) -> dict:
    """The paper's SI parameters in lattice units, with dx, dt and the solvent density as the units
    of length, time and mass density.  tau = 1/2 + 3 nu dt / dx^2 (Eq. BGK, c_s^2 = 1/3); a stress or
    modulus sigma [Pa] becomes sigma dt^2 / (rho dx^2), a viscosity eta [Pa s] eta dt / (rho dx^2), a
    diffusivity D [m^2/s] D dt / dx^2.  Reading for the two-dimensional model (the paper states its
    droplet constants in three-dimensional units): a lattice cell is dx deep, so a force [N] acts on
    a layer of cells and a stiffness k [N/m] becomes k dt^2 / (rho dx^3), a bending stiffness eps
    [N m] eps dt^2 / (rho dx^5)."""
    dx, dt, rho = si["dx"], si["dt"], si["rho"]
    stress = dt * dt / (rho * dx * dx)
    return dict(
        tau=0.5 + 3.0 * si["eta_s"] / rho * dt / (dx * dx),
        C=si["C"] * stress, K=tuple(k * stress for k in si["K"]),
        eta_p=si["eta_p"] * dt / (rho * dx * dx), Dp=si["Dp"] * dt / (dx * dx),
        R=si["R"] / dx, l_eq=si["l_eq"] / dx, d_pull=si["d_pull"] / dx, T_pull=si["T_pull"] / dt,
        k_spring=si["k_spring"] * dt * dt / (rho * dx ** 3), eps_angle=si["eps_angle"] * dt * dt / (rho * dx ** 5),
        k_trap=si["k_trap"] * dt * dt / (rho * dx ** 3), nx=si["nx"], ny=si["ny"], n_steps=si["n_steps"])


def paper_setup(model: str = "scalar", seed: int = 1, every: int = 100, **si_overrides) -> dict:
    """The paper's pulling experiment with its default parameters (App. C): a 250^2 closed box, the
    droplet (radius 0.5 um, nodes 20 nm apart) centred 2 um left of the box centre on its mid-line,
    held by the trap, dragged 4 um along x over 0.2 s after 30 steps of equilibration (sigmoid width
    30 steps) and left to recoil to 187 500 steps; Table IV's scalar modulus (model="scalar") or its
    K^x with the Beris-Edwards field of Table III (model="tensorial", director along x, no noise).
    si_overrides replace entries of PAPER_SI (e.g. Dp=1e-15, R=3.2e-7, T_pull=0.1)."""
    si = dict(PAPER_SI)
    si.update(si_overrides)
    lu = lattice_units(si)
    n_nodes = int(round(2.0 * math.pi * lu["R"] / lu["l_eq"]))
    x_mid, y_mid = (lu["nx"] - 1) / 2.0, (lu["ny"] - 1) / 2.0
    centre = (x_mid - 2e-6 / si["dx"], y_mid)
    trap = dict(k=lu["k_trap"], dx=lu["d_pull"], dy=0.0, t_eq=30, pull=float(round(lu["T_pull"])), width=30)
    rings = [ring(n_nodes, lu["R"], centre, k_spring=lu["k_spring"], eps_angle=lu["eps_angle"],
                  pull_force=0.0, trap=trap)]
    if model == "scalar":
        physics = scalar_physics(lu["C"])
    elif model == "tensorial":
        physics = dict(K=lu["K"])
    else:
        raise ValueError("model must be 'scalar' or 'tensorial'")
    physics.update(tau=lu["tau"], eta_p=lu["eta_p"], Dp=lu["Dp"], walls_x=1, walls_y=1)
    return make(lu["nx"], lu["ny"], rings=rings, seed=seed, noise_amp=0.0, steps=lu["n_steps"], every=every,
                **physics)


# ---------------------------------------------------------------------------------------
# Three-dimensional workloads (the D3Q19 form of Sec. IV's first extension)
# ---------------------------------------------------------------------------------------

# Recipe: D3Q19 BGK, tau = 0.8, rho0 = 1, periodic in x, y and z, fluid at rest; K^x = G0 (2, 1,
# 1, 1, 1/2) for (K1111, K1122, K2222, K1212, K2233), G0 = 1e-3 (the two-dimensional ratios, with
# K2233 inside the interval (0, K2222) where the transversely isotropic K^x is positive
# definite); eta_p and D_p given directly; the Beris-Edwards parameters of the two-dimensional
# recipe; P = P_eq d + noise with the director d along x and noise uniform in [-0.05, 0.05] per
# component; sigma = 0.
DEFAULT_PHYSICS_3D = dict(tau=0.8, rho0=1.0, K=(2e-3, 1e-3, 1e-3, 1e-3, 5e-4), eta_p=0.05, Dp=0.05,
                          alpha=-0.9, beta=1.0, xi=1.1, Gamma=1.0, kappa=0.001, P_cap=0.99, ericksen=1,
                          director=(1.0, 0.0, 0.0), n_quad=24, fext=None)


def make3d(nx: int, ny: int, nz: int, seed: int = 1, noise_amp: float = 0.05, steps: int = 100,
           every: int = 10, **physics) -> dict:
    """A three-dimensional workload: physics + seeded orientation noise [3, nz, ny, nx]."""
    w = dict(DEFAULT_PHYSICS_3D)
    w.update(physics)
    w.update(nx=nx, ny=ny, nz=nz, seed=seed, steps=steps, every=every, dim=3)
    rng = np.random.Generator(np.random.PCG64(seed))
    w["noise"] = rng.uniform(-noise_amp, noise_amp, size=(3, nz, ny, nx)) if noise_amp > 0 else None
    w["noise_amp"] = noise_amp
    return w


def cube3d(seed: int = 7) -> dict:
    """The measured three-dimensional workload: a 256^3 periodic box of the default physics
    (2 x 28 planes x 67 M cells x 4 B = 3.8 GB of state)."""
    return make3d(256, 256, 256, seed=seed, steps=100, every=10)
