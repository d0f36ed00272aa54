"""Throughput of the fused viscoelastic IB-LB step on GB300 (one JSON line on rank 0).

Workload: the 1024 x 1024 periodic lattice with one 256-node ring of radius 24 pulled at 30
degrees to the director with 5e-4, D_p = 0.1, relaxation time 200 steps (Tables III-IV
ratios, synthetic seeded input).  One bench step = lb_step(10): ten LB time steps, i.e. one
readout period (restoring force, mass, momentum, total force recorded once).  Every rank runs
its own independent lattice: the lattice would shard by domain decomposition (one halo exchange
per step) and a batch by instances, but every call here runs on one GPU, so N ranks are
replicas (weak scaling, no collective).

value     MLUPS = cells x LB steps / device time, inputs resident in HBM, L2 flushed (256 MB
          write) between timed steps, each timed step bracketed by CUDA events.
roofline  fused lattice kernel (the node step runs in its tail; --separate-nodes runs it as its
          own kernel instead): algorithmic bytes (112 B/cell: 14 FP32 fields read + written)
          x cells / mean launch duration (CUDA events around each launch in a second pass over
          the same steps), against the measured HBM copy bandwidth.
e2e       the same metric through the C ABI with host buffers: per step the whole stored state is
          uploaded from pinned host memory in one copy, ten steps run, and the newest readout row
          is copied back; the next step's upload runs on a copy stream while the current step
          computes (lb_stage_state / lb_commit_state) and the row comes back while the next step
          runs (lb_series_latest_async / lb_series_wait).  serial_value: the same with the upload
          in line (lb_write_state) and a synchronous row read (lb_series_latest).
cpu_baseline         the FP64 oracle on one host core, one LB step of the 1024 x 1024 workload;
cpu_baseline_openmp  the same oracle source with OpenMP on all host cores (bitwise the same).
forms     the 4096^2 sixteen-ring workload in FP32, in the FP16/BF16 storage form and with the
          scalar model (state 0.9-1.9 GB: the clean HBM roofline; the warp-strip kernel); the
          batched form (256 lattices); the protocol form (Return against D_p, radius and pulling
          time in 250^2 closed boxes, scalar model, lattice-unit parameters); the anisotropy form
          (Return, deflection and rotation against alpha and theta0, tensorial model); the
          paper's own setup (App. C parameters, 187 500 steps: Return against D_p and radius);
          the learned form (a 16-step U-Net stepper with residual checks).
--impl reference   the FP64 CPU oracle on the host cores, on a bounded sample (512 x 512 with
          the same physics and ring), one LB time step per bench step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS of fused viscoelastic LB step + % HBM roofline; restoring-force err vs FP64"
LB_STEPS_PER_STEP = 10
WORKLOAD = ("1024x1024 periodic D2Q9, tau 0.8; one ring of 256 nodes, radius 24, pulled with "
            "5e-4 at 30 deg to the director; D_p 0.1, relaxation 200 steps; FP32 state")


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), \
        int(os.environ.get("WORLD_SIZE", 1))


def max_over_ranks(value: float, world: int, device: str = "cuda") -> float:
    """The largest value over the ranks (the slowest rank's time sets the whole job's), or the
    value itself on one rank.  device: where the process group's backend reduces (cuda for NCCL,
    cpu for gloo)."""
    if world <= 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


KERNEL_SOURCES = ["lb_fused.cu", "lb_tile.cuh", "lb_cell.cuh", "lb_vec.cuh", "lb_internal.h", "lb_node.cuh"]
STRIP_SOURCES = ["lb_strip.cu", "lb_strip.cuh", "lb_cell.cuh", "lb_vec.cuh", "lb_internal.h"]
LB3D_SOURCES = ["lb3d.cu"]


def kernel_source_sha1(sources=KERNEL_SOURCES):
    """SHA-1 over the sources of a lattice kernel (the counters in profiles/ are valid only for
    the source they were taken on)."""
    h = hashlib.sha1()
    for f in sources:
        h.update(open(os.path.join(ROOT, "paper_2209_14889_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def profile_values(name, sources):
    """key: value lines of a committed ncu summary, or {} when the kernel's sources changed
    since its counters were taken."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return {}
    info = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            info[k.strip()] = v.strip()
    return info if info.get("kernel_source_sha1") == kernel_source_sha1(sources) else {}


# Instruction issue of a GB300: 152 SMs x 4 schedulers x one warp instruction per cycle at the SM
# clock (the nominal unit counts; the clock is the median sampled under load, else the maximum).
def issue_roofline(warp_inst_per_launch, launch_s, sm_mhz):
    if not warp_inst_per_launch or not launch_s:
        return None
    peak = 152 * 4 * sm_mhz * 1e6
    achieved = warp_inst_per_launch / launch_s
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "T warp-instr/s",
            "frac": achieved / peak, "warp_instructions_per_launch": warp_inst_per_launch,
            "peak_from": "152 SMs x 4 schedulers x 1 warp instruction/cycle x %.0f MHz" % sm_mhz}


def ncu_traffic():
    """DRAM bytes per launch of the fused kernel from the committed ncu summary, or None when
    the kernel source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "fused_step_1024x1024.txt")
    if not os.path.exists(path):
        return None
    info = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            info[k.strip()] = v.strip()
    sha = kernel_source_sha1()
    if info.get("kernel_source_sha1") != sha or "dram_bytes_per_launch" not in info:
        return None
    return float(info["dram_bytes_per_launch"])


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = "/tmp/vlb_clocks_%d.csv" % os.getpid()

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            # the timed region starts once sampling is live (first line written), within 5 s
            t0 = time.time()
            while time.time() - t0 < 5.0 and self.proc.poll() is None:
                if os.path.getsize(self.path) > 0:
                    break
                time.sleep(0.02)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def frest_error_check():
    """Restoring-force error of the GPU path vs the FP64 oracle on the 64 x 64 workload for 200
    steps (20 readouts): relative L2 over the series."""
    import numpy as np

    import oracle as O
    from paper_2209_14889_gb300 import lb, workloads as W
    w = W.cfg1()
    s = lb.Solver.from_workload(w)
    s.step(200)
    s.sync()
    g = s.series()[:, 6:8]
    s.close()
    sim = O.Sim.from_workload(w)
    sim.step(200, every=10)
    r = np.array(sim.series)[:, 6:8]
    return float(np.linalg.norm(g - r) / np.linalg.norm(r))


def run_reference(args, rank, world):
    """FP64 oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import numpy as np

    import oracle as O
    from paper_2209_14889_gb300 import workloads as W
    w = W.make(512, 512, rings=[W.ring(256, 24.0, (256.0, 256.0), pull_force=5e-4,
                                       pull_angle=math.radians(30))],
               seed=2, lambda_steps=200.0, Dp=0.1)
    sim = O.Sim.from_workload(w)
    cells = 512 * 512
    for _ in range(args.warmup):
        sim.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sim.step(1, every=10)
    dt = time.perf_counter() - t0
    v = cells * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "512x512 lattice, same physics and ring, "
                       "one LB time step per bench step", "parallelism": "replicas"},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                             "sample": "512x512, 1 LB step per bench step, %d steps" % args.steps},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measure_forms(args, lb, W, torch):
    """The 4096^2 workload with 16 rings (128 nodes, radius 12, seeded positions and pull angles)
    in the FP32 and the FP16/BF16 storage forms and with the scalar model (one modulus, no P
    field) in FP32 (state 0.94-1.9 GB, larger than L2, so no flush), and the precision form's
    restoring-force error against the FP32 step (256^2, 2000 steps)."""
    import numpy as np
    peaks, _ = measured_peaks()
    out = {"workload": "4096x4096 periodic, 16 rings of 128 nodes (radius 12, seeded), pull 5e-4 "
                       "at seeded angles in [0, 90] deg, D_p 0.1, relaxation 200 steps"}
    w = W.cfg3()
    cells = w["nx"] * w["ny"]
    steps = max(3, min(args.steps, 10))
    ws = dict(w, **W.scalar_physics())
    for name, prec, wk in [("fp32", lb.LB_FP32, w), ("fp16_bf16", lb.LB_FP16_BF16, w),
                           ("scalar_fp32", lb.LB_FP32, ws)]:
        s = lb.Solver.from_workload(wk, precision=prec)
        stream = torch.cuda.current_stream()
        for _ in range(2):
            s.step(LB_STEPS_PER_STEP)
        s.sync()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        torch.cuda.synchronize()
        for k in range(steps):
            ev[k][0].record(stream)
            s.step(LB_STEPS_PER_STEP)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        s.timing(True)
        for k in range(steps):
            s.step(LB_STEPS_PER_STEP)
        kt = s.kernel_time()
        s.timing(False)
        fused_s = kt["fused_ms"] * 1e-3 / max(kt["fused_launches"], 1)
        gbs = s.bytes_per_cell * cells / fused_s / 1e9
        prof = profile_values("strip_step_4096x4096_counters.txt", STRIP_SOURCES)
        inst = float(prof["warp_inst_per_launch_" + name]) if ("warp_inst_per_launch_" + name) in prof else None
        out[name] = {"value": cells * LB_STEPS_PER_STEP * steps / (ms * 1e-3) / 1e6, "unit": "MLUPS",
                     "kernel": s.lattice_kernel,
                     "issue_roofline": issue_roofline(inst, fused_s, args.sm_mhz) if s.lattice_kernel == "strip" else None,
                     "traffic": float(prof["dram_bytes_per_launch_" + name])
                     if s.lattice_kernel == "strip" and ("dram_bytes_per_launch_" + name) in prof else None,
                     "bytes_per_cell_step": s.bytes_per_cell, "fused_mean_us": fused_s * 1e6,
                     "node_mean_us": kt["node_ms"] * 1e3 / max(kt["node_launches"], 1),
                     "roofline_frac": gbs / peaks["hbm_gbs"], "achieved_gbs": gbs, "steps": steps}
        s.sync()
        s.close()
    # restoring-force error of the precision form against the FP32 step on this GPU
    wr = W.make(256, 256, rings=[W.ring(128, 12.0, (128.3, 127.6), pull_force=5e-4,
                                        pull_angle=math.radians(35))],
                seed=3, steps=2000, every=10, lambda_steps=200.0, Dp=0.1)
    series = {}
    for name, prec in [("fp32", lb.LB_FP32), ("fp16_bf16", lb.LB_FP16_BF16)]:
        s = lb.Solver.from_workload(wr, precision=prec)
        s.step(2000)
        s.sync()
        series[name] = s.series()[:, 6:8]
        s.close()
    d = series["fp16_bf16"] - series["fp32"]
    out["fp16_bf16"]["frest_err_vs_fp32"] = {
        "value": float(np.linalg.norm(d) / np.linalg.norm(series["fp32"])),
        "workload": "256x256, one ring of 128 nodes, 2000 steps, relative L2 over 200 readouts"}
    return out


def _protocol_batch(lb, W, torch, runs, n_steps, d_pull=40.0):
    """One batch of 250 x 250 closed boxes (walls on all four sides, App. C) with the scalar model:
    per run (radius, nodes, pull steps, D_p, seed) a ring held by the harmonic trap, dragged by
    d_pull cells along x after 30 steps of equilibration and released, relaxation 2000 steps.
    Returns the Return (Eq. Rec) of each run at n_steps and the batch's device time (ms)."""
    ws = [W.make(250, 250, rings=[W.ring(nodes, radius, (60.3, 125.2), pull_force=0.0,
                                         trap=dict(k=0.02, dx=d_pull, dy=0.0, t_eq=30, pull=pull, width=30))],
                 seed=seed, walls_y=1, walls_x=1, Dp=dp, lambda_steps=2000.0, every=100, steps=n_steps,
                 **W.scalar_physics())
          for radius, nodes, pull, dp, seed in runs]
    ss = [lb.Solver.from_workload(w, max_samples=n_steps // 100 + 2) for w in ws]
    b = lb.Batch(ss)
    try:
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(torch.cuda.current_stream())
        b.step(n_steps)
        e1.record(torch.cuda.current_stream())
        b.sync()
        torch.cuda.synchronize()
        rets = [lb.return_metric(s_.series(), 0, d_pull, 250, 250) for s_ in ss]
        return rets, e0.elapsed_time(e1)
    finally:
        b.close()
        for s_ in ss:
            s_.close()


# The paper's own setup (App. C, Tables I-IV; workloads.paper_setup) swept as in Sec. III B.  The
# paper plots the Return against D_p and against the droplet radius without printing the values
# it used; the sweeps are taken around its defaults (D_p = 1e-13 m^2/s, R = 0.5 um): D_p over four
# decades on both sides within the order of magnitude the paper cites for micellar solutions, R
# over 0.3-0.8 um (nodes 20 nm apart, at most 251).
PAPER_DP_SI = [1e-15, 3e-15, 1e-14, 3e-14, 1e-13, 3e-13, 1e-12, 3e-12]
PAPER_R_SI = [3e-7, 4e-7, 5e-7, 6e-7, 7e-7, 8e-7]
PAPER_EVERY = 500


def _paper_batch(lb, W, torch, overrides, seed0):
    """One batch of paper_setup boxes (scalar model), each with its SI overrides, run for the
    paper's 187 500 steps plus one (so that the final state is a readout row); returns the Return
    of each box, the batch's device time (ms) and the step count."""
    ws = [W.paper_setup("scalar", seed=seed0 + i, every=PAPER_EVERY, **o) for i, o in enumerate(overrides)]
    n_steps = ws[0]["steps"] + 1
    d_pull = ws[0]["rings"][0]["trap"]["dx"]
    ss = [lb.Solver.from_workload(w, max_samples=n_steps // PAPER_EVERY + 2) for w in ws]
    b = lb.Batch(ss)
    try:
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(torch.cuda.current_stream())
        b.step(n_steps)
        e1.record(torch.cuda.current_stream())
        b.sync()
        torch.cuda.synchronize()
        rets = [lb.return_metric(s_.series(), 0, d_pull, ws[0]["nx"], ws[0]["ny"]) for s_ in ss]
        return rets, e0.elapsed_time(e1), n_steps
    finally:
        b.close()
        for s_ in ss:
            s_.close()


def measure_3d(args, W):
    """The three-dimensional step (D3Q19, stiffness averaged over the unit sphere; four kernels
    per step) on the 256^3 periodic box of the default three-dimensional physics (3.8 GB of state,
    larger than L2, so no flush), timed with CUDA events around every step on the handle's own
    stream.  Its HBM roofline takes the algorithmic 224 B per cell and step (the 28 FP32 planes
    read once and written once); traffic is the DRAM bytes per step of the four kernels from the
    committed ncu counters at 192^3, scaled by the cell count (the kernels stream every plane, so
    traffic grows with the cells), or null when the source changed since."""
    from paper_2209_14889_gb300 import lb3d
    peaks, src = measured_peaks()
    w = W.cube3d()
    cells = w["nx"] * w["ny"] * w["nz"]
    s = lb3d.Solver3D.from_workload(w)
    s.step(3)
    s.sync()
    steps = max(5, min(args.steps, 40))
    s.timing(True)
    s.step(steps)
    s.sync()
    ms, n = s.kernel_time()
    s.timing(False)
    s.sync()
    bpc = s.bytes_per_cell
    launches = s.launches_per_step
    s.close()
    step_s = ms * 1e-3 / n
    prof = profile_values("step3d_192x192x192_counters.txt", LB3D_SOURCES)
    traffic = float(prof["dram_bytes_per_cell_step"]) * cells if "dram_bytes_per_cell_step" in prof else None
    inst = float(prof["warp_inst_per_cell_step"]) * cells if "warp_inst_per_cell_step" in prof else None
    gbs = bpc * cells / step_s / 1e9
    cpu = None
    if not args.no_cpu_baseline:
        # the three-dimensional oracle as it stands, one host core, one step of a 32^3 box
        import oracle.o3d as O3
        sim = O3.Sim3.from_workload(W.make3d(32, 32, 32, seed=7))
        t0 = time.perf_counter()
        sim.step(1)
        dt = time.perf_counter() - t0
        cpu = {"value": 32 ** 3 / dt / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
               "sample": "1 step of a 32^3 box of the same physics (%.2f s)" % dt}
    return {"workload": "256x256x256 periodic D3Q19 box, default three-dimensional physics (K^x = 1e-3 (2, 1, "
                        "1, 1, 1/2), eta_p 0.05, D_p 0.05, P = P_eq x + noise 0.05)",
            "value": cells / step_s / 1e6, "unit": "MLUPS", "ms_per_step": step_s * 1e3, "steps": n,
            "launches_per_step": launches,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": gbs / peaks["hbm_gbs"], "traffic": traffic, "peak_source": src,
                         "bytes_per_cell_step": bpc},
            "issue_roofline": issue_roofline(inst, step_s, args.sm_mhz), "cpu_baseline": cpu}


def measure_paper_setup(args, lb, W, torch):
    """The paper's pulling experiment at its own parameters (App. C: 250^2 closed box, tau 1.25,
    157-node droplet of radius 12.5 cells, trap 0.05 dragging it 100 cells over 25 000 steps after
    30 steps of equilibration, 187 500 steps, scalar modulus of Table IV), as batched runs: the
    Return (Eq. Rec) against D_p and against the droplet radius (Sec. III B)."""
    rd, ms_d, n = _paper_batch(lb, W, torch, [dict(Dp=d) for d in PAPER_DP_SI], 900)
    rr, ms_r, _ = _paper_batch(lb, W, torch, [dict(R=r) for r in PAPER_R_SI], 920)
    cells = 250 * 250
    return {"workload": "paper_setup (App. C, Tables I-IV): 250x250 closed box, tau 1.25, droplet 0.5 um "
                        "(157 nodes), trap 1e-6 N/m dragging 4 um over 0.2 s, %d steps, scalar model" % (n - 1),
            "Dp_m2_per_s": PAPER_DP_SI, "return_vs_Dp": rd,
            "radius_m": PAPER_R_SI, "return_vs_radius": rr,
            "steps": n, "seconds": (ms_d + ms_r) * 1e-3,
            "value": cells * n * (len(PAPER_DP_SI) + len(PAPER_R_SI)) / ((ms_d + ms_r) * 1e-3) / 1e6,
            "unit": "MLUPS"}


def run_only_paper(args):
    import torch
    from paper_2209_14889_gb300 import lb, workloads as W
    torch.cuda.set_device(0)
    print(json.dumps({"paper_setup": measure_paper_setup(args, lb, W, torch)}), flush=True)


def measure_protocol(args, lb, W, torch):
    """The paper's pulling experiments of its scalar-viscoelasticity results (Sec. III B) as
    batched runs of 250 x 250 closed boxes with the scalar model: the trapped ring is dragged by
    40 cells and released.  (1) Return against D_p: eight boxes, D_p log-spaced over [1e-3, 0.25],
    a ring of 128 nodes (radius 16), dragged over 8000 steps, 20000 steps.  (2) Return against the
    ring's radius: 8 .. 28 cells (nodes at 0.785-cell spacing), D_p = 0.01, the same protocol.
    (3) Return against the pulling time: 2000 .. 16000 steps over the same 40 cells, radius 16,
    D_p = 0.01, 30000 steps.  Synthetic stand-in for the paper's runs: same protocol shape and
    lattice size, these lattice-unit parameters."""
    import numpy as np
    dps = [float(x) for x in np.geomspace(1e-3, 0.25, 8)]
    rets, ms = _protocol_batch(lb, W, torch, [(16.0, 128, 8000, dp, 700 + i) for i, dp in enumerate(dps)], 20000)
    out = {"workload": "8 x 250x250 closed boxes, scalar model, trapped ring (128 nodes, r 16) dragged 40 cells over "
                       "8000 steps then released, 20000 steps, relaxation 2000 steps",
           "Dp": dps, "return": rets, "value": 8 * 250 * 250 * 20000 / (ms * 1e-3) / 1e6, "unit": "MLUPS",
           "seconds": ms * 1e-3}
    radii = [8.0, 12.0, 16.0, 20.0, 24.0, 28.0]
    rr, ms_r = _protocol_batch(lb, W, torch, [(r, int(round(2 * math.pi * r / 0.785)), 8000, 0.01, 720 + i)
                                             for i, r in enumerate(radii)], 20000)
    out["radius_sweep"] = {"workload": "6 boxes, D_p 0.01, radius 8..28 (nodes at 0.785 spacing), dragged 40 cells "
                                       "over 8000 steps, 20000 steps", "radius": radii, "return": rr,
                           "seconds": ms_r * 1e-3}
    pulls = [2000, 4000, 8000, 12000, 16000]
    rp, ms_p = _protocol_batch(lb, W, torch, [(16.0, 128, tp, 0.01, 740 + i) for i, tp in enumerate(pulls)], 30000)
    out["pull_time_sweep"] = {"workload": "5 boxes, D_p 0.01, radius 16, dragged 40 cells over 2000..16000 steps, "
                                          "30000 steps", "pull_steps": pulls, "return": rp, "seconds": ms_p * 1e-3}
    return out


ANISO_THETAS = [0.0, math.pi / 6, math.pi / 3, math.pi / 2, 2 * math.pi / 3, 5 * math.pi / 6, math.pi]
ANISO_ALPHAS = [0.0, -0.45, -0.9]


def measure_anisotropy(args, lb, W, torch):
    """The paper's anisotropy study (Sec. III C): the Return (Eq. Rec) of the trapped ring against
    the equilibrium polarisation P = sqrt(-alpha/beta) (beta = 1, alpha in {0, -0.45, -0.9}) and
    the initial director angle theta0 to the pulling axis x (0 .. pi by pi/6; at alpha = 0 only
    theta0 = 0 and pi/3), with the tensorial model in 250 x 250 closed boxes: no orientation
    noise, the ring (128 nodes, radius 16) on the box's mirror line, the trap of the protocol form
    (dragged 40 cells over 8000 steps, released, 20000 steps), relaxation 2000 steps, D_p = 0.01,
    and the Ericksen force on.  One batch per alpha.  Reports, per alpha, the Return per theta0, its residuals under theta0 ->
    theta0 + pi and theta0 -> pi - theta0, and the deflection (centre of mass across the pulling
    axis, cells) and rotation (of the node that starts on the +x side, about the centre of mass,
    degrees) at the end of each run."""
    import numpy as np
    n_steps, d_pull, side, cy = 20000, 40.0, 250, 124.5
    trap = dict(k=0.02, dx=d_pull, dy=0.0, t_eq=30, pull=8000, width=30)
    out = {"workload": "250x250 closed boxes, tensorial model with the Ericksen force, no noise, "
                       "trapped ring (128 nodes, r 16) on the mirror line dragged 40 cells along x over "
                       "8000 steps then released, 20000 steps, relaxation 2000 steps, D_p 0.01",
           "theta0": ANISO_THETAS, "alpha": ANISO_ALPHAS, "per_alpha": {}}
    cells_steps, seconds = 0, 0.0
    for alpha in ANISO_ALPHAS:
        thetas = ANISO_THETAS if alpha != 0.0 else [0.0, math.pi / 3]
        ws = [W.make(side, side, rings=[W.ring(128, 16.0, (60.3, cy), pull_force=0.0, trap=trap)],
                     seed=900, noise_amp=0.0, walls_y=1, walls_x=1, Dp=0.01, lambda_steps=2000.0,
                     every=100, steps=n_steps, alpha=alpha, director_angle=th)
              for th in thetas]
        ss = [lb.Solver.from_workload(w, max_samples=n_steps // 100 + 2) for w in ws]
        X0 = [s_.nodes() for s_ in ss]
        b = lb.Batch(ss)
        rec = {"theta0": thetas}
        try:
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(torch.cuda.current_stream())
            b.step(n_steps)
            e1.record(torch.cuda.current_stream())
            b.sync()
            torch.cuda.synchronize()
            seconds += e0.elapsed_time(e1) * 1e-3
            cells_steps += len(ss) * side * side * n_steps
            rets, defl, rot = [], [], []
            for s_, x0 in zip(ss, X0):
                ser = s_.series()
                rets.append(lb.return_metric(ser, 0, d_pull, side, side))
                x1 = s_.nodes()
                c0, c1 = x0.mean(0), x1.mean(0)
                defl.append(float(c1[1] - c0[1]))
                a0 = math.atan2(x0[0, 1] - c0[1], x0[0, 0] - c0[0])
                a1 = math.atan2(x1[0, 1] - c1[1], x1[0, 0] - c1[0])
                rot.append(math.degrees(math.remainder(a1 - a0, 2 * math.pi)))
            rec.update(ret=rets, deflection=defl, rotation_deg=rot)
            if len(thetas) == len(ANISO_THETAS):
                rec["period_pi_residual"] = abs(rets[0] - rets[-1])
                rec["mirror_pi_2_residual"] = max(abs(rets[i] - rets[-1 - i]) for i in range(len(rets)))
                rec["theta0_spread"] = max(rets) - min(rets)
            else:
                rec["theta0_spread"] = max(rets) - min(rets)
        except lb.LBError as e:
            rec["error"] = str(e)
        finally:
            b.close()
            for s_ in ss:
                s_.close()
        out["per_alpha"]["%g" % alpha] = rec
    out["value"] = cells_steps / seconds / 1e6 if seconds > 0 else None
    out["unit"] = "MLUPS"
    out["seconds"] = seconds
    return out


def run_only_aniso(args):
    """The anisotropy form alone (one JSON line)."""
    import torch
    from paper_2209_14889_gb300 import lb, workloads as W
    print(json.dumps({"anisotropy": measure_anisotropy(args, lb, W, torch)}))


def measure_batched(args, lb, W, torch):
    """The batched workload: 256 independent periodic lattices of sides {128, ..., 512} (28.9M
    cells, 3.2 GB of FP32 state, larger than L2, so no flush) with one ring each, advanced by the
    persistent kernel in graph-replayed chunks of 10 steps after the tile-shape autotuner; and
    the restoring-force difference of batched instances against lb_step on the same inputs."""
    import numpy as np
    ws = W.cfg4()
    cells = sum(w["nx"] * w["ny"] for w in ws)
    ss = [lb.Solver.from_workload(w) for w in ws]
    b = lb.Batch(ss)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    b.autotune(args.tune_cache, steps=20)
    tune_s = time.perf_counter() - t0
    shapes = {}
    for i, w in enumerate(ws):
        sh = lb.TILE_SHAPES[b.shape(i)]
        shapes["%dx%d" % (w["nx"], w["ny"])] = sh if isinstance(sh, str) else "%dx%d" % sh
    chunk = 10
    steps = max(3, min(args.steps, 10))
    b.step(2 * chunk)
    b.sync()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        ev[k][0].record(stream)
        b.step(chunk)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(x.elapsed_time(y) for x, y in ev)
    b.sync()
    out = {"workload": "256 periodic lattices, sides uniform over {128,192,256,384,512} (%.1fM "
                       "cells), one ring each (r U[4,32], N=clamp(round(2 pi r/0.78),32,256), pull "
                       "5e-4 at U[0,90] deg), D_p log-uniform [1e-3,1] with ceil(D_p/0.2) "
                       "diffusion sub-steps above 0.2, relaxation U[20,500] steps" % (cells / 1e6),
           "value": cells * chunk * steps / (ms * 1e-3) / 1e6, "unit": "MLUPS",
           "ms_per_lb_step": ms / (chunk * steps), "graph": b.uses_graph, "grid_ctas": b.grid,
           "tile_shapes": shapes, "autotune_s": tune_s, "steps": chunk * steps}
    peaks, _ = measured_peaks()
    gbs = 112.0 * cells * chunk * steps / (ms * 1e-3) / 1e9
    out["roofline_frac"] = gbs / peaks["hbm_gbs"]
    out["achieved_gbs"] = gbs
    b.close()
    for s_ in ss:
        s_.close()
    # batched instances against lb_step on the same inputs (restoring force over 500 steps)
    errs = []
    sub = [w for w in W.cfg4(n_instances=8)]
    sb = [lb.Solver.from_workload(w) for w in sub]
    bb = lb.Batch(sb)
    bb.step(500)
    bb.sync()
    for w, s_ in zip(sub, sb):
        r = lb.Solver.from_workload(w)
        r.step(500)
        r.sync()
        a, c = s_.series()[:, 6:8], r.series()[:, 6:8]
        errs.append(float(np.linalg.norm(a - c) / max(np.linalg.norm(c), 1e-300)))
        r.close()
    bb.close()
    for s_ in sb:
        s_.close()
    out["frest_err_vs_fp32"] = {"value": max(errs), "workload": "first 8 instances, 500 steps, "
                                "batched vs lb_step, relative L2 over 50 readouts"}
    return out


# (level, Ci, Co) of the network's 3x3 convolutions (level l at 1/2^l resolution)
NET_CONVS = [(0, 16, 32), (0, 32, 32), (1, 32, 64), (1, 64, 64), (2, 64, 96), (2, 96, 96), (3, 96, 128),
             (3, 128, 128), (2, 224, 96), (2, 96, 96), (1, 160, 64), (1, 64, 64), (0, 96, 32), (0, 32, 32),
             (0, 32, 16)]


def run_only_net(args):
    """Forward passes of the network at 256^2, batch 1, with the default (tcgen05) convolutions."""
    import torch
    from paper_2209_14889_gb300 import lb
    net = lb.Net(1, 256, 256, seed=1)
    x = torch.zeros((1, 256, 256, 16), dtype=torch.bfloat16, device="cuda")
    for _ in range(args.warmup):
        net.forward(x)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        net.forward(x)
    e1.record()
    torch.cuda.synchronize()
    lb.conv_status()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    flop = 2.0 * 9 * 256 * 256 * sum(ci * co * 4 ** -lev for lev, ci, co in NET_CONVS)
    print(json.dumps({"network_forward_ms": ms, "tflops": flop / (ms * 1e-3) / 1e12, "steps": args.steps}))
    net.close()


def measure_learned(args, lb, torch):
    """The learned form at 256^2: training pairs from seeded trajectories of the batched recipe's
    physics (one lattice side), GPU training of the U-Net for a time budget, residual bounds
    fixed on a validation trajectory, then 64 calls (1024 steps) on a held-out trajectory
    against the plain FP32 solver on the same GPU."""
    import numpy as np
    from paper_2209_14889_gb300 import learned as LR
    side, calls = 256, 64
    t0 = time.perf_counter()
    data = LR.Dataset(LR.learned_workloads(500, LEARNED_TRAJ, side=side), pairs_per_traj=2, warmup=64, stride=256,
                      batch=250)
    t_data = time.perf_counter() - t0
    net = lb.Net(4, side, side, seed=1)
    held = list(range(0, data.n, 8))
    val0 = LR.evaluate(net, data, held)
    t0 = time.perf_counter()
    net, losses = LR.train(data, batch=4, seconds=args.learned_seconds, lr=5e-4, seed=1, net=net)
    t_train = time.perf_counter() - t0
    val1 = LR.evaluate(net, data, held)
    inf = LR.inference_net(net, side, side)
    eps, acc_val, err_val = LR.calibrate(inf, data.norm, LR.learned_workloads(501, 1, side=side)[0], calls=16,
                                         grid=(0.05, 0.2, 1.0, 5.0, 20.0, 100.0))
    w = LR.learned_workloads(502, 1, side=side)[0]
    fr_p, ms_p, _ = LR.run(w, calls=calls)
    fr_l, ms_l, stt = LR.run(w, inf, data.norm, calls=calls, eps=eps)
    err = float(np.linalg.norm(fr_l - fr_p) / np.linalg.norm(fr_p))
    cells = side * side
    # network forward throughput at 256^2, batch 1, per convolution kernel (CUDA events)
    flop = 2.0 * 9 * cells * sum(ci * co * 4 ** -lev for lev, ci, co in NET_CONVS)
    xin = torch.zeros((1, side, side, 16), dtype=torch.bfloat16, device="cuda")
    fwd = {}
    for name, k in (("mma_sync", 0), ("tcgen05", 1)):
        lb.conv_kernel(k)
        for _ in range(3):
            inf.forward(xin)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(20):
            inf.forward(xin)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 20
        fwd[name] = {"ms": ms, "tflops": flop / (ms * 1e-3) / 1e12}
    lb.conv_kernel(1)
    lb.conv_status()
    peaks, _ = measured_peaks()
    out = {"workload": "256x256 periodic, one ring (batched-recipe physics, seed 502), 64 calls of 16 steps",
           "network_forward": {"gflop": flop / 1e9, "batch": 1, "by_kernel": fwd,
                               "tensor_roofline": {"bound": "tensor", "achieved": fwd["tcgen05"]["tflops"],
                                                   "peak": peaks.get("bf16_tflops"), "unit": "TFLOP/s",
                                                   "frac": fwd["tcgen05"]["tflops"] / peaks.get("bf16_tflops", 1.0)}},
           "value": cells * calls * 16 / (ms_l * 1e-3) / 1e6, "unit": "MLUPS",
           "plain_fp32_mlups": cells * calls * 16 / (ms_p * 1e-3) / 1e6,
           "accepted_calls": stt["accepted"], "calls": calls,
           "frest_err_vs_fp32": {"value": err, "workload": "64 readouts (every 16 steps), relative L2"},
           "residual_bounds": {"momentum": eps[0], "tendency": eps[1],
                               "validation_accepted": acc_val, "validation_frest_err": err_val},
           "training": {"trajectories": LEARNED_TRAJ, "pairs": data.n, "data_s": t_data,
                        "data": "batched kernel, 250 trajectories at a time, pairs at steps 64 and 320",
                        "adam_steps": len(losses), "train_s": t_train,
                        "batch": 4, "loss_subset_before": val0, "loss_subset_after": val1}}
    inf.close()
    net.close()
    return out


LEARNED_TRAJ = 2000


def measure_learned_curve(args, lb, torch, budgets=(45.0, 180.0, 540.0)):
    """The learned form against its training budget: one network trained on the 2000-trajectory
    data set in segments (each a cosine schedule of its own), and after each segment the loss on
    pairs of 64 unseen trajectories, the residual bounds calibrated for 1 % and the calls they
    accept on a held-out trajectory, the restoring-force error with every call accepted, and the
    time of 64 calls against 1024 plain steps."""
    import numpy as np
    from paper_2209_14889_gb300 import learned as LR
    side, calls = 256, 64
    data = LR.Dataset(LR.learned_workloads(500, LEARNED_TRAJ, side=side), pairs_per_traj=2, warmup=64, stride=256,
                      batch=250)
    val = LR.Dataset(LR.learned_workloads(600, 64, side=side), pairs_per_traj=2, warmup=64, stride=256, batch=64,
                     norm=data.norm)
    net = lb.Net(4, side, side, seed=1)
    w = LR.learned_workloads(502, 1, side=side)[0]
    fr_p, ms_p, _ = LR.run(w, calls=calls)
    points, spent = [], 0.0
    for b in budgets:
        net, losses = LR.train(data, batch=4, seconds=b - spent, lr=5e-4, seed=int(b), net=net)
        spent = b
        vloss = LR.evaluate(net, val, range(val.n))
        inf = LR.inference_net(net, side, side)
        eps, acc_val, err_val = LR.calibrate(inf, data.norm, LR.learned_workloads(501, 1, side=side)[0], calls=16,
                                             grid=(0.05, 0.2, 1.0, 5.0, 20.0, 100.0))
        fr_l, ms_l, stt = LR.run(w, inf, data.norm, calls=calls, eps=eps)
        fr_a, ms_a, st_a = LR.run(w, inf, data.norm, calls=calls, eps=(1e30, 1e30))
        nrm = np.linalg.norm(fr_p)
        points.append({"train_s": b, "adam_steps_segment": len(losses), "val_loss": vloss,
                       "bounds": list(eps), "accepted": stt["accepted"],
                       "frest_err_calibrated": float(np.linalg.norm(fr_l - fr_p) / nrm),
                       "frest_err_all_accepted": float(np.linalg.norm(fr_a - fr_p) / nrm),
                       "all_accepted_calls": st_a["accepted"], "ms_learned_all_accepted": ms_a,
                       "ms_learned_calibrated": ms_l})
        inf.close()
    net.close()
    return {"workload": "256x256, batched-recipe physics; %d trajectories (%d pairs) for training, 64 unseen "
                        "for the loss, held-out trajectory 502 (64 calls = 1024 steps)" % (LEARNED_TRAJ, data.n),
            "ms_plain": ms_p, "points": points}


PROFILE_CASES = ("tile_fp32", "tile_lp", "tile_scalar", "strip_fp32", "strip_lp", "strip_scalar", "sweep_fp32",
                 "diffuse_fp32", "batch", "batch_cfg4", "cube3d_128", "cube3d_192", "cube3d_256")


def run_case(args):
    """One lattice kernel on its profiling workload for --steps lattice steps (the commands under
    profiles/ capture these): tile_* and sweep_fp32 on cfg3 at 2048^2 with 4 rings, strip_* on
    cfg3 at 4096^2 with 16 rings (FP32, FP16/BF16 storage, scalar model), diffuse_fp32 on the
    2048^2 lattice with D_p = 0.6 in 3 sub-steps, batch: 64 lattices of 256^2 (cfg4 recipe,
    D_p = 0.05, no sub-steps) in one batch with the 32 x 16 tile shape, batch_cfg4: the batched
    workload of the bench (256 lattices, sides 128-512, stress diffusion with sub-steps) with the
    warp-strip shape for every instance (the autotuner's choice), cube3d_N: the
    three-dimensional step on an N^3 periodic box of the default three-dimensional physics."""
    import torch
    from paper_2209_14889_gb300 import lb, workloads as W
    torch.cuda.set_device(0)
    case = args.case
    if case.startswith("cube3d"):
        from paper_2209_14889_gb300 import lb3d
        n = int(case.split("_")[1])
        w = W.make3d(n, n, n, seed=7)
        s3 = lb3d.Solver3D.from_workload(w)
        s3.step(args.steps)
        s3.sync()
        print(json.dumps({"case": case, "cells": n ** 3, "steps": args.steps}))
        s3.close()
        return
    if case == "batch_cfg4":
        ws = W.cfg4()
        ss = [lb.Solver.from_workload(w) for w in ws]
        b = lb.Batch(ss)
        b.set_shape(4)
        b.step(args.steps)
        b.sync()
        print(json.dumps({"case": case, "cells": sum(w["nx"] * w["ny"] for w in ws), "steps": args.steps}))
        b.close()
        for s_ in ss:
            s_.close()
        return
    if case == "batch":
        ws = W.cfg4(n_instances=64, sides=(256,))
        for w in ws:
            w["Dp"], w["diffusion_substeps"] = 0.05, 0
        ss = [lb.Solver.from_workload(w) for w in ws]
        b = lb.Batch(ss)
        b.set_shape(0)
        b.step(args.steps)
        b.sync()
        print(json.dumps({"case": case, "cells": sum(w["nx"] * w["ny"] for w in ws), "steps": args.steps}))
        b.close()
        return
    side = 4096 if case.startswith("strip") else 2048
    w = W.cfg3(side=side, n_rings=max(1, 16 * side * side // (4096 * 4096)))
    if case.endswith("_scalar"):
        w = dict(w, **W.scalar_physics())
    if case.startswith("diffuse"):
        w = dict(w, Dp=0.6, diffusion_substeps=3)
    prec = lb.LB_FP16_BF16 if case.endswith("_lp") else lb.LB_FP32
    s = lb.Solver.from_workload(w, precision=prec)
    s.set_kernel({"tile": lb.LB_KERNEL_TILE, "strip": lb.LB_KERNEL_STRIP, "sweep": lb.LB_KERNEL_SWEEP,
                  "diffuse": lb.LB_KERNEL_TILE}[case.split("_")[0]])
    s.step(args.steps)
    s.sync()
    print(json.dumps({"case": case, "kernel": s.lattice_kernel, "cells": w["nx"] * w["ny"], "steps": args.steps}))
    s.close()


def run_learned_curve(args):
    import torch
    from paper_2209_14889_gb300 import lb
    torch.cuda.set_device(0)
    print(json.dumps({"learned_curve": measure_learned_curve(args, lb, torch)}), flush=True)


def cpu_baseline_sample():
    """The oracle as it stands on one host core, on a bounded sample of the workload: one LB
    time step of the 1024 x 1024 lattice."""
    import oracle as O
    from paper_2209_14889_gb300 import workloads as W
    w = W.cfg2()
    sim = O.Sim.from_workload(w)
    t0 = time.perf_counter()
    sim.step(1)
    dt = time.perf_counter() - t0
    return {"value": 1024 * 1024 / dt / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": "1 LB time step of the 1024x1024 workload (%.1f s)" % dt}


_OMP_CHILD = r"""
import json, sys, time
sys.path.insert(0, sys.argv[1])
import oracle as O
from paper_2209_14889_gb300 import workloads as W
assert O._OPENMP
O.lib()
sim = O.Sim.from_workload(W.cfg2())
sim.step(1)
t0 = time.perf_counter()
sim.step(3)
print(json.dumps({"dt": time.perf_counter() - t0}))
"""


def cpu_baseline_openmp():
    """The same oracle source built with OpenMP over rows (bitwise the serial results) on all host
    cores, in a child process: three LB time steps of the 1024 x 1024 lattice after one untimed."""
    cores = os.cpu_count() or 1
    env = dict(os.environ, VLB_ORACLE_OPENMP="1", OMP_NUM_THREADS=str(cores))
    try:
        r = subprocess.run([sys.executable, "-c", _OMP_CHILD, ROOT], env=env, cwd=ROOT, capture_output=True,
                           text=True, timeout=600)
        dt = json.loads(r.stdout.strip().splitlines()[-1])["dt"]
    except Exception as e:                     # the figure is context only: report why it is missing
        return {"error": str(e)[:200]}
    return {"value": 3 * 1024 * 1024 / dt / 1e6, "unit": "MLUPS", "cores": cores,
            "kind": "oracle, OpenMP over rows (same source, bitwise the serial results)",
            "sample": "3 LB time steps of the 1024x1024 workload after one untimed (%.1f s)" % dt}


KERNEL_NAMES = {"auto": "k_fused (fused lattice step, one cell per thread)",
                "pair": "k_fused_pair (fused lattice step, two cells per thread)",
                "tile": "k_fused (fused lattice step, one cell per thread)",
                "sweep": "k_sweep (column-strip sweep)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--side", type=int, default=1024,
                    help="lattice side (profiling captures use 2048 so that the state exceeds L2)")
    ap.add_argument("--kernel", default="auto", choices=["auto", "tile", "pair", "sweep"],
                    help="lattice kernel (auto: the fastest measured, the one-cell tile kernel)")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched workload")
    ap.add_argument("--separate-nodes", action="store_true",
                    help="run the node step as its own kernel instead of in the tile kernel's tail")
    ap.add_argument("--only-net", action="store_true",
                    help="time the network's forward pass at 256^2 (batch 1) only (for profiling)")
    ap.add_argument("--only-aniso", action="store_true",
                    help="run the anisotropy study (Return against alpha and theta0) only")
    ap.add_argument("--only-paper", action="store_true",
                    help="run the paper's own setup (Return against D_p and radius) only")
    ap.add_argument("--case", default=None, choices=PROFILE_CASES,
                    help="run one lattice kernel's profiling workload for --steps steps (only)")
    ap.add_argument("--learned-curve", action="store_true",
                    help="train the learned form for growing budgets and report each point (only)")
    ap.add_argument("--learned-seconds", type=float, default=45.0,
                    help="training budget of the learned form (0: skip it)")
    ap.add_argument("--tune-cache", default=None,
                    help="JSON cache of the batched tile-shape autotuner (default: none)")
    ap.add_argument("--no-extras", action="store_true",
                    help="time the device steps only (no e2e, parity check or CPU baseline)")
    args = ap.parse_args()
    rank, local, world = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.only_net:
        return run_only_net(args)
    if args.only_aniso:
        return run_only_aniso(args)
    if args.only_paper:
        return run_only_paper(args)
    if args.learned_curve:
        return run_learned_curve(args)
    if args.case:
        return run_case(args)

    import numpy as np
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2209_14889_gb300 import lb, workloads as W

    w = W.cfg2(seed=2 + rank)
    if args.side != 1024:
        w = W.make(args.side, args.side,
                   rings=[W.ring(256, 24.0, (args.side / 2, args.side / 2), pull_force=5e-4,
                                 pull_angle=math.radians(30))],
                   seed=2 + rank, steps=20000, every=10, lambda_steps=200.0, Dp=0.1)
    cells = w["nx"] * w["ny"]
    s = lb.Solver.from_workload(w)
    s.set_kernel({"auto": lb.LB_KERNEL_AUTO, "tile": lb.LB_KERNEL_TILE, "pair": lb.LB_KERNEL_PAIR,
                  "sweep": lb.LB_KERNEL_SWEEP}[args.kernel])
    s.set_node_tail(not args.separate_nodes)
    launches_per_step = s.launches_per_step
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # warm-up
    for _ in range(args.warmup):
        flush.zero_()
        s.step(LB_STEPS_PER_STEP)
    s.sync()

    # timed steps (device time; consecutive kernels overlap by programmatic dependent launch)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with Clocks(local) as clk:
        barrier()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            s.step(LB_STEPS_PER_STEP)
            ev[k][1].record(stream)
        barrier()
    s.sync()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    # per-kernel durations for the roofline: the same steps again with events around each
    # launch (which serialises the kernels), L2 flushed between steps as above
    s.timing(True)
    for k in range(args.steps):
        flush.zero_()
        s.step(LB_STEPS_PER_STEP)
    s.sync()
    kt = s.kernel_time()
    s.timing(False)
    ms = max_over_ranks(ms, world)
    total_cells = cells * LB_STEPS_PER_STEP * args.steps * world
    value = total_cells / (ms * 1e-3) / 1e6

    # roofline of the fused lattice kernel
    peaks, peak_kind = measured_peaks()
    fused_avg_s = kt["fused_ms"] * 1e-3 / max(kt["fused_launches"], 1)
    bytes_launch = s.bytes_per_cell * cells
    achieved = bytes_launch / fused_avg_s / 1e9
    traffic = ncu_traffic() if args.kernel in ("auto", "tile") and args.side == 1024 else None
    csum = clk.summary()
    args.sm_mhz = csum.get("sm_mhz") or csum.get("sm_max_mhz") or 2070.0
    prof = profile_values("fused_step_1024x1024.txt", KERNEL_SOURCES) if args.kernel in ("auto", "tile") \
        and args.side == 1024 else {}
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
            "issue": issue_roofline(float(prof["warp_inst_per_launch"]) if "warp_inst_per_launch" in prof else None,
                                    fused_avg_s, args.sm_mhz),
            "kernel": KERNEL_NAMES[args.kernel], "peak_kind": peak_kind,
            "algorithmic_bytes_per_launch": bytes_launch,
            "mean_launch_us": fused_avg_s * 1e6,
            "node_step": ("separate node kernel, mean %.2f us" % (kt["node_ms"] * 1e3 / max(kt["node_launches"], 1))
                          if kt["node_launches"] else "in the lattice kernel's tail (timed with it)")}

    if args.no_extras:
        s.close()
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
                              "steps": args.steps, "ms_per_step": ms / args.steps,
                              "config": {"lattice": [w["nx"], w["ny"]]}, "roofline": roof,
                              "note": "device steps only (--no-extras)"}), flush=True)
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    # end to end through the C ABI with host buffers: every bench step takes a whole stored state
    # uploaded from pinned host memory in one copy, runs the 10 LB steps on it and reads the
    # newest readout row back.  The upload of step k + 1's state runs on the handle's copy stream
    # while step k computes (lb_stage_state), each step starts by making its uploaded state
    # current (lb_commit_state), and step k's row comes back while step k + 1 runs
    # (lb_series_latest_async / lb_series_wait); e2e_serial is the same loop with the upload in
    # line (lb_write_state) and a synchronous row read (lb_series_latest).
    nbytes = s.state_bytes
    pinned = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    s.read_state(pinned)
    e2e_steps = max(3, min(args.steps, 10))
    d2h = 0
    rows_pin = [torch.empty(lb.lib().lb_series_row_len(s.h), dtype=torch.float64).pin_memory() for _ in range(2)]

    def e2e_run(overlap):
        nonlocal d2h
        barrier()
        t0 = time.perf_counter()
        if overlap:
            s.stage_state(pinned)
        for k in range(e2e_steps):
            if overlap:
                s.commit_state()
                if k + 1 < e2e_steps:
                    s.stage_state(pinned)
                s.step(LB_STEPS_PER_STEP)
                if k > 0:
                    s.series_wait()          # step k - 1's row, while step k runs
                s.series_latest_async(rows_pin[k % 2], 1)
                d2h = rows_pin[k % 2].numel() * 8
            else:
                s.write_state(pinned)
                s.step(LB_STEPS_PER_STEP)
                row = s.series_latest(1)
                d2h = row.nbytes
        if overlap:
            s.series_wait()
        barrier()
        return cells * LB_STEPS_PER_STEP * e2e_steps * world / (time.perf_counter() - t0) / 1e6

    e2e_serial = e2e_run(False)
    e2e = {"value": e2e_run(True), "unit": "MLUPS",
           "h2d_bytes_per_step": int(nbytes), "d2h_bytes_per_step": int(d2h),
           "steps": e2e_steps,
           "pipeline": "upload of the next state and read-back of the previous row overlap the steps",
           "serial_value": e2e_serial}

    rc = lb.lib().lb_sync(s.h)
    s.close()
    del flush
    forms = None if world > 1 else measure_forms(args, lb, W, torch)
    if forms is not None and not args.no_batched:
        forms["batched"] = measure_batched(args, lb, W, torch)
        try:
            forms["protocol"] = measure_protocol(args, lb, W, torch)
        except lb.LBError as e:
            forms["protocol"] = {"error": str(e)}
        try:
            forms["anisotropy"] = measure_anisotropy(args, lb, W, torch)
        except lb.LBError as e:
            forms["anisotropy"] = {"error": str(e)}
        try:
            forms["paper_setup"] = measure_paper_setup(args, lb, W, torch)
        except lb.LBError as e:
            forms["paper_setup"] = {"error": str(e)}
    if forms is not None and not args.no_batched:
        forms["three_d"] = measure_3d(args, W)
    if forms is not None and args.learned_seconds > 0:
        forms["learned"] = measure_learned(args, lb, torch)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    frest_err = frest_error_check()
    cpu = None if args.no_cpu_baseline else cpu_baseline_sample()
    cpu_omp = None if args.no_cpu_baseline else cpu_baseline_openmp()
    line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "lattice": [w["nx"], w["ny"]],
                       "lb_steps_per_step": LB_STEPS_PER_STEP,
                       "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": roof, "cpu_baseline": cpu, "cpu_baseline_openmp": cpu_omp, "e2e": e2e, "clocks": clk.summary(),
            "gpu_launches": launches_per_step * LB_STEPS_PER_STEP * args.steps,
            "kernel_timing": "roofline durations from a second pass with events around each launch",
            "frest_err_vs_fp64": {"value": frest_err, "workload": "64x64, 200 steps, 20 readouts"},
            "forms": forms,
            "status": int(rc)}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
