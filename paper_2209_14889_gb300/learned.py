"""The learned stepper: data from the solver's own trajectories, GPU training of the U-Net with
the library's kernels, and the stepper with its residual check and plain-solver fallback.

Everything numerical runs in libvlb.so (lb_learned_*, lb_net_*); this module only schedules it:
it creates solvers, asks the library to pack their fields, keeps the training pairs in device
memory (torch tensors as plain buffers) and calls the training step.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import lb
from . import workloads as W

CHANNELS = ["ux", "uy", "sxx", "sxy", "syy", "dPx", "dPy", "body"]
JUMP = 16                     # lattice steps per learned call
OUT_MASK = np.array([1.0] * 7 + [0.0] * 9, dtype=np.float32)
IDENTITY_NORM = np.concatenate([np.zeros(8), np.ones(8), np.ones(7)]).astype(np.float32)


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def learned_workloads(seed: int, n: int, side: int = 256, steps: int = 4096) -> list:
    """The batched recipe's physics (radius, node count, pull angle, D_p with sub-steps,
    relaxation time) at one lattice side, readouts every 16 steps."""
    ws = W.cfg4(seed=seed, n_instances=n, sides=(side,), steps=steps)
    for w in ws:
        w["every"] = JUMP
    return ws


def pack(solver, norm, x=None, raw=None):
    """Network input (BF16 [ny, nx, 16]) and raw fields (FP32 [ny, nx, 8]) of a solver's state."""
    nm = np.ascontiguousarray(norm, dtype=np.float32)
    lb._check(solver.h, lb.lib().lb_learned_pack(solver.h, nm.ctypes.data, lb._ptr(x), lb._ptr(raw)))


def target(raw0, raw1, norm, out):
    nm = np.ascontiguousarray(norm, dtype=np.float32)
    cells = raw0.numel() // 8
    lb._check(None, lb.lib().lb_learned_target(lb._ptr(raw0), lb._ptr(raw1), nm.ctypes.data, lb._ptr(out),
                                               cells, _stream()))


def normalize(raw, norm, x):
    nm = np.ascontiguousarray(norm, dtype=np.float32)
    cells = raw.numel() // 8
    lb._check(None, lb.lib().lb_learned_normalize(lb._ptr(raw), nm.ctypes.data, lb._ptr(x), cells, _stream()))


def fit_norm(samples0, samples1) -> np.ndarray:
    """Input shift/scale per channel (mean, 1/std over the samples) and output scales (1/std of
    the 16-step changes); samples: host FP32 [..., 8] raw fields at t and t + 16."""
    a = np.concatenate([s.reshape(-1, 8) for s in samples0]).astype(np.float64)
    b = np.concatenate([s.reshape(-1, 8) for s in samples1]).astype(np.float64)
    shift = a.mean(axis=0)
    sd = a.std(axis=0)
    scale = 1.0 / np.where(sd > 0, sd, 1.0)
    dsd = (b - a)[:, :7].std(axis=0)
    oscale = 1.0 / np.where(dsd > 0, dsd, 1.0)
    return np.concatenate([shift, scale, oscale]).astype(np.float32)


class Dataset:
    """Pairs (x(t), target(t -> t + 16)) of seeded trajectories, held on the GPU.  batch > 0: the
    trajectories are generated `batch` at a time by the batched kernel (lb_batch_*), which
    advances them together; else one solver at a time."""

    def __init__(self, workloads, pairs_per_traj: int, warmup: int = 32, stride: int = JUMP, norm=None,
                 batch: int = 0):
        import torch
        ny, nx = workloads[0]["ny"], workloads[0]["nx"]
        n = len(workloads) * pairs_per_traj
        self.raw0 = torch.empty((n, ny, nx, 8), dtype=torch.float32, device="cuda")
        self.raw1 = torch.empty((n, ny, nx, 8), dtype=torch.float32, device="cuda")
        if batch > 0:
            for g0 in range(0, len(workloads), batch):
                group = workloads[g0:g0 + batch]
                ss = [lb.Solver.from_workload(w) for w in group]
                b = lb.Batch(ss)
                b.step(warmup)
                for p in range(pairs_per_traj):
                    b.sync()
                    for j, s in enumerate(ss):
                        pack(s, IDENTITY_NORM, raw=self.raw0[(g0 + j) * pairs_per_traj + p])
                    b.step(JUMP)
                    b.sync()
                    for j, s in enumerate(ss):
                        pack(s, IDENTITY_NORM, raw=self.raw1[(g0 + j) * pairs_per_traj + p])
                    if stride > JUMP:
                        b.step(stride - JUMP)
                b.sync()
                b.close()
                for s in ss:
                    s.close()
        else:
            k = 0
            for w in workloads:
                s = lb.Solver.from_workload(w)
                s.step(warmup)
                for _ in range(pairs_per_traj):
                    pack(s, IDENTITY_NORM, raw=self.raw0[k])
                    s.step(JUMP)
                    pack(s, IDENTITY_NORM, raw=self.raw1[k])
                    if stride > JUMP:
                        s.step(stride - JUMP)
                    k += 1
                s.sync()
                s.close()
        torch.cuda.synchronize()
        if norm is None:
            pick = list(range(0, n, max(1, n // 16)))
            norm = fit_norm([self.raw0[j].cpu().numpy() for j in pick],
                            [self.raw1[j].cpu().numpy() for j in pick])
        self.norm = np.asarray(norm, dtype=np.float32)
        self.x = torch.empty((n, ny, nx, 16), dtype=torch.bfloat16, device="cuda")
        self.t = torch.empty((n, ny, nx, 16), dtype=torch.float32, device="cuda")
        for j in range(n):
            normalize(self.raw0[j], self.norm, self.x[j])
            target(self.raw0[j], self.raw1[j], self.norm, self.t[j])
        torch.cuda.synchronize()
        self.n = n
        self.shape = (ny, nx)


def train(data: Dataset, batch: int = 4, seconds: float = 60.0, max_steps: int = 100000, lr: float = 1e-3,
          seed: int = 0, net=None, log=None):
    """Adam on minibatches of the dataset (seeded order) for a time budget; returns the network
    and the loss history.  The minibatch is gathered on the device by plain copies."""
    import time
    import torch
    ny, nx = data.shape
    if net is None:
        net = lb.Net(batch, ny, nx, seed=seed)
    rng = np.random.Generator(np.random.PCG64(seed + 77))
    xb = torch.empty((batch, ny, nx, 16), dtype=torch.bfloat16, device="cuda")
    tb = torch.empty((batch, ny, nx, 16), dtype=torch.float32, device="cuda")
    losses = []
    t0 = time.perf_counter()
    step = 0
    while step < max_steps and time.perf_counter() - t0 < seconds:
        idx = rng.integers(0, data.n, size=batch)
        for b, j in enumerate(idx):
            xb[b].copy_(data.x[int(j)])
            tb[b].copy_(data.t[int(j)])
        # cosine decay over the budget
        frac = min(1.0, (time.perf_counter() - t0) / seconds)
        lr_k = lr * 0.5 * (1.0 + np.cos(np.pi * frac))
        losses.append(net.train_step(xb, tb, OUT_MASK, max(lr_k, lr * 0.02)))
        step += 1
        if log and step % 50 == 0:
            log("step %d loss %.4f" % (step, losses[-1]))
    return net, losses


def evaluate(net, data: Dataset, idx) -> float:
    """Mean loss of the network over the given pairs (forward only, in batches of the net's
    batch size; a short last batch is padded with the first pair and not counted)."""
    import torch
    ny, nx = data.shape
    B = net.B
    xb = torch.empty((B, ny, nx, 16), dtype=torch.bfloat16, device="cuda")
    tb = torch.empty((B, ny, nx, 16), dtype=torch.float32, device="cuda")
    idx = list(idx)
    total, count = 0.0, 0
    for k in range(0, len(idx), B):
        chunk = idx[k:k + B]
        for b in range(B):
            j = chunk[b] if b < len(chunk) else chunk[0]
            xb[b].copy_(data.x[j])
            tb[b].copy_(data.t[j])
        net.forward(xb)
        # the loss of a padded batch counts the padding once per pad; weight by the real share
        total += net.mse(tb, OUT_MASK) * len(chunk)
        count += len(chunk)
    return total / max(count, 1)


def inference_net(trained, ny: int, nx: int):
    """A batch-1 network with the trained parameters."""
    net = lb.Net(1, ny, nx, seed=0)
    net.set_params(trained.params())
    return net


def run(workload, net=None, norm=None, calls: int = 32, eps=(0.25, 0.5), warmup: int = 32):
    """One trajectory: warm-up plain steps, then `calls` x 16 steps learned (net given) or plain;
    returns (restoring-force series of the ring, device ms of the timed part, stepper stats)."""
    import torch
    s = lb.Solver.from_workload(workload)
    s.step(warmup)
    s.sync()
    st = Stepper(s, net, norm, eps[0], eps[1]) if net is not None else None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    if st:
        st.step(calls)
    else:
        s.step(calls * JUMP)
    e1.record()
    s.sync()
    torch.cuda.synchronize()
    out = (s.series()[:, 6:8], e0.elapsed_time(e1), st.stats() if st else None)
    if st:
        st.close()
    s.close()
    return out


def calibrate(net, norm, workload, calls: int = 32, target_err: float = 1e-2,
              grid=(0.02, 0.05, 0.1, 0.2, 0.5, 1.0, 2.0, 5.0, 20.0, 100.0)):
    """Residual bounds fixed on a validation trajectory: of the (eps_momentum, eps_tendency)
    pairs on the grid whose run keeps the restoring force within target_err (relative L2 over
    the readouts) of the plain solver, the one that accepts the most calls (ties: the tighter
    bounds).  Returns (eps, accepted, error), or the tightest pair with 0 accepted if none
    accepts a call within the bound."""
    ref, _, _ = run(workload, calls=calls)
    nref = np.linalg.norm(ref)
    best = ((grid[0], grid[0]), 0, 0.0)
    for em in grid:
        for et in grid:
            fr, _, stt = run(workload, net, norm, calls=calls, eps=(em, et))
            err = float(np.linalg.norm(fr - ref) / nref)
            if err <= target_err and stt["accepted"] > best[1]:
                best = ((em, et), stt["accepted"], err)
    return best


class Stepper:
    """lb_learned_*: 16 lattice steps per call with the plain solver as check and fallback."""

    def __init__(self, solver, net, norm, eps_momentum: float = 0.25, eps_tendency: float = 0.5):
        self.solver, self.net = solver, net
        self.norm = np.ascontiguousarray(norm, dtype=np.float32)
        self.L = lb._L()
        rc = lb.lib().lb_learned_create(solver.h, net.n, self.norm.ctypes.data, eps_momentum, eps_tendency,
                                        ctypes.byref(self.L))
        if rc != lb.LB_OK:
            raise lb.LBError(rc, "lb_learned_create failed")

    def step(self, calls: int) -> int:
        fb = ctypes.c_int64(0)
        rc = lb.lib().lb_learned_step(self.L, int(calls), ctypes.byref(fb))
        if rc != lb.LB_OK:
            raise lb.LBError(rc, lb.lib().lb_learned_last_error(self.L).decode())
        return fb.value

    def stats(self) -> dict:
        out = np.zeros(4)
        lb.lib().lb_learned_stats(self.L, out.ctypes.data)
        return {"r_momentum": out[0], "r_tendency": out[1], "calls": int(out[2]), "accepted": int(out[3])}

    def close(self):
        if self.L:
            lb.lib().lb_learned_destroy(self.L)
            self.L = lb._L()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
