"""FP64 CPU oracle of the learned time-stepper's network (the U-Net of the learned form).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU legs may import it; the product path never does.

Plain numpy in FP64, written from the definitions:
  * 3x3 convolution, stride 1, zero padding 1, NHWC activations x[B, H, W, Ci], weights
    w[9, Co, Ci] with tap t = (dy + 1) * 3 + (dx + 1), bias b[Co]:
        y[b, i, j, o] = b[o] + sum_{dy, dx, c} x[b, i + dy, j + dx, c] w[t(dy, dx), o, c];
  * LeakyReLU with slope 0.1 on the negative side;
  * 2x2 average pooling and nearest-neighbour 2x upsampling;
  * channel concatenation (the skip connections);
  * mean squared error.
Every backward is the transpose of its forward, written out; the tests pin them by finite
differences and by adjointness, and the forward convolution by scipy's correlate.

The network (fixed): 4 levels at full, 1/2, 1/4, 1/8 resolution with 32, 64, 96, 128 channels;
two conv + LeakyReLU per level on the way down, average pooling between levels, nearest
upsampling + concatenation with the skip + two conv + LeakyReLU on the way up, and a final
3x3 conv to 16 output channels without activation.  Input 16 channels (7 fields, a body
indicator, zero padding).
"""
from __future__ import annotations

import numpy as np

SLOPE = 0.1
# (name, Ci, Co, activation) in execution order; "pool" / "up+cat:<skip>" are the joins
LAYERS = [
    ("e0a", 16, 32, True), ("e0b", 32, 32, True),
    ("e1a", 32, 64, True), ("e1b", 64, 64, True),
    ("e2a", 64, 96, True), ("e2b", 96, 96, True),
    ("bta", 96, 128, True), ("btb", 128, 128, True),
    ("d2a", 128 + 96, 96, True), ("d2b", 96, 96, True),
    ("d1a", 96 + 64, 64, True), ("d1b", 64, 64, True),
    ("d0a", 64 + 32, 32, True), ("d0b", 32, 32, True),
    ("head", 32, 16, False),
]
C_IN, C_OUT = 16, 16


# ---------------------------------------------------------------- elementary operations

def round_bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as FP64: the FP32 value's upper
    16 bits after adding 0x7FFF + (bit 16) to its bit pattern (finite inputs)."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def conv3x3(x, w, b):
    B, H, W, Ci = x.shape
    Co = w.shape[1]
    xp = np.zeros((B, H + 2, W + 2, Ci))
    xp[:, 1:-1, 1:-1] = x
    y = np.broadcast_to(b, (B, H, W, Co)).astype(np.float64).copy()
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            t = (dy + 1) * 3 + (dx + 1)
            xs = xp[:, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
            y += np.einsum("bhwc,oc->bhwo", xs, w[t])
    return y


def conv3x3_bwd(x, w, gy):
    """Gradients (gx, gw, gb) of sum(gy * conv3x3(x, w, b))."""
    B, H, W, Ci = x.shape
    xp = np.zeros((B, H + 2, W + 2, Ci))
    xp[:, 1:-1, 1:-1] = x
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w, dtype=np.float64)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            t = (dy + 1) * 3 + (dx + 1)
            xs = xp[:, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
            gw[t] = np.einsum("bhwo,bhwc->oc", gy, xs)
            gxp[:, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W] += np.einsum("bhwo,oc->bhwc", gy, w[t])
    gb = gy.sum(axis=(0, 1, 2))
    return gxp[:, 1:-1, 1:-1], gw, gb


def leaky(x):
    return np.where(x > 0, x, SLOPE * x)


def leaky_bwd(y, gy):
    """Gradient through LeakyReLU given its OUTPUT y (same sign as its input)."""
    return np.where(y > 0, gy, SLOPE * gy)


def pool2(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool2_bwd(gy):
    return np.repeat(np.repeat(gy, 2, axis=1), 2, axis=2) / 4.0


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_bwd(gy):
    B, H, W, C = gy.shape
    return gy.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def mse(pred, target, mask):
    """Mean over the masked (used) channels of (pred - target)^2, and its gradient."""
    d = (pred - target) * mask
    n = pred.shape[0] * pred.shape[1] * pred.shape[2] * mask.sum()
    return float((d * d).sum() / n), 2.0 * d / n


# ---------------------------------------------------------------- the network

def init_params(seed=0):
    """He-style initialisation (weights N(0, 2 / (9 Ci)), zero bias); FP64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    P = {}
    for name, ci, co, act in LAYERS:
        std = np.sqrt(2.0 / (9 * ci)) if act else np.sqrt(1.0 / (9 * ci)) * 0.1
        P[name + ".w"] = rng.normal(0.0, std, size=(9, co, ci))
        P[name + ".b"] = np.zeros(co)
    return P


def forward(P, x, q=None):
    """The network on x[B, H, W, 16] (H, W multiples of 8); returns (y, cache).  q: optional
    rounding applied where a reduced-precision implementation stores a value (every
    activated convolution output and every pooled value); the head output is not rounded."""
    cache = {}
    q = q or (lambda v: v)

    def conv(name, inp, act):
        z = conv3x3(inp, P[name + ".w"], P[name + ".b"])
        out = q(leaky(z)) if act else z
        cache[name] = (inp, out)
        return out

    e0 = conv("e0b", conv("e0a", x, True), True)
    e1 = conv("e1b", conv("e1a", q(pool2(e0)), True), True)
    e2 = conv("e2b", conv("e2a", q(pool2(e1)), True), True)
    bt = conv("btb", conv("bta", q(pool2(e2)), True), True)
    d2 = conv("d2b", conv("d2a", np.concatenate([up2(bt), e2], axis=3), True), True)
    d1 = conv("d1b", conv("d1a", np.concatenate([up2(d2), e1], axis=3), True), True)
    d0 = conv("d0b", conv("d0a", np.concatenate([up2(d1), e0], axis=3), True), True)
    y = conv("head", d0, False)
    return y, cache


def backward(P, cache, gy, q=None):
    """Gradients of sum(gy * forward(P, x)) with respect to every parameter and x.  q: optional
    rounding where a reduced-precision implementation stores a back-propagated gradient (the
    output gradient, every pre-activation gradient, every input gradient of a convolution, of
    an upsampling and of a pooling join); parameter gradients are not rounded."""
    G = {}
    q = q or (lambda v: v)

    def conv_b(name, g_out, act):
        inp, out = cache[name]
        gz = q(leaky_bwd(out, g_out)) if act else g_out
        gx, gw, gb = conv3x3_bwd(inp, P[name + ".w"], gz)
        G[name + ".w"] = gw
        G[name + ".b"] = gb
        return q(gx)

    g = conv_b("head", q(gy), False)
    g = conv_b("d0a", conv_b("d0b", g, True), True)
    g_up, g_e0 = g[..., :64], g[..., 64:]
    g = conv_b("d1a", conv_b("d1b", q(up2_bwd(g_up)), True), True)
    g_up, g_e1 = g[..., :96], g[..., 96:]
    g = conv_b("d2a", conv_b("d2b", q(up2_bwd(g_up)), True), True)
    g_up, g_e2 = g[..., :128], g[..., 128:]
    g = conv_b("bta", conv_b("btb", q(up2_bwd(g_up)), True), True)
    g = conv_b("e2a", conv_b("e2b", q(pool2_bwd(g) + g_e2), True), True)
    g = conv_b("e1a", conv_b("e1b", q(pool2_bwd(g) + g_e1), True), True)
    gx = conv_b("e0a", conv_b("e0b", q(pool2_bwd(g) + g_e0), True), True)
    return G, gx
