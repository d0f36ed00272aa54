"""The learned stepper's network kernels (BF16 tensor cores, FP32 accumulation) against the FP64
network oracle (oracle/unet.py), through the C ABI.

Single kernels take inputs that are exact in BF16, so the oracle sees the same numbers; the
differences are then the FP32 accumulation (relative ~1e-6 over a few hundred products) and,
for BF16 outputs, one final rounding (2^-9 relative).  The whole network rounds every
activation and every back-propagated gradient to BF16 (2^-9 relative each) through 15 layers in
sequence, so it is compared in relative L2 with the bounds derived in the tests.
"""
import numpy as np
import pytest

from oracle import unet as U

pytestmark = pytest.mark.gpu


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_14889_gb300 import lb
    return torch, lb


def bf(torch, a):
    """numpy -> BF16 CUDA tensor, and the BF16-rounded values back as FP64 numpy."""
    t = torch.tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).cuda().contiguous()
    return t, t.float().cpu().numpy().astype(np.float64)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


KERNELS = [0, 1]      # mma.sync tiles, tcgen05 with tensor-memory accumulators


@pytest.fixture(params=KERNELS, ids=["mma_sync", "tcgen05"])
def conv_kernel(request):
    torch, lb = _gpu()
    lb.conv_kernel(request.param)
    yield request.param
    lb.conv_status()
    lb.conv_kernel(1)


@pytest.mark.parametrize("B,H,W,Ci,Co,act", [(2, 16, 32, 32, 48, False), (1, 8, 4, 16, 96, True),
                                             (1, 24, 16, 224, 16, True), (1, 16, 16, 32, 160, False)])
def test_conv_forward_vs_oracle(B, H, W, Ci, Co, act, conv_kernel):
    torch, lb = _gpu()
    r = np.random.Generator(np.random.PCG64(10 + Ci))
    xt, x = bf(torch, r.normal(size=(B, H, W, Ci)))
    wt, w = bf(torch, r.normal(size=(9, Co, Ci)) / np.sqrt(9 * Ci))
    b = r.normal(size=Co).astype(np.float32)
    bt = torch.tensor(b).cuda()
    y = lb.conv3x3(xt, wt, bt, act=act, out_f32=True)
    torch.cuda.synchronize()
    ref = U.conv3x3(x, w, b.astype(np.float64))
    if act:
        ref = U.leaky(ref)
    got = y.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
    # BF16 output: one rounding of the FP32 result
    yb = lb.conv3x3(xt, wt, bt, act=act, out_f32=False)
    torch.cuda.synchronize()
    gotb = yb.float().cpu().numpy()
    assert np.all(np.abs(gotb - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-5 * np.abs(ref).max())


def test_conv_into_channel_slice(conv_kernel):
    # the skip connections write into a channel slice of a wider buffer
    torch, lb = _gpu()
    r = np.random.Generator(np.random.PCG64(3))
    xt, x = bf(torch, r.normal(size=(1, 16, 16, 32)))
    wt, w = bf(torch, r.normal(size=(9, 32, 32)) / 17.0)
    buf = torch.full((1, 16, 16, 96), 7.0, dtype=torch.bfloat16, device="cuda")
    lb.conv3x3(xt, wt, None, act=True, out_f32=False, ldy=96, yoff=64, y=buf)
    torch.cuda.synchronize()
    got = buf.float().cpu().numpy()
    assert np.all(got[..., :64] == 7.0)
    ref = U.leaky(U.conv3x3(x, w, np.zeros(32)))
    assert np.all(np.abs(got[..., 64:] - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-5 * np.abs(ref).max())


@pytest.mark.parametrize("B,H,W,Ci,Co", [(2, 16, 16, 32, 64), (1, 8, 8, 96, 128), (1, 32, 16, 16, 32)])
def test_conv_gradients_vs_oracle(B, H, W, Ci, Co, conv_kernel):
    torch, lb = _gpu()
    r = np.random.Generator(np.random.PCG64(20 + Co))
    xt, x = bf(torch, r.normal(size=(B, H, W, Ci)))
    wt, w = bf(torch, r.normal(size=(9, Co, Ci)) / np.sqrt(9 * Ci))
    gzt, gz = bf(torch, r.normal(size=(B, H, W, Co)))
    gx_ref, gw_ref, gb_ref = U.conv3x3_bwd(x, w, gz)
    gx = lb.conv3x3_dgrad(gzt, wt)
    gw, gb = lb.conv3x3_wgrad(xt, gzt)
    torch.cuda.synchronize()
    gx = gx.float().cpu().numpy()
    assert np.all(np.abs(gx - gx_ref) <= 2.0 ** -8 * np.abs(gx_ref) + 1e-5 * np.abs(gx_ref).max())
    # FP32 sums over B H W pixels
    assert np.abs(gw.cpu().numpy() - gw_ref).max() <= 1e-5 * np.abs(gw_ref).max()
    assert np.abs(gb.cpu().numpy() - gb_ref).max() <= 1e-5 * np.abs(gb_ref).max()


def _flat(P):
    return np.concatenate([np.concatenate([P[n + ".w"].ravel(), P[n + ".b"].ravel()])
                           for n, _, _, _ in U.LAYERS]).astype(np.float32)


def _unflat(v):
    out, k = {}, 0
    for n, ci, co, _ in U.LAYERS:
        out[n + ".w"] = v[k:k + 9 * co * ci].reshape(9, co, ci)
        k += 9 * co * ci
        out[n + ".b"] = v[k:k + co]
        k += co
    return out


def _gpu_cache(net, x, y):
    """The oracle's per-layer (input, output) cache built from the GPU's stored activations."""
    A = {k: net.activation(k).astype(np.float64) for k, _, _ in net.ACTIVATIONS}
    c0, c1, c2 = A["cat0"], A["cat1"], A["cat2"]
    return {"e0a": (x, A["e0a"]), "e0b": (A["e0a"], c0[..., 64:]), "e1a": (A["p1"], A["e1a"]),
            "e1b": (A["e1a"], c1[..., 96:]), "e2a": (A["p2"], A["e2a"]), "e2b": (A["e2a"], c2[..., 128:]),
            "bta": (A["p3"], A["bta"]), "btb": (A["bta"], A["btb"]), "d2a": (c2, A["d2a"]),
            "d2b": (A["d2a"], A["d2b"]), "d1a": (c1, A["d1a"]), "d1b": (A["d1a"], A["d1b"]),
            "d0a": (c0, A["d0a"]), "d0b": (A["d0a"], A["d0b"]), "head": (A["d0b"], y)}


def test_network_forward_and_gradients_vs_oracle(conv_kernel):
    torch, lb = _gpu()
    B, H, W = 2, 32, 32
    P = U.init_params(seed=7)
    for name, _, _, _ in U.LAYERS:          # small random biases exercise the bias paths
        P[name + ".b"] = np.random.Generator(np.random.PCG64(len(name))).normal(0, 0.05, P[name + ".b"].shape)
    net = lb.Net(B, H, W, seed=1)
    flat = _flat(P)
    assert flat.size == net.n_params
    net.set_params(flat)
    # the oracle runs on the weights the GPU multiplies: BF16-rounded (biases stay FP32)
    wq = _unflat(flat.astype(np.float64))
    for name, _, _, _ in U.LAYERS:
        wq[name + ".w"] = torch.tensor(wq[name + ".w"], dtype=torch.float32).to(torch.bfloat16).float().numpy()
    r = np.random.Generator(np.random.PCG64(8))
    xt, x = bf(torch, r.normal(size=(B, H, W, 16)))
    y = net.forward(xt)
    torch.cuda.synchronize()
    y = y.cpu().numpy().astype(np.float64)
    cache = _gpu_cache(net, x, y)
    # (1) layer by layer on the GPU's own inputs: one BF16 rounding of an FP32 accumulation, so
    # a value differs from the oracle's only where FP32 and FP64 round to different BF16
    # neighbours (one ulp, 2^-8 relative, in a small fraction of the elements)
    for name, _, _, act in U.LAYERS:
        inp, out = cache[name]
        z = U.conv3x3(inp, wq[name + ".w"], wq[name + ".b"])
        ref = U.round_bf16(U.leaky(z)) if act else z
        e = rel_l2(out, ref)
        assert e < (1e-3 if act else 1e-5), (name, e)
        if act:
            assert np.mean(out != ref) < 0.02, name
    # the joins: pooled and upsampled copies
    assert np.array_equal(cache["e1a"][0], U.round_bf16(U.pool2(cache["e0b"][1])))
    assert np.array_equal(cache["d0a"][0][..., :64], U.up2(cache["d1b"][1]))
    # (2) end to end against the independent rounded oracle: the per-layer differences above
    # carried through 15 layers
    yref, _ = U.forward(wq, x, q=U.round_bf16)
    assert rel_l2(y, yref) < 8e-3
    # (3) gradients on the same forward state (LeakyReLU's derivative jumps at 0, so the
    # activation masks must be the GPU's): the back-propagated gradients are rounded to BF16 at
    # the same places on both sides
    g = r.normal(size=(B, H, W, 16)).astype(np.float32)
    net.backward(torch.tensor(g).cuda())
    torch.cuda.synchronize()
    G, _ = U.backward(wq, cache, g.astype(np.float64), q=U.round_bf16)
    got = _unflat(net.grads().astype(np.float64))
    errs = {n + p: rel_l2(got[n + p], G[n + p]) for n, _, _, _ in U.LAYERS for p in (".w", ".b")}
    assert max(errs.values()) < 5e-3, " ".join("%s=%.1e" % kv for kv in errs.items())


def _bf16_output_bound(P, x, seed=11):
    """First-order bound on the relative L2 error of the network's output when every weight and
    every stored activation (each activated convolution output and each pooled value) carries a
    relative rounding error of at most u = 2^-9 (BF16 keeps 8 significant bits; round to nearest).
    For each such tensor the unrounded FP64 network is run with that tensor alone scaled by
    (1 + u s), s = +-1 at random per element, and the output changes are added: to first order
    the errors of different tensors add, and their sum bounds the combined error.  It needs no
    knowledge of where a kernel rounds beyond what the BF16 format stores."""
    u = 2.0 ** -9
    r = np.random.Generator(np.random.PCG64(seed))
    y0, _ = U.forward(P, x)
    total = 0.0
    n_points = 17        # 14 activated convolution outputs and 3 pooled tensors, in call order
    for k in range(n_points):
        calls = [0]

        def q(v, k=k):
            hit = calls[0] == k
            calls[0] += 1
            return v * (1.0 + u * r.choice([-1.0, 1.0], size=v.shape)) if hit else v
        yk, _ = U.forward(P, x, q=q)
        assert calls[0] == n_points
        total += np.linalg.norm(yk - y0)
    for name, _, _, _ in U.LAYERS:
        Pk = dict(P)
        Pk[name + ".w"] = P[name + ".w"] * (1.0 + u * r.choice([-1.0, 1.0], size=P[name + ".w"].shape))
        yk, _ = U.forward(Pk, x)
        total += np.linalg.norm(yk - y0)
    return y0, total / np.linalg.norm(y0)


def test_network_forward_vs_unrounded_fp64_within_derived_bound(conv_kernel):
    # The GPU network (BF16 weights and activations, FP32 accumulation) against the FP64 network
    # with no rounding at all, on the FP32 weights before their BF16 rounding: the difference
    # must stay within the first-order bound of BF16 storage derived above.  This check does not
    # rely on the rounded oracle reproducing the kernels' rounding points.
    torch, lb = _gpu()
    B, H, W = 2, 32, 32
    P = U.init_params(seed=5)
    for name, _, _, _ in U.LAYERS:
        P[name + ".b"] = np.random.Generator(np.random.PCG64(3 + len(name))).normal(0, 0.05, P[name + ".b"].shape)
    flat = _flat(P).astype(np.float32)
    net = lb.Net(B, H, W, seed=1)
    net.set_params(flat)
    P64 = _unflat(flat.astype(np.float64))
    r = np.random.Generator(np.random.PCG64(12))
    xt, x = bf(torch, r.normal(size=(B, H, W, 16)))
    y = net.forward(xt)
    torch.cuda.synchronize()
    y = y.cpu().numpy().astype(np.float64)
    yref, bound = _bf16_output_bound(P64, x)
    err = rel_l2(y, yref)
    assert 0.0 < err <= bound, (err, bound)
    # the bound is tight enough to catch a fault: one layer's taps mirrored moves the output by
    # far more than it
    Pbad = dict(P64)
    Pbad["d1b.w"] = P64["d1b.w"][::-1].copy()
    ybad, _ = U.forward(Pbad, x)
    assert rel_l2(ybad, yref) > 3 * bound
    net.close()


def test_training_reduces_loss_and_is_deterministic():
    torch, lb = _gpu()
    B, H, W = 2, 32, 32
    r = np.random.Generator(np.random.PCG64(9))
    x = torch.tensor(r.normal(size=(B, H, W, 16)).astype(np.float32)).to(torch.bfloat16).cuda()
    # a smooth target the network can fit: a fixed linear map of the input channels
    A = r.normal(size=(16, 16)).astype(np.float32) / 4.0
    target = (x.float() @ torch.tensor(A).cuda()).contiguous()
    mask = np.ones(16, dtype=np.float32)
    mask[7:] = 0.0
    runs = []
    for _ in range(2):
        net = lb.Net(B, H, W, seed=3)
        losses = [net.train_step(x, target, mask, 2e-3) for _ in range(100)]
        runs.append((losses, net.params()))
        net.close()
    losses = runs[0][0]
    assert losses[-1] < 0.5 * losses[0], (losses[0], losses[-1])
    assert runs[0][0] == runs[1][0]
    assert np.array_equal(runs[0][1], runs[1][1])
