"""Pins of the FP64 network oracle (oracle/unet.py): the convolution against scipy's 2-D
correlation, every backward against central finite differences and adjointness, and the
whole network's gradient against finite differences on an 8 x 8 input."""
import numpy as np
import pytest

from oracle import unet as U


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def test_conv_matches_scipy_correlate():
    signal = pytest.importorskip("scipy.signal")
    r = rng(1)
    x = r.normal(size=(2, 7, 9, 5))
    w = r.normal(size=(9, 4, 5))
    b = r.normal(size=4)
    y = U.conv3x3(x, w, b)
    for bi in range(2):
        for o in range(4):
            ref = np.full((7, 9), b[o])
            for c in range(5):
                k = w[:, o, c].reshape(3, 3)             # k[dy + 1, dx + 1]
                ref += signal.correlate2d(x[bi, :, :, c], k, mode="same", boundary="fill")
            assert np.allclose(y[bi, :, :, o], ref, rtol=1e-12, atol=1e-12)


def _fd(f, a, idx, h=1e-6):
    a0 = a[idx]
    a[idx] = a0 + h
    fp = f()
    a[idx] = a0 - h
    fm = f()
    a[idx] = a0
    return (fp - fm) / (2 * h)


def test_conv_backward_finite_differences():
    r = rng(2)
    x = r.normal(size=(2, 5, 6, 3))
    w = r.normal(size=(9, 4, 3))
    b = r.normal(size=4)
    g = r.normal(size=(2, 5, 6, 4))
    loss = lambda: float((U.conv3x3(x, w, b) * g).sum())
    gx, gw, gb = U.conv3x3_bwd(x, w, g)
    for idx in [(0, 0, 0, 0), (1, 4, 5, 2), (0, 2, 3, 1), (1, 0, 5, 0)]:
        assert abs(_fd(loss, x, idx) - gx[idx]) < 1e-6
    for idx in [(0, 0, 0), (4, 3, 2), (8, 1, 1), (2, 2, 0)]:
        assert abs(_fd(loss, w, idx) - gw[idx]) < 1e-6
    for idx in [(0,), (3,)]:
        assert abs(_fd(loss, b, idx) - gb[idx]) < 1e-6


def test_adjointness_of_conv_pool_up():
    r = rng(3)
    x = r.normal(size=(1, 8, 8, 3))
    w = r.normal(size=(9, 2, 3))
    g = r.normal(size=(1, 8, 8, 2))
    gx, _, _ = U.conv3x3_bwd(x, w, g)
    assert np.isclose((U.conv3x3(x, w, np.zeros(2)) * g).sum(), (x * gx).sum(), rtol=1e-12)
    gp = r.normal(size=(1, 4, 4, 3))
    assert np.isclose((U.pool2(x) * gp).sum(), (x * U.pool2_bwd(gp)).sum(), rtol=1e-12)
    gu = r.normal(size=(1, 16, 16, 3))
    assert np.isclose((U.up2(x) * gu).sum(), (x * U.up2_bwd(gu)).sum(), rtol=1e-12)
    # pooling a constant keeps it; upsampling then pooling is the identity
    assert np.allclose(U.pool2(U.up2(x)), x)


def test_leaky_and_mse_gradients():
    r = rng(4)
    z = r.normal(size=(3, 4))
    g = r.normal(size=(3, 4))
    y = U.leaky(z)
    gz = U.leaky_bwd(y, g)
    for idx in [(0, 0), (1, 2), (2, 3)]:
        assert abs(_fd(lambda: float((U.leaky(z) * g).sum()), z, idx) - gz[idx]) < 1e-6
    p = r.normal(size=(1, 2, 2, 4))
    t = r.normal(size=(1, 2, 2, 4))
    mask = np.array([1.0, 1.0, 0.0, 1.0])
    val, gp = U.mse(p, t, mask)
    assert np.isclose(val, (((p - t) * mask) ** 2).sum() / (4 * 3))
    for idx in [(0, 0, 0, 0), (0, 1, 1, 3), (0, 1, 0, 2)]:
        assert abs(_fd(lambda: U.mse(p, t, mask)[0], p, idx) - gp[idx]) < 1e-7


def test_network_gradient_finite_differences():
    P = U.init_params(seed=5)
    r = rng(6)
    x = r.normal(size=(1, 8, 8, U.C_IN))
    g = r.normal(size=(1, 8, 8, U.C_OUT))
    y, cache = U.forward(P, x)
    assert y.shape == (1, 8, 8, U.C_OUT)
    G, gx = U.backward(P, cache, g)
    loss = lambda: float((U.forward(P, x)[0] * g).sum())
    checks = [("e0a.w", (4, 3, 2)), ("e1b.w", (0, 5, 7)), ("bta.w", (8, 100, 90)),
              ("d2a.w", (2, 10, 200)), ("d1a.w", (6, 3, 150)), ("d0a.w", (7, 30, 70)),
              ("head.w", (4, 2, 17)), ("e2b.b", (50,)), ("head.b", (3,))]
    for name, idx in checks:
        fd = _fd(loss, P[name], idx)
        assert abs(fd - G[name][idx]) <= 1e-5 * max(1.0, abs(fd)), (name, fd, G[name][idx])
    for idx in [(0, 0, 0, 0), (0, 7, 3, 9), (0, 4, 4, 15)]:
        fd = _fd(loss, x, idx)
        assert abs(fd - gx[idx]) <= 1e-5 * max(1.0, abs(fd)), (idx, fd, gx[idx])


def test_bf16_rounding_matches_library_and_ties_to_even():
    torch = pytest.importorskip("torch")
    r = rng(7)
    a = np.concatenate([r.normal(size=1000) * 10.0 ** r.integers(-20, 20, size=1000),
                        [0.0, -0.0, 1.0, -3.5, 65504.0, 1e-38]]).astype(np.float32)
    ref = torch.tensor(a).to(torch.bfloat16).float().numpy().astype(np.float64)
    assert np.array_equal(U.round_bf16(a), ref)
    # ties: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7 and rounds to the even 1;
    # 1 + 3 * 2^-8 rounds up to the even 1 + 2^-6
    assert U.round_bf16(np.float32(1 + 2 ** -8)) == 1.0
    assert U.round_bf16(np.float32(1 + 3 * 2 ** -8)) == 1 + 2 ** -6


def test_rounded_network_reduces_to_exact_one_without_rounding():
    P = U.init_params(seed=2)
    x = rng(3).normal(size=(1, 8, 8, U.C_IN))
    y0, c0 = U.forward(P, x)
    y1, c1 = U.forward(P, x, q=lambda v: v)
    assert np.array_equal(y0, y1)
    yq, _ = U.forward(P, x, q=U.round_bf16)
    assert 0 < np.linalg.norm(yq - y0) / np.linalg.norm(y0) < 2e-2
