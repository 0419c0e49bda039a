"""Pins of the learned-guess network's CPU reference (oracle/cnn_oracle.py):
BF16 rounding against torch's own conversion, the dilated convolution
against scipy's 2D correlation, the backward pass against central finite
differences of the loss, and the BF16 mode against the exact network."""
import numpy as np
import pytest

from oracle import cnn_oracle as cnn


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-6, 6, 10000),
                        # exact ties between two BF16 values, both parities
                        (np.arange(1, 200) * 2 + 1) * 2.0 ** -8 + 1.0])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cnn.bf16_round(x), ref)


@pytest.mark.parametrize("d", [1, 2, 5])
def test_conv_matches_scipy_correlation(d):
    sig = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(d)
    x = rng.standard_normal((2, 3, 17, 13))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    z = cnn.conv3x3(x, w, b, d)
    for n in range(2):
        for o in range(4):
            ref = np.full((17, 13), b[o])
            for c in range(3):
                k = np.zeros((2 * d + 1, 2 * d + 1))
                k[::d, ::d] = w[o, c]          # the dilated 3x3 kernel
                ref += sig.correlate2d(x[n, c], k, mode="same", boundary="fill")
            assert np.abs(z[n, o] - ref).max() < 1e-12


def _loss(net, x, t, m):
    out, _ = net.forward(x)
    return cnn.masked_mse(out, t, m)[0]


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(5)
    params = cnn.init_params(3)
    params = [(w, rng.standard_normal(b.shape) * 0.1) for w, b in params]
    dil = (1, 2, 1, 3, 2, 1)
    net = cnn.CnnOracle(params, dil, bf16=False)
    x = rng.standard_normal((2, 4, 11, 10))
    t = rng.standard_normal((2, 2, 11, 10))
    m = (rng.uniform(size=(2, 2, 11, 10)) < 0.7).astype(float)
    out, acts = net.forward(x)
    _, dout = cnn.masked_mse(out, t, m)
    grads = net.backward(acts, dout)
    eps = 1e-6
    for l in range(6):
        w, b = net.params[l]
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in w.shape)
            w0 = w[idx]
            w[idx] = w0 + eps
            lp = _loss(net, x, t, m)
            w[idx] = w0 - eps
            lm = _loss(net, x, t, m)
            w[idx] = w0
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - grads[l][0][idx]) <= 1e-6 * max(1.0, abs(fd)), (l, idx, fd, grads[l][0][idx])
        o = int(rng.integers(0, b.shape[0]))
        b0 = b[o]
        b[o] = b0 + eps
        lp = _loss(net, x, t, m)
        b[o] = b0 - eps
        lm = _loss(net, x, t, m)
        b[o] = b0
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - grads[l][1][o]) <= 1e-6 * max(1.0, abs(fd)), (l, o)


def test_bf16_mode_is_close_to_exact():
    rng = np.random.default_rng(8)
    params = cnn.init_params(1)
    x = rng.standard_normal((1, 4, 20, 20))
    ex, _ = cnn.CnnOracle(params, bf16=False).forward(x)
    bf, acts = cnn.CnnOracle(params, bf16=True).forward(x)
    assert np.abs(bf - ex).max() < 0.05 * np.abs(ex).max()
    for a in acts:    # every stored activation is a BF16 value
        assert np.array_equal(a, cnn.bf16_round(a))


def test_laplacian_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(9)
    out = rng.standard_normal((2, 2, 9, 8))
    t = rng.standard_normal((2, 2, 9, 8))
    m = np.zeros((2, 2, 9, 8))
    m[:, 0] = rng.uniform(size=(2, 9, 8)) < 0.8
    m[:, 1] = (rng.uniform(size=(2, 9, 8)) < 0.6) * m[:, 0]
    L, g = cnn.laplacian_loss(out, t, m, 3.0)
    # closed form: a unit error at one node, the term taken at that node
    # only: s = -4 there, L = 16
    e = np.zeros_like(out)
    e[0, 0, 4, 4] = 1.0
    mm = np.zeros_like(m)
    mm[0, 0] = 1.0
    mm[0, 1, 4, 4] = 1.0
    assert abs(cnn.laplacian_loss(e, 0 * e, mm, 1.0)[0] - 16.0) < 1e-12
    eps = 1e-6
    for _ in range(20):
        idx = tuple(rng.integers(0, s) for s in out.shape)
        o0 = out[idx]
        out[idx] = o0 + eps
        lp = cnn.laplacian_loss(out, t, m, 3.0)[0]
        out[idx] = o0 - eps
        lm = cnn.laplacian_loss(out, t, m, 3.0)[0]
        out[idx] = o0
        assert abs((lp - lm) / (2 * eps) - g[idx]) <= 1e-6 * max(1.0, abs(g[idx]))
