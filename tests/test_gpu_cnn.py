"""The learned-guess network on the GPU (tcgen05 BF16 kernels) against its
CPU reference (oracle/cnn_oracle.py).

Each layer is compared on the GPU's own BF16 input, so the only differences
are accumulation order (FP32 on the GPU, FP64 in the reference) and the BF16
rounding decisions that order can flip: stored activations agree to one BF16
ulp (and almost all exactly), the FP32 output to 1e-5 relative, parameter
gradients to 1e-3 of their largest magnitude per layer.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import cnn_oracle as co  # noqa: E402


def _net(B, H, W, params, dil=co.DILATIONS):
    from paper_1111_0983_gb300 import cnn
    net = cnn.Net(B, H, W, dil)
    net.set_params(cnn.pack_params(params))
    return net


def _params(seed):
    rng = np.random.default_rng(seed)
    return [(w, rng.standard_normal(b.shape) * 0.1) for w, b in co.init_params(seed)]


def _acts(net, B, H, W):
    out = []
    for l in range(6):
        a = torch.zeros((B, 4 if l == 0 else 32, H, W), dtype=torch.float32, device="cuda")
        net.activation(l, a)
        out.append(a.cpu().numpy().astype(np.float64))
    return out


@pytest.mark.parametrize("B,H,W,dil", [(2, 40, 37, co.DILATIONS), (1, 129, 129, (1, 1, 2, 3, 1, 1)),
                                       (3, 17, 150, (2, 4, 1, 16, 8, 1))])
def test_forward_layers_match_reference(B, H, W, dil):
    from paper_1111_0983_gb300 import cnn
    params = _params(B + H)
    net = _net(B, H, W, params, dil)
    rng = np.random.default_rng(H)
    x = rng.standard_normal((B, 4, H, W)).astype(np.float32)
    out = torch.zeros((B, 2, H, W), dtype=torch.float32, device="cuda")
    net.forward(torch.from_numpy(x).cuda(), out)
    acts = _acts(net, B, H, W)
    assert np.array_equal(acts[0], co.bf16_round(x))
    P = cnn.unpack_params(cnn.pack_params(params))
    for l in range(6):
        w, b = P[l]
        z = co.conv3x3(acts[l], co.bf16_round(w), b, dil[l])
        if l < 5:
            ref = co.bf16_round(np.maximum(z, 0.0).astype(np.float32))
            got = acts[l + 1]
            d = np.abs(got - ref)
            # one BF16 step of the larger value, plus the FP32 accumulation
            # error (1e-6 of the sum of absolute products) where the ReLU
            # clamps a sum that lies within rounding of zero
            S = co.conv3x3(np.abs(acts[l]), np.abs(co.bf16_round(w)), np.zeros_like(b), dil[l])
            assert np.all(d <= 2.0 ** -7 * np.maximum(np.abs(ref), np.abs(got)) + 1e-6 * S), l
            assert (d > 0).mean() < 1e-3, l         # almost all exact
        else:
            got = out.cpu().numpy()
            assert np.abs(got - z).max() <= 1e-5 * np.abs(z).max()


def test_backward_matches_reference():
    from paper_1111_0983_gb300 import cnn
    B, H, W = 2, 48, 45
    params = _params(7)
    net = _net(B, H, W, params)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((B, 4, H, W)).astype(np.float32)
    out = torch.zeros((B, 2, H, W), dtype=torch.float32, device="cuda")
    net.forward(torch.from_numpy(x).cuda(), out)
    acts = _acts(net, B, H, W)
    dout = rng.standard_normal((B, 2, H, W)).astype(np.float32)
    g = torch.zeros(cnn.num_params(), dtype=torch.float32, device="cuda")
    net.backward(torch.from_numpy(dout).cuda(), g)
    got = cnn.unpack_params(g.cpu().numpy())
    ref = co.CnnOracle(cnn.unpack_params(cnn.pack_params(params))).backward(acts, dout.astype(np.float64))
    for l in range(6):
        for a, r in zip(got[l], ref[l]):
            assert np.abs(a - r).max() <= 1e-3 * np.abs(r).max(), l


def test_train_step_reduces_a_fitting_loss():
    """Adam on the masked squared error: the GPU's loss before each step
    equals the reference loss of its own output, and fitting a fixed smooth
    target lowers it."""
    from paper_1111_0983_gb300 import cnn
    B, H, W = 2, 64, 64
    params = _params(11)
    net = _net(B, H, W, params)
    rng = np.random.default_rng(5)
    x = torch.from_numpy(rng.standard_normal((B, 4, H, W)).astype(np.float32)).cuda()
    yy, xx = np.meshgrid(np.linspace(-1, 1, H), np.linspace(-1, 1, W), indexing="ij")
    t = np.zeros((B, 2, H, W), np.float32)
    t[:, 0] = np.sin(2 * xx) * np.cos(yy)
    m = np.zeros_like(t)
    m[:, 0] = 1.0
    td, md = torch.from_numpy(t).cuda(), torch.from_numpy(m).cuda()
    out = torch.zeros((B, 2, H, W), dtype=torch.float32, device="cuda")
    net.forward(x, out)
    l_ref = co.masked_mse(out.cpu().numpy().astype(np.float64), t, m)[0]
    losses = [net.train_step(x, td, md, float(m.sum()), 3e-3) for _ in range(60)]
    assert abs(losses[0] - l_ref) <= 1e-5 * l_ref
    assert losses[-1] < 0.2 * losses[0], losses[::10]
    # with the residual term (mask channel 1: the pixels where it is taken)
    m2 = m.copy()
    m2[:, 1] = (np.random.default_rng(2).uniform(size=(B, H, W)) < 0.5).astype(np.float32)
    net.forward(x, out)
    o = out.cpu().numpy().astype(np.float64)
    l_lap, _ = co.laplacian_loss(o, t, m2, 50.0)
    inner = float((m2[:, 1, 1:-1, 1:-1] > 0).sum())
    l_ref = co.masked_mse(o, t, m)[0] + l_lap
    got = net.train_step(x, td, torch.from_numpy(m2).cuda(), float(m.sum()), 1e-4, 50.0, inner)
    assert abs(got - l_ref) <= 1e-4 * l_ref
