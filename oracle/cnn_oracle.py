"""CPU reference of the learned initial-guess network (test infrastructure).

Only tests, the smoke check and the benchmark's CPU baseline may use this
module; the product path never calls it.

The paper has no learned part: this network is the data-driven initial guess
that the multigrid solve starts from.  Six 3x3 convolution layers with
channels 4 -> 32 -> 32 -> 32 -> 32 -> 32 -> 2, ReLU after the first five, zero
padding ("same" size), dilation d_l per layer.  Images are NCHW, weights
[C_out][C_in][3][3], biases [C_out].

``bf16=True`` reproduces the rounding points of the GPU path (BF16 operands,
FP32 accumulation): the input, every weight tensor and every hidden
activation are rounded to BF16 (round to nearest even), the output stays
FP32; in the backward pass the gradient entering each layer is rounded to
BF16 (after the ReLU mask), weight and bias gradients are accumulated
exactly.  Accumulation here is FP64, so GPU and reference differ only by
accumulation order and by BF16 rounding decisions that order can flip.
``bf16=False`` is the exact FP64 network (for finite-difference checks).
"""
import numpy as np

LAYERS = [(4, 32), (32, 32), (32, 32), (32, 32), (32, 32), (32, 2)]
DILATIONS = (1, 3, 9, 27, 81, 1)


def bf16_round(x):
    """Round to the nearest BF16 value, ties to even (via FP32), as FP64."""
    x32 = np.ascontiguousarray(x, dtype=np.float32)
    u = x32.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def conv3x3(x, w, b, d):
    """z[n,o,i,j] = b[o] + sum_{c,ki,kj} w[o,c,ki,kj] x[n,c,i+(ki-1)d,j+(kj-1)d],
    zero outside the image."""
    n, c, h, wd = x.shape
    xp = np.zeros((n, c, h + 2 * d, wd + 2 * d))
    xp[:, :, d:d + h, d:d + wd] = x
    z = np.zeros((n, w.shape[0], h, wd))
    for ki in range(3):
        for kj in range(3):
            xs = xp[:, :, ki * d:ki * d + h, kj * d:kj * d + wd]
            z += np.einsum("oc,nchw->nohw", w[:, :, ki, kj], xs)
    return z + b[None, :, None, None]


def conv3x3_backward(x, w, dz, d):
    """Gradients of conv3x3 with respect to w, b and x given dz = dL/dz."""
    n, c, h, wd = x.shape
    xp = np.zeros((n, c, h + 2 * d, wd + 2 * d))
    xp[:, :, d:d + h, d:d + wd] = x
    dw = np.zeros_like(w)
    dxp = np.zeros_like(xp)
    for ki in range(3):
        for kj in range(3):
            xs = xp[:, :, ki * d:ki * d + h, kj * d:kj * d + wd]
            dw[:, :, ki, kj] = np.einsum("nohw,nchw->oc", dz, xs)
            dxp[:, :, ki * d:ki * d + h, kj * d:kj * d + wd] += np.einsum("oc,nohw->nchw", w[:, :, ki, kj], dz)
    db = dz.sum(axis=(0, 2, 3))
    return dw, db, dxp[:, :, d:d + h, d:d + wd]


def init_params(seed=0):
    """He-initialised weights, zero biases (FP32 values as FP64)."""
    rng = np.random.default_rng(seed)
    out = []
    for ci, co in LAYERS:
        w = rng.standard_normal((co, ci, 3, 3)) * np.sqrt(2.0 / (9 * ci))
        out.append((w.astype(np.float32).astype(np.float64), np.zeros(co)))
    return out


class CnnOracle:
    def __init__(self, params, dilations=DILATIONS, bf16=True):
        self.params = [(np.asarray(w, np.float64), np.asarray(b, np.float64)) for w, b in params]
        self.dil = tuple(dilations)
        self.bf16 = bf16

    def _r(self, x):
        return bf16_round(x) if self.bf16 else x

    def forward(self, x):
        """Returns (out [N,2,H,W], cache).  x: [N,4,H,W]."""
        a = self._r(np.asarray(x, np.float64))
        acts = [a]
        for l, (w, b) in enumerate(self.params):
            z = conv3x3(a, self._r(w), b, self.dil[l])
            if l + 1 < len(self.params):
                a = np.maximum(z, 0.0)
                if self.bf16:
                    a = bf16_round(a.astype(np.float32))
                acts.append(a)
            else:
                out = z.astype(np.float32).astype(np.float64) if self.bf16 else z
        return out, acts

    def backward(self, acts, dout):
        """Parameter gradients [(dw, db)] for dL/dout = dout."""
        dz = self._r(np.asarray(dout, np.float64))
        grads = [None] * len(self.params)
        for l in range(len(self.params) - 1, -1, -1):
            w, _ = self.params[l]
            dw, db, dx = conv3x3_backward(acts[l], self._r(w), dz, self.dil[l])
            grads[l] = (dw, db)
            if l > 0:
                g = dx * (acts[l] > 0)
                dz = bf16_round(g.astype(np.float32)) if self.bf16 else g
        return grads


def masked_mse(out, target, mask):
    """L = sum(mask * (out - target)^2) / sum(mask) over all channels given
    (target, mask: [N,C,H,W]); returns (L, dL/dout)."""
    cnt = max(float(mask.sum()), 1.0)
    diff = (out - target) * mask
    return float((diff * diff).sum() / cnt), 2.0 * diff / cnt


def laplacian_loss(out, target, mask, beta):
    """Residual term of the training loss: with e = (out_0 - target_0) m_0 (the
    error of channel 0 on the unknowns), s = e_N + e_S + e_E + e_W - 4 e (h^2
    times the 5-point Laplacian) at the nodes where m_1 = 1 (away from the
    image edge), L = beta sum(s^2) / sum(m_1); returns (L, dL/dout)."""
    e = (out[:, 0] - target[:, 0]) * mask[:, 0]
    inner = np.zeros_like(e, dtype=bool)
    inner[:, 1:-1, 1:-1] = mask[:, 1, 1:-1, 1:-1] > 0
    s = np.zeros_like(e)
    s[:, 1:-1, 1:-1] = (e[:, :-2, 1:-1] + e[:, 2:, 1:-1] + e[:, 1:-1, :-2] + e[:, 1:-1, 2:]
                        - 4.0 * e[:, 1:-1, 1:-1])
    s = np.where(inner, s, 0.0)
    cnt = max(float(inner.sum()), 1.0)
    g = -4.0 * s
    g[:, 1:, :] += s[:, :-1, :]
    g[:, :-1, :] += s[:, 1:, :]
    g[:, :, 1:] += s[:, :, :-1]
    g[:, :, :-1] += s[:, :, 1:]
    dout = np.zeros_like(out)
    dout[:, 0] = 2.0 * beta / cnt * g * mask[:, 0]
    return float(beta * (s * s).sum() / cnt), dout
