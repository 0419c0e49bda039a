"""Python binding of the learned initial-guess network (include/gcmg_cnn.h):
argument marshalling only; every step runs in libgcmg.so."""
import ctypes as C

import numpy as np

from . import gcmg

LAYERS = [(4, 32), (32, 32), (32, 32), (32, 32), (32, 32), (32, 2)]
DILATIONS = (1, 3, 9, 27, 81, 1)

_bound = False


def _lib():
    global _bound
    L = gcmg.lib()
    if not _bound:
        vp, i32, i64, f32, dbl, st = C.c_void_p, C.c_int, C.c_int64, C.c_float, C.c_double, C.c_int
        sig = {
            "gcmg_cnn_num_params": (i64, []),
            "gcmg_cnn_create": (st, [i32, i32, i32, vp, vp, C.POINTER(vp)]),
            "gcmg_cnn_destroy": (None, [vp]),
            "gcmg_cnn_last_error": (C.c_char_p, [vp]),
            "gcmg_cnn_set_params": (st, [vp, vp, i64]),
            "gcmg_cnn_get_params": (st, [vp, vp, i64]),
            "gcmg_cnn_forward": (st, [vp, vp, vp]),
            "gcmg_cnn_activation": (st, [vp, i32, vp]),
            "gcmg_cnn_backward": (st, [vp, vp, vp]),
            "gcmg_cnn_train_step": (st, [vp, vp, vp, vp, f32, f32, f32, f32, C.POINTER(dbl)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _bound = True
    return L


def num_params():
    return int(_lib().gcmg_cnn_num_params())


def pack_params(params):
    """[(w [co][ci][3][3], b [co])] -> one FP32 vector in the library's order."""
    return np.concatenate([np.concatenate([np.asarray(w, np.float32).ravel(), np.asarray(b, np.float32).ravel()])
                           for w, b in params]).astype(np.float32)


def unpack_params(vec):
    out, o = [], 0
    for ci, co in LAYERS:
        w = vec[o:o + co * ci * 9].reshape(co, ci, 3, 3)
        o += co * ci * 9
        b = vec[o:o + co]
        o += co
        out.append((w.astype(np.float64), b.astype(np.float64)))
    return out


class Net:
    """Network for batches of `batch` images of H x W pixels."""

    def __init__(self, batch, H, W, dilations=DILATIONS, stream=None):
        self.batch, self.H, self.W = batch, H, W
        d = (C.c_int * 6)(*dilations)
        h = C.c_void_p()
        s = _lib().gcmg_cnn_create(batch, H, W, d, C.c_void_p(stream.cuda_stream) if stream else None, C.byref(h))
        self._h = h
        if s != gcmg.GCMG_OK:
            msg = _lib().gcmg_cnn_last_error(h).decode() if h.value else ""
            self.close()
            raise gcmg.GcmgError(s, msg)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib().gcmg_cnn_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, s):
        if s != gcmg.GCMG_OK:
            raise gcmg.GcmgError(s, _lib().gcmg_cnn_last_error(self._h).decode())

    def set_params(self, vec):
        vec = np.ascontiguousarray(vec, np.float32)
        self._check(_lib().gcmg_cnn_set_params(self._h, gcmg._ptr(vec), vec.size))

    def get_params(self):
        vec = np.empty(num_params(), np.float32)
        self._check(_lib().gcmg_cnn_get_params(self._h, gcmg._ptr(vec), vec.size))
        return vec

    def forward(self, inp, out):
        self._check(_lib().gcmg_cnn_forward(self._h, gcmg._ptr(inp), gcmg._ptr(out)))

    def activation(self, layer, dst):
        self._check(_lib().gcmg_cnn_activation(self._h, layer, gcmg._ptr(dst)))

    def backward(self, dout, grad):
        self._check(_lib().gcmg_cnn_backward(self._h, gcmg._ptr(dout), gcmg._ptr(grad)))

    def train_step(self, inp, target, mask, mask_count, lr, lap_weight=0.0, lap_count=0.0):
        loss = C.c_double()
        self._check(_lib().gcmg_cnn_train_step(self._h, gcmg._ptr(inp), gcmg._ptr(target), gcmg._ptr(mask),
                                               float(mask_count), float(lap_weight), float(lap_count), float(lr),
                                               C.byref(loss)))
        return loss.value
