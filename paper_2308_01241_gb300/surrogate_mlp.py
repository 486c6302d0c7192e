"""ctypes binding of the surrogate MLP (include/dtb_surrogate.h): marshalling only."""
from __future__ import annotations

import ctypes

import numpy as np

from . import dtb

_lib = dtb._lib
_vp, _i32, _i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
for _n, (_a, _r) in {
    "dtb_mlp_create": ([_i32, _i32, _i32, _i32, _i64, _vp, ctypes.POINTER(ctypes.c_void_p)], _i32),
    "dtb_mlp_destroy": ([_vp], _i32),
    "dtb_mlp_forward": ([_vp, _vp, _vp, _i64, _vp], _i32),
    "dtb_mlp_gradients": ([_vp, _vp, _vp, _i64, _vp, _vp, _vp], _i32),
    "dtb_mlp_train_step": ([_vp, _vp, _vp, _i64, ctypes.c_float, _vp, _vp], _i32),
    "dtb_mlp_get_params": ([_vp, _vp], _i32),
}.items():
    getattr(_lib, _n).argtypes = _a
    getattr(_lib, _n).restype = _r


def flatten(params) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params]).astype(np.float32)


def unflatten(flat, n_in, width, depth, n_out):
    sizes = [n_in] + [width] * depth + [n_out]
    out, o = [], 0
    for i in range(len(sizes) - 1):
        w = flat[o:o + sizes[i] * sizes[i + 1]].reshape(sizes[i], sizes[i + 1])
        o += w.size
        b = flat[o:o + sizes[i + 1]]
        o += b.size
        out.append((w, b))
    return out


class MLP:
    """The surrogate network on the GPU (dtb_mlp handle)."""

    def __init__(self, params, n_in, width, depth, n_out, max_batch):
        self.shape = (n_in, width, depth, n_out)
        flat = np.ascontiguousarray(flatten(params))
        h = ctypes.c_void_p()
        dtb._check(_lib.dtb_mlp_create(n_in, width, depth, n_out, int(max_batch), flat.ctypes.data, ctypes.byref(h)),
                   "dtb_mlp_create")
        self.h = h.value
        self.n_params = flat.size

    def close(self):
        if getattr(self, "h", None):
            _lib.dtb_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, x, y, stream=None):
        """x [B][n_in], y [B][n_out]: float32 torch device tensors."""
        dtb._check(_lib.dtb_mlp_forward(self.h, x.data_ptr(), y.data_ptr(), x.shape[0], stream), "dtb_mlp_forward")

    def gradients(self, x, t, stream=None):
        g = np.zeros(self.n_params, np.float32)
        loss = ctypes.c_float()
        dtb._check(_lib.dtb_mlp_gradients(self.h, x.data_ptr(), t.data_ptr(), x.shape[0], g.ctypes.data,
                                          ctypes.byref(loss), stream), "dtb_mlp_gradients")
        return unflatten(g, *self.shape), float(loss.value)

    def train_step(self, x, t, lr, stream=None) -> float:
        loss = ctypes.c_float()
        dtb._check(_lib.dtb_mlp_train_step(self.h, x.data_ptr(), t.data_ptr(), x.shape[0], float(lr),
                                           ctypes.byref(loss), stream), "dtb_mlp_train_step")
        return float(loss.value)

    def params(self):
        p = np.zeros(self.n_params, np.float32)
        dtb._check(_lib.dtb_mlp_get_params(self.h, p.ctypes.data), "dtb_mlp_get_params")
        return unflatten(p, *self.shape)
