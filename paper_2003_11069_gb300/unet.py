"""ctypes binding of the warm-start U-Net (include/lbnci_unet.h): argument marshalling only.

Host arrays are numpy float32; device arrays are contiguous CUDA tensors (torch), used
for their memory only. Every forward, backward and optimiser step runs in the library's
CUDA kernels; without the library or a GPU these calls raise.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import lbnci

EXPORTS = ("lbu_layer_count", "lbu_layer_shape", "lbu_param_count", "lbu_create", "lbu_destroy",
           "lbu_last_error", "lbu_kernel_launches", "lbu_set_params", "lbu_get_params", "lbu_set_adam",
           "lbu_forward", "lbu_loss_grad", "lbu_train_step", "lbu_conv3x3", "lbu_conv3x3_wgrad_work",
           "lbu_conv3x3_wgrad")


class lbu_config(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("base", ctypes.c_int), ("in_ch", ctypes.c_int),
                ("out_ch", ctypes.c_int), ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("max_batch", ctypes.c_int), ("stream", ctypes.c_void_p)]


_done = False


def load() -> ctypes.CDLL:
    global _done
    lib = lbnci.load()
    if _done:
        return lib
    vp, cp = ctypes.c_void_p, ctypes.POINTER(lbu_config)
    i, f = ctypes.c_int, ctypes.c_float
    sig = {
        "lbu_layer_count": ([cp], i),
        "lbu_layer_shape": ([cp, i, ctypes.POINTER(ctypes.c_int)], i),
        "lbu_param_count": ([cp, ctypes.POINTER(ctypes.c_longlong)], i),
        "lbu_create": ([cp, ctypes.POINTER(vp)], i),
        "lbu_destroy": ([vp], None),
        "lbu_last_error": ([vp], ctypes.c_char_p),
        "lbu_kernel_launches": ([vp], ctypes.c_longlong),
        "lbu_set_params": ([vp, vp, i], i),
        "lbu_get_params": ([vp, vp, i], i),
        "lbu_set_adam": ([vp, f, f, f], i),
        "lbu_forward": ([vp, vp, i, vp, i], i),
        "lbu_loss_grad": ([vp, vp, vp, vp, i, vp, vp, vp], i),
        "lbu_train_step": ([vp, vp, vp, vp, i, vp, f, vp], i),
        "lbu_conv3x3": ([vp, i, i, i, i, i, i, vp, vp, i, vp, i, i, vp], i),
        "lbu_conv3x3_wgrad_work": ([i, i, i, i, i], ctypes.c_size_t),
        "lbu_conv3x3_wgrad": ([vp, i, i, i, i, i, i, vp, i, i, vp, vp, vp, ctypes.c_size_t, vp], i),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _done = True
    return lib


def _check(st, h=None):
    if st != lbnci.LB_OK:
        msg = load().lbu_last_error(h)
        raise lbnci.LBError(st, msg.decode() if msg else "")


def make_config(levels=4, base=32, in_ch=5, out_ch=3, H=64, W=256, max_batch=16, stream=None) -> lbu_config:
    return lbu_config(levels, base, in_ch, out_ch, H, W, max_batch, stream)


def layer_shapes(cfg: lbu_config):
    """[(C_out, kh, kw, C_in)] of every layer, in parameter order (from the library)."""
    lib = load()
    n = lib.lbu_layer_count(ctypes.byref(cfg))
    if n < 0:
        _check(lbnci.LB_EINVAL)
    out = []
    for k in range(n):
        s = (ctypes.c_int * 4)()
        _check(lib.lbu_layer_shape(ctypes.byref(cfg), k, s))
        out.append(tuple(s))
    return out


def param_count(cfg: lbu_config) -> int:
    c = ctypes.c_longlong()
    _check(load().lbu_param_count(ctypes.byref(cfg), ctypes.byref(c)))
    return c.value


def _ptr(t):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not (lbnci._is_torch(t) and t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class Net:
    """Owning wrapper of an lbu_net handle."""

    def __init__(self, cfg: lbu_config):
        self.cfg = cfg
        self.h = ctypes.c_void_p()
        _check(load().lbu_create(ctypes.byref(cfg), ctypes.byref(self.h)))
        self.nparams = param_count(cfg)

    def close(self):
        if self.h:
            load().lbu_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_params(self, flat):
        if lbnci._is_torch(flat):
            _check(load().lbu_set_params(self.h, _ptr(flat), 1), self.h)
        else:
            a = np.ascontiguousarray(flat, dtype=np.float32)
            assert a.size == self.nparams
            _check(load().lbu_set_params(self.h, a.ctypes.data_as(ctypes.c_void_p), 0), self.h)

    def get_params(self) -> np.ndarray:
        a = np.empty(self.nparams, dtype=np.float32)
        _check(load().lbu_get_params(self.h, a.ctypes.data_as(ctypes.c_void_p), 0), self.h)
        return a

    def set_adam(self, b1=0.9, b2=0.999, eps=1e-8):
        _check(load().lbu_set_adam(self.h, b1, b2, eps), self.h)

    def forward(self, x, y=None):
        """x: numpy float32 [B][H][W][in_ch] (returns numpy) or a CUDA tensor (writes y)."""
        c = self.cfg
        if lbnci._is_torch(x):
            _check(load().lbu_forward(self.h, _ptr(x), x.shape[0], _ptr(y), 1), self.h)
            return y
        a = np.ascontiguousarray(x, dtype=np.float32)
        out = np.empty((a.shape[0], c.H, c.W, c.out_ch), dtype=np.float32)
        _check(load().lbu_forward(self.h, a.ctypes.data_as(ctypes.c_void_p), a.shape[0],
                                  out.ctypes.data_as(ctypes.c_void_p), 0), self.h)
        return out

    def loss_grad(self, X, T, idx=None, batch=None, lam=None, grads=None):
        """X, T, idx (int32), grads: CUDA tensors; returns the loss (host float)."""
        batch = X.shape[0] if batch is None else batch
        lam_a = None if lam is None else (ctypes.c_float * len(lam))(*lam)
        loss = ctypes.c_float()
        _check(load().lbu_loss_grad(self.h, _ptr(X), _ptr(T), _ptr(idx), batch, lam_a, ctypes.byref(loss),
                                    _ptr(grads)), self.h)
        return loss.value

    def train_step(self, X, T, idx=None, batch=None, lam=None, lr=1e-3, want_loss=False):
        batch = X.shape[0] if batch is None else batch
        lam_a = None if lam is None else (ctypes.c_float * len(lam))(*lam)
        loss = ctypes.c_float()
        _check(load().lbu_train_step(self.h, _ptr(X), _ptr(T), _ptr(idx), batch, lam_a, lr,
                                     ctypes.byref(loss) if want_loss else None), self.h)
        return loss.value if want_loss else None

    def launches(self) -> int:
        return int(load().lbu_kernel_launches(self.h))


def flatten(params) -> np.ndarray:
    """[(w, b)] in layer order -> the flat parameter vector (float32)."""
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in params]).astype(np.float32)


def unflatten(flat, shapes) -> list:
    """Inverse of flatten for shapes [(C_out, kh, kw, C_in)] (head: kh = kw = 1 -> [C_out, C_in])."""
    out, o = [], 0
    for co, kh, kw, ci in shapes:
        ws = (co, kh, kw, ci) if kh == 3 else (co, ci)
        n = int(np.prod(ws))
        w = np.asarray(flat[o:o + n], dtype=np.float64).reshape(ws)
        o += n
        b = np.asarray(flat[o:o + co], dtype=np.float64)
        o += co
        out.append((w, b))
    return out


def conv3x3(x, x_stride, batch, h, w, c_in, upsample, wgt, bias, relu, y, y_stride, c_out, stream=None):
    """Single convolution on device tensors (x, wgt, y: bfloat16 CUDA tensors; bias float32)."""
    _check(load().lbu_conv3x3(_ptr(x), x_stride, batch, h, w, c_in, int(upsample), _ptr(wgt), _ptr(bias),
                              int(relu), _ptr(y), y_stride, c_out, stream))


def conv3x3_wgrad(x, x_stride, batch, h, w, c_in, upsample, dy, dy_stride, c_out, dw, db, work, stream=None):
    _check(load().lbu_conv3x3_wgrad(_ptr(x), x_stride, batch, h, w, c_in, int(upsample), _ptr(dy), dy_stride,
                                    c_out, _ptr(dw), _ptr(db), _ptr(work), work.numel() * work.element_size(),
                                    stream))


def conv3x3_wgrad_work(batch, h, w, c_in, c_out) -> int:
    return int(load().lbu_conv3x3_wgrad_work(batch, h, w, c_in, c_out))
