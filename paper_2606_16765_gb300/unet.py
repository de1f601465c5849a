"""Python binding of the U-Net C ABI in include/unet.h (argument marshalling only).

The network runs in ``lib/libunet.so``; arrays may be numpy (host) or torch
tensors (device).  If the library is missing, loading it raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libunet.so")


class unet_config(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("cin", C.c_int32), ("cout", C.c_int32), ("stages", C.c_int32),
                ("channels", C.c_int32 * 4), ("bottleneck", C.c_int32), ("max_batch", C.c_int32),
                ("reserved", C.c_int32 * 2), ("seed", C.c_uint64)]


class UNetError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lib = None
_vp = C.c_void_p
_i32 = C.c_int32


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"CUDA library not built: {_LIB_PATH} (run __graft_entry__.build())")
        L = C.CDLL(_LIB_PATH)
        P = C.POINTER(unet_config)
        conv = (C.c_int, [_vp, _vp, _vp, _i32, _i32, _i32, _i32, _i32, _i32, _vp])
        sig = {
            "unet_config_default": (None, [P]),
            "unet_create": (C.c_int, [P, _vp, C.POINTER(_vp)]),
            "unet_destroy": (C.c_int, [_vp]),
            "unet_num_params": (C.c_int64, [_vp]),
            "unet_set_params": (C.c_int, [_vp, _vp]),
            "unet_get_params": (C.c_int, [_vp, _vp]),
            "unet_get_grads": (C.c_int, [_vp, _vp]),
            "unet_forward": (C.c_int, [_vp, _vp, _vp, _i32]),
            "unet_loss_grad": (C.c_int, [_vp, _vp, _vp, _vp, _i32, C.POINTER(C.c_double)]),
            "unet_adam_step": (C.c_int, [_vp, C.c_float, C.c_float, C.c_float, C.c_float]),
            "unet_train_step": (C.c_int, [_vp, _vp, _vp, _vp, _i32, C.c_float, C.POINTER(C.c_double)]),
            "unet_sync": (C.c_int, [_vp]),
            "unet_last_error": (C.c_char_p, [_vp]),
            "unet_conv3_forward": conv,
            "unet_conv3_backward_data": conv,
            "unet_conv3_backward_weights": conv,
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(st, h):
    if st != 0:
        raise UNetError(st, lib().unet_last_error(h).decode())


def _ptr(a):
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


def unet_config_default() -> unet_config:
    c = unet_config()
    lib().unet_config_default(C.byref(c))
    return c


def make_config(**kw) -> unet_config:
    c = unet_config_default()
    for k, v in kw.items():
        if k == "channels":
            v = list(v) + [0] * (4 - len(v))
            c.channels = (C.c_int32 * 4)(*v)
        else:
            setattr(c, k, v)
    return c


def conv3_forward(x, w, y, stream=0):
    """y [B, nz, ny, nx, cout] = conv3(x [B, nz, ny, nx, cin], w [cout, cin, 27]); CUDA tensors."""
    B, nz, ny, nx, cin = x.shape
    _check(lib().unet_conv3_forward(_ptr(x), _ptr(w), _ptr(y), B, nx, ny, nz, cin, w.shape[0], _vp(stream)), None)


def conv3_backward_data(gy, w, gx, stream=0):
    B, nz, ny, nx, cout = gy.shape
    _check(lib().unet_conv3_backward_data(_ptr(gy), _ptr(w), _ptr(gx), B, nx, ny, nz, w.shape[1], cout, _vp(stream)),
           None)


def conv3_backward_weights(x, gy, gw, stream=0):
    B, nz, ny, nx, cin = x.shape
    _check(lib().unet_conv3_backward_weights(_ptr(x), _ptr(gy), _ptr(gw), B, nx, ny, nz, cin, gy.shape[-1],
                                             _vp(stream)), None)


class UNet:
    """The U-Net surrogate on the current CUDA device (work on the current torch stream)."""

    def __init__(self, **cfg):
        import torch
        self.cfg = make_config(**cfg)
        self.stream = torch.cuda.current_stream()
        h = C.c_void_p()
        _check(lib().unet_create(C.byref(self.cfg), C.c_void_p(self.stream.cuda_stream), C.byref(h)), None)
        self.h = h
        self.n = self.cfg.nx * self.cfg.ny * self.cfg.nz

    def close(self):
        if getattr(self, "h", None):
            _check(lib().unet_destroy(self.h), None)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_params(self):
        return int(lib().unet_num_params(self.h))

    def params(self):
        out = np.zeros(self.num_params, np.float32)
        _check(lib().unet_get_params(self.h, _ptr(out)), self.h)
        return out

    def set_params(self, p):
        _check(lib().unet_set_params(self.h, _ptr(np.ascontiguousarray(p, dtype=np.float32))), self.h)

    def grads(self):
        out = np.zeros(self.num_params, np.float32)
        _check(lib().unet_get_grads(self.h, _ptr(out)), self.h)
        return out

    def forward(self, x, out=None):
        """x [B, cin, nz, ny, nx] float32 (numpy or CUDA tensor)."""
        B = x.shape[0]
        if out is None:
            out = np.zeros((B, self.cfg.cout) + tuple(x.shape[2:]), np.float32)
        _check(lib().unet_forward(self.h, _ptr(x), _ptr(out), B), self.h)
        return out

    def loss_grad(self, x, t, m):
        loss = C.c_double()
        _check(lib().unet_loss_grad(self.h, _ptr(x), _ptr(t), _ptr(m), x.shape[0], C.byref(loss)), self.h)
        return loss.value

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(lib().unet_adam_step(self.h, float(lr), float(beta1), float(beta2), float(eps)), self.h)

    def train_step(self, x, t, m, lr):
        loss = C.c_double()
        _check(lib().unet_train_step(self.h, _ptr(x), _ptr(t), _ptr(m), x.shape[0], float(lr), C.byref(loss)), self.h)
        return loss.value

    def sync(self):
        _check(lib().unet_sync(self.h), self.h)


# ---------------------------------------------------------------------------
# flat parameter layout (see include/unet.h)
# ---------------------------------------------------------------------------
def blocks(cfg):
    """Convolution blocks in forward order: (name, in channels, out channels)."""
    S = cfg.stages
    ch = [cfg.channels[e] for e in range(S)]
    out, cin = [], cfg.cin
    for e in range(S):
        out += [(f"enc{e}a", cin, ch[e]), (f"enc{e}b", ch[e], ch[e])]
        cin = ch[e]
    out += [("mida", cin, cfg.bottleneck), ("midb", cfg.bottleneck, cfg.bottleneck)]
    below = cfg.bottleneck
    for d in reversed(range(S)):
        out += [(f"dec{d}a", ch[d] + below, ch[d]), (f"dec{d}b", ch[d], ch[d])]
        below = ch[d]
    return out


def layout(cfg):
    """[(name, shape)] in the order of the flat vector."""
    out = []
    for name, ci, co in blocks(cfg):
        out += [(name + "_w", (co, ci, 3, 3, 3)), (name + "_g", (co,)), (name + "_b", (co,))]
    out += [("out_w", (cfg.cout, cfg.channels[0])), ("out_b", (cfg.cout,))]
    return out


def unflatten(cfg, flat):
    d, o = {}, 0
    for name, shape in layout(cfg):
        n = int(np.prod(shape))
        d[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return d


def flatten(cfg, d):
    return np.concatenate([np.asarray(d[name]).reshape(-1) for name, _ in layout(cfg)]).astype(np.float32)
