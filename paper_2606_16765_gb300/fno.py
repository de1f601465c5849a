"""Python binding of the FNO C ABI in include/fno.h (argument marshalling only).

The network runs in ``lib/libfno.so``; arrays may be numpy (host) or torch
tensors (device).  If the library is missing, loading it raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libfno.so")


class fno_config(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("cin", C.c_int32), ("width", C.c_int32), ("cout", C.c_int32),
                ("mx", C.c_int32), ("my", C.c_int32), ("mz", C.c_int32),
                ("layers", C.c_int32), ("hidden", C.c_int32), ("max_batch", C.c_int32),
                ("act_bf16", C.c_int32), ("tensor_cores", C.c_int32),
                ("lift_hidden", C.c_int32), ("omega0", C.c_float), ("umma", C.c_int32), ("reserved", C.c_int32),
                ("seed", C.c_uint64)]


class FNOError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lib = None
_vp = C.c_void_p


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"CUDA library not built: {_LIB_PATH} (run __graft_entry__.build())")
        L = C.CDLL(_LIB_PATH)
        P = C.POINTER(fno_config)
        sig = {
            "fno_config_default": (None, [P]),
            "fno_create": (C.c_int, [P, _vp, C.POINTER(_vp)]),
            "fno_destroy": (C.c_int, [_vp]),
            "fno_num_params": (C.c_int64, [_vp]),
            "fno_set_params": (C.c_int, [_vp, _vp]),
            "fno_get_params": (C.c_int, [_vp, _vp]),
            "fno_get_grads": (C.c_int, [_vp, _vp]),
            "fno_forward": (C.c_int, [_vp, _vp, _vp, C.c_int32]),
            "fno_loss_grad": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int32, C.POINTER(C.c_double)]),
            "fno_adam_step": (C.c_int, [_vp, C.c_float, C.c_float, C.c_float, C.c_float]),
            "fno_train_step": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int32, C.c_float, C.POINTER(C.c_double)]),
            "fno_sync": (C.c_int, [_vp]),
            "fno_save": (C.c_int, [_vp, C.c_char_p]),
            "fno_load": (C.c_int, [_vp, C.c_char_p]),
            "fno_last_error": (C.c_char_p, [_vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(st, h):
    if st != 0:
        raise FNOError(st, lib().fno_last_error(h).decode())


def _ptr(a):
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


def fno_config_default() -> fno_config:
    c = fno_config()
    lib().fno_config_default(C.byref(c))
    return c


def fno_create(cfg, stream=None):
    h = C.c_void_p()
    _check(lib().fno_create(C.byref(cfg), C.c_void_p(stream or 0), C.byref(h)), None)
    return h


def fno_destroy(h):
    _check(lib().fno_destroy(h), None)


def fno_num_params(h):
    return int(lib().fno_num_params(h))


def fno_set_params(h, src):
    _check(lib().fno_set_params(h, _ptr(src)), h)


def fno_get_params(h, dst):
    _check(lib().fno_get_params(h, _ptr(dst)), h)


def fno_get_grads(h, dst):
    _check(lib().fno_get_grads(h, _ptr(dst)), h)


def fno_forward(h, x, y, batch):
    _check(lib().fno_forward(h, _ptr(x), _ptr(y), int(batch)), h)


def fno_loss_grad(h, x, t, m, batch):
    loss = C.c_double()
    _check(lib().fno_loss_grad(h, _ptr(x), _ptr(t), _ptr(m), int(batch), C.byref(loss)), h)
    return loss.value


def fno_adam_step(h, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    _check(lib().fno_adam_step(h, float(lr), float(beta1), float(beta2), float(eps)), h)


def fno_train_step(h, x, t, m, batch, lr):
    loss = C.c_double()
    _check(lib().fno_train_step(h, _ptr(x), _ptr(t), _ptr(m), int(batch), float(lr), C.byref(loss)), h)
    return loss.value


def fno_sync(h):
    _check(lib().fno_sync(h), h)


def fno_save(h, path):
    _check(lib().fno_save(h, str(path).encode()), h)


def fno_load(h, path):
    _check(lib().fno_load(h, str(path).encode()), h)


def make_config(**kw) -> fno_config:
    c = fno_config_default()
    for k, v in kw.items():
        setattr(c, k, v)
    return c


class FNO:
    """The surrogate on the current CUDA device (work on the current torch stream)."""

    def __init__(self, **cfg):
        import torch
        self.cfg = make_config(**cfg)
        self.stream = torch.cuda.current_stream()
        self.h = fno_create(self.cfg, self.stream.cuda_stream)
        self.n = self.cfg.nx * self.cfg.ny * self.cfg.nz

    def close(self):
        if getattr(self, "h", None):
            fno_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_params(self):
        return fno_num_params(self.h)

    def params(self):
        out = np.zeros(self.num_params, np.float32)
        fno_get_params(self.h, out)
        return out

    def set_params(self, p):
        fno_set_params(self.h, np.ascontiguousarray(p, dtype=np.float32))

    def grads(self):
        out = np.zeros(self.num_params, np.float32)
        fno_get_grads(self.h, out)
        return out

    def forward(self, x, out=None):
        """x [B, cin, nz, ny, nx] float32 (numpy or CUDA tensor)."""
        B = x.shape[0]
        if out is None:
            out = np.zeros((B, self.cfg.cout) + tuple(x.shape[2:]), np.float32)
        fno_forward(self.h, x, out, B)
        return out

    def loss_grad(self, x, t, m):
        return fno_loss_grad(self.h, x, t, m, x.shape[0])

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        fno_adam_step(self.h, lr, beta1, beta2, eps)

    def train_step(self, x, t, m, lr):
        return fno_train_step(self.h, x, t, m, x.shape[0], lr)

    def sync(self):
        fno_sync(self.h)

    def save(self, path):
        fno_save(self.h, path)

    def load(self, path):
        fno_load(self.h, path)


# ---------------------------------------------------------------------------
# flat parameter layout (see include/fno.h)
# ---------------------------------------------------------------------------
def layout(cfg):
    """[(name, shape, complex)] in the order of the flat vector."""
    K = cfg.mz * 2 * cfg.my * 2 * cfg.mx
    W, H, LH = cfg.width, cfg.hidden, cfg.lift_hidden
    out = [(f"R{l}", (K, W, W), True) for l in range(cfg.layers)]
    out += [("P1_w", (LH, cfg.cin), False), ("P1_b", (LH,), False),
            ("P2_w", (W, LH), False), ("P2_b", (W,), False)]
    for l in range(cfg.layers):
        out += [(f"W{l}_w", (W, W), False), (f"W{l}_b", (W,), False)]
    out += [("Q1_w", (H, W), False), ("Q1_b", (H,), False), ("Q2_w", (cfg.cout, H), False),
            ("Q2_b", (cfg.cout,), False)]
    return out


def unflatten(cfg, flat):
    """Flat vector -> dict of arrays; spectral weights as complex [K][i][o]."""
    d, o = {}, 0
    for name, shape, cplx in layout(cfg):
        n = int(np.prod(shape)) * (2 if cplx else 1)
        a = np.asarray(flat[o:o + n], dtype=np.float64)
        d[name] = (a[0::2] + 1j * a[1::2]).reshape(shape) if cplx else a.reshape(shape)
        o += n
    return d


def flatten(cfg, d):
    parts = []
    for name, shape, cplx in layout(cfg):
        a = np.asarray(d[name]).reshape(shape)
        if cplx:
            parts.append(np.stack([a.real, a.imag], -1).reshape(-1))
        else:
            parts.append(a.reshape(-1))
    return np.concatenate(parts).astype(np.float32)
