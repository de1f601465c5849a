"""Python binding of the factorised FNO C ABI in include/ffno.h (argument
marshalling only).

The network runs in ``lib/libffno.so``; arrays may be numpy (host) or torch
tensors (device).  If the library is missing, loading it raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libffno.so")


class ffno_config(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("cin", C.c_int32), ("width", C.c_int32), ("cout", C.c_int32),
                ("mx", C.c_int32), ("my", C.c_int32), ("mz", C.c_int32),
                ("layers", C.c_int32), ("ff_hidden", C.c_int32), ("hidden", C.c_int32),
                ("lift_hidden", C.c_int32), ("max_batch", C.c_int32), ("omega0", C.c_float),
                ("reserved", C.c_int32), ("seed", C.c_uint64)]


class FFNOError(RuntimeError):
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
        P = C.POINTER(ffno_config)
        sig = {
            "ffno_config_default": (None, [P]),
            "ffno_create": (C.c_int, [P, _vp, C.POINTER(_vp)]),
            "ffno_destroy": (C.c_int, [_vp]),
            "ffno_num_params": (C.c_int64, [_vp]),
            "ffno_set_params": (C.c_int, [_vp, _vp]),
            "ffno_get_params": (C.c_int, [_vp, _vp]),
            "ffno_get_grads": (C.c_int, [_vp, _vp]),
            "ffno_forward": (C.c_int, [_vp, _vp, _vp, C.c_int32]),
            "ffno_loss_grad": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int32, C.POINTER(C.c_double)]),
            "ffno_adam_step": (C.c_int, [_vp, C.c_float, C.c_float, C.c_float, C.c_float]),
            "ffno_sync": (C.c_int, [_vp]),
            "ffno_last_error": (C.c_char_p, [_vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(st, h):
    if st != 0:
        raise FFNOError(st, lib().ffno_last_error(h).decode())


def _ptr(a):
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


def make_config(**kw) -> ffno_config:
    c = ffno_config()
    lib().ffno_config_default(C.byref(c))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


class FFNO:
    """The factorised surrogate on the current CUDA device (work on the current torch stream)."""

    def __init__(self, **cfg):
        import torch
        self.cfg = make_config(**cfg)
        self.stream = torch.cuda.current_stream()
        self.h = C.c_void_p()
        _check(lib().ffno_create(C.byref(self.cfg), C.c_void_p(self.stream.cuda_stream), C.byref(self.h)), None)

    def close(self):
        if getattr(self, "h", None):
            _check(lib().ffno_destroy(self.h), None)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_params(self):
        return int(lib().ffno_num_params(self.h))

    def params(self):
        out = np.zeros(self.num_params, np.float32)
        _check(lib().ffno_get_params(self.h, _ptr(out)), self.h)
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(lib().ffno_set_params(self.h, _ptr(p)), self.h)

    def grads(self):
        out = np.zeros(self.num_params, np.float32)
        _check(lib().ffno_get_grads(self.h, _ptr(out)), self.h)
        return out

    def forward(self, x, out=None):
        """x [B, cin, nz, ny, nx] float32 (numpy or CUDA tensor)."""
        B = x.shape[0]
        if out is None:
            out = np.zeros((B, self.cfg.cout) + tuple(x.shape[2:]), np.float32)
        _check(lib().ffno_forward(self.h, _ptr(x), _ptr(out), int(B)), self.h)
        return out

    def loss_grad(self, x, t, m):
        loss = C.c_double()
        _check(lib().ffno_loss_grad(self.h, _ptr(x), _ptr(t), _ptr(m), int(x.shape[0]), C.byref(loss)), self.h)
        return loss.value

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(lib().ffno_adam_step(self.h, float(lr), float(beta1), float(beta2), float(eps)), self.h)

    def sync(self):
        _check(lib().ffno_sync(self.h), self.h)


# ---------------------------------------------------------------------------
# flat parameter layout (see include/ffno.h)
# ---------------------------------------------------------------------------
def layout(cfg):
    """[(name, shape, complex)] in the order of the flat vector; spectral
    weights R{l}{z,y,x} as complex [width_in][width_out][m_d]."""
    W, H, LH = cfg.width, cfg.ff_hidden, cfg.lift_hidden
    out = [("P1_w", (LH, cfg.cin), False), ("P1_b", (LH,), False),
           ("P2_w", (W, LH), False), ("P2_b", (W,), False)]
    for l in range(cfg.layers):
        for name, m in (("z", cfg.mz), ("y", cfg.my), ("x", cfg.mx)):
            out.append((f"R{l}{name}", (W, W, m), True))
        out += [(f"F{l}a_w", (H, W), False), (f"F{l}a_b", (H,), False),
                (f"F{l}b_w", (W, H), False), (f"F{l}b_b", (W,), False)]
    out += [("Q1_w", (cfg.hidden, W), False), ("Q1_b", (cfg.hidden,), False),
            ("Q2_w", (cfg.cout, cfg.hidden), False), ("Q2_b", (cfg.cout,), False)]
    return out


def unflatten(cfg, flat):
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
        parts.append(np.stack([a.real, a.imag], -1).reshape(-1) if cplx else a.reshape(-1))
    return np.concatenate(parts).astype(np.float32)


def time_ffno(batch=8, reps=2, warmup=1):
    """Forward and training-step time (ms, CUDA events) of the default
    factorised surrogate (128x64x64, batch 8) on random inputs resident on
    the device."""
    import torch
    net = FFNO(max_batch=batch)
    c = net.cfg
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.rand((batch, c.cin, c.nz, c.ny, c.nx), device="cuda", generator=g)
    t = torch.rand((batch, c.cout, c.nz, c.ny, c.nx), device="cuda", generator=g)
    w = torch.ones((batch, c.nz, c.ny, c.nx), device="cuda")
    y = torch.zeros((batch, c.cout, c.nz, c.ny, c.nx), device="cuda")
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    fwd = timed(lambda: net.forward(x, y))
    train = timed(lambda: (net.loss_grad(x, t, w), net.adam(1e-6)))
    net.close()
    return {"batch": batch, "forward_ms_per_batch": fwd, "train_step_ms": train,
            "train_samples_per_s": batch / train * 1e3}


if __name__ == "__main__":
    import json
    print(json.dumps(time_ffno()))
