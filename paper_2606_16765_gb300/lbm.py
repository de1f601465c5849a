"""Python binding of the C ABI in include/lbm.h (argument marshalling only).

Every step of the lattice Boltzmann path runs in the CUDA library
``lib/liblbm.so``; this module only converts arguments.  PyTorch supplies the
device memory (the context's workspace is a torch tensor) and the stream (the
current torch stream).  If the library is missing the import of the binding
fails; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "liblbm.so")

LBM_OK, LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_OOM, LBM_ERR_UNSTABLE, LBM_ERR_TIMEOUT, LBM_ERR_STATE, LBM_ERR_IO = range(8)
LBM_F64, LBM_F32, LBM_F16S, LBM_BF16S, LBM_F16C = range(5)
LBM_FACE_WALL, LBM_FACE_PERIODIC, LBM_FACE_INLET, LBM_FACE_OUTLET, LBM_FACE_OUTFLOW = range(5)
STORAGE = {"f64": LBM_F64, "f32": LBM_F32, "f16s": LBM_F16S, "bf16s": LBM_BF16S, "f16c": LBM_F16C}
FACES = {"wall": LBM_FACE_WALL, "periodic": LBM_FACE_PERIODIC, "inlet": LBM_FACE_INLET, "outlet": LBM_FACE_OUTLET,
         "outflow": LBM_FACE_OUTFLOW}


class lbm_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32)]


class lbm_params(C.Structure):
    _fields_ = [
        ("re", C.c_double), ("u_in", C.c_double), ("l_ref", C.c_double),
        ("omega1", C.c_double), ("omega_bulk", C.c_double), ("omega_higher", C.c_double),
        ("rho_in", C.c_double), ("rho_out", C.c_double),
        ("storage", C.c_int32), ("galilean_correction", C.c_int32),
        ("face_x_lo", C.c_int32), ("face_x_hi", C.c_int32), ("face_y", C.c_int32), ("face_z", C.c_int32),
        ("mean_start", C.c_int64), ("mean_end", C.c_int64), ("mean_every", C.c_int64),
        ("snap_first", C.c_int64), ("snap_every", C.c_int64), ("snap_count", C.c_int64),
        ("snap_halfres", C.c_int32), ("force_every", C.c_int32),
        ("force_capacity", C.c_int64),
        ("block_x", C.c_int32), ("block_y", C.c_int32), ("stats", C.c_int32),
        ("param4", C.c_int32), ("limiter", C.c_double), ("xface_edge", C.c_int32), ("reserved", C.c_int32 * 1),
    ]


class lbm_info(C.Structure):
    _fields_ = [("cells", C.c_int64), ("fluid_cells", C.c_int64), ("edge_cells", C.c_int64),
                ("bulk_cells", C.c_int64), ("launches", C.c_int64), ("workspace_bytes", C.c_uint64),
                ("storage", C.c_int32), ("block_x", C.c_int32), ("omega1", C.c_double),
                ("interior_cells", C.c_int64), ("wall_cells", C.c_int64)]


class lbm_timing_report(C.Structure):
    _fields_ = [("steps", C.c_int64), ("bulk_ms", C.c_double * 4), ("bulk_n", C.c_int64 * 4),
                ("rowend_ms", C.c_double), ("edge_ms", C.c_double)]


class lbm_batch_info(C.Structure):
    _fields_ = [("t", C.c_int64), ("chunk", C.c_int64), ("members", C.c_int32), ("live", C.c_int32),
                ("block_x", C.c_int32), ("block_y", C.c_int32), ("graph_captures", C.c_int64),
                ("graph_launches", C.c_int64), ("kernel_launches", C.c_int64), ("lattice_updates", C.c_int64)]


class LBMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lib = None

_vp, _dp, _i64 = C.c_void_p, C.POINTER(C.c_double), C.c_int64


def lib():
    """Load liblbm.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"CUDA library not built: {_LIB_PATH} (run __graft_entry__.build())")
        L = C.CDLL(_LIB_PATH)
        G, P = C.POINTER(lbm_grid), C.POINTER(lbm_params)
        sig = {
            "lbm_params_default": (None, [P]),
            "lbm_workspace_bytes": (C.c_size_t, [G, _vp, P]),
            "lbm_create": (C.c_int, [G, _vp, P, _vp, C.POINTER(_vp)]),
            "lbm_create_in": (C.c_int, [G, _vp, P, _vp, _vp, C.c_size_t, C.POINTER(_vp)]),
            "lbm_destroy": (C.c_int, [_vp]),
            "lbm_step": (C.c_int, [_vp, _i64]),
            "lbm_sync": (C.c_int, [_vp]),
            "lbm_time": (_i64, [_vp]),
            "lbm_read_mean": (C.c_int, [_vp, C.c_int32, C.c_int32, _vp, C.POINTER(_i64)]),
            "lbm_read_stats": (C.c_int, [_vp, C.c_int32, _vp, C.POINTER(_i64)]),
            "lbm_set_probes": (C.c_int, [_vp, _i64, _vp, _i64, _i64]),
            "lbm_init_equilibrium": (C.c_int, [_vp, _vp]),
            "lbm_read_probes": (C.c_int, [_vp, _vp, _i64, C.POINTER(_i64)]),
            "lbm_set_plane_monitor": (C.c_int, [_vp, C.c_int32, _i64, _i64]),
            "lbm_read_plane_monitor": (C.c_int, [_vp, _vp, _i64, C.POINTER(_i64), _vp]),
            "lbm_set_wall_distances": (C.c_int, [_vp, _i64, _vp, _vp, _vp]),
            "lbm_batch_set_wall_distances": (C.c_int, [_vp, C.c_int32, _i64, _vp, _vp, _vp]),
            "lbm_read_snapshot": (C.c_int, [_vp, C.c_int32, _vp]),
            "lbm_read_macros": (C.c_int, [_vp, _vp, _vp]),
            "lbm_read_forces": (C.c_int, [_vp, _vp, _i64, C.POINTER(_i64)]),
            "lbm_get_pdfs": (C.c_int, [_vp, _vp]),
            "lbm_set_pdfs": (C.c_int, [_vp, _vp]),
            "lbm_get_cells": (C.c_int, [_vp, _i64, _vp, _vp]),
            "lbm_init_noise": (C.c_int, [_vp, C.c_uint64, C.c_double]),
            "lbm_totals": (C.c_int, [_vp, _vp]),
            "lbm_get_info": (C.c_int, [_vp, C.POINTER(lbm_info)]),
            "lbm_timing": (C.c_int, [_vp, C.c_int32]),
            "lbm_timing_read": (C.c_int, [_vp, C.POINTER(lbm_timing_report), C.c_int32]),
            "lbm_batch_create": (C.c_int, [C.c_int32, G, C.POINTER(_vp), P, _vp, C.POINTER(_vp)]),
            "lbm_batch_destroy": (C.c_int, [_vp]),
            "lbm_batch_set_end": (C.c_int, [_vp, C.POINTER(_i64)]),
            "lbm_batch_set_flowthroughs": (C.c_int, [_vp, C.c_double]),
            "lbm_batch_run": (C.c_int, [_vp, _i64]),
            "lbm_batch_run_to_end": (C.c_int, [_vp]),
            "lbm_batch_sync": (C.c_int, [_vp]),
            "lbm_batch_member": (C.c_int, [_vp, C.c_int32, C.POINTER(_vp)]),
            "lbm_batch_get_info": (C.c_int, [_vp, C.POINTER(lbm_batch_info)]),
            "lbm_batch_autotune": (C.c_int, [_vp, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                             C.POINTER(C.c_double)]),
            "lbm_autotune": (C.c_int, [_vp, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                       C.POINTER(C.c_double)]),
            "lbm_reset": (C.c_int, [_vp]),
            "lbm_save": (C.c_int, [_vp, C.c_char_p]),
            "lbm_load": (C.c_int, [_vp, C.c_char_p]),
            "lbm_totals_noalloc": (C.c_int, [_vp, C.c_int32, C.c_int64, _vp, C.c_int32, C.c_int32,
                                             C.c_int32, _vp, _vp]),
            "lbm_resample": (C.c_int, [_vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _vp,
                                       C.c_int32, C.c_int32, C.c_int32, _vp]),
            "lbm_last_error": (C.c_char_p, [_vp]),
            "lbm_status_string": (C.c_char_p, [C.c_int]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status, ctx=None):
    if status != LBM_OK:
        msg = lib().lbm_last_error(ctx).decode() if ctx is not None or status else ""
        raise LBMError(status, msg or lib().lbm_status_string(status).decode())


def _ptr(a):
    """Raw pointer of a numpy array or a torch tensor (host or device)."""
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


# ---------------------------------------------------------------------------
# functions with the C names
# ---------------------------------------------------------------------------
def lbm_params_default() -> lbm_params:
    p = lbm_params()
    lib().lbm_params_default(C.byref(p))
    return p


def lbm_workspace_bytes(grid: lbm_grid, mask, p: lbm_params) -> int:
    return int(lib().lbm_workspace_bytes(C.byref(grid), _ptr(mask) if mask is not None else None, C.byref(p)))


def lbm_create(grid, mask, p, stream=None):
    h = C.c_void_p()
    st = lib().lbm_create(C.byref(grid), _ptr(mask) if mask is not None else None, C.byref(p),
                          C.c_void_p(stream or 0), C.byref(h))
    _check(st, None)
    return h


def lbm_create_in(grid, mask, p, stream, workspace, nbytes):
    h = C.c_void_p()
    st = lib().lbm_create_in(C.byref(grid), _ptr(mask) if mask is not None else None, C.byref(p),
                             C.c_void_p(stream or 0), _ptr(workspace), nbytes, C.byref(h))
    _check(st, None)
    return h


def lbm_destroy(h):
    _check(lib().lbm_destroy(h), None)


def lbm_step(h, n):
    _check(lib().lbm_step(h, int(n)), h)


def lbm_sync(h):
    _check(lib().lbm_sync(h), h)


def lbm_time(h):
    return int(lib().lbm_time(h))


def lbm_read_mean(h, dst, dtype, halfres):
    s = C.c_int64()
    _check(lib().lbm_read_mean(h, int(dtype), int(halfres), _ptr(dst), C.byref(s)), h)
    return s.value


def lbm_set_wall_distances(h, cell, direction, q):
    cell = np.ascontiguousarray(cell, dtype=np.int64)
    direction = np.ascontiguousarray(direction, dtype=np.int8)
    q = np.ascontiguousarray(q, dtype=np.float64)
    n = len(cell)
    _check(lib().lbm_set_wall_distances(h, n, _ptr(cell), _ptr(direction), _ptr(q)), h)


def lbm_set_probes(h, cells, every=1, capacity=65536):
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    _check(lib().lbm_set_probes(h, len(cells), _ptr(cells), int(every), int(capacity)), h)


def lbm_set_plane_monitor(h, z=-1, every=1, capacity=64):
    _check(lib().lbm_set_plane_monitor(h, int(z), int(every), int(capacity)), h)


def lbm_read_plane_monitor(h, nx, ny):
    """(planes [k, ny, nx, 4] float32, steps [k] int64) recorded so far."""
    rows = _i64()
    _check(lib().lbm_read_plane_monitor(h, None, 0, C.byref(rows), None), h)
    out = np.zeros((rows.value, ny, nx, 4), np.float32)
    steps = np.zeros(rows.value, np.int64)
    if rows.value:
        _check(lib().lbm_read_plane_monitor(h, _ptr(out), rows.value, C.byref(rows), _ptr(steps)), h)
    return out, steps


def lbm_read_probes(h, n_probes):
    rows = C.c_int64()
    _check(lib().lbm_read_probes(h, None, 0, C.byref(rows)), h)
    out = np.zeros((rows.value, n_probes, 4), np.float32)
    if rows.value:
        _check(lib().lbm_read_probes(h, _ptr(out), rows.value, C.byref(rows)), h)
    return out


def lbm_read_stats(h, dst, dtype):
    s = C.c_int64()
    _check(lib().lbm_read_stats(h, int(dtype), _ptr(dst), C.byref(s)), h)
    return s.value


def lbm_read_snapshot(h, k, dst):
    _check(lib().lbm_read_snapshot(h, int(k), _ptr(dst)), h)


def lbm_read_macros(h, rho, u):
    _check(lib().lbm_read_macros(h, _ptr(rho), _ptr(u)), h)


def lbm_read_forces(h, dst, max_rows):
    n = C.c_int64()
    _check(lib().lbm_read_forces(h, _ptr(dst) if dst is not None else None, int(max_rows), C.byref(n)), h)
    return n.value


def lbm_get_pdfs(h, dst):
    _check(lib().lbm_get_pdfs(h, _ptr(dst)), h)


def lbm_set_pdfs(h, src):
    _check(lib().lbm_set_pdfs(h, _ptr(src)), h)


def lbm_get_cells(h, cells, dst):
    _check(lib().lbm_get_cells(h, len(cells), _ptr(cells), _ptr(dst)), h)


def lbm_init_noise(h, seed, amplitude):
    _check(lib().lbm_init_noise(h, C.c_uint64(seed), float(amplitude)), h)


def lbm_totals(h, out):
    _check(lib().lbm_totals(h, _ptr(out)), h)


def lbm_get_info(h) -> lbm_info:
    out = lbm_info()
    _check(lib().lbm_get_info(h, C.byref(out)), h)
    return out


def lbm_timing(h, enable):
    _check(lib().lbm_timing(h, int(bool(enable))), h)


def lbm_timing_read(h, reset=True) -> lbm_timing_report:
    out = lbm_timing_report()
    _check(lib().lbm_timing_read(h, C.byref(out), int(bool(reset))), h)
    return out


def lbm_totals_noalloc(pdf, storage, slot_stride, mask, grid, stream, out):
    """Totals of a caller-owned device population array (see include/lbm.h);
    allocates no device memory."""
    nx, ny, nz = grid
    _check(lib().lbm_totals_noalloc(_ptr(pdf), int(storage), int(slot_stride),
                                    _ptr(mask) if mask is not None else None, nx, ny, nz,
                                    C.c_void_p(stream or 0), _ptr(out)), None)


def lbm_resample(src, grid, channels, src_layout, dst, out_grid, stream=None):
    """Cell-centred trilinear resampling of device fields (see include/lbm.h):
    src on grid (nx, ny, nz), layout 0 = [z][y][x][C], 1 = [C][z][y][x];
    dst [C][mz][my][mx] on out_grid (mx, my, mz)."""
    nx, ny, nz = grid
    mx, my, mz = out_grid
    _check(lib().lbm_resample(_ptr(src), nx, ny, nz, int(channels), int(src_layout), _ptr(dst), mx, my, mz,
                              C.c_void_p(stream or 0)), None)


def lbm_reset(h):
    _check(lib().lbm_reset(h), h)


def lbm_autotune(h, trials):
    bx, by, ms = C.c_int32(), C.c_int32(), C.c_double()
    _check(lib().lbm_autotune(h, int(trials), C.byref(bx), C.byref(by), C.byref(ms)), h)
    return bx.value, by.value, ms.value


def lbm_batch_create(grids, masks, params, stream=None):
    n = len(grids)
    G = (lbm_grid * n)(*grids)
    M = (C.c_void_p * n)(*[(_ptr(m).value if m is not None else None) for m in masks])
    P = (lbm_params * n)(*params)
    h = C.c_void_p()
    _check(lib().lbm_batch_create(n, G, M, P, C.c_void_p(stream or 0), C.byref(h)), None)
    return h


def lbm_batch_destroy(b):
    _check(lib().lbm_batch_destroy(b), None)


def lbm_batch_set_end(b, t_end):
    arr = (C.c_int64 * len(t_end))(*[int(v) for v in t_end])
    _check(lib().lbm_batch_set_end(b, arr), None)


def lbm_batch_set_flowthroughs(b, n_ft):
    _check(lib().lbm_batch_set_flowthroughs(b, float(n_ft)), None)


def lbm_batch_run(b, n):
    _check(lib().lbm_batch_run(b, int(n)), None)


def lbm_batch_run_to_end(b):
    _check(lib().lbm_batch_run_to_end(b), None)


def lbm_batch_sync(b):
    _check(lib().lbm_batch_sync(b), None)


def lbm_batch_member(b, g):
    h = C.c_void_p()
    _check(lib().lbm_batch_member(b, int(g), C.byref(h)), None)
    return h


def lbm_batch_get_info(b) -> lbm_batch_info:
    out = lbm_batch_info()
    _check(lib().lbm_batch_get_info(b, C.byref(out)), None)
    return out


def lbm_batch_autotune(b, trials):
    bx, by, ms = C.c_int32(), C.c_int32(), C.c_double()
    _check(lib().lbm_batch_autotune(b, int(trials), C.byref(bx), C.byref(by), C.byref(ms)), None)
    return bx.value, by.value, ms.value


def lbm_save(h, path):
    _check(lib().lbm_save(h, os.fsencode(path)), h)


def lbm_load(h, path):
    _check(lib().lbm_load(h, os.fsencode(path)), h)


# ---------------------------------------------------------------------------
# convenience wrapper: torch workspace + current torch stream
# ---------------------------------------------------------------------------
def make_params(**kw) -> lbm_params:
    p = lbm_params_default()
    faces = kw.pop("faces", None)
    if faces is not None:
        p.face_x_lo, p.face_x_hi, p.face_y, p.face_z = (FACES[f] for f in faces)
    st = kw.pop("storage", None)
    if st is not None:
        p.storage = STORAGE[st] if isinstance(st, str) else int(st)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class _Lattice:
    """Read/write methods shared by owned contexts and batch members."""

    h = None
    shape = None
    p = None

    @property
    def t(self):
        return lbm_time(self.h)

    def sync(self):
        lbm_sync(self.h)

    def pdfs(self):
        out = np.zeros((27,) + self.shape)
        lbm_get_pdfs(self.h, out)
        return out

    def set_pdfs(self, f):
        lbm_set_pdfs(self.h, np.ascontiguousarray(f, dtype=np.float64))

    def init_equilibrium(self, fields):
        """Equilibrium of fields [nz, ny, nx, 4] (ux, uy, uz, p) in every fluid cell."""
        if hasattr(fields, "data_ptr"):
            _check(lib().lbm_init_equilibrium(self.h, _ptr(fields.contiguous())), self.h)
        else:
            _check(lib().lbm_init_equilibrium(self.h, _ptr(np.ascontiguousarray(fields, dtype=np.float32))), self.h)

    def cells(self, idx):
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        out = np.zeros((len(idx), 27))
        lbm_get_cells(self.h, idx, out)
        return out

    def macros(self):
        rho = np.zeros(self.shape)
        u = np.zeros(self.shape + (3,))
        lbm_read_macros(self.h, rho, u)
        return rho, u

    def mean(self, halfres=False, dtype=np.float64):
        shape = tuple((s + 1) // 2 for s in self.shape) if halfres else self.shape
        out = np.zeros(shape + (4,), dtype=dtype)
        s = lbm_read_mean(self.h, out, 1 if dtype == np.float32 else 0, halfres)
        return out, s

    def set_wall_distances(self, links):
        """Interpolated bounce-back on the listed obstacle links: (cell,
        direction, q) arrays as returned by inputs.link_wall_distances."""
        lbm_set_wall_distances(self.h, *links)

    def set_probes(self, cells, every=1, capacity=65536):
        """Record (u, v, w, p) at the cells (flat indices) every `every` steps."""
        self._n_probes = len(cells)
        lbm_set_probes(self.h, cells, every, capacity)

    def probes(self):
        """[rows, n_probes, 4] float32: (u, v, w, p) per recorded step."""
        return lbm_read_probes(self.h, getattr(self, "_n_probes", 0))

    def set_plane_monitor(self, z=-1, every=1, capacity=64):
        """Record the (u, v, w, p) of the plane z (default nz/2) every `every` steps."""
        lbm_set_plane_monitor(self.h, z, every, capacity)

    def plane_monitor(self):
        """(planes [k, ny, nx, 4], steps [k]) recorded so far."""
        return lbm_read_plane_monitor(self.h, self.grid.nx, self.grid.ny)

    def stats(self, dtype=np.float64):
        """Velocity covariances [nz, ny, nx, 6] (xx, yy, zz, xy, xz, yz) over
        the averaging samples, and the sample count."""
        out = np.zeros(self.shape + (6,), dtype=dtype)
        s = lbm_read_stats(self.h, out, 1 if dtype == np.float32 else 0)
        return out, s

    def snapshot(self, k):
        shape = tuple((s + 1) // 2 for s in self.shape) if self.p.snap_halfres else self.shape
        out = np.zeros(shape + (4,), dtype=np.float32)
        lbm_read_snapshot(self.h, k, out)
        return out

    def forces(self):
        n = lbm_read_forces(self.h, None, 0)
        out = np.zeros((n, 3))
        if n:
            lbm_read_forces(self.h, out, n)
        return out

    def totals(self):
        out = np.zeros(4)
        lbm_totals(self.h, out)
        return out

    def info(self):
        return lbm_get_info(self.h)


class Solver(_Lattice):
    """One channel-flow lattice on the current CUDA device.

    grid = (nx, ny, nz); mask: uint8 [nz, ny, nx] (1 = solid) or None;
    keyword arguments set lbm_params fields (storage='f32', faces=(...), ...).
    """

    def __init__(self, grid, mask=None, **params):
        import torch

        self.grid = lbm_grid(*grid)
        self.p = make_params(**params)
        self.shape = (grid[2], grid[1], grid[0])
        self.n = int(np.prod(grid))
        self._torch = torch
        m = None
        if mask is not None:
            m = np.ascontiguousarray(mask, dtype=np.uint8)
            assert m.shape == self.shape, (m.shape, self.shape)
        self._mask = m
        nbytes = lbm_workspace_bytes(self.grid, m, self.p)
        if nbytes == 0:
            raise LBMError(LBM_ERR_ARG, "invalid grid or parameters")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.stream = torch.cuda.current_stream()
        self.h = lbm_create_in(self.grid, m, self.p, self.stream.cuda_stream, self.workspace, nbytes)

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        lbm_step(self.h, n)

    def init_noise(self, seed, amplitude):
        lbm_init_noise(self.h, seed, amplitude)

    def reset(self):
        lbm_reset(self.h)

    def autotune(self, trials=10):
        return lbm_autotune(self.h, trials)

    def timing(self, enable=True):
        lbm_timing(self.h, enable)

    def timing_read(self, reset=True):
        return lbm_timing_read(self.h, reset)

    def save(self, path):
        lbm_save(self.h, path)

    def load(self, path):
        lbm_load(self.h, path)


class BatchMember(_Lattice):
    """Borrowed view of one lattice of a Batch (reads only)."""

    def __init__(self, batch, g):
        self._batch = batch
        self.h = lbm_batch_member(batch.h, g)
        d = batch.members[g]
        self.grid = lbm_grid(*d["grid"])
        self.shape = (d["grid"][2], d["grid"][1], d["grid"][0])
        self.p = batch.params[g]


class Batch:
    """Many lattices stepped together (graph-captured batched launches).

    members: list of dicts with keys grid, mask and lbm_params fields.
    """

    def __init__(self, members):
        import torch

        self.members = members
        self.params = []
        grids, masks = [], []
        self._masks = []
        for d in members:
            kw = {k: v for k, v in d.items() if k not in ("grid", "mask")}
            self.params.append(make_params(**kw))
            grids.append(lbm_grid(*d["grid"]))
            m = d.get("mask")
            if m is not None:
                m = np.ascontiguousarray(m, dtype=np.uint8)
            self._masks.append(m)
            masks.append(m)
        self.stream = torch.cuda.current_stream()
        self.h = lbm_batch_create(grids, masks, self.params, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "h", None):
            lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return len(self.members)

    def member(self, g):
        return BatchMember(self, g)

    def set_end(self, t_end):
        lbm_batch_set_end(self.h, t_end)

    def set_flowthroughs(self, n_ft):
        lbm_batch_set_flowthroughs(self.h, n_ft)

    def set_wall_distances(self, g, links):
        """Interpolated bounce-back for member g: (cell, direction, q) arrays
        as returned by inputs.link_wall_distances."""
        cell = np.ascontiguousarray(links[0], dtype=np.int64)
        direction = np.ascontiguousarray(links[1], dtype=np.int8)
        q = np.ascontiguousarray(links[2], dtype=np.float64)
        st = lib().lbm_batch_set_wall_distances(self.h, int(g), len(cell), _ptr(cell), _ptr(direction), _ptr(q))
        if st != 0:
            raise LBMError(st, "lbm_batch_set_wall_distances failed")

    def run(self, n):
        lbm_batch_run(self.h, n)

    def run_to_end(self):
        lbm_batch_run_to_end(self.h)

    def sync(self):
        lbm_batch_sync(self.h)

    def info(self):
        return lbm_batch_get_info(self.h)

    def autotune(self, trials=4):
        return lbm_batch_autotune(self.h, trials)
