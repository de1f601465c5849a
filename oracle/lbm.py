"""ctypes front end of the FP64 C oracle (test infrastructure only).

Layouts: pdfs are direction-major ``f[i, z, y, x]`` (full populations, not the
shifted ones), macros ``rho[z, y, x]`` and ``u[z, y, x, 3]``, means
``[z, y, x, 4]`` holding (ux, uy, uz, p) with p = (rho - 1)/3.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

FACE_WALL, FACE_PERIODIC, FACE_INLET, FACE_OUTLET, FACE_OUTFLOW = 0, 1, 2, 3, 4
Q = 27


class OracleParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("face_x_lo", C.c_int32), ("face_x_hi", C.c_int32),
        ("face_y", C.c_int32), ("face_z", C.c_int32),
        ("omega1", C.c_double), ("omega2", C.c_double), ("omega3", C.c_double),
        ("galilean", C.c_int32), ("pad0", C.c_int32),
        ("u_in", C.c_double), ("rho_in", C.c_double), ("rho_out", C.c_double),
        ("mean_start", C.c_int64), ("mean_end", C.c_int64), ("mean_every", C.c_int64),
        ("param4", C.c_int32), ("pad1", C.c_int32), ("limiter", C.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        P = C.POINTER(OracleParams)
        L.oracle_weights.argtypes = [dp]
        L.oracle_omega_from_re.argtypes = [C.c_double] * 3
        L.oracle_omega_from_re.restype = C.c_double
        L.oracle_param4_rates.argtypes = [C.c_double, C.c_double, dp]
        L.oracle_equilibrium.argtypes = [C.c_double] * 4 + [dp]
        L.oracle_macros.argtypes = [dp, dp, dp]
        L.oracle_central_moments.argtypes = [dp, dp, dp, dp]
        L.oracle_cumulants_from_moments.argtypes = [dp, dp]
        L.oracle_moments_from_cumulants.argtypes = [dp, dp]
        L.oracle_relax.argtypes = [P, dp, dp, dp]
        L.oracle_pdfs_from_moments.argtypes = [dp, C.c_double, dp, dp]
        L.oracle_collide.argtypes = [P, dp, dp, dp, dp]
        L.oracle_lbm_create.argtypes = [P, C.c_void_p]
        L.oracle_lbm_create.restype = C.c_void_p
        L.oracle_lbm_destroy.argtypes = [C.c_void_p]
        L.oracle_lbm_set_f.argtypes = [C.c_void_p, dp]
        L.oracle_lbm_get_f.argtypes = [C.c_void_p, dp]
        L.oracle_lbm_time.argtypes = [C.c_void_p]
        L.oracle_lbm_time.restype = C.c_int64
        L.oracle_lbm_set_time.argtypes = [C.c_void_p, C.c_int64]
        L.oracle_lbm_macros.argtypes = [C.c_void_p, dp, dp]
        L.oracle_lbm_means.argtypes = [C.c_void_p, dp]
        L.oracle_lbm_means.restype = C.c_int64
        L.oracle_lbm_stats.argtypes = [C.c_void_p, dp]
        L.oracle_lbm_stats.restype = C.c_int64
        L.oracle_lbm_set_q.argtypes = [C.c_void_p, C.c_void_p]
        L.oracle_lbm_set_q.restype = None
        L.oracle_lbm_forces.argtypes = [C.c_void_p, dp]
        L.oracle_lbm_step.argtypes = [C.c_void_p, C.c_int]
        L.oracle_lbm_totals.argtypes = [C.c_void_p, dp]
        _lib = L
    return _lib


def _dp(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def weights():
    w = np.zeros(Q)
    lib().oracle_weights(_dp(w))
    return w


def velocities():
    i = np.arange(Q)
    return np.stack([i % 3 - 1, (i // 3) % 3 - 1, i // 9 - 1], axis=1)


def omega_from_re(re, u, l_ref):
    return lib().oracle_omega_from_re(re, u, l_ref)


def params(nx, ny, nz, omega1, omega2=1.0, omega3=1.0, galilean=1, u_in=0.0,
           rho_in=1.0, rho_out=1.0, faces=("inlet", "outlet", "wall", "wall"),
           mean=(0, 0, 0), param4=0, limiter=0.01):
    kinds = {"wall": FACE_WALL, "periodic": FACE_PERIODIC,
             "inlet": FACE_INLET, "outlet": FACE_OUTLET, "outflow": FACE_OUTFLOW}
    p = OracleParams()
    p.nx, p.ny, p.nz = nx, ny, nz
    p.face_x_lo, p.face_x_hi, p.face_y, p.face_z = (kinds[f] for f in faces)
    p.omega1, p.omega2, p.omega3 = omega1, omega2, omega3
    p.galilean = int(galilean)
    p.u_in, p.rho_in, p.rho_out = u_in, rho_in, rho_out
    p.mean_start, p.mean_end, p.mean_every = mean
    p.param4, p.limiter = int(param4), float(limiter)
    return p


def param4_rates(w1, w2=1.0):
    """(omega3, omega4, omega5, A, B) of the fourth-order parametrisation."""
    out = np.zeros(5)
    lib().oracle_param4_rates(float(w1), float(w2), _dp(out))
    return out


def equilibrium(rho, ux, uy, uz):
    f = np.zeros(Q)
    lib().oracle_equilibrium(rho, ux, uy, uz, _dp(f))
    return f


def central_moments(f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    k = np.zeros(Q)
    rho = C.c_double()
    u = np.zeros(3)
    lib().oracle_central_moments(_dp(f), _dp(k), C.byref(rho), _dp(u))
    return k, rho.value, u


def cumulants(k):
    k = np.ascontiguousarray(k, dtype=np.float64)
    c = np.zeros(Q)
    lib().oracle_cumulants_from_moments(_dp(k), _dp(c))
    return c


def moments_from_cumulants(c):
    c = np.ascontiguousarray(c, dtype=np.float64)
    k = np.zeros(Q)
    lib().oracle_moments_from_cumulants(_dp(c), _dp(k))
    return k


def pdfs_from_moments(k, rho, u):
    k = np.ascontiguousarray(k, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    f = np.zeros(Q)
    lib().oracle_pdfs_from_moments(_dp(k), rho, _dp(u), _dp(f))
    return f


def collide(p, f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(Q)
    lib().oracle_collide(C.byref(p), _dp(f), _dp(out), None, None)
    return out


class Lattice:
    """FP64 two-array pull-streaming lattice."""

    def __init__(self, p, solid=None):
        self.p = p
        self.shape = (p.nz, p.ny, p.nx)
        self.n = p.nx * p.ny * p.nz
        if solid is not None:
            solid = np.ascontiguousarray(solid, dtype=np.uint8)
            assert solid.shape == self.shape
            self.solid = solid
            ptr = solid.ctypes.data_as(C.c_void_p)
        else:
            self.solid = np.zeros(self.shape, np.uint8)
            ptr = None
        self.h = lib().oracle_lbm_create(C.byref(p), ptr)

    def __del__(self):
        if getattr(self, "h", None):
            lib().oracle_lbm_destroy(self.h)
            self.h = None

    @property
    def t(self):
        return lib().oracle_lbm_time(self.h)

    @t.setter
    def t(self, v):
        lib().oracle_lbm_set_time(self.h, int(v))

    def set_f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(Q, *self.shape)
        lib().oracle_lbm_set_f(self.h, _dp(f))

    def get_f(self):
        f = np.zeros((Q,) + self.shape)
        lib().oracle_lbm_get_f(self.h, _dp(f))
        return f

    def step(self, n=1):
        lib().oracle_lbm_step(self.h, int(n))

    def macros(self):
        rho = np.zeros(self.shape)
        u = np.zeros(self.shape + (3,))
        lib().oracle_lbm_macros(self.h, _dp(rho), _dp(u))
        return rho, u

    def means(self):
        out = np.zeros(self.shape + (4,))
        s = lib().oracle_lbm_means(self.h, _dp(out))
        return out, s

    def set_q(self, q):
        """Wall distances [27, nz, ny, nx] of the links x -> x + c_j into
        obstacle cells (interpolated bounce-back), or None for halfway."""
        if q is None:
            lib().oracle_lbm_set_q(self.h, None)
        else:
            q = np.ascontiguousarray(q, dtype=np.float64)
            lib().oracle_lbm_set_q(self.h, q.ctypes.data)

    def stats(self):
        """Velocity covariances [..., 6] (xx, yy, zz, xy, xz, yz) over the
        averaging samples, and the sample count."""
        out = np.zeros(self.shape + (6,))
        s = lib().oracle_lbm_stats(self.h, _dp(out))
        return out, s

    def forces(self):
        out = np.zeros((self.t, 3))
        if self.t:
            lib().oracle_lbm_forces(self.h, _dp(out))
        return out

    def totals(self):
        out = np.zeros(4)
        lib().oracle_lbm_totals(self.h, _dp(out))
        return out


def halfres(field):
    """2x2x2 box mean of a [z, y, x, ...] field; a trailing odd cell forms a
    block of its own (averaged over the cells it has)."""
    f = np.asarray(field, dtype=np.float64)
    nz, ny, nx = f.shape[:3]
    hz, hy, hx = (nz + 1) // 2, (ny + 1) // 2, (nx + 1) // 2
    acc = np.zeros((hz, hy, hx) + f.shape[3:])
    cnt = np.zeros((hz, hy, hx))
    for dz in range(2):
        for dy in range(2):
            for dx in range(2):
                sub = f[dz::2, dy::2, dx::2]
                acc[:sub.shape[0], :sub.shape[1], :sub.shape[2]] += sub
                cnt[:sub.shape[0], :sub.shape[1], :sub.shape[2]] += 1
    return acc / cnt.reshape(cnt.shape + (1,) * (f.ndim - 3))
