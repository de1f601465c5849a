"""Shared case descriptions for the parity tests: one dict describes a
lattice, and the helpers build the same case on the FP64 oracle and on the
CUDA library.  Inputs come from paper_2606_16765_gb300.inputs only."""
import numpy as np

from paper_2606_16765_gb300 import inputs as I

Q = 27


def case(grid, mask=None, omega1=1.8, omega_bulk=1.0, omega_higher=1.0, galilean=1, u_in=0.05,
         faces=("inlet", "outlet", "wall", "wall"), mean=(0, 0, 0), noise=None, param4=0):
    return dict(grid=tuple(grid), mask=mask, omega1=omega1, omega_bulk=omega_bulk,
                omega_higher=omega_higher, galilean=galilean, u_in=u_in, faces=tuple(faces),
                mean=tuple(mean), noise=noise, param4=param4)


def noise_state(grid, mask, seed, amp, weights):
    """Full populations w_i + amp * r(seed, cell*27 + i) for fluid cells,
    w_i for solid cells, direction-major [27, nz, ny, nx]."""
    nx, ny, nz = grid
    n = nx * ny * nz
    r = I.pdf_noise(seed, np.arange(n))
    f = weights[:, None] + amp * r
    if mask is not None:
        f[:, mask.reshape(-1) != 0] = weights[:, None]
    return f.reshape(Q, nz, ny, nx)


def run_oracle(c, steps):
    import oracle.lbm as O
    nx, ny, nz = c["grid"]
    p = O.params(nx, ny, nz, c["omega1"], c["omega_bulk"], c["omega_higher"], galilean=c["galilean"],
                 u_in=c["u_in"], faces=c["faces"], mean=c["mean"], param4=c.get("param4", 0))
    L = O.Lattice(p, c["mask"])
    if c["noise"] is not None:
        seed, amp = c["noise"]
        L.set_f(noise_state(c["grid"], c["mask"], seed, amp, O.weights()))
    if steps:
        L.step(steps)
    return L


def make_solver(c, storage, **extra):
    from paper_2606_16765_gb300.lbm import Solver
    m, e, v = c["mean"]
    s = Solver(c["grid"], c["mask"], storage=storage, omega1=c["omega1"], omega_bulk=c["omega_bulk"],
               omega_higher=c["omega_higher"], galilean_correction=c["galilean"], u_in=c["u_in"],
               faces=c["faces"], mean_start=m, mean_end=e, mean_every=v, param4=c.get("param4", 0), **extra)
    if c["noise"] is not None:
        s.init_noise(*c["noise"])
    return s


def rel_u_err(u, u_ref, fluid):
    """max |u - u_ref| / max |u_ref| over fluid cells (velocity components jointly)."""
    d = np.abs(u - u_ref)[fluid]
    return d.max() / max(np.abs(u_ref[fluid]).max(), 1e-300)


def rho_err(rho, rho_ref, fluid):
    return np.abs(rho - rho_ref)[fluid].max()
