"""Host logic of the FFNO binding: the flat parameter layout of
include/ffno.h holds exactly the oracle's parameters, and flattening is
exact in both directions."""
import numpy as np

from oracle import ffno as F
from paper_2606_16765_gb300 import ffno as G


class Cfg:
    """The binding's layout reads only these fields."""
    nx, ny, nz, cin, width, cout = 8, 5, 6, 2, 3, 2
    mx, my, mz, layers, ff_hidden, hidden, lift_hidden = 4, 3, 2, 2, 4, 5, 3


def oracle_cfg():
    return F.FFNOConfig(grid=(6, 5, 8), cin=2, width=3, cout=2, modes=(2, 3, 4), layers=2, ff_hidden=4, hidden=5,
                        lift_hidden=3)


def test_layout_holds_the_oracle_parameters():
    p = F.init_params(oracle_cfg(), seed=3)
    names = [n for n, _, _ in G.layout(Cfg)]
    assert sorted(names) == sorted(p)
    for n, shape, cplx in G.layout(Cfg):
        assert p[n].shape == shape and np.iscomplexobj(p[n]) == cplx, n


def test_flatten_round_trip():
    p = F.init_params(oracle_cfg(), seed=4)
    flat = G.flatten(Cfg, p)
    n = sum(int(np.prod(s)) * (2 if c else 1) for _, s, c in G.layout(Cfg))
    assert flat.size == n
    q = G.unflatten(Cfg, flat)
    for k in p:
        assert np.array_equal(q[k], p[k].astype(np.complex64 if np.iscomplexobj(p[k]) else np.float32)), k
