"""GPU parity of the FNO forward x stage on tcgen05 tensor cores (TMEM
accumulators, tensor-map loads; fno_config.umma = 1) against the mma.sync
stage and the FP64 oracle."""
import numpy as np
import pytest

import oracle.fno as F
from tests.test_gpu_fno import GCFG_CACHE, problem, rel_l2, to_gpu_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_16765_gb300 import _build
    _build.build()


def test_tcgen05_x_stage_matches_the_mma_sync_stage_and_the_oracle():
    """umma = 1: the forward x stage of the layer inputs on tcgen05 tensor
    cores (TMEM accumulators, tensor-map loads).  Same contraction as the
    mma.sync stage (BF16 rows exact, twiddles as hi + lo): the forward and
    the gradients agree with the umma = 0 network to 1e-4 and with the
    oracle at the BF16 bounds; no bounded wait gives up."""
    from paper_2606_16765_gb300 import fno as G
    ocfg = F.FNOConfig(grid=(16, 16, 128), modes=(8, 8, 16))
    gcfg = dict(nx=128, ny=16, nz=16, max_batch=8, act_bf16=1, tensor_cores=1)
    GCFG_CACHE["g"] = gcfg
    x, t, m, p = problem(ocfg, B=8, seed=43)
    flat = to_gpu_params(ocfg, p)
    nets = {u: G.FNO(umma=u, **gcfg) for u in (0, 1)}
    out = {}
    for u, net in nets.items():
        net.set_params(flat)
        y = net.forward(x)
        L = net.loss_grad(x, t, m)
        net.sync()
        out[u] = (y, L, net.grads())
    y_ref = F.forward(p, x.astype(np.float64), ocfg)
    print(f"tcgen05 x stage: forward rel L2 vs mma.sync {rel_l2(out[1][0], out[0][0]):.2e}, vs oracle "
          f"{rel_l2(out[1][0], y_ref):.2e}; gradients rel L2 vs mma.sync {rel_l2(out[1][2], out[0][2]):.2e}")
    assert rel_l2(out[1][0], out[0][0]) < 1e-4
    assert abs(out[1][1] - out[0][1]) < 1e-4 * abs(out[0][1])
    assert rel_l2(out[1][2], out[0][2]) < 1e-4
    assert rel_l2(out[1][0], y_ref) < 2e-2
