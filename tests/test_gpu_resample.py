"""GPU parity of lbm_resample (mean fields onto the surrogate's 128x64x64
grid) against the FP64 reference oracle.resample: FP32 arithmetic, max error
<= 1e-6 of the field's scale, for every grid of the batched configuration's
set {128,192,256} x {64,96,128}^2 that the tests sample and both source
layouts."""
import numpy as np
import pytest

import oracle.resample as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_16765_gb300 import _build
    _build.build()


@pytest.mark.parametrize("grid", [(192, 96, 128), (256, 128, 64), (128, 64, 96), (128, 64, 64), (100, 30, 70)])
@pytest.mark.parametrize("layout", [0, 1])
def test_resample_matches_oracle(grid, layout):
    import torch
    from paper_2606_16765_gb300 import lbm as B
    nx, ny, nz = grid
    r = np.random.default_rng(nx + 7 * ny + 31 * nz + layout)
    f = r.normal(size=(4, nz, ny, nx)).astype(np.float32)             # [C][z][y][x]
    src_host = f if layout == 1 else np.ascontiguousarray(np.moveaxis(f, 0, -1))
    src = torch.from_numpy(np.ascontiguousarray(src_host)).cuda()
    out = (128, 64, 64)
    dst = torch.full((4, 64, 64, 128), float("nan"), device="cuda")
    B.lbm_resample(src, grid, 4, layout, dst, out, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    ref = R.resample(f.astype(np.float64), (64, 64, 128))
    err = np.abs(dst.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < 1e-6, err


def test_resample_refuses_host_arrays():
    import torch
    from paper_2606_16765_gb300 import lbm as B
    host = np.zeros((4, 8, 8, 8), np.float32)
    dst = torch.zeros((4, 4, 4, 4), device="cuda")
    with pytest.raises(B.LBMError) as e:
        B.lbm_resample(host, (8, 8, 8), 4, 1, dst, (4, 4, 4))
    assert e.value.status == B.LBM_ERR_ARG
