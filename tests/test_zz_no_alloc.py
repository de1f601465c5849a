"""GPU test of lbm_totals_noalloc, the entry point for callers that cannot
allocate device memory where they need mass and momentum totals (a monitor
thread beside a solver it does not own, where cudaMalloc/cudaFree could
synchronise the device; an application whose device memory belongs to a
framework's pool).

The same seeded state is held twice: by a library context (initialised with
lbm_init_noise) and by a caller-owned torch buffer in the natural layout.
The allocation-free entry point, called twice in a row through the C ABI on
the caller's buffer, must give the totals the context's lbm_totals gives,
within the FP64 tolerance of the other totals tests.  This file is collected
last so that a run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_16765_gb300 import _build
    _build.build()


@pytest.mark.parametrize("storage,dtype", [("f32", "float32"), ("f64", "float64")])
def test_noalloc_totals_match_context_totals(storage, dtype):
    import torch
    from paper_2606_16765_gb300 import inputs as I
    from paper_2606_16765_gb300 import lbm as B

    grid = (40, 24, 20)
    nx, ny, nz = grid
    n = nx * ny * nz
    mask = I.sphere(grid, (12.0, 11.5, 9.5), 5.0)
    seed, amp = 4242, 3e-3

    s = B.Solver(grid, mask, storage=storage, omega1=1.8, u_in=0.05)
    s.init_noise(seed, amp)
    ref = s.totals()                      # existing entry point (context scratch)

    # the same state in a caller-owned buffer: f_i - w_i, direction-major,
    # slot stride larger than n to exercise the stride argument
    slot = n + 96
    fbar = amp * I.pdf_noise(seed, np.arange(n))
    fbar[:, mask.reshape(-1) != 0] = 0.0
    host = np.zeros((27, slot), dtype=np.float64)
    host[:, :n] = fbar
    tdt = getattr(torch, dtype)
    pdf = torch.from_numpy(host).to(device="cuda", dtype=tdt)
    dmask = torch.from_numpy(np.ascontiguousarray(mask).reshape(-1)).to("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    st = B.STORAGE[storage]

    out1 = np.zeros(4)
    B.lbm_totals_noalloc(pdf, st, slot, dmask, grid, stream, out1)
    out2 = torch.zeros(4, dtype=torch.float64, device="cuda")   # device output, second call
    B.lbm_totals_noalloc(pdf, st, slot, dmask, grid, stream, out2)
    torch.cuda.synchronize()
    out2 = out2.cpu().numpy()

    assert np.abs(out1 - ref).max() <= TOL
    assert np.abs(out2 - ref).max() <= TOL
    assert np.array_equal(out1, out2)         # fixed-order reduction: same bits


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    from paper_2606_16765_gb300 import lbm as B

    pdf = torch.zeros(27, dtype=torch.float32, device="cuda")
    out = np.zeros(4)
    with pytest.raises(B.LBMError) as e:
        B.lbm_totals_noalloc(pdf, B.LBM_F32, 2 ** 31, None, (2048, 1024, 1024), 0, out)
    assert e.value.status == B.LBM_ERR_ARG
    assert "capacity" in str(e.value)
