"""GPU test of lbm_totals_noalloc, the entry point for callers that cannot
allocate device memory where they need mass and momentum totals (a monitor
thread beside a solver it does not own, where cudaMalloc/cudaFree could
synchronise the device; an application whose device memory belongs to a
framework's pool).

The same seeded state is held twice: by a library context (initialised with
lbm_init_noise) and by a caller-owned torch buffer that holds the context's
stored values in the natural layout, encoded in the same storage format.  The
allocation-free entry point, called twice in a row through the C ABI on the
caller's buffer, must give the totals the context's lbm_totals gives and the
exactly rounded sums (math.fsum) of the same values.  Both sides reduce the
same decoded values in FP64, so one FP64 tolerance serves every storage
format.  This file is collected last so that a run stopping at the first
failure has run everything else.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12
STORAGES = ["f64", "f32", "f16s", "bf16s", "f16c"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_16765_gb300 import _build
    _build.build()


def encode_f16c(v):
    """Bits of the library's 16-bit F16C code (sign, 4 exponent bits with bias
    15, 11 mantissa bits) for values that the code represents exactly: the
    FP32 pattern of v * 2^-112 with its low 12 mantissa bits dropped."""
    f = (np.asarray(v, np.float64) * 2.0 ** -112).astype(np.float32)
    assert np.array_equal(f.astype(np.float64) * 2.0 ** 112, v)      # exact scaling
    u = f.view(np.uint32)
    assert not np.any(u & 0xFFF)                                     # representable
    return (((u >> 16) & 0x8000) | ((u >> 12) & 0x7FFF)).astype(np.uint16)


def caller_buffer(fbar, storage, slot):
    """Device buffer [27][slot] holding fbar (exactly representable in
    `storage`) in that storage's encoding."""
    import torch
    host = np.zeros((27, slot), dtype=np.float64)
    host[:, :fbar.shape[1]] = fbar
    if storage == "f16c":
        return torch.from_numpy(encode_f16c(host).view(np.int16)).to("cuda")
    tdt = {"f64": torch.float64, "f32": torch.float32, "f16s": torch.float16, "bf16s": torch.bfloat16}[storage]
    t = torch.from_numpy(host).to(dtype=tdt)
    assert np.array_equal(t.to(torch.float64).numpy(), host)         # exactly representable
    return t.to("cuda")


@pytest.mark.parametrize("storage", STORAGES)
def test_noalloc_totals_match_context_totals(storage):
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
    tw = lambda k: 2.0 / 3.0 if k == 1 else 1.0 / 6.0
    w = np.array([tw(i % 3) * tw((i // 3) % 3) * tw(i // 9) for i in range(27)])   # the library's own product
    fl = mask.reshape(-1) == 0
    if storage == "f64":
        fbar = amp * I.pdf_noise(seed, np.arange(n))
    else:
        # the context's stored values: (f_i - w_i) + w_i - w_i is exact in FP64
        # for values with at most 24 significant bits
        fbar = s.pdfs().reshape(27, n) - w[:, None]
    fbar[:, ~fl] = 0.0
    s.close()
    cv = np.stack([np.arange(27) % 3 - 1, (np.arange(27) // 3) % 3 - 1, np.arange(27) // 9 - 1], 1)
    exact = np.array([math.fsum(fbar[:, fl].ravel())] +
                     [math.fsum((cv[:, a, None] * fbar[:, fl]).ravel()) for a in range(3)])

    # caller-owned buffer with a slot stride larger than n (the stride argument)
    slot = n + 96
    pdf = caller_buffer(fbar, storage, slot)
    dmask = torch.from_numpy(np.ascontiguousarray(mask).reshape(-1)).to("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    st = B.STORAGE[storage]

    out1 = np.zeros(4)
    B.lbm_totals_noalloc(pdf, st, slot, dmask, grid, stream, out1)
    out2 = torch.zeros(4, dtype=torch.float64, device="cuda")   # device output, second call
    B.lbm_totals_noalloc(pdf, st, slot, dmask, grid, stream, out2)
    torch.cuda.synchronize()
    out2 = out2.cpu().numpy()

    assert np.abs(exact - ref).max() <= TOL          # the two references agree
    assert np.abs(out1 - ref).max() <= TOL
    assert np.abs(out2 - ref).max() <= TOL
    assert np.abs(out1 - exact).max() <= TOL
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


def test_noalloc_rejects_host_arrays_before_launching():
    import torch
    from paper_2606_16765_gb300 import lbm as B

    grid = (8, 4, 4)
    n = 8 * 4 * 4
    out = np.zeros(4)
    host_pdf = np.zeros(27 * n, np.float32)
    with pytest.raises(B.LBMError) as e:
        B.lbm_totals_noalloc(host_pdf, B.LBM_F32, n, None, grid, 0, out)
    assert e.value.status == B.LBM_ERR_ARG and "device" in str(e.value)
    dev_pdf = torch.zeros(27 * n, dtype=torch.float32, device="cuda")
    host_mask = np.zeros(n, np.uint8)
    with pytest.raises(B.LBMError) as e:
        B.lbm_totals_noalloc(dev_pdf, B.LBM_F32, n, host_mask, grid, 0, out)
    assert e.value.status == B.LBM_ERR_ARG and "device" in str(e.value)
    torch.cuda.synchronize()                       # the context is still usable
    B.lbm_totals_noalloc(dev_pdf, B.LBM_F32, n, None, grid, 0, out)
    assert np.array_equal(out, np.zeros(4))
