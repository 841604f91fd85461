"""The allocation-free 2-D real DFT (gfdeconv_fft2_r2c_noalloc) against the
allocating entry point (gfdeconv_fft2_r2c) on the same inputs.

Both run the same row and column passes, so the spectra must agree to the FFT
tolerance of the parity tests (relative rms 1e-6; in practice bit for bit).
The file is named to be collected last: it must pass alone and after every
other GPU test in the same process."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1609_01839_gb300 as gfd  # noqa: E402

DEV = torch.device("cuda:0")
FFT_RTOL = 1e-6


@pytest.fixture(scope="module")
def ctx():
    c = gfd.Context(0)
    yield c
    c.close()


def _image(M, N, seed):
    rng = np.random.default_rng(seed)
    return torch.from_numpy(rng.random((M, N), dtype=np.float64).astype(np.float32)).to(DEV)


def _rel_rms(a, b):
    a = a.cpu().numpy().astype(np.complex128)
    b = b.cpu().numpy().astype(np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("M,N", [(8, 8), (64, 256), (512, 512), (1024, 1024), (4096, 256),
                                 (256, 4096)])
def test_two_calls_in_a_row_match_allocating_entry_point(ctx, M, N):
    x1, x2 = _image(M, N, 1), _image(M, N, 2)
    ref1, ref2 = ctx.fft2_r2c(x1), ctx.fft2_r2c(x2)
    X1 = torch.empty((M, N // 2), dtype=torch.complex64, device=DEV)
    X2 = torch.empty_like(X1)
    X3 = torch.empty_like(X1)
    torch.cuda.synchronize()
    ctx.fft2_r2c_noalloc(x1, X1)
    ctx.fft2_r2c_noalloc(x2, X2)  # second call reuses the same static scratch
    ctx.fft2_r2c_noalloc(x1, X3)
    torch.cuda.synchronize()
    assert _rel_rms(X1, ref1) <= FFT_RTOL
    assert _rel_rms(X2, ref2) <= FFT_RTOL
    assert _rel_rms(X3, ref1) <= FFT_RTOL


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info(DEV)[0]


def test_calls_allocate_no_device_memory(ctx):
    """On a context that has made no call yet, the first two no-alloc calls
    leave free device memory unchanged; as a control, the allocating entry
    point's first call on another fresh context takes its workspace (4 MiB
    here), which shows that the probe sees an allocation of that size."""
    M, N = 1024, 1024
    x = _image(M, N, 3)
    X = torch.empty((M, N // 2), dtype=torch.complex64, device=DEV)
    stream = torch.cuda.current_stream(DEV).cuda_stream
    ctx.fft2_r2c_noalloc(x, X)  # the per-device symbol lookup is done once per process
    fresh = gfd.Context(0)
    try:
        free0 = _free_bytes()
        for _ in range(2):
            rc = gfd.lib.gfdeconv_fft2_r2c_noalloc(fresh._h, x.data_ptr(), M, N, X.data_ptr(),
                                                   stream)
            assert rc == 0
        assert _free_bytes() == free0
    finally:
        fresh.close()
    control = gfd.Context(0)
    try:
        free0 = _free_bytes()
        rc = gfd.lib.gfdeconv_fft2_r2c(control._h, x.data_ptr(), M, N, X.data_ptr(), stream)
        assert rc == 0
        assert free0 - _free_bytes() >= 4 * M * N
    finally:
        control.close()


def test_size_beyond_static_scratch_rejected(ctx):
    M, N = 2048, 1024  # 2 M pixels > 1024 * 1024
    x = torch.zeros((M, N), dtype=torch.float32, device=DEV)
    X = torch.empty((M, N // 2), dtype=torch.complex64, device=DEV)
    with pytest.raises(gfd.GfdError) as ei:
        ctx.fft2_r2c_noalloc(x, X)
    assert ei.value.code == gfd.ERR_SCRATCH_LIMIT
    assert "static scratch" in str(ei.value)
