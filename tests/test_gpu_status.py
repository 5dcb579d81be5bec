"""Plan-level device status (the problem-and-plan interface of sec. 4.1: an
execution's outcome must reach the caller).  Every wait in the kernels is
bounded; a wait that runs out records FFT_ERR_DEVICE_TIMEOUT in the plan's
status word.  FFT_DEBUG_STALL adds one wait, bounded at 50 ms, on an mbarrier
nothing arrives on, so the timeout path runs without any fault: the test
checks that fft_sync_status reports it once, that the next fft_execute reports
an uncollected one without enqueuing, and that the context then still
computes a correct transform."""
import numpy as np
import pytest

import fft_inputs
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2602_23525_gb300 import gbfft  # noqa: E402

n, b = 4096, 16


def rel(y, ref):
    return (np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)).max()


def test_timeout_reported_by_sync_status_then_cleared():
    x = torch.from_numpy(fft_inputs.uniform_c64(n * b, 901)).cuda()
    y = torch.empty_like(x)
    stall = gbfft.Plan([(n, 1, 1)], [(b, n, n)], -1, gbfft.FFT_ESTIMATE | gbfft.FFT_DEBUG_STALL)
    assert "debug stall" in stall.info
    stall.execute(x, y)
    assert gbfft.fft_sync_status(stall.handle) == gbfft.FFT_ERR_DEVICE_TIMEOUT
    assert gbfft.fft_sync_status(stall.handle) == gbfft.FFT_OK  # collected once
    # the transform after the stall ran, and a plain plan still matches the oracle
    ref = oracle.dft(x.cpu().numpy(), [(n, 1, 1)], [(b, n, n)], -1).reshape(b, n)
    assert rel(y.cpu().numpy().astype(np.complex128).reshape(b, n), ref) <= 2e-6
    plain = gbfft.Plan([(n, 1, 1)], [(b, n, n)], -1, gbfft.FFT_ESTIMATE)
    y2 = torch.empty_like(x)
    plain.execute(x, y2)
    assert gbfft.fft_sync_status(plain.handle) == gbfft.FFT_OK
    assert rel(y2.cpu().numpy().astype(np.complex128).reshape(b, n), ref) <= 2e-6
    stall.destroy()
    plain.destroy()


def test_uncollected_timeout_is_returned_by_next_execute():
    x = torch.from_numpy(fft_inputs.uniform_c64(n * b, 902)).cuda()
    y = torch.empty_like(x)
    stall = gbfft.Plan([(n, 1, 1)], [(b, n, n)], 1, gbfft.FFT_ESTIMATE | gbfft.FFT_DEBUG_STALL)
    stall.execute(x, y)
    torch.cuda.synchronize()  # the stall kernel has run: its status is visible to the host
    with pytest.raises(gbfft.GbfftError) as e:
        stall.execute(x, y)
    assert e.value.code == gbfft.FFT_ERR_DEVICE_TIMEOUT
    assert gbfft.fft_last_error() == gbfft.FFT_ERR_DEVICE_TIMEOUT
    # cleared by being reported: the next call runs (and stalls again)
    y.zero_()
    stall.execute(x, y)
    assert gbfft.fft_sync_status(stall.handle) == gbfft.FFT_ERR_DEVICE_TIMEOUT
    ref = oracle.dft(x.cpu().numpy(), [(n, 1, 1)], [(b, n, n)], 1).reshape(b, n)
    assert rel(y.cpu().numpy().astype(np.complex128).reshape(b, n), ref) <= 2e-6
    stall.destroy()


def test_sync_status_without_execution_and_null():
    p = gbfft.Plan([(256, 1, 1)], [(4, 256, 256)], -1, gbfft.FFT_ESTIMATE)
    assert gbfft.fft_sync_status(p.handle) == gbfft.FFT_OK
    p.destroy()
    assert gbfft.load().fft_sync_status(None) == gbfft.FFT_ERR_INVALID_ARG
