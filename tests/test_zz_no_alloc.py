"""fft_execute_1d_noalloc: the entry point for callers that cannot allocate device
memory when they need a transform (it takes its scratch, tables and pass
descriptors from a static device array).  Through the C ABI, two calls in a
row are compared with the planned path (fft_plan_dft + fft_execute) on the
same inputs, within the parity tolerance; sizes beyond the static array's
limit are refused.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import fft_inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import __graft_entry__  # noqa: E402
from paper_2602_23525_gb300 import gbfft  # noqa: E402

TOL = 2e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()


def planned(x, n, batch, sign):
    y = torch.empty_like(x)
    plan = gbfft.Plan([(n, 1, 1)], [(batch, n, n)], sign, gbfft.FFT_ESTIMATE)
    plan.execute(x, y)
    torch.cuda.synchronize()
    plan.destroy()
    return y.cpu().numpy().astype(np.complex128).reshape(batch, n)


def noalloc(x, n, batch, sign):
    y = torch.empty_like(x)
    gbfft.fft_execute_1d_noalloc(n, batch, sign, x.data_ptr(), y.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.complex128).reshape(batch, n)


def rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def test_two_calls_in_a_row_match_planned_path():
    cases = [(65536, 8, -1), (3000, 17, +1)]   # second call: other size and sign
    for i, (n, batch, sign) in enumerate(cases):
        x = torch.from_numpy(fft_inputs.uniform_c64(n * batch, 700 + i)).cuda()
        a = noalloc(x, n, batch, sign)
        b = planned(x, n, batch, sign)
        err = rel(a, b)
        assert np.all(np.isfinite(err)) and err.max() <= TOL, (n, batch, sign, err.max())


def test_in_place_and_the_largest_accepted_size():
    """in == out is accepted; n * batch = GBFFT_NOALLOC_MAX_POINTS is the largest
    call (n = 2^21, batch 1: the largest split-twiddle tables, S = 1449)."""
    n, batch = 1 << 21, 1
    assert n * batch == gbfft.GBFFT_NOALLOC_MAX_POINTS
    x = torch.from_numpy(fft_inputs.uniform_c64(n * batch, 710)).cuda()
    b = planned(x, n, batch, -1)
    a = noalloc(x, n, batch, -1)
    assert rel(a, b).max() <= TOL
    # in place, twice in a row (the second call sees the first call's output)
    for sign, n, batch in ((-1, 4096, 64), (1, 1000, 33)):
        x = torch.from_numpy(fft_inputs.uniform_c64(n * batch, 720 + n)).cuda()
        want = planned(x, n, batch, sign)
        y = x.clone()
        for _ in range(2):
            gbfft.fft_execute_1d_noalloc(n, batch, sign, y.data_ptr(), y.data_ptr(),
                                         torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        twice = y.cpu().numpy().astype(np.complex128).reshape(batch, n)
        want2 = planned(torch.from_numpy(want.astype(np.complex64).reshape(-1)).cuda(), n, batch, sign)
        assert rel(twice, want2).max() <= 4 * TOL


def test_matches_the_oracle():
    import oracle
    n, batch = 3000, 17
    x = fft_inputs.uniform_c64(n * batch, 730)
    a = noalloc(torch.from_numpy(x).cuda(), n, batch, -1)
    ref = oracle.dft(x, [(n, 1, 1)], [(batch, n, n)], -1).reshape(batch, n)
    assert rel(a, ref).max() <= TOL


def test_sizes_beyond_the_static_array_are_refused():
    n = 4096
    batch = gbfft.GBFFT_NOALLOC_MAX_POINTS // n + 1
    x = torch.empty(8, dtype=torch.complex64, device="cuda")
    with pytest.raises(gbfft.GbfftError) as e:
        gbfft.fft_execute_1d_noalloc(n, batch, -1, x.data_ptr(), x.data_ptr(), 0)
    assert e.value.code == gbfft.FFT_ERR_UNSUPPORTED
