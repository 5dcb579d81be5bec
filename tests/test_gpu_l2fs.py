"""The four-step of eq. (2) in one persistent kernel with its intermediate in an
L2-resident ring (sec. 3.3: blocking so that the radix-sqrt(n) step's data
stays in cache): every supported split n1 x n2 = 2^14 .. 2^22, both signs,
several ring lags (many transforms, a few, one), a padded vector stride, an
unaligned input (no tensor map: plain loads), in place, and the measured plan
at the benchmark's full size on sampled transforms, each against the FP64
oracle within 2e-6 per transform."""
import numpy as np
import pytest

import fft_inputs
import oracle
from parity import check

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2602_23525_gb300 import gbfft  # noqa: E402


def force(n, how, n1, inplace=False):
    v = "[" + ",".join(f"({a},{b},{c})" for a, b, c in how) + "]"
    gbfft.fft_forget_wisdom()
    gbfft.fft_import_wisdom(f"gbfft-wisdom 1\nr1 n={n} is=1 os=1 v={v} ip={1 if inplace else 0}\tl2fs:{n1}\n")


SPLITS = [(7, 7, 24), (7, 8, 12), (8, 8, 9), (8, 9, 5), (9, 9, 3), (9, 10, 3), (10, 10, 2), (10, 11, 2),
          (11, 11, 1)]


@pytest.mark.parametrize("l1,l2,b", SPLITS)
@pytest.mark.parametrize("sign", [-1, 1])
def test_every_split(l1, l2, b, sign):
    n, n1 = 1 << (l1 + l2), 1 << l1
    how = [(b, n, n)] if b > 1 else []
    force(n, how, n1)
    try:
        x = fft_inputs.uniform_c64(n * b, fft_inputs.seed_for(8, l1 + l2))
        err, info = check([(n, 1, 1)], how, sign, x, flags=gbfft.FFT_ESTIMATE, algo="ct")
        assert "pass l2-fourstep" in info, info
    finally:
        gbfft.fft_forget_wisdom()


def test_many_transforms_long_ring_padded_stride():
    n, b = 1 << 14, 300  # lag and ring of many transforms; vector stride n + 2
    how = [(b, n + 2, n + 6)]
    force(n, how, 128)
    try:
        x = fft_inputs.uniform_c64((n + 2) * b, fft_inputs.seed_for(8, 1))
        err, info = check([(n, 1, 1)], how, -1, x, flags=gbfft.FFT_ESTIMATE, algo="ct")
        assert "pass l2-fourstep" in info
    finally:
        gbfft.fft_forget_wisdom()


def test_unaligned_input_uses_plain_loads():
    n, b = 1 << 16, 4
    how = [(b, n, n)]
    force(n, how, 256)
    try:
        x = fft_inputs.uniform_c64(n * b + 1, fft_inputs.seed_for(8, 2))
        # element 0 at an odd element offset: 8-byte but not 16-byte aligned
        err, info = check([(n, 1, 1)], how, 1, x, flags=gbfft.FFT_ESTIMATE, algo="ct", in_offset=1)
        assert "pass l2-fourstep" in info
    finally:
        gbfft.fft_forget_wisdom()


def test_in_place():
    n, b = 1 << 18, 6
    how = [(b, n, n)]
    force(n, how, 512, inplace=True)
    try:
        x = fft_inputs.uniform_c64(n * b, fft_inputs.seed_for(8, 3))
        err, info = check([(n, 1, 1)], how, -1, x, flags=gbfft.FFT_ESTIMATE, algo="ct", inplace=True)
        assert "pass l2-fourstep" in info
    finally:
        gbfft.fft_forget_wisdom()


@pytest.mark.parametrize("e", [14, 17, 20])
def test_full_size_measured_plan_sampled(e):
    """2^26 points with the measured plan, repeated: sampled transforms vs the oracle."""
    n = 1 << e
    b = (1 << 26) // n
    x = fft_inputs.uniform_c64(n * b, fft_inputs.seed_for(1, e))
    xin = torch.from_numpy(x).cuda()
    y = torch.empty_like(xin)
    gbfft.fft_forget_wisdom()
    plan = gbfft.Plan([(n, 1, 1)], [(b, n, n)], -1, gbfft.FFT_MEASURE)
    for _ in range(3):
        plan.execute(xin, y)
    assert gbfft.fft_sync_status(plan.handle) == gbfft.FFT_OK
    yh = y.cpu().numpy()
    print(plan.info.splitlines()[1])
    for v in (0, 1, b // 2, b - 1):
        ref = oracle.dft(x[v * n:(v + 1) * n], [(n, 1, 1)], [], -1, algo="ct")
        got = yh[v * n:(v + 1) * n].astype(np.complex128)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 2e-6, (v, err)
    plan.destroy()


@pytest.mark.parametrize("e,b", [(22, 2), (23, 1), (24, 1)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_group_mode_inner_transforms(e, b, sign):
    """2^22..2^24 as n1 x 65536 (eq. (2)): the n1-point column pass, then the
    65536-point rows in the L2-resident four-step whose B items take one row
    of 8 transforms, two rows each, and store their outputs n1 apart (group
    mode), against
    the FP64 oracle on every transform."""
    n = 1 << e
    how = [(b, n, n)] if b > 1 else []
    x = fft_inputs.uniform_c64(n * b, fft_inputs.seed_for(8, e + b))
    err, info = check([(n, 1, 1)], how, sign, x, flags=gbfft.FFT_ESTIMATE, algo="ct")
    assert f"= {1 << (e - 16)} x 65536" in info and "B items over 2 rows of 8 transforms" in info, info


def test_group_mode_padded_batch_and_full_size_sampled():
    """A padded batch stride (the column pass writes the rows contiguously, so
    the group kernel sees the same layout) and 2^24 x 4 at full size with the
    measured plan, on sampled transforms."""
    n, b = 1 << 22, 3
    how = [(b, n + 8, n + 16)]
    x = fft_inputs.uniform_c64((n + 8) * b, fft_inputs.seed_for(8, 40))
    err, info = check([(n, 1, 1)], how, -1, x, flags=gbfft.FFT_ESTIMATE, algo="ct")
    assert "B items over 2 rows of 8 transforms" in info, info
    n, b = 1 << 24, 4
    x = fft_inputs.uniform_c64(n * b, fft_inputs.seed_for(8, 41))
    xin = torch.from_numpy(x).cuda()
    y = torch.empty_like(xin)
    gbfft.fft_forget_wisdom()
    plan = gbfft.Plan([(n, 1, 1)], [(b, n, n)], 1, gbfft.FFT_MEASURE)
    for _ in range(2):
        plan.execute(xin, y)
    assert gbfft.fft_sync_status(plan.handle) == gbfft.FFT_OK
    print(plan.info)
    yh = y.cpu().numpy()
    for v in (0, b - 1):
        ref = oracle.dft(x[v * n:(v + 1) * n], [(n, 1, 1)], [], 1, algo="ct")
        got = yh[v * n:(v + 1) * n].astype(np.complex128)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 2e-6, v
    plan.destroy()
