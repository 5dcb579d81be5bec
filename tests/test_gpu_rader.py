"""Rader's algorithm for prime lengths (sec. 4.2.5, "Plans for prime sizes"):
the nonzero indices permuted by powers of a generator g of the group modulo p
turn the DFT into a cyclic convolution of length p - 1, evaluated by FFTs of
length p - 1 (when it is smooth) or of a zero-padded power of two.  Every
transform is compared with the FP64 oracle (the DFT's definition) within the
2e-6 relative-L2 gate; both signs, strided and in-place layouts, estimated,
wisdom-forced and measured plans."""
import numpy as np
import pytest

import fft_inputs
from parity import check

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2602_23525_gb300 import gbfft  # noqa: E402


def forced(n, howmany, L, inplace=False):
    """Wisdom text that makes the planner take Rader with convolution length L."""
    v = "[" + ",".join(f"({a},{b},{c})" for a, b, c in howmany) + "]"
    return f"gbfft-wisdom 1\nr1 n={n} is=1 os=1 v={v} ip={1 if inplace else 0}\trader:{L}\n"


@pytest.mark.parametrize("p,b", [(1153, 32), (2689, 16), (7681, 8), (12289, 6)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_smooth_p_minus_1_estimated(p, b, sign):
    x = fft_inputs.uniform_c64(p * b, fft_inputs.seed_for(6, p))
    err, info = check([(p, 1, 1)], [(b, p, p)], sign, x, flags=gbfft.FFT_ESTIMATE)
    assert f"rader p={p}" in info and f"L={p - 1}" in info, info
    print(f"rader p={p} sign={sign}: max rel-L2 {err:.3e}")


@pytest.mark.parametrize("p,L", [(10007, 32768), (17, 32), (61, 128), (1009, 2048), (4099, 16384), (97, 96),
                                 (257, 256)])
def test_wisdom_forced_lengths(p, L):
    b = 5
    how = [(b, p, p)]
    gbfft.fft_import_wisdom(forced(p, how, L))
    try:
        x = fft_inputs.uniform_c64(p * b, fft_inputs.seed_for(6, p + 1))
        for sign in (-1, 1):
            err, info = check([(p, 1, 1)], how, sign, x, flags=gbfft.FFT_ESTIMATE)
            assert f"rader p={p}" in info and f"L={L}" in info, info
            assert ("zero-padded" in info) == (L != p - 1)
    finally:
        gbfft.fft_forget_wisdom()


def test_strided_and_transposed_layouts():
    p, b = 7681, 12
    # transforms down the columns of a p x b row-major array (batch fastest)
    x = fft_inputs.gaussian_c64(p * b, fft_inputs.seed_for(6, 2))
    err, info = check([(p, b, b)], [(b, 1, 1)], -1, x, flags=gbfft.FFT_ESTIMATE)
    assert "rader" in info
    # batch-fastest input into transform-contiguous output
    err, info = check([(p, b, 1)], [(b, 1, p)], 1, x, flags=gbfft.FFT_ESTIMATE)
    assert "rader" in info


def test_in_place():
    p, b = 12289, 4
    x = fft_inputs.uniform_c64(p * b, fft_inputs.seed_for(6, 3))
    err, info = check([(p, 1, 1)], [(b, p, p)], -1, x, flags=gbfft.FFT_ESTIMATE, inplace=True)
    assert "rader" in info and "in-place" in info


def test_single_transform_and_repeat():
    p = 65537
    x = fft_inputs.uniform_c64(p, fft_inputs.seed_for(6, 4))
    err, info = check([(p, 1, 1)], [], -1, x, flags=gbfft.FFT_ESTIMATE, repeat=3)
    assert "rader" in info


@pytest.mark.parametrize("p,b", [(12289, 16), (10007, 16)])
def test_measured_plan(p, b):
    """The measuring planner times Rader against Bluestein; whatever it picks
    matches the oracle."""
    x = fft_inputs.uniform_c64(p * b, fft_inputs.seed_for(6, 5))
    err, info = check([(p, 1, 1)], [(b, p, p)], -1, x, flags=gbfft.FFT_MEASURE)
    assert "rader" in info or "bluestein" in info
    print(info.splitlines()[1])
