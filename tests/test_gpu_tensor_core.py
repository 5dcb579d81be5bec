"""Tensor-core radix-16 stages (FP16 / BF16 operands, FP32 accumulation, plain
and split): each form's error against the FP64 oracle, per transform.  The
split forms must meet the 2e-6 relative-L2 gate of the FP32 path: FP16 as
hi + lo (~22 bits), BF16 as hi + mid + lo (~24 bits).  The plain forms have
their own stated bounds (one rounding to 11 or 8 bits per stage)."""
import numpy as np
import pytest

import fft_inputs
from parity import check, run_gpu, reference, per_transform_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2602_23525_gb300 import gbfft  # noqa: E402

F16, BF16, SPLIT = gbfft.FFT_PREC_TC_FP16, gbfft.FFT_PREC_TC_BF16, gbfft.FFT_PREC_SPLIT
FORMS = {  # flags -> (plan label, bound on the per-transform relative L2 error)
    "fp16": (F16, "tc-fp16 ", 2e-3),
    "bf16": (BF16, "tc-bf16 ", 2e-2),
    "fp16-split": (F16 | SPLIT, "tc-fp16-split", 2e-6),
    "bf16-split": (BF16 | SPLIT, "tc-bf16-split", 2e-6),
}


@pytest.mark.parametrize("form", sorted(FORMS))
@pytest.mark.parametrize("sign", [-1, 1])
def test_batched_4096(form, sign):
    flags, label, tol = FORMS[form]
    n, b = 4096, 37
    x = fft_inputs.uniform_c64(n * b, fft_inputs.seed_for(3, 7))
    err, info = check([(n, 1, 1)], [(b, n, n)], sign, x, flags=flags | gbfft.FFT_ESTIMATE, tol=tol)
    assert label in info
    print(f"{form} n=4096 sign={sign}: max rel-L2 {err:.3e}")


@pytest.mark.parametrize("form", sorted(FORMS))
def test_batched_256_and_columns(form):
    flags, label, tol = FORMS[form]
    n, b = 256, 50
    x = fft_inputs.uniform_c64(n * b, fft_inputs.seed_for(3, 8))
    err, info = check([(n, 1, 1)], [(b, n, n)], -1, x, flags=flags | gbfft.FFT_ESTIMATE, tol=tol)
    assert label in info
    # columns of a 256 x 64 matrix (the strided tile shape)
    x = fft_inputs.uniform_c64(n * 64, fft_inputs.seed_for(3, 9))
    err, info = check([(n, 64, 64)], [(64, 1, 1)], -1, x, flags=flags | gbfft.FFT_ESTIMATE, tol=tol)
    assert label in info and "load=rows" in info


@pytest.mark.parametrize("form", ["fp16-split", "bf16-split", "bf16"])
def test_rank3_64x256x256(form):
    flags, label, tol = FORMS[form]
    shape = (64, 256, 256)
    x = fft_inputs.uniform_c64(int(np.prod(shape)), fft_inputs.seed_for(3, 10))
    dims = [(64, 65536, 65536), (256, 256, 256), (256, 1, 1)]
    err, info = check(dims, [], -1, x, flags=flags | gbfft.FFT_ESTIMATE, tol=tol, algo="ct")
    assert label in info


# the precision workload's 3-D shape: one 256 x 256 x 256 transform, every form
# and plain FP32 on the same input, against one oracle evaluation
DIMS3 = [(256, 65536, 65536), (256, 256, 256), (256, 1, 1)]


@pytest.fixture(scope="module")
def cube():
    x = fft_inputs.uniform_c64(256 ** 3, fft_inputs.seed_for(3, 11))
    ref = reference(DIMS3, [], -1, x, algo="ct")
    return x, ref


@pytest.mark.parametrize("form", sorted(FORMS) + ["fp32"])
def test_rank3_256_cubed(cube, form):
    x, ref = cube
    flags, label, tol = FORMS.get(form, (0, "p2-tma", 2e-6))
    y, info = run_gpu(DIMS3, [], -1, x, flags=flags | gbfft.FFT_ESTIMATE)
    err = float(per_transform_error(y, ref, DIMS3, []).max())
    print(f"256^3 {form}: rel-L2 {err:.3e}")
    assert label in info
    assert np.isfinite(err) and err <= tol, (form, err)
