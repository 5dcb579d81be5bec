"""DFTs of real data (sec. 5: a real input's conjugate-symmetric spectrum halves
the work; sec. 7: real-data transforms) against the FP64 oracle's real-data
definitions, per transform within 2e-6 relative L2: real-input forward
(half spectrum) and real-output backward (unnormalised) transforms, even
lengths (half-length complex DFT and the pairwise step) and odd or strided
ones (widened to complex), batched and rank-2/3 layouts, and the round trip
c2r(r2c(x)) = N x."""
import numpy as np
import pytest

import fft_inputs
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2602_23525_gb300 import gbfft  # noqa: E402

TOL = 2e-6


def dense(shape):
    return oracle._dense(list(shape))


def r2c_layout(shape):
    """dims (n, is in reals, os in complex) of dense row-major arrays"""
    half = list(shape[:-1]) + [shape[-1] // 2 + 1]
    return [(n, a, b) for (n, a, _), (_, b, _) in zip(dense(shape), dense(half))], int(np.prod(half))


def rel_rows(a, b, rows):
    a = a.reshape(rows, -1)
    b = b.reshape(rows, -1)
    return (np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)).max()


def run(plan, x, out_elems, out_dtype):
    xin = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    y = torch.zeros(out_elems, dtype=out_dtype, device="cuda")
    gbfft.fft_execute(plan, xin.data_ptr(), y.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("n,b", [(4096, 64), (1000, 33), (1 << 16, 8), (30, 100), (4097, 7), (2, 5), (1 << 20, 2),
                                 (10007, 3)])
def test_r2c_batched(n, b):
    x = fft_inputs.uniform_c64(n * b, fft_inputs.seed_for(9, n)).real.astype(np.float32).copy()
    h = n // 2 + 1
    p = gbfft.fft_plan_dft_r2c([(n, 1, 1)], [(b, n, h)], gbfft.FFT_ESTIMATE)
    info = gbfft.fft_plan_info(p)
    y = run(p, x, h * b, torch.complex64)
    gbfft.fft_destroy(p)
    ref = oracle.rdft_r2c(x, [(n, 1, 1)], [(b, n, h)], algo="ct")
    assert ("complex pairs" in info) == (n % 2 == 0), info
    assert rel_rows(y.astype(np.complex128), ref, b) <= TOL, info


@pytest.mark.parametrize("n,b", [(4096, 64), (1000, 33), (1 << 16, 8), (30, 100), (4097, 7), (2, 5), (1 << 20, 2)])
def test_c2r_batched(n, b):
    h = n // 2 + 1
    X = fft_inputs.uniform_c64(h * b, fft_inputs.seed_for(9, n + 1))
    p = gbfft.fft_plan_dft_c2r([(n, 1, 1)], [(b, h, n)], gbfft.FFT_ESTIMATE)
    info = gbfft.fft_plan_info(p)
    y = run(p, X, n * b, torch.float32)
    gbfft.fft_destroy(p)
    ref = oracle.rdft_c2r(X, [(n, 1, 1)], [(b, h, n)], algo="ct")
    assert ("real pairs" in info) == (n % 2 == 0), info
    assert rel_rows(y.astype(np.float64), ref, b) <= TOL, info


def test_strided_layouts_take_the_general_path():
    n, b = 256, 24
    # r2c: input transform stride 3 reals, batch fastest output
    x = np.random.default_rng(5).uniform(-1, 1, 3 * n * b).astype(np.float32)
    h = n // 2 + 1
    p = gbfft.fft_plan_dft_r2c([(n, 3, b)], [(b, 3 * n, 1)], gbfft.FFT_ESTIMATE)
    assert "widened to complex" in gbfft.fft_plan_info(p)
    y = run(p, x, h * b, torch.complex64)
    gbfft.fft_destroy(p)
    ref = oracle.rdft_r2c(x, [(n, 3, b)], [(b, 3 * n, 1)], out_len=h * b)
    assert rel_rows(y.reshape(h, b).T.astype(np.complex128), ref.reshape(h, b).T, b) <= TOL
    # c2r into a strided real output
    X = fft_inputs.uniform_c64(h * b, 77)
    p = gbfft.fft_plan_dft_c2r([(n, b, 2)], [(b, 1, 2 * n)], gbfft.FFT_ESTIMATE)
    assert "conjugate-symmetric extension" in gbfft.fft_plan_info(p)
    y = run(p, X, 2 * n * b, torch.float32)
    gbfft.fft_destroy(p)
    ref = oracle.rdft_c2r(X, [(n, b, 2)], [(b, 1, 2 * n)], out_len=2 * n * b)
    assert rel_rows(y.reshape(b, n, 2)[:, :, 0].astype(np.float64), ref.reshape(b, n, 2)[:, :, 0], b) <= TOL


@pytest.mark.parametrize("shape", [(64, 128), (256, 256), (48, 30), (16, 32, 64), (9, 10, 12)])
def test_multidimensional(shape):
    fwd, hsize = r2c_layout(shape)
    x = np.random.default_rng(len(shape)).uniform(-1, 1, int(np.prod(shape))).astype(np.float32)
    p = gbfft.fft_plan_dft_r2c(fwd, [], gbfft.FFT_ESTIMATE)
    y = run(p, x, hsize, torch.complex64)
    gbfft.fft_destroy(p)
    ref = oracle.rdft_r2c(x, fwd, algo="ct")
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert err <= TOL, (shape, err)
    bwd = [(n, b, a) for n, a, b in fwd]
    p = gbfft.fft_plan_dft_c2r(bwd, [], gbfft.FFT_ESTIMATE)
    z = run(p, y, int(np.prod(shape)), torch.float32)
    gbfft.fft_destroy(p)
    ref2 = oracle.rdft_c2r(y.astype(np.complex128), bwd, algo="ct")
    assert np.linalg.norm(z - ref2) / np.linalg.norm(ref2) <= TOL
    # the round trip: prod(n) x
    assert np.linalg.norm(z / np.prod(shape) - x) / np.linalg.norm(x) <= 4 * TOL


def test_round_trip_and_measured_plans():
    n, b = 1 << 14, 32
    x = np.random.default_rng(9).uniform(-1, 1, n * b).astype(np.float32)
    h = n // 2 + 1
    pf = gbfft.fft_plan_dft_r2c([(n, 1, 1)], [(b, n, h)], gbfft.FFT_MEASURE)
    pb = gbfft.fft_plan_dft_c2r([(n, 1, 1)], [(b, h, n)], gbfft.FFT_MEASURE)
    y = run(pf, x, h * b, torch.complex64)
    z = run(pb, y, n * b, torch.float32)
    assert gbfft.fft_plan_flops(pf) == pytest.approx(2.5 * n * np.log2(n) * b)
    assert gbfft.fft_plan_bytes(pf) == pytest.approx((4 * n + 8 * h) * b)
    gbfft.fft_destroy(pf)
    gbfft.fft_destroy(pb)
    assert rel_rows(z.astype(np.float64) / n, x.astype(np.float64), b) <= 4 * TOL


def test_misaligned_real_array_and_bad_flags_are_refused():
    n = 64
    p = gbfft.fft_plan_dft_r2c([(n, 1, 1)], [], gbfft.FFT_ESTIMATE)
    x = torch.zeros(n + 1, dtype=torch.float32, device="cuda")
    y = torch.zeros(n, dtype=torch.complex64, device="cuda")
    with pytest.raises(gbfft.GbfftError) as e:
        gbfft.fft_execute(p, x.data_ptr() + 4, y.data_ptr(), 0)  # 4-byte aligned real array
    assert e.value.code == gbfft.FFT_ERR_INVALID_ARG
    gbfft.fft_destroy(p)
    for fl in (gbfft.FFT_INPLACE, gbfft.FFT_PREC_TC_FP16):
        with pytest.raises(gbfft.GbfftError) as e:
            gbfft.fft_plan_dft_r2c([(n, 1, 1)], [], fl)
        assert e.value.code == gbfft.FFT_ERR_UNSUPPORTED
