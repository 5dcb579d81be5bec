"""Device twiddle and chirp tables read back and checked entry by entry against
a host FP64 evaluation (sec. 6: twiddles accurate to about machine precision,
computed from an exactly reduced exponent, rounded once to FP32).

The host reference takes each entry's exponent from Python integers, reduces
the angle to a quadrant exactly in integers, evaluates cos and sin of the
remaining angle (at most pi/4) in FP64, and rotates.  A device entry must lie
within half an FP32 ulp (of the reference's magnitude) plus 1e-15 of it, i.e.
be the FP32 rounding of the exact value up to FP64 noise -- and at most one
FP32 ulp from the reference in every case."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2602_23525_gb300 import gbfft  # noqa: E402


def host_root(m, N, half=False):
    """exp(-2 pi i m / N) (half: exp(-pi i m / N)) for integer arrays m >= 0; m = -1 gives 1."""
    m = np.asarray(m, dtype=np.int64)
    one = m < 0
    m = np.where(one, 0, m)
    num = (2 if half else 4) * m  # angle = (pi / 2) * num / N
    k = (2 * num + N) // (2 * N)  # nearest quadrant
    u = num - k * N               # |u| <= N / 2, exact
    phi = (np.pi / 2) * (u.astype(np.float64) / float(N))
    c, s = np.cos(phi), np.sin(phi)
    q = k % 4
    cos_t = np.select([q == 0, q == 1, q == 2, q == 3], [c, -s, -c, s])
    sin_t = np.select([q == 0, q == 1, q == 2, q == 3], [s, c, -s, -c])
    z = cos_t - 1j * sin_t
    return np.where(one, 1.0 + 0j, z)


def device_table(kind, N, a, b, count):
    out = torch.empty(count, dtype=torch.complex64, device="cuda")
    gbfft.fft_twiddle_table(kind, N, a, b, count, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def check(dev, ref):
    for d, r in ((dev.real, ref.real), (dev.imag, ref.imag)):
        ulp = np.spacing(np.abs(r).astype(np.float32)).astype(np.float64)
        err = np.abs(d.astype(np.float64) - r)
        assert np.all(err <= 0.5 * ulp + 1e-15), (err.max(), np.argmax(err - 0.5 * ulp))
        # at most one FP32 ulp (of the reference's magnitude, floored at 2^-30 so
        # that an exactly-zero reference tolerates FP64 noise)
        ulp1 = np.spacing(np.maximum(np.abs(r), 2.0 ** -30).astype(np.float32)).astype(np.float64)
        assert np.all(err <= ulp1)


@pytest.mark.parametrize("N,mult,count", [(4096, 1, 4096), (10007, 1, 10007), (1 << 24, 1, 1 << 24),
                                          (1 << 24, 4096, 4097), (12289, 11, 12289), (2 ** 31 - 1, 7, 65536)])
def test_root_tables(N, mult, count):
    dev = device_table(gbfft.FFT_TABLE_ROOTS, N, mult, 0, count)
    e = gbfft.fft_twiddle_exponents(gbfft.FFT_TABLE_ROOTS, N, mult, 0, count)
    assert e.tolist()[:64] == [(i * mult) % N for i in range(min(64, count))]
    check(dev, host_root(e, N))


@pytest.mark.parametrize("N,L,R", [(4096, 16, 16), (4096, 256, 16), (8192, 512, 16), (1 << 24, 1 << 20, 16)])
def test_stage_tables(N, L, R):
    dev = device_table(gbfft.FFT_TABLE_STAGE, N, L, R, 4 * L)
    check(dev, host_root(gbfft.fft_twiddle_exponents(gbfft.FFT_TABLE_STAGE, N, L, R, 4 * L), N))


@pytest.mark.parametrize("L,R", [(125, 8), (243, 9), (1024, 7), (128, 59)])
def test_mixed_radix_stage_tables(L, R):
    cnt = L * (R & ~1)
    dev = device_table(gbfft.FFT_TABLE_FULL_STAGE, L * R, L, R, cnt)
    check(dev, host_root(gbfft.fft_twiddle_exponents(gbfft.FFT_TABLE_FULL_STAGE, L * R, L, R, cnt), L * R))


@pytest.mark.parametrize("N,L,ncols", [(1 << 20, 64, 1024), (1 << 24, 256, 4096), (65536 * 7, 16, 448)])
def test_four_step_twiddle_tables(N, L, ncols):
    cnt = ncols * (L + 4)
    dev = device_table(gbfft.FFT_TABLE_POSTTW, N, L, ncols, cnt)
    check(dev, host_root(gbfft.fft_twiddle_exponents(gbfft.FFT_TABLE_POSTTW, N, L, ncols, cnt), N))


@pytest.mark.parametrize("n", [17, 1000, 10007, (1 << 20) + 7])
def test_chirp_tables(n):
    dev = device_table(gbfft.FFT_TABLE_CHIRP, n, 0, 0, n)
    e = gbfft.fft_twiddle_exponents(gbfft.FFT_TABLE_CHIRP, n, 0, 0, n)
    assert e.tolist()[-8:] == [(k * k) % (2 * n) for k in range(n - 8, n)]
    check(dev, host_root(e, n, half=True))
