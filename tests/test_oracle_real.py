"""Pins of the oracle's real-data transforms (DFTs of real data, sec. 5 and
sec. 7) against what mathematics and an independent library fix: numpy's
pocketfft rfftn / irfftn, the conjugate symmetry of a real input's spectrum,
closed forms (real delta, constant, single cosine), the round trip
c2r(r2c(x)) = N x, and the drop-out of the imaginary parts a real output
cannot carry.  Strided and batched layouts use the I/O-tensor strides of
sec. 4.1 (real elements on the real side, complex on the complex side)."""
import numpy as np
import pytest

import oracle

rng = np.random.default_rng(20260)


@pytest.mark.parametrize("shape", [(16,), (17,), (2,), (1,), (64,), (6, 10), (5, 7), (4, 6, 8), (3, 5, 9)])
def test_r2c_matches_numpy_rfftn(shape):
    x = rng.standard_normal(int(np.prod(shape)))
    dims = oracle._dense(list(shape))
    half = shape[-1] // 2 + 1
    hshape = list(shape[:-1]) + [half]
    odims = [(n, s_in, s_out) for (n, s_in, _), (_, s_out, _) in zip(dims, oracle._dense(hshape))]
    y = oracle.rdft_r2c(x, odims)
    want = np.fft.rfftn(x.reshape(shape))
    assert np.allclose(y.reshape(hshape), want, rtol=0, atol=1e-11 * np.abs(want).max())


@pytest.mark.parametrize("shape", [(16,), (17,), (2,), (64,), (6, 10), (5, 7), (4, 6, 8)])
def test_c2r_matches_numpy_irfftn(shape):
    half = shape[-1] // 2 + 1
    hshape = list(shape[:-1]) + [half]
    X = rng.standard_normal(int(np.prod(hshape))) + 1j * rng.standard_normal(int(np.prod(hshape)))
    idims = [(n, s_in, s_out) for (n, s_in, _), (_, s_out, _) in zip(
        [(n, s, s) for n, s, _ in oracle._dense(hshape)], oracle._dense(list(shape)))]
    idims[-1] = (shape[-1], idims[-1][1], idims[-1][2])
    y = oracle.rdft_c2r(X, idims)
    want = np.fft.irfftn(X.reshape(hshape), s=shape, axes=tuple(range(len(shape)))) * np.prod(shape)
    assert np.allclose(y.reshape(shape), want, rtol=0, atol=1e-11 * np.abs(want).max())


def test_batched_strided_layouts():
    n, b = 12, 5
    # input: transform stride 2 (every other real), batch stride 30; output: batch-fastest
    x = rng.standard_normal(30 * b + 5)
    y = oracle.rdft_r2c(x, [(n, 2, b)], [(b, 30, 1)], in_offset=3)
    got = y[: (n // 2 + 1) * b].reshape(n // 2 + 1, b).T
    want = np.fft.rfft(np.stack([x[3 + 30 * v: 3 + 30 * v + 2 * n: 2] for v in range(b)]))
    assert np.allclose(got, want, atol=1e-12)
    # c2r back through a different layout recovers n x
    z = oracle.rdft_c2r(y, [(n, b, 3)], [(b, 1, 3 * n)], out_len=3 * n * b)
    assert np.allclose(z.reshape(b, n, 3)[:, :, 0], n * np.stack(
        [x[3 + 30 * v: 3 + 30 * v + 2 * n: 2] for v in range(b)]), atol=1e-11)


def test_conjugate_symmetry_and_complex_oracle():
    n = 40
    x = rng.standard_normal(n)
    full = oracle.dft(x.astype(np.complex128), [(n, 1, 1)], [], -1)
    half = oracle.rdft_r2c(x, [(n, 1, 1)])
    assert np.array_equal(half, full[: n // 2 + 1])
    k = np.arange(1, n)
    assert np.allclose(full[n - k], np.conj(full[k]), atol=1e-12)


def test_closed_forms():
    n = 32
    for l0 in (0, 1, 7):
        x = np.zeros(n)
        x[l0] = 1.0
        y = oracle.rdft_r2c(x, [(n, 1, 1)])
        k = np.arange(n // 2 + 1)
        assert np.allclose(y, np.exp(-2j * np.pi * l0 * k / n), atol=1e-14)
    y = oracle.rdft_r2c(np.full(n, 2.0), [(n, 1, 1)])
    assert abs(y[0] - 2 * n) < 1e-12 and np.abs(y[1:]).max() < 1e-12
    k0 = 5
    y = oracle.rdft_r2c(np.cos(2 * np.pi * k0 * np.arange(n) / n), [(n, 1, 1)])
    want = np.zeros(n // 2 + 1, dtype=complex)
    want[k0] = n / 2
    assert np.allclose(y, want, atol=1e-12)
    # c2r of one bin 0 < k0 < n/2: 2 cos(2 pi k0 l / n)
    X = np.zeros(n // 2 + 1, dtype=complex)
    X[k0] = 1.0
    z = oracle.rdft_c2r(X, [(n, 1, 1)])
    assert np.allclose(z, 2 * np.cos(2 * np.pi * k0 * np.arange(n) / n), atol=1e-13)


@pytest.mark.parametrize("shape", [(10,), (11,), (4, 6), (3, 4, 7)])
def test_round_trip(shape):
    x = rng.standard_normal(int(np.prod(shape)))
    dims = oracle._dense(list(shape))
    half = shape[-1] // 2 + 1
    hd = oracle._dense(list(shape[:-1]) + [half])
    fwd = [(n, s, t) for (n, s, _), (_, t, _) in zip(dims, hd)]
    bwd = [(n, t, s) for (n, s, _), (_, t, _) in zip(dims, hd)]
    y = oracle.rdft_r2c(x, fwd)
    z = oracle.rdft_c2r(y, bwd)
    assert np.allclose(z, np.prod(shape) * x, atol=1e-11)


def test_c2r_ignores_imaginary_parts_of_self_conjugate_bins():
    n = 16
    X = rng.standard_normal(n // 2 + 1) + 1j * rng.standard_normal(n // 2 + 1)
    Y = X.copy()
    Y[0] = Y[0].real
    Y[-1] = Y[-1].real
    assert np.allclose(oracle.rdft_c2r(X, [(n, 1, 1)]), oracle.rdft_c2r(Y, [(n, 1, 1)]), atol=1e-13)
    # odd n: only the k = 0 bin is self-conjugate
    n = 15
    X = rng.standard_normal(n // 2 + 1) + 1j * rng.standard_normal(n // 2 + 1)
    Y = X.copy()
    Y[0] = Y[0].real
    a, b = oracle.rdft_c2r(X, [(n, 1, 1)]), oracle.rdft_c2r(Y, [(n, 1, 1)])
    assert np.allclose(a, b, atol=1e-13)
    X2 = X.copy()
    X2[-1] += 1j  # k = 7 is not self-conjugate for n = 15: it must matter
    assert not np.allclose(oracle.rdft_c2r(X2, [(n, 1, 1)]), a)
