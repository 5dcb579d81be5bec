"""Pins for the FP64 oracle against what the paper's definitions fix.

Nothing here re-types the oracle's formula: each check is a closed form of
eq. (1) for a special input, an invariant of the DFT (shift theorem,
linearity, Parseval, inversion), a brute-force sum on tiny inputs, agreement
of the oracle's two independent algorithms (direct eq. (1) vs the recursive
Cooley-Tukey of eq. (2) / Algorithm 1), a hand-written fixture of the 3- and
4-point DFT matrices, or an independent library routine (numpy.fft, pocketfft).
"""
import cmath
import math
import os

import numpy as np
import pytest

import fft_inputs
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

SIZES_SMALL = list(range(1, 65))
SIZES_MIXED = [96, 100, 128, 210, 243, 625, 1000, 1024, 2187, 3125, 4096]
SIZES_LARGE = [5000, 7168, 8192, 10007, 65536]


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    d = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (d if d > 0 else 1.0))


def one(n, x, sign=-1, algo="auto"):
    return oracle.dft(x, [(n, 1, 1)], [], sign, algo=algo, threads=1)


def load_matrix(name):
    rows = []
    h = math.sqrt(3.0) / 2.0
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            vals = []
            for tok in line.split():
                neg = tok.startswith("-")
                t = tok.lstrip("-")
                v = h if t == "h" else float(t)
                vals.append(-v if neg else v)
            rows.append([complex(vals[i], vals[i + 1]) for i in range(0, len(vals), 2)])
    return np.array(rows)


# ---------------------------------------------------------------- fixtures

@pytest.mark.parametrize("algo", ["direct", "ct"])
def test_dft4_matrix_fixture(algo):
    """Columns of the 4-point DFT matrix (eq. (1), w_4 = -i) from the fixture."""
    F = load_matrix("dft4_matrix.txt")
    for l in range(4):
        e = np.zeros(4, complex)
        e[l] = 1
        # FP64 roots of unity at quarter turns carry ~1e-16 residue
        assert np.allclose(one(4, e, -1, algo), F[:, l], rtol=0, atol=1e-15)
        # sign +1 is the backward transform: the conjugate matrix
        assert np.allclose(one(4, e, +1, algo), np.conj(F[:, l]), rtol=0, atol=1e-15)


@pytest.mark.parametrize("algo", ["direct", "ct"])
def test_dft3_matrix_fixture(algo):
    F = load_matrix("dft3_matrix.txt")
    for l in range(3):
        e = np.zeros(3, complex)
        e[l] = 1
        assert np.allclose(one(3, e, -1, algo), F[:, l], rtol=0, atol=1e-15)


@pytest.mark.parametrize("algo", ["direct", "ct"])
def test_n1_and_n2(algo):
    x = np.array([0.25 - 0.5j])
    assert np.array_equal(one(1, x, -1, algo), x)
    x = np.array([1.5 + 2j, -0.25 + 1j])
    assert np.allclose(one(2, x, -1, algo), np.array([x[0] + x[1], x[0] - x[1]]), rtol=0,
                       atol=1e-15)


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", SIZES_SMALL[::7] + SIZES_MIXED[::2] + SIZES_LARGE)
def test_delta_gives_exponential(n):
    """x = delta at l0  ->  Y[k] = w_n^{l0 k} (eq. (1) with one nonzero term)."""
    for l0 in sorted({0, min(1, n - 1), n // 3, n - 1}):
        x = np.zeros(n, complex)
        x[l0] = 1.0
        y = one(n, x)
        k = np.arange(n)
        expect = np.exp(-2j * np.pi * ((l0 * k) % n) / n)
        assert np.max(np.abs(y - expect)) < 1e-12 * max(1, math.log2(n))
        if l0 == 0:
            assert np.all(y == 1.0)


@pytest.mark.parametrize("n", [7, 12, 64, 1000, 4096, 10007, 65536])
def test_exponential_gives_scaled_delta(n):
    """x[l] = w_n^{-l k0}  ->  Y = n * delta[k - k0]."""
    for k0 in sorted({0, 1, n // 2, n - 1}):
        l = np.arange(n)
        x = np.exp(2j * np.pi * ((l * k0) % n) / n)
        y = one(n, x)
        expect = np.zeros(n, complex)
        expect[k0] = n
        assert np.max(np.abs(y - expect)) < 1e-10 * n ** 0.5


@pytest.mark.parametrize("n", [5, 16, 30, 243, 1024, 5000, 8192])
def test_shift_theorem(n):
    """x'[l] = x[(l - s) mod n]  ->  Y'[k] = Y[k] w_n^{s k}."""
    x = fft_inputs.uniform_c64(n, 11).astype(np.complex128)
    y = one(n, x)
    k = np.arange(n)
    for s in sorted({1, 3 % n, n // 2, n - 1}):
        ys = one(n, np.roll(x, s))
        expect = y * np.exp(-2j * np.pi * ((s * k) % n) / n)
        assert rel_l2(ys, expect) < 1e-13


@pytest.mark.parametrize("n", [9, 64, 360, 4096, 6000])
def test_linearity(n):
    """Ergun-style random linearity check: DFT(a x + b z) = a DFT(x) + b DFT(z)."""
    x = fft_inputs.uniform_c64(n, 1).astype(np.complex128)
    z = fft_inputs.gaussian_c64(n, 2).astype(np.complex128)
    a, b = 0.75 - 1.25j, -2.0 + 0.5j
    assert rel_l2(one(n, a * x + b * z), a * one(n, x) + b * one(n, z)) < 1e-13


@pytest.mark.parametrize("n", [1, 13, 100, 2048, 4096, 9000, 16384])
def test_parseval(n):
    x = fft_inputs.gaussian_c64(n, 5).astype(np.complex128)
    y = one(n, x)
    assert abs(np.vdot(y, y).real - n * np.vdot(x, x).real) <= 1e-12 * n * np.vdot(x, x).real


@pytest.mark.parametrize("n", [3, 64, 1000, 4096, 4100, 32768])
def test_forward_then_backward_is_n_times_x(n):
    x = fft_inputs.uniform_c64(n, 9).astype(np.complex128)
    assert rel_l2(one(n, one(n, x, -1), +1), n * x) < 1e-13


# ---------------------------------------------------------------- two algorithms

@pytest.mark.parametrize("sign", [-1, 1])
def test_direct_and_ct_agree_all_small_n(sign):
    for n in SIZES_SMALL:
        x = fft_inputs.uniform_c64(n, 100 + n).astype(np.complex128)
        assert rel_l2(one(n, x, sign, "ct"), one(n, x, sign, "direct")) < 1e-13, n


@pytest.mark.parametrize("n", SIZES_MIXED + [997, 4093])
def test_direct_and_ct_agree_sampled(n):
    x = fft_inputs.gaussian_c64(n, 200 + n).astype(np.complex128)
    assert rel_l2(one(n, x, -1, "ct"), one(n, x, -1, "direct")) < 1e-13


# ---------------------------------------------------------------- library cross-check

@pytest.mark.parametrize("n", [8, 15, 101, 1000, 4096, 7168, 10007, 65536, 2 ** 18])
def test_matches_numpy_fft(n):
    x = fft_inputs.uniform_c64(n, 3).astype(np.complex128)
    assert rel_l2(one(n, x, -1), np.fft.fft(x)) < 1e-13
    assert rel_l2(one(n, x, +1), n * np.fft.ifft(x)) < 1e-13


# ---------------------------------------------------------------- multi-dimensional

def brute_nd(x, sign):
    """Full multi-dimensional sum prod_j w_{n_j}^{l_j k_j}, pure Python loops."""
    shape = x.shape
    out = np.zeros(shape, complex)
    idx = list(np.ndindex(*shape))
    for k in idx:
        acc = 0j
        for l in idx:
            ph = sum(lj * kj / nj for lj, kj, nj in zip(l, k, shape))
            acc += x[l] * cmath.exp(sign * 2j * math.pi * ph)
        out[k] = acc
    return out


@pytest.mark.parametrize("shape", [(3, 7), (4, 6, 5), (2, 3, 2, 2)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_multidim_separable_vs_brute_force(shape, sign):
    x = fft_inputs.gaussian_c64(int(np.prod(shape)), 7).astype(np.complex128).reshape(shape)
    assert rel_l2(oracle.dft_nd(x, sign), brute_nd(x, sign)) < 1e-13


def test_multidim_matches_numpy_fftn():
    x = fft_inputs.uniform_c64(16 * 12 * 10, 8).astype(np.complex128).reshape(16, 12, 10)
    assert rel_l2(oracle.dft_nd(x, -1), np.fft.fftn(x)) < 1e-13


def test_multidim_dim_order_irrelevant():
    """The separable definition does not depend on the order of dims[]."""
    n1, n2 = 12, 20
    x = fft_inputs.uniform_c64(n1 * n2, 4)
    a = oracle.dft(x, [(n1, n2, n2), (n2, 1, 1)], [], -1)
    b = oracle.dft(x, [(n2, 1, 1), (n1, n2, n2)], [], -1)
    assert rel_l2(a, b) < 1e-14


# ---------------------------------------------------------------- I/O tensor semantics

def test_rows_and_columns_examples():
    """Sec. 4.1.1: rows dft({(n2,1,1)},{(n1,n2,n2)}) and columns dft({(n1,n2,n2)},{(n2,1,1)})."""
    n1, n2 = 6, 10
    x = fft_inputs.uniform_c64(n1 * n2, 21).astype(np.complex128)
    rows = oracle.dft(x, [(n2, 1, 1)], [(n1, n2, n2)], -1)
    cols = oracle.dft(x, [(n1, n2, n2)], [(n2, 1, 1)], -1)
    m = x.reshape(n1, n2)
    assert rel_l2(rows.reshape(n1, n2), np.fft.fft(m, axis=1)) < 1e-14
    assert rel_l2(cols.reshape(n1, n2), np.fft.fft(m, axis=0)) < 1e-14


def test_rank0_copy_and_transpose_exact():
    """Rank-0 problems are copies and permutations (sec. 4.1.1): bit-exact."""
    n1, n2 = 5, 7
    x = fft_inputs.uniform_c64(n1 * n2, 22).astype(np.complex128)
    assert np.array_equal(oracle.dft(x, [], [(n1 * n2, 1, 1)], -1), x)
    t = oracle.dft(x, [], [(n1, n2, 1), (n2, 1, n1)], -1)
    assert np.array_equal(t.reshape(n2, n1), x.reshape(n1, n2).T)


def test_negative_and_zero_input_strides():
    n = 24
    x = fft_inputs.uniform_c64(n, 23).astype(np.complex128)
    rev = oracle.dft(x, [(n, -1, 1)], [], -1, in_offset=n - 1, out_len=n)
    assert rel_l2(rev, np.fft.fft(x[::-1])) < 1e-14
    # zero input stride broadcasts one value: the DFT of a constant
    z = oracle.dft(x, [(n, 0, 1)], [], -1, out_len=n)
    expect = np.zeros(n, complex)
    expect[0] = n * x[0]
    assert np.max(np.abs(z - expect)) < 1e-12


def test_strided_output_and_vector_offsets():
    n, b = 16, 5
    x = fft_inputs.uniform_c64(n * b, 24).astype(np.complex128)
    # output transposed: element k of transform v at v + k*b
    y = oracle.dft(x, [(n, 1, b)], [(b, n, 1)], -1)
    assert rel_l2(y.reshape(n, b).T, np.fft.fft(x.reshape(b, n), axis=1)) < 1e-14


def test_empty_problem_is_noop():
    x = np.zeros(4, complex)
    out = np.full(4, 7 + 7j)
    oracle.dft(x, [(0, 1, 1)], [], -1, out=out)
    oracle.dft(x, [(4, 1, 1)], [(0, 4, 4)], -1, out=out)
    assert np.all(out == 7 + 7j)


def test_threads_do_not_change_results():
    n, b = 256, 33
    x = fft_inputs.gaussian_c64(n * b, 25)
    a = oracle.dft(x, [(n, 1, 1)], [(b, n, n)], -1, threads=1)
    c = oracle.dft(x, [(n, 1, 1)], [(b, n, n)], -1, threads=7)
    assert np.array_equal(a, c)
