"""Bit-exact pins of the integer exponent arithmetic behind every twiddle and
chirp table (sec. 6: twiddles are accurate only when the exponent of w_N^m is
reduced exactly before the angle is formed; sec. 4.2.5: Bluestein's chirp
exponent k^2 mod 2n and Rader's permutation g^i mod p).

The library evaluates, on the host, the same inline integer code its device
generators run (fft_twiddle_exponents); each table is compared entry by entry
with Python's arbitrary-precision integers, on full tables or on every entry
of long prefixes, at lengths up to 2^31 where a 32-bit product or a missing
reduction would overflow."""
import numpy as np
import pytest

from paper_2602_23525_gb300 import gbfft



@pytest.fixture(scope="module", autouse=True)
def library():
    try:
        gbfft.load()
    except RuntimeError as e:  # the library is built by __graft_entry__.build()
        pytest.skip(str(e))


def exps(kind, N, a, b, count):
    return gbfft.fft_twiddle_exponents(kind, N, a, b, count).tolist()


PRIMES_AND_POWERS = [2 ** 12, 2 ** 24, 2 ** 31, 3 ** 7, 5 ** 5, 7168, 10007, 12289, 65537, 1000003,
                     2 ** 31 - 1]


@pytest.mark.parametrize("N", PRIMES_AND_POWERS)
def test_root_exponents(N):
    S = int(np.ceil(np.sqrt(N)))
    while S * S < N:
        S += 1
    count = min(N, 1 << 16)
    for mult in (1, S, N - 1, N + 3, 2 ** 31 + 5):
        got = exps(gbfft.FFT_TABLE_ROOTS, N, mult, 0, count)
        assert got == [(i * mult) % N for i in range(count)], (N, mult)


def test_root_exponents_full_tables():
    for N in (4096, 10007, 1 << 20):
        assert exps(gbfft.FFT_TABLE_ROOTS, N, 1, 0, N) == list(range(N))
        S = int(np.ceil(np.sqrt(N)))
        while S * S < N:
            S += 1
        hi = exps(gbfft.FFT_TABLE_ROOTS, N, S, 0, N // S + 1)
        assert hi == [(i * S) % N for i in range(N // S + 1)]


@pytest.mark.parametrize("N,L,R", [(4096, 1, 16), (4096, 16, 16), (4096, 256, 16), (2 ** 13, 2, 16),
                                   (2 ** 13, 512, 16), (2 ** 24, 2 ** 20, 16), (64, 4, 16), (8, 1, 8)])
def test_power_of_two_stage_exponents(N, L, R):
    got = exps(gbfft.FFT_TABLE_STAGE, N, L, R, 4 * L)
    step = N // (L * R)
    want = []
    for k in range(L):
        for t in range(4):
            p = 1 << t
            want.append(-1 if p >= R else (p * k * step) % N)
    assert got == want


@pytest.mark.parametrize("L,R", [(125, 8), (1, 5), (243, 9), (64, 11), (7, 13), (25, 5), (1, 61), (128, 59),
                                 (3125, 2), (1024, 7)])
def test_mixed_radix_stage_exponents(L, R):
    W = R & ~1
    got = exps(gbfft.FFT_TABLE_FULL_STAGE, L * R, L, R, L * W)
    want = [((r * k) % (L * R)) if r < R else -1 for k in range(L) for r in range(1, W + 1)]
    assert got == want


@pytest.mark.parametrize("N,L,ncols", [(2 ** 16, 16, 256), (2 ** 20, 64, 1024), (2 ** 24, 256, 256),
                                       (1000 * 64, 25, 64), (2 ** 31, 4096, 8)])
def test_four_step_twiddle_exponents(N, L, ncols):
    """w_N^{l2 k1} of eq. (2): table A = (c j) mod N, table B = (c L 2^t) mod N."""
    got = exps(gbfft.FFT_TABLE_POSTTW, N, L, ncols, ncols * (L + 4))
    want = [(c * j) % N for c in range(ncols) for j in range(L)]
    want += [(c * L * (1 << t)) % N for c in range(ncols) for t in range(4)]
    assert got == want
    # every k1 = j + q L: A[c][j] * B-powers reach exponent (c k1) mod N
    for c in (0, 1, ncols - 1):
        for k1 in (0, 1, L - 1, L, 15 * L + L - 1):
            j, q = k1 % L, k1 // L
            e = want[c * L + j] + sum(want[ncols * L + 4 * c + t] for t in range(4) if (q >> t) & 1)
            assert e % N == (c * k1) % N


@pytest.mark.parametrize("n", [2, 3, 17, 61, 1000, 10007, 65537, 1 << 20, 2 ** 31 - 1])
def test_chirp_exponents(n):
    count = min(n, 1 << 16)
    got = exps(gbfft.FFT_TABLE_CHIRP, n, 0, 0, count)
    assert got == [(k * k) % (2 * n) for k in range(count)]


def test_chirp_exponents_full_and_symmetric():
    for n in (10007, 1 << 18):
        e = exps(gbfft.FFT_TABLE_CHIRP, n, 0, 0, n)
        assert e == [(k * k) % (2 * n) for k in range(n)]
        # (n - k)^2 = k^2 + n (n - 2k): the chirp identity the convolution uses
        for k in (1, 2, n // 3, n - 1):
            assert (e[n - k] - e[k] - n * (n - 2 * k)) % (2 * n) == 0


def order(g, p):
    # multiplicative order of g mod p, brute force over divisors of p - 1
    m, f, q = p - 1, [], 2
    while q * q <= m:
        while m % q == 0:
            f.append(q)
            m //= q
        q += 1
    if m > 1:
        f.append(m)
    o = p - 1
    for q in set(f):
        while o % q == 0 and pow(g, o // q, p) == 1:
            o //= q
    return o


@pytest.mark.parametrize("p,g", [(17, 3), (257, 3), (7681, 17), (10007, 5), (12289, 11), (65537, 3)])
def test_rader_permutation_exponents(p, g):
    assert order(g, p) == p - 1  # g generates the multiplicative group
    got = exps(gbfft.FFT_TABLE_RADER, p, g, 0, p - 1)
    assert got == [pow(g, i, p) for i in range(p - 1)]
    assert sorted(got) == list(range(1, p))  # a permutation of 1..p-1


def test_rader_large_prime_prefix():
    p, g = 2 ** 31 - 1, 7
    got = exps(gbfft.FFT_TABLE_RADER, p, g, 0, 4096)
    assert got == [pow(g, i, p) for i in range(4096)]


def test_inconsistent_table_arguments_are_refused():
    bad = [(gbfft.FFT_TABLE_STAGE, 4096, 300, 16, 4),      # L R does not divide N
           (gbfft.FFT_TABLE_FULL_STAGE, 100, 10, 11, 4),   # N != L R
           (gbfft.FFT_TABLE_POSTTW, 4096, 16, 4, 1000),    # count beyond the table
           (gbfft.FFT_TABLE_CHIRP, 0, 0, 0, 1),
           (gbfft.FFT_TABLE_RADER, 17, 17, 0, 4),          # generator not below p
           (99, 16, 1, 0, 1)]
    for kind, N, a, b, count in bad:
        with pytest.raises(gbfft.GbfftError) as e:
            gbfft.fft_twiddle_exponents(kind, N, a, b, count)
        assert e.value.code == gbfft.FFT_ERR_INVALID_ARG
