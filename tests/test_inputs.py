"""The seeded input generators against the workload recipes they implement
(CPU): value ranges and moments, determinism, layouts, and the serving
request mix (rank, size, batch and sign proportions; Poisson arrivals)."""
import numpy as np

import fft_inputs


def test_seed_formula():
    assert fft_inputs.seed_for(0) == 20260
    assert fft_inputs.seed_for(3, 2) == 20260 + 3 + 2000


def test_uniform_values_and_determinism():
    x = fft_inputs.uniform_c64(200000, 7)
    assert x.dtype == np.complex64
    for part in (x.real, x.imag):
        assert part.min() >= -1.0 and part.max() < 1.0
        assert abs(part.mean()) < 0.01
        assert abs(part.var() - 1.0 / 3.0) < 0.01  # variance of U[-1, 1)
    assert abs(np.corrcoef(x.real, x.imag)[0, 1]) < 0.01
    assert np.array_equal(x, fft_inputs.uniform_c64(200000, 7))
    assert not np.array_equal(x[:100], fft_inputs.uniform_c64(100, 8))


def test_gaussian_moments_and_determinism():
    x = fft_inputs.gaussian_c64(200000, 9)
    for part in (x.real, x.imag):
        assert abs(part.mean()) < 0.01
        assert abs(part.std() - 1.0) < 0.01
    assert np.array_equal(x, fft_inputs.gaussian_c64(200000, 9))


def test_layouts():
    assert fft_inputs.batched_1d(8, 3) == ([(8, 1, 1)], [(3, 8, 8)])
    # batch-fastest: element l of transform b at l * batch + b in, b * n + l out
    assert fft_inputs.transposed_1d(8, 3) == ([(8, 3, 1)], [(3, 1, 8)])
    assert fft_inputs.POW2_SWEEP[0] == 16 and fft_inputs.POW2_SWEEP[-1] == 2 ** 24
    assert set(fft_inputs.UNEVEN_TRANSPOSED) <= set(fft_inputs.UNEVEN_SIZES)


def test_split_pow2():
    for e in range(6, 21):
        for r in (1, 2, 3):
            f = fft_inputs._split_pow2(e, r)
            assert len(f) == r and int(np.prod(f)) == 2 ** e
            exps = [int(np.log2(v)) for v in f]
            assert max(exps) - min(exps) <= 1


def test_serving_request_mix():
    reqs = fft_inputs.serving_requests(20000, 5)
    assert reqs == fft_inputs.serving_requests(20000, 5)
    ranks = np.array([len(s) for s, _, _ in reqs])
    for r, p in ((1, 0.7), (2, 0.2), (3, 0.1)):
        assert abs((ranks == r).mean() - p) < 0.015
    pts = np.array([int(np.prod(s)) for s, _, _ in reqs])
    pow2 = (pts & (pts - 1)) == 0
    assert abs(pow2.mean() - 0.8) < 0.015
    e = np.log2(pts[pow2]).astype(int)
    assert e.min() == 6 and e.max() == 20
    # every exponent about equally likely
    counts = np.bincount(e, minlength=21)[6:]
    assert counts.min() > 0.8 * counts.mean()
    for s, _, _ in reqs:
        n = int(np.prod(s))
        if n & (n - 1):
            r = len(s)
            lo, hi = int(np.ceil(100 ** (1.0 / r))), int(np.floor((10 ** 5) ** (1.0 / r)))
            assert all(lo <= d <= hi and d & (d - 1) for d in s), s
    batches = np.array([b for _, b, _ in reqs])
    assert batches.min() == 1 and batches.max() == 256
    assert abs(batches.mean() - 128.5) < 2.0
    signs = np.array([g for _, _, g in reqs])
    assert set(signs.tolist()) == {-1, 1} and abs((signs == 1).mean() - 0.5) < 0.015


def test_poisson_arrivals():
    t = fft_inputs.poisson_arrivals(50000, 400.0, 3)
    assert np.all(np.diff(t) > 0) and t[0] > 0
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 400.0) < 0.02 / 400.0
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.02  # exponential: std = mean
