"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Every case compares each transform's output with the oracle (relative L2
<= 2e-6, the FP32 tolerance of the workload definition); copies and
repeated runs must be bit-exact.  Sizes are chosen so the oracle finishes in
seconds while spanning several CTA tiles and ragged tails.
"""
import numpy as np
import pytest

import fft_inputs
from parity import TOL, check, reference, run_gpu, per_transform_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2602_23525_gb300 import gbfft  # noqa: E402

EST = gbfft.FFT_ESTIMATE


def u(count, seed):
    return fft_inputs.uniform_c64(count, seed)


# ---------------------------------------------------------------- the small workload

@pytest.mark.parametrize("flags", [EST, gbfft.FFT_MEASURE])
def test_config1_n4096_batch64_forward(flags):
    n, b = 4096, 64
    x = u(n * b, fft_inputs.seed_for(0))
    err, info = check([(n, 1, 1)], [(b, n, n)], -1, x, flags=flags)
    print(f"config-1 max rel-L2 {err:.3e}\n{info}")


# ---------------------------------------------------------------- sizes

@pytest.mark.parametrize("e", range(0, 21))
@pytest.mark.parametrize("sign", [-1, 1])
def test_pow2_sizes(e, sign):
    n = 2 ** e
    b = max(1, min(2 ** 18 // n, 64)) + (3 if n <= 4096 else 0)  # ragged batch for small n
    x = u(n * b, fft_inputs.seed_for(1, e))
    check([(n, 1, 1)], [(b, n, n)], sign, x, flags=EST, algo="ct" if n > 4096 else "auto")


@pytest.mark.parametrize("n", [3, 5, 6, 7, 9, 10, 11, 12, 13, 14, 15, 18, 20, 21, 25, 27, 30, 35, 36, 45, 49,
                               60, 63, 77, 81, 99, 100, 121, 125, 143, 169, 243, 343, 360, 625, 1000,
                               1001, 2187, 3125, 3600, 3840, 7168, 10000, 15625])
def test_mixed_radix_sizes(n):
    b = max(1, 2 ** 15 // n) + 1
    x = fft_inputs.gaussian_c64(n * b, n)
    check([(n, 1, 1)], [(b, n, n)], -1, x, flags=EST)


@pytest.mark.parametrize("n", [17, 19, 23, 29, 31, 37, 61, 67, 97, 127, 257, 1009, 4099, 8191, 10007,
                               2 * 17, 34 * 9, 4 * 1009])
def test_bluestein_sizes(n):
    b = max(1, 2 ** 14 // n) + 1
    x = fft_inputs.gaussian_c64(n * b, n + 7)
    check([(n, 1, 1)], [(b, n, n)], -1, x, flags=EST, algo="ct" if n > 4096 else "auto")
    check([(n, 1, 1)], [(b, n, n)], +1, x, flags=EST, algo="ct" if n > 4096 else "auto")


@pytest.mark.parametrize("n", [2 ** 21, 2 ** 22, 3 * 2 ** 18, 65536 * 5])
def test_large_multipass(n):
    x = u(n, 77)
    check([(n, 1, 1)], [], -1, x, flags=EST, algo="ct")


@pytest.mark.parametrize("exps", [range(4, 10), range(10, 15), range(15, 19), range(19, 22), range(22, 25)])
def test_sweep_full_size_measured_sampled(exps):
    """The benchmark step's transforms at their full sizes (2^26 points: n = 2^e,
    batch 2^26 / n) with the plans the measuring planner picks, as the bench
    runs them; sampled transforms (first, middle, last) against the oracle."""
    total = 2 ** 26
    x = torch.from_numpy(u(total, fft_inputs.seed_for(1, 98))).cuda()
    y = torch.empty_like(x)
    for e in exps:
        n, sign = 2 ** e, (-1 if e % 2 == 0 else 1)
        b = total // n
        p = gbfft.Plan([(n, 1, 1)], [(b, n, n)], sign, gbfft.FFT_MEASURE)
        p.execute(x, y)
        torch.cuda.synchronize()
        for v in sorted({0, b // 2, b - 1}):
            xi = x[v * n:(v + 1) * n].cpu().numpy()
            yi = y[v * n:(v + 1) * n].cpu().numpy()
            ref = reference([(n, 1, 1)], [], sign, xi, algo="ct" if n > 4096 else "auto")
            err = np.linalg.norm(yi.astype(np.complex128) - ref) / np.linalg.norm(ref)
            assert err <= TOL, (n, v, err, p.info)
        p.destroy()


def test_single_2_24_measured():
    """The single 2^24-point transform with the measured plan (as the bench)."""
    n = 2 ** 24
    x = u(n, fft_inputs.seed_for(1, 97))
    check([(n, 1, 1)], [], 1, x, flags=gbfft.FFT_MEASURE, algo="ct")


def test_single_2_24():
    n = 2 ** 24
    x = u(n, fft_inputs.seed_for(1, 99))
    check([(n, 1, 1)], [], -1, x, flags=EST, algo="ct")


# ---------------------------------------------------------------- layouts (sec. 4.1)

def test_transposed_layout_columns():
    """dft({(n, b, 1)}, {(b, 1, n)}): columns of an n x b matrix in, rows out."""
    for n, b in [(2187, 40), (7168, 24), (64, 100), (1000, 33)]:
        x = fft_inputs.gaussian_c64(n * b, n)
        check([(n, b, 1)], [(b, 1, n)], -1, x, flags=EST)


def test_columns_in_place_example():
    """Sec. 4.1.1 columns example, in place: dft({(n1,n2,n2)},{(n2,1,1)},X,X)."""
    n1, n2 = 256, 96
    x = u(n1 * n2, 5)
    y, info = run_gpu([(n1, n2, n2)], [(n2, 1, 1)], -1, x, flags=EST, inplace=True)
    ref = reference([(n1, n2, n2)], [(n2, 1, 1)], -1, x)
    err = per_transform_error(y, ref, [(n1, n2, n2)], [(n2, 1, 1)])
    assert err.max() <= TOL, info


def test_rows_in_place_example():
    n1, n2 = 50, 1024
    x = u(n1 * n2, 6)
    y, info = run_gpu([(n2, 1, 1)], [(n1, n2, n2)], +1, x, flags=EST, inplace=True)
    ref = reference([(n2, 1, 1)], [(n1, n2, n2)], +1, x)
    assert per_transform_error(y, ref, [(n2, 1, 1)], [(n1, n2, n2)]).max() <= TOL, info


def test_negative_and_padded_strides():
    n, b = 512, 9
    x = u(2 * n * b + 8, 8)
    # reversed input transform order and reversed elements, padded output
    check([(n, -1, 2)], [(b, -n, 2 * n + 1)], -1, x, flags=EST, in_offset=n * b - 1)


def test_vector_rank_two_unmergeable():
    n = 128
    x = u(n * 6 * 5 * 2, 9)
    check([(n, 1, 1)], [(6, 2 * n * 5, n * 5), (5, 2 * n, n)], -1, x, flags=EST)


def test_broadcast_zero_input_stride():
    x = u(4, 10)
    check([(256, 0, 1)], [(4, 1, 256)], -1, x, flags=EST)


def test_rank0_copy_bit_exact():
    x = u(1000, 11)
    y, _ = run_gpu([], [(40, 25, 1), (25, 1, 40)], -1, x, flags=EST)
    assert np.array_equal(y.reshape(25, 40), x.reshape(40, 25).T)


def test_length_zero_is_noop():
    x = u(16, 12)
    y, _ = run_gpu([(0, 1, 1)], [], -1, x, out_len=16, fill=3.0, flags=EST)
    assert np.all(y == 3.0)


# ---------------------------------------------------------------- multi-dimensional

@pytest.mark.parametrize("shape", [(12, 20), (3, 5, 7), (64, 128, 32), (256, 48), (30, 30, 30)])
def test_multidim_small(shape):
    dims = []
    st = 1
    for nn in reversed(shape):
        dims.append((nn, st, st))
        st *= nn
    dims.reverse()
    x = u(int(np.prod(shape)), 13)
    check(dims, [], -1, x, flags=EST)
    check(dims, [(2, st, st)], +1, np.concatenate([x, x[::-1]]), flags=EST)


def test_rank2_4096x4096():
    n = 4096
    x = u(n * n, fft_inputs.seed_for(1, 50))
    check([(n, n, n), (n, 1, 1)], [], -1, x, flags=EST, algo="ct")


def _force(key, choice):
    gbfft.fft_forget_wisdom()
    gbfft.fft_import_wisdom(f"gbfft-wisdom 1\n{key}\t{choice}\n")


@pytest.mark.parametrize("sign", [-1, 1])
def test_fourstep_columns_innermost(sign):
    """Four-step (eq. (2)) of transforms that run down columns: the scratch keeps
    the unit-stride loop innermost, both passes tile along it and the pass-1
    twiddle takes its column from a vector loop.  A rank-2 column dimension
    (in place on the output), a rank-1 batch with two loops (out of place), and
    the same with an input that is 8- but not 16-byte aligned (the generic pass
    with the twiddle column from vector dim 1)."""
    try:
        x = u(4096 * 64, 91)
        _force("r1 n=4096 is=64 os=64 v=[(64,1,1)] ip=1", "split:64")
        err, info = check([(4096, 64, 64), (64, 1, 1)], [], sign, x, flags=EST, algo="ct")
        assert "columns innermost" in info and "^(v1*k)" in info, info
        x = u(4096 * 128 * 3 + 1, 92)
        _force("r1 n=4096 is=128 os=128 v=[(3,524288,524288),(128,1,1)] ip=0", "split:64")
        err, info = check([(4096, 128, 128)], [(128, 1, 1), (3, 524288, 524288)], sign, x, flags=EST, algo="ct")
        assert "columns innermost" in info and "load=rows store=cols T=64" in info, info
        err, info = check([(4096, 128, 128)], [(128, 1, 1), (3, 524288, 524288)], sign, x, flags=EST, algo="ct",
                          in_offset=1)
        assert "columns innermost" in info, info
    finally:
        gbfft.fft_forget_wisdom()


@pytest.mark.parametrize("sign", [-1, 1])
def test_bluestein_fused_fourstep(sign):
    """Bluestein (sec. 4.2, prime sizes) with m a power of two beyond one CTA:
    the multiply and the output step ride on the stores of the last passes of
    the two convolution FFTs.  n = 10007 (m = 2^15, contiguous), and n = 8193
    (m = 2^16) with two padded vector loops, out of place with an output
    offset (8-byte aligned stores) and an input offset."""
    try:
        b = 8
        x = u(10007 * b, 93)
        _force(f"r1 n=10007 is=1 os=1 v=[({b},10007,10007)] ip=0", "blue:32768")
        err, info = check([(10007, 1, 1)], [(b, 10007, 10007)], sign, x, flags=EST, algo="ct")
        assert "multiply fused" in info and "epilogue" in info and "pointwise Z" not in info, info
        how = [(3, 8193, 8193), (2, 3 * 8193 + 5, 2 * 3 * 8193 + 7)]
        x = u(2 * (3 * 8193 + 5) + 8, 94)
        _force("r1 n=8193 is=1 os=1 v=[(2,24584,49165),(3,8193,8193)] ip=0", "blue:65536")
        err, info = check([(8193, 1, 1)], how, sign, x, flags=EST, algo="ct", out_offset=1)
        assert "y = " in info and "epilogue" in info, info
        err, info = check([(8193, 1, 1)], how, sign, x, flags=EST, algo="ct", in_offset=3)
    finally:
        gbfft.fft_forget_wisdom()


@pytest.mark.parametrize("sign", [-1, 1])
def test_fourstep_batch_fastest_input(sign):
    """Four-step (eq. (2)) of a batch-fastest input with transform-contiguous
    output: the scratch [l2][b][k1]; pass 1 loads rows of adjacent transforms
    and stores whole transforms with the twiddle column taken from a vector
    loop, pass 2 loads rows of adjacent k1.  One loop and two loops (padded
    strides), and an input that is 8- but not 16-byte aligned (the generic
    passes)."""
    try:
        x = u(4096 * 64, 101)
        _force("r1 n=4096 is=64 os=1 v=[(64,1,4096)] ip=0", "split:64")
        err, info = check([(4096, 64, 1)], [(64, 1, 4096)], sign, x, flags=EST, algo="ct")
        assert "scratch [l2][b][k1]" in info and "load=rows store=contig" in info, info
        how = [(64, 1, 4096), (3, 4096 * 64 + 8, 4096 * 64 + 16)]
        x = u(3 * (4096 * 64 + 8) + 4, 102)
        _force("r1 n=4096 is=64 os=1 v=[(3,262152,262160),(64,1,4096)] ip=0", "split:64")
        err, info = check([(4096, 64, 1)], how, sign, x, flags=EST, algo="ct")
        assert "scratch [l2][b][k1]" in info and "^(v2*k)" in info, info
        err, info = check([(4096, 64, 1)], how, sign, x, flags=EST, algo="ct", in_offset=1)
        assert "scratch [l2][b][k1]" in info, info
    finally:
        gbfft.fft_forget_wisdom()


def test_rank2_4096x4096_measured():
    """The measuring planner over the rank-2 workload (its column dimension
    chooses between one column-tile pass and a four-step)."""
    n = 4096
    x = u(n * n, fft_inputs.seed_for(1, 51))
    err, info = check([(n, n, n), (n, 1, 1)], [], 1, x, flags=gbfft.FFT_MEASURE, algo="ct")
    print(info)


def test_rank3_256_cubed():
    n = 256
    x = u(n ** 3, fft_inputs.seed_for(3, 1))
    check([(n, n * n, n * n), (n, n, n), (n, 1, 1)], [], -1, x, flags=EST, algo="ct")


# ---------------------------------------------------------------- determinism, planner

def test_repeatable_bit_exact():
    n, b = 2048, 33
    x = u(n * b, 14)
    y1, _ = run_gpu([(n, 1, 1)], [(b, n, n)], -1, x, flags=EST)
    y2, _ = run_gpu([(n, 1, 1)], [(b, n, n)], -1, x, flags=EST, repeat=3)
    assert np.array_equal(y1, y2)


def test_measure_and_wisdom_replay_bit_identical():
    gbfft.fft_forget_wisdom()
    dims, how = [(8192, 1, 1)], [(16, 8192, 8192)]
    x = u(8192 * 16, 15)
    y1, info1 = run_gpu(dims, how, -1, x, flags=gbfft.FFT_MEASURE)
    wis = gbfft.fft_export_wisdom()
    assert "r1 n=8192" in wis
    gbfft.fft_forget_wisdom()
    gbfft.fft_import_wisdom(wis)
    y2, info2 = run_gpu(dims, how, -1, x, flags=gbfft.FFT_WISDOM_ONLY)
    assert info1.replace(" estimate", "") == info2.replace(" estimate", "")
    assert np.array_equal(y1, y2)
    ref = reference(dims, how, -1, x, algo="ct")
    assert per_transform_error(y2, ref, dims, how).max() <= TOL
    gbfft.fft_forget_wisdom()


def test_wisdom_only_without_entry_fails():
    gbfft.fft_forget_wisdom()
    with pytest.raises(gbfft.GbfftError) as e:
        gbfft.Plan([(4096, 1, 1)], [], -1, gbfft.FFT_WISDOM_ONLY)
    assert e.value.code == gbfft.FFT_ERR_WISDOM


def test_alias_rejected_at_execute():
    n = 1024
    x = torch.zeros(2 * n, dtype=torch.complex64, device="cuda")
    plan = gbfft.Plan([(n, 1, 1)], [], -1, EST)
    with pytest.raises(gbfft.GbfftError) as e:
        gbfft.fft_execute(plan.handle, x.data_ptr(), x.data_ptr() + 8 * (n // 2), 0)
    assert e.value.code == gbfft.FFT_ERR_ALIAS
    plan.destroy()


# ---------------------------------------------------------------- power-of-two TMA kernel

@pytest.mark.parametrize("e", range(8, 14))
def test_pow2_kernel_padded_batch_stride(e):
    """Batch stride n + 2 (tiles are not one contiguous block: one bulk copy per
    transform) and a ragged last tile."""
    n = 2 ** e
    b = 37
    x = u((n + 2) * b, 30 + e)
    err, info = check([(n, 1, 1)], [(b, n + 2, n)], -1, x, flags=EST)
    assert "p2-tma" in info


def test_pow2_kernel_unaligned_input_falls_back():
    """An input pointer that is 8- but not 16-byte aligned cannot feed a bulk copy;
    the plan's generic pass runs instead, with the same result."""
    n, b = 1024, 9
    x = u(n * b + 1, 31)
    err, info = check([(n, 1, 1)], [(b, n, n)], +1, x, flags=EST, in_offset=1)
    assert "p2-tma" in info


def test_pow2_kernel_matches_generic_pass_bit_for_bit_tolerance():
    """The specialised kernel and the generic pass run the same stage schedule;
    both stay within the oracle tolerance for every size (forward, in place)."""
    for e in range(8, 14):
        n = 2 ** e
        b = 2 ** 20 // n
        x = u(n * b, 40 + e)
        y, info = run_gpu([(n, 1, 1)], [(b, n, n)], -1, x, flags=EST, inplace=True)
        assert "p2-tma" in info
        ref = reference([(n, 1, 1)], [(b, n, n)], -1, x, algo="ct")
        assert per_transform_error(y, ref, [(n, 1, 1)], [(b, n, n)]).max() <= TOL


def test_p2_strided_tile_shapes():
    """Column tiles (rows of adjacent columns in, rows or columns out) of the TMA
    pass kernels, with two extra vector loops and ragged column counts rejected
    back to the generic pass."""
    for n, cols, b in [(64, 192, 3), (128, 96, 2), (512, 32, 2), (1024, 16, 2), (4096, 4, 2)]:
        x = u(n * cols * b, 50 + n)
        # columns of a row-major n x cols matrix, b matrices
        err, info = check([(n, cols, cols)], [(cols, 1, 1), (b, n * cols, n * cols)], +1, x, flags=EST)
        assert "p2-tma" in info and "load=rows" in info
        err, info = check([(n, cols, 1)], [(cols, 1, n), (b, n * cols, n * cols)], -1, x, flags=EST)
        # long transforms of a batch-fastest input are transposed first
        assert ("transpose first" in info) if n >= 4096 else ("load=rows store=contig" in info), info
    x = u(1024 * 24, 60)
    err, info = check([(1024, 1, 24)], [(24, 1024, 1)], -1, x, flags=EST)
    assert "load=contig store=cols" in info
    x = u(1024 * 18, 61)  # 18 columns: not a whole number of 4-column tiles
    err, info = check([(1024, 1, 18)], [(18, 1024, 1)], -1, x, flags=EST)
    assert "p2-tma" not in info and "pass stockham" in info


def test_p2_rows_tensor_map_layouts():
    """Column tiles loaded through a tensor map: padded row pitch and two
    unmergeable vector loops in either stride order; and a layout whose vector
    stride is below the row stride (no tensor map: one bulk copy per row)."""
    n, cols, b1, b2 = 256, 32, 3, 2
    pitch = cols + 8
    s2 = n * pitch
    s1 = b2 * s2 + 64
    x = u(b1 * s1, 81)
    for how in ([(cols, 1, 1), (b1, s1, n * cols * b2), (b2, s2, n * cols)],
                [(cols, 1, 1), (b2, s2, n * cols), (b1, s1, n * cols * b2)]):
        err, info = check([(n, pitch, cols)], how, -1, x, flags=EST)
        assert "load=rows" in info
    B = 4
    x = u(n * B * (cols + 2), 82)
    err, info = check([(n, B * (cols + 2), cols)], [(cols, 1, 1), (B, cols + 2, n * cols)], 1, x, flags=EST)
    assert "load=rows" in info


@pytest.mark.parametrize("e", [4, 5, 6, 7])
@pytest.mark.parametrize("sign", [-1, 1])
def test_small_transform_kernel(e, sign):
    """n = 16..128: the tile is re-laid into odd-pitch rows; ragged last tile."""
    n = 2 ** e
    b = (4096 // n) * 5 + 3
    x = u(n * b, 70 + e)
    err, info = check([(n, 1, 1)], [(b, n, n)], sign, x, flags=EST)
    assert "p2-tma" in info


# ---------------------------------------------------------------- mixed-radix TMA kernel

@pytest.mark.parametrize("n", [12, 60, 100, 240, 1000, 2187, 3125, 4374, 7000])
@pytest.mark.parametrize("sign", [-1, 1])
def test_mr_kernel_contiguous(n, sign):
    """Mixed-radix lengths through the TMA pass kernel: several tiles and a
    ragged last tile; odd lengths (whole 16-byte copies need an even tile)."""
    b = max(3, 20000 // n) | 1
    for bb in (b, b + 1):  # odd batch: ragged tile (plain loads for odd n); even: copy engine
        x = u(n * bb, 700 + n + bb)
        err, info = check([(n, 1, 1)], [(bb, n, n)], sign, x, flags=EST)
        assert "pass mr-tma" in info, info


@pytest.mark.parametrize("n,sched", [(1000, "R=8.5.5.5"), (2187, "R=9.9.9.3"), (3125, "R=5.5.5.5.5"),
                                     (3600, "R=16.9.5.5"), (3840, "R=16.16.3.5"), (7168, "R=16.16.4.7")])
def test_mr_compile_time_schedules(n, sched):
    """The lengths with a compile-time radix schedule (stockham_mrc.cu): both
    signs, contiguous batches with a ragged tile, and strided columns through
    tensor-map boxes (load=rows) where two transforms fit one CTA (3600 and
    7168 need 400 and 448 threads each: the generic pass takes their columns)."""
    b = max(3, 12000 // n) | 1
    for sign in (-1, 1):
        x = u(n * b, 760 + n)
        err, info = check([(n, 1, 1)], [(b, n, n)], sign, x, flags=EST)
        assert "pass mr-tma" in info and sched in info, info
    cols = 16
    x = u(n * cols, 770 + n)
    err, info = check([(n, cols, 1)], [(cols, 1, n)], -1, x, flags=EST)
    if n not in (3600, 7168):
        assert "pass mr-tma" in info and "load=rows" in info, info


def test_mr_kernel_layouts():
    """Strided columns (tensor-map boxes, several boxes of 256 rows and a partial
    one), non-adjacent transforms (one copy each / plain loads for odd n), an
    8-byte aligned input (plain loads), and two vector loops."""
    for n, cols in [(2187, 64), (300, 48), (45, 32)]:
        x = u(n * cols * 2, 710 + n)
        err, info = check([(n, cols, 1)], [(cols, 1, n), (2, n * cols, n * cols)], -1, x, flags=EST)
        assert "pass mr-tma" in info and "load=rows" in info, info
    for n, pad in [(1000, 8), (1125, 5)]:
        b = 37
        x = u((n + pad) * b, 720 + n)
        err, info = check([(n, 1, 1)], [(b, n + pad, n)], 1, x, flags=EST)
        assert "pass mr-tma" in info, info
    n, b = 3000, 11
    x = u(n * b + 1, 730)
    err, info = check([(n, 1, 1)], [(b, n, n)], -1, x, flags=EST, in_offset=1)
    assert "pass mr-tma" in info
    n = 360
    x = u(5 * (6 * (n + 7) + 3), 731)
    err, info = check([(n, 1, 1)], [(6, n + 7, n), (5, 6 * (n + 7) + 3, 6 * n)], -1, x, flags=EST)
    assert "pass mr-tma" in info


def test_mr_kernel_fourstep_bluestein():
    """Bluestein for a prime (m = 20160 = 140 x 144: mixed-radix four-step
    passes with the post twiddle) and a mixed-radix four-step length."""
    try:
        for n, b in [(10007, 3), (20160, 4)]:
            x = u(n * b, 740 + n)
            # estimate mode takes the fused power of two for 10007: force the
            # smooth length through wisdom
            _force(f"r1 n={n} is=1 os=1 v=[({b},{n},{n})] ip=0", "blue:20160" if n == 10007 else "split:140")
            err, info = check([(n, 1, 1)], [(b, n, n)], -1, x, flags=EST, algo="ct")
            assert "pass mr-tma" in info and "post-twiddle" in info, info
    finally:
        gbfft.fft_forget_wisdom()


# ---------------------------------------------------------------- transpose first

def test_rank0_transposes_bit_exact():
    """Rank-0 copies that transpose go through the tiled transpose kernel:
    ragged tiles, a batch loop, padded strides; results are bit-exact."""
    for r, c in [(37, 41), (64, 64), (1000, 9), (9, 1000)]:
        x = u(r * c, 900 + r)
        y, _ = run_gpu([], [(r, c, 1), (c, 1, r)], -1, x, flags=EST)
        assert np.array_equal(y.reshape(c, r), x.reshape(r, c).T), (r, c)
    r, c, b = 33, 70, 3
    x = u(b * (r * c + 5), 910)
    y, _ = run_gpu([], [(r, c, 1), (c, 1, r), (b, r * c + 5, r * c)], 1, x, flags=EST)
    for k in range(b):
        src = x[k * (r * c + 5):k * (r * c + 5) + r * c].reshape(r, c)
        assert np.array_equal(y[k * r * c:(k + 1) * r * c].reshape(c, r), src.T)


@pytest.mark.parametrize("n,b", [(4096, 24), (7168, 40), (65536, 8), (12288, 16)])
def test_transpose_first_plans(n, b):
    """Transposed batches of long transforms: the input is copied into the
    output's layout first, then transformed with the same-layout kernels."""
    x = u(n * (b + 3), 920 + n)
    for is_ in (b, b + 3):  # dense and padded input rows
        err, info = check([(n, is_, 1)], [(b, 1, n)], -1, x, flags=EST, algo="ct")
        assert "transpose first" in info, info


# ---------------------------------------------------------------- generic prime stage

@pytest.mark.parametrize("n", [17, 19, 23, 61, 68, 177, 345, 3904, 4070, 4880])
@pytest.mark.parametrize("sign", [-1, 1])
def test_generic_prime_stage(n, sign):
    """One prime factor 17..61 (the generic O(p^2) DFT in conjugate-pair form,
    sec. 4.2.5) as the first stage of the mixed-radix kernel."""
    b = max(3, 30000 // n)
    x = u(n * b, 950 + n)
    err, info = check([(n, 1, 1)], [(b, n, n)], sign, x, flags=EST, algo="direct" if n <= 4096 else "ct")
    assert "pass mr-tma" in info and "R=" in info, info


def test_generic_prime_strided_and_group():
    """Strided columns with a generic prime radix; a group with such a plan
    (no generic one-CTA form) uses the graph of plan launches."""
    n, cols = 61 * 8, 32
    x = u(n * cols, 960)
    err, info = check([(n, cols, 1)], [(cols, 1, n)], 1, x, flags=EST)
    assert "pass mr-tma n=488 R=61.8 load=rows" in info, info
    p = gbfft.Plan([(59, 1, 1)], [(40, 59, 59)], -1, EST)
    q = gbfft.Plan([(4096, 1, 1)], [(4, 4096, 4096)], -1, EST)
    try:
        g = gbfft.fft_group_create([p.handle, q.handle])
        assert gbfft.fft_group_mode(g) == 2
        with pytest.raises(gbfft.GbfftError):
            gbfft.fft_group_create([p.handle, q.handle], gbfft.FFT_GROUP_PERSISTENT)
        xa = torch.from_numpy(u(59 * 40, 961)).cuda()
        xb = torch.from_numpy(u(4096 * 4, 962)).cuda()
        ya, yb = torch.zeros_like(xa), torch.zeros_like(xb)
        gbfft.fft_group_execute(g, [xa.data_ptr(), xb.data_ptr()], [ya.data_ptr(), yb.data_ptr()],
                                torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        gbfft.fft_group_destroy(g)
        ref = reference([(59, 1, 1)], [(40, 59, 59)], -1, xa.cpu().numpy())
        assert per_transform_error(ya.cpu().numpy(), ref, [(59, 1, 1)], [(40, 59, 59)]).max() <= TOL
    finally:
        p.destroy()
        q.destroy()
