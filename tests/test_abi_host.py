"""The C-ABI library on the host: it loads, exports every entry point declared in
include/gbfft.h, and its host logic (problem canonicalisation and validation,
plan construction in estimate mode) behaves as documented.  No GPU needed:
fft_plan_explain builds the plan text without touching a device.
"""
import ctypes
import os
import re
import subprocess

import pytest

import __graft_entry__
from paper_2602_23525_gb300 import gbfft

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbfft.h")


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(fft_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_core_entry_points():
    names = declared_functions()
    for n in ("fft_plan_dft", "fft_execute", "fft_destroy", "fft_last_error", "fft_error_string",
              "fft_plan_info", "fft_export_wisdom", "fft_import_wisdom"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(gbfft.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", gbfft.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (fft_\w+)", out))
    assert set(declared_functions()) <= exported


def test_binding_covers_header():
    assert set(declared_functions()) <= set(gbfft._SIGNATURES)


def test_error_strings():
    assert gbfft.fft_error_string(0) == "ok"
    for code in range(1, 12):
        assert gbfft.fft_error_string(code) not in ("ok", "unknown error")
    assert gbfft.fft_error_string(999) == "unknown error"


def explain(dims, howmany=(), sign=-1, flags=0):
    return gbfft.fft_plan_explain(dims, howmany, sign, flags)


def explain_err(dims, howmany=(), sign=-1, flags=0):
    with pytest.raises(gbfft.GbfftError) as e:
        explain(dims, howmany, sign, flags)
    return e.value.code


# ---------------------------------------------------------------- validation

def test_invalid_arguments():
    assert explain_err([(8, 1, 1)], sign=0) == gbfft.FFT_ERR_INVALID_ARG
    assert explain_err([(8, 1, 1)], sign=2) == gbfft.FFT_ERR_INVALID_ARG
    assert explain_err([(-1, 1, 1)]) == gbfft.FFT_ERR_INVALID_ARG
    assert explain_err([(8, 1, 1)], [(-3, 8, 8)]) == gbfft.FFT_ERR_INVALID_ARG
    assert explain_err([(8, 1, 1)], flags=1 << 20) == gbfft.FFT_ERR_INVALID_ARG
    assert explain_err([(2, 1, 1)] * 4) == gbfft.FFT_ERR_UNSUPPORTED


def test_output_overlap_rejected():
    # zero output stride with n > 1
    assert explain_err([(8, 1, 0)]) == gbfft.FFT_ERR_OUTPUT_OVERLAP
    # vector stride smaller than the transform's span
    assert explain_err([(8, 1, 1)], [(4, 8, 4)]) == gbfft.FFT_ERR_OUTPUT_OVERLAP
    # zero input stride is a broadcast and is allowed
    assert "pass" in explain([(8, 0, 1)])


def test_inplace_requires_equal_strides():
    assert explain_err([(8, 1, 2)], flags=gbfft.FFT_INPLACE) == gbfft.FFT_ERR_INPLACE_MISMATCH
    assert "in-place" in explain([(8, 1, 1)], [(4, 8, 8)], flags=gbfft.FFT_INPLACE)


def test_empty_problem_is_noop():
    assert "no-op" in explain([(0, 1, 1)])
    assert "no-op" in explain([(16, 1, 1)], [(0, 16, 16)])


def test_length_one_dims_dropped_and_runs_merged():
    t = explain([(64, 1, 1), (1, 5, 7)], [(4, 64 * 3, 64 * 3), (3, 64, 64), (1, 9, 9)])
    assert "n=[(64,1,1)]" in t
    assert "howmany=[(12,64,64)]" in t


def test_rank0_is_a_copy():
    t = explain([], [(10, 1, 1)])
    assert "copy" in t


# ---------------------------------------------------------------- plan structure

def test_plan_single_pass_pow2():
    t = explain([(4096, 1, 1)], [(64, 4096, 4096)])
    assert "pass stockham n=4096" in t and "R=16.16.16" in t and "cooley-tukey" not in t


def test_plan_mixed_radix():
    t = explain([(1000, 1, 1)], [(512, 1000, 1000)])
    assert "pass stockham n=1000" in t
    assert "R=8.5.5.5" in t
    assert "R=9.9.9.3" in explain([(2187, 512, 1)], [(512, 1, 2187)])


def test_plan_large_is_multi_pass():
    """Radix-sqrt(n) steps (sec. 3.3): 2^24 = 256 x 65536, the 256-point column
    pass with its twiddle, then the 65536 rows as 256 x 256 in the L2-resident
    four-step, its B items over two rows of 8 transforms (their outputs
    interleave 256 apart); with wisdom for the rows' sub-problem, three one-CTA
    TMA passes as before."""
    t = explain([(2 ** 24, 1, 1)])
    assert "cooley-tukey n=16777216 = 256 x 65536" in t
    assert t.count("pass p2-tma") == 1 and "post-twiddle" in t
    assert "pass l2-fourstep n=65536 = 256 x 256" in t and "B items over 2 rows of 8 transforms" in t, t
    assert "output element stride 256" in t, t
    for e, n1 in ((22, 64), (23, 128)):
        t = explain([(2 ** e, 1, 1)], [(2 ** (26 - e), 2 ** e, 2 ** e)])
        assert f"= {n1} x 65536" in t and "B items over 2 rows of 8 transforms" in t, t
    gbfft.fft_forget_wisdom()
    gbfft.fft_import_wisdom("gbfft-wisdom 1\nr1 n=65536 is=1 os=256 v=[(256,65536,1)] ip=0\tsplit:256\n")
    try:
        t = explain([(2 ** 24, 1, 1)])
    finally:
        gbfft.fft_forget_wisdom()
    assert "cooley-tukey n=65536 = 256 x 256" in t
    assert t.count("pass p2-tma") == 3, t
    assert t.count("post-twiddle") >= 2
    t = explain([(2 ** 20, 1, 1)], [(4, 2 ** 20, 2 ** 20)])
    assert "= 1024 x 1024" in t and t.count("pass p2-tma") == 2


def test_plan_prime_is_bluestein():
    t = explain([(10007, 1, 1)], [(512, 10007, 10007)])
    assert "bluestein n=10007" in t
    t = explain([(97, 1, 1)])
    assert "bluestein n=97" in t and "bluestein-fused" in t


def test_plan_prime_rader():
    """Rader (sec. 4.2.5) where p - 1 is smooth and p is beyond the one-CTA
    Bluestein pass; a wisdom entry can force it, padded or not, for any prime."""
    for p in (1153, 7681, 12289, 65537):
        t = explain([(p, 1, 1)], [(8, p, p)])
        assert f"rader p={p}" in t and f"L={p - 1}" in t, t
        assert t.count("pointwise") == 3
    t = explain([(10007, 1, 1)], [(8, 10007, 10007)])  # 10006 = 2 x 5003: Bluestein
    assert "bluestein" in t and "rader" not in t
    gbfft.fft_forget_wisdom()
    try:
        gbfft.fft_import_wisdom("gbfft-wisdom 1\nr1 n=10007 is=1 os=1 v=[(8,10007,10007)] ip=0\trader:32768\n")
        t = explain([(10007, 1, 1)], [(8, 10007, 10007)])
        assert "rader p=10007 g=5 L=32768 (zero-padded" in t
        # a convolution length Rader cannot use is a wisdom error at plan time
        gbfft.fft_import_wisdom("gbfft-wisdom 1\nr1 n=10007 is=1 os=1 v=[(8,10007,10007)] ip=0\trader:16384\n")
        with pytest.raises(gbfft.GbfftError) as e:
            explain([(10007, 1, 1)], [(8, 10007, 10007)])
        assert e.value.code == gbfft.FFT_ERR_WISDOM
    finally:
        gbfft.fft_forget_wisdom()


def test_plan_multidim_separable():
    """Rank 2 is one rank-1 problem per dimension (sec. 4.2): the rows in one
    pass, the 4096-long columns as a four-step whose scratch keeps the columns
    innermost (both passes tile 64 adjacent columns)."""
    t = explain([(4096, 4096, 4096), (4096, 1, 1)])
    assert "separable rank-2" in t
    assert t.count("pass stockham n=4096") == 1
    assert "cooley-tukey n=4096 = 64 x 64" in t and "columns innermost" in t
    assert t.count("load=rows store=cols T=64") == 2, t


def test_size30_radix_decomposition():
    """Fig. 3 of the paper decomposes a size-30 DFT with radices 3, 2 and 5; the
    planner's codelet stages cover the same factors."""
    t = explain([(30, 1, 1)])
    m = re.search(r"R=([0-9.]+)", t)
    assert m and sorted(int(r) for r in m.group(1).split(".")) == [2, 3, 5]


def test_explain_is_deterministic():
    a = explain([(7168, 1, 1)], [(512, 7168, 7168)])
    b = explain([(7168, 1, 1)], [(512, 7168, 7168)])
    assert a == b


def test_wisdom_text_roundtrip_and_rejection():
    gbfft.fft_forget_wisdom()
    good = "gbfft-wisdom 1\nr1 n=64 is=1 os=1 v=[] ip=0\tsingle:R=16.4:T=4:f=0:l=1:s=1:lc=0:sc=0\n"
    gbfft.fft_import_wisdom(good)
    assert "single:R=16.4" in gbfft.fft_export_wisdom()
    for bad in ("nonsense", "gbfft-wisdom 1\nr1 x\tsingle:R=6\n", "gbfft-wisdom 1\nfoo\tbar\n"):
        with pytest.raises(gbfft.GbfftError) as e:
            gbfft.fft_import_wisdom(bad)
        assert e.value.code == gbfft.FFT_ERR_WISDOM
    gbfft.fft_forget_wisdom()
    assert gbfft.fft_export_wisdom().strip() == "gbfft-wisdom 1"


def test_wisdom_decides_estimate_plan():
    gbfft.fft_forget_wisdom()
    key = "r1 n=64 is=1 os=1 v=[] ip=0"
    gbfft.fft_import_wisdom(f"gbfft-wisdom 1\n{key}\tsingle:R=4.4.4:T=1:f=0:l=1:s=1:lc=0:sc=0\n")
    assert "R=4.4.4" in explain([(64, 1, 1)])
    gbfft.fft_forget_wisdom()
    assert "R=16.4" in explain([(64, 1, 1)])


def test_cluster_plans_and_wisdom():
    """Estimate mode takes the one-pass cluster kernel for contiguous 2^14
    batches and two TMA passes for 2^15..2^17 (the faster of the two when
    measured); wisdom selects any instantiated (n1, n2, C, buffers) and rejects
    configurations that are not built."""
    txt = explain([(16384, 1, 1)], [(8, 16384, 16384)])
    assert "pass cluster n=16384 = " in txt, txt
    for e in (15, 16, 17):
        n = 2 ** e
        txt = explain([(n, 1, 1)], [(8, n, n)])
        assert "pass cluster" not in txt and f"cooley-tukey n={n}" in txt, txt
    # strided transforms or two vector loops keep the four-step plan
    assert "pass cluster" not in explain([(65536, 8, 8)], [(8, 1, 1)])
    gbfft.fft_forget_wisdom()
    key = "r1 n=65536 is=1 os=1 v=[(8,65536,65536)] ip=0"
    gbfft.fft_import_wisdom(f"gbfft-wisdom 1\n{key}\tcluster:8.8.16.1\n")
    assert "C=16 buffers=1" in explain([(65536, 1, 1)], [(8, 65536, 65536)])
    for bad in ("cluster:9.9.9.1", "cluster:8.8.16", "cluster:7.9.8.1", "cluster:8.8.16.3"):
        with pytest.raises(gbfft.GbfftError) as ei:
            gbfft.fft_import_wisdom(f"gbfft-wisdom 1\n{key}\t{bad}\n")
        assert ei.value.code == gbfft.FFT_ERR_WISDOM
    gbfft.fft_forget_wisdom()


def test_plan_l2_resident_four_step():
    """Estimate mode takes the four-step in one persistent kernel with its
    intermediate in an L2 ring (eq. (2), one HBM round trip) for contiguous
    2^14..2^21 batches that fill the GPU several times over, split n1 = 2^floor(e/2);
    small batches, 2^22 and strided layouts keep the cluster or TMA passes."""
    for e in range(14, 22):
        n = 2 ** e
        txt = explain([(n, 1, 1)], [(2 ** 26 // n, n, n)])
        assert f"pass l2-fourstep n={n} = {2 ** (e // 2)} x {n >> (e // 2)}" in txt, txt
        assert txt.count("pass ") == 1, txt
    # 2^22 takes a 64-point column pass and its 65536-point rows in groups, not one 2048 x 2048 kernel
    assert "pass l2-fourstep n=4194304" not in explain([(2 ** 22, 1, 1)], [(16, 2 ** 22, 2 ** 22)])
    assert "l2-fourstep" not in explain([(65536, 1, 1)], [(8, 65536, 65536)])
    assert "l2-fourstep" not in explain([(65536, 1024, 1024)], [(1024, 1, 1)])


def test_plan_layout_specific_four_steps():
    """The four-step (eq. (2)) picks its scratch layout from the problem's
    strides: columns innermost for transforms down the columns of a row-major
    array, [l2][b][k1] for a batch-fastest input into transform-contiguous
    output (from 2^14 on in estimate mode; shorter ones transpose first), and
    the plain [vector][k1][l2] for contiguous batches."""
    t = explain([(65536, 512, 1)], [(512, 1, 65536)])
    assert "batch-fastest input, scratch [l2][b][k1]" in t and "transpose first" not in t, t
    assert t.count("pass p2-tma") == 2 and "load=rows store=contig" in t and "^(v1*k)" in t, t
    t = explain([(4096, 512, 1)], [(512, 1, 4096)])
    assert "transpose first" in t, t
    t = explain([(8192, 64, 64), (64, 1, 1)])
    assert "columns innermost" in t and t.count("load=rows store=cols T=64") == 1, t
    t = explain([(65536, 1, 1)], [(8, 65536, 65536)])
    assert "cooley-tukey n=65536" in t and "columns innermost" not in t and "[l2][b][k1]" not in t, t
    # a column count that no 64-column tile divides keeps the column-tile pass
    t = explain([(4096, 40, 40), (40, 1, 1)])
    assert "columns innermost" not in t, t


def test_plan_bluestein_store_epilogues():
    """Bluestein with a power-of-two convolution length (sec. 4.2.5 prime sizes):
    the multiply and the output step ride on the stores of the FFT passes;
    a smooth non-power-of-two length keeps the separate pointwise steps."""
    gbfft.fft_forget_wisdom()
    try:
        gbfft.fft_import_wisdom("gbfft-wisdom 1\nr1 n=10007 is=1 os=1 v=[(8,10007,10007)] ip=0\tblue:32768\n")
        t = explain([(10007, 1, 1)], [(8, 10007, 10007)])
        assert "multiply fused" in t and "epilogue Z = conj(y Bhat) for k < 32768" in t, t
        assert "epilogue y = w conj(D) for k < 10007" in t and "pointwise Z" not in t, t
        t = explain([(10007, 1, 1)], [(8, 10007, 10007)], sign=1)
        assert "epilogue y = conj(w conj(D))" in t, t
        gbfft.fft_forget_wisdom()
        # estimate mode: the fused power of two where the smooth length would
        # need several passes; the smooth length where it fits one CTA or where
        # the output layout rules out the fused stores (stride 2 along k)
        t = explain([(10007, 1, 1)], [(8, 10007, 10007)])
        assert "bluestein n=10007 m=32768" in t and "multiply fused" in t, t
        t = explain([(4099, 1, 1)], [(8, 4099, 4099)])
        assert "bluestein n=4099 m=8232" in t and "bluestein-fused" in t, t
        t = explain([(10007, 1, 2)], [(8, 10007, 20014)])
        assert "bluestein n=10007 m=20160" in t and "pointwise Z = conj(A Bhat)" in t, t
    finally:
        gbfft.fft_forget_wisdom()


def test_real_data_plan_validation():
    """Real-data planners (sec. 5, 7) validate before touching a device."""
    def code(fn, dims, how=(), flags=0):
        with pytest.raises(gbfft.GbfftError) as e:
            fn(dims, how, flags)
        return e.value.code
    r2c, c2r = gbfft.fft_plan_dft_r2c, gbfft.fft_plan_dft_c2r
    assert code(r2c, []) == gbfft.FFT_ERR_INVALID_ARG                        # rank 0
    assert code(r2c, [(8, 1, 1)], (), gbfft.FFT_INPLACE) == gbfft.FFT_ERR_UNSUPPORTED
    assert code(c2r, [(8, 1, 1)], (), gbfft.FFT_PREC_TC_BF16) == gbfft.FFT_ERR_UNSUPPORTED
    assert code(r2c, [(-1, 1, 1)]) == gbfft.FFT_ERR_INVALID_ARG
    # r2c of n = 8 has 5 outputs per transform: a batch stride of 4 overlaps
    assert code(r2c, [(8, 1, 1)], [(3, 8, 4)]) == gbfft.FFT_ERR_OUTPUT_OVERLAP
    # c2r writes 8 reals per transform: stride 8 is fine, 7 overlaps
    assert code(c2r, [(8, 1, 1)], [(3, 5, 7)]) == gbfft.FFT_ERR_OUTPUT_OVERLAP


def test_in_place_plans_without_scratch():
    """In place (sec. 4.2): n = s^2 as columns, rows and an in-place square
    transpose; rank-0 in-place square transposes; non-square refused."""
    IP = gbfft.FFT_INPLACE
    t = explain([(1 << 20, 1, 1)], [(4, 1 << 20, 1 << 20)], -1, IP)
    assert "1024 x 1024 in place without scratch" in t
    assert "load=rows store=cols" in t and "transpose in place 1024 x 1024" in t
    t = explain([(4096, 4096, 4096), (4096, 1, 1)], [], -1, IP)
    assert "cooley-tukey" not in t and t.count("pass p2-tma") == 2
    t = explain([], [(64, 64, 1), (64, 1, 64), (3, 4096, 4096)], -1, IP)
    assert "transpose in place 64 x 64" in t
    assert explain_err([], [(64, 32, 1), (32, 1, 64)], -1, IP) == gbfft.FFT_ERR_UNSUPPORTED
    # a transform in place still needs equal strides
    assert explain_err([(64, 1, 2)], [], -1, IP) == gbfft.FFT_ERR_INPLACE_MISMATCH


def test_indirect_plan_from_wisdom():
    gbfft.fft_forget_wisdom()
    try:
        gbfft.fft_import_wisdom("gbfft-wisdom 1\nr1 n=4096 is=64 os=1 v=[(64,1,4096)] ip=0\tindirect\n")
        t = explain([(4096, 64, 1)], [(64, 1, 4096)])
        assert "indirect: copy into the output's layout" in t and "copy (rank-0)" in t
    finally:
        gbfft.fft_forget_wisdom()
