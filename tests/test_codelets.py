"""The codelet generator (sec. 5): every emitted radix, unparsed to C in FP64 and
compiled with gcc, must equal the direct DFT of eq. (1); the committed CUDA
codelets must be what the generator emits now."""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2602_23525_gb300", "csrc")
sys.path.insert(0, CSRC)
import gen_codelets  # noqa: E402


@pytest.fixture(scope="module")
def host_lib(tmp_path_factory):
    d = tmp_path_factory.mktemp("codelets")
    src = gen_codelets.render_host_c()
    wrap = "\n".join(
        f"void call{R}(const double* re, const double* im, double* o, double* p) "
        f"{{ host_dft{R}(re, im, o, p); }}" for R in gen_codelets.RADICES)
    c = d / "codelets.c"
    c.write_text(src + "\n" + wrap + "\n")
    so = d / "codelets.so"
    subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", str(c), "-o", str(so)])
    return ctypes.CDLL(str(so))


def direct(x):
    n = len(x)
    k = np.arange(n)
    W = np.exp(-2j * np.pi * ((k[:, None] * k[None, :]) % n) / n)
    return W @ x


@pytest.mark.parametrize("R", gen_codelets.RADICES)
def test_codelet_equals_direct_dft(host_lib, R):
    rng = np.random.default_rng(R)
    f = getattr(host_lib, f"call{R}")
    for trial in range(4):
        x = rng.standard_normal(R) + 1j * rng.standard_normal(R)
        re, im = np.ascontiguousarray(x.real), np.ascontiguousarray(x.imag)
        o, p = np.zeros(R), np.zeros(R)
        f(*(a.ctypes.data_as(ctypes.c_void_p) for a in (re, im, o, p)))
        y = o + 1j * p
        assert np.max(np.abs(y - direct(x))) < 1e-13 * R


@pytest.mark.parametrize("R", gen_codelets.RADICES)
def test_codelet_columns_are_the_dft_matrix(host_lib, R):
    """Unit impulses give the columns w_R^{l k} of the DFT matrix exactly where
    the root is trivial (+-1, +-i)."""
    f = getattr(host_lib, f"call{R}")
    for l in range(R):
        re = np.zeros(R)
        re[l] = 1.0
        im = np.zeros(R)
        o, p = np.zeros(R), np.zeros(R)
        f(*(a.ctypes.data_as(ctypes.c_void_p) for a in (re, im, o, p)))
        k = np.arange(R)
        expect = np.exp(-2j * np.pi * ((l * k) % R) / R)
        assert np.max(np.abs(o + 1j * p - expect)) < 1e-14
        if l == 0:
            assert np.all(o == 1.0) and np.all(p == 0.0)


def test_trivial_twiddles_folded():
    """Radix 2 and 4 need no multiplications; radix 8 only the four by 1/sqrt(2)."""
    for R, muls in ((2, 0), (4, 0), (8, 4)):
        dag, y = gen_codelets.build(R)
        assert gen_codelets.count_ops(dag, y)[1] == muls


def test_committed_cuda_codelets_are_current():
    with open(os.path.join(CSRC, "codelets.cuh")) as fh:
        assert fh.read() == gen_codelets.render_cuda()
