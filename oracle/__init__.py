"""FP64 CPU oracle for the DFT problem dft(N, V, I, O).

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
never imports, links or executes anything here, and this package imports
nothing from the product library: the two share no code.

What it computes (Johnson & Frigo, *Implementing FFTs in Practice*):

* ``dft``: the problem dft(N, V, I, O) of sec. 4.1 -- a loop over the vector
  I/O tensor V of rank-|N| DFTs, each I/O dimension a triple (n, is, os) with
  strides in complex elements; a multi-dimensional DFT is the separable
  product over its dimensions, all with the same sign.
* each 1-D transform is eq. (1), Y[k] = sum_l X[l] w_n^{l k},
  w_n = exp(sign * 2 pi i / n) (sign -1 is the paper's forward transform;
  sign +1 is the unnormalised backward transform), evaluated either directly
  (``algo="direct"``, the Theta(n^2) generic plan of sec. 4.2) or by the
  recursive mixed-radix decimation-in-time Cooley-Tukey of eq. (2) and
  Algorithm 1 (``algo="ct"``); ``"auto"`` takes direct for n <= 4096.

* ``rdft_r2c`` / ``rdft_c2r``: DFTs of real data (sec. 5 and 7): the forward
  transform of a real input restricted to the non-redundant half of its
  conjugate-symmetric spectrum (last index <= n/2), and the unnormalised
  backward transform of such a half spectrum to real data.  Both are ``dft``
  applied to the data widened or extended in a dense array, plus index work.

Every transform is computed in IEEE FP64 in plain C (``oracle.c``), threaded
over the vector loops with pthreads.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ALGOS = {"auto": 0, "direct": 1, "ct": 2}


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` with gcc into ``liboracle.so`` (no GPU code)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-shared", "-fPIC",
                           _SRC, "-o", tmp, "-lpthread", "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def open_library(path: str):
    """Load a compiled oracle library and declare its entry point."""
    lib = ctypes.CDLL(path)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_dft.argtypes = [ctypes.c_int, i64p, i64p, i64p, ctypes.c_int, i64p, i64p,
                               i64p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                               ctypes.c_int, ctypes.c_int]
    lib.oracle_dft.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = open_library(build())
    return _lib


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _arr(vals):
    a = (ctypes.c_int64 * max(1, len(vals)))()
    for i, v in enumerate(vals):
        a[i] = int(v)
    return a


def dft(x, dims, howmany=(), sign=-1, *, out=None, out_len=None, in_offset=0, out_offset=0,
        algo="auto", threads=None, lib=None):
    """Evaluate dft(N, V, I, O) (sec. 4.1) in FP64.

    x          : 1-D complex array (any complex dtype; widened exactly to FP64)
    dims       : N, a sequence of (n, is, os) triples (rank 0 = copy)
    howmany    : V, a sequence of (n, is, os) triples (the vector loops)
    sign       : -1 forward (eq. (1)), +1 backward (unnormalised)
    out        : optional complex128 1-D output buffer, written in place
    out_len    : length of a freshly allocated zero output buffer
    in_offset  : element index of I inside ``x`` (strides may be negative)
    out_offset : element index of O inside ``out``
    lib        : an alternative library from ``open_library`` (default: oracle.c)
    Returns the complex128 output buffer.
    """
    lib = lib if lib is not None else _load()
    if sign not in (-1, 1):
        raise ValueError("sign must be -1 or +1")
    xin = np.ascontiguousarray(np.asarray(x).reshape(-1), dtype=np.complex128)
    if out is None:
        if out_len is None:
            out_len = xin.size
        out = np.zeros(int(out_len), dtype=np.complex128)
    if out.dtype != np.complex128 or not out.flags.c_contiguous:
        raise ValueError("out must be a contiguous complex128 array")
    dims = [tuple(int(v) for v in d) for d in dims]
    howmany = [tuple(int(v) for v in d) for d in howmany]
    _check_bounds(xin.size, in_offset, [(n, s) for n, s, _ in dims] + [(n, s) for n, s, _ in howmany])
    _check_bounds(out.size, out_offset, [(n, s) for n, _, s in dims] + [(n, s) for n, _, s in howmany])
    nthr = threads if threads is not None else default_threads()
    rc = lib.oracle_dft(len(dims), _arr([d[0] for d in dims]), _arr([d[1] for d in dims]),
                        _arr([d[2] for d in dims]), len(howmany), _arr([d[0] for d in howmany]),
                        _arr([d[1] for d in howmany]), _arr([d[2] for d in howmany]),
                        ctypes.c_void_p(xin.ctypes.data + 16 * int(in_offset)),
                        ctypes.c_void_p(out.ctypes.data + 16 * int(out_offset)),
                        int(sign), ALGOS[algo], int(nthr))
    if rc != 0:
        raise RuntimeError("oracle_dft failed")
    return out


def _check_bounds(size, offset, dims):
    """Every addressed element must lie inside the buffer (the C code trusts us)."""
    if any(n == 0 for n, _ in dims):
        return
    lo = hi = int(offset)
    for n, s in dims:
        ext = (n - 1) * s
        if ext < 0:
            lo += ext
        else:
            hi += ext
    if lo < 0 or hi >= size:
        raise ValueError(f"problem addresses [{lo}, {hi}] outside a buffer of {size} elements")


def dft_rows(x, sign=-1, algo="auto", threads=None):
    """Batched 1-D DFTs along the last axis of a C-contiguous array:
    dft({(n,1,1)}, {(batch, n, n)}, X, Y) -- the row example of sec. 4.1.1."""
    x = np.asarray(x)
    n = x.shape[-1]
    b = x.size // n if n else 0
    y = dft(x.reshape(-1), [(n, 1, 1)], [(b, n, n)], sign, algo=algo, threads=threads)
    return y.reshape(x.shape)


def dft_nd(x, sign=-1, algo="auto", threads=None):
    """Rank-d DFT over all axes of a C-contiguous array (separable, sec. 4.1)."""
    x = np.asarray(x)
    dims = []
    stride = 1
    for n in reversed(x.shape):
        dims.append((n, stride, stride))
        stride *= n
    dims.reverse()
    y = dft(x.reshape(-1), dims, [], sign, algo=algo, threads=threads)
    return y.reshape(x.shape)


# --------------------------------------------------------------------------- real data

def _loop_offsets(loops, k):
    """Offsets (flattened, row-major over `loops`) of stride component k (1 in, 2 out)."""
    off = np.zeros(1, dtype=np.int64)
    for d in loops:
        off = (off[:, None] + np.arange(d[0], dtype=np.int64)[None, :] * int(d[k])).reshape(-1)
    return off


def _dense(shape_loops):
    """(n, s, s) triples of a dense row-major layout of the given lengths."""
    out, st = [], 1
    for n in reversed(shape_loops):
        out.append((n, st, st))
        st *= n
    return list(reversed(out))


def rdft_r2c(x, dims, howmany=(), *, out_len=None, in_offset=0, out_offset=0, algo="auto", threads=None):
    """DFT of real data (sec. 5 and sec. 7: real-input transforms), forward.

    x       : real array; dims (n, is, os) and howmany as in ``dft``, with the
              input strides counted in real elements and the output strides in
              complex elements
    returns : the complex128 output buffer holding Y[k] = sum_l x[l] prod_j
              w_{n_j}^{l_j k_j} (w = exp(-2 pi i / n)) for every k whose last
              index is at most n_last / 2 (integer division): the non-redundant
              half of the conjugate-symmetric spectrum of a real input
    The spectrum is the complex DFT of eq. (1) over all dimensions, computed by
    ``dft`` on the input widened to complex; nothing else is computed here.
    """
    dims = [tuple(int(v) for v in d) for d in dims]
    howmany = [tuple(int(v) for v in d) for d in howmany]
    if not dims:
        raise ValueError("a real-data transform has rank >= 1")
    xr = np.asarray(x, dtype=np.float64).reshape(-1)
    loops = howmany + dims
    shape = [d[0] for d in loops]
    half = dims[-1][0] // 2 + 1
    hshape = shape[:-1] + [half]
    hloops = loops[:-1] + [(half, dims[-1][1], dims[-1][2])]
    if out_len is None:
        _, hi = _span([(d[0], d[2]) for d in hloops])
        out_len = out_offset + hi + 1
    out = np.zeros(int(out_len), dtype=np.complex128)
    if any(n == 0 for n in shape):
        return out
    dense = xr[in_offset + _loop_offsets(loops, 1)].astype(np.complex128)
    ld = _dense(shape)
    full = dft(dense, ld[len(howmany):], ld[:len(howmany)], -1, algo=algo, threads=threads)
    full = full.reshape(shape)[..., :half].reshape(-1)
    out[out_offset + _loop_offsets(hloops, 2)] = full
    return out


def rdft_c2r(X, dims, howmany=(), *, out_len=None, in_offset=0, out_offset=0, algo="auto", threads=None):
    """Real-output DFT (sec. 5 and sec. 7), backward and unnormalised: the inverse
    of ``rdft_r2c`` up to the factor prod(n).

    X       : complex array holding the half spectrum, k_last <= n_last / 2 (the
              last dimension has n_last // 2 + 1 entries); dims (n, is, os) with
              the input strides in complex elements and the output strides in
              real elements
    returns : the float64 output buffer holding
              y[l] = Re( sum_{k, k_last <= n_last/2} c(k_last) X[k] prod_j w_{n_j}^{-l_j k_j} ),
              c = 1 for k_last = 0 and, for even n_last, k_last = n_last / 2,
              else 2 -- for a conjugate-symmetric spectrum this is the sum over
              all k of its full extension; the imaginary parts the extension
              cannot carry (those of the k_last = 0 and n_last / 2 planes) drop out
    Evaluated as the real part of ``dft`` (sign +1) of the weighted half
    spectrum placed in a full-length array, zero beyond n_last / 2.
    """
    dims = [tuple(int(v) for v in d) for d in dims]
    howmany = [tuple(int(v) for v in d) for d in howmany]
    if not dims:
        raise ValueError("a real-data transform has rank >= 1")
    Xc = np.asarray(X, dtype=np.complex128).reshape(-1)
    loops = howmany + dims
    shape = [d[0] for d in loops]
    nl = dims[-1][0]
    half = nl // 2 + 1
    hloops = loops[:-1] + [(half, dims[-1][1], dims[-1][2])]
    if out_len is None:
        _, hi = _span([(d[0], d[2]) for d in loops])
        out_len = out_offset + hi + 1
    out = np.zeros(int(out_len), dtype=np.float64)
    if any(n == 0 for n in shape):
        return out
    hx = Xc[in_offset + _loop_offsets(hloops, 1)].reshape(shape[:-1] + [half])
    c = np.full(half, 2.0)
    c[0] = 1.0
    if nl % 2 == 0:
        c[-1] = 1.0
    full = np.zeros(shape, dtype=np.complex128)
    full[..., :half] = hx * c
    ld = _dense(shape)
    y = dft(full.reshape(-1), ld[len(howmany):], ld[:len(howmany)], 1, algo=algo, threads=threads)
    out[out_offset + _loop_offsets(loops, 2)] = y.real
    return out


def _span(pairs):
    lo = hi = 0
    for n, s in pairs:
        e = (n - 1) * s
        if e < 0:
            lo += e
        else:
            hi += e
    return lo, hi
