"""Python binding of the C ABI in ``include/gbfft.h`` (ctypes, marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of the transform: all of it runs in the CUDA library
``libgbfft.so``.  If the library is missing, ``load()`` raises -- there is no
fallback of any kind.

``Plan`` is a convenience wrapper for torch tensors: it reads sizes and
strides (torch.complex64 strides are already in complex elements) and passes
``torch.cuda.current_stream().cuda_stream``.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbfft.so")

FFT_OK = 0
FFT_ERR_INVALID_ARG = 1
FFT_ERR_UNSUPPORTED = 2
FFT_ERR_ALIAS = 3
FFT_ERR_INPLACE_MISMATCH = 4
FFT_ERR_OOM = 5
FFT_ERR_BUDGET = 6
FFT_ERR_CUDA = 7
FFT_ERR_DEVICE_TIMEOUT = 8
FFT_ERR_WISDOM = 9
FFT_ERR_NO_DEVICE = 10
FFT_ERR_OUTPUT_OVERLAP = 11

FFT_MEASURE = 0
FFT_ESTIMATE = 1 << 0
FFT_WISDOM_ONLY = 1 << 1
FFT_INPLACE = 1 << 2
FFT_EXTERNAL_SCRATCH = 1 << 3
FFT_PREC_TC_FP16 = 1 << 4
FFT_PREC_TC_BF16 = 1 << 5
FFT_PREC_SPLIT = 1 << 6
FFT_DEBUG_STALL = 1 << 11
FFT_GROUP_DEBUG_STALL = 1 << 8
FFT_TABLE_ROOTS = 0
FFT_TABLE_STAGE = 1
FFT_TABLE_FULL_STAGE = 2
FFT_TABLE_POSTTW = 3
FFT_TABLE_CHIRP = 4
FFT_TABLE_RADER = 5
FFT_GROUP_PERSISTENT = 1 << 9
FFT_GROUP_GRAPH = 1 << 10


class fft_iodim(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("is_", ctypes.c_int64), ("os", ctypes.c_int64)]


class GbfftError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {fft_error_string(code)} (code {code})" if what else
                         f"{fft_error_string(code)} (code {code})")


_lock = threading.Lock()
_lib = None

_SIGNATURES = {
    "fft_plan_dft": (ctypes.c_void_p, [ctypes.c_int, ctypes.POINTER(fft_iodim), ctypes.c_int,
                                       ctypes.POINTER(fft_iodim), ctypes.c_int, ctypes.c_uint]),
    "fft_plan_dft_r2c": (ctypes.c_void_p, [ctypes.c_int, ctypes.POINTER(fft_iodim), ctypes.c_int,
                                           ctypes.POINTER(fft_iodim), ctypes.c_uint]),
    "fft_plan_dft_c2r": (ctypes.c_void_p, [ctypes.c_int, ctypes.POINTER(fft_iodim), ctypes.c_int,
                                           ctypes.POINTER(fft_iodim), ctypes.c_uint]),
    "fft_execute": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "fft_destroy": (None, [ctypes.c_void_p]),
    "fft_sync_status": (ctypes.c_int, [ctypes.c_void_p]),
    "fft_execute_scratch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p]),
    "fft_last_error": (ctypes.c_int, []),
    "fft_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "fft_plan_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t]),
    "fft_plan_explain": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(fft_iodim), ctypes.c_int,
                                        ctypes.POINTER(fft_iodim), ctypes.c_int, ctypes.c_uint,
                                        ctypes.c_char_p, ctypes.c_size_t]),
    "fft_plan_bytes": (ctypes.c_double, [ctypes.c_void_p]),
    "fft_plan_flops": (ctypes.c_double, [ctypes.c_void_p]),
    "fft_plan_launches": (ctypes.c_int, [ctypes.c_void_p]),
    "fft_plan_scratch_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "fft_export_wisdom": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_size_t]),
    "fft_import_wisdom": (ctypes.c_int, [ctypes.c_char_p]),
    "fft_forget_wisdom": (None, []),
    "fft_group_create": (ctypes.c_void_p, [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p), ctypes.c_uint]),
    "fft_group_execute": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                                         ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]),
    "fft_group_status": (ctypes.c_int, [ctypes.c_void_p]),
    "fft_group_launches": (ctypes.c_int, [ctypes.c_void_p]),
    "fft_group_mode": (ctypes.c_int, [ctypes.c_void_p]),
    "fft_group_destroy": (None, [ctypes.c_void_p]),
    "fft_server_create": (ctypes.c_void_p, [ctypes.c_size_t, ctypes.c_int, ctypes.c_uint]),
    "fft_server_now": (ctypes.c_double, [ctypes.c_void_p]),
    "fft_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                         ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_double, ctypes.POINTER(ctypes.c_uint64)]),
    "fft_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "fft_server_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_double]),
    "fft_server_drain": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "fft_server_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t]),
    "fft_server_destroy": (None, [ctypes.c_void_p]),
    "fft_twiddle_exponents": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_int64, ctypes.c_void_p]),
    "fft_twiddle_table": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "fft_execute_1d_noalloc": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p]),
}

GBFFT_NOALLOC_MAX_POINTS = 1 << 21


def load():
    """Load ``libgbfft.so`` (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                                   "(run __graft_entry__.build())")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _dims(dims):
    dims = [tuple(int(v) for v in d) for d in dims]
    arr = (fft_iodim * max(1, len(dims)))()
    for i, (n, s_in, s_out) in enumerate(dims):
        arr[i].n, arr[i].is_, arr[i].os = n, s_in, s_out
    return len(dims), arr


def _text(fn, *args):
    need = fn(*args, None, 0)
    if need < 0:
        return None
    buf = ctypes.create_string_buffer(need + 1)
    fn(*args, buf, need + 1)
    return buf.value.decode()


# ------------------------------------------------------------------ C ABI names

def fft_last_error() -> int:
    return load().fft_last_error()


def fft_error_string(code: int) -> str:
    return load().fft_error_string(int(code)).decode()


def fft_plan_dft(dims, howmany=(), sign=-1, flags=0):
    """Plan dft(N, V, I, O); returns an opaque handle (int) or raises GbfftError."""
    r, d = _dims(dims)
    hr, h = _dims(howmany)
    p = load().fft_plan_dft(r, d, hr, h, int(sign), int(flags))
    if not p:
        raise GbfftError(fft_last_error(), "fft_plan_dft")
    return p


def fft_plan_dft_r2c(dims, howmany=(), flags=0):
    """Plan a real-input DFT (real strides on the input side, complex on the output)."""
    r, d = _dims(dims)
    hr, h = _dims(howmany)
    p = load().fft_plan_dft_r2c(r, d, hr, h, int(flags))
    if not p:
        raise GbfftError(fft_last_error(), "fft_plan_dft_r2c")
    return p


def fft_plan_dft_c2r(dims, howmany=(), flags=0):
    """Plan a real-output DFT (complex strides on the input side, real on the output)."""
    r, d = _dims(dims)
    hr, h = _dims(howmany)
    p = load().fft_plan_dft_c2r(r, d, hr, h, int(flags))
    if not p:
        raise GbfftError(fft_last_error(), "fft_plan_dft_c2r")
    return p


def fft_execute(plan, in_ptr: int, out_ptr: int, stream: int = 0) -> None:
    rc = load().fft_execute(plan, ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream))
    if rc != FFT_OK:
        raise GbfftError(rc, "fft_execute")


def fft_execute_scratch(plan, in_ptr: int, out_ptr: int, scratch_ptr: int, stream: int = 0) -> None:
    rc = load().fft_execute_scratch(plan, ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr),
                                    ctypes.c_void_p(scratch_ptr), ctypes.c_void_p(stream))
    if rc != FFT_OK:
        raise GbfftError(rc, "fft_execute_scratch")


def fft_sync_status(plan) -> int:
    """Wait for the plan's last execution; its device status (FFT_OK or the error), cleared."""
    return load().fft_sync_status(plan)


def fft_destroy(plan) -> None:
    if plan:
        load().fft_destroy(plan)


def fft_plan_info(plan) -> str:
    return _text(load().fft_plan_info, plan)


def fft_plan_explain(dims, howmany=(), sign=-1, flags=0) -> str:
    r, d = _dims(dims)
    hr, h = _dims(howmany)
    s = _text(load().fft_plan_explain, r, d, hr, h, int(sign), int(flags))
    if s is None:
        raise GbfftError(fft_last_error(), "fft_plan_explain")
    return s


def fft_plan_bytes(plan) -> float:
    return load().fft_plan_bytes(plan)


def fft_plan_flops(plan) -> float:
    return load().fft_plan_flops(plan)


def fft_plan_launches(plan) -> int:
    return load().fft_plan_launches(plan)


def fft_plan_scratch_bytes(plan) -> int:
    return load().fft_plan_scratch_bytes(plan)


def fft_export_wisdom() -> str:
    return _text(load().fft_export_wisdom)


def fft_import_wisdom(text: str) -> None:
    rc = load().fft_import_wisdom(text.encode())
    if rc != FFT_OK:
        raise GbfftError(rc, "fft_import_wisdom")


def fft_forget_wisdom() -> None:
    load().fft_forget_wisdom()


def _ptrs(vals):
    arr = (ctypes.c_void_p * max(1, len(vals)))()
    for i, v in enumerate(vals):
        arr[i] = int(v)
    return arr


def fft_group_create(plans, flags=0):
    """Group plan handles for one persistent launch; returns a handle or raises."""
    g = load().fft_group_create(len(plans), _ptrs(plans), int(flags))
    if not g:
        raise GbfftError(fft_last_error(), "fft_group_create")
    return g


def fft_group_execute(group, in_ptrs, out_ptrs, stream=0) -> None:
    rc = load().fft_group_execute(group, _ptrs(in_ptrs), _ptrs(out_ptrs), ctypes.c_void_p(stream))
    if rc != FFT_OK:
        raise GbfftError(rc, "fft_group_execute")


def fft_group_status(group) -> int:
    return load().fft_group_status(group)


def fft_group_launches(group) -> int:
    return load().fft_group_launches(group)


def fft_group_mode(group) -> int:
    """1: persistent queue, 2: graph of plan launches."""
    return load().fft_group_mode(group)


def fft_group_destroy(group) -> None:
    if group:
        load().fft_group_destroy(group)


def fft_server_create(budget_bytes: int, nstreams: int = 4, flags: int = 0):
    s = load().fft_server_create(int(budget_bytes), int(nstreams), int(flags))
    if not s:
        raise GbfftError(fft_last_error(), "fft_server_create")
    return s


def fft_server_now(server) -> float:
    return load().fft_server_now(server)


def fft_server_submit(server, n, batch, sign, host_in_ptr, host_out_ptr, arrival=-1.0) -> int:
    """Submit a dense row-major transform (lengths n, last fastest); returns the ticket."""
    arr = (ctypes.c_int64 * 3)(*(list(n) + [1] * (3 - len(n))))
    t = ctypes.c_uint64(0)
    rc = load().fft_server_submit(server, len(n), arr, int(batch), int(sign), ctypes.c_void_p(host_in_ptr),
                                  ctypes.c_void_p(host_out_ptr), float(arrival), ctypes.byref(t))
    if rc != FFT_OK:
        raise GbfftError(rc, "fft_server_submit")
    return t.value


def fft_server_poll(server, ticket) -> int:
    return load().fft_server_poll(server, int(ticket))


def fft_server_wait(server, ticket, timeout_s=60.0) -> int:
    return load().fft_server_wait(server, int(ticket), float(timeout_s))


def fft_server_drain(server, timeout_s=600.0) -> int:
    return load().fft_server_drain(server, float(timeout_s))


def fft_server_stats(server) -> dict:
    import json
    return json.loads(_text(load().fft_server_stats, server))


def fft_server_destroy(server) -> None:
    if server:
        load().fft_server_destroy(server)


def fft_twiddle_exponents(kind: int, N: int, a: int, b: int, count: int):
    """Exponent of every entry of one twiddle / chirp table (host evaluation of
    the generators' integer code); returns a numpy int64 array."""
    import numpy as np
    out = np.empty(max(0, int(count)), dtype=np.int64)
    rc = load().fft_twiddle_exponents(int(kind), int(N), int(a), int(b), int(count),
                                      ctypes.c_void_p(out.ctypes.data if count else 0))
    if rc != FFT_OK:
        raise GbfftError(rc, "fft_twiddle_exponents")
    return out


def fft_twiddle_table(kind: int, N: int, a: int, b: int, count: int, out_ptr: int, stream: int = 0) -> None:
    """Run the device generator of one table into a complex64 device array."""
    rc = load().fft_twiddle_table(int(kind), int(N), int(a), int(b), int(count), ctypes.c_void_p(out_ptr),
                                  ctypes.c_void_p(stream))
    if rc != FFT_OK:
        raise GbfftError(rc, "fft_twiddle_table")


def fft_execute_1d_noalloc(n: int, batch: int, sign: int, in_ptr: int, out_ptr: int, stream: int = 0) -> None:
    """Batched contiguous 1-D DFT that allocates no device memory (static scratch);
    raises GbfftError with the library's code on failure."""
    rc = load().fft_execute_1d_noalloc(int(n), int(batch), int(sign), ctypes.c_void_p(in_ptr),
                                       ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream))
    if rc != FFT_OK:
        raise GbfftError(rc, "fft_execute_1d_noalloc")


# ------------------------------------------------------------------ torch helper

class Plan:
    """Owns a plan; ``execute(x, y)`` runs it on complex64 CUDA tensors (element 0
    of each is ``tensor.data_ptr()`` -- pass ``offset`` for negative strides)."""

    def __init__(self, dims, howmany=(), sign=-1, flags=0):
        self.dims = [tuple(d) for d in dims]
        self.howmany = [tuple(d) for d in howmany]
        self.sign = sign
        self.flags = flags
        self.handle = fft_plan_dft(self.dims, self.howmany, sign, flags)

    def execute(self, x, y, stream=None, in_offset=0, out_offset=0):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        fft_execute(self.handle, x.data_ptr() + 8 * in_offset, y.data_ptr() + 8 * out_offset, stream)

    @property
    def info(self):
        return fft_plan_info(self.handle)

    @property
    def bytes(self):
        return fft_plan_bytes(self.handle)

    @property
    def flops(self):
        return fft_plan_flops(self.handle)

    @property
    def launches(self):
        return fft_plan_launches(self.handle)

    def destroy(self):
        if self.handle:
            fft_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
