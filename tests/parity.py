"""Shared helpers for the GPU parity tests: run a problem through the C ABI and
compare it with the FP64 oracle, transform by transform.

The gate is the relative L2 error per transform, ||y_gpu - y_ref|| / ||y_ref||
(computed in FP64), at most 2e-6; rank-0 problems (copies) must be bit-exact.
"""
import itertools

import numpy as np

import oracle

TOL = 2e-6


def index_map(dims, howmany, side):
    """Element indices, shape (count, points): row = vector index (row-major over
    howmany), column = transform point (row-major over dims)."""
    k = 1 if side == "in" else 2

    def offsets(ds):
        off = np.zeros(1, dtype=np.int64)
        for d in ds:
            off = (off[:, None] + np.arange(d[0], dtype=np.int64)[None, :] * d[k]).reshape(-1)
        return off

    return offsets(howmany)[:, None] + offsets(dims)[None, :]


def extent(dims, howmany, side):
    k = 1 if side == "in" else 2
    lo = hi = 0
    for d in list(dims) + list(howmany):
        e = (d[0] - 1) * d[k]
        if e < 0:
            lo += e
        else:
            hi += e
    return lo, hi


def run_gpu(dims, howmany, sign, x, *, flags=0, in_offset=None, out_len=None, out_offset=None,
            inplace=False, fill=0.0, repeat=1):
    """Run the plan on cuda:0; returns the whole output buffer (complex64, numpy)
    and the plan info text."""
    import torch

    from paper_2602_23525_gb300 import gbfft

    lo, _ = extent(dims, howmany, "in")
    olo, ohi = extent(dims, howmany, "out")
    if in_offset is None:
        in_offset = -lo
    if out_offset is None:
        out_offset = -olo
    if out_len is None:
        out_len = out_offset + ohi + 1
    dev = torch.device("cuda:0")
    xin = torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex64)).to(dev)
    if inplace:
        yout = xin
        flags |= gbfft.FFT_INPLACE
    else:
        yout = torch.full((int(out_len),), complex(fill), dtype=torch.complex64, device=dev)
    plan = gbfft.Plan(dims, howmany, sign, flags)
    try:
        for _ in range(repeat):
            plan.execute(xin, yout, in_offset=in_offset, out_offset=out_offset if not inplace else in_offset)
        torch.cuda.synchronize()
        info = plan.info
    finally:
        plan.destroy()
    return yout.cpu().numpy(), info


def reference(dims, howmany, sign, x, *, in_offset=None, out_len=None, out_offset=None, algo="auto"):
    lo, _ = extent(dims, howmany, "in")
    olo, ohi = extent(dims, howmany, "out")
    if in_offset is None:
        in_offset = -lo
    if out_offset is None:
        out_offset = -olo
    if out_len is None:
        out_len = out_offset + ohi + 1
    return oracle.dft(x, dims, howmany, sign, out_len=out_len, in_offset=in_offset, out_offset=out_offset,
                      algo=algo)


def per_transform_error(y, ref, dims, howmany, out_offset=None):
    olo, _ = extent(dims, howmany, "out")
    if out_offset is None:
        out_offset = -olo
    idx = index_map(dims, howmany, "out") + out_offset
    a = y[idx].astype(np.complex128)
    b = ref[idx]
    num = np.linalg.norm(a - b, axis=1)
    den = np.linalg.norm(b, axis=1)
    den[den == 0] = 1.0
    return num / den


def check(dims, howmany, sign, x, *, tol=TOL, algo="auto", **kw):
    """Run GPU and oracle; assert every transform is within tol.  Returns (max error, info)."""
    y, info = run_gpu(dims, howmany, sign, x, **{k: v for k, v in kw.items() if k != "out_offset_ref"})
    ref = reference(dims, howmany, sign, x, in_offset=kw.get("in_offset"), out_len=len(y),
                    out_offset=kw.get("out_offset"), algo=algo)
    err = per_transform_error(y, ref, dims, howmany, out_offset=kw.get("out_offset"))
    assert np.all(np.isfinite(err)), info
    assert err.max() <= tol, f"max rel-L2 {err.max():.3e} > {tol:.1e} (worst transform {err.argmax()})\n{info}"
    return float(err.max()), info


def all_tuples(howmany):
    return itertools.product(*[range(d[0]) for d in howmany])
