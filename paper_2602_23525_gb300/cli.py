r"""Run and time one DFT problem from the command line.

    python -m paper_2602_23525_gb300.cli --dims 4096,1,1 --howmany 8192,4096,4096 \
        --sign -1 --reps 5 [--estimate]

Dimensions are "n,is,os" triples (strides in complex elements), as in
dft(N, V, I, O).  Prints the plan tree and the median device time per
execution with its GFLOP/s (5 N log2 N) and algorithmic GB/s (16 B/point).
--wisdom takes wisdom entries ("key\tchoice" lines, with \t and \n written
as escapes) to import before planning, e.g. to replay one plan choice:
    --wisdom 'r1 n=10007 is=1 os=1 v=[(512,10007,10007)] ip=0\tblue:32768'
"""
import argparse
import math
import statistics
import sys


def parse_dims(items):
    out = []
    for it in items or []:
        n, a, b = (int(v) for v in it.split(","))
        out.append((n, a, b))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", nargs="*", default=[])
    ap.add_argument("--howmany", nargs="*", default=[])
    ap.add_argument("--sign", type=int, default=-1)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--estimate", action="store_true")
    ap.add_argument("--inplace", action="store_true")
    ap.add_argument("--wisdom", default="")
    a = ap.parse_args(argv)
    import torch

    from . import gbfft
    if a.wisdom:
        body = a.wisdom.replace("\\t", "\t").replace("\\n", "\n")
        gbfft.fft_import_wisdom("gbfft-wisdom 1\n" + body.rstrip("\n") + "\n")
    dims, how = parse_dims(a.dims), parse_dims(a.howmany)
    flags = (gbfft.FFT_ESTIMATE if a.estimate else 0) | (gbfft.FFT_INPLACE if a.inplace else 0)

    def span(k):
        lo = hi = 0
        for d in dims + how:
            e = (d[0] - 1) * d[k]
            lo, hi = (lo + e, hi) if e < 0 else (lo, hi + e)
        return lo, hi

    ilo, ihi = span(1)
    olo, ohi = span(2)
    x = torch.randn(ihi - ilo + 1, dtype=torch.complex64, device="cuda")
    y = x if a.inplace else torch.empty(ohi - olo + 1, dtype=torch.complex64, device="cuda")
    plan = gbfft.Plan(dims, how, a.sign, flags)
    print(plan.info)
    s = torch.cuda.current_stream().cuda_stream
    for _ in range(a.warmup):
        gbfft.fft_execute(plan.handle, x.data_ptr() - 8 * ilo, y.data_ptr() - 8 * (ilo if a.inplace else olo), s)
    times = []
    for _ in range(a.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        gbfft.fft_execute(plan.handle, x.data_ptr() - 8 * ilo, y.data_ptr() - 8 * (ilo if a.inplace else olo), s)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    print(f"median {ms:.4f} ms  {plan.flops / ms / 1e6:.1f} GFLOP/s  {plan.bytes / ms / 1e6:.1f} GB/s algorithmic"
          f"  launches/exec {plan.launches}")
    plan.destroy()
    return 0


if __name__ == "__main__":
    sys.exit(main())
