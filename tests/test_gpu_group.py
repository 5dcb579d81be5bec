"""Uneven batches (fft_group_*), with each executor (persistent queue, graph
of plan launches) and the measured choice: every transform of every plan
matches the FP64 oracle (relative L2 <= 2e-6) and its own plan run alone (bit
for bit with the graph of plan launches); CUDA-graph replays and pointer
changes keep results; a device wait that runs out reports
FFT_ERR_DEVICE_TIMEOUT and leaves the context usable."""
import numpy as np
import pytest

import fft_inputs
from parity import TOL, per_transform_error, reference

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2602_23525_gb300 import gbfft  # noqa: E402

EST = gbfft.FFT_ESTIMATE


def uneven_problems(batch):
    probs = []
    for i, n in enumerate(fft_inputs.UNEVEN_SIZES):
        if n in fft_inputs.UNEVEN_TRANSPOSED:
            dims, how = fft_inputs.transposed_1d(n, batch)
        else:
            dims, how = fft_inputs.batched_1d(n, batch)
        x = fft_inputs.gaussian_c64(n * batch, fft_inputs.seed_for(2, i))
        probs.append((n, dims, how, x))
    return probs


def run_group(probs, sign, stream, flags=0, repeat=1, plan_flags=EST):
    plans = [gbfft.Plan(d, h, sign, plan_flags) for _, d, h, _ in probs]
    ins = [torch.from_numpy(x).cuda() for *_, x in probs]
    outs = [torch.zeros_like(t) for t in ins]
    g = gbfft.fft_group_create([p.handle for p in plans], flags)
    try:
        for _ in range(repeat):
            gbfft.fft_group_execute(g, [t.data_ptr() for t in ins], [t.data_ptr() for t in outs], stream)
        torch.cuda.synchronize()
        status = gbfft.fft_group_status(g)
        alone = []
        for p, t in zip(plans, ins):
            y = torch.zeros_like(t)
            p.execute(t, y)
            alone.append(y)
        torch.cuda.synchronize()
    finally:
        gbfft.fft_group_destroy(g)
    res = [o.cpu().numpy() for o in outs], [a.cpu().numpy() for a in alone], status
    for p in plans:
        p.destroy()
    return res


MODES = [gbfft.FFT_GROUP_PERSISTENT, gbfft.FFT_GROUP_GRAPH, 0]


@pytest.mark.parametrize("flags", MODES)
def test_group_with_fused_bluestein(flags):
    """A plan whose Bluestein steps ride on the FFT stores (store epilogues)
    in a group: the persistent queue runs their generic passes with the same
    epilogue."""
    gbfft.fft_forget_wisdom()
    gbfft.fft_import_wisdom("gbfft-wisdom 1\nr1 n=10007 is=1 os=1 v=[(4,10007,10007)] ip=0\tblue:32768\n")
    try:
        probs = [(10007, [(10007, 1, 1)], [(4, 10007, 10007)], fft_inputs.gaussian_c64(10007 * 4, 95)),
                 (1000, [(1000, 1, 1)], [(4, 1000, 1000)], fft_inputs.gaussian_c64(4000, 96))]
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            outs, alone, status = run_group(probs, 1, s.cuda_stream, flags=flags)
        assert status == gbfft.FFT_OK
        for (n, dims, how, x), y, a in zip(probs, outs, alone):
            ref = reference(dims, how, 1, x, algo="ct" if n > 4096 else "auto")
            assert per_transform_error(y, ref, dims, how).max() <= TOL, n
    finally:
        gbfft.fft_forget_wisdom()


@pytest.mark.parametrize("sign", [-1, 1])
@pytest.mark.parametrize("flags", MODES)
def test_uneven_group_matches_oracle_and_alone(sign, flags):
    probs = uneven_problems(8)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        outs, alone, status = run_group(probs, sign, s.cuda_stream, flags=flags, repeat=2)
    assert status == gbfft.FFT_OK
    for (n, dims, how, x), y, a in zip(probs, outs, alone):
        ref = reference(dims, how, sign, x, algo="ct" if n > 4096 else "auto")
        err = per_transform_error(y, ref, dims, how)
        assert err.max() <= TOL, (n, err.max())
        assert per_transform_error(y, a.astype(np.complex128), dims, how).max() <= TOL
        if flags == gbfft.FFT_GROUP_GRAPH:
            assert np.array_equal(y, a)


@pytest.mark.parametrize("flags", MODES)
def test_group_on_legacy_stream_and_pointer_change(flags):
    probs = uneven_problems(4)[:4]
    plans = [gbfft.Plan(d, h, -1, EST) for _, d, h, _ in probs]
    ins = [torch.from_numpy(x).cuda() for *_, x in probs]
    g = gbfft.fft_group_create([p.handle for p in plans], flags)
    mode = gbfft.fft_group_mode(g)
    assert mode == {gbfft.FFT_GROUP_PERSISTENT: 1, gbfft.FFT_GROUP_GRAPH: 2}.get(flags, mode) and mode in (1, 2)
    assert gbfft.fft_group_launches(g) == (1 if mode == 1 else sum(p.launches for p in plans))
    s = torch.cuda.Stream()
    results = []
    for stream in (0, s.cuda_stream, s.cuda_stream):
        outs = [torch.zeros_like(t) for t in ins]  # new pointers every time
        gbfft.fft_group_execute(g, [t.data_ptr() for t in ins], [t.data_ptr() for t in outs], stream)
        torch.cuda.synchronize()
        results.append([o.cpu().numpy() for o in outs])
    assert gbfft.fft_group_status(g) == gbfft.FFT_OK
    gbfft.fft_group_destroy(g)
    for r in results[1:]:
        for a, b in zip(results[0], r):
            assert np.array_equal(a, b)
    for (n, dims, how, x), y in zip(probs, results[0]):
        ref = reference(dims, how, -1, x)
        assert per_transform_error(y, ref, dims, how).max() <= TOL
    for p in plans:
        p.destroy()


def test_group_wait_timeout_is_reported_and_context_survives():
    probs = uneven_problems(2)[:2]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        outs, alone, status = run_group(probs, -1, s.cuda_stream, flags=gbfft.FFT_GROUP_DEBUG_STALL)
    assert status == gbfft.FFT_ERR_DEVICE_TIMEOUT
    # the real items still completed, and the context still runs plans
    for (n, dims, how, x), y in zip(probs, outs):
        ref = reference(dims, how, -1, x)
        assert per_transform_error(y, ref, dims, how).max() <= TOL
    n = 4096
    x = fft_inputs.uniform_c64(n * 4, 5)
    xt = torch.from_numpy(x).cuda()
    yt = torch.zeros_like(xt)
    p = gbfft.Plan([(n, 1, 1)], [(4, n, n)], -1, EST)
    p.execute(xt, yt)
    torch.cuda.synchronize()
    ref = reference([(n, 1, 1)], [(4, n, n)], -1, x)
    assert per_transform_error(yt.cpu().numpy(), ref, [(n, 1, 1)], [(4, n, n)]).max() <= TOL
    p.destroy()


@pytest.mark.parametrize("plan_flags", [EST, gbfft.FFT_MEASURE])
def test_uneven_full_size_sampled(plan_flags):
    """The full uneven workload (6 sizes x 512, mixed layouts) in one group
    execution, with estimated plans and with the measured plans the benchmark
    runs; sampled transforms (first, middle, last of each size) against the
    oracle."""
    batch = fft_inputs.UNEVEN_BATCH
    probs = uneven_problems(batch)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        outs, alone, status = run_group(probs, -1, s.cuda_stream, plan_flags=plan_flags)
    assert status == gbfft.FFT_OK
    for (n, dims, how, x), y in zip(probs, outs):
        for v in (0, batch // 2, batch - 1):
            if n in fft_inputs.UNEVEN_TRANSPOSED:
                xi = x[v::batch]        # column v in, row v out
                yi = y[v * n:(v + 1) * n]
            else:
                xi = x[v * n:(v + 1) * n]
                yi = y[v * n:(v + 1) * n]
            ref = reference([(n, 1, 1)], [], -1, xi, algo="ct" if n > 4096 else "auto")
            err = np.linalg.norm(yi.astype(np.complex128) - ref) / np.linalg.norm(ref)
            assert err <= TOL, (n, v, err)
