"""The serving loop (fft_server_*): requests of mixed shapes, ranks, batches and
signs arriving while others run are admitted by the byte budget, merged when
compatible, and each result matches the FP64 oracle and the same transform run
alone, within the relative-L2 tolerance 2e-6."""
import time

import numpy as np
import pytest

import fft_inputs
from parity import TOL, per_transform_error, reference

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2602_23525_gb300 import gbfft  # noqa: E402

SHAPES = [(256,), (1000,), (4096,), (97,), (64, 48), (16, 8, 12), (2187,), (32768,)]


def dense(shape, batch):
    dims, st = [], 1
    for n in reversed(shape):
        dims.append((n, st, st))
        st *= n
    dims.reverse()
    return dims, [(batch, st, st)]


def alone(shape, batch, sign, x):
    dims, how = dense(shape, batch)
    xt = torch.from_numpy(x).cuda()
    yt = torch.zeros_like(xt)
    p = gbfft.Plan(dims, how, sign, gbfft.FFT_ESTIMATE)
    p.execute(xt, yt)
    torch.cuda.synchronize()
    p.destroy()
    return yt.cpu().numpy()


def test_mixed_requests_match_oracle_and_alone():
    rng = np.random.default_rng(123)
    server = gbfft.fft_server_create(256 << 20, 3)
    reqs = []
    for i in range(48):
        shape = SHAPES[int(rng.integers(len(SHAPES)))] if i % 3 else SHAPES[0]  # repeats merge
        batch = int(rng.integers(1, 9))
        sign = int(rng.choice([-1, 1]))
        pts = int(np.prod(shape))
        x = fft_inputs.uniform_c64(pts * batch, 900 + i)
        hin = torch.from_numpy(x).pin_memory()
        hout = torch.zeros_like(hin).pin_memory()
        t = gbfft.fft_server_submit(server, shape, batch, sign, hin.data_ptr(), hout.data_ptr())
        reqs.append((t, shape, batch, sign, x, hin, hout))
        if i % 7 == 0:
            time.sleep(0.002)  # arrivals while earlier requests are on the device
    for t, *_ in reqs:
        assert gbfft.fft_server_wait(server, t, 120.0) == gbfft.FFT_OK
    stats = gbfft.fft_server_stats(server)
    gbfft.fft_server_destroy(server)
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert 0 < stats["budget_high_water_bytes"] <= 256 << 20
    assert stats["p99_latency_s"] >= stats["p50_latency_s"] > 0
    for t, shape, batch, sign, x, hin, hout in reqs:
        y = hout.numpy()
        dims, how = dense(shape, batch)
        ref = reference(dims, how, sign, x)
        assert per_transform_error(y, ref, dims, how).max() <= TOL, (shape, batch, sign)
        solo = alone(shape, batch, sign, x).astype(np.complex128)
        assert per_transform_error(y, solo, dims, how).max() <= TOL


def test_budget_admission_and_rejection():
    budget = 6 << 20  # a few requests at a time
    server = gbfft.fft_server_create(budget, 2)
    keep = []
    for i in range(12):
        x = fft_inputs.uniform_c64(4096 * 32, 950 + i)  # 1 MiB in, 1 MiB out
        hin = torch.from_numpy(x).pin_memory()
        hout = torch.zeros_like(hin).pin_memory()
        t = gbfft.fft_server_submit(server, (4096,), 32, -1, hin.data_ptr(), hout.data_ptr())
        keep.append((t, x, hout, hin))
    big_in = torch.zeros(1 << 20, dtype=torch.complex64).pin_memory()  # 8 MiB: never fits
    big_out = torch.zeros_like(big_in).pin_memory()
    tb = gbfft.fft_server_submit(server, (1 << 20,), 1, -1, big_in.data_ptr(), big_out.data_ptr())
    assert gbfft.fft_server_drain(server, 120.0) == gbfft.FFT_OK
    assert gbfft.fft_server_poll(server, tb) == gbfft.FFT_ERR_BUDGET
    for t, x, hout, _ in keep:
        assert gbfft.fft_server_poll(server, t) == gbfft.FFT_OK
        ref = reference([(4096, 1, 1)], [(32, 4096, 4096)], -1, x)
        assert per_transform_error(hout.numpy(), ref, [(4096, 1, 1)], [(32, 4096, 4096)]).max() <= TOL
    stats = gbfft.fft_server_stats(server)
    gbfft.fft_server_destroy(server)
    assert stats["budget_high_water_bytes"] <= budget
    assert stats["rejected"] == 1


def test_requests_merge_behind_a_blocked_head():
    """Admission keeps arrival order: a head request waiting for budget holds
    back the requests behind it, and the waiting ones of the same shape and
    sign are then merged into one launch."""
    big_n, big_b = 65536, 32               # 16 MiB in, 16 MiB out (+ scratch)
    server = gbfft.fft_server_create(64 << 20, 2)
    bufs = []
    for i in range(2):
        x = fft_inputs.uniform_c64(big_n * big_b, 970 + i)
        bufs.append(((big_n,), big_b, x, torch.from_numpy(x).pin_memory(), torch.zeros(big_n * big_b,
                     dtype=torch.complex64).pin_memory()))
    for i in range(8):
        x = fft_inputs.uniform_c64(4096 * 2, 980 + i)
        bufs.append(((4096,), 2, x, torch.from_numpy(x).pin_memory(), torch.zeros(8192, dtype=torch.complex64).pin_memory()))
    tickets = [gbfft.fft_server_submit(server, shape, b, -1, hin.data_ptr(), hout.data_ptr())
               for shape, b, _, hin, hout in bufs]
    assert gbfft.fft_server_drain(server, 120.0) == gbfft.FFT_OK
    stats = gbfft.fft_server_stats(server)
    gbfft.fft_server_destroy(server)
    assert stats["completed"] == len(bufs) and stats["failed"] == 0
    assert stats["merged_requests"] > 0, stats
    assert stats["budget_high_water_bytes"] <= 64 << 20
    for (shape, b, x, hin, hout) in bufs:
        n = shape[0]
        ref = reference([(n, 1, 1)], [(b, n, n)], -1, x)
        assert per_transform_error(hout.numpy(), ref, [(n, 1, 1)], [(b, n, n)]).max() <= TOL
