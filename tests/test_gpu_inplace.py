"""In-place transforms without full-size scratch (sec. 4.2: in-place plans from
DIT/DIF steps and in-place transposes; the rank-0 in-place transpose of
sec. 4.1.1; the indirect plan), against the FP64 oracle within 2e-6 per
transform, and bit-exact for the transposes:
  * 1-D n = s^2 in place: column DFTs in place (twiddle fused), row DFTs in
    place, an in-place square transpose -- the plan holds no scratch;
  * rank-2 4096 x 4096 in place with no scratch;
  * rank-0 in-place square transposes, batched, with ragged tiles;
  * the indirect plan (copy into the output's layout, transform in place)."""
import numpy as np
import pytest

import fft_inputs
from parity import check

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2602_23525_gb300 import gbfft  # noqa: E402

IP, EST = gbfft.FFT_INPLACE, gbfft.FFT_ESTIMATE


@pytest.mark.parametrize("e,b", [(14, 16), (16, 8), (18, 4), (20, 2), (24, 1)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_one_dimensional_in_place_without_scratch(e, b, sign):
    n = 1 << e
    how = [(b, n, n)] if b > 1 else []
    p = gbfft.Plan([(n, 1, 1)], how, sign, IP | EST)
    assert "in place without scratch" in p.info and gbfft.fft_plan_scratch_bytes(p.handle) == 0, p.info
    p.destroy()
    x = fft_inputs.uniform_c64(n * b, fft_inputs.seed_for(10, e))
    err, info = check([(n, 1, 1)], how, sign, x, flags=EST, inplace=True, algo="ct")


def test_rank2_4096_in_place_without_scratch():
    dims = [(4096, 4096, 4096), (4096, 1, 1)]
    p = gbfft.Plan(dims, [], -1, IP | EST)
    assert gbfft.fft_plan_scratch_bytes(p.handle) == 0, p.info
    p.destroy()
    x = fft_inputs.uniform_c64(4096 * 4096, fft_inputs.seed_for(10, 30))
    check(dims, [], -1, x, flags=EST, inplace=True, algo="ct")


@pytest.mark.parametrize("s,batch", [(64, 5), (1000, 2), (4096, 1), (33, 7)])
def test_rank0_in_place_square_transpose(s, batch):
    x = fft_inputs.uniform_c64(s * s * batch, fft_inputs.seed_for(10, s))
    t = torch.from_numpy(x).cuda()
    how = [(s, s, 1), (s, 1, s)] + ([(batch, s * s, s * s)] if batch > 1 else [])
    p = gbfft.Plan([], how, -1, IP | EST)
    assert "transpose in place" in p.info
    p.execute(t, t)
    torch.cuda.synchronize()
    got = t.cpu().numpy().reshape(batch, s, s)
    assert np.array_equal(got, x.reshape(batch, s, s).transpose(0, 2, 1))
    p.destroy()


def test_non_square_in_place_transpose_is_refused():
    with pytest.raises(gbfft.GbfftError) as e:
        gbfft.Plan([], [(64, 32, 1), (32, 1, 64)], -1, IP | EST)
    assert e.value.code == gbfft.FFT_ERR_UNSUPPORTED


@pytest.mark.parametrize("n,how", [(4096, [(64, 1, 4096)]), (1000, [(20, 1000, 1000)]), (65536, [(8, 1, 65536)])])
def test_indirect_plan(n, how):
    is_ = how[0][1] * how[0][0] if how[0][1] == 1 else 1
    dims = [(n, is_, 1)]
    v = "[" + ",".join(f"({a},{b},{c})" for a, b, c in how) + "]"
    gbfft.fft_forget_wisdom()
    gbfft.fft_import_wisdom(f"gbfft-wisdom 1\nr1 n={n} is={is_} os=1 v={v} ip=0\tindirect\n")
    try:
        x = fft_inputs.uniform_c64(n * how[0][0], fft_inputs.seed_for(10, n))
        for sign in (-1, 1):
            err, info = check(dims, how, sign, x, flags=EST, algo="ct")
            assert "indirect" in info, info
    finally:
        gbfft.fft_forget_wisdom()


def test_measured_in_place_plan():
    n, b = 1 << 20, 4
    x = fft_inputs.uniform_c64(n * b, fft_inputs.seed_for(10, 40))
    err, info = check([(n, 1, 1)], [(b, n, n)], -1, x, flags=gbfft.FFT_MEASURE, inplace=True, algo="ct")
    print(info.splitlines()[1])
