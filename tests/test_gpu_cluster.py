"""The one-pass cluster kernel (n = 2^13 .. 2^17 over a thread-block cluster,
eq. (2) with the exchange through distributed shared memory) against the FP64
oracle, relative L2 <= 2e-6 per transform.

Every instantiated (n1, n2, C) configuration is forced through imported wisdom;
batches are larger than the number of co-resident clusters (several
iterations of the persistent loop, ragged last round), both signs; layouts
cover the tensor-map load (padded batch stride), the plain-load path (odd batch
stride, 8-byte aligned input), in-place execution and a single transform."""
import numpy as np
import pytest

import fft_inputs
from parity import TOL, check, per_transform_error, reference, run_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2602_23525_gb300 import gbfft  # noqa: E402

CONFIGS = [(6, 7, 2, 1), (6, 7, 2, 2), (7, 7, 4, 1), (7, 7, 4, 2), (7, 7, 2, 2), (7, 8, 8, 1), (7, 8, 8, 2),
           (7, 8, 4, 2), (7, 9, 16, 1), (8, 8, 8, 2), (8, 8, 16, 1), (8, 9, 16, 2)]


def u(count, seed):
    return fft_inputs.uniform_c64(count, seed)


def force(n, how, choice, inplace=False):
    """Import a wisdom entry that makes the planner take `choice` for this problem."""
    gbfft.fft_forget_wisdom()
    v = ",".join(f"({a},{b},{c})" for a, b, c in how if a > 1)  # the canonical problem drops n = 1 loops
    gbfft.fft_import_wisdom(f"gbfft-wisdom 1\nr1 n={n} is=1 os=1 v=[{v}] ip={1 if inplace else 0}\t{choice}\n")


@pytest.mark.parametrize("cfg", CONFIGS)
@pytest.mark.parametrize("sign", [-1, 1])
def test_cluster_configs(cfg, sign):
    l1, l2, c, nb = cfg
    n = 2 ** (l1 + l2)
    batch = {13: 45, 14: 41, 15: 37, 16: 27, 17: 19}[l1 + l2] + 40 * (nb == 1)
    how = [(batch, n, n)]
    force(n, how, f"cluster:{l1}.{l2}.{c}.{nb}")
    try:
        err, info = check([(n, 1, 1)], how, sign, u(n * batch, 300 + l1 + l2 + c), flags=gbfft.FFT_WISDOM_ONLY,
                          algo="ct")
    finally:
        gbfft.fft_forget_wisdom()
    assert f"pass cluster n={n} = {2 ** l1} x {2 ** l2} C={c} buffers={nb}" in info


@pytest.mark.parametrize("n", [2 ** 13, 2 ** 14, 2 ** 16, 2 ** 17])
def test_cluster_layouts(n):
    """padded (even) batch stride: tensor-map loads; odd batch stride: plain
    loads; input at an 8-byte (not 16-byte) boundary: plain loads."""
    e = n.bit_length() - 1
    cfg = [c for c in CONFIGS if c[0] + c[1] == e][0]
    choice = "cluster:" + ".".join(str(v) for v in cfg)
    b = 23
    for k, (vis, vos, off) in enumerate([(n + 2, n + 6, 0), (n + 1, n + 3, 0), (n, n, 1)]):
        how = [(b, vis, vos)]
        force(n, how, choice)
        x = u(vis * b + 2, 400 + k + e)
        try:
            kw = {"in_offset": off} if off else {}
            y, info = run_gpu([(n, 1, 1)], how, -1, x, flags=gbfft.FFT_WISDOM_ONLY, **kw)
        finally:
            gbfft.fft_forget_wisdom()
        assert "pass cluster" in info
        ref = reference([(n, 1, 1)], how, -1, x, in_offset=off if off else None, out_len=len(y), algo="ct")
        assert per_transform_error(y, ref, [(n, 1, 1)], how).max() <= TOL


def test_cluster_inplace_and_single_transform():
    n = 2 ** 16
    for batch in (1, 21):
        how = [(batch, n, n)]
        x = u(n * batch, 500 + batch)
        for inplace, sign in ((True, 1), (False, -1)):
            force(n, how, "cluster:8.8.8.2", inplace=inplace)
            try:
                err, info = check([(n, 1, 1)], how, sign, x, flags=gbfft.FFT_WISDOM_ONLY, inplace=inplace, algo="ct")
            finally:
                gbfft.fft_forget_wisdom()
            assert "pass cluster" in info


def test_cluster_full_size_sampled():
    """n = 65536 x 512 transforms (256 MiB in, the single-pass workload), with
    the oracle on sampled transforms."""
    n, batch = 2 ** 16, 512
    x = u(n * batch, 510)
    dims, how = [(n, 1, 1)], [(batch, n, n)]
    force(n, how, "cluster:8.8.8.2")
    try:
        y, info = run_gpu(dims, how, -1, x, flags=gbfft.FFT_WISDOM_ONLY)
    finally:
        gbfft.fft_forget_wisdom()
    assert "pass cluster" in info
    for t in (0, 1, 255, 511):
        seg = x[t * n:(t + 1) * n]
        ref = reference(dims, [], -1, seg, algo="ct")
        got = y[t * n:(t + 1) * n].astype(np.complex128)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= TOL, (t, err)


def test_cluster_plan_in_group():
    """n = 2^14 has a one-CTA fallback the persistent queue runs; n = 2^16 has
    none: the queue is refused and the group uses the graph of plan launches."""
    p14 = gbfft.Plan([(2 ** 14, 1, 1)], [(4, 2 ** 14, 2 ** 14)], -1, gbfft.FFT_ESTIMATE)
    force(2 ** 16, [(4, 2 ** 16, 2 ** 16)], "cluster:8.8.8.2")
    try:
        p16 = gbfft.Plan([(2 ** 16, 1, 1)], [(4, 2 ** 16, 2 ** 16)], -1, gbfft.FFT_WISDOM_ONLY)
    finally:
        gbfft.fft_forget_wisdom()
    try:
        assert "pass cluster" in p14.info and "pass cluster" in p16.info
        g = gbfft.fft_group_create([p14.handle], gbfft.FFT_GROUP_PERSISTENT)
        gbfft.fft_group_destroy(g)
        with pytest.raises(gbfft.GbfftError) as ei:
            gbfft.fft_group_create([p16.handle], gbfft.FFT_GROUP_PERSISTENT)
        assert ei.value.code == gbfft.FFT_ERR_UNSUPPORTED
        g = gbfft.fft_group_create([p14.handle, p16.handle])
        assert gbfft.fft_group_mode(g) == 2
        x = fft_inputs.uniform_c64(4 * 2 ** 16, 520)
        a = torch.from_numpy(x[:4 * 2 ** 14]).cuda()
        b = torch.from_numpy(x).cuda()
        ya, yb = torch.zeros_like(a), torch.zeros_like(b)
        gbfft.fft_group_execute(g, [a.data_ptr(), b.data_ptr()], [ya.data_ptr(), yb.data_ptr()],
                                torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert gbfft.fft_group_status(g) == gbfft.FFT_OK
        gbfft.fft_group_destroy(g)
        for y, xs, n in ((ya, x[:4 * 2 ** 14], 2 ** 14), (yb, x, 2 ** 16)):
            ref = reference([(n, 1, 1)], [(4, n, n)], -1, xs, algo="ct")
            assert per_transform_error(y.cpu().numpy(), ref, [(n, 1, 1)], [(4, n, n)]).max() <= TOL
    finally:
        p14.destroy()
        p16.destroy()
