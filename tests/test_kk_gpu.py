"""GPU parity of the per-spectrum KK kernel (Eq. KCARS with the surrogate,
Eq. K) against the FP64 oracle, through the C ABI.

Tolerance: relative L2 error of Im{K} <= 1e-4 (the FP32-path bound), and a
per-element bound of 2e-5 * max|Im| + 1e-5 * |Im| that the FP32 arithmetic
(log, two length-L FFTs, exp, sin) stays well inside."""
import numpy as np
import pytest

import oracle as O
from gpu_util import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_L2 = 1e-4


@pytest.fixture(scope="module")
def ctx():
    from paper_2005_07132_gb300 import build, Context
    build.build()
    c = Context(0)
    yield c
    c.close()


def _run(ctx, i, i_ref, pad_len=0, ld=None, ld_out=None, re=True):
    from paper_2005_07132_gb300 import kk_per_spectrum
    n, m = i.shape
    ld = ld or m
    ld_out = ld_out or m
    buf = torch.zeros((n, ld), dtype=torch.float32, device="cuda")
    buf[:, :m] = torch.from_numpy(np.ascontiguousarray(i, np.float32))
    x = buf[:, :m]
    ref_t = torch.from_numpy(np.ascontiguousarray(i_ref, np.float32)).cuda()
    im = torch.full((n, ld_out), 7.0, dtype=torch.float32, device="cuda")[:, :m]
    rr = torch.full((n, ld_out), 7.0, dtype=torch.float32, device="cuda")[:, :m] if re else None
    out = kk_per_spectrum(ctx, x, ref_t, pad_len=pad_len, im_out=im, re_out=rr)
    torch.cuda.synchronize()
    if re:
        return out[1].cpu().numpy(), out[0].cpu().numpy(), im
    return None, out.cpu().numpy(), im


def _check(im_gpu, re_gpu, i, i_ref, pad_len=0):
    re_o, im_o = O.kk_per_spectrum(i.astype(np.float64), i_ref.astype(np.float64),
                                   L=pad_len or None)
    assert rel_l2(im_gpu, im_o) <= RTOL_L2
    tol = 2e-5 * np.abs(im_o).max() + 1e-5 * np.abs(im_o)
    assert np.all(np.abs(im_gpu - im_o) <= tol)
    if re_gpu is not None:
        assert rel_l2(re_gpu, re_o) <= RTOL_L2


def test_kk_img64_m512(ctx):
    from paper_2005_07132_gb300.synth import CONFIGS, make_cube
    cube = make_cube(CONFIGS["img64_m512"])
    re, im, _ = _run(ctx, cube.i_cars, cube.i_ref)
    _check(im, re, cube.i_cars, cube.i_ref)


@pytest.mark.parametrize("n,m,pad", [(1, 37, 0), (3, 37, 0), (1001, 878, 0), (257, 1000, 4096),
                                      (64, 1600, 0), (5, 64, 64), (9, 2, 0), (33, 4096, 8192),
                                      # pad length 2,048 at both ends of its range: the widest
                                      # edge padding (513) and none to spare (1,024)
                                      (3, 513, 0), (2, 1024, 0), (4099, 1000, 0)])
def test_kk_ragged_shapes(ctx, n, m, pad):
    r = np.random.default_rng(n * 7919 + m)
    i_ref = r.uniform(0.5, 2.0, m).astype(np.float32)
    i = (i_ref * np.exp(2 * (0.3 * r.standard_normal((n, m))))).astype(np.float32)
    re, im, _ = _run(ctx, i, i_ref, pad_len=pad)
    _check(im, re, i, i_ref, pad)


@pytest.mark.parametrize("n,m", [(50, 300), (37, 1000)])
def test_kk_strided_rows_and_untouched_padding(ctx, n, m):
    r = np.random.default_rng(11)
    i_ref = r.uniform(0.5, 2.0, m).astype(np.float32)
    i = (i_ref * np.exp(0.4 * r.standard_normal((n, m)))).astype(np.float32)
    re, im, im_view = _run(ctx, i, i_ref, ld=m + 13, ld_out=m + 5)
    _check(im, re, i, i_ref)
    full = im_view.as_strided((n, m + 5), (m + 5, 1)).cpu().numpy()
    assert np.all(full[:, m:] == 7.0)  # stride padding never written


def test_kk_clamp_count(ctx):
    r = np.random.default_rng(5)
    n, m = 20, 128
    i_ref = np.ones(m, np.float32)
    i = r.uniform(0.5, 2.0, (n, m)).astype(np.float32)
    i[3, 10] = -1.0
    i[7, :5] = 0.0
    ctx.sync_status()
    re, im, _ = _run(ctx, i, i_ref)
    st, clamped = ctx.sync_status()
    assert st == 0 and clamped == 6
    _check(im, re, i, i_ref)


def test_kk_empty_and_errors(ctx):
    from paper_2005_07132_gb300 import FkkError, kk_per_spectrum
    x = torch.zeros((0, 10), device="cuda")
    ref = torch.ones(10, device="cuda")
    kk_per_spectrum(ctx, x, ref)
    y = torch.ones((4, 10), device="cuda")
    with pytest.raises(FkkError):
        kk_per_spectrum(ctx, y, ref, pad_len=12)  # not a power of two
    with pytest.raises(FkkError):
        kk_per_spectrum(ctx, y, ref, pad_len=8)  # shorter than the spectrum
    with pytest.raises(FkkError):
        kk_per_spectrum(ctx, y, ref, ratio_floor=0.0)


def test_kk_full_size_703026x1000_sampled(ctx):
    """Paper-shaped image (846 x 831 spectra, 1,000 channels) in the launch
    configuration the benchmark times; sampled rows checked against the
    oracle one by one."""
    from paper_2005_07132_gb300.synth import CONFIGS, make_cube
    from paper_2005_07132_gb300 import kk_per_spectrum
    cube = make_cube(CONFIGS["img846x831_m1000"])
    x = torch.from_numpy(cube.i_cars).cuda()
    ref = torch.from_numpy(cube.i_ref).cuda()
    im = kk_per_spectrum(ctx, x, ref)
    torch.cuda.synchronize()
    N = x.shape[0]
    rows = np.unique(np.concatenate([[0, 1, N - 2, N - 1],
                                     np.random.default_rng(0).integers(0, N, 3000)]))
    got = im[torch.from_numpy(rows).cuda()].cpu().numpy()
    _check(got, None, cube.i_cars[rows], cube.i_ref)
