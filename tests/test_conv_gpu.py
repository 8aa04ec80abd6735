"""GPU parity of the conventional per-spectrum workflow (Sec. 2.1, Eq.
KCARS_from_K: KK, PEC by the ALS-detrended phase error, SEC by the trendline
of Re K) against the FP64 oracle, through the C ABI.

Tolerance: relative L2 error of Im{K_CARS} <= 1e-4 (the FP32-path bound).
The detrend runs in double-word arithmetic on an FP32 phase, the transforms
and the final exp / sin in FP32."""
import numpy as np
import pytest

import oracle as O
from gpu_util import rel_l2
from paper_2005_07132_gb300.synth import CubeSpec, make_cube

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_L2 = 1e-4


@pytest.fixture(scope="module")
def fk():
    from paper_2005_07132_gb300 import build
    build.build()
    import paper_2005_07132_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(fk):
    c = fk.Context(0)
    yield c
    c.close()


def _params(fk, **kw):
    mode = kw.pop("sec_mode", "sg")
    p = fk.fit_params(sec_mode=fk.SEC_SAVGOL if mode == "sg" else fk.SEC_MEAN, **kw)
    po = O.FitParams(pec=bool(p.pec), sec=bool(p.sec), als_lambda=(p.als_lambda or None), als_p=p.als_p,
                     als_iters=p.als_iters, sec_mode=mode, sg_window=p.sg_window, sg_order=p.sg_order,
                     pad_len=p.pad_len, ratio_floor=p.ratio_floor, denoise_k=p.denoise_k, k_max=p.k_max,
                     rank_eps=p.rank_eps)
    return p, po


def _cube(h, w, m, seed):
    c = make_cube(CubeSpec(h, w, m, 6, "gauss", 50.0, seed=seed))
    return c.i_cars, c.i_ref


def _gpu(fk, ctx, i, ref, p, re=True):
    x = torch.from_numpy(np.ascontiguousarray(i, np.float32)).cuda()
    r = torch.from_numpy(np.ascontiguousarray(ref, np.float32)).cuda()
    im = torch.full_like(x, float("nan"))
    rr = torch.full_like(x, float("nan")) if re else None
    out = fk.conventional_per_spectrum(ctx, x, r, p, im_out=im, re_out=rr)
    torch.cuda.synchronize()
    if re:
        return out[0].cpu().numpy(), out[1].cpu().numpy()
    return out.cpu().numpy(), None


@pytest.mark.parametrize("h,w,m", [(7, 11, 200), (5, 13, 512), (3, 23, 1000)])
@pytest.mark.parametrize("pec,sec,mode", [(1, 1, "sg"), (1, 1, "mean"), (1, 0, "sg"), (0, 1, "sg")])
def test_conventional_matches_oracle(fk, ctx, h, w, m, pec, sec, mode):
    i, ref = _cube(h, w, m, seed=31 + m)
    p, po = _params(fk, pec=pec, sec=sec, sec_mode=mode)
    im, re = _gpu(fk, ctx, i, ref, p)
    re_o, im_o = O.conventional(i.astype(np.float64), ref.astype(np.float64), po)
    assert np.all(np.isfinite(im)) and np.all(np.isfinite(re))
    assert rel_l2(im, im_o) <= RTOL_L2
    assert rel_l2(re, re_o) <= RTOL_L2


@pytest.mark.parametrize("order,window", [(0, 31), (1, 45), (2, 101), (2, 199)])
def test_conventional_trendline_orders(fk, ctx, order, window):
    i, ref = _cube(4, 9, 200, seed=5)
    p, po = _params(fk, sg_order=order, sg_window=window)
    im, _ = _gpu(fk, ctx, i, ref, p, re=False)
    _, im_o = O.conventional(i.astype(np.float64), ref.astype(np.float64), po)
    assert rel_l2(im, im_o) <= RTOL_L2


def test_conventional_als_settings(fk, ctx):
    i, ref = _cube(6, 6, 300, seed=9)
    for lam, pp, iters in [(50.0, 0.05, 5), (3e4, 0.001, 30), (1.0, 0.5, 1)]:
        p, po = _params(fk, als_lambda=lam, als_p=pp, als_iters=iters)
        im, _ = _gpu(fk, ctx, i, ref, p, re=False)
        _, im_o = O.conventional(i.astype(np.float64), ref.astype(np.float64), po)
        assert rel_l2(im, im_o) <= RTOL_L2, (lam, pp, iters)


def test_conventional_without_pec_sec_equals_kk_bitwise(fk, ctx):
    """PEC and SEC off: the same float operations as kk_per_spectrum."""
    i, ref = _cube(9, 9, 512, seed=2)
    p, _ = _params(fk, pec=0, sec=0)
    im, re = _gpu(fk, ctx, i, ref, p)
    x = torch.from_numpy(i).cuda()
    r = torch.from_numpy(ref).cuda()
    im_k, re_k = fk.kk_per_spectrum(ctx, x, r, im_out=torch.empty_like(x), re_out=torch.empty_like(x))
    torch.cuda.synchronize()
    assert np.array_equal(im, im_k.cpu().numpy())
    assert np.array_equal(re, re_k.cpu().numpy())


def test_conventional_chunks_do_not_change_results(fk, ctx):
    """A budget that forces chunks of a few dozen spectra gives bit-identical
    output (spectra are independent; the ragged last chunk included)."""
    i, ref = _cube(11, 17, 256, seed=4)  # 187 spectra
    p, _ = _params(fk)
    im1, re1 = _gpu(fk, ctx, i, ref, p)
    small = fk.Context(0, hbm_budget_bytes=600_000)
    try:
        im2, re2 = _gpu(fk, small, i, ref, p)
    finally:
        small.close()
    assert np.array_equal(im1, im2)
    assert np.array_equal(re1, re2)


def test_conventional_strided_rows(fk, ctx):
    i, ref = _cube(3, 9, 200, seed=12)
    n, m = i.shape
    p, po = _params(fk)
    buf = torch.zeros((n, m + 24), dtype=torch.float32, device="cuda")
    buf[:, :m] = torch.from_numpy(i)
    out = torch.full((n, m + 40), 7.0, device="cuda")
    r = torch.from_numpy(ref).cuda()
    fk.conventional_per_spectrum(ctx, buf[:, :m], r, p, im_out=out[:, :m])
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert np.all(o[:, m:] == 7.0)
    _, im_o = O.conventional(i.astype(np.float64), ref.astype(np.float64), po)
    assert rel_l2(o[:, :m], im_o) <= RTOL_L2


def test_conventional_rejects_bad_arguments(fk, ctx):
    i, ref = _cube(2, 4, 64, seed=1)
    x = torch.from_numpy(i).cuda()
    r = torch.from_numpy(ref).cuda()
    for kw in [dict(sg_order=3, sg_window=31), dict(sg_window=30), dict(pad_len=100), dict(als_p=1.5)]:
        p, _ = _params(fk, **kw)
        with pytest.raises(fk.FkkError):
            fk.conventional_per_spectrum(ctx, x, r, p)
    p, _ = _params(fk)
    with pytest.raises(fk.FkkError):
        fk.conventional_per_spectrum(ctx, x[:, :7].contiguous(), r[:7].contiguous(), p)
    # zero spectra is a no-op
    fk.conventional_per_spectrum(ctx, x[:0], r, p, im_out=torch.empty((0, 64), device="cuda"))


def test_conventional_full_size_sampled_rows(fk, ctx):
    """The 846 x 831 x 1,000 cube (the benchmark workload) in one call, checked
    on sampled spectra the oracle computes one by one."""
    from paper_2005_07132_gb300.synth import CONFIGS
    cube = make_cube(CONFIGS["img846x831_m1000"])
    x = torch.from_numpy(cube.i_cars).cuda()
    r = torch.from_numpy(cube.i_ref).cuda()
    p, po = _params(fk)
    im = fk.conventional_per_spectrum(ctx, x, r, p)
    torch.cuda.synchronize()
    n = x.shape[0]
    rows = np.unique(np.concatenate([[0, 1, n - 2, n - 1], np.random.default_rng(3).integers(0, n, 12)]))
    got = im[torch.from_numpy(rows).cuda()].cpu().numpy()
    _, want = O.conventional(cube.i_cars[rows].astype(np.float64), cube.i_ref.astype(np.float64), po)
    assert np.all(np.isfinite(got))
    assert rel_l2(got, want) <= RTOL_L2


# ---------------------------------------------------------------------------
# The workflow's SVD denoising of the raw spectra (Fig. 1(a)): k is chosen
# where the singular values have a clear gap (s_5 / s_6 = 2.2 and 3.0 on the
# two cubes), so the kept subspace is well determined.
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("h,w,m,seed,k,pec", [(32, 40, 256, 3, 5, True), (48, 48, 200, 5, 5, False),
                                              (48, 48, 200, 5, 1, False)])
def test_conventional_denoise_matches_oracle(fk, ctx, h, w, m, seed, k, pec):
    i, ref = _cube(h, w, m, seed)
    p, po = _params(fk, denoise_k=k, pec=int(pec), sec=int(pec))
    im, re = _gpu(fk, ctx, i, ref, p)
    re_o, im_o = O.conventional(i.astype(np.float64), ref.astype(np.float64), po)
    assert rel_l2(im, im_o) <= RTOL_L2
    assert rel_l2(re, re_o) <= RTOL_L2
    assert ctx.sync_status()[0] == 0


def test_conventional_denoise_rank_rule_on_the_simulation(fk, ctx):
    """The noiseless simulation-shaped cube: the rank rule keeps 3 singular
    vectors of the raw spectra (s_3 = 3.3e-3 s_1 above the cutoff 5.4e-4 s_1,
    s_4 = 2.2e-5 s_1 below it)."""
    from paper_2005_07132_gb300.synth import make_sim_cube
    cube = make_sim_cube(0.5)
    i = cube.i_cars.astype(np.float64)
    assert O.svd_denoise(i, -1)[1] == 3
    p, po = _params(fk, denoise_k=-1, pec=0, sec=1, sec_mode="mean")
    im, re = _gpu(fk, ctx, cube.i_cars, cube.i_ref, p)
    re_o, im_o = O.conventional(i, cube.i_ref.astype(np.float64), po)
    assert rel_l2(im, im_o) <= RTOL_L2
    assert rel_l2(re, re_o) <= RTOL_L2


def test_conventional_full_rank_denoise_changes_nothing(fk, ctx):
    """k = M keeps every singular vector: X V V^T = X up to rounding."""
    i, ref = _cube(16, 16, 64, 7)
    p0, _ = _params(fk)
    p1, _ = _params(fk, denoise_k=64)
    im0, _ = _gpu(fk, ctx, i, ref, p0, re=False)
    im1, _ = _gpu(fk, ctx, i, ref, p1, re=False)
    assert rel_l2(im1, im0) <= 1e-5


def test_conventional_denoise_rejects_bad_arguments(fk, ctx):
    i, ref = _cube(16, 16, 64, 7)
    for kw in (dict(denoise_k=81), dict(denoise_k=65), dict(denoise_k=-1, k_max=0), dict(denoise_k=-1, k_max=81),
               dict(denoise_k=-1, rank_eps=-1.0)):
        p, _ = _params(fk, **kw)
        with pytest.raises(fk.FkkError):
            _gpu(fk, ctx, i, ref, p, re=False)
