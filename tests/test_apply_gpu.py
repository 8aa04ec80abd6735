"""GPU parity of ML:fKK-EC apply (Sec. 2.6: Eq. ML_Unew, then Eq. fKKEC on
new spectra) against the FP64 oracle, through the C ABI.

fkk_apply runs one fused launch (projection of the raw spectra on the
tensor cores, P kept on chip, reconstruction with the exp / sin epilogue)
whenever the row strides are multiples of 4 floats, the arrays 16-byte
aligned and k <= 62, and a projection kernel followed by the reconstruction
otherwise; both forms are tested here.  The fused kernel shifts the log
ratios by the basis' offset (the training mean; fkk_basis_set_offset) and
adds the shift's share back through two extra K columns.

Tolerances:
  * FKK_PREC_BF16X3 (three bf16 products per GEMM, fp32 accumulation):
    relative L2 of Im{K} <= 1e-4 (the fp32-path bound) and, per element,
    |dIm| <= 1e-4 max|Im| + 1e-4 |Im| -- the projection's split operands
    carry ~2^-16 relative error per product, the phase error that reaches
    sin() is below 1e-5 rad, and exp / sin are the SFU forms (2^-21 abs);
  * FKK_PREC_BF16 (one bf16 product in the projection, two in the
    reconstruction): relative L2 <= 1e-3, the bound the reduced-precision
    served form is held to; the measured value is printed for k = 20, 40 and
    80 (a CPU emulation of the same roundings gives 6.7e-4, 7.6e-4, 8.4e-4
    on this scene).
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


@pytest.fixture(scope="module")
def cube1():
    from paper_2005_07132_gb300.synth import CONFIGS, make_cube
    return make_cube(CONFIGS["img64_m512"])


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _oracle_basis(fk, ctx, cube, k, ml_lambda=0.0, precision=0, offset=True):
    """The oracle's basis, imported; with offset=True it also carries the
    training mean of the log ratios that fkk_fit_basis would store."""
    b_o, _, _ = O.fit(cube.i_cars, cube.i_ref, O.FitParams(k=k, ml_lambda=ml_lambda))
    prm = fk.fit_params(k=k, ml_lambda=ml_lambda, precision=precision)
    basis = fk.fkk_basis_from_arrays(ctx, prm, b_o.f, b_o.s, b_o.V, b_o.c_amp, b_o.c_ph, b_o.i_ref)
    if offset:
        basis.set_offset(O.log_ratio(cube.i_cars, cube.i_ref).mean(0))
    return b_o, basis


def _bound_ok(got, ref, abs_rel=1e-4, rel=1e-4):
    tol = abs_rel * np.abs(ref).max() + rel * np.abs(ref)
    worst = float(np.max(np.abs(got - ref) / tol))
    return worst <= 1.0, worst


@pytest.mark.parametrize("k", [20, 40, 80])
def test_apply_bf16x3_matches_oracle(fk, ctx, cube1, k):
    from paper_2005_07132_gb300.synth import make_cube
    b_o, basis = _oracle_basis(fk, ctx, cube1, k, ml_lambda=0.5)
    new = make_cube(cube1.scene.spec, image=3, height=33, width=31, scene=cube1.scene)
    re_o, im_o = O.apply(b_o, new.i_cars)
    im, re = fk.fkk_apply(ctx, basis, _dev(new.i_cars), re_out=torch.empty(new.i_cars.shape, device="cuda"))
    im, re = im.cpu().numpy(), re.cpu().numpy()
    assert rel_l2(im, im_o) <= 1e-4
    assert rel_l2(re, re_o) <= 1e-4
    ok, worst = _bound_ok(im, im_o)
    print(f"apply bf16x3 k={k}: rel-L2 {rel_l2(im, im_o):.3e}, worst element / bound {worst:.3f}")
    assert ok
    basis.close()


@pytest.mark.parametrize("k", [20, 40, 80])
def test_apply_bf16_reduced_precision(fk, ctx, cube1, k):
    """The reduced-precision served form (at k = 80 the fused kernel runs
    its P and coefficient operands in two K atoms)."""
    from paper_2005_07132_gb300.synth import make_cube
    b_o, basis = _oracle_basis(fk, ctx, cube1, k, precision=fk.PREC_BF16)
    new = make_cube(cube1.scene.spec, image=4, height=40, width=40, scene=cube1.scene)
    _, im_o = O.apply(b_o, new.i_cars)
    im = fk.fkk_apply(ctx, basis, _dev(new.i_cars)).cpu().numpy()
    err = rel_l2(im, im_o)
    print(f"apply bf16 k={k}: rel-L2(Im) = {err:.3e}")
    assert err <= 1e-3
    # the same basis switched to the fp32-accurate form
    basis.set_precision(fk.PREC_BF16X3)
    im3 = fk.fkk_apply(ctx, basis, _dev(new.i_cars)).cpu().numpy()
    assert rel_l2(im3, im_o) <= 1e-4
    basis.close()


@pytest.mark.parametrize("n,m,k,ld_pad,ldo_pad", [
    (1, 64, 8, 0, 0),        # one spectrum, one chunk
    (127, 301, 13, 3, 5),    # ragged rows and channels; strides not multiples of 4: two-kernel path
    (129, 301, 13, 4, 8),    # one spectrum past a tile; padded strides
    (130, 301, 13, 3, 3),    # strides multiples of 4 but M is not: the stride padding stays untouched
    (129, 300, 13, 4, 8),    # one spectrum past a tile; padded strides (fused path)
    (1000, 878, 40, 0, 0),
    (200, 1000, 62, 0, 0),   # the largest k of the fused kernel
    (300, 1600, 64, 0, 4),
    (257, 2048, 80, 0, 0),   # widest basis, k > 64 (two K atoms)
])
def test_apply_ragged_shapes(fk, ctx, n, m, k, ld_pad, ldo_pad):
    from paper_2005_07132_gb300.synth import CubeSpec, make_cube
    train = make_cube(CubeSpec(24, 24, m, 6, "gauss", 50.0, seed=1000 + m))
    b_o, basis = _oracle_basis(fk, ctx, train, k)
    new = make_cube(train.scene.spec, image=2, height=1, width=n, scene=train.scene)
    x = torch.zeros((n, m + ld_pad), dtype=torch.float32, device="cuda")
    x[:, :m] = _dev(new.i_cars)
    im_full = torch.full((n, m + ldo_pad), 7.0, dtype=torch.float32, device="cuda")
    im = fk.fkk_apply(ctx, basis, x[:, :m], im_out=im_full[:, :m])
    torch.cuda.synchronize()
    _, im_o = O.apply(b_o, new.i_cars)
    got = im.cpu().numpy()
    assert rel_l2(got, im_o) <= 1e-4
    ok, worst = _bound_ok(got, im_o)
    assert ok, worst
    if ldo_pad:
        assert torch.all(im_full[:, m:] == 7.0)  # stride padding never written
    basis.close()


@pytest.mark.parametrize("n,m,k", [(257, 2048, 80), (129, 1600, 63), (300, 878, 72)])
def test_apply_bf16_two_atoms_ragged(fk, ctx, n, m, k):
    """The reduced form with k > 62 (P and coefficients in two 64-wide K
    atoms, the bias columns in the second), with Re, ragged rows and padded
    output rows."""
    from paper_2005_07132_gb300.synth import CubeSpec, make_cube
    train = make_cube(CubeSpec(24, 24, m, 6, "gauss", 50.0, seed=2000 + m))
    b_o, basis = _oracle_basis(fk, ctx, train, k, precision=fk.PREC_BF16)
    new = make_cube(train.scene.spec, image=2, height=1, width=n, scene=train.scene)
    re_o, im_o = O.apply(b_o, new.i_cars)
    im_full = torch.full((n, m + 4), 7.0, dtype=torch.float32, device="cuda")
    re_full = torch.full((n, m + 4), 7.0, dtype=torch.float32, device="cuda")
    im, re = fk.fkk_apply(ctx, basis, _dev(new.i_cars), im_out=im_full[:, :m], re_out=re_full[:, :m])
    torch.cuda.synchronize()
    e_im, e_re = rel_l2(im.cpu().numpy(), im_o), rel_l2(re.cpu().numpy(), re_o)
    print(f"apply bf16 two atoms n={n} m={m} k={k}: rel-L2 Im {e_im:.3e}, Re {e_re:.3e}")
    assert e_im <= 1e-3 and e_re <= 1e-3
    assert torch.all(im_full[:, m:] == 7.0) and torch.all(re_full[:, m:] == 7.0)
    basis.close()


def test_apply_offset_changes_only_rounding(fk, ctx, cube1):
    """Any offset gives the same apply up to rounding (it is subtracted
    before the projection and added back through the reconstruction);
    a wrong-sized offset is rejected."""
    from paper_2005_07132_gb300.synth import make_cube
    b_o, basis = _oracle_basis(fk, ctx, cube1, 20, offset=False)
    new = make_cube(cube1.scene.spec, image=5, height=20, width=20, scene=cube1.scene)
    _, im_o = O.apply(b_o, new.i_cars)
    x = _dev(new.i_cars)
    im0 = fk.fkk_apply(ctx, basis, x).cpu().numpy()
    basis.set_offset(np.linspace(-1.0, 2.0, 512))
    im1 = fk.fkk_apply(ctx, basis, x).cpu().numpy()
    assert rel_l2(im0, im_o) <= 1e-4 and rel_l2(im1, im_o) <= 1e-4
    with pytest.raises(fk.FkkError):
        basis.set_offset(np.zeros(511))
    basis.close()


def test_fit_stores_training_offset(fk, ctx, cube1):
    """fkk_fit_basis stores the training mean of 1/2 ln max(I/I_ref, floor)
    as the apply offset: the reduced form of its own basis meets 1e-3."""
    from paper_2005_07132_gb300.synth import make_cube
    basis, _, _ = fk.fkk_fit_basis(ctx, _dev(cube1.i_cars), _dev(cube1.i_ref), fk.fit_params(k=40))
    new = make_cube(cube1.scene.spec, image=6, height=30, width=30, scene=cube1.scene)
    x = _dev(new.i_cars)
    ref = fk.fkk_apply(ctx, basis, x).cpu().numpy()
    basis.set_precision(fk.PREC_BF16)
    red = fk.fkk_apply(ctx, basis, x).cpu().numpy()
    err = rel_l2(red, ref)
    print(f"reduced form on a fitted basis (k=40): rel-L2 vs the fp32-accurate apply {err:.3e}")
    assert err <= 1e-3
    basis.close()


def test_apply_clamps_counted_once(fk, ctx, cube1):
    """Non-positive samples are clamped to the floor and counted; rows and
    channels of the padded tiles are not."""
    b_o, basis = _oracle_basis(fk, ctx, cube1, 20)
    x = cube1.i_cars[:200].copy()
    x[3, 10] = -1.0
    x[150, :7] = 0.0
    ctx.sync_status()
    im = fk.fkk_apply(ctx, basis, _dev(x)).cpu().numpy()
    st, clamped = ctx.sync_status()
    assert st == 0 and clamped == 8
    _, im_o = O.apply(b_o, x)
    assert rel_l2(im, im_o) <= 1e-4
    basis.close()


def test_apply_empty_and_repeatable(fk, ctx, cube1):
    b_o, basis = _oracle_basis(fk, ctx, cube1, 20)
    fk.fkk_apply(ctx, basis, torch.zeros((0, 512), device="cuda"))
    x = _dev(cube1.i_cars)
    a = fk.fkk_apply(ctx, basis, x).cpu().numpy()
    b = fk.fkk_apply(ctx, basis, x).cpu().numpy()
    assert np.array_equal(a, b)  # fixed reduction order: bit-identical reruns
    basis.close()


def test_apply_full_size_703026x1000_sampled(fk, ctx):
    """The paper-shaped image (846 x 831 spectra, 1,000 channels, k = 40) in
    the benchmark's launch configuration, on a basis the oracle trained on
    a 100 x 100 crop of the same scene; sampled rows against the oracle's
    apply, in both precisions."""
    from paper_2005_07132_gb300.synth import CONFIGS, make_cube
    cube = make_cube(CONFIGS["img846x831_m1000"])
    N = cube.i_cars.shape[0]
    train = cube.i_cars[:10000]
    mean_i = cube.i_cars[:10000].astype(np.float64).mean(0)
    f = O.noise_scale(mean_i, cube.alpha, cube.sigma_g)
    b_o, _, _ = O.fit(train, cube.i_ref, O.FitParams(k=40), f=f)
    prm = fk.fit_params(k=40)
    basis = fk.fkk_basis_from_arrays(ctx, prm, b_o.f, b_o.s, b_o.V, b_o.c_amp, b_o.c_ph, b_o.i_ref)
    basis.set_offset(O.log_ratio(train, cube.i_ref).mean(0))
    rows = np.unique(np.concatenate([[0, 1, N - 2, N - 1], np.random.default_rng(2).integers(0, N, 3000)]))
    _, im_o = O.apply(b_o, cube.i_cars[rows])
    x = _dev(cube.i_cars)
    im = fk.fkk_apply(ctx, basis, x)
    got = im[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert rel_l2(got, im_o) <= 1e-4
    ok, worst = _bound_ok(got, im_o)
    assert ok, worst
    basis.set_precision(fk.PREC_BF16)
    im = fk.fkk_apply(ctx, basis, x, im_out=im)
    got = im[torch.from_numpy(rows).cuda()].cpu().numpy()
    err = rel_l2(got, im_o)
    print(f"apply bf16 full size: rel-L2(Im) = {err:.3e}")
    assert err <= 1e-3
    basis.close()
