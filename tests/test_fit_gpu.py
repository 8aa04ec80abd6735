"""GPU parity of the fKK-EC fit pipeline (Secs. 2.2-2.6) against the FP64
oracle, step by step (each CUDA step fed the oracle's inputs) and end to
end, through the C ABI.

Tolerances and where they come from:
  * Gram: each product of the centred log ratios d is formed from two bf16
    terms per factor (three products), relative error <= 3 * 2^-17 of
    |d_i d_j|, fp32 accumulation in TMEM and fp64 across splits; centring
    makes |d| ~30x smaller than |a|, so |dG| <= 2e-6 max|G|.
  * eigenpairs: Householder tridiagonalisation, Sturm multisection and
    twisted-factorisation eigenvectors in double-word (about 48-bit)
    arithmetic, back-transformed and orthonormalised; eigenvalues to
    1e-12 lambda_1, ||V^T V - I|| <= 1e-12, ||G V - V L|| <= 1e-12 ||G||.
  * projection: fp32 accumulation of bf16-pair inputs, |dP| <= 5e-6 max|P|;
    argmax / argmin rows equal to the oracle's wherever the oracle's margin
    between the two largest (smallest) values exceeds that bound.
  * basis math: fp64 on both sides; rel <= 1e-9.
  * reconstruction / end to end: relative L2 of Im{K} <= 1e-4 (the FP32-path
    bound); the sub-sampled rows q must be identical end to end; and per
    element |dIm| <= 2e-4 max|Im| + 1e-4 |Im| (PER_ELEM), so that an error
    concentrated in a few channels cannot hide inside the norm: a relative
    perturbation of the Gram matrix moves the output by about 500 times as
    much at k = 40 (the noise-floor singular values at the cut are 4e-5 to
    1e-3 apart, relatively), and the Gram's own error is about 1e-7.
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import elementwise_ratio, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


PER_ELEM = (2e-4, 1e-4)


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


def _dev(a, dtype=None):
    a = np.ascontiguousarray(a if dtype is None else np.asarray(a, dtype))
    return torch.from_numpy(a).cuda()


def test_gram_matches_oracle(fk, ctx, cube1):
    A = O.log_ratio(cube1.i_cars, cube1.i_ref)
    G_o = A.T @ A
    G = fk.fkk_gram(ctx, _dev(cube1.i_cars), _dev(cube1.i_ref)).cpu().numpy()
    assert np.abs(G - G_o).max() <= 2e-6 * np.abs(G_o).max()
    np.testing.assert_allclose(G, G.T, rtol=0, atol=0)


@pytest.mark.parametrize("n,m", [(1000, 37), (777, 300), (130, 878)])
def test_gram_ragged_with_f(fk, ctx, n, m):
    r = np.random.default_rng(n + m)
    i_ref = r.uniform(0.5, 2.0, m).astype(np.float32)
    i = (i_ref * np.exp(2 * (0.3 * r.standard_normal((n, m)) + 0.1))).astype(np.float32)
    f = r.uniform(0.5, 2.0, m)
    A = O.log_ratio(i, i_ref, f)
    G_o = A.T @ A
    G = fk.fkk_gram(ctx, _dev(i), _dev(i_ref), f=_dev(f)).cpu().numpy()
    # per-element bound of the three-product bf16 split (without the gain of
    # centring, which random data does not give): 2^-15 sum_n |a_ni a_nj|
    bound = 2.0**-15 * (np.abs(A).T @ np.abs(A))
    assert np.all(np.abs(G - G_o) <= bound)


def test_eig_matches_oracle(fk, ctx, cube1):
    A = O.log_ratio(cube1.i_cars, cube1.i_ref)
    G_o = A.T @ A
    k = 20
    lam_o, V_o = O.eig_desc(G_o)
    lam, V = fk.fkk_eig_topk(ctx, _dev(G_o), k)
    st, _ = ctx.sync_status()
    assert st == 0
    lam = lam.cpu().numpy()
    V = V.cpu().numpy()
    assert np.abs(lam - lam_o[:k]).max() <= 1e-8 * lam_o[0]
    assert np.abs(V.T @ V - np.eye(k)).max() <= 1e-10
    assert np.linalg.norm(G_o @ V - V * lam) <= 1e-6 * np.linalg.norm(G_o)
    # well-separated eigenvalues: the vectors themselves (sign fixed by the
    # largest-magnitude component, as in the oracle)
    gaps = np.minimum(np.abs(np.diff(lam_o[: k + 1]))[:k], np.abs(np.diff(np.r_[np.inf, lam_o[:k]]))[:k])
    sep = gaps > 1e-3 * lam_o[0]
    assert sep.sum() >= 3
    np.testing.assert_allclose((V * V_o[:, :k]).sum(0)[sep], 1.0, atol=1e-6)


def test_eig_known_spectrum(fk, ctx):
    r = np.random.default_rng(3)
    m, k = 200, 12
    Q, _ = np.linalg.qr(r.standard_normal((m, m)))
    lam = np.sort(r.uniform(0.1, 1.0, m))[::-1] * np.geomspace(1e3, 1.0, m)
    G = (Q * lam) @ Q.T
    lg, V = fk.fkk_eig_topk(ctx, _dev(G), k)
    lg = lg.cpu().numpy()
    V = V.cpu().numpy()
    np.testing.assert_allclose(lg, lam[:k], rtol=1e-9)
    np.testing.assert_allclose(np.abs((V * Q[:, :k]).sum(0)), 1.0, atol=1e-8)


def _eig_check(fk, ctx, G, k, lam_tol=1e-12, res_tol=1e-12):
    lam, V = fk.fkk_eig_topk(ctx, _dev(G), k)
    st, _ = ctx.sync_status()
    assert st == 0
    lam = lam.cpu().numpy()
    V = V.cpu().numpy()
    w = np.linalg.eigvalsh(G)[::-1]
    assert np.abs(lam - w[:k]).max() <= lam_tol * abs(w[0])
    assert np.abs(V.T @ V - np.eye(k)).max() <= 1e-12
    assert np.linalg.norm(G @ V - V * lam) <= res_tol * np.linalg.norm(G)
    big = np.abs(V).argmax(0)
    assert np.all(V[big, np.arange(k)] > 0)
    return lam, V


@pytest.mark.parametrize("m", [2, 3, 33])
def test_eig_small(fk, ctx, m):
    B = np.random.default_rng(m).standard_normal((50, m))
    _eig_check(fk, ctx, B.T @ B, min(m, 3))


def test_eig_split_with_equal_eigenvalues(fk, ctx):
    """Two identical diagonal blocks: the tridiagonal form splits and every
    eigenvalue is double; the two vectors of each pair must be orthogonal."""
    B = np.random.default_rng(5).standard_normal((300, 60))
    G = np.zeros((120, 120))
    G[:60, :60] = B.T @ B
    G[60:, 60:] = B.T @ B
    _eig_check(fk, ctx, G, 10)


@pytest.mark.parametrize("m", [512, 2048])
def test_eig_dominant_rank_one(fk, ctx, m):
    """Gram of log-ratio-like data: one eigenvalue ~2e5 times the noise
    floor, noise eigenvalues a fraction of a percent apart; m = 2048 keeps
    the working columns in global memory instead of shared memory."""
    r = np.random.default_rng(m)
    A = (1.0 + 0.3 * np.sin(np.arange(m) / 37.0)[None, :] * r.standard_normal((20000, 1))
         + 0.05 * r.standard_normal((20000, m)))
    _eig_check(fk, ctx, A.T @ A, 80 if m == 2048 else 40)


def test_project_and_argext(fk, ctx, cube1):
    A = O.log_ratio(cube1.i_cars, cube1.i_ref)
    _, V_o = O.eig_desc(A.T @ A)
    Vk = np.ascontiguousarray(V_o[:, :20])
    P_o = A @ Vk
    P, qmax, qmin = fk.fkk_project(ctx, _dev(cube1.i_cars), _dev(cube1.i_ref), _dev(Vk))
    P = P.cpu().numpy()
    tol = 5e-6 * np.abs(P_o).max()
    assert np.abs(P - P_o).max() <= tol
    qmax, qmin = qmax.cpu().numpy(), qmin.cpu().numpy()
    for i in range(Vk.shape[1]):
        col = P_o[:, i]
        srt = np.sort(col)
        if srt[-1] - srt[-2] > 2 * tol:
            assert qmax[i] == np.argmax(col)
        else:
            assert col[qmax[i]] >= srt[-1] - 2 * tol
        if srt[1] - srt[0] > 2 * tol:
            assert qmin[i] == np.argmin(col)
        else:
            assert col[qmin[i]] <= srt[0] + 2 * tol


@pytest.mark.parametrize("pec,sec_mode", [(1, 0), (1, 1), (0, 0), (0, 1)])
def test_basis_math(fk, ctx, cube1, pec, sec_mode):
    M = cube1.i_cars.shape[1]
    A = O.log_ratio(cube1.i_cars, cube1.i_ref)
    _, V_o = O.eig_desc(A.T @ A)
    k = 20
    Vk = np.ascontiguousarray(V_o[:, :k])
    P_o = A @ Vk
    f = np.random.default_rng(1).uniform(0.8, 1.2, M)
    prm = O.FitParams(k=k, pec=bool(pec), sec_mode=["sg", "mean"][sec_mode])
    out = O.basis_math(Vk, P_o, f, prm, O.pad_len(M))
    q = out[7]
    x_rows = _dev(P_o[q]) if pec else None
    ca, cp = fk.fkk_basis_math(ctx, _dev(Vk), fk.fit_params(k=k, pec=pec, sec_mode=sec_mode), x_rows=x_rows,
                               f=_dev(f))
    assert rel_l2(ca.cpu().numpy(), out[5]) <= 1e-9
    assert rel_l2(cp.cpu().numpy(), out[6]) <= 1e-9


@pytest.mark.parametrize("n,k,m,ld_pad", [(1000, 80, 300, 0), (129, 13, 877, 3), (131, 20, 300, 4), (5000, 64, 512, 0), (1, 1, 8, 0)])
def test_reconstruct_shapes(fk, ctx, n, k, m, ld_pad):
    """Tensor-core reconstruction: K padded to 64 / 128, ragged rows and
    channels, row stride above M, Im and Re."""
    r = np.random.default_rng(n + k + m)
    P = (r.standard_normal((n, k)) * 0.05).astype(np.float32)
    ca = r.standard_normal((k, m)) * 0.5
    cp = r.standard_normal((k, m)) * 0.5
    re_o, im_o = O.reconstruct(P.astype(np.float64), ca, cp)
    ld = m + ld_pad
    im_buf = torch.full((n, ld), 9.0, device="cuda")
    re_buf = torch.full((n, ld), 9.0, device="cuda")
    fk.fkk_reconstruct(ctx, _dev(P), _dev(ca), _dev(cp), im_out=im_buf[:, :m], re_out=re_buf[:, :m])
    im = im_buf.cpu().numpy()
    re = re_buf.cpu().numpy()
    assert rel_l2(im[:, :m], im_o) <= 1e-5
    assert rel_l2(re[:, :m], re_o) <= 1e-5
    assert np.all(im[:, m:] == 9.0) and np.all(re[:, m:] == 9.0)


def test_reconstruct(fk, ctx, cube1):
    A = O.log_ratio(cube1.i_cars, cube1.i_ref)
    b, P_o, _ = O.fit(cube1.i_cars, cube1.i_ref, O.FitParams(k=20))
    re_o, im_o = O.reconstruct(P_o, b.c_amp, b.c_ph)
    im, re = fk.fkk_reconstruct(ctx, _dev(P_o, np.float32), _dev(b.c_amp), _dev(b.c_ph),
                                re_out=torch.empty(P_o.shape[0], A.shape[1], device="cuda"))
    assert rel_l2(im.cpu().numpy(), im_o) <= 1e-5
    assert rel_l2(re.cpu().numpy(), re_o) <= 1e-5


@pytest.mark.parametrize("pec,sec", [(0, 0), (1, 1)])
def test_fit_end_to_end_img64(fk, ctx, cube1, pec, sec):
    k = 20
    b_o, _, res = O.fit(cube1.i_cars, cube1.i_ref, O.FitParams(k=k, pec=bool(pec), sec=bool(sec)))
    basis, im, _ = fk.fkk_fit_basis(ctx, _dev(cube1.i_cars), _dev(cube1.i_ref), fk.fit_params(k=k, pec=pec, sec=sec))
    st, _ = ctx.sync_status()
    assert st == 0
    assert rel_l2(im.cpu().numpy(), res["im"]) <= 1e-4
    assert elementwise_ratio(im.cpu().numpy(), res["im"], *PER_ELEM) <= 1.0
    if pec:
        np.testing.assert_array_equal(basis.get("q").astype(np.int64), res["q"])
    # the dominant singular value is unique; noise-floor ones move with the
    # Gram's rounding and are checked through the output instead
    np.testing.assert_allclose(basis.get("s")[0], b_o.s[0], rtol=1e-6)
    basis.close()


@pytest.mark.parametrize("k", [20, 40, 80])
def test_fit_precision_by_k(fk, ctx, cube1, k):
    """rel-L2 of Im{K} against the fp64 oracle with PEC and SEC on, at
    k = 20, 40 and 80 (the bound of the fp32-accurate path is 1e-4)."""
    _, _, res = O.fit(cube1.i_cars, cube1.i_ref, O.FitParams(k=k))
    basis, im, _ = fk.fkk_fit_basis(ctx, _dev(cube1.i_cars), _dev(cube1.i_ref), fk.fit_params(k=k))
    st, _ = ctx.sync_status()
    assert st == 0
    err = rel_l2(im.cpu().numpy(), res["im"])
    worst = elementwise_ratio(im.cpu().numpy(), res["im"], *PER_ELEM)
    print(f"precision k={k}: rel-L2(Im) = {err:.3e}, worst element / bound {worst:.3f}")
    assert err <= 1e-4 and worst <= 1.0
    basis.close()


def test_fit_ragged_poisson_f(fk, ctx):
    """Odd channel count, N not a multiple of 64, k not a multiple of 8, and
    f(w) from the Poisson-Gaussian noise model (Sec. 2.2)."""
    from paper_2005_07132_gb300.synth import CubeSpec, make_cube
    cube = make_cube(CubeSpec(37, 41, 301, 6, "poisson_gauss", 30.0, seed=77))
    k = 13
    mean_i = cube.i_cars.astype(np.float64).mean(0)
    f = O.noise_scale(mean_i, cube.alpha, cube.sigma_g)
    b_o, _, res = O.fit(cube.i_cars, cube.i_ref, O.FitParams(k=k), f=f)
    basis, im, _ = fk.fkk_fit_basis(ctx, _dev(cube.i_cars), _dev(cube.i_ref),
                                    fk.fit_params(k=k, noise_alpha=cube.alpha, noise_sigma_g=cube.sigma_g))
    np.testing.assert_allclose(basis.get("f"), f, rtol=1e-6)
    assert rel_l2(im.cpu().numpy(), res["im"]) <= 1e-4
    np.testing.assert_array_equal(basis.get("q").astype(np.int64), res["q"])


def test_apply_with_oracle_basis(fk, ctx, cube1):
    """ML:fKK-EC (Eq. ML_Unew) on new spectra with the oracle's basis."""
    from paper_2005_07132_gb300.synth import make_cube
    k = 20
    b_o, _, _ = O.fit(cube1.i_cars, cube1.i_ref, O.FitParams(k=k, ml_lambda=0.5))
    new = make_cube(cube1.scene.spec, image=3, height=33, width=31, scene=cube1.scene)
    re_o, im_o = O.apply(b_o, new.i_cars)
    prm = fk.fit_params(k=k, ml_lambda=0.5)
    basis = fk.fkk_basis_from_arrays(ctx, prm, b_o.f, b_o.s, b_o.V, b_o.c_amp, b_o.c_ph, b_o.i_ref)
    im = fk.fkk_apply(ctx, basis, _dev(new.i_cars))
    assert rel_l2(im.cpu().numpy(), im_o) <= 1e-4
    assert elementwise_ratio(im.cpu().numpy(), im_o, *PER_ELEM) <= 1.0


def test_apply_on_training_equals_fit(fk, ctx, cube1):
    basis, im, _ = fk.fkk_fit_basis(ctx, _dev(cube1.i_cars), _dev(cube1.i_ref), fk.fit_params(k=20))
    im2 = fk.fkk_apply(ctx, basis, _dev(cube1.i_cars))
    assert rel_l2(im2.cpu().numpy(), im.cpu().numpy()) <= 1e-5


def test_fit_errors(fk, ctx, cube1):
    x = _dev(cube1.i_cars)
    ref = _dev(cube1.i_ref)
    for bad in (dict(k=0, k_max=0), dict(k=81), dict(als_p=1.5), dict(ratio_floor=0.0), dict(sg_window=4),
                dict(pad_len=100)):
        with pytest.raises(fk.FkkError):
            fk.fkk_fit_basis(ctx, x, ref, fk.fit_params(**bad))


@pytest.mark.slow
def test_fit_full_size_703026x1000_sampled(fk, ctx):
    """Paper-shaped image (846 x 831 spectra, 1,000 channels, k = 40, Poisson +
    Gaussian noise, PEC and SEC on) in the configuration the benchmark
    times: the oracle fits the whole cube in fp64; sampled output rows are
    compared."""
    from paper_2005_07132_gb300.synth import CONFIGS, make_cube
    cube = make_cube(CONFIGS["img846x831_m1000"])
    N = cube.i_cars.shape[0]
    rows = np.unique(np.concatenate([[0, N - 1], np.random.default_rng(1).integers(0, N, 2000)]))
    mean_i = cube.i_cars.astype(np.float64).mean(0)
    f = O.noise_scale(mean_i, cube.alpha, cube.sigma_g)
    b_o, _, res = O.fit(cube.i_cars, cube.i_ref, O.FitParams(k=40), f=f, out_rows=rows)
    basis, im, _ = fk.fkk_fit_basis(ctx, _dev(cube.i_cars), _dev(cube.i_ref),
                                    fk.fit_params(k=40, noise_alpha=cube.alpha, noise_sigma_g=cube.sigma_g))
    st, _ = ctx.sync_status()
    assert st == 0
    got = im[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert rel_l2(got, res["im"]) <= 1e-4
    worst = elementwise_ratio(got, res["im"], *PER_ELEM)
    print(f"full size: worst element / bound {worst:.3f}")
    assert worst <= 1.0
    np.testing.assert_array_equal(basis.get("q").astype(np.int64), res["q"])


def test_fit_with_host_buffers(fk, ctx, cube1):
    """Host inputs and outputs (pinned and pageable, a strided cube) go
    through the same kernels: the output equals the device-buffer fit's bit
    for bit."""
    x = torch.from_numpy(np.ascontiguousarray(cube1.i_cars))
    r = torch.from_numpy(np.ascontiguousarray(cube1.i_ref))
    prm = fk.fit_params(k=20)
    b0, im0, _ = fk.fkk_fit_basis(ctx, x.cuda(), r.cuda(), prm)
    torch.cuda.synchronize()
    ref = im0.cpu()
    n, m = x.shape
    padded = torch.zeros((n, m + 3), dtype=torch.float32)
    padded[:, :m] = x
    for xh, rh, pin in ((x.pin_memory(), r.pin_memory(), True), (x.clone(), r.clone(), False),
                        (padded[:, :m], r.clone(), False)):
        oh = torch.full((n, m), float("nan"))
        if pin:
            oh = oh.pin_memory()
        b1, im1, _ = fk.fkk_fit_basis(ctx, xh, rh, prm, im_out=oh)
        torch.cuda.synchronize()
        assert torch.equal(im1, ref)
        b1.close()
    with pytest.raises(fk.FkkError):
        fk.fkk_fit_basis(ctx, x.cuda(), r.cuda(), prm, im_out=torch.empty((n, m)),
                         re_out=torch.empty((n, m), device="cuda"))
    b0.close()
