"""GPU: the randomised SVD (Sec. 5; Halko, Martinsson & Tropp 2011) through
the C ABI against the FP64 oracle running the same algorithm on the same
Philox4x64-10 test matrix.

The generator's doubles agree to the last bits (the same integer stream,
Box-Muller in fp64).  The fitted subspace is a random sketch refined by
power iterations, so the comparison is with the oracle's randomised fit, not
the exact one; tolerance rel-L2(Im) <= 1e-4 as for the exact path."""
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


@pytest.mark.parametrize("seed", [0, 7, 2**64 - 3])
def test_philox_normals_match_oracle(fk, ctx, seed):
    got = fk.fkk_philox_normals(ctx, 1001, seed).cpu().numpy()
    np.testing.assert_allclose(got, O.philox_normals(1001, seed), rtol=1e-14, atol=1e-14)


def _fit_pair(fk, ctx, cube_i, cube_ref, **kw):
    x = torch.from_numpy(cube_i).cuda()
    r = torch.from_numpy(cube_ref).cuda()
    basis, im, _ = fk.fkk_fit_basis(ctx, x, r, fk.fit_params(svd=fk.SVD_RANDOMIZED, **kw))
    torch.cuda.synchronize()
    st, _ = ctx.sync_status()
    po = O.FitParams(svd="randomized", k=kw["k"], rsvd_oversample=kw.get("rsvd_oversample", 10),
                     rsvd_power_iters=kw.get("rsvd_power_iters", 2), rsvd_seed=kw.get("rsvd_seed", 0))
    bo, _, res = O.fit(cube_i.astype(np.float64), cube_ref.astype(np.float64), po)
    return basis, im.cpu().numpy(), st, bo, res


@pytest.mark.parametrize("k,p,q", [(20, 10, 2), (8, 8, 0), (40, 10, 1)])
def test_rsvd_fit_matches_oracle(fk, ctx, k, p, q):
    from paper_2005_07132_gb300.synth import CONFIGS, make_cube
    cube = make_cube(CONFIGS["img64_m512"])
    basis, im, st, bo, res = _fit_pair(fk, ctx, cube.i_cars, cube.i_ref, k=k, rsvd_oversample=p,
                                       rsvd_power_iters=q, rsvd_seed=11)
    assert st == 0
    lam = basis.get("lambda")
    np.testing.assert_allclose(lam, res["lam"], rtol=0, atol=1e-6 * res["lam"][0])
    V = basis.get("v")
    dots = np.abs(np.sum(V * bo.V, 0))
    assert np.all(dots > 1 - 1e-6), dots.min()
    assert rel_l2(im, res["im"]) <= 1e-4
    # the training residual uses the transform's sum of squares here
    assert abs(basis.training_residual() - (1 - res["lam"].sum() / bo.extras["energy"])) < 1e-6
    basis.close()


def test_rsvd_fit_on_the_simulation(fk, ctx):
    from paper_2005_07132_gb300.synth import make_sim_cube
    cube = make_sim_cube(0.5)
    basis, im, st, bo, res = _fit_pair(fk, ctx, cube.i_cars, cube.i_ref, k=3, rsvd_seed=5)
    assert st == 0
    assert rel_l2(im, res["im"]) <= 1e-4
    np.testing.assert_array_equal(np.sort(basis.get("q").astype(np.int64)), np.sort(res["q"]))
    basis.close()


def test_rsvd_arguments(fk, ctx):
    from paper_2005_07132_gb300.synth import CONFIGS, make_cube
    cube = make_cube(CONFIGS["img64_m512"])
    x = torch.from_numpy(cube.i_cars).cuda()
    r = torch.from_numpy(cube.i_ref).cuda()
    for kw in (dict(k=0), dict(k=75, rsvd_oversample=10), dict(k=10, rsvd_power_iters=21),
               dict(k=10, rsvd_oversample=-1), dict(k=10, svd=5)):
        kw.setdefault("svd", fk.SVD_RANDOMIZED)
        with pytest.raises(fk.FkkError):
            fk.fkk_fit_basis(ctx, x, r, fk.fit_params(**kw))


@pytest.mark.slow
def test_rsvd_full_size_sampled(fk, ctx):
    """The 846 x 831 x 1,000 cube (k = 40, the benchmark's configuration
    with the randomised SVD), sampled rows against the oracle's randomised
    fit of the whole cube."""
    from paper_2005_07132_gb300.synth import CONFIGS, make_cube
    cube = make_cube(CONFIGS["img846x831_m1000"])
    N = cube.i_cars.shape[0]
    rows = np.unique(np.concatenate([[0, N - 1], np.random.default_rng(2).integers(0, N, 1000)]))
    f = O.noise_scale(cube.i_cars.astype(np.float64).mean(0), cube.alpha, cube.sigma_g)
    po = O.FitParams(k=40, svd="randomized")
    b_o, _, res = O.fit(cube.i_cars, cube.i_ref, po, f=f, out_rows=rows)
    x = torch.from_numpy(cube.i_cars).cuda()
    r = torch.from_numpy(cube.i_ref).cuda()
    basis, im, _ = fk.fkk_fit_basis(ctx, x, r, fk.fit_params(k=40, svd=fk.SVD_RANDOMIZED, noise_alpha=cube.alpha,
                                                               noise_sigma_g=cube.sigma_g))
    st, _ = ctx.sync_status()
    assert st == 0
    got = im[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert rel_l2(got, res["im"]) <= 1e-4
    basis.close()
