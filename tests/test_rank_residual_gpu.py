"""GPU: the rank rule choosing k (Sec. 4.1) and the residual fraction that
tells whether a trained basis supports new data (Sec. 5), through the C ABI,
against the FP64 oracle.

The rule keeps singular values above s_1 max(N, M) eps (eps = the float32
epsilon of the input).  The GPU's Gram resolves singular values down to about
1e-4 s_1, so the rule is compared where its cutoff lies clear of that: on the
noiseless simulation-shaped cube (cutoff 5.4e-4 s_1 between s_3 = 3.8e-3 and
s_4 = 3.4e-5) and on a noisy cube whose noise floor (1e-2 s_1) is far above
the cutoff, so that k_max binds."""
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


def test_rank_rule_on_the_noiseless_simulation(fk, ctx):
    from paper_2005_07132_gb300.synth import make_sim_cube
    cube = make_sim_cube(0.5)
    x = torch.from_numpy(cube.i_cars).cuda()
    r = torch.from_numpy(cube.i_ref).cuda()
    basis, im, _ = fk.fkk_fit_basis(ctx, x, r, fk.fit_params(k=0))
    torch.cuda.synchronize()
    _, _, res = O.fit(cube.i_cars.astype(np.float64), cube.i_ref.astype(np.float64), O.FitParams(k=0))
    assert res["k"] == 3
    assert basis.info()["k"] == res["k"]
    assert rel_l2(im.cpu().numpy(), res["im"]) <= 1e-4
    basis.close()


def test_rank_rule_capped_by_k_max(fk, ctx):
    from paper_2005_07132_gb300.synth import CONFIGS, make_cube
    cube = make_cube(CONFIGS["img64_m512"])
    x = torch.from_numpy(cube.i_cars).cuda()
    r = torch.from_numpy(cube.i_ref).cuda()
    basis, im, _ = fk.fkk_fit_basis(ctx, x, r, fk.fit_params(k=0, k_max=24))
    torch.cuda.synchronize()
    _, _, res = O.fit(cube.i_cars.astype(np.float64), cube.i_ref.astype(np.float64), O.FitParams(k=0, k_max=24))
    assert res["k"] == 24 == basis.info()["k"]
    assert rel_l2(im.cpu().numpy(), res["im"]) <= 1e-4
    # the chosen-k basis equals a fixed-k fit bit for bit
    b2, im2, _ = fk.fkk_fit_basis(ctx, x, r, fk.fit_params(k=24))
    torch.cuda.synchronize()
    assert torch.equal(im, im2)
    for art in ("lambda", "v", "c_amp", "c_ph"):
        np.testing.assert_array_equal(basis.get(art), b2.get(art))
    basis.close()
    b2.close()


def test_rank_rule_arguments(fk, ctx):
    from paper_2005_07132_gb300.synth import CONFIGS, make_cube
    cube = make_cube(CONFIGS["img64_m512"])
    x = torch.from_numpy(cube.i_cars).cuda()
    r = torch.from_numpy(cube.i_ref).cuda()
    for kw in (dict(k=0, k_max=0), dict(k=0, k_max=81), dict(k=0, rank_eps=-1.0)):
        with pytest.raises(fk.FkkError):
            fk.fkk_fit_basis(ctx, x, r, fk.fit_params(**kw))


def test_residual_flags_data_the_basis_does_not_support(fk, ctx):
    from paper_2005_07132_gb300.synth import CONFIGS, CubeSpec, Scene, make_cube
    spec = CONFIGS["img64_m512"]
    scene = Scene.from_spec(spec)
    train = make_cube(spec, scene=scene)
    new = make_cube(spec, image=1, scene=scene)
    other = make_cube(CubeSpec(64, 64, 512, 8, "gauss", 50.0, seed=4242))
    x = torch.from_numpy(train.i_cars).cuda()
    r = torch.from_numpy(train.i_ref).cuda()
    basis, _, _ = fk.fkk_fit_basis(ctx, x, r, fk.fit_params(k=20))
    bo, _, _ = O.fit(train.i_cars.astype(np.float64), train.i_ref.astype(np.float64), O.FitParams(k=20))
    r_train = fk.fkk_residual(ctx, basis, x)
    assert abs(r_train - basis.training_residual()) < 1e-5
    assert abs(r_train - O.residual_fraction(bo, train.i_cars.astype(np.float64))) < 1e-5
    r_new = fk.fkk_residual(ctx, basis, torch.from_numpy(new.i_cars).cuda())
    r_other = fk.fkk_residual(ctx, basis, torch.from_numpy(other.i_cars).cuda())
    assert abs(r_new - O.residual_fraction(bo, new.i_cars.astype(np.float64))) < 1e-5
    assert abs(r_other - O.residual_fraction(bo, other.i_cars.astype(np.float64))) < 1e-4
    assert r_new < 1.5 * r_train        # same scene: supported
    assert r_other > 5.0 * r_train      # new species: retrain
    basis.close()
