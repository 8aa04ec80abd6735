"""GPU tests of the batched multi-image workload: 16 independent cubes, each
its own scene (species, NRB, surrogate), with sides, channel counts
(512 / 878 / 1,000 / 1,600) and k (10 / 20 / 40 / 80) drawn by a seeded
stream, fitted end to end (Gram, eigensolve, fKK / fPEC / fSEC on the basis,
reconstruction; Fig. 1(b) on each image) by one fkk_fit_many call.

  * parity: every cube at 64 x 64 spectra (its own M and k) against the fp64
    oracle's fit -- rel-L2 of Im{K} <= 1e-4 and the same sub-sampled rows.
    The sub-sample q (argmax / argmin rows of each column of P = U S) can
    hinge on a near-degenerate pair of eigenvectors inside the kept set: a
    rotation within the pair moves the extremes.  A cube whose q, in fp64,
    changes when G is perturbed by random symmetric matrices of 1e-8 max|G|
    (three fixed draws) is not determined at the precision of an
    fp32-accurate Gram matrix (its error is ~1e-7 of ||G||); for such a cube
    (found from the oracle alone: two of this draw's sixteen) the output
    depends on the choice and is compared with PEC off, where it is unique;
  * at the workload's sizes (128^2 .. 1,024^2 spectra, tiled from a 128 x 128
    draw of each scene): every cube's output and basis equal those of
    fkk_fit_basis on that cube alone, bit for bit.
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import rel_l2
from paper_2005_07132_gb300.synth import CubeSpec, make_cube, make_tiled_cube, multi_image_specs

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


def _q_stable(cube, k, eps=1e-8, draws=3):
    """Whether the fp64 sub-sample q survives random symmetric perturbations
    of G = A^T A of eps max|G|."""
    A = O.log_ratio(cube.i_cars, cube.i_ref)
    G = A.T @ A

    def q_of(Gm):
        V = np.linalg.eigh(Gm)[1][:, ::-1][:, :k]
        P = A @ V
        return np.unique(np.concatenate([P.argmax(0), P.argmin(0)]))

    q0 = q_of(G)
    r = np.random.default_rng(1)
    for _ in range(draws):
        E = r.standard_normal(G.shape)
        E = (E + E.T) / 2
        if not np.array_equal(q_of(G + eps * np.abs(G).max() * E / np.abs(E).max()), q0):
            return False
    return True


def test_multi_image_parity_small(fk, ctx):
    jobs, cubes = [], []
    for spec, k in multi_image_specs():
        small = CubeSpec(64, 64, spec.n_channels, spec.n_species, spec.noise, spec.snr, seed=spec.seed)
        cube = make_cube(small)
        x = torch.from_numpy(cube.i_cars).cuda()
        ref = torch.from_numpy(cube.i_ref).cuda()
        jobs.append((x, ref, fk.fit_params(k=k), torch.empty_like(x)))
        cubes.append((cube, k))
    bases = fk.fkk_fit_many(ctx, jobs)
    torch.cuda.synchronize()
    st, _ = ctx.sync_status()
    assert st == 0
    degenerate = 0
    for (cube, k), (x, ref, prm, out), b in zip(cubes, jobs, bases):
        _, _, res = O.fit(cube.i_cars, cube.i_ref, O.FitParams(k=k))
        assert b.info()["k"] == k
        if _q_stable(cube, k):
            err = rel_l2(out.cpu().numpy(), res["im"])
            assert err <= 1e-4, (cube.i_cars.shape, k, err)
            np.testing.assert_array_equal(b.get("q").astype(np.int64), res["q"])
        else:
            degenerate += 1
            _, _, res0 = O.fit(cube.i_cars, cube.i_ref, O.FitParams(k=k, pec=False))
            b0, im0, _ = fk.fkk_fit_basis(ctx, x, ref, fk.fit_params(k=k, pec=0))
            assert rel_l2(im0.cpu().numpy(), res0["im"]) <= 1e-4
            b0.close()
        b.close()
    assert degenerate <= 2


def test_multi_image_full_size_equals_single_fits(fk, ctx):
    specs = multi_image_specs()
    jobs = []
    for spec, k in specs:
        cube = make_tiled_cube(spec)
        x = torch.from_numpy(cube.i_cars).cuda()
        ref = torch.from_numpy(cube.i_ref).cuda()
        jobs.append((x, ref, fk.fit_params(k=k), torch.empty_like(x)))
    bases = fk.fkk_fit_many(ctx, jobs)
    torch.cuda.synchronize()
    st, _ = ctx.sync_status()
    assert st == 0
    for (x, ref, prm, out), b in zip(jobs, bases):
        b1, im1, _ = fk.fkk_fit_basis(ctx, x, ref, prm)
        torch.cuda.synchronize()
        assert torch.equal(im1, out)
        np.testing.assert_array_equal(b1.get("c_amp"), b.get("c_amp"))
        np.testing.assert_array_equal(b1.get("q"), b.get("q"))
        b1.close()
        b.close()
        del im1


def test_multi_image_empty_and_errors(fk, ctx):
    assert fk.fkk_fit_many(ctx, []) == []
    x = torch.ones((100, 64), device="cuda")
    ref = torch.ones(64, device="cuda")
    with pytest.raises(fk.FkkError):  # k larger than the channel count
        fk.fkk_fit_many(ctx, [(x, ref, fk.fit_params(k=20), None), (x, ref, fk.fit_params(k=70), None)])
