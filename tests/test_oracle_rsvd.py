"""Pins for the oracle's randomised SVD (Sec. 5 proposes it; Halko,
Martinsson & Tropp 2011): its counter-based generator against NumPy's own
Philox4x64-10, and the algorithm against what randomised subspace iteration
must give (exact recovery at low rank, convergence to the exact SVD, the
range-finder error bound)."""
import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("key", [(0, 0), (12345, 678), (2**64 - 1, 2**63 + 5)])
def test_philox_matches_numpy(key):
    """NumPy's Philox bit generator increments its counter before each block,
    so its i-th block of four words is ours at counter i + 1."""
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.zeros(4, dtype=np.uint64))
    raw = bg.random_raw(4 * 6)
    for b in range(6):
        assert tuple(int(v) for v in raw[4 * b: 4 * b + 4]) == O.philox4x64((b + 1, 0, 0, 0), key)


@pytest.mark.parametrize("seed", [0, 3, 2**64 - 7])
def test_philox_normals_mapping_by_hand(seed):
    """The mapping of the normals, computed here from NumPy's Philox words
    and the textbook Box-Muller formula: NumPy increments its 256-bit counter
    before each block, so a counter of all ones yields the block at counter
    (0, 0, 0, 0), then (1, 0, 0, 0); entries 2b and 2b + 1 are
    sqrt(-2 ln u1) (cos, sin)(2 pi u2) with u = (w >> 11 + 1/2) 2^-53 of
    words 0 and 1 of block b."""
    ones = np.full(4, 2**64 - 1, dtype=np.uint64)
    bg = np.random.Philox(key=np.array([seed, 0], dtype=np.uint64), counter=ones)
    raw = [int(v) for v in bg.random_raw(8)]
    want = []
    for b in range(2):
        w0, w1 = raw[4 * b], raw[4 * b + 1]
        u1 = ((w0 >> 11) + 0.5) / 2.0**53
        u2 = ((w1 >> 11) + 0.5) / 2.0**53
        r = (-2.0 * np.log(u1)) ** 0.5
        want += [r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)]
    np.testing.assert_allclose(O.philox_normals(4, seed), want, rtol=1e-15, atol=1e-15)


def test_philox_normals_are_standard_normal():
    z = O.philox_normals(200_001, seed=9)
    assert z.shape == (200_001,)
    assert abs(z.mean()) < 5 * (1 / np.sqrt(z.size))
    assert abs(z.std() - 1.0) < 5 * np.sqrt(0.5 / z.size)
    assert abs(np.mean(np.abs(z)) - np.sqrt(2 / np.pi)) < 0.01
    # a different seed gives a different stream; the same seed the same one
    assert not np.allclose(O.philox_normals(64, 1), O.philox_normals(64, 2))
    np.testing.assert_array_equal(O.philox_normals(65, 7)[:64], O.philox_normals(64, 7))


def _lowrank(s, n=400, m=60, seed=0, noise=0.0):
    r = np.random.default_rng(seed)
    U, _ = np.linalg.qr(r.standard_normal((n, len(s))))
    V, _ = np.linalg.qr(r.standard_normal((m, len(s))))
    return (U * np.asarray(s)) @ V.T + noise * r.standard_normal((n, m))


def _rsvd(A, k, p, q, seed=0):
    return O.rsvd(lambda X: A @ X, lambda Y: A.T @ Y, *A.shape, k, p, q, seed)


@pytest.mark.parametrize("q", [0, 1, 3])
def test_rsvd_exact_at_low_rank(q):
    """rank(A) <= l: the sketch spans the whole range, so the top-k pairs are
    exact for any number of power iterations."""
    s = [9.0, 5.0, 3.0, 1.0, 0.5, 0.2, 0.1, 0.05]
    A = _lowrank(s)
    lam, V = _rsvd(A, 5, 5, q)
    np.testing.assert_allclose(np.sqrt(lam), s[:5], rtol=1e-12)
    lam_e, V_e = O.eig_desc(A.T @ A)
    np.testing.assert_allclose(np.abs(np.sum(V * V_e[:, :5], 0)), 1.0, atol=1e-10)
    np.testing.assert_allclose(V.T @ V, np.eye(5), atol=1e-12)


def test_rsvd_converges_to_the_exact_svd():
    """A full-rank matrix with a decaying spectrum: with enough power
    iterations the k leading pairs converge to those of the exact SVD."""
    s = 0.8 ** np.arange(60)
    A = _lowrank(s, n=500, m=60)
    lam_e, V_e = O.eig_desc(A.T @ A)
    lam, V = _rsvd(A, 6, 6, 25)
    np.testing.assert_allclose(lam, lam_e[:6], rtol=1e-10)
    np.testing.assert_allclose(np.abs(np.sum(V * V_e[:, :6], 0)), 1.0, atol=1e-8)
    # fewer iterations: still within the first pairs' gaps, less exact at the cut
    lam1, _ = _rsvd(A, 6, 6, 1)
    assert np.all(lam1 <= lam_e[:6] * (1 + 1e-12)) and lam1[0] > 0.999 * lam_e[0]


def test_rsvd_range_finder_error_bound():
    """Halko et al. eq. (1.9): with q = 0, ||A - Q Q^T A|| <= (1 + 11 sqrt(l
    min(n, m))) s_{k+1} except with probability 6 p^-p; checked through the
    reconstruction error of the returned rank-k factorisation."""
    s = np.concatenate([[10, 7, 5, 3, 2], 0.01 * np.ones(55)])
    A = _lowrank(s, n=300, m=60, seed=4)
    k, p = 5, 6
    lam, V = _rsvd(A, k, p, 0, seed=3)
    err = np.linalg.norm(A - (A @ V) @ V.T, 2)
    assert err <= (1 + 11 * np.sqrt((k + p) * 60)) * s[k]
    assert err < 0.1                                     # in practice near s_{k+1}


def test_fit_with_randomized_svd_close_to_exact():
    """On a cube whose leading singular values are well separated, the fit
    with the randomised SVD approaches the exact fit as q grows."""
    r = np.random.default_rng(6)
    A = _lowrank([4.0, 2.0, 1.0, 0.5], n=800, m=32, seed=6, noise=1e-3)
    i = np.exp(2.0 * A)
    base = dict(k=3, pec=False, sec=False)
    _, _, ex = O.fit(i, np.ones(32), O.FitParams(**base))
    _, _, rq = O.fit(i, np.ones(32), O.FitParams(**base, svd="randomized", rsvd_power_iters=4))
    assert np.linalg.norm(rq["im"] - ex["im"]) / np.linalg.norm(ex["im"]) < 1e-8
