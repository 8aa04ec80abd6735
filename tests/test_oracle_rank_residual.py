"""Pins for the oracle's rank rule (Sec. 4.1: keep the singular values above
s_1 max(N, M) eps) and for the residual fraction that tests whether a
trained basis still supports new data (Sec. 5)."""
import numpy as np
import pytest

import oracle as O


def _matrix_with_singular_values(s, n=300, m=40, seed=0):
    r = np.random.default_rng(seed)
    U, _ = np.linalg.qr(r.standard_normal((n, len(s))))
    V, _ = np.linalg.qr(r.standard_normal((m, len(s))))
    return (U * np.asarray(s)) @ V.T


@pytest.mark.parametrize("s,want", [([1.0, 0.5, 0.1, 1e-3, 1e-9, 1e-11], 4),
                                    ([2.0, 1.0, 1e-7], 2),
                                    ([1.0], 1)])
def test_rank_rule_matches_numpy_matrix_rank(s, want):
    """The rule is NumPy's matrix_rank cutoff: with float32 data both count
    the same singular values (none lies near the threshold here)."""
    A = _matrix_with_singular_values(s).astype(np.float32)
    lam = O.eig_desc(O.gram(A))[0]
    k = O.rank_k(lam, *A.shape, k_max=80)
    assert k == want == np.linalg.matrix_rank(A)


def test_rank_rule_k_max_and_eps():
    A = _matrix_with_singular_values([1.0, 0.5, 0.1, 1e-3, 1e-5])
    lam = O.eig_desc(O.gram(A))[0]
    n, m = A.shape
    assert O.rank_k(lam, n, m, k_max=2) == 2                     # capped
    assert O.rank_k(lam, n, m, k_max=80, eps=1e-9) == 5          # finer epsilon keeps more
    assert O.rank_k(lam, n, m, k_max=80, eps=1.0) == 1           # never below 1


def _basis_from(A_log, k):
    """A trained basis whose A (f = 1, I_ref = 1) is exactly A_log."""
    i = np.exp(2.0 * A_log)
    basis, P, res = O.fit(i, np.ones(A_log.shape[1]), O.FitParams(k=k, pec=False, sec=False))
    return basis, i


def test_residual_of_training_data_is_the_discarded_eigenvalue_mass():
    """For the training data, ||A V_k||^2 = sum of the k largest eigenvalues
    of A^T A (Ky Fan), so the residual is 1 - sum(lambda_1..k) / trace."""
    r = np.random.default_rng(2)
    A = 0.1 * r.standard_normal((400, 30)) @ np.diag(np.linspace(2.0, 0.1, 30))
    basis, i = _basis_from(A, 7)
    lam = basis.extras["lam"]
    want = 1.0 - lam[:7].sum() / basis.extras["energy"]
    assert abs(O.residual_fraction(basis, i) - want) < 1e-12
    np.testing.assert_allclose(basis.extras["energy"], np.sum(A * A), rtol=1e-12)


def test_residual_of_data_in_and_orthogonal_to_the_span():
    r = np.random.default_rng(3)
    A = 0.1 * r.standard_normal((200, 20))
    basis, _ = _basis_from(A, 5)
    V = basis.V
    inside = r.standard_normal((50, 5)) @ V.T                   # rows in span(V)
    assert abs(O.residual_fraction(basis, np.exp(2.0 * inside))) < 1e-12
    Q, _ = np.linalg.qr(np.concatenate([V, r.standard_normal((20, 3))], axis=1))
    outside = r.standard_normal((50, 3)) @ Q[:, 5:].T           # rows orthogonal to V
    assert abs(O.residual_fraction(basis, np.exp(2.0 * outside)) - 1.0) < 1e-12


def test_fit_with_rank_rule_uses_the_rule():
    A = _matrix_with_singular_values([3.0, 1.0, 0.2, 1e-9], n=500, m=24) + 0.0
    i = np.exp(2.0 * A)
    _, _, res = O.fit(i, np.ones(24), O.FitParams(k=0, pec=False, sec=False))
    assert res["k"] == 3
