"""Pins of the oracle's basis refinement (refine_basis: one subspace
iteration V <- orth(A^T (A V)) = orth(G V) and the Rayleigh-Ritz pairs of G
on the new span), against facts of the mathematics rather than a retyped
formula: exact eigenvectors are fixed points; a basis rotated inside the
right subspace comes back un-mixed (Rayleigh-Ritz, not just the iteration);
the subspace error shrinks by the eigenvalue gap ratio per step; the Ritz
values interlace the eigenvalues; and the iteration through A equals the one
through G."""
import numpy as np
import pytest

import oracle as O


def _spd(m, lam, seed):
    r = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(r.standard_normal((m, m)))
    return (Q * lam) @ Q.T, Q


def _sin_theta(V, W):
    """Largest principal angle sine between span(V) and span(W)."""
    Qv, _ = np.linalg.qr(V)
    Qw, _ = np.linalg.qr(W)
    return np.linalg.norm(Qv - Qw @ (Qw.T @ Qv), 2)


def test_exact_eigenvectors_are_fixed_points():
    m, k = 60, 8
    lam = np.geomspace(100.0, 0.01, m)
    G, _ = _spd(m, lam, 1)
    lam_o, V = O.eig_desc(G)
    mu, V1 = O.refine_basis(G, V[:, :k], 1)
    np.testing.assert_allclose(mu, lam_o[:k], rtol=1e-12)
    assert np.abs(V1 - V[:, :k]).max() <= 1e-10


def test_rotation_inside_the_subspace_is_undone():
    """Any orthonormal basis of the right span refines to the eigenvectors:
    the Rayleigh-Ritz step, not only the orthonormalised iteration."""
    m, k = 50, 6
    lam = np.concatenate([np.linspace(10.0, 5.0, k), np.linspace(1.0, 0.1, m - k)])
    G, _ = _spd(m, lam, 2)
    lam_o, V = O.eig_desc(G)
    R, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((k, k)))
    mu, V1 = O.refine_basis(G, V[:, :k] @ R, 1)
    np.testing.assert_allclose(mu, lam_o[:k], rtol=1e-12)
    assert np.abs(V1 - V[:, :k]).max() <= 1e-10


@pytest.mark.parametrize("steps", [1, 2, 3])
def test_error_shrinks_by_the_gap_ratio(steps):
    m, k = 80, 5
    ratio = 0.5  # lambda_{k+1} / lambda_k
    lam = np.concatenate([np.linspace(2.0, 1.0, k), ratio * np.linspace(1.0, 0.01, m - k)])
    G, _ = _spd(m, lam, 4)
    _, V = O.eig_desc(G)
    r = np.random.default_rng(5)
    V0, _ = np.linalg.qr(V[:, :k] + 1e-3 * r.standard_normal((m, k)))
    e0 = _sin_theta(V0, V[:, :k])
    _, V1 = O.refine_basis(G, V0, steps)
    e1 = _sin_theta(V1, V[:, :k])
    assert e1 <= 1.05 * ratio**steps * e0 + 1e-13
    assert e1 >= 0.2 * ratio**steps * e0  # a true step, not an exact solve


def test_ritz_values_interlace():
    m, k = 40, 7
    lam = np.geomspace(50.0, 0.5, m)
    G, _ = _spd(m, lam, 6)
    lam_o, _ = O.eig_desc(G)
    V0, _ = np.linalg.qr(np.random.default_rng(7).standard_normal((m, k)))
    mu, V1 = O.refine_basis(G, V0, 1)
    assert np.all(mu <= lam_o[:k] * (1 + 1e-12))  # Cauchy interlacing
    assert np.all(np.diff(mu) <= 0)
    np.testing.assert_allclose(V1.T @ V1, np.eye(k), atol=1e-12)
    np.testing.assert_allclose(V1.T @ G @ V1, np.diag(mu), atol=1e-10 * lam_o[0])


def test_iteration_through_a_equals_through_g():
    r = np.random.default_rng(8)
    A = r.standard_normal((300, 30)) * np.geomspace(1.0, 0.05, 30)
    G = A.T @ A
    V0, _ = np.linalg.qr(r.standard_normal((30, 4)))
    Qa, _ = np.linalg.qr(A.T @ (A @ V0))
    Qg, _ = np.linalg.qr(G @ V0)
    assert _sin_theta(Qa, Qg) <= 1e-10
    mu, V1 = O.refine_basis(G, V0, 1)
    assert _sin_theta(V1, Qa) <= 1e-10


def test_fit_with_refinement_equals_fit_without():
    """With exact eigenvectors the refinement leaves the fit's output as is."""
    from paper_2005_07132_gb300.synth import CubeSpec, make_cube
    cube = make_cube(CubeSpec(12, 12, 96, 4, "gauss", 50.0, seed=9))
    _, _, r0 = O.fit(cube.i_cars, cube.i_ref, O.FitParams(k=6))
    _, _, r1 = O.fit(cube.i_cars, cube.i_ref, O.FitParams(k=6, refine_steps=1))
    assert np.abs(r1["im"] - r0["im"]).max() <= 1e-9 * np.abs(r0["im"]).max()
