"""Pins for the FP64 oracle: each test ties one oracle step to something other
than the oracle itself (a hand-derived value, a closed form, an invariant, a
different library routine, or brute force on a tiny input)."""
import json
import os

import numpy as np
import pytest

import oracle as O

RNG = np.random.default_rng(20200514)


# ---------------------------------------------------------------- Hilbert ---

def _dft_hilbert_bruteforce(x):
    """O(L^2) DFT sums written out: the periodic discrete Hilbert transform."""
    L = x.size
    n = np.arange(L)
    X = np.array([np.sum(x * np.exp(-2j * np.pi * m * n / L)) for m in range(L)])
    mult = np.array([0 if (m == 0 or 2 * m == L) else (-1j if m < L / 2 else 1j) for m in range(L)])
    H = X * mult
    return np.array([np.sum(H * np.exp(2j * np.pi * np.arange(L) * t / L)) / L for t in range(L)]).real


def test_hilbert_golden_impulse(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "hilbert_delta.json")))
    for c in g["cases"]:
        h = O.hilbert(np.array(c["x"], float)[None, :], L=c["L"])[0]
        np.testing.assert_allclose(h, c["h"], atol=1e-15)


@pytest.mark.parametrize("L", [8, 16, 32, 64])
def test_hilbert_vs_bruteforce_dft_periodic(L):
    x = RNG.standard_normal(L)
    np.testing.assert_allclose(O.hilbert(x[None], L=L)[0], _dft_hilbert_bruteforce(x), atol=1e-12)


@pytest.mark.parametrize("M", [5, 13, 24, 31])
def test_hilbert_vs_bruteforce_dft_padded(M):
    """Padded transform = brute-force periodic transform of the edge-padded
    signal, cropped (padding rule: centred, floor((L-M)/2) on the left)."""
    x = RNG.standard_normal(M)
    L = O.pad_len(M)
    assert L >= 2 * M and (L & (L - 1)) == 0 and L // 2 < 2 * M
    left = (L - M) // 2
    xp = np.concatenate([np.full(left, x[0]), x, np.full(L - M - left, x[-1])])
    ref = _dft_hilbert_bruteforce(xp)[left:left + M]
    np.testing.assert_allclose(O.hilbert(x[None])[0], ref, atol=1e-12)


@pytest.mark.parametrize("m", [1, 3, 7, 31])
def test_hilbert_cos_is_sin(m):
    L = 64
    t = np.arange(L)
    h = O.hilbert(np.cos(2 * np.pi * m * t / L)[None], L=L)[0]
    np.testing.assert_allclose(h, np.sin(2 * np.pi * m * t / L), atol=1e-13)


def test_hilbert_twice_is_minus_identity():
    """H{H{x}} = -(x - mean) for x with no Nyquist content (periodic)."""
    L = 64
    X = np.fft.fft(RNG.standard_normal(L))
    X[L // 2] = 0
    x = np.fft.ifft(X).real
    hh = O.hilbert(O.hilbert(x[None], L=L), L=L)[0]
    np.testing.assert_allclose(hh, -(x - x.mean()), atol=1e-13)


# ------------------------------------------------------ KK closed form -----

def _lorentzian_case(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "lorentzian_kk.json")))
    w = np.linspace(g["grid"]["w_min"], g["grid"]["w_max"], g["grid"]["n_channels"])
    Om, Ga = g["peak"]["Omega"], g["peak"]["Gamma"]
    chi_r = g["peak"]["A_over_Gamma"] * Ga / (Om - w - 1j * Ga)
    chi_nr = g["chi_nr"]
    i_cars = np.abs(chi_r + chi_nr) ** 2
    i_nrb = np.full_like(w, chi_nr**2)
    win = np.abs(w - Om) <= g["window_half_widths"] * Ga
    return g, w, chi_r, chi_nr, i_cars, i_nrb, win


def test_kk_lorentzian_closed_form(golden_dir):
    g, w, chi_r, chi_nr, i_cars, i_nrb, win = _lorentzian_case(golden_dir)
    re, im = O.kk_per_spectrum(i_cars[None], i_nrb)
    truth = chi_r.imag / chi_nr
    err = np.linalg.norm(im[0, win] - truth[win]) / np.linalg.norm(truth[win])
    assert err < g["rel_l2_max"], err
    # the real part is 1 + Re{chi_r}/chi_nr
    err_re = np.linalg.norm(re[0, win] - (1 + chi_r.real / chi_nr)[win]) / np.linalg.norm(chi_r.real[win])
    assert err_re < 1e-2, err_re


def test_kk_lorentzian_sign_flip_fails(golden_dir):
    """The opposite Hilbert sign must fail the same closed-form check."""
    g, w, chi_r, chi_nr, i_cars, i_nrb, win = _lorentzian_case(golden_dir)
    a = O.log_ratio(i_cars[None], i_nrb)
    phi = -O.hilbert(a)
    im = np.exp(a) * np.sin(phi)
    truth = chi_r.imag / chi_nr
    err = np.linalg.norm(im[0, win] - truth[win]) / np.linalg.norm(truth[win])
    assert err > 0.5


def test_log_ratio_floor_and_scale():
    i = np.array([[4.0, 0.0, -1.0, 1.0]])
    ref = np.array([1.0, 2.0, 1.0, 1.0])
    a = O.log_ratio(i, ref, ratio_floor=1e-6)
    np.testing.assert_allclose(a[0], [np.log(2.0), 0.5 * np.log(1e-6), 0.5 * np.log(1e-6), 0.0])
    f = np.array([2.0, 1.0, 1.0, 3.0])
    np.testing.assert_allclose(O.log_ratio(i, ref, f)[0], a[0] * f)


def test_noise_scale_definition():
    """1/f = sqrt(alpha <I> + sg^2) / (2 <I>) at hand-checked points."""
    f = O.noise_scale(np.array([1.0, 4.0]), alpha=0.0, sigma_g=2.0)
    np.testing.assert_allclose(f, [1.0, 4.0])  # 2<I>/sg
    f = O.noise_scale(np.array([4.0]), alpha=1.0, sigma_g=0.0)
    np.testing.assert_allclose(f, [4.0])  # 2*4/sqrt(4)


# ------------------------------------------------------------- eigen -------

def test_eig_desc_known_spectrum():
    M = 40
    Q, _ = np.linalg.qr(RNG.standard_normal((M, M)))
    lam = np.sort(RNG.uniform(0.1, 10.0, M))[::-1] + np.arange(M)[::-1] * 0.01
    G = (Q * lam) @ Q.T
    l2, V = O.eig_desc(G)
    np.testing.assert_allclose(l2, lam, rtol=1e-12, atol=1e-12)
    cos = np.abs(np.sum(V * Q, axis=0))
    np.testing.assert_allclose(cos, 1.0, atol=1e-9)
    idx = np.argmax(np.abs(V), axis=0)
    assert np.all(V[idx, np.arange(M)] > 0)


def test_singular_values_match_svd():
    """Gram route gives the singular values of a well-conditioned A
    (numpy.linalg.svd as an independent routine)."""
    A = RNG.standard_normal((300, 20)) * np.linspace(1, 5, 20)
    lam, _ = O.eig_desc(O.gram(A))
    np.testing.assert_allclose(O.singular_from_eig(lam), np.linalg.svd(A, compute_uv=False), rtol=1e-10)


def test_select_rows_hand_case():
    P = np.array([[0.0, 5.0], [3.0, -1.0], [3.0, 5.0], [-2.0, 0.0]])
    # col0: max 3 at rows 1,2 -> 1 (lowest); min -2 at row 3
    # col1: max 5 at rows 0,2 -> 0; min -1 at row 1
    np.testing.assert_array_equal(O.select_rows(P), [0, 1, 3])


# ------------------------------------------------------------- ALS ---------

def test_als_linear_is_fixed_point():
    y = np.linspace(-2.0, 3.0, 200) * 0.7 + 0.3
    for p in (1e-3, 0.5):
        z = O.als_baseline(y, 1e4, p, 10)
        np.testing.assert_allclose(z, y, atol=1e-9)


def test_als_large_lambda_is_weighted_line_fit():
    """lambda -> infinity forces D2 z = 0: z is the weighted least-squares
    line; with p = 0.5 all weights are equal (numpy.polyfit)."""
    x = np.arange(30, dtype=float)
    y = np.sin(x / 3.0) + 0.01 * x
    z = O.als_baseline(y, 1e10, 0.5, 3)
    np.testing.assert_allclose(z, np.polyval(np.polyfit(x, y, 1), x), atol=1e-4)


def test_als_symmetric_is_whittaker_dense():
    """p = 0.5 keeps W = I/2 after the first pass: z solves
    (I + 2 lam D2^T D2) z = y, checked against a dense D2 built from np.diff."""
    n = 60
    y = RNG.standard_normal(n)
    lam = 3.0
    D = np.diff(np.eye(n), 2, axis=0)
    ref = np.linalg.solve(np.eye(n) + 2 * lam * D.T @ D, y)
    np.testing.assert_allclose(O.als_baseline(y, lam, 0.5, 5), ref, atol=1e-10)


def test_als_recovers_baseline_under_positive_peaks():
    x = np.arange(1000, dtype=float)
    base = 0.05 * np.cos(2 * np.pi * x / 700.0) + 0.02 * np.sin(2 * np.pi * x / 330.0)
    peaks = sum(0.3 * 4.0**2 / ((x - c) ** 2 + 4.0**2) for c in (120, 400, 410, 777))
    z = O.als_baseline(base + peaks, O.default_als_lambda(1000), 1e-2, 20)
    assert np.sqrt(np.mean((z - base) ** 2)) < 0.01
    assert np.max(np.abs(z - base)) < 0.04


# ------------------------------------------------------------- ridge -------

def test_ridge_zero_lambda_is_lstsq():
    X = RNG.standard_normal((50, 8))
    Y = RNG.standard_normal((50, 30))
    np.testing.assert_allclose(O.ridge(X, Y, 0.0), np.linalg.lstsq(X, Y, rcond=None)[0], atol=1e-12)


def test_ridge_shrinks_like_svd_filter():
    """(X^T X + lam I)^-1 X^T Y = V diag(s/(s^2+lam)) U^T Y (SVD filter form)."""
    X = RNG.standard_normal((30, 6))
    Y = RNG.standard_normal((30, 4))
    U, s, Vt = np.linalg.svd(X, full_matrices=False)
    lam = 0.7
    ref = Vt.T @ np.diag(s / (s**2 + lam)) @ U.T @ Y
    np.testing.assert_allclose(O.ridge(X, Y, lam), ref, atol=1e-12)


# ------------------------------------------------------------- SG ----------

@pytest.mark.parametrize("M,win,order", [(101, 51, 2), (512, 255, 2), (64, 31, 3)])
def test_savgol_matches_scipy_interp(M, win, order):
    from scipy.signal import savgol_filter
    x = RNG.standard_normal((3, M))
    np.testing.assert_allclose(O.savgol_trend(x, win, order),
                               savgol_filter(x, win, order, mode="interp", axis=-1), atol=1e-10)


def test_savgol_reproduces_polynomials():
    t = np.linspace(-1, 1, 200)
    x = 0.3 - 2 * t + 1.5 * t**2
    np.testing.assert_allclose(O.savgol_trend(x[None], 99, 2)[0], x, atol=1e-11)


# ------------------------------------------------ composition pins ---------

def _small_cube(N=600, M=24, seed=3):
    r = np.random.default_rng(seed)
    i_ref = r.uniform(0.5, 2.0, M)
    i = i_ref * np.exp(2 * (0.2 * r.standard_normal((N, M)) + 0.05))
    return i, i_ref


def test_fkk_full_rank_equals_per_spectrum_kk():
    """With k = M and no PEC/SEC, fKK reproduces per-spectrum KK exactly
    (linearity of H, Eq. HilbertA_Derivation), for any f (Sec. 2.2)."""
    i, i_ref = _small_cube()
    M = i.shape[1]
    f = np.random.default_rng(9).uniform(0.5, 2.0, M)
    p = O.FitParams(k=M, pec=False, sec=False)
    _, _, res = O.fit(i, i_ref, p, f=f)
    re, im = O.kk_per_spectrum(i, i_ref)
    np.testing.assert_allclose(res["im"], im, atol=1e-10)
    np.testing.assert_allclose(res["re"], re, atol=1e-10)


def _conventional_linear(i, i_ref, lam_w, L):
    """Per-spectrum KK + PEC + SEC (Eq. KCARS_from_K in log form) with a
    LINEAR detrend (Whittaker, the p = 0.5 ALS) and the mean as trendline."""
    a = O.log_ratio(i, i_ref)
    phi = O.hilbert(a, L)
    phi_err = np.stack([O.als_baseline(r, lam_w, 0.5, 3) for r in phi])
    logamp = a + O.hilbert(phi_err, L)
    logamp = logamp - logamp.mean(axis=1, keepdims=True)
    return np.exp(logamp) * np.sin(phi - phi_err)


def test_fkk_ec_full_rank_equals_conventional_with_linear_operators():
    """k = M, ridge lambda = 0 and linear D / M: the factorised workflow must
    equal the per-spectrum workflow (fPEC regression is then exact).  Pins the
    orientation of X = U_ss S, the signs of H{Phi_PEC} and Phi_PEC, the V_SEC
    subtraction and the f scaling (f != 1)."""
    i, i_ref = _small_cube(N=500, M=20)
    M = i.shape[1]
    f = np.random.default_rng(5).uniform(0.5, 2.0, M)
    lam_w = 2.0
    p = O.FitParams(k=M, pec=True, sec=True, als_lambda=lam_w, als_p=0.5, als_iters=3,
                    ridge_rel=0.0, sec_mode="mean")
    basis, P, res = O.fit(i, i_ref, p, f=f)
    assert len(res["q"]) >= M
    ref = _conventional_linear(i, i_ref, lam_w, O.pad_len(M))
    np.testing.assert_allclose(res["im"], ref, atol=1e-8)


def test_sec_mean_zeroes_mean_log_amplitude():
    """Eq. fSEC: with the mean trendline every reconstructed spectrum has a
    zero mean log-amplitude."""
    i, i_ref = _small_cube(N=800, M=32)
    p = O.FitParams(k=6, sec_mode="mean")
    basis, P, res = O.fit(i, i_ref, p)
    np.testing.assert_allclose(basis.c_amp.mean(axis=1), 0.0, atol=1e-13)
    logamp = np.log(np.hypot(res["re"], res["im"]))
    np.testing.assert_allclose(logamp.mean(axis=1), 0.0, atol=1e-12)


def test_ml_apply_on_training_data_equals_fit():
    """Eq. ML_Unew with lambda = 0 on the training data returns U S, so the
    ML output equals the fit's output."""
    i, i_ref = _small_cube(N=700, M=28)
    p = O.FitParams(k=8)
    basis, P, res = O.fit(i, i_ref, p)
    re, im = O.apply(basis, i)
    np.testing.assert_allclose(im, res["im"], atol=1e-11)
    np.testing.assert_allclose(re, res["re"], atol=1e-11)


def test_ml_ridge_shrinks_projection():
    i, i_ref = _small_cube(N=300, M=16)
    p = O.FitParams(k=5, ml_lambda=0.0)
    basis, P, _ = O.fit(i, i_ref, p)
    basis.params.ml_lambda = 2.0
    W = O.apply_projector(basis)
    s = basis.s
    np.testing.assert_allclose(W, basis.V * (s**2 / (s**2 + 2.0)), atol=1e-14)
    # ridge projection equals the explicit ridge of A_new on X = S V^T
    A = O.log_ratio(i, i_ref)
    X = np.diag(s) @ basis.V.T
    U_new = A @ X.T @ np.linalg.inv(X @ X.T + 2.0 * np.eye(5))
    np.testing.assert_allclose(A @ W, U_new * s, atol=1e-10)
