"""Pins for the oracle's conventional per-spectrum workflow (Sec. 2.1,
Eq. KCARS_from_K: KK, then PEC by a detrended phase error, then SEC by the
trendline of the real part).  Its parts (Hilbert transform, ALS, trendline)
are pinned in test_oracle_pins.py; these tie their composition to what the
equations fix independently of the code."""
import numpy as np
import pytest

import oracle as O


def _cars_like(N=12, M=96, seed=11, scale=1.0):
    """Spectra with narrow positive phase features on a smooth background,
    and a surrogate reference with a smooth spectral error xi(w)."""
    r = np.random.default_rng(seed)
    w = np.linspace(0.0, 1.0, M)
    nrb = 1.0 + 0.3 * np.exp(-((w - 0.5) ** 2) / 0.1)
    chi_r = np.zeros((N, M), complex)
    for n in range(N):
        for _ in range(3):
            om, g, amp = r.uniform(0.2, 0.8), r.uniform(0.01, 0.03), r.uniform(0.02, 0.1)
            chi_r[n] += amp * g / (om - w - 1j * g)
    i_cars = nrb * np.abs(chi_r + 1.0) ** 2
    xi = np.exp(0.05 * np.cos(2 * np.pi * w) + 0.03 * np.sin(3 * np.pi * w))
    i_ref = scale * 1.05 * xi * nrb
    return i_cars, i_ref


def test_conventional_without_pec_sec_is_plain_kk():
    """PEC and SEC off: Eq. KCARS_from_K reduces to Eq. K."""
    i, ref = _cars_like()
    p = O.FitParams(pec=False, sec=False)
    re, im = O.conventional(i, ref, p)
    re0, im0 = O.kk_per_spectrum(i, ref)
    np.testing.assert_allclose(im, im0, rtol=0, atol=1e-14)
    np.testing.assert_allclose(re, re0, rtol=0, atol=1e-14)


@pytest.mark.parametrize("pec", [False, True])
@pytest.mark.parametrize("mode", ["mean", "sg"])
@pytest.mark.parametrize("xi_scale", [0.37, 4.2])
def test_conventional_is_invariant_to_the_reference_scale(pec, mode, xi_scale):
    """I_ref -> c I_ref only multiplies K by 1/sqrt(c) (H of a constant is 0,
    so phi and the phase error do not change); SEC divides that constant
    out again (Sec. 2.1: SEC finds the constant Xi)."""
    i, ref = _cars_like(N=6, M=80)
    p = O.FitParams(pec=pec, sec=True, sec_mode=mode, sg_window=31)
    re1, im1 = O.conventional(i, ref, p)
    re2, im2 = O.conventional(i, xi_scale * ref, p)
    np.testing.assert_allclose(im2, im1, rtol=0, atol=1e-12)
    np.testing.assert_allclose(re2, re1, rtol=0, atol=1e-12)
    # without SEC the output scales as 1/sqrt(c): the invariance above is SEC's
    p.sec = False
    _, im3 = O.conventional(i, ref, p)
    _, im4 = O.conventional(i, xi_scale * ref, p)
    np.testing.assert_allclose(im4, im3 / np.sqrt(xi_scale), rtol=1e-12, atol=1e-15)


def test_conventional_sec_mean_normalises_the_real_part():
    """With the plain mean as trendline (Eq. KCARS_from_K as written), the
    mean of Re K_CARS over frequency is exactly 1 for every spectrum."""
    i, ref = _cars_like(N=9, M=64)
    p = O.FitParams(pec=True, sec=True, sec_mode="mean")
    re, _ = O.conventional(i, ref, p)
    np.testing.assert_allclose(re.mean(axis=1), 1.0, rtol=0, atol=1e-13)


def test_conventional_pec_phase_is_equivariant_to_linear_phase():
    """The ALS baseline moves with any added linear function (D2 annihilates
    it and the weights compare y - z, which it leaves unchanged), so the
    PEC-corrected phase phi - phi_err ignores a linear phase.  A sign error
    in the subtraction, or a baseline taken of anything but phi, fails."""
    i, ref = _cars_like(N=5, M=120, seed=4)
    a = O.log_ratio(i, ref)
    phi = O.hilbert(a)
    p = O.FitParams(pec=True, sec=False)
    ell = 0.3 - 0.002 * np.arange(a.shape[1])
    re1, im1 = O.conventional_from_phase(a, phi, p)
    re2, im2 = O.conventional_from_phase(a, phi + ell, p)
    ang1 = np.arctan2(im1, re1)
    ang2 = np.arctan2(im2, re2)
    np.testing.assert_allclose(ang2, ang1, rtol=0, atol=1e-9)
    # and the corrected phase is not the raw one: PEC removed something
    assert np.max(np.abs(ang1 - np.arctan2(np.sin(phi), np.cos(phi)))) > 1e-3


def test_conventional_pec_removes_a_pure_phase_error():
    """No Raman signal (I_CARS = I_NRB) and a reference with a smooth
    spectral error: K is then exp(a) exp(i phi) with phi the phase error
    alone, so the ideal K_CARS is 1.  ALS recovers the smooth phase error up
    to its smoothing bias: the corrected phase is far smaller than phi."""
    M = 256
    w = np.linspace(0.0, 1.0, M)
    nrb = np.ones((3, M))
    xi = np.exp(0.2 * np.cos(np.pi * w) + 0.1 * w)
    i_ref = xi * nrb[0]
    a = O.log_ratio(nrb, i_ref)
    phi = O.hilbert(a)
    p = O.FitParams(pec=True, sec=True, sec_mode="mean", als_p=0.5)
    re, im = O.conventional(nrb, i_ref, p)
    assert np.max(np.abs(im)) < 0.05 * np.max(np.abs(phi))


def test_conventional_pec_exact_phase_error_gives_unit_k():
    """Fixes the sign of H{phi_err} in the amplitude (Eq. K: the amplitude
    error is exp(-H{phi_err}) / Xi).  Periodic transform (L = M) and an ALS
    with a vanishing penalty return phi_err = phi exactly; with a
    band-limited a, H{H{a}} = -(a - <a>), so K_pec = exp(<a>) and the mean
    SEC makes K_CARS = 1 at every frequency."""
    M = 64
    r = np.random.default_rng(8)
    t = np.arange(M)
    a = 0.1 * sum(r.standard_normal() * np.cos(2 * np.pi * q * t / M + r.uniform(0, 6)) for q in range(1, 12))
    a = a[None, :] + 0.3
    phi = O.hilbert(a, M)
    p = O.FitParams(pec=True, sec=True, sec_mode="mean", als_lambda=1e-10, als_p=0.5, als_iters=1)
    re, im = O.conventional_from_phase(a, phi, p, M)
    np.testing.assert_allclose(re, 1.0, rtol=0, atol=1e-9)
    np.testing.assert_allclose(im, 0.0, rtol=0, atol=1e-9)


# ---------------------------------------------------------------------------
# The conventional workflow's SVD denoising of the raw spectra (Fig. 1(a))
# ---------------------------------------------------------------------------


def _known_svd(s, n=300, m=48, seed=5):
    """X = U diag(s) V^T with U, V random orthonormal: its truncations are
    known without computing an SVD."""
    r = np.random.default_rng(seed)
    U, _ = np.linalg.qr(r.standard_normal((n, len(s))))
    V, _ = np.linalg.qr(r.standard_normal((m, len(s))))
    return U, np.asarray(s, float), V


def test_denoise_keeps_the_largest_triplets():
    """Eckart-Young: the rank-j truncation is U_j S_j V_j^T of the largest
    j singular values; a matrix of rank r is returned unchanged for k >= r."""
    U, s, V = _known_svd([7.0, 3.0, 2.0, 0.5, 0.1])
    X = (U * s) @ V.T
    for j in (1, 2, 4):
        got, k = O.svd_denoise(X, j)
        assert k == j
        np.testing.assert_allclose(got, (U[:, :j] * s[:j]) @ V[:, :j].T, atol=1e-12)
        assert abs(np.linalg.norm(X - got) ** 2 - np.sum(s[j:] ** 2)) < 1e-10
    got, k = O.svd_denoise(X, 9)
    assert k == 9
    np.testing.assert_allclose(got, X, atol=1e-12)


def test_denoise_rank_rule():
    """k < 0: the rank rule of Sec. 4.1 (cutoff s_1 max(N, M) eps) on
    singular values chosen on both sides of the cutoff 300 x 1.19e-7 =
    3.6e-5 (relative)."""
    U, s, V = _known_svd([1.0, 0.3, 1e-3, 1e-4, 1e-6, 1e-8])
    X = (U * s) @ V.T
    got, k = O.svd_denoise(X, -1)
    assert k == 4
    np.testing.assert_allclose(got, (U[:, :4] * s[:4]) @ V[:, :4].T, atol=1e-12)
    assert O.svd_denoise(X, -1, k_max=2)[1] == 2


def test_conventional_with_full_rank_denoise_is_unchanged():
    i, ref = _cars_like(N=20, M=64)
    p = O.FitParams()
    re0, im0 = O.conventional(i, ref, p)
    p.denoise_k = 64
    re1, im1 = O.conventional(i, ref, p)
    np.testing.assert_allclose(im1, im0, atol=1e-9)
    np.testing.assert_allclose(re1, re0, atol=1e-9)
    # a truncation changes it
    p.denoise_k = 3
    _, im3 = O.conventional(i, ref, p)
    assert np.abs(im3 - im0).max() > 1e-4


def test_denoise_reduces_the_error_against_the_truth():
    """On the noisy synthetic cube (SNR 50) the conventional workflow on
    SVD-denoised spectra lands much closer to the known Im{chi/chi_NR}: the
    rows span 6 dominant singular vectors above a flat noise floor."""
    from paper_2005_07132_gb300.synth import CONFIGS, make_cube
    c = make_cube(CONFIGS["img64_m512"])
    rows = np.arange(384)
    I = c.i_cars[rows].astype(np.float64)
    truth = c.truth_im(rows)
    rss = {}
    for k in (0, 6):
        _, im = O.conventional(I, c.i_ref.astype(np.float64), O.FitParams(denoise_k=k))
        rss[k] = np.mean(np.sum((im - truth) ** 2, 1))
    assert rss[6] < 0.25 * rss[0], rss
