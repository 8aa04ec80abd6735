"""FP64 CPU oracle for fKK-EC and per-spectrum KK  --  TEST INFRASTRUCTURE ONLY.

This module is the independent, slow, plain reference that the CUDA path is
checked against.  Only the test-suite, the smoke check of the package entry
point and the benchmark's CPU-baseline / reference legs may import it; the
product path never does.  It shares no code with the CUDA library.

Everything is float64 numpy.  Library primitives used as single steps: FFT
(numpy.fft), symmetric eigendecomposition (numpy.linalg.eigh), the SVD
(numpy.linalg.svd, for the conventional workflow's denoising), dense and
banded linear solves (numpy.linalg.solve, scipy.linalg.solveh_banded), and
matrix products.

Notation follows the paper (Camp, Bender & Lee, "Real-time and high-throughput
Raman signal extraction and processing in CARS hyperspectral imaging"), with
one deliberate renaming: here N is the number of spectra (rows) and M the
number of channels (columns); the paper uses the opposite letters (Sec. 2.2).

Readings where the paper is silent (each is also a keyword argument):
  * ratio floor: I/I_ref is clamped below at 1e-6 before the logarithm;
  * discrete Hilbert transform: edge-replicate pad to L = nextpow2(2M),
    centred (floor((L-M)/2) samples on the left), multiply bin m of the DFT by
    -i*sgn(m) with 0 at DC and at the Nyquist bin, inverse DFT, crop;
  * no mean-centring before the SVD (Sec. 2.2 factorises A itself);
  * eigenvector sign: the largest-magnitude component is made positive
    (cosmetic; every use is bilinear in V or a union of argmax and argmin);
  * detrending operator D (Eq. phi_err_USphi_b) = asymmetric least squares
    with a second-difference penalty, lambda = 1e4 * (M/1000)^4, p = 1e-2,
    20 iterations, weights start at 1 (chosen by the error against the known
    truth on the synthetic workload; the paper gives no values);
  * ridge weight (Eq. PEC_Ridge) lambda_r = 1e-3 * ||X||_F^2 / k;
  * trendline M{} (Eq. fSEC_VT) = Savitzky-Golay of order 2 over the largest
    odd window <= M/2, edges from the polynomial fitted to the first / last
    full window ("interp" edges); the alternative is the plain mean;
  * ML apply (Eq. ML_Unew): U_new S = A_new V diag(s^2 / (s^2 + lambda_ml)).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

F64 = np.float64

# ---------------------------------------------------------------------------
# Parameters
# ---------------------------------------------------------------------------


@dataclass
class FitParams:
    k: int = 20
    pad_len: int = 0  # 0 -> nextpow2(2M)
    pec: bool = True
    sec: bool = True
    als_lambda: float | None = None  # None -> 1e4 * (M/1000)^4
    als_p: float = 1e-2
    als_iters: int = 20
    ridge_rel: float = 1e-3
    sec_mode: str = "sg"  # "sg" | "mean"
    sg_window: int = 0  # 0 -> largest odd <= M/2
    sg_order: int = 2
    ml_lambda: float = 0.0
    ratio_floor: float = 1e-6
    k_max: int = 80          # k = 0: the rank rule picks k <= k_max
    rank_eps: float = 0.0    # epsilon of the rank rule; 0 -> float32 machine epsilon
    svd: str = "exact"       # "exact" (eigenpairs of A^T A) or "randomized" (Sec. 5: Halko et al.)
    rsvd_oversample: int = 10
    rsvd_power_iters: int = 2
    rsvd_seed: int = 0
    denoise_k: int = 0       # conventional workflow: 0 no SVD denoising of the raw spectra; > 0 keep that
                             # many singular triplets; < 0 the rank rule (at most k_max)
    refine_steps: int = 0    # exact SVD: refinement steps on the kept basis (refine_basis)


def pad_len(n_channels: int) -> int:
    """L = nextpow2(2M): the discrete Hilbert transform's padded length."""
    L = 1
    while L < 2 * n_channels:
        L *= 2
    return L


def default_als_lambda(n_channels: int) -> float:
    return 1e4 * (n_channels / 1000.0) ** 4


def default_sg_window(n_channels: int) -> int:
    w = n_channels // 2
    if w % 2 == 0:
        w -= 1
    return max(w, 3)


# ---------------------------------------------------------------------------
# Eq. KCARS / Eq. K: log ratio and Hilbert transform
# ---------------------------------------------------------------------------


def log_ratio(i_cars, i_ref, f=None, ratio_floor: float = 1e-6) -> np.ndarray:
    """A = f(w) * 1/2 ln(I_CARS / I_ref) row-wise (Sec. 2.2, the scaled A of
    the heteroscedastic addendum; f = None means f = 1)."""
    r = np.asarray(i_cars, F64) / np.asarray(i_ref, F64)
    a = 0.5 * np.log(np.maximum(r, ratio_floor))
    if f is not None:
        a = a * np.asarray(f, F64)
    return a


def hilbert(x, L: int | None = None) -> np.ndarray:
    """Discrete Hilbert transform of each row of x (last axis), Eq. KCARS.

    Rows are edge-padded to length L (centred), transformed with the DFT,
    bin m multiplied by -i*sgn(m) (sgn = +1 for 0 < m < L/2, -1 for m > L/2,
    0 at m = 0 and m = L/2), inverse-transformed and cropped back.  With
    L == M there is no padding (the periodic transform)."""
    x = np.asarray(x, F64)
    M = x.shape[-1]
    if L is None:
        L = pad_len(M)
    if L < M:
        raise ValueError("pad length shorter than the signal")
    left = (L - M) // 2
    right = L - M - left
    pad = [(0, 0)] * (x.ndim - 1) + [(left, right)]
    xp = np.pad(x, pad, mode="edge") if L > M else x
    X = np.fft.fft(xp, axis=-1)
    m = np.arange(L)
    mult = np.zeros(L, np.complex128)
    mult[(m > 0) & (m < L // 2)] = -1j
    mult[m > L // 2] = 1j
    h = np.fft.ifft(X * mult, axis=-1).real
    return h[..., left : left + M]


def kk_per_spectrum(i_cars, i_ref, L: int | None = None, ratio_floor: float = 1e-6):
    """Conventional per-spectrum KK, Eq. KCARS with the surrogate of Eq. K:
    K = sqrt(I/I_ref) exp(i H{1/2 ln(I/I_ref)}).  Returns (Re K, Im K)."""
    a = log_ratio(i_cars, i_ref, None, ratio_floor)
    phi = hilbert(a, L)
    amp = np.exp(a)
    return amp * np.cos(phi), amp * np.sin(phi)


# ---------------------------------------------------------------------------
# Sec. 2.1 / Fig. 1(a): the conventional per-spectrum workflow (KK, PEC, SEC)
# ---------------------------------------------------------------------------


def conventional_from_phase(a, phi, params: "FitParams", L: int | None = None):
    """PEC and SEC of Eq. KCARS_from_K on each spectrum, given its log
    amplitude a = 1/2 ln(I/I_ref) and KK phase phi = H{a}.

    PEC: phi_err = D{phi} (the ALS baseline, the same detrending operator as
    fPEC), K_pec = exp(a + H{phi_err}) exp(i (phi - phi_err)).
    SEC: K_CARS = K_pec / M{Re K_pec}, M the trendline operator (the plain
    mean for sec_mode "mean"); with sec off the divisor is 1.
    Returns (Re K_CARS, Im K_CARS)."""
    a = np.atleast_2d(np.asarray(a, F64))
    phi = np.atleast_2d(np.asarray(phi, F64))
    M = a.shape[-1]
    if params.pec:
        lam = params.als_lambda if params.als_lambda is not None else default_als_lambda(M)
        phi_err = np.stack([als_baseline(r, lam, params.als_p, params.als_iters) for r in phi])
        h_err = hilbert(phi_err, L)
    else:
        phi_err = np.zeros_like(phi)
        h_err = np.zeros_like(phi)
    amp = np.exp(a + h_err)
    ph = phi - phi_err
    re = amp * np.cos(ph)
    im = amp * np.sin(ph)
    if params.sec:
        win = params.sg_window or default_sg_window(M)
        div = trend(re, params.sec_mode, win, params.sg_order)
    else:
        div = np.ones_like(re)
    return re / div, im / div


def svd_denoise(i_cars, k: int, k_max: int = 80, eps: float = 0.0):
    """The denoising step of the conventional workflow (Fig. 1(a); Sec. 2.2:
    drop the singular vectors that carry noise): the truncated SVD of the raw
    spectra (rows = spectra), U_k S_k V_k^T with the k largest singular
    values, or with k < 0 the rank rule of Sec. 4.1 (at most k_max).
    Returns (denoised spectra, k)."""
    X = np.asarray(i_cars, F64)
    U, s, Vt = np.linalg.svd(X, full_matrices=False)
    if k < 0:
        k = rank_k(s * s, X.shape[0], X.shape[1], k_max, eps)
    k = min(k, s.size)
    return (U[:, :k] * s[:k]) @ Vt[:k], k


def conventional(i_cars, i_ref, params: "FitParams", L: int | None = None):
    """The conventional workflow of Fig. 1(a): optionally the SVD denoising
    of the raw spectra (params.denoise_k), then per-spectrum KK (Eq. K),
    PEC and SEC (Eq. KCARS_from_K).  Returns (Re K_CARS, Im K_CARS)."""
    if params.denoise_k:
        i_cars, _ = svd_denoise(i_cars, params.denoise_k, params.k_max, params.rank_eps)
    a = log_ratio(i_cars, i_ref, None, params.ratio_floor)
    phi = hilbert(a, L or params.pad_len or None)
    return conventional_from_phase(a, phi, params, L or params.pad_len or None)


# ---------------------------------------------------------------------------
# Sec. 2.2 (heteroscedastic addendum): noise-normalising spectrum f(w)
# ---------------------------------------------------------------------------


def noise_scale(mean_i, alpha: float, sigma_g: float) -> np.ndarray:
    """f(w) from 1/f = sqrt(alpha <I> + sigma_g^2) / (2 <I>)."""
    mean_i = np.asarray(mean_i, F64)
    return 2.0 * mean_i / np.sqrt(alpha * mean_i + sigma_g**2)


# ---------------------------------------------------------------------------
# Sec. 2.2: SVD through the Gram matrix
# ---------------------------------------------------------------------------


def gram(A) -> np.ndarray:
    """G = A^T A (M x M)."""
    A = np.asarray(A, F64)
    return A.T @ A


def eig_desc(G):
    """Eigenpairs of the symmetric G sorted by descending eigenvalue, each
    eigenvector's largest-magnitude component made positive."""
    lam, V = np.linalg.eigh(np.asarray(G, F64))
    order = np.argsort(lam)[::-1]
    lam = lam[order]
    V = V[:, order]
    idx = np.argmax(np.abs(V), axis=0)
    sign = np.sign(V[idx, np.arange(V.shape[1])])
    sign[sign == 0] = 1.0
    return lam, V * sign


def refine_basis(G, V, steps: int):
    """Refinement of a computed basis V (M x k) of the k largest eigenpairs of
    G = A^T A (Sec. 2.2 needs V and S of the SVD of A): each step is one
    subspace iteration, Q = orth(G V) = orth(A^T (A V)), then the
    Rayleigh-Ritz pairs of G on span(Q): the k x k matrix Q^T G Q =
    U diag(mu) U^T gives V = Q U and the eigenvalues mu.  Exact eigenvectors
    come back unchanged (up to rounding); the error of an approximate basis
    shrinks about as lambda_{k+1} / lambda_k per step.  Returns (mu, V),
    descending, each column's largest-magnitude component positive."""
    G = np.asarray(G, F64)
    V = np.asarray(V, F64)
    mu = np.diag(V.T @ G @ V).copy()
    for _ in range(steps):
        Q, _ = np.linalg.qr(G @ V)
        H = Q.T @ G @ Q
        mu, U = np.linalg.eigh((H + H.T) / 2.0)
        order = np.argsort(mu)[::-1]
        mu, U = mu[order], U[:, order]
        V = Q @ U
    idx = np.argmax(np.abs(V), axis=0)
    sign = np.sign(V[idx, np.arange(V.shape[1])])
    sign[sign == 0] = 1.0
    return mu, V * sign


def rank_k(lam, n: int, m: int, k_max: int, eps: float = 0.0) -> int:
    """The rank rule of Sec. 4.1: the number of singular values s_i of A
    (s = sqrt(lambda)) above s_1 * max(N, M) * eps, among the k_max largest
    (at least 1).  eps = 0 means the float32 machine epsilon, the epsilon of
    the input data type."""
    eps = eps or float(np.finfo(np.float32).eps)
    s = np.sqrt(np.maximum(np.asarray(lam, F64)[:k_max], 0.0))
    tol = s[0] * max(n, m) * eps
    return max(1, int(np.sum(s > tol)))


def residual_fraction(basis: "Basis", i_new) -> float:
    """||A - A V V^T||_F^2 / ||A||_F^2 of new spectra on a trained basis:
    how much of the new data the basis does not represent (Sec. 5: retrain
    when the basis vectors do not adequately support new data)."""
    A = log_ratio(i_new, basis.i_ref, basis.f, basis.params.ratio_floor)
    PV = A @ basis.V
    return float(1.0 - np.sum(PV * PV) / np.sum(A * A))


# ---------------------------------------------------------------------------
# Sec. 5 (the randomised SVD the paper proposes, Halko, Martinsson & Tropp
# 2011): counter-based random numbers and randomised subspace iteration
# ---------------------------------------------------------------------------

_PHILOX_M = (0xD2E7470EE14C6C93, 0xCA5A826395121157)  # Philox4x64 multipliers
_PHILOX_W = (0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B)  # key increments (Weyl)
_U64 = (1 << 64) - 1


def philox4x64(ctr, key, rounds: int = 10):
    """Philox4x64-10 (Salmon, Moraes, Dror & Shaw, SC'11): 4 x 64-bit counter,
    2 x 64-bit key; each round multiplies words 0 and 2 by the constants,
    mixes the high halves with words 1, 3 and the key, then bumps the key."""
    x0, x1, x2, x3 = (int(v) & _U64 for v in ctr)
    k0, k1 = (int(v) & _U64 for v in key)
    for _ in range(rounds):
        p0 = _PHILOX_M[0] * x0
        p1 = _PHILOX_M[1] * x2
        x0, x1, x2, x3 = ((p1 >> 64) ^ x1 ^ k0) & _U64, p1 & _U64, ((p0 >> 64) ^ x3 ^ k1) & _U64, p0 & _U64
        k0 = (k0 + _PHILOX_W[0]) & _U64
        k1 = (k1 + _PHILOX_W[1]) & _U64
    return x0, x1, x2, x3


def philox_normals(count: int, seed: int) -> np.ndarray:
    """count standard normals: entry e comes from Philox4x64-10 at counter
    (e // 2, 0, 0, 0) with key (seed, 0); its first two words give uniforms
    u = (w >> 11 + 1/2) 2^-53 in (0, 1), and Box-Muller gives
    sqrt(-2 ln u1) cos(2 pi u2) (even e) or sin(2 pi u2) (odd e)."""
    out = np.empty(count)
    for b in range((count + 1) // 2):
        w0, w1, _, _ = philox4x64((b, 0, 0, 0), (seed, 0))
        u1 = ((w0 >> 11) + 0.5) * 2.0**-53
        u2 = ((w1 >> 11) + 0.5) * 2.0**-53
        r = np.sqrt(-2.0 * np.log(u1))
        out[2 * b] = r * np.cos(2.0 * np.pi * u2)
        if 2 * b + 1 < count:
            out[2 * b + 1] = r * np.sin(2.0 * np.pi * u2)
    return out


def _orth(Y) -> np.ndarray:
    """An orthonormal basis of the range of Y (Householder QR)."""
    return np.linalg.qr(Y)[0]


def rsvd(matvec, rmatvec, n: int, m: int, k: int, oversample: int, power_iters: int, seed: int):
    """Randomised SVD of an n x m matrix A given A X (matvec) and A^T Y
    (rmatvec): randomised subspace iteration (Halko et al. 2011, Alg. 4.4)
    with l = k + oversample Gaussian test vectors, then the SVD of the small
    B = Q^T A through the eigenpairs of B B^T.  Returns (lambda, V) for the k
    largest: lambda = s^2, V (m x k) with its largest-magnitude component
    positive in each column."""
    l = min(k + oversample, m)
    Om = philox_normals(m * l, seed).reshape(m, l)
    Y = matvec(Om)
    for _ in range(power_iters):
        Q = _orth(Y)
        Z = _orth(rmatvec(Q))
        Y = matvec(Z)
    Q = _orth(Y)
    B = rmatvec(Q).T  # l x m
    lam, U = np.linalg.eigh(B @ B.T)
    order = np.argsort(lam)[::-1][:k]
    lam, U = lam[order], U[:, order]
    s = np.sqrt(np.maximum(lam, 0.0))
    V = (B.T @ U) / np.where(s > 0, s, 1.0)
    idx = np.argmax(np.abs(V), axis=0)
    sign = np.sign(V[idx, np.arange(k)])
    sign[sign == 0] = 1.0
    return lam, V * sign


def singular_from_eig(lam) -> np.ndarray:
    """s = sqrt(max(lambda, 0)): singular values of A from eigenvalues of A^T A."""
    return np.sqrt(np.maximum(np.asarray(lam, F64), 0.0))


# ---------------------------------------------------------------------------
# Sec. 2.3 (fPEC): sub-sampling, detrending, ridge regression
# ---------------------------------------------------------------------------


def select_rows(P) -> np.ndarray:
    """q = q_max U q_min: the rows holding the largest and the smallest value
    of each column of U (equivalently of U S, since s > 0), Eqs. q_max/q_min.
    Ties go to the lowest row index.  Returned sorted and unique."""
    P = np.asarray(P)
    qmax = np.argmax(P, axis=0)
    qmin = np.argmin(P, axis=0)
    return np.unique(np.concatenate([qmax, qmin]))


def als_baseline(y, lam: float, p: float, iters: int) -> np.ndarray:
    """Asymmetric least squares baseline of one signal (the detrending operator
    D of Eq. phi_err_USphi_b; P. Eilers' ALS as cited for PEC in Sec. 2.1).

    Repeats `iters` times: solve (W + lam D2^T D2) z = W y with W = diag(w),
    D2 the second-difference operator; then w_i = p where y_i > z_i, else 1-p.
    Weights start at 1.  Returns z."""
    y = np.asarray(y, F64)
    n = y.size
    # D2^T D2 is symmetric pentadiagonal: accumulate the outer products of the
    # rows (1, -2, 1) of D2 into its three bands (upper banded storage).
    d0 = np.zeros(n)
    d1 = np.zeros(n - 1)
    d2 = np.zeros(n - 2)
    d0[: n - 2] += 1.0
    d0[1 : n - 1] += 4.0
    d0[2:] += 1.0
    d1[: n - 2] += -2.0
    d1[1 : n - 1] += -2.0
    d2 += 1.0
    w = np.ones(n)
    z = y.copy()
    for _ in range(iters):
        ab = np.zeros((3, n))
        ab[2] = lam * d0 + w
        ab[1, 1:] = lam * d1
        ab[0, 2:] = lam * d2
        z = scipy.linalg.solveh_banded(ab, w * y)
        w = np.where(y > z, p, 1.0 - p)
    return z


def ridge(X, Y, lam: float) -> np.ndarray:
    """(X^T X + lam I)^-1 X^T Y, Eq. PEC_Ridge."""
    X = np.asarray(X, F64)
    k = X.shape[1]
    return np.linalg.solve(X.T @ X + lam * np.eye(k), X.T @ np.asarray(Y, F64))


# ---------------------------------------------------------------------------
# Sec. 2.4 (fSEC): trendline
# ---------------------------------------------------------------------------


def savgol_trend(x, window: int, order: int) -> np.ndarray:
    """Savitzky-Golay trendline of each row: the value at j of the degree-
    `order` least-squares polynomial over the window centred at j; within half
    a window of either edge, the polynomial fitted to the first / last full
    window evaluated at j."""
    x = np.asarray(x, F64)
    M = x.shape[-1]
    if window > M or window % 2 == 0 or window <= order:
        raise ValueError("bad Savitzky-Golay window")
    h = window // 2
    t = np.arange(-h, h + 1, dtype=F64)
    V = np.vander(t, order + 1, increasing=True)  # window x (order+1)
    fit = np.linalg.pinv(V)  # (order+1) x window: polynomial coefficients
    out = np.empty_like(x)
    rows = x.reshape(-1, M)
    o = out.reshape(-1, M)
    centre = fit[0]  # value of the polynomial at t = 0
    for r in range(rows.shape[0]):
        for j in range(h, M - h):
            o[r, j] = centre @ rows[r, j - h : j + h + 1]
        c_lo = fit @ rows[r, :window]
        c_hi = fit @ rows[r, M - window :]
        for j in range(h):
            o[r, j] = np.polyval(c_lo[::-1], j - h)
            o[r, M - h + j] = np.polyval(c_hi[::-1], j + 1)
    return out


def trend(x, mode: str, window: int, order: int) -> np.ndarray:
    """The trendline operator M{} of Eq. fSEC_VT: Savitzky-Golay or the mean."""
    x = np.asarray(x, F64)
    if mode == "mean":
        return np.repeat(x.mean(axis=-1, keepdims=True), x.shape[-1], axis=-1)
    if mode == "sg":
        return savgol_trend(x, window, order)
    raise ValueError(mode)


# ---------------------------------------------------------------------------
# Sec. 2.2-2.5: fKK-EC fit and reconstruction; Sec. 2.6: ML apply
# ---------------------------------------------------------------------------


@dataclass
class Basis:
    """The trained artefacts listed in Sec. 2.6 (f, S, V, Phi_PEC, V_SEC),
    in the combined form used by the reconstruction Eq. fKKEC."""

    f: np.ndarray  # (M,)
    s: np.ndarray  # (k,) singular values
    V: np.ndarray  # (M, k) right singular vectors of A
    B: np.ndarray  # (k, M) V^T / f
    H_B: np.ndarray  # (k, M) H{V^T / f}
    phi_pec_t: np.ndarray  # (k, M) Phi_PEC^T
    H_phi: np.ndarray  # (k, M) H{Phi_PEC^T}
    v_sec_t: np.ndarray  # (k, M) V_SEC^T
    c_amp: np.ndarray  # (k, M) V^T/f + H{Phi_PEC} - V_SEC^T
    c_ph: np.ndarray  # (k, M) H{V^T/f} - Phi_PEC^T
    i_ref: np.ndarray  # (M,)
    params: FitParams
    extras: dict = field(default_factory=dict)


def reconstruct(P, c_amp, c_ph):
    """Eq. fKKEC with U S = P: K = exp(P C_amp) exp(i P C_ph).
    Returns (Re K, Im K)."""
    P = np.asarray(P, F64)
    amp = np.exp(P @ c_amp)
    ph = P @ c_ph
    return amp * np.cos(ph), amp * np.sin(ph)


def basis_math(V, P, f, params: FitParams, L: int):
    """fKK, fPEC and fSEC on the k basis vectors (Secs. 2.2-2.4).

    V: (M, k) right singular vectors of A; P = A V = U S (N, k); f: (M,).
    Returns the Basis pieces (without s / i_ref) and the row set q."""
    V = np.asarray(V, F64)
    P = np.asarray(P, F64)
    f = np.asarray(f, F64)
    M, k = V.shape
    B = V.T / f  # V^T / f(w)
    H_B = hilbert(B, L)  # fKK: H{V^T / f}, Eq. fKK (scaled form)
    q = np.zeros(0, np.int64)
    phi_pec_t = np.zeros((k, M))
    if params.pec:
        q = select_rows(P)
        X = P[q]  # U_ss S
        phi_ph = X @ H_B  # U_ss S H{V^T/f}
        lam_als = params.als_lambda if params.als_lambda is not None else default_als_lambda(M)
        phi_err = np.stack([als_baseline(r, lam_als, params.als_p, params.als_iters) for r in phi_ph])
        lam_r = params.ridge_rel * float(np.sum(X * X)) / k
        phi_pec_t = ridge(X, phi_err, lam_r)  # Eq. PEC_Ridge
    H_phi = hilbert(phi_pec_t, L)
    corrected = B + H_phi  # PEC-corrected log-amplitude basis, Eq. fPEC_K
    if params.sec:
        win = params.sg_window or default_sg_window(M)
        v_sec_t = trend(corrected, params.sec_mode, win, params.sg_order)  # Eq. fSEC_VT
    else:
        v_sec_t = np.zeros((k, M))
    c_amp = corrected - v_sec_t
    c_ph = H_B - phi_pec_t
    return B, H_B, phi_pec_t, H_phi, v_sec_t, c_amp, c_ph, q


def fit(i_cars, i_ref, params: FitParams, f=None, out_rows=None, chunk: int = 65536):
    """Full fKK-EC (Fig. 1(b)): A, Gram, eigen, top-k, fKK, fPEC, fSEC, and the
    reconstruction Eq. fKKEC.

    The Gram matrix and P = A V are accumulated over row blocks of `chunk`
    rows (the same sums in block order) so a large cube fits in memory.
    Returns (Basis, P, result) where result holds Im/Re K for `out_rows`
    (all rows if None), the eigenvalues and q."""
    i_cars = np.asarray(i_cars)
    N, M = i_cars.shape
    L = params.pad_len or pad_len(M)
    f = np.ones(M) if f is None else np.asarray(f, F64)
    def blocks():
        for a in range(0, N, chunk):
            yield a, log_ratio(i_cars[a : a + chunk], i_ref, f, params.ratio_floor)

    G = None
    if params.svd == "randomized":
        if not params.k:
            raise ValueError("the randomised SVD needs a fixed k")
        k = params.k

        def matvec(X):
            out = np.empty((N, X.shape[1]))
            for a, A in blocks():
                out[a : a + A.shape[0]] = A @ X
            return out

        def rmatvec(Y):
            out = np.zeros((M, Y.shape[1]))
            for a, A in blocks():
                out += A.T @ Y[a : a + A.shape[0]]
            return out

        lam, V = rsvd(matvec, rmatvec, N, M, k, params.rsvd_oversample, params.rsvd_power_iters, params.rsvd_seed)
    elif params.svd == "exact":
        G = np.zeros((M, M))
        for _, A in blocks():
            G += A.T @ A
        lam, Vall = eig_desc(G)
        k = params.k or rank_k(lam, N, M, params.k_max, params.rank_eps)
        V = Vall[:, :k]
        if params.refine_steps:
            lam_k, V = refine_basis(G, V, params.refine_steps)
            lam = np.concatenate([lam_k, lam[k:]])
    else:
        raise ValueError(params.svd)
    s = singular_from_eig(lam[:k])
    P = np.empty((N, k))
    for a in range(0, N, chunk):
        P[a : a + chunk] = log_ratio(i_cars[a : a + chunk], i_ref, f, params.ratio_floor) @ V
    B, H_B, phi_pec_t, H_phi, v_sec_t, c_amp, c_ph, q = basis_math(V, P, f, params, L)
    basis = Basis(f, s, V, B, H_B, phi_pec_t, H_phi, v_sec_t, c_amp, c_ph,
                  np.asarray(i_ref, F64), params, {"lam": lam, "q": q, "G": G, "k": k,
                   "energy": float(np.trace(G)) if G is not None else float(sum(np.sum(A * A) for _, A in blocks()))})
    rows = slice(None) if out_rows is None else out_rows
    re, im = reconstruct(P[rows], c_amp, c_ph)
    return basis, P, {"re": re, "im": im, "lam": lam, "q": q, "k": k}


def apply_projector(basis: Basis) -> np.ndarray:
    """W with U_new S = A_new W: Eq. ML_Unew read as the ridge solution
    U_new = A_new X^T (X X^T + lambda I)^-1, X = S V^T, which gives
    U_new S = A_new V diag(s^2 / (s^2 + lambda))."""
    s = basis.s
    lam = basis.params.ml_lambda
    return basis.V * (s**2 / (s**2 + lam))[None, :]


def apply(basis: Basis, i_new, out_rows=None):
    """ML:fKK-EC (Sec. 2.6): project new spectra on the trained basis and
    reuse Eq. fKKEC.  Returns (Re K, Im K)."""
    A = log_ratio(i_new if out_rows is None else np.asarray(i_new)[out_rows],
                  basis.i_ref, basis.f, basis.params.ratio_floor)
    P = A @ apply_projector(basis)
    return reconstruct(P, basis.c_amp, basis.c_ph)
