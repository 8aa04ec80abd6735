"""Seeded synthetic CARS hyperspectral cubes (the input generator).

This module holds the forward model only: the CARS signal model of Eq. ICARS
(Sec. 2.1), a Lorentzian resonant susceptibility chi_R = sum_s A_s/(Omega_s - w
- i Gamma_s) with a constant real chi_NR (the form assumed below Eq.
Mean_PEC_Corrected_Magnitude), and the surrogate relation I_ref = Xi xi(w)
I_NRB of Eq. K.  No step of the fKK-EC method (logarithm of ratios, Hilbert
transform, factorisation, error correction) is computed here, so both the
oracle and the CUDA path can consume these cubes without sharing arithmetic.

Recipe (stand-in for the paper's simulation of Sec. 4.1 and its chicken
cartilage image of Sec. 4.2, neither of which is available):

* grid: w_j linear on [w_min, w_max] with M points;
* S species, one Lorentzian each: Omega ~ U(band), Gamma ~ U(5, 20) cm^-1,
  A = a * Gamma with a ~ U(0.05, 0.5) (so the peak of Im chi_R is a);
* concentration maps: per species, U(0,1) noise on the H x W pixel grid,
  periodic Gaussian blur (sigma = 4 px), min-max normalised to [0, 1];
* stimulation envelope C(w) = exp(-(w - 2150)^2 / (2 * 1200^2)), so
  I_NRB = C^2 chi_NR^2 and I_CARS = C^2 |chi_R + chi_NR|^2 + noise;
* noise "gauss": sigma(w) = <I_clean>(w) / snr;  "poisson_gauss": with the
  band mean Ibar of <I_clean>, total sigma = Ibar/snr split half/half in
  variance between a Poisson term (I = alpha * Poisson(I_clean/alpha)) and
  additive Gaussian sigma_g;
* surrogate: I_ref = Xi * xi(w) * I_NRB with Xi = 1.05 and
  ln xi = -2 eps sum_{j=1..3} b_j cos(2 pi j u + theta_j), u the normalised
  band coordinate; eps is set so that the nominal phase error of the
  continuous transform, eps * max_u |sum_j b_j sin(2 pi j u + theta_j)|,
  equals 0.05 rad.

Random numbers come from numpy's PCG64 streams keyed by (seed, image, chunk),
so a cube does not depend on the thread count used to build it.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

CHUNK_ROWS = 16384


@dataclass(frozen=True)
class CubeSpec:
    height: int
    width: int
    n_channels: int
    n_species: int
    noise: str = "gauss"  # "gauss" | "poisson_gauss" | "none"
    snr: float = 50.0
    seed: int = 1001
    w_min: float = 500.0
    w_max: float = 3800.0
    gamma_min: float = 5.0
    gamma_max: float = 20.0
    amp_min: float = 0.05
    amp_max: float = 0.5
    blur_px: float = 4.0
    xi_scale: float = 1.05
    phase_err: float = 0.05
    envelope_center: float = 2150.0
    envelope_width: float = 1200.0
    chi_nr: float = 1.0

    @property
    def n_spectra(self) -> int:
        return self.height * self.width


# Workloads: shapes and noise of the paper-shaped benchmarks.
CONFIGS = {
    # 64 x 64 pixels, 512 channels, 8 species, Gaussian noise at SNR 50.
    "img64_m512": CubeSpec(64, 64, 512, 8, "gauss", 50.0, seed=1001),
    # 846 x 831 = 703,026 pixels (the stitched tissue image size of Sec. 4.2),
    # 1,000 channels, 30 species, Poisson + Gaussian noise at SNR 20.
    "img846x831_m1000": CubeSpec(846, 831, 1000, 30, "poisson_gauss", 20.0, seed=1002),
    # 400 x 500 = 200,000-pixel training cube for the served (ML) form.
    "train400x500_m1000": CubeSpec(400, 500, 1000, 30, "poisson_gauss", 20.0, seed=1004),
}


# The batched multi-image workload: 16 independent cubes, each its own scene
# (species, NRB, surrogate) with sides, channel counts and k drawn from the
# lists below by the seeded stream 1005; cube i has seed 1005 + i.
MULTI_SIDES = (128, 256, 512, 1024)
MULTI_CHANNELS = (512, 878, 1000, 1600)
MULTI_K = (10, 20, 40, 80)


def multi_image_specs(count: int = 16, seed: int = 1005):
    """(CubeSpec, k) of each cube of the multi-image workload."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        side = int(rng.choice(MULTI_SIDES))
        m = int(rng.choice(MULTI_CHANNELS))
        k = int(rng.choice(MULTI_K))
        species = int(rng.integers(8, 31))
        out.append((CubeSpec(side, side, m, species, "gauss", 50.0, seed=seed + i), k))
    return out


@dataclass
class Scene:
    """Species, NRB and surrogate shared by every image drawn from one spec."""

    spec: CubeSpec
    omega: np.ndarray  # (M,) float64, cm^-1
    omega0: np.ndarray  # (S,) centres
    gamma: np.ndarray  # (S,) widths
    amp: np.ndarray  # (S,) A_s = a_s * Gamma_s
    envelope: np.ndarray  # (M,) C(w)
    i_nrb: np.ndarray  # (M,) float64
    i_ref: np.ndarray  # (M,) float64 surrogate
    ln_xi: np.ndarray  # (M,)
    noise_sigma: np.ndarray | None = None  # (M,) for "gauss"
    alpha: float = 0.0
    sigma_g: float = 0.0
    lor_re: np.ndarray = field(default=None, repr=False)  # (S, M)
    lor_im: np.ndarray = field(default=None, repr=False)

    @classmethod
    def from_spec(cls, spec: CubeSpec) -> "Scene":
        rng = np.random.default_rng(np.random.SeedSequence([spec.seed, 0]))
        M, S = spec.n_channels, spec.n_species
        omega = np.linspace(spec.w_min, spec.w_max, M)
        omega0 = rng.uniform(spec.w_min, spec.w_max, S)
        gamma = rng.uniform(spec.gamma_min, spec.gamma_max, S)
        amp = rng.uniform(spec.amp_min, spec.amp_max, S) * gamma
        env = np.exp(-((omega - spec.envelope_center) ** 2) / (2.0 * spec.envelope_width**2))
        i_nrb = env**2 * spec.chi_nr**2
        # smooth surrogate error: 3-term cosine series over the band
        b = rng.uniform(0.5, 1.0, 3) / np.arange(1, 4)
        theta = rng.uniform(0.0, 2.0 * np.pi, 3)
        j = np.arange(1, 4)[:, None]
        u_fine = np.linspace(0.0, 1.0, 8193)
        peak = np.abs((b[:, None] * np.sin(2 * np.pi * j * u_fine + theta[:, None])).sum(0)).max()
        eps = spec.phase_err / peak
        u = (omega - spec.w_min) / (spec.w_max - spec.w_min)
        ln_xi = -2.0 * eps * (b[:, None] * np.cos(2 * np.pi * j * u + theta[:, None])).sum(0)
        i_ref = spec.xi_scale * np.exp(ln_xi) * i_nrb
        den = (omega0[:, None] - omega[None, :]) ** 2 + gamma[:, None] ** 2
        lor_re = amp[:, None] * (omega0[:, None] - omega[None, :]) / den
        lor_im = amp[:, None] * gamma[:, None] / den
        return cls(spec, omega, omega0, gamma, amp, env, i_nrb, i_ref, ln_xi,
                   lor_re=lor_re, lor_im=lor_im)

    # -- concentrations -------------------------------------------------
    def concentrations(self, height: int, width: int, image: int) -> np.ndarray:
        """(H*W, S) smooth maps in [0, 1] (periodic Gaussian blur)."""
        rng = np.random.default_rng(np.random.SeedSequence([self.spec.seed, 1, image]))
        S = self.spec.n_species
        ky = np.fft.fftfreq(height)[:, None]
        kx = np.fft.fftfreq(width)[None, :]
        kern = np.exp(-2.0 * np.pi**2 * self.spec.blur_px**2 * (kx**2 + ky**2))
        out = np.empty((height * width, S))
        for s in range(S):
            u = rng.uniform(size=(height, width))
            sm = np.fft.ifft2(np.fft.fft2(u) * kern).real
            lo, hi = sm.min(), sm.max()
            out[:, s] = ((sm - lo) / (hi - lo if hi > lo else 1.0)).ravel()
        return out

    # -- clean intensities ------------------------------------------------
    def chi_r(self, conc: np.ndarray):
        """Resonant susceptibility (real, imag) for rows of concentrations."""
        return conc @ self.lor_re, conc @ self.lor_im

    def clean(self, conc: np.ndarray) -> np.ndarray:
        re, im = self.chi_r(conc)
        nr = self.spec.chi_nr
        return self.envelope[None, :] ** 2 * ((re + nr) ** 2 + im**2)

    def truth_im(self, conc: np.ndarray) -> np.ndarray:
        """Im{chi/chi_NR} = Im{chi_R}/chi_NR for rows of concentrations."""
        return self.chi_r(conc)[1] / self.spec.chi_nr

    def set_noise(self, mean_clean: np.ndarray) -> None:
        sp = self.spec
        if sp.noise == "gauss":
            self.noise_sigma = mean_clean / sp.snr
        elif sp.noise == "poisson_gauss":
            ibar = float(mean_clean.mean())
            tot = ibar / sp.snr
            self.alpha = tot**2 / (2.0 * ibar)
            self.sigma_g = tot / np.sqrt(2.0)
        elif sp.noise != "none":
            raise ValueError(f"unknown noise model {sp.noise!r}")

    def noisy(self, clean: np.ndarray, rng: np.random.Generator) -> np.ndarray:
        sp = self.spec
        if sp.noise == "gauss":
            return clean + rng.standard_normal(clean.shape) * self.noise_sigma[None, :]
        if sp.noise == "poisson_gauss":
            counts = rng.poisson(clean / self.alpha)
            return self.alpha * counts + self.sigma_g * rng.standard_normal(clean.shape)
        return clean


@dataclass
class Cube:
    scene: Scene
    conc: np.ndarray  # (N, S)
    i_cars: np.ndarray  # (N, M) float32
    i_ref: np.ndarray  # (M,) float32
    image: int

    @property
    def omega(self):
        return self.scene.omega

    @property
    def alpha(self):
        return self.scene.alpha

    @property
    def sigma_g(self):
        return self.scene.sigma_g

    def truth_im(self, rows=None) -> np.ndarray:
        c = self.conc if rows is None else self.conc[rows]
        return self.scene.truth_im(c)


def _threads() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def _render(scene: Scene, conc: np.ndarray, image: int, out: np.ndarray | None,
            noise: bool) -> np.ndarray:
    n = conc.shape[0]
    M = scene.spec.n_channels
    if out is None:
        out = np.empty((n, M), np.float32)
    starts = list(range(0, n, CHUNK_ROWS))

    def work(ci):
        a = starts[ci]
        b = min(n, a + CHUNK_ROWS)
        cl = scene.clean(conc[a:b])
        if noise:
            rng = np.random.default_rng(np.random.SeedSequence([scene.spec.seed, 2, image, ci]))
            cl = scene.noisy(cl, rng)
        out[a:b] = cl
        return None

    with ThreadPoolExecutor(_threads()) as ex:
        list(ex.map(work, range(len(starts))))
    return out


def _mean_clean(scene: Scene, conc: np.ndarray) -> np.ndarray:
    n = conc.shape[0]
    acc = np.zeros(scene.spec.n_channels)
    for a in range(0, n, CHUNK_ROWS):
        acc += scene.clean(conc[a : a + CHUNK_ROWS]).sum(0)
    return acc / n


def make_cube(spec: CubeSpec, *, image: int = 0, height: int | None = None,
              width: int | None = None, scene: Scene | None = None) -> Cube:
    """Draw one image of the scene.  Image 0 fixes the noise level of the
    scene (from its own clean mean spectrum); later images reuse it, so a
    stream of tiles shares species, NRB, surrogate and noise model."""
    if scene is None:
        scene = Scene.from_spec(spec)
    h = spec.height if height is None else height
    w = spec.width if width is None else width
    conc = scene.concentrations(h, w, image)
    if scene.noise_sigma is None and scene.alpha == 0.0 and spec.noise != "none":
        scene.set_noise(_mean_clean(scene, conc))
    i_cars = _render(scene, conc, image, None, spec.noise != "none")
    return Cube(scene, conc, i_cars, scene.i_ref.astype(np.float32), image)


def make_tiled_cube(spec: CubeSpec, base: int = 128) -> Cube:
    """A cube of the spec's size made by repeating a base x base draw of its
    scene over the image (the full-size multi-image cubes, whose fit cost
    does not depend on the repetition, without drawing up to 10^6 spectra
    each); spec.height and spec.width must be multiples of base."""
    if spec.height % base or spec.width % base:
        raise ValueError("cube sides must be multiples of the base tile")
    c = make_cube(spec, height=base, width=base)
    ry, rx = spec.height // base, spec.width // base
    img = c.i_cars.reshape(base, base, -1)
    full = np.tile(img, (ry, rx, 1)).reshape(spec.height * spec.width, -1)
    conc = np.tile(c.conc.reshape(base, base, -1), (ry, rx, 1)).reshape(spec.height * spec.width, -1)
    return Cube(c.scene, conc, np.ascontiguousarray(full), c.i_ref, c.image)


def tile_stream(scene: Scene, sizes, first_image: int = 1):
    """Yield (image_id, Cube) tiles of the given spectrum counts, each a
    1-pixel-high strip with fresh concentrations and noise."""
    for i, n in enumerate(sizes):
        yield make_cube(scene.spec, image=first_image + i, height=1, width=int(n), scene=scene)


# ---------------------------------------------------------------------------
# The simulation-shaped workload of Sec. 4.1 (shape only: the paper's random
# draws are not published)
# ---------------------------------------------------------------------------

SIM_BASE = (74, 246)            # base image, 18,204 spectra
SIM_SIDE_SCALES = (0.5, 1, 2, 3, 4)
SIM_PEAKS = (22, 25, 10)        # Lorentzian peaks of chemicals 1, 2, 3


@dataclass
class SimCube:
    i_cars: np.ndarray   # (N, M) float32, noiseless
    i_ref: np.ndarray    # (M,) float32
    omega: np.ndarray    # (M,) cm^-1
    conc: np.ndarray     # (N, 3) concentrations, each row summing to 1
    chi_r: np.ndarray    # (3, M) complex resonant susceptibility of each chemical
    chi_nr: np.ndarray   # (3, M) real non-resonant susceptibility of each chemical

    def truth_im(self, rows=None) -> np.ndarray:
        """Im{chi / chi_nr} of the mixture: the ideal K_CARS's imaginary part."""
        c = self.conc if rows is None else self.conc[rows]
        chi = c @ (self.chi_r + self.chi_nr)
        return (chi / (c @ self.chi_nr)).imag


def make_sim_cube(side_scale: float = 1.0, seed: int = 2005, n_channels: int = 810) -> SimCube:
    """A noiseless three-chemical mixture shaped like the simulation of
    Sec. 4.1: 810 channels over -500..2,500 cm^-1; chemicals with 22, 25 and
    10 complex Lorentzian peaks (centre U(500, 1700) cm^-1, width U(5, 20),
    amplitude U(0.02, 0.3) x width); each chemical's chi_nr a quadratic
    polynomial in the normalised frequency with non-negative random
    coefficients; chi_ref a linear polynomial with non-negative
    coefficients; I_CARS = |sum_s c_s (chi_R,s + chi_nr,s)|^2 and
    I_ref = chi_ref^2 (constant stimulation profile).  Concentrations: three
    smooth random maps on the 74 x 246 base image, normalised to sum to 1 at
    every pixel (a ternary mixture), then side-scaled by `side_scale` with
    bilinear resampling -- 0.5, 1, 2, 3, 4 give 4,551, 18,204, 72,816,
    163,836 and 291,264 spectra."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 7]))
    M = n_channels
    omega = np.linspace(-500.0, 2500.0, M)
    u = (omega - omega[0]) / (omega[-1] - omega[0])
    chi_r = np.zeros((3, M), complex)
    for s, npk in enumerate(SIM_PEAKS):
        om = rng.uniform(500.0, 1700.0, npk)
        g = rng.uniform(5.0, 20.0, npk)
        a = rng.uniform(0.02, 0.3, npk) * g
        chi_r[s] = (a[:, None] / (om[:, None] - omega[None, :] - 1j * g[:, None])).sum(0)
    coef = rng.uniform(0.2, 1.0, (3, 3))  # c0 + c1 u + c2 u^2, non-negative
    chi_nr = coef[:, :1] + coef[:, 1:2] * u[None, :] + coef[:, 2:3] * u[None, :] ** 2
    d = rng.uniform(0.3, 1.0, 2)
    chi_ref = d[0] + d[1] * u
    # ternary concentration maps on the base image
    h0, w0 = SIM_BASE
    ky = np.fft.fftfreq(h0)[:, None]
    kx = np.fft.fftfreq(w0)[None, :]
    kern = np.exp(-2.0 * np.pi**2 * 6.0**2 * (kx**2 + ky**2))
    maps = np.stack([np.fft.ifft2(np.fft.fft2(rng.uniform(size=(h0, w0))) * kern).real for _ in range(3)])
    maps = maps - maps.min(axis=(1, 2), keepdims=True) + 0.05
    maps = maps / maps.sum(0, keepdims=True)
    h, w = int(round(h0 * side_scale)), int(round(w0 * side_scale))
    conc = np.stack([_bilinear(mp, h, w) for mp in maps], axis=-1).reshape(h * w, 3)
    conc = conc / conc.sum(1, keepdims=True)
    chi = conc @ (chi_r + chi_nr)
    i_cars = (np.abs(chi) ** 2).astype(np.float32)
    return SimCube(i_cars, (chi_ref**2).astype(np.float32), omega, conc, chi_r, chi_nr)


def _bilinear(img: np.ndarray, h: int, w: int) -> np.ndarray:
    """Resample img to h x w, pixel centres aligned (edge-clamped)."""
    h0, w0 = img.shape
    y = np.clip((np.arange(h) + 0.5) * h0 / h - 0.5, 0.0, h0 - 1.0)
    x = np.clip((np.arange(w) + 0.5) * w0 / w - 0.5, 0.0, w0 - 1.0)
    y0 = np.floor(y).astype(int)
    x0 = np.floor(x).astype(int)
    y1 = np.minimum(y0 + 1, h0 - 1)
    x1 = np.minimum(x0 + 1, w0 - 1)
    fy = (y - y0)[:, None]
    fx = (x - x0)[None, :]
    top = img[y0][:, x0] * (1 - fx) + img[y0][:, x1] * fx
    bot = img[y1][:, x0] * (1 - fx) + img[y1][:, x1] * fx
    return top * (1 - fy) + bot * fy
