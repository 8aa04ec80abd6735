"""The simulation-shaped workload (Sec. 4.1; shape only): sizes, the
forward model and its ideal output."""
import numpy as np

from paper_2005_07132_gb300.synth import SIM_PEAKS, SIM_SIDE_SCALES, make_sim_cube


def test_sim_sizes_match_the_paper():
    """Side scales 0.5, 1, 2, 3, 4 of the 74 x 246 base give the paper's
    4,551, 18,204, 72,816, 163,836 and 291,264 spectra of 810 channels."""
    want = [4551, 18204, 72816, 163836, 291264]
    for s, n in zip(SIM_SIDE_SCALES, want):
        c = make_sim_cube(s)
        assert c.i_cars.shape == (n, 810)
    assert SIM_PEAKS == (22, 25, 10)


def test_sim_forward_model():
    c = make_sim_cube(0.5, seed=3)
    assert np.allclose(c.conc.sum(1), 1.0) and np.all(c.conc > 0)       # ternary mixture
    assert np.all(c.chi_nr > 0)                                          # non-negative coefficients
    u = (c.omega - c.omega[0]) / (c.omega[-1] - c.omega[0])
    for s in range(3):                                                   # quadratic chi_nr
        assert np.allclose(np.polyval(np.polyfit(u, c.chi_nr[s], 2), u), c.chi_nr[s])
    ref = np.sqrt(c.i_ref.astype(np.float64))                            # linear chi_ref
    assert np.allclose(np.polyval(np.polyfit(u, ref, 1), u), ref, rtol=1e-6)
    peaks = c.omega[np.argmax(np.abs(c.chi_r.imag), axis=1)]
    assert np.all((peaks > 450) & (peaks < 1750))                        # Raman band 500-1700
    # noiseless: I = |chi|^2 exactly (to float32 rounding)
    chi = c.conc @ (c.chi_r + c.chi_nr)
    np.testing.assert_allclose(c.i_cars, np.abs(chi) ** 2, rtol=2e-7)


def test_sim_truth_is_the_ideal_kk_output():
    """With the true NRB as the reference, K = chi / chi_nr, whose imaginary
    part is truth_im (Eq. KCARS); checked directly from the susceptibilities."""
    c = make_sim_cube(0.5, seed=4)
    rows = np.arange(0, c.i_cars.shape[0], 97)
    chi = c.conc[rows] @ (c.chi_r + c.chi_nr)
    nr = c.conc[rows] @ c.chi_nr
    np.testing.assert_allclose(c.truth_im(rows), (chi / nr).imag, rtol=0, atol=1e-15)
