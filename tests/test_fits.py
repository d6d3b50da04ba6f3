"""Host fits on synthetic series with known answers (no GPU)."""
import numpy as np

from paper_2303_08163_gb300 import fits


def test_energy_decay_rate_exact_exponential():
    t = np.arange(0, 500, 10.0)
    assert abs(fits.energy_decay_rate(t, 3.0 * np.exp(-2.5e-3 * t)) - 2.5e-3) < 1e-12


def test_mode_multipliers_recover_two_modes():
    """Two damped travelling modes seen through two channels (like rho and j_x)."""
    lam = np.array([0.999 * np.exp(-0.3j), 0.998 * np.exp(0.2j)])
    vec = np.array([[1.0, 0.4 - 0.1j], [0.5 + 0.2j, 1.0]])
    amp = np.array([1e-4, 7e-5])
    s = np.arange(300)
    series = (vec[:, None, :] * (amp[None, :] * lam[None, :] ** s[:, None])[None]).sum(axis=2).T
    mu = fits.mode_multipliers(series, nmodes=2)
    for m in lam:
        assert np.min(np.abs(mu - m)) < 1e-10


def test_per_step_branch_and_rates():
    """lambda^K loses the phase branch; a hint one branch away recovers it."""
    k, c, gamma, K = 0.4, 0.9, 1e-3, 10
    lam = np.exp(-gamma - 1j * k * c)        # exp(-i Omega), Omega = k c - i gamma
    mu = lam ** K
    got = fits.per_step(mu, K, phase_hint=-k * c * 1.05)
    decay, speed = fits.rates(got, k)
    assert abs(decay - gamma) < 1e-12 and abs(speed - c) < 1e-12
