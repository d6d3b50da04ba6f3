"""Host-side fits of the measured series (post-processing, not part of the step).

* ``energy_decay_rate``: least-squares slope of ln E(t) (Sec. V.B.2: the pressure-wave
  energy decays as exp(-2 nu A' k^2 t)).
* ``mode_multipliers``: dynamic mode decomposition of a probe series.  The probes of one
  instance (rho, j_x, j_y projected on exp(-i k.r) every K steps) follow
  v(s + 1) = M v(s) once the fast non-hydrodynamic modes have decayed; the eigenvalues
  of the least-squares M are the per-sample multipliers mu = lambda^K of the
  hydrodynamic modes.
* ``per_step``: lambda from mu.  The modulus is unambiguous; the phase per sample is
  known only modulo 2 pi, so the branch is chosen nearest to a given per-step phase
  estimate (e.g. -k c from the closed-form sound speed) and the choice is reported.
* ``rates``: decay per step -ln|lambda| and phase speed -arg(lambda)/|k| (convention of
  the von Neumann eigenproblem, Eq. eq:VN_eigen, with perturbations exp(i (k.r - w t))).
"""
import numpy as np


def energy_decay_rate(t, energy, skip=0):
    """Slope of -ln E against t (least squares), after dropping `skip` samples."""
    t = np.asarray(t, dtype=np.float64)[skip:]
    e = np.asarray(energy, dtype=np.float64)[skip:]
    return float(-np.polyfit(t, np.log(e), 1)[0])


def mode_multipliers(series, nmodes=None, skip=0):
    """Eigenvalues (per sample) of the least-squares linear map between consecutive
    samples of a complex series with shape (samples, channels)."""
    X = np.asarray(series, dtype=np.complex128)[skip:]
    if X.ndim == 1:
        X = X[:, None]
    # drop channels that carry no signal
    scale = np.max(np.abs(X), axis=0)
    keep = scale > 1e-12 * max(float(scale.max()), 1e-300)
    X = X[:, keep] / scale[keep]
    X0, X1 = X[:-1], X[1:]
    M, *_ = np.linalg.lstsq(X0, X1, rcond=None)
    mu = np.linalg.eigvals(M)
    mu = mu[np.argsort(-np.abs(mu))]
    return mu if nmodes is None else mu[:nmodes]


def per_step(mu, every_k, phase_hint=0.0):
    """Per-step multiplier from a per-sample multiplier mu = lambda^K; the phase branch
    is the one closest to K * phase_hint (phase_hint = expected arg(lambda))."""
    mu = np.asarray(mu, dtype=np.complex128)
    mag = np.abs(mu) ** (1.0 / every_k)
    base = np.angle(mu)
    m = np.round((every_k * np.asarray(phase_hint) - base) / (2 * np.pi))
    return mag * np.exp(1j * (base + 2 * np.pi * m) / every_k)


def rates(lam, k):
    """(decay per step, phase speed) of per-step multipliers for wave number |k|."""
    lam = np.asarray(lam, dtype=np.complex128)
    return -np.log(np.abs(lam)), -np.angle(lam) / k
