"""Tolerance of the full-size sampled-cell checks (shared by tests/test_gpu_fullsize.py
and the CPU test of its power, tests/test_fullsize_power.py).

Each binary16 (FP32) store rounds f - w rho0 by at most half an ulp: u = 2^-11 (2^-24)
relative; below 2^-14 a binary16 value is a subnormal, rounded to a multiple of 2^-24, an
absolute error of up to 2^-25.  A sampled value after n steps has been rounded n + 1
times directly; the roundings of the other populations reach it through rho and u, to
first order amplified by at most omega K (omega = 1/tau, K the bound of `sensitivity` on
|d f^eq_i / d f_j| / w_i at the field's largest |u_a|); the FP32 collision is a chain of
at most 32 roundings of operands bounded by w_i (1 + S).  So, with S = sum_j |f_j - w_j|,

  |f_gpu - f_ref| <= (n + 2) [u (|f_i - w_i| + omega K w_i S) + 2^-25 (1 + omega K Q w_i)]
                     + 32 n 2^-24 w_i (1 + S) (1 + omega K)

(the 2^-25 term for binary16 only).  A data-movement error (a wrong neighbour, direction
or layout) changes f_i by the difference of f_i between neighbouring cells: of order
w_i |grad(rho, u)| on a smooth field, which at 512^3 lies inside this bound, and of order
w_i |delta rho + 3 delta u| on a field that varies from cell to cell, far outside it.
"""
import numpy as np

UNIT = {1: 2.0 ** -24, 2: 2.0 ** -11}
# half the spacing of the subnormal numbers: below 2^-14 a binary16 store rounds to a
# multiple of 2^-24, an absolute error of up to 2^-25 that no relative bound covers
FLOOR = {1: 0.0, 2: 2.0 ** -25}


def sensitivity(D, umax, rho_min=0.9):
    """Bound K on |d f^eq_i / d f_j| / w_i for |u_a| <= umax, rho >= rho_min: f^eq_i =
    w_i rho (1 + h_i(u)) with u = j / rho, so a change of f_j moves f^eq_i through rho
    (factor 1 + |h_i|) and through u (factor sum_a |dh_i/du_a| (1 + |u_a|) / rho).  For the
    entropic and product forms h_i = prod_a t_a - 1 with t <= 1 + 3u + 3u^2 and |dt/du| <=
    3 + 6u; for the quadratic form |dh/du_a| <= 3 + 9 D u + 3u."""
    t = 1 + 3 * umax + 3 * umax ** 2
    hmax = max(t ** D - 1, 3 * D * umax + 4.5 * (D * umax) ** 2 + 1.5 * D * umax ** 2)
    g = max((3 + 6 * umax) * t ** (D - 1), 3 + 9 * D * umax + 3 * umax)
    return 1 + hmax + D * g * (1 + umax) / rho_min


def sampled_tolerance(ref, w, D, tau, prec, nsteps, umax, rho_min=0.9):
    """Per-population bound on |f_gpu - f_ref| for reference populations ref (m, Q)."""
    shifted = np.abs(ref - w)
    S = shifted.sum(axis=1, keepdims=True)
    ok = (1.0 / tau) * sensitivity(D, umax, rho_min)
    return ((nsteps + 2) * UNIT[prec] * (shifted + ok * w * S)
            + (nsteps + 2) * FLOOR[prec] * (1 + ok * w * len(w))
            + 32 * nsteps * 2.0 ** -24 * w * (1 + S) * (1 + ok))
