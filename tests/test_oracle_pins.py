"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test would fail for a plausible mistake in the oracle: a dropped term or wrong sign
in an equilibrium (moment identities, minimiser, P* closed form), a transposed velocity
component (axis-permutation symmetry), a wrong streaming direction (free flight, advected
shear wave), a wrong tau-nu relation (Taylor-Green decay), or a wrong bulk coefficient or
local collision frequency (von Neumann acoustic dissipation against the Chapman-Enskog
result of Sec. IV).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import analysis, core
from paper_2303_08163_gb300 import inputs

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
EQS = [core.EQ_ENTROPIC, core.EQ_POLY2, core.EQ_PRODUCT]
VS2 = 1.0 / 3.0


def rand_states(D, n, seed, umax=0.9):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.5, 2.0, n), rng.uniform(-umax, umax, (n, D))


# ----------------------------------------------------------------------------- lattice

@pytest.mark.parametrize("D", [1, 2, 3])
def test_lattice_weights_and_isotropy(D):
    """Sec. II: D1Q3 weights {1/6, 2/3, 1/6}; tensor products; sum w c c = vs^2 delta."""
    c, w = core.lattice(D)
    assert len(w) == 3 ** D
    np.testing.assert_allclose(core.lattice(1)[1], GOLD["d1q3_weights"]["value"], rtol=0, atol=1e-16)
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(c[:, :D].T @ w, 0.0, atol=1e-16)
    second = (c[:, :D].T * w) @ c[:, :D]
    np.testing.assert_allclose(second, VS2 * np.eye(D), atol=1e-15)
    # population index convention and opposite = Q - 1 - i
    Q = len(w)
    for i in range(Q):
        np.testing.assert_array_equal(c[Q - 1 - i], -c[i])
        assert i == sum((c[i, a] + 1) * 3 ** a for a in range(D))
        assert all(c[i, a] == 0 for a in range(D, 3))
    if D == 2:
        assert sorted(set(np.round(w * 36).astype(int))) == [1, 4, 16]
    if D == 3:
        assert sorted(set(np.round(w * 216).astype(int))) == [1, 4, 16, 64]


# ----------------------------------------------------------------------------- equilibria

@pytest.mark.parametrize("D", [1, 2, 3])
@pytest.mark.parametrize("eq", EQS)
def test_feq_mass_momentum(D, eq):
    """Constraints of Sec. II.A: sum f^eq = rho, sum c f^eq = rho u (all three forms)."""
    c, _ = core.lattice(D)
    rhos, us = rand_states(D, 40, 11 + D + 7 * eq, umax=0.9 if eq == core.EQ_ENTROPIC else 0.5)
    for rho, u in zip(rhos, us):
        f = core.feq(D, eq, rho, u)
        assert abs(f.sum() - rho) < 2e-14 * rho
        np.testing.assert_allclose(c[:, :D].T @ f, rho * u, atol=2e-14 * rho)


@pytest.mark.parametrize("D", [1, 2, 3])
@pytest.mark.parametrize("eq", EQS)
def test_feq_rest_state(D, eq):
    """f^eq(rho, 0) = w_i rho for every form."""
    _, w = core.lattice(D)
    for rho in (0.7, 1.0, 1.9):
        np.testing.assert_allclose(core.feq(D, eq, rho, np.zeros(D)), w * rho, rtol=1e-15, atol=0)


@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("eq", EQS)
def test_feq_mirror_and_axis_symmetry(D, eq):
    """f^eq_i(rho, u) = f^eq_opp(i)(rho, -u); swapping two velocity components permutes
    the populations the same way (catches a transposed operand)."""
    c, _ = core.lattice(D)
    Q = len(c)
    rhos, us = rand_states(D, 10, 5 + D, umax=0.4)
    for rho, u in zip(rhos, us):
        f = core.feq(D, eq, rho, u)
        fm = core.feq(D, eq, rho, -u)
        np.testing.assert_allclose(f[::-1], fm, rtol=1e-14)
        us_ = u.copy()
        us_[[0, 1]] = us_[[1, 0]]
        fs = core.feq(D, eq, rho, us_)
        perm = [int(np.nonzero((c[:, 0] == c[i, 1]) & (c[:, 1] == c[i, 0]) & (c[:, 2] == c[i, 2]))[0][0])
                for i in range(Q)]
        np.testing.assert_allclose(fs[perm], f, rtol=1e-14)


@pytest.mark.parametrize("D", [1, 2, 3])
def test_entropic_feq_is_H_minimiser(D):
    """Sec. II.A: the entropic equilibrium minimises H = sum f ln(f / w) under the mass and
    momentum constraints (Newton solve of the dual, no closed form used)."""
    rhos, us = rand_states(D, 12, 101 + D, umax=0.8)
    for rho, u in zip(rhos, us):
        f_min = analysis.newton_entropic(D, rho, u)
        np.testing.assert_allclose(core.feq(D, core.EQ_ENTROPIC, rho, u), f_min, rtol=5e-13)


@pytest.mark.parametrize("D", [2, 3])
def test_poly2_second_moments(D):
    """Eq. (eq:Poly2_isothermal_EDF) matches the Maxwell-Boltzmann pressure tensor:
    sum c_a c_b f^eq = rho (vs^2 delta_ab + u_a u_b)."""
    c, _ = core.lattice(D)
    C = c[:, :D].astype(float)
    rhos, us = rand_states(D, 10, 21 + D, umax=0.4)
    for rho, u in zip(rhos, us):
        f = core.feq(D, core.EQ_POLY2, rho, u)
        np.testing.assert_allclose((C.T * f) @ C, rho * (VS2 * np.eye(D) + np.outer(u, u)), atol=1e-14)


@pytest.mark.parametrize("D", [2, 3])
def test_product_form_second_moments(D):
    """Eq. (eq:Product_isothermal_EDF) enforces the diagonal second moments:
    sum c_a^2 f^eq = rho (vs^2 + u_a^2); its off-diagonal moments are rho u_a u_b."""
    c, _ = core.lattice(D)
    C = c[:, :D].astype(float)
    rhos, us = rand_states(D, 10, 31 + D, umax=0.4)
    for rho, u in zip(rhos, us):
        f = core.feq(D, core.EQ_PRODUCT, rho, u)
        np.testing.assert_allclose((C.T * f) @ C, rho * (VS2 * np.eye(D) + np.outer(u, u)), atol=1e-14)


def test_entropic_pressure_deviation_closed_form():
    """Sec. III.A: sum (c - u)^2 f^eq - rho vs^2 = -rho vs^2 [x^2 - 2 sqrt(x^2 + 1) + 2],
    x = u_a / vs, for the entropic equilibrium; zero for the polynomial forms."""
    for D in (1, 2, 3):
        rhos, us = rand_states(D, 10, 41 + D, umax=0.95)
        for rho, u in zip(rhos, us):
            for a in range(D):
                num = analysis.pstar_numeric(D, core.EQ_ENTROPIC, rho, u, a)
                assert abs(num - analysis.pstar_closed(rho, u[a])) < 1e-14
                ul = np.clip(u, -0.4, 0.4)
                assert abs(analysis.pstar_numeric(D, core.EQ_POLY2, rho, ul, a)) < 1e-14
                assert abs(analysis.pstar_numeric(D, core.EQ_PRODUCT, rho, ul, a)) < 1e-14


# ----------------------------------------------------------------------------- bulk A, omega

def test_entropic_bulk_A_matches_general_form():
    """Eq. (eq:entropic_bulk) equals the general Eq. (eq:entorpic_bulk) evaluated with the
    entropic P* (derivatives by finite differences); B of Eq. (eq:entorpic_bulk_2) is 0."""
    for u in np.linspace(-0.95, 0.95, 39):
        A_gen = analysis.bulk_A_general(1.3, u)
        assert abs(core.bulk_A(core.EQ_ENTROPIC, u) - A_gen) < 1e-9
        assert abs(analysis.bulk_B_general(1.3, u)) < 1e-9


def test_bulk_A_printed_values():
    """A(0) = 1; entropic A -> 0 as u -> 1 (Sec. IV.A); polynomial A = 0 at
    |u| = vs sqrt(2/3) (Eq. eq:bulk_poly_positivity) and the general form with P* = 0."""
    assert core.bulk_A(core.EQ_ENTROPIC, 0.0) == 1.0
    assert core.bulk_A(core.EQ_POLY2, 0.0) == 1.0
    assert abs(core.bulk_A(core.EQ_ENTROPIC, 1.0) - GOLD["entropic_bulk_A_at_u1"]["value"]) < 1e-14
    assert core.bulk_A(core.EQ_ENTROPIC, 0.999) > 0
    u_star = math.sqrt(VS2) * math.sqrt(2.0 / 3.0)
    assert abs(core.bulk_A(core.EQ_POLY2, u_star)) < 1e-14
    assert abs(u_star - 0.4714) < 5e-5
    zero = lambda rho, u: 0.0 * rho
    for u in (-0.3, 0.1, 0.4):
        assert abs(core.bulk_A(core.EQ_POLY2, u) - analysis.bulk_A_general(1.0, u, pstar=zero)) < 1e-12
        assert abs(analysis.bulk_B_general(1.0, u, pstar=zero) + u ** 3) < 1e-12
    # entropic A stays positive on (-1, 1) (Sec. IV.A)
    assert min(core.bulk_A(core.EQ_ENTROPIC, u) for u in np.linspace(-0.999, 0.999, 2001)) > 0


@pytest.mark.parametrize("eq", EQS)
def test_omega(eq):
    """2 beta = 1 / tau without correction (Eq. eq:relaxation_frequency with
    nu = vs^2 (tau - 1/2)); the corrected rate reduces to it at u = 0 and lies in
    [0, 2] (beta in [0, 1]) whenever A >= 0."""
    for tau in (0.5005, 0.8, 1.5):
        assert abs(core.omega(3, eq, 0, tau, [0.3, -0.2, 0.1]) - 1.0 / tau) < 1e-15
        assert abs(core.omega(3, eq, 1, tau, [0.0, 0.0, 0.0]) - 1.0 / tau) < 1e-15
        for u in ([0.3, 0.0, 0.0], [0.1, -0.2, 0.05]):
            om = core.omega(3, eq, 1, tau, u)
            assert 0.0 <= om <= 2.0
    # the cell's A is the smallest over axes (flow along one axis reduces to the 1-D case)
    tau = 0.7
    a1 = core.omega(1, eq, 1, tau, [0.25])
    assert abs(core.omega(3, eq, 1, tau, [0.0, -0.25, 0.1]) - a1) < 1e-15


# ----------------------------------------------------------------------------- full step

@pytest.mark.parametrize("D,dims", [(2, (7, 5, 1)), (3, (5, 4, 3))])
@pytest.mark.parametrize("eq", EQS)
@pytest.mark.parametrize("bulk", [0, 1])
def test_step_conserves_mass_and_momentum(D, dims, eq, bulk):
    """Eq. (1) with periodic streaming conserves global mass and momentum."""
    n = int(np.prod(dims))
    rho, u = inputs.random_state(D, dims, 7 + eq + 3 * bulk, u_max=0.15)
    f0 = core.init(D, dims, eq, rho, u)
    d0 = core.diagnostics(D, dims, f0)
    f1 = core.step(D, dims, eq, bulk, 0.6, 60, f0)
    d1 = core.diagnostics(D, dims, f1)
    assert abs(d1["mass"] - d0["mass"]) < 1e-13 * n
    np.testing.assert_allclose(d1["momentum"], d0["momentum"], atol=1e-13 * n)
    # initial diagnostics equal the input fields (f = f^eq conserves rho and rho u)
    assert abs(d0["mass"] - rho.sum()) < 1e-12
    np.testing.assert_allclose(d0["momentum"][:D], (rho * u).sum(axis=1), atol=1e-12)
    assert abs(d0["kinetic"] - 0.5 * (rho * (u * u).sum(axis=0)).sum()) < 1e-12


@pytest.mark.parametrize("D,dims", [(2, (6, 5, 1)), (3, (4, 5, 3))])
def test_free_flight_and_full_relaxation(D, dims):
    """tau -> infinity: one step only moves f_i from r to r + c_i.  tau = 1 (2 beta = 1):
    the new f_i(r) is the equilibrium of cell r - c_i."""
    c, _ = core.lattice(D)
    rng = np.random.default_rng(3)
    n = int(np.prod(dims))
    f0 = rng.uniform(0.01, 0.2, (len(c), n))
    f1 = core.step(D, dims, core.EQ_ENTROPIC, 0, 1e12, 1, f0)
    nx, ny, nz = dims
    grid0 = f0.reshape(len(c), nz, ny, nx)
    grid1 = f1.reshape(len(c), nz, ny, nx)
    for i in range(len(c)):
        shifted = np.roll(grid0[i], shift=(c[i, 2], c[i, 1], c[i, 0]), axis=(0, 1, 2))
        np.testing.assert_allclose(grid1[i], shifted, atol=1e-11)
    rho, u = core.moments(D, dims, f0)
    feq0 = core.init(D, dims, core.EQ_ENTROPIC, rho, u).reshape(len(c), nz, ny, nx)
    f2 = core.step(D, dims, core.EQ_ENTROPIC, 0, 1.0, 1, f0).reshape(len(c), nz, ny, nx)
    for i in range(len(c)):
        np.testing.assert_allclose(
            f2[i], np.roll(feq0[i], shift=(c[i, 2], c[i, 1], c[i, 0]), axis=(0, 1, 2)), rtol=1e-14)


def test_translation_invariance():
    """Shifting the initial state by one cell shifts the result by one cell."""
    D, dims = 2, (9, 7, 1)
    rho, u = inputs.random_state(D, dims, 19, u_max=0.2)
    f = core.init(D, dims, core.EQ_ENTROPIC, rho, u)
    Q = f.shape[0]
    g = np.roll(f.reshape(Q, 7, 9), shift=(2, 3), axis=(1, 2)).reshape(Q, -1)
    a = core.step(D, dims, core.EQ_ENTROPIC, 1, 0.55, 25, f).reshape(Q, 7, 9)
    b = core.step(D, dims, core.EQ_ENTROPIC, 1, 0.55, 25, g).reshape(Q, 7, 9)
    np.testing.assert_allclose(np.roll(a, shift=(2, 3), axis=(1, 2)), b, rtol=1e-13)


def _fit_rate(t, y):
    return -np.polyfit(t, np.log(y), 1)[0]


def test_taylor_green_energy_decay():
    """2-D Taylor-Green vortex (64^2, u0 = 0.05, tau = 0.8): the kinetic energy decays at
    2 nu (k_x^2 + k_y^2) with nu = (tau - 1/2) / 3, k = 2 pi / 64 (within 1%)."""
    n, tau = 64, 0.8
    nu = (tau - 0.5) / 3.0
    rho, u = inputs.taylor_green_2d(n, u0=0.05)
    dims = (n, n, 1)
    f = core.init(2, dims, core.EQ_ENTROPIC, rho, u)
    ts, es = [], []
    for t in range(0, 601, 100):
        ts.append(t)
        es.append(core.diagnostics(2, dims, f)["kinetic"])
        if t < 600:
            f = core.step(2, dims, core.EQ_ENTROPIC, 0, tau, 100, f)
    rate = _fit_rate(np.array(ts[1:]), np.array(es[1:]))
    k = 2 * math.pi / n
    assert abs(rate / (2 * nu * 2 * k * k) - 1.0) < 0.01


def test_shear_wave_decay_at_rest():
    """Shear wave u_y = a sin(k x) at U0 = 0 decays at nu k^2 (amplitude)."""
    nx, ny, tau = 64, 2, 0.9
    nu = (tau - 0.5) / 3.0
    k = 2 * math.pi / nx
    table = {"nx": [nx], "ny": [ny], "nmode": [1], "U0": [0.0], "tau": [tau], "kind": [0], "amp": 1e-4}
    rho, u = inputs.linear_mode_fields(table, 0)
    f = core.init(2, (nx, ny, 1), core.EQ_ENTROPIC, rho, u)
    _, series = core.run_probed(2, (nx, ny, 1), core.EQ_ENTROPIC, 0, tau, 801, 100, (1, 0, 0), f)
    amp = np.abs(series[:, 2])
    rate = _fit_rate(np.arange(len(amp))[2:] * 100.0, amp[2:])
    assert abs(rate / (nu * k * k) - 1.0) < 0.01


@pytest.mark.parametrize("D", [2, 3])
def test_diagnostics_closed_form(D):
    """Diagnostics of f = f^eq(rho = 1, u) for the Taylor-Green velocity on an n^D grid
    (the equilibrium reproduces rho and rho u exactly): mass n^D, momentum 0 (the field
    is odd), kinetic energy 1/2 sum |u|^2 = u0^2 n^2 / 4 in 2-D and u0^2 n^3 / 8 in 3-D
    (the mean of sin^2 cos^2 products), max |u_a| = u0 (reached where x = pi/2, y = z = 0)."""
    n, u0 = 16, 0.07
    if D == 2:
        _, u = inputs.taylor_green_2d(n, u0=u0)
        dims = (n, n, 1)
        expect_ke = u0 * u0 * n ** 2 / 4
    else:
        _, u = inputs.taylor_green_3d(n, u0=u0)
        dims = (n, n, n)
        expect_ke = u0 * u0 * n ** 3 / 8
    rho = np.ones(int(np.prod(dims)))
    for eq in (core.EQ_ENTROPIC, core.EQ_POLY2, core.EQ_PRODUCT):
        d = core.diagnostics(D, dims, core.init(D, dims, eq, rho, u))
        assert abs(d["mass"] - np.prod(dims)) < 1e-11
        assert np.all(np.abs(d["momentum"]) < 1e-12)
        assert abs(d["kinetic"] / expect_ke - 1) < 1e-12
        assert abs(d["max_u"] - u0) < 1e-15


def test_probe_of_sine_density():
    """sum_x (1 + a sin(2 pi n x / N)) exp(-i 2 pi n x / N) = -i a N / 2 per row."""
    nx, ny, a = 48, 3, 1e-3
    table = {"nx": [nx], "ny": [ny], "nmode": [2], "U0": [0.0], "tau": [0.8], "kind": [1], "amp": a}
    rho, u = inputs.linear_mode_fields(table, 0)
    f = core.init(2, (nx, ny, 1), core.EQ_ENTROPIC, rho, u)
    p = core.probe(2, (nx, ny, 1), f, (2, 0, 0))
    assert abs(p[0] - (-1j * a * nx * ny / 2)) < 1e-13
    assert abs(p[1]) < 1e-13 and abs(p[2]) < 1e-13


def test_local_patch_matches_full_lattice():
    """The sampled-cell evaluation on a (2n+1)^D patch equals the full periodic run."""
    D, dims, n = 3, (9, 8, 7), 2
    rho_fn, u_fn = inputs.taylor_green_3d_fields(8, u0=0.1)
    iz, iy, ix = np.meshgrid(np.arange(7), np.arange(8), np.arange(9), indexing="ij")
    rho = rho_fn(ix, iy, iz).reshape(-1)
    u = u_fn(ix, iy, iz).reshape(3, -1)
    f = core.step(D, dims, core.EQ_ENTROPIC, 1, 0.52, n, core.init(D, dims, core.EQ_ENTROPIC, rho, u))
    cells = np.array([[0, 0, 0], [8, 7, 6], [4, 3, 2], [1, 6, 5]])
    got = core.local_populations(D, dims, core.EQ_ENTROPIC, 1, 0.52, n, rho_fn, u_fn, cells)
    for m, (x, y, z) in enumerate(cells):
        np.testing.assert_allclose(got[m], f[:, x + 9 * (y + 8 * z)], rtol=1e-15)


# ----------------------------------------------------------------------------- linear theory

def _mode_rates(lam, k):
    return -np.log(np.abs(lam)), -np.angle(lam) / k


@pytest.mark.parametrize("eq", [core.EQ_ENTROPIC, core.EQ_POLY2])
@pytest.mark.parametrize("U0", [0.0, 0.15, 0.3])
def test_time_stepping_matches_von_neumann(eq, U0):
    """A small-amplitude shear wave advanced by the oracle decays and travels exactly as
    the eigenvalue of M = E (delta + J) (Eq. eq:VN_eigen) predicts; it travels at +U0
    (streaming direction of Eq. 1)."""
    nx, ny, tau, n = 32, 1, 0.8, 1
    k = 2 * math.pi * n / nx
    table = {"nx": [nx], "ny": [ny], "nmode": [n], "U0": [U0], "tau": [tau], "kind": [0], "amp": 1e-6}
    rho, u = inputs.linear_mode_fields(table, 0)
    f = core.init(2, (nx, ny, 1), eq, rho, u)
    K = 5
    _, s = core.run_probed(2, (nx, ny, 1), eq, 0, tau, 301, K, (n, 0, 0), f)
    jy = s[:, 2]
    lam_meas = (jy[-1] / jy[-11]) ** (1.0 / (10 * K))
    lams, vecs = analysis.hydrodynamic_modes(2, eq, 0, tau, 1.0, [U0, 0.0], [k, 0.0])
    # the shear mode is the one whose eigenvector carries j_y
    c, _ = core.lattice(2)
    jy_w = np.abs(c[:, 1] @ vecs)
    lam_vn = lams[np.argmax(jy_w)]
    assert abs(lam_meas - lam_vn) < 1e-7
    decay, speed = _mode_rates(lam_vn, k)
    assert abs(speed - U0) < 2e-3


@pytest.mark.parametrize("U0", [0.0, 0.2, 0.5, 0.8])
def test_von_neumann_entropic_sound_speeds(U0):
    """At k -> 0 the acoustic eigenvalues of M travel at c_s^{e+-}(U0) of Eqs.
    (eq:cs_plus_ent), (eq:cs_minus_ent), and their k^2 damping coefficients follow the
    general form of Sec. IV.B with B = 0."""
    tau = 0.8
    nu = (tau - 0.5) / 3.0
    k = 2 * math.pi / 2048
    lams, vecs = analysis.hydrodynamic_modes(1, core.EQ_ENTROPIC, 0, tau, 1.0, [U0], [k])
    decay, speed = _mode_rates(lams, k)
    order = np.argsort(-speed)
    cp, cm = analysis.cs_entropic(U0)
    assert abs(speed[order[0]] - cp) < 1e-5
    assert abs(speed[order[1]] - cm) < 1e-5
    gp, gm = analysis.acoustic_dissipation_entropic(U0, nu)
    assert abs(decay[order[0]] / (k * k) - gp) < 1e-3 * nu
    assert abs(decay[order[1]] / (k * k) - gm) < 1e-3 * nu


@pytest.mark.parametrize("eq", [core.EQ_ENTROPIC, core.EQ_POLY2])
@pytest.mark.parametrize("U0", [0.1, 0.25])
def test_von_neumann_bulk_correction(eq, U0):
    """Sec. V.B: without correction the mean k^2 damping of the two acoustic modes is
    nu A(U0); with the redefined beta it is nu."""
    tau = 0.7
    nu = (tau - 0.5) / 3.0
    k = 2 * math.pi / 2048
    for bulk, expect in ((0, nu * core.bulk_A(eq, U0)), (1, nu)):
        lams, _ = analysis.hydrodynamic_modes(1, eq, bulk, tau, 1.0, [U0], [k])
        decay, _ = _mode_rates(lams, k)
        assert abs(np.mean(decay) / (k * k) - expect) < 1e-3 * nu


@pytest.mark.parametrize("eq", [core.EQ_ENTROPIC, core.EQ_POLY2])
def test_von_neumann_shear_coefficient(eq):
    """Sec. IV.C: the shear mode (k along x, U0 along x) damps at nu A^s_xy k^2."""
    tau = 0.8
    nu = (tau - 0.5) / 3.0
    k = 2 * math.pi / 2048
    for U0 in (0.1, 0.3):
        lams, vecs = analysis.hydrodynamic_modes(2, eq, 0, tau, 1.0, [U0, 0.0], [k, 0.0])
        c, _ = core.lattice(2)
        lam = lams[np.argmax(np.abs(c[:, 1] @ vecs))]
        decay = -math.log(abs(lam))
        assert abs(decay / (k * k) - nu * analysis.shear_As(eq, U0, 0.0)) < 1e-3 * nu


def test_entropic_sound_speed_limits():
    """Limits of Eqs. (eq:cs_plus_ent), (eq:cs_minus_ent) as printed in Sec. III.C."""
    g = GOLD["entropic_cs_limits"]
    cp, cm = analysis.cs_entropic(1.0)
    assert abs(cp - g["cs_plus_u_to_1"]) < 1e-15 and abs(cm - g["cs_minus_u_to_1"]) < 1e-15
    cp, cm = analysis.cs_entropic(-1.0)
    assert abs(cp - g["cs_plus_u_to_m1"]) < 1e-15 and abs(cm - g["cs_minus_u_to_m1"]) < 1e-15


def test_poly_cfl_limit_printed_constant():
    """Sec. III.C: at large viscosity the polynomial equilibrium is linearly stable up to
    |u| = 1 - vs = 0.4226 (flow along x); the entropic one stays stable beyond it."""
    umax = GOLD["poly_cfl_umax"]["value"]
    assert abs((1 - math.sqrt(VS2)) - umax) < 5e-5
    tau = 0.5 + 3 * 1.2  # nu = 1.2, the largest viscosity of the stability study
    kgrid = np.linspace(0.0, math.pi, 25)
    grow = lambda eq, u: max(float(np.max(np.abs(np.linalg.eigvals(
        analysis.vn_matrix(1, eq, 0, tau, 1.0, [u], [kk]))))) for kk in kgrid)
    assert grow(core.EQ_POLY2, umax - 0.01) <= 1 + 1e-12
    assert grow(core.EQ_POLY2, umax + 0.02) > 1 + 1e-6
    assert grow(core.EQ_ENTROPIC, 0.9) <= 1 + 1e-12


def test_entropic_unconditional_linear_stability():
    """Sec. V.A.2: the entropic equilibrium is linearly stable for |u| < 1 at any
    viscosity of the study (two end points checked on a coarse k, theta grid)."""
    kgrid = np.linspace(0.0, math.pi, 9)
    for nu in (1e-5, 0.1):
        tau = 0.5 + 3 * nu
        for theta in (0.0, math.pi / 8, math.pi / 4):
            assert analysis.growth_max(2, core.EQ_ENTROPIC, tau, 0.6, theta, kgrid) <= 1 + 1e-10


def test_product_form_diagonal_limit():
    """Sec. V.A.2: along a diagonal link the product form is stable up to
    sqrt(2) (1 - vs) = 0.598 at large viscosity."""
    lim = GOLD["product_diagonal_umax"]["value"]
    assert abs(math.sqrt(2) * (1 - math.sqrt(VS2)) - lim) < 5e-4
    tau = 0.5 + 3 * 1.2
    kgrid = np.linspace(0.0, math.pi, 13)
    assert analysis.growth_max(2, core.EQ_PRODUCT, tau, lim - 0.02, math.pi / 4, kgrid) <= 1 + 1e-12
    assert analysis.growth_max(2, core.EQ_PRODUCT, tau, lim + 0.03, math.pi / 4, kgrid) > 1 + 1e-6


@pytest.mark.parametrize("D,dims", [(2, (23, 17, 1)), (3, (9, 7, 5))])
@pytest.mark.parametrize("eq", [core.EQ_ENTROPIC, core.EQ_POLY2, core.EQ_PRODUCT])
def test_threaded_step_is_bitwise_single_thread(D, dims, eq):
    """The all-core oracle (rows of the lattice shared out between host threads) computes
    every cell exactly as the single-thread oracle does: the states agree bit for bit."""
    rho, u = inputs.random_state(D, dims, seed=61 + eq, u_max=0.15)
    f0 = core.init(D, dims, eq, rho, u)
    core.set_threads(1)
    one = core.step(D, dims, eq, 1, 0.57, 6, f0)
    used = core.set_threads(4)
    try:
        many = core.step(D, dims, eq, 1, 0.57, 6, f0)
    finally:
        core.set_threads(1)
    assert used in (1, 4)
    assert np.array_equal(one.view(np.uint64), many.view(np.uint64))
