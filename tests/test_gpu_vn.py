"""von Neumann analysis on the GPU (Sec. V.A): eigenvalues of M = E (delta + J)
(Eq. eq:VN_eigen) against the oracle's matrices (NumPy eigensolver, Jacobian by
fourth-order finite differences of the oracle's equilibrium), and the stability limits
the paper prints (Sec. III.C and V.A.2).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import analysis, core

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


@pytest.fixture(scope="module", autouse=True)
def cuda_library():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2303_08163_gb300 import build, lbm
    build.build()
    lbm.load()
    yield


@pytest.mark.parametrize("eq", [core.EQ_ENTROPIC, core.EQ_POLY2, core.EQ_PRODUCT])
@pytest.mark.parametrize("bulk", [0, 1])
def test_eigenvalues_match_oracle(eq, bulk):
    from paper_2303_08163_gb300 import lbm
    rng = np.random.default_rng(31 + eq + 5 * bulk)
    n = 40
    umax = 0.6 if eq == core.EQ_ENTROPIC else 0.35
    params = np.stack([0.5 + 10 ** rng.uniform(-3, 0.3, n), rng.uniform(0.9, 1.1, n),
                       rng.uniform(-umax, umax, n), rng.uniform(-umax, umax, n),
                       rng.uniform(0, math.pi, n), rng.uniform(0, math.pi, n)], axis=1)
    lam = lbm.vn_eigenvalues(eq, bulk, params)
    for p in range(n):
        ref = np.linalg.eigvals(analysis.vn_matrix(2, eq, bulk, params[p, 0], params[p, 1],
                                                   params[p, 2:4], params[p, 4:6]))
        dist = max(float(np.min(np.abs(lam[p] - r))) for r in ref)
        assert dist < 1e-8, (p, dist)
        assert np.all(np.diff(np.abs(lam[p])) <= 1e-15)  # sorted by decreasing modulus


def test_zero_wavevector_has_conserved_modes():
    """At k = 0 the mass and momentum modes have lambda = 1 exactly (three of them)."""
    from paper_2303_08163_gb300 import lbm
    params = np.array([[0.7, 1.0, 0.2, -0.1, 0.0, 0.0]])
    lam = lbm.vn_eigenvalues(core.EQ_ENTROPIC, 0, params)[0]
    assert np.sum(np.abs(lam - 1.0) < 1e-12) == 3


def test_printed_stability_limits():
    """Largest linearly stable |u| at nu = 1.2 (the largest viscosity of the study):
    polynomial along x: 1 - vs = 0.4226 (Eq. eq:CFL_lmit_absolute_poly); product form along
    a diagonal: sqrt(2)(1 - vs) = 0.598 (Sec. V.A.2); the entropic equilibrium is stable up
    to |u| -> 1 in every direction, at every viscosity of the study (Sec. V.A.2)."""
    from paper_2303_08163_gb300 import lbm
    nk = 41
    poly = lbm.vn_stability_limit(core.EQ_POLY2, [1.2], [0.0], nk=nk)[0]
    prod = lbm.vn_stability_limit(core.EQ_PRODUCT, [1.2], [math.pi / 4], nk=nk)[0]
    print(f"nu = 1.2: polynomial along x {poly:.4f}, product form along the diagonal {prod:.4f}")
    assert abs(poly - GOLD["poly_cfl_umax"]["value"]) < 0.01
    assert abs(prod - GOLD["product_diagonal_umax"]["value"]) < 0.01
    nus = GOLD["stability_nu_grid"]["value"]
    thetas = np.linspace(0, math.pi / 2, 7)
    nu_g, th_g = np.meshgrid(nus, thetas, indexing="ij")
    ent = lbm.vn_stability_limit(core.EQ_ENTROPIC, nu_g.ravel(), th_g.ravel(), nk=17, u_hi=0.95,
                                 iterations=8)
    assert np.all(ent >= 0.95 - 1e-12)


def test_stability_domain_vs_viscosity():
    """Sec. V.A.2, Fig. stability_all: the polynomial and product-form limits fall towards
    zero as nu -> 0 and approach the CFL values at large nu; the entropic limit does not
    depend on nu."""
    from paper_2303_08163_gb300 import lbm
    nus = np.array(GOLD["stability_nu_grid"]["value"])
    thetas = np.linspace(0, math.pi / 2, 9)
    rows = {}
    for eq in (core.EQ_POLY2, core.EQ_PRODUCT, core.EQ_ENTROPIC):
        nu_g, th_g = np.meshgrid(nus, thetas, indexing="ij")
        lim = lbm.vn_stability_limit(eq, nu_g.ravel(), th_g.ravel(), nk=25, u_hi=0.95, iterations=14)
        rows[eq] = lim.reshape(len(nus), len(thetas)).min(axis=1)
    print("nu        poly2   product entropic")
    for i, nu in enumerate(nus):
        print(f"{nu:8.1e} {rows[core.EQ_POLY2][i]:.4f} {rows[core.EQ_PRODUCT][i]:.4f} {rows[core.EQ_ENTROPIC][i]:.4f}")
    assert np.all(rows[core.EQ_ENTROPIC] >= 0.95 - 1e-3)
    for eq in (core.EQ_POLY2, core.EQ_PRODUCT):
        assert rows[eq][0] < 0.5 * rows[eq][-1]      # smallest viscosity far less stable
        assert rows[eq][-1] < 0.45                   # bounded by the CFL value at large nu
