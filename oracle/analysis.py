"""Host FP64 analysis of the entropic lattice-BGK scheme (test infrastructure only).

Each function restates a passage of arXiv 2303.08163 in NumPy, or checks the C oracle
against something the paper or the mathematics fixes:

- ``newton_entropic``: Sec. II.A, the equilibrium as the minimiser of
  H = sum_i f_i ln(f_i / w_i) under the mass and momentum constraints, solved by Newton's
  method on the convex dual.  Independent of the closed form.
- ``pstar_closed`` / ``pstar_numeric``: Sec. III.A, the pressure deviation P*_aa.
- ``bulk_A_general``: Eq. (eq:entorpic_bulk), A from P* and its derivatives.
- ``cs_entropic``: Eqs. (eq:cs_plus_ent), (eq:cs_minus_ent).
- ``acoustic_dissipation_entropic``: the k^2 coefficients of the entropic acoustic modes,
  from the general form of Sec. IV.B with B = 0 (the printed entropic special case is
  garbled; this reading is listed in the design notes).
- ``shear_As``: Sec. IV.C, A^s for the three equilibria.
- ``vn_matrix`` / ``vn_eigs``: Sec. V.A, M = E (delta + J), Eq. (eq:VN_eigen), with J the
  Jacobian of the collision operator taken by fourth-order central differences of the
  oracle's f^eq (the printed Jacobian of App. C is not transcribed).
"""
import numpy as np

from . import core

VS2 = 1.0 / 3.0  # lattice sound speed squared, vs = dr / (sqrt(3) dt)


def newton_entropic(D, rho, u, tol=1e-15, maxit=100):
    """Minimiser of H = sum f ln(f/w) subject to sum f = rho, sum c f = rho u.

    Stationarity gives f_i = w_i exp(l0 + l . c_i); the multipliers minimise the convex
    dual G(l) = sum_i w_i exp(l0 + l . c_i) - l0 rho - l . rho u.
    """
    c, w = core.lattice(D)
    C = np.concatenate([np.ones((len(w), 1)), c[:, :D].astype(np.float64)], axis=1)
    target = np.concatenate([[rho], rho * np.asarray(u, dtype=np.float64)[:D]])
    lam = np.zeros(D + 1)
    lam[0] = np.log(rho)
    for _ in range(maxit):
        f = w * np.exp(C @ lam)
        grad = C.T @ f - target
        hess = (C * f[:, None]).T @ C
        dl = np.linalg.solve(hess, grad)
        lam -= dl
        if np.max(np.abs(dl)) < tol:
            break
    return w * np.exp(C @ lam)


def pstar_closed(rho, ua):
    """P*_aa = -rho vs^2 [x^2 - 2 sqrt(x^2 + 1) + 2], x = u_a / vs (Sec. III.A)."""
    x2 = ua * ua / VS2
    return -rho * VS2 * (x2 - 2.0 * np.sqrt(x2 + 1.0) + 2.0)


def pstar_numeric(D, eq_kind, rho, u, axis):
    """sum_i (c_ia - u_a)^2 f_i^eq - rho vs^2 from the oracle's equilibrium."""
    c, _ = core.lattice(D)
    f = core.feq(D, eq_kind, rho, u)
    return float(np.sum((c[:, axis] - u[axis]) ** 2 * f) - rho * VS2)


def _d1(fn, x, h):
    """Fourth-order central difference of a scalar function."""
    return (-fn(x + 2 * h) + 8 * fn(x + h) - 8 * fn(x - h) + fn(x - 2 * h)) / (12 * h)


def bulk_A_general(rho, ux, pstar=pstar_closed, h=1e-3):
    """Eq. (eq:entorpic_bulk): A from a pressure deviation P*(rho, u_x)."""
    dPu = _d1(lambda v: pstar(rho, v), ux, h)
    dPr = _d1(lambda r: pstar(r, ux), rho, h)
    return (1.0 - 1.5 * ux * ux / VS2 - 1.5 / (rho * VS2) * ux * dPu
            - dPu * dPu / (2.0 * rho * rho * VS2) - dPr / (2.0 * VS2))


def bulk_B_general(rho, ux, pstar=pstar_closed, h=1e-3):
    """Eq. (eq:entorpic_bulk_2): the compressibility error B."""
    dPu = _d1(lambda v: pstar(rho, v), ux, h)
    dPr = _d1(lambda r: pstar(r, ux), rho, h)
    return -3.0 * ux * dPr - VS2 / rho * dPu - dPu * dPr / rho - ux ** 3


def cs_entropic(ux):
    """Entropic sound speeds (c_s^{e+}, c_s^{e-}), Eqs. (eq:cs_plus_ent), (eq:cs_minus_ent)."""
    vs = np.sqrt(VS2)
    S = np.sqrt(ux * ux / VS2 + 1.0)
    root = np.sqrt(2.0 * S - 1.0)
    return (ux + vs * root) / S, (ux - vs * root) / S


def acoustic_dissipation_entropic(ux, nu):
    """k^2 coefficients of the entropic acoustic modes (c_s^{e+}, c_s^{e-}).

    General form of Sec. IV.B with B = 0 (Eq. eq:bulk_compressibility_error_entropic):
    nu A [1 +- vs^2 dP*/du / (2 rho vs^2 sqrt(vs^2 + dP*/drho + (dP*/du / 2 rho)^2))].
    With x = u / vs and S = sqrt(x^2 + 1) this is nu A [1 -+ x (S - 1) / sqrt(2 S - 1)].
    """
    rho = 1.0
    A = bulk_A_general(rho, ux)
    dPu = _d1(lambda v: pstar_closed(rho, v), ux, 1e-3)
    dPr = _d1(lambda r: pstar_closed(r, ux), rho, 1e-3)
    root = np.sqrt(VS2 + dPr + (dPu / (2 * rho)) ** 2)
    frac = VS2 * dPu / (2 * rho * VS2 * root)
    return nu * A * (1 + frac), nu * A * (1 - frac)


def shear_As(eq_kind, ua, ub=0.0):
    """Effective shear coefficient A^s_ab of Sec. IV.C."""
    if eq_kind == core.EQ_ENTROPIC:
        x2 = ua * ua / VS2
        return 2.0 * np.sqrt(x2 + 1.0) - x2 - 1.0
    if eq_kind == core.EQ_POLY2:
        return 1.0 - ua / VS2 * (ua + 2.0 * ub)
    return 1.0


def feq_jacobian(D, eq_kind, rho, u, h=1e-4):
    """d f^eq_i / d f_j at f = f^eq(rho, u), by the chain rule through rho(f), u(f).

    rho = sum f, u = sum c f / rho, so d rho / d f_j = 1 and
    d u_a / d f_j = (c_ja - u_a) / rho.  The partial derivatives of f^eq(rho, u) are
    fourth-order central differences of the oracle's equilibrium.
    """
    c, _ = core.lattice(D)
    u = np.asarray(u, dtype=np.float64)[:D]
    dfr = _d1(lambda r: core.feq(D, eq_kind, r, u), rho, h)
    J = np.outer(dfr, np.ones(len(c)))
    for a in range(D):
        def fa(v, a=a):
            uu = u.copy()
            uu[a] = v
            return core.feq(D, eq_kind, rho, uu)
        dfu = _d1(fa, u[a], h)
        J += np.outer(dfu, (c[:, a] - u[a]) / rho)
    return J


def vn_matrix(D, eq_kind, bulk_corr, tau, rho, u, k):
    """M = E (delta + J) of Eq. (eq:VN_eigen) for wave vector k (length D).

    J_ij = omega (d f^eq_i / d f_j - delta_ij) with omega = 2 beta at the mean state; the
    derivative of a local omega multiplies (f^eq - f), which vanishes at equilibrium.
    E_ij = exp(-i c_i . k) delta_ij.
    """
    c, _ = core.lattice(D)
    om = core.omega(D, eq_kind, bulk_corr, tau, u)
    Q = len(c)
    J = om * (feq_jacobian(D, eq_kind, rho, u) - np.eye(Q))
    phase = np.exp(-1j * (c[:, :D] @ np.asarray(k, dtype=np.float64)[:D]))
    return phase[:, None] * (np.eye(Q) + J)


def vn_eigs(D, eq_kind, bulk_corr, tau, rho, u, k):
    """Eigenvalues and right eigenvectors of M."""
    return np.linalg.eig(vn_matrix(D, eq_kind, bulk_corr, tau, rho, u, k))


def hydrodynamic_modes(D, eq_kind, bulk_corr, tau, rho, u, k, nmodes=None):
    """The nmodes (default D + 1) eigenvalues of M whose eigenvectors lie closest to the
    conserved-moment subspace spanned by (1, c_i) weighted by f^eq.

    Returns them sorted by the argument's sign convention: exp(-i Omega) with
    phase speed -arg(lambda) / |k| and decay rate -ln|lambda| per step.
    """
    c, _ = core.lattice(D)
    lam, vec = vn_eigs(D, eq_kind, bulk_corr, tau, rho, u, k)
    Q = len(c)
    # moments of each eigenvector: rho' = sum F, j' = sum c F
    mom = np.vstack([np.ones(Q), c[:, :D].T.astype(np.float64)]) @ vec
    weight = np.linalg.norm(mom, axis=0) / np.linalg.norm(vec, axis=0)
    if nmodes is None:
        nmodes = D + 1
    sel = np.argsort(-weight)[:nmodes]
    return lam[sel], vec[:, sel]


def growth_max(D, eq_kind, tau, umag, theta, kgrid):
    """Largest |lambda| of M over the given (k_x, k_y) grid for a mean velocity of
    magnitude umag at angle theta to the x axis (Sec. V.A.2 stability domain)."""
    u = np.array([umag * np.cos(theta), umag * np.sin(theta), 0.0])
    best = 0.0
    for kx in kgrid:
        for ky in kgrid:
            lam = np.linalg.eigvals(vn_matrix(D, eq_kind, 0, tau, 1.0, u, [kx, ky]))
            best = max(best, float(np.max(np.abs(lam))))
    return best
