"""ctypes wrapper of the plain-C FP64 oracle (test infrastructure only).

Each function follows the paper (arXiv 2303.08163) as cited in ``lbm_oracle.c``:
Sec. II lattice and equilibria (Eqs. eq:Entropic_isothermal_EDF, eq:Poly2_isothermal_EDF,
eq:Product_isothermal_EDF), Eq. (1) collide-then-stream, Eq. (eq:relaxation_frequency),
and the bulk correction of Sec. V.B (Eqs. eq:entropic_bulk, eq:LBGK_bulk,
eq:redefined_relaxation rate).

Pins (tests/test_oracle_pins.py): moments of every equilibrium, f^eq(rho, 0) = w rho,
mirror symmetry, the entropic equilibrium equals a Newton minimiser of H, the P* closed
form of Sec. III.A, the bulk A closed form against the general Chapman-Enskog form,
global conservation, pure streaming, Taylor-Green and shear-wave decay, and the
time-stepped oracle against the von Neumann eigenvalues of Eq. (eq:VN_eigen).

Array conventions: dims = (Nx, Ny, Nz), cell index x + Nx (y + Ny z); populations f
have shape (Q, ncell); velocities u have shape (D, ncell); population index
i = (c_x+1) + 3 (c_y+1) + 9 (c_z+1).
"""
import ctypes
import os

import numpy as np

from . import build as _build

EQ_ENTROPIC, EQ_POLY2, EQ_PRODUCT = 0, 1, 2

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lp = ctypes.POINTER(ctypes.c_int64)
        i64, ci, cd = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        sig = {
            "oracle_lattice": (ci, [ci, ip, dp]),
            "oracle_feq": (ci, [ci, ci, cd, dp, dp]),
            "oracle_bulk_A": (cd, [ci, cd]),
            "oracle_omega": (cd, [ci, ci, ci, cd, dp]),
            "oracle_init": (ci, [ci, lp, ci, dp, dp, dp]),
            "oracle_step": (ci, [ci, lp, ci, ci, cd, i64, dp, dp]),
            "oracle_moments": (ci, [ci, lp, dp, dp, dp]),
            "oracle_diagnostics": (ci, [ci, lp, dp, dp]),
            "oracle_probe": (ci, [ci, lp, dp, ip, dp]),
            "oracle_run_probed": (ci, [ci, lp, ci, ci, cd, i64, i64, ip, dp, dp, dp]),
            "oracle_set_threads": (ci, [ci]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _lp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _dims(dims):
    d = [int(v) for v in dims] + [1] * (3 - len(dims))
    return np.ascontiguousarray(d[:3], dtype=np.int64)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed (rc={rc})")


def lattice(D):
    """Velocities c (Q, 3) and weights w (Q,) of the D-dimensional tensor-product lattice."""
    c = np.zeros((27, 3), dtype=np.int32)
    w = np.zeros(27)
    Q = _load().oracle_lattice(int(D), _ip(c), _dp(w))
    if Q < 0:
        raise ValueError("D must be 1, 2 or 3")
    return c[:Q].copy(), w[:Q].copy()


def feq(D, eq_kind, rho, u):
    """Equilibrium populations (Q,) at density rho and velocity u (length D)."""
    uu = np.zeros(3)
    uu[:D] = np.asarray(u, dtype=np.float64)[:D]
    out = np.zeros(27)
    _check(_load().oracle_feq(int(D), int(eq_kind), float(rho), _dp(uu), _dp(out)), "feq")
    return out[: 3 ** D].copy()


def bulk_A(eq_kind, u):
    """Bulk coefficient A(u) of Eq. (eq:entropic_bulk) or Eq. (eq:LBGK_bulk)."""
    return _load().oracle_bulk_A(int(eq_kind), float(u))


def omega(D, eq_kind, bulk_corr, tau, u):
    """Collision frequency 2 beta of a cell with velocity u."""
    uu = np.zeros(3)
    uu[:D] = np.asarray(u, dtype=np.float64)[:D]
    return _load().oracle_omega(int(D), int(eq_kind), int(bulk_corr), float(tau), _dp(uu))


def init(D, dims, eq_kind, rho, u):
    """f = f^eq(rho, u) per cell; rho (ncell,), u (D, ncell) -> f (Q, ncell)."""
    d = _dims(dims)
    n = int(np.prod(d))
    rho = np.ascontiguousarray(np.asarray(rho, dtype=np.float64).reshape(n))
    uu = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(D, n))
    f = np.zeros((3 ** D, n))
    _check(_load().oracle_init(int(D), _lp(d), int(eq_kind), _dp(rho), _dp(uu), _dp(f)), "init")
    return f


def set_threads(n):
    """Host threads used by `step` from now on (1 by default); returns the number the
    library will use (1 when it was built without OpenMP).  Every thread count gives the
    same result bit for bit."""
    return _load().oracle_set_threads(int(n))


def step(D, dims, eq_kind, bulk_corr, tau, n, f):
    """Return the state after n steps of Eq. (1) from state f (not modified)."""
    d = _dims(dims)
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    g = np.empty_like(f)
    _check(_load().oracle_step(int(D), _lp(d), int(eq_kind), int(bulk_corr), float(tau),
                               int(n), _dp(f), _dp(g)), "step")
    return f


def moments(D, dims, f):
    """rho (ncell,) and u (D, ncell) of state f."""
    d = _dims(dims)
    n = int(np.prod(d))
    f = np.ascontiguousarray(f, dtype=np.float64)
    rho = np.zeros(n)
    u = np.zeros((D, n))
    _check(_load().oracle_moments(int(D), _lp(d), _dp(f), _dp(rho), _dp(u)), "moments")
    return rho, u


def diagnostics(D, dims, f):
    """Compensated global sums: mass, momentum (3,), kinetic energy, max |u_a|."""
    d = _dims(dims)
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(6)
    _check(_load().oracle_diagnostics(int(D), _lp(d), _dp(f), _dp(out)), "diagnostics")
    return {"mass": out[0], "momentum": out[1:4].copy(), "kinetic": out[4], "max_u": out[5]}


def probe(D, dims, f, kvec):
    """Complex projections (rho, j_x, j_y, j_z) on exp(-i k.r), k = 2 pi n / N."""
    d = _dims(dims)
    f = np.ascontiguousarray(f, dtype=np.float64)
    k = np.ascontiguousarray((list(kvec) + [0, 0, 0])[:3], dtype=np.int32)
    out = np.zeros(8)
    _check(_load().oracle_probe(int(D), _lp(d), _dp(f), _ip(k), _dp(out)), "probe")
    return out[0::2] + 1j * out[1::2]


def run_probed(D, dims, eq_kind, bulk_corr, tau, n, every_k, kvec, f):
    """n steps from f, probing at t = 0, K, 2K, ... (< n); returns (f_final, series (S, 4))."""
    d = _dims(dims)
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    g = np.empty_like(f)
    k = np.ascontiguousarray((list(kvec) + [0, 0, 0])[:3], dtype=np.int32)
    ns = (int(n) + int(every_k) - 1) // int(every_k)
    out = np.zeros((max(ns, 1), 8))
    _check(_load().oracle_run_probed(int(D), _lp(d), int(eq_kind), int(bulk_corr), float(tau),
                                     int(n), int(every_k), _ip(k), _dp(f), _dp(g), _dp(out)),
           "run_probed")
    series = out[:ns, 0::2] + 1j * out[:ns, 1::2]
    return f, series


def local_populations(D, dims, eq_kind, bulk_corr, tau, nsteps, rho_fn, u_fn, cells):
    """Populations at sampled cells after nsteps steps from f = f^eq(rho, u) on a periodic
    lattice of size dims, computed on a (2 nsteps + 1)^D patch around each cell.

    After n steps a cell depends only on cells within Chebyshev distance n, so a periodic
    patch of side 2n + 1 centred on it gives the same value as the full lattice.
    rho_fn(ix, iy, iz) and u_fn(ix, iy, iz) return the initial fields on integer index
    arrays (already wrapped); cells is an (m, 3) array of (x, y, z).  Returns (m, Q).
    """
    dims3 = [int(v) for v in _dims(dims)]
    side = 2 * int(nsteps) + 1
    sides = [min(side, dims3[a]) if a < D else 1 for a in range(3)]
    Q = 3 ** D
    out = np.zeros((len(cells), Q))
    for m, cell in enumerate(np.asarray(cells, dtype=np.int64)):
        offs = []
        for a in range(3):
            if a < D:
                if sides[a] == dims3[a]:
                    offs.append(np.arange(dims3[a]))
                else:
                    offs.append((cell[a] + np.arange(-nsteps, nsteps + 1)) % dims3[a])
            else:
                offs.append(np.array([cell[a]]))
        iz, iy, ix = np.meshgrid(offs[2], offs[1], offs[0], indexing="ij")
        rho = np.asarray(rho_fn(ix, iy, iz), dtype=np.float64).reshape(-1)
        u = np.asarray(u_fn(ix, iy, iz), dtype=np.float64).reshape(D, -1)
        pd = (len(offs[0]), len(offs[1]), len(offs[2]))
        f = init(D, pd, eq_kind, rho, u)
        f = step(D, pd, eq_kind, bulk_corr, tau, nsteps, f)
        centre = []
        for a in range(3):
            hit = np.nonzero(offs[a] == cell[a])[0]
            centre.append(int(hit[0]))
        cidx = centre[0] + pd[0] * (centre[1] + pd[1] * centre[2])
        out[m] = f[:, cidx]
    return out
