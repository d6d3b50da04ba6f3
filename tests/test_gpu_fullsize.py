"""GPU parity at the full benchmark sizes, in the launch shape the benchmark uses (the
autotuned one), on outputs the oracle can compute one by one:

- D3Q27 512^3 Taylor-Green (Re = 1600), binary16 and FP32 shifted storage: populations of
  sampled cells after 1 and 2 steps (the oracle evaluates a (2n+1)^3 patch around each
  cell), and global mass / momentum over 40 steps.
- D2Q9 4096^2 double shear layer, FP32: sampled cells after 1 and 2 steps.
- 4096 batched D2Q9 instances (FP64): probe series and final populations of sampled
  instances equal the oracle's to 1e-12.
- D3Q27 1024 x 512 x 512 decaying turbulence, binary16 and FP32: sampled cells after 1 and
  2 steps.
- The largest lattice: 1304^3 cells (more than 2^31), binary16, both step kernels.

Tolerances for stored binary16 / FP32 values: each storage rounding moves f - w rho0 by
at most half an ulp (u = 2^-11 resp. 2^-24 relative; below 2^-14 a binary16 value is a
subnormal, rounded to a multiple of 2^-24, an absolute error of up to 2^-25).  A sampled
value after n steps has been rounded n + 1 times directly; the roundings of the other
populations reach it through rho and u, to first order amplified by at most omega K
(omega = 1/tau, K the bound of `sensitivity` on |d f^eq_i / d f_j| / w_i at the field's
largest |u_a|); the FP32 collision is a chain of at most 32 roundings of operands bounded
by w_i (1 + S).  So, with S = sum_j |f_j - w_j|,
|f_gpu - f_ref| <= (n + 2) [u (|f_i - w_i| + omega K w_i S) + 2^-25 (1 + omega K Q w_i)]
                   + 32 n 2^-24 w_i (1 + S) (1 + omega K)
(the 2^-25 term for binary16 only).  Data-movement errors (a wrong neighbour, direction or
layout) are of order w_i |u| and stay well outside this bound.
"""
import math

import numpy as np
import pytest

from oracle import core
from paper_2303_08163_gb300 import inputs

pytestmark = pytest.mark.gpu

UNIT = {1: 2.0 ** -24, 2: 2.0 ** -11}
# half the spacing of the subnormal numbers: below 2^-14 a binary16 store rounds to a
# multiple of 2^-24, an absolute error of up to 2^-25 that no relative bound covers
FLOOR = {1: 0.0, 2: 2.0 ** -25}


@pytest.fixture(scope="module", autouse=True)
def cuda_library():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2303_08163_gb300 import build, lbm
    build.build()
    lbm.load()
    yield


def sample_cells(dims, count, seed):
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    pts = [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (0, ny - 1, 0), (nx - 1, 0, nz - 1)]
    pts += [tuple(int(rng.integers(0, d)) for d in dims) for _ in range(count)]
    return np.array(pts, dtype=np.int64)


def flat(cells, dims):
    nx, ny, _ = dims
    return cells[:, 0] + nx * (cells[:, 1] + ny * cells[:, 2])


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


def check_sampled(lat, D, dims, eq, bulk, tau, prec, rho_fn, u_fn, nsteps, cells, umax):
    got = lat.sample_populations(flat(cells, dims))
    ref = core.local_populations(D, dims, eq, bulk, tau, nsteps, rho_fn, u_fn, cells)
    _, w = core.lattice(D)
    shifted = np.abs(ref - w)
    S = shifted.sum(axis=1, keepdims=True)
    # storage roundings of this population, plus those reaching it through rho and u
    # (first order, amplified by at most omega K), plus the FP32 collision arithmetic
    ok = (1.0 / tau) * sensitivity(D, umax)
    tol = ((nsteps + 2) * UNIT[prec] * (shifted + ok * w * S)
           + (nsteps + 2) * FLOOR[prec] * (1 + ok * w * len(w))
           + 32 * nsteps * 2.0 ** -24 * w * (1 + S) * (1 + ok))
    bad = np.abs(got - ref) > tol
    assert not bad.any(), f"{bad.sum()} sampled populations off; worst {np.max(np.abs(got - ref) - tol):.3e}"


@pytest.mark.parametrize("prec", [2, 1])
def test_tgv_512_sampled_and_conservation(prec):
    import torch
    from paper_2303_08163_gb300 import lbm
    n, u0 = 512, 0.1
    nu = u0 * (n / (2 * math.pi)) / 1600.0
    tau = 0.5 + 3 * nu
    dims = (n, n, n)
    rho, u = inputs.taylor_green_3d(n, u0=u0)
    rho_fn, u_fn = inputs.taylor_green_3d_fields(n, u0=u0)
    lat = lbm.Lattice(lbm.D3Q27, dims, tau, lbm.ENTROPIC, 0, prec)
    lat.init_fields(rho, u)
    lat.set_option(lbm.OPT_TUNE, 1)  # the benchmark's launch shape
    assert lat.launch_info()["kernel"] == lbm.KERNEL_TMA
    lat.init_fields(rho, u)
    cells = sample_cells(dims, 48, seed=prec)
    lat.step(1)
    check_sampled(lat, 3, dims, core.EQ_ENTROPIC, 0, tau, prec, rho_fn, u_fn, 1, cells, u0)
    lat.step(1)
    check_sampled(lat, 3, dims, core.EQ_ENTROPIC, 0, tau, prec, rho_fn, u_fn, 2, cells, u0)
    d0 = lat.diagnostics()
    nsteps = 40
    lat.step(nsteps)
    d1 = lat.diagnostics()
    assert d1["nonfinite"] == 0
    # Conservation to round-off: every step rounds each stored f - w rho0 once (unit u of
    # the storage format) and the FP32 collision adds a few ulp; sum |f - w rho0| over a
    # cell is below 0.3 rho for |u| <= 0.1, so |d mass| <= steps * 2u * 0.3 * mass.
    bound = nsteps * 2 * UNIT[prec] * 0.3 * d0["mass"]
    drift = abs(d1["mass"] - d0["mass"])
    print(f"prec={prec}: mass drift {drift:.3e} over {nsteps} steps (bound {bound:.3e})")
    assert drift <= bound
    assert np.all(np.abs(d1["momentum"] - d0["momentum"]) <= bound)
    lat.close()
    del rho, u
    torch.cuda.empty_cache()


def test_shear_layer_4096_sampled():
    from paper_2303_08163_gb300 import lbm
    n = 4096
    dims = (n, n, 1)
    tau = 0.5 + 3e-5
    rho, u = inputs.double_shear_layer(n)
    rho_fn, u_fn = inputs.double_shear_layer_fields(n)
    for eq in (core.EQ_ENTROPIC, core.EQ_POLY2):
        lat = lbm.Lattice(lbm.D2Q9, dims, tau, eq, 0, lbm.F32)
        lat.init_fields(rho, u)
        lat.set_option(lbm.OPT_TUNE, 1)
        lat.init_fields(rho, u)
        cells = sample_cells(dims, 48, seed=11)
        cells[:, 2] = 0
        lat.step(1)
        check_sampled(lat, 2, dims, eq, 0, tau, 1, rho_fn, u_fn, 1, cells, 0.1)
        lat.step(1)
        check_sampled(lat, 2, dims, eq, 0, tau, 1, rho_fn, u_fn, 2, cells, 0.1)
        lat.close()


def test_batch_4096_sampled_instances():
    from paper_2303_08163_gb300 import lbm
    table = inputs.linear_mode_batch(count=4096, seed=2303)
    count = len(table["nx"])
    dims = np.stack([table["nx"], table["ny"], np.ones(count, dtype=np.int32)], axis=1)
    fields = [inputs.linear_mode_fields(table, k) for k in range(count)]
    rho = np.concatenate([f[0] for f in fields])
    u = np.concatenate([f[1].reshape(-1) for f in fields])
    kvec = np.stack([table["nmode"], np.zeros(count, np.int32), np.zeros(count, np.int32)], axis=1)
    b = lbm.Batch(lbm.D2Q9, dims, table["tau"], core.EQ_ENTROPIC, 0)
    b.init_fields(rho, u)
    b.set_probe(kvec, 10)
    steps = 61
    b.step(steps)
    series = b.probe_series()
    pops = b.get_populations()
    assert np.all(b.status() == 0)
    ncells = dims.prod(axis=1)
    order = np.argsort(ncells)
    picks = list(order[:4]) + list(np.random.default_rng(1).choice(order[: count // 2], 4, replace=False))
    for k in picks:
        d3 = (int(dims[k, 0]), int(dims[k, 1]), 1)
        f0 = core.init(2, d3, core.EQ_ENTROPIC, fields[k][0], fields[k][1])
        fk, sk = core.run_probed(2, d3, core.EQ_ENTROPIC, 0, float(table["tau"][k]), steps, 10,
                                 tuple(kvec[k]), f0)
        c0, c1 = b.cell_start[k], b.cell_start[k + 1]
        gk = pops[9 * c0: 9 * c1].reshape(9, -1)
        assert float(np.max(np.abs(gk - fk) / np.abs(fk))) <= 1e-12
        assert np.all(np.abs(series[k] - sk) <= 1e-12 * np.abs(sk) + 1e-13 * int(c1 - c0))
    b.close()


@pytest.mark.parametrize("shape", [(2, 256, 2, 1, 1304, 4096), (1, 256)])
def test_lattice_over_2_31_cells(shape):
    """The largest lattice the 280 GB of HBM holds comfortably: 1304^3 = 2.22e9 cells
    (more than 2^31), 120 GB of binary16 populations.  Cell and population indices exceed
    32 bits, so this checks the 64-bit indexing of the initialisation, of the TMA step
    (whole 2608-byte rows, one per job) and of the one-cell step, and the sampled export,
    against the oracle on sampled cells after an even and an odd number of steps."""
    import torch
    from paper_2303_08163_gb300 import lbm
    n, u0 = 1304, 0.1
    assert n ** 3 > 2 ** 31
    tau = 0.5 + 3 * u0 * (n / (2 * math.pi)) / 1600.0
    dims = (n, n, n)
    rho, u = inputs.taylor_green_3d_torch(n, u0=u0, device="cuda")
    rho_fn, u_fn = inputs.taylor_green_3d_fields(n, u0=u0)
    lat = lbm.Lattice(lbm.D3Q27, dims, tau, lbm.ENTROPIC, 0, lbm.F16S)
    lat.set_launch_shape(*shape)
    lat.init_fields(rho, u, dtype=np.float32)
    del rho, u
    torch.cuda.empty_cache()
    assert lat.launch_info()["kernel"] == shape[0]
    cells = sample_cells(dims, 32, seed=13)
    cells[-1] = (n - 1, n - 1, n - 1)  # the last cell: index n^3 - 1 > 2^31
    lat.step(1)
    check_sampled(lat, 3, dims, core.EQ_ENTROPIC, 0, tau, 2, rho_fn, u_fn, 1, cells, u0)
    lat.step(1)
    check_sampled(lat, 3, dims, core.EQ_ENTROPIC, 0, tau, 2, rho_fn, u_fn, 2, cells, u0)
    lat.close()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", [2, 1])
def test_turbulence_1024x512x512_sampled(prec):
    """The decaying-turbulence box at full size (1024 x 512 x 512, tau - 1/2 = 1e-4, the
    random solenoidal field with E(k) ~ k^4 exp(-2 (k/8)^2), u_rms = 0.05) in the autotuned
    launch shape: sampled cells after 1 and 2 steps against the oracle, which starts from
    the same generated field values (gathered at each patch)."""
    import torch
    from paper_2303_08163_gb300 import lbm
    dims = (1024, 512, 512)
    nx, ny, _ = dims
    tau = 0.5 + 1e-4
    rho, u = inputs.random_solenoidal_torch(dims, u_rms=0.05, device="cuda")
    umax = 1.1 * float(u.abs().max())  # of the input field, with room for two steps

    def gather(t, ix, iy, iz):
        flat = torch.from_numpy(np.ascontiguousarray(ix + nx * (iy + ny * iz), dtype=np.int64).reshape(-1))
        return t[..., flat.to(t.device)].double().cpu().numpy()

    def rho_fn(ix, iy, iz):
        return gather(rho, ix, iy, iz).reshape(np.shape(ix))

    def u_fn(ix, iy, iz):
        return gather(u, ix, iy, iz).reshape((3,) + np.shape(ix))

    lat = lbm.Lattice(lbm.D3Q27, dims, tau, lbm.ENTROPIC, 0, prec)
    lat.init_fields(rho, u, dtype=np.float32)
    lat.set_option(lbm.OPT_TUNE, 1)  # the benchmark's launch shape
    assert lat.launch_info()["kernel"] == lbm.KERNEL_TMA
    lat.init_fields(rho, u, dtype=np.float32)
    cells = sample_cells(dims, 32, seed=29 + prec)
    lat.step(1)
    check_sampled(lat, 3, dims, core.EQ_ENTROPIC, 0, tau, prec, rho_fn, u_fn, 1, cells, umax)
    lat.step(1)
    check_sampled(lat, 3, dims, core.EQ_ENTROPIC, 0, tau, prec, rho_fn, u_fn, 2, cells, umax)
    lat.close()
    del rho, u
    torch.cuda.empty_cache()
