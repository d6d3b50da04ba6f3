"""GPU parity at the full benchmark sizes, in the launch shape the benchmark uses (the
autotuned one), on outputs the oracle can compute one by one:

- D3Q27 512^3 Taylor-Green (Re = 1600), binary16 and FP32 shifted storage: populations of
  sampled cells after 1 and 2 steps (the oracle evaluates a (2n+1)^3 patch around each
  cell), and global mass / momentum over 40 steps.
- D2Q9 4096^2 double shear layer, FP32: sampled cells after 1 and 2 steps.
- 4096 batched D2Q9 instances (FP64) in the batch tuner's launch shape: probe series and
  final populations of sampled instances equal the oracle's to 1e-12.
- D3Q27 1024 x 512 x 512 decaying turbulence, binary16 and FP32: sampled cells after 1 and
  2 steps.
- The largest lattice: 1304^3 cells (more than 2^31), binary16, both step kernels.

- The same 512^3 lattice filled with a field that varies from cell to cell (uniform
  random rho and u per cell), binary16 and FP32: sampled cells after 1 and 2 steps.  On
  the smooth vortex a wrong-neighbour read changes a population by about w_i |grad u|,
  which lies inside the rounding bound; on this field it changes it by about
  w_i |delta rho + 3 delta u|, far outside (tests/test_fullsize_power.py shows both on the
  CPU with the oracle).
- The autotuned TMA kernel against the one-cell kernel at 512^3 (binary16 and FP32), on
  the 1024 x 512 x 512 turbulence box (binary16) and on the 4096^2 D2Q9 shear layer (FP32
  in segments with halos, binary16 in whole 8 KB rows with the paired bodies): the stored
  states after 1, 2 and 3 steps are identical bit for bit (both kernels evaluate the same
  collision on the same stored values, so any data-movement error shows up as a
  difference).

The rounding bound of the sampled checks is derived in tests/fullsize_bounds.py.
"""
import math

import numpy as np
import pytest

from fullsize_bounds import UNIT, sampled_tolerance
from oracle import core
from paper_2303_08163_gb300 import inputs

pytestmark = pytest.mark.gpu


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


def check_sampled(lat, D, dims, eq, bulk, tau, prec, rho_fn, u_fn, nsteps, cells, umax, rho_min=0.9):
    got = lat.sample_populations(flat(cells, dims))
    ref = core.local_populations(D, dims, eq, bulk, tau, nsteps, rho_fn, u_fn, cells)
    _, w = core.lattice(D)
    # storage roundings of this population, plus those reaching it through rho and u
    # (first order, amplified by at most omega K), plus the FP32 collision arithmetic
    tol = sampled_tolerance(ref, w, D, tau, prec, nsteps, umax, rho_min)
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
    b.autotune(steps=4)  # the benchmark's launch shape
    print(f"batch tuned shape {b.launch_info()}")
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


def test_tune_lattice_larger_than_half_of_hbm():
    """The tuner needs no copy of the state: a binary16 D3Q27 lattice holding more than half
    of the device's memory (1400^3 cells, about 148 GB, on a 284 GB GB300) is tuned in
    place (the candidates run on a proxy of at most 2 GiB); the tuned TMA step then
    matches the oracle on sampled cells after 1 and 2 steps."""
    import torch
    from paper_2303_08163_gb300 import lbm
    total = torch.cuda.get_device_properties(0).total_memory
    n = 8
    while n ** 3 * 27 * 2 <= 0.52 * total:
        n += 8
    u0 = 0.1
    tau = 0.5 + 3 * u0 * (n / (2 * math.pi)) / 1600.0
    dims = (n, n, n)
    lat = lbm.Lattice(lbm.D3Q27, dims, tau, lbm.ENTROPIC, 0, lbm.F16S)
    state = lat.launch_info()["storage_bytes"]
    assert state > total / 2
    rho, u = inputs.taylor_green_3d_torch(n, u0=u0, device="cuda")
    lat.init_fields(rho, u, dtype=np.float32)
    del rho, u
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    assert free < state  # a full copy of the state would not fit
    lat.set_option(lbm.OPT_TUNE, 1)
    info = lat.launch_info()
    print(f"{n}^3: state {state / 1e9:.1f} GB of {total / 1e9:.1f} GB, tuned shape {info}")
    assert info["kernel"] == lbm.KERNEL_TMA and lat.step_count == 0
    rho_fn, u_fn = inputs.taylor_green_3d_fields(n, u0=u0)
    cells = sample_cells(dims, 24, seed=14)
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


@pytest.mark.parametrize("case,prec", [("tgv512", 2), ("tgv512", 1), ("turb", 2), ("shear4096", 1),
                                       ("shear4096", 2)])
def test_fullsize_tma_equals_one_cell_bitwise(case, prec):
    """At the full benchmark sizes and in the autotuned launch shape (whatever it is on
    this device: rows per job, segments, stages, threads, the paired binary16 body), the
    TMA kernel's stored state equals the one-cell kernel's bit for bit after 1, 2 and 3
    steps (Eq. 1: collide, then stream; both kernels evaluate the same collision on the
    same stored values, so only a data-movement error can make them differ).  The tuner
    must also leave the state it was called on untouched."""
    import torch
    from paper_2303_08163_gb300 import lbm
    lattice = lbm.D3Q27
    if case == "tgv512":
        n, u0 = 512, 0.1
        dims = (n, n, n)
        tau = 0.5 + 3 * u0 * (n / (2 * math.pi)) / 1600.0
        rho, u = inputs.taylor_green_3d_torch(n, u0=u0, device="cuda")
    elif case == "shear4096":
        # the double shear layer: FP32 rows of 16 KB run as segments with halos, binary16
        # rows of 8 KB whole, with up to 512 threads and the paired D2Q9 bodies
        lattice = lbm.D2Q9
        dims = (4096, 4096, 1)
        tau = 0.5 + 3e-5
        r_np, u_np = inputs.double_shear_layer(4096, dtype=np.float32)
        rho, u = torch.from_numpy(r_np).cuda(), torch.from_numpy(np.ascontiguousarray(u_np)).cuda()
    else:
        dims = (1024, 512, 512)
        tau = 0.5 + 1e-4
        rho, u = inputs.random_solenoidal_torch(dims, u_rms=0.05, device="cuda")
    ncell = int(np.prod(dims))
    Q = 27 if lattice == lbm.D3Q27 else 9
    store = {1: torch.int32, 2: torch.int16}[prec]
    a = lbm.Lattice(lattice, dims, tau, lbm.ENTROPIC, 0, prec)
    a.init_fields(rho, u, dtype=np.float32)
    before = torch.empty(Q * ncell, dtype=store, device="cuda")
    a.get_populations("storage", out=before)
    a.set_option(lbm.OPT_TUNE, 1)  # the benchmark's launch shape
    after = torch.empty_like(before)
    a.get_populations("storage", out=after)
    assert torch.equal(before, after), "the tuner changed the state"
    assert a.step_count == 0
    del before
    info = a.launch_info()
    print(f"{case} prec={prec}: tuned shape {info}")
    assert info["kernel"] == lbm.KERNEL_TMA
    b = lbm.Lattice(lattice, dims, tau, lbm.ENTROPIC, 0, prec)
    b.set_launch_shape(lbm.KERNEL_GENERIC, 256)
    b.init_fields(rho, u, dtype=np.float32)
    del rho, u
    torch.cuda.empty_cache()
    other = torch.empty_like(after)
    for n in (1, 2, 3):
        a.step(1)
        b.step(1)
        a.get_populations("storage", out=after)
        b.get_populations("storage", out=other)
        same = torch.equal(after, other)
        if not same:
            idx = torch.nonzero(after != other)[:4].flatten().tolist()
            raise AssertionError(f"after {n} steps the kernels differ at flat indices {idx} "
                                 f"(direction = index // {ncell})")
    a.sync()
    b.sync()
    for x in (a, b):
        x.close()
    del after, other
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", [2, 1])
def test_512_nonsmooth_field_sampled(prec):
    """512^3 lattice in the autotuned shape, filled with uniform random rho in [0.9, 1.1]
    and u_a in [-0.1, 0.1] drawn independently for every cell (a seeded generator on the
    device), tau of the Re = 1600 vortex: sampled cells after 1 and 2 steps against the
    oracle, which starts from the same generated values (gathered at each patch).  Here a
    wrong neighbour, direction or layout moves a population far outside the rounding bound."""
    import torch
    from paper_2303_08163_gb300 import lbm
    n, u0 = 512, 0.1
    dims = (n, n, n)
    nx, ny, _ = dims
    tau = 0.5 + 3 * u0 * (n / (2 * math.pi)) / 1600.0
    rho, u = inputs.random_state_torch(3, dims, seed=512 + prec, rho_range=(0.9, 1.1), u_max=0.1,
                                       device="cuda")

    def gather(t, ix, iy, iz):
        idx = torch.from_numpy(np.ascontiguousarray(ix + nx * (iy + ny * iz), dtype=np.int64).reshape(-1))
        return t[..., idx.to(t.device)].double().cpu().numpy()

    def rho_fn(ix, iy, iz):
        return gather(rho, ix, iy, iz).reshape(np.shape(ix))

    def u_fn(ix, iy, iz):
        return gather(u, ix, iy, iz).reshape((3,) + np.shape(ix))

    lat = lbm.Lattice(lbm.D3Q27, dims, tau, lbm.ENTROPIC, 0, prec)
    lat.init_fields(rho, u, dtype=np.float32)
    lat.set_option(lbm.OPT_TUNE, 1)
    assert lat.launch_info()["kernel"] == lbm.KERNEL_TMA
    cells = sample_cells(dims, 40, seed=77 + prec)
    lat.step(1)
    # bounds of the field a step or two later: |u_a| <= 0.12, rho >= 0.85
    check_sampled(lat, 3, dims, core.EQ_ENTROPIC, 0, tau, prec, rho_fn, u_fn, 1, cells, 0.12, rho_min=0.85)
    lat.step(1)
    check_sampled(lat, 3, dims, core.EQ_ENTROPIC, 0, tau, prec, rho_fn, u_fn, 2, cells, 0.12, rho_min=0.85)
    lat.close()
    del rho, u
    torch.cuda.empty_cache()
