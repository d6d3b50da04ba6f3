"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle, element by
element on the same seeded inputs.

Tolerances:
- FP64 storage: max relative error per population <= 1e-12 (after up to 1000 steps).
  Both sides evaluate the same formulas in IEEE FP64; they differ only by rounding
  order (the GPU uses fused multiply-adds, 1/rho then a product, and the identity
  (2 - S) Z = 2 S - 1 + 3u instead of the division by 1 - u), about 1e-16 per step.
- FP32 storage of f - w rho0 with FP32 collision: relative L2 error of the velocity
  field <= 1e-4, a tenth of the binary16 target (the FP32 collision arithmetic, a few
  ulp of O(w) quantities per step, dominates the FP32 storage rounding).
- binary16 storage with FP32 collision: relative L2 velocity error <= 1e-3 on
  Taylor-Green (the target accuracy of the reduced-precision path).
"""
import math

import numpy as np
import pytest

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


def lbm_mod():
    from paper_2303_08163_gb300 import lbm
    return lbm


def max_rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_gpu(D, dims, eq, bulk, tau, prec, rho, u, steps, shape=None, graph=False):
    lbm = lbm_mod()
    lat = lbm.Lattice(lbm.D2Q9 if D == 2 else lbm.D3Q27, dims, tau, eq, bulk, prec)
    if shape is not None:
        lat.set_launch_shape(*shape)
    if graph:
        lat.set_option(lbm.OPT_USE_GRAPH, 1)
    lat.init_fields(rho, u)
    lat.step(steps)
    f = lat.get_populations()
    info = lat.launch_info()
    lat.close()
    return f, info


def run_oracle(D, dims, eq, bulk, tau, rho, u, steps):
    return core.step(D, dims, eq, bulk, tau, steps, core.init(D, dims, eq, rho, u))


# --------------------------------------------------------------------------- FP64 parity

@pytest.mark.parametrize("kernel", ["generic", "tma"])
def test_taylor_green_64_fp64_1000_steps(kernel):
    """The small Taylor-Green configuration: D2Q9 64^2, u0 = 0.05, tau = 0.8, entropic,
    FP64, 1000 steps (and one more, to check the odd-step layout)."""
    lbm = lbm_mod()
    n, tau = 64, 0.8
    rho, u = inputs.taylor_green_2d(n, u0=0.05)
    shape = (lbm.KERNEL_GENERIC, 256) if kernel == "generic" else (lbm.KERNEL_TMA, 256, 4, 4, n, 2048)
    lat = lbm.Lattice(lbm.D2Q9, (n, n, 1), tau, lbm.ENTROPIC, 0, lbm.F64)
    lat.set_launch_shape(*shape)
    lat.init_fields(rho, u)
    lat.step(1000)
    ref = run_oracle(2, (n, n, 1), core.EQ_ENTROPIC, 0, tau, rho, u, 1000)
    assert max_rel(lat.get_populations(), ref) <= 1e-12
    lat.step(1)
    ref1 = core.step(2, (n, n, 1), core.EQ_ENTROPIC, 0, tau, 1, ref)
    assert lat.step_count == 1001
    assert max_rel(lat.get_populations(), ref1) <= 1e-12
    lat.close()


@pytest.mark.parametrize("eq", [core.EQ_POLY2, core.EQ_PRODUCT, core.EQ_ENTROPIC])
def test_d2q9_fp64_1000_steps_bulk_all_equilibria(eq):
    """D2Q9 64^2 Taylor-Green (u0 = 0.05, tau = 0.8), FP64, bulk correction on (Eq.
    eq:redefined_relaxation rate), each equilibrium, TMA and one-cell paths, the TMA path
    replayed from a CUDA graph: after 1000 and 1001 steps every population equals the
    oracle's to 1e-12 (maximum relative error)."""
    import os
    lbm = lbm_mod()
    n, tau = 64, 0.8
    rho, u = inputs.taylor_green_2d(n, u0=0.05)
    core.set_threads(os.cpu_count() or 1)  # the same result bit for bit as one thread
    try:
        ref = run_oracle(2, (n, n, 1), eq, 1, tau, rho, u, 1000)
        ref1 = core.step(2, (n, n, 1), eq, 1, tau, 1, ref)
    finally:
        core.set_threads(1)
    for shape, graph in (((lbm.KERNEL_TMA, 128, 3, 8, n, 4096), True), ((lbm.KERNEL_GENERIC, 128), False)):
        lat = lbm.Lattice(lbm.D2Q9, (n, n, 1), tau, eq, 1, lbm.F64)
        lat.set_launch_shape(*shape)
        if graph:
            lat.set_option(lbm.OPT_USE_GRAPH, 1)
        lat.init_fields(rho, u)
        lat.step(1000)
        assert max_rel(lat.get_populations(), ref) <= 1e-12
        lat.step(1)
        assert max_rel(lat.get_populations(), ref1) <= 1e-12
        lat.close()


def test_batch_fp64_1000_steps():
    """Batched D2Q9 instances (ragged sizes, per-instance tau, shear and acoustic waves on
    background flows), entropic with the bulk correction, FP64: 1000 steps in three calls
    (three persistent launches from CUDA graphs), probes every 50 steps; populations and
    probe series equal the oracle's instance by instance to 1e-12."""
    lbm = lbm_mod()
    table = inputs.linear_mode_batch(count=10, seed=19, nmin=6, nmax=32)
    count = len(table["nx"])
    dims = np.stack([table["nx"], table["ny"], np.ones(count, dtype=np.int32)], axis=1)
    fields = [inputs.linear_mode_fields(table, k) for k in range(count)]
    rho = np.concatenate([f[0] for f in fields])
    u = np.concatenate([f[1].reshape(-1) for f in fields])
    kvec = np.stack([table["nmode"], np.zeros(count, np.int32), np.zeros(count, np.int32)], axis=1)
    b = lbm.Batch(lbm.D2Q9, dims, table["tau"], core.EQ_ENTROPIC, 1)
    b.init_fields(rho, u)
    b.set_probe(kvec, 50)
    for n in (333, 444, 223):
        b.step(n)
    assert b.info()["step"] == 1000
    series, pops = b.probe_series(), b.get_populations()
    assert np.all(b.status() == 0)
    for k in range(count):
        d3 = (int(dims[k, 0]), int(dims[k, 1]), 1)
        f0 = core.init(2, d3, core.EQ_ENTROPIC, fields[k][0], fields[k][1])
        fk, sk = core.run_probed(2, d3, core.EQ_ENTROPIC, 1, float(table["tau"][k]), 1000, 50, tuple(kvec[k]), f0)
        c0, c1 = b.cell_start[k], b.cell_start[k + 1]
        assert max_rel(pops[9 * c0: 9 * c1].reshape(9, -1), fk) <= 1e-12
        assert np.all(np.abs(series[k] - sk) <= 1e-12 * np.abs(sk) + 1e-13 * int(c1 - c0))
    b.close()


# D3Q27 FP64 over 1000 steps: (name, dims, fields, tau, launch shapes).  The TMA shapes
# cover several whole rows per job with a ragged last row group (y wrap) and aligned
# row segments with halos; the one-cell kernel is the second path.
D3Q27_1000 = [
    ("taylor-green 16^3", (16, 16, 16), "tgv", 0.8,
     [(2, 128, 3, 4, 16, 1024), (1, 256)]),
    ("random 12x10x8", (12, 10, 8), "random", 0.6,
     [(2, 128, 2, 3, 12, 1024), (2, 128, 2, 1, 4, 1024), (1, 128)]),
]


@pytest.mark.parametrize("name,dims,field,tau,shapes", D3Q27_1000, ids=[c[0] for c in D3Q27_1000])
@pytest.mark.parametrize("bulk", [0, 1])
@pytest.mark.parametrize("eq", [core.EQ_ENTROPIC, core.EQ_POLY2, core.EQ_PRODUCT])
def test_d3q27_fp64_1000_steps(name, dims, field, tau, shapes, bulk, eq):
    """D3Q27, FP64, each equilibrium (entropic Eq. eq:Entropic_isothermal_EDF, quadratic
    Eq. eq:Poly2_isothermal_EDF, product form Eq. eq:Product_isothermal_EDF), bulk
    correction off and on (Eq. eq:redefined_relaxation rate): after 1000 steps every
    population of every kernel path equals the oracle's to 1e-12 (maximum relative
    error), and again one step later (the other AA layout)."""
    import os
    lbm = lbm_mod()
    n = int(np.prod(dims))
    if field == "tgv":
        rho, u = inputs.taylor_green_3d(dims[0], u0=0.05)
    else:
        rho, u = inputs.random_state(3, dims, seed=1000 + bulk + 10 * eq, rho_range=(0.9, 1.1), u_max=0.1)
    assert rho.shape == (n,)
    core.set_threads(os.cpu_count() or 1)  # the same result bit for bit as one thread
    try:
        ref = run_oracle(3, dims, eq, bulk, tau, rho, u, 1000)
        ref1 = core.step(3, dims, eq, bulk, tau, 1, ref)
    finally:
        core.set_threads(1)
    for shape in shapes:
        lat = lbm.Lattice(lbm.D3Q27, dims, tau, eq, bulk, lbm.F64)
        lat.set_launch_shape(*shape)
        assert lat.launch_info()["kernel"] == shape[0]
        lat.init_fields(rho, u)
        lat.step(1000)
        err = max_rel(lat.get_populations(), ref)
        lat.step(1)
        err1 = max_rel(lat.get_populations(), ref1)
        print(f"{name} eq={eq} bulk={bulk} shape={shape}: max rel error {err:.2e} (1000 steps), {err1:.2e} (1001)")
        assert err <= 1e-12 and err1 <= 1e-12
        lat.close()


# (D, dims, launch shape) covering: whole rows with several rows per job and y wrap,
# aligned segments with halos and a shorter last segment, ragged Nx (generic only).
SHAPES = [
    (2, (40, 18, 1), (2, 256, 3, 4, 40, 2048)),
    (2, (40, 18, 1), (2, 128, 2, 1, 16, 1024)),
    (2, (13, 11, 1), (1, 128)),
    (3, (12, 10, 6), (2, 128, 3, 3, 12, 1024)),
    (3, (12, 10, 6), (2, 256, 2, 1, 4, 1024)),
    (3, (7, 5, 6), (1, 256)),
]


@pytest.mark.parametrize("D,dims,shape", SHAPES)
@pytest.mark.parametrize("eq", [core.EQ_ENTROPIC, core.EQ_POLY2, core.EQ_PRODUCT])
@pytest.mark.parametrize("bulk", [0, 1])
def test_fp64_parity_all_paths(D, dims, shape, eq, bulk):
    """Every equilibrium, with and without the bulk correction, through every kernel
    path, after an odd number of steps: max relative error per population <= 1e-12."""
    rho, u = inputs.random_state(D, dims, seed=100 + 7 * eq + bulk + D, u_max=0.12)
    steps, tau = 11, 0.57
    got, info = run_gpu(D, dims, eq, bulk, tau, 0, rho, u, steps, shape=shape)
    assert info["kernel"] == shape[0]
    ref = run_oracle(D, dims, eq, bulk, tau, rho, u, steps)
    assert max_rel(got, ref) <= 1e-12


# Launch shapes of the reduced-precision TMA kernels (rows must be 16-byte multiples):
# whole rows with several rows per job and y wrap, and aligned segments with halos and a
# shorter last segment.
RP_SHAPES = [
    (2, (40, 18, 1), (2, 256, 3, 4, 40, 2048)),
    (2, (40, 18, 1), (2, 128, 2, 1, 16, 1024)),
    (3, (24, 10, 6), (2, 128, 3, 3, 24, 1024)),
    (3, (24, 10, 6), (2, 256, 2, 1, 8, 1024)),
]


@pytest.mark.parametrize("D,dims,shape", RP_SHAPES)
@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("eq", [core.EQ_ENTROPIC, core.EQ_POLY2, core.EQ_PRODUCT])
@pytest.mark.parametrize("bulk", [0, 1])
def test_reduced_precision_tma_shapes(D, dims, shape, prec, eq, bulk):
    """FP32 and binary16 storage through every TMA job layout, after an even and two odd
    numbers of steps.  The TMA kernel and the one-cell-per-thread kernel evaluate the same
    collision on the same stored values, so their stored states must agree bit for bit
    (this checks the data movement of every layout: rows, y wrap, segments and their
    halos, paired binary16 accesses); the velocity field must match the oracle within the
    reduced-precision tolerance (relative L2 1e-4 for FP32, 1e-3 for binary16)."""
    lbm = lbm_mod()
    rho, u = inputs.random_state(D, dims, seed=300 + 11 * eq + 3 * bulk + D + prec, u_max=0.12)
    tau = 0.57
    lats = []
    for sh in (shape, (1, 128)):
        lat = lbm.Lattice(lbm.D2Q9 if D == 2 else lbm.D3Q27, dims, tau, eq, bulk, prec)
        lat.set_launch_shape(*sh)
        lat.init_fields(rho, u)
        lats.append(lat)
    assert lats[0].launch_info()["kernel"] == 2 and lats[1].launch_info()["kernel"] == 1
    ref = core.init(D, dims, eq, rho, u)
    done = 0
    for n in (2, 3, 5):
        for lat in lats:
            lat.step(n - done)
        ref = core.step(D, dims, eq, bulk, tau, n - done, ref)
        done = n
        a, b = (lat.get_populations("storage") for lat in lats)
        diff = np.argwhere(a.view(np.uint8) != b.view(np.uint8))
        assert diff.size == 0, f"after {n} steps the TMA and one-cell kernels differ at {diff[:4].tolist()}"
        _, ug = core.moments(D, dims, lats[0].get_populations())
        _, ur = core.moments(D, dims, ref)
        err = rel_l2(ug, ur)
        assert err <= {1: 1e-4, 2: 1e-3}[prec], f"after {n} steps rel-L2 velocity error {err:.3e}"
    for lat in lats:
        lat.close()


@pytest.mark.parametrize("prec", [0, 2])
def test_host_buffers_pinned_pageable_device_agree(prec):
    """lbm_init_fields and lbm_moments with page-locked host buffers (read and written by
    the kernels across the link), pageable host buffers (staged) and device buffers give the
    same state and the same moments bit for bit, for a single lattice and for a batch."""
    import torch
    lbm = lbm_mod()
    dims = (40, 12, 9)
    n = int(np.prod(dims))
    rho, u = inputs.random_state(3, dims, seed=71, u_max=0.1)
    rho32, u32 = rho.astype(np.float32), u.astype(np.float32)
    srcs = {"pageable": (rho32, u32),
            "pinned": (torch.from_numpy(rho32).pin_memory(), torch.from_numpy(u32).pin_memory()),
            "device": (torch.from_numpy(rho32).cuda(), torch.from_numpy(u32).cuda())}
    states, moms = {}, {}
    for name, (r, v) in srcs.items():
        lat = lbm.Lattice(lbm.D3Q27, dims, 0.6, lbm.ENTROPIC, 1, prec)
        lat.init_fields(r, v, dtype=np.float32)
        lat.step(3)
        states[name] = lat.get_populations("storage")
        if name == "pageable":
            moms[name] = lat.moments(dtype=np.float32)
        else:
            out = (torch.empty(n, dtype=torch.float32), torch.empty(3, n, dtype=torch.float32))
            if name == "pinned":
                out = tuple(t.pin_memory() for t in out)
            else:
                out = tuple(t.cuda() for t in out)
            lat.moments(dtype=np.float32, out=out)
            torch.cuda.synchronize()
            moms[name] = tuple(t.cpu().numpy() for t in out)
        lat.close()
    for name in ("pinned", "device"):
        assert np.array_equal(states[name].view(np.uint8), states["pageable"].view(np.uint8)), name
        for a, b in zip(moms[name], moms["pageable"]):
            assert np.array_equal(a.reshape(-1).view(np.uint32), b.reshape(-1).view(np.uint32)), name
    # batch: pinned fields in and pinned moments out against pageable
    table = inputs.linear_mode_batch(count=9, seed=3, nmin=5, nmax=30)
    bd = np.stack([table["nx"], table["ny"], np.ones(9, dtype=np.int32)], axis=1)
    fields = [inputs.linear_mode_fields(table, k) for k in range(9)]
    br = np.concatenate([f[0] for f in fields])
    bu = np.concatenate([f[1].reshape(-1) for f in fields])
    res = {}
    for name in ("pageable", "pinned"):
        b = lbm.Batch(lbm.D2Q9, bd, table["tau"], lbm.ENTROPIC, 0)
        if name == "pinned":
            b.init_fields(torch.from_numpy(br).pin_memory(), torch.from_numpy(bu).pin_memory())
        else:
            b.init_fields(br, bu)
        b.step(5)
        if name == "pinned":
            out = (torch.empty(len(br), dtype=torch.float64).pin_memory(),
                   torch.empty(len(bu), dtype=torch.float64).pin_memory())
            b.moments(out=out)
            res[name] = (b.get_populations(), out[0].numpy().copy(), out[1].numpy().copy())
        else:
            r2, u2 = b.moments()
            res[name] = (b.get_populations(), r2, u2)
        b.close()
    for a, c in zip(res["pinned"], res["pageable"]):
        assert np.array_equal(a.view(np.uint64), c.view(np.uint64))


def test_init_and_moments_fp64():
    """f = f^eq(rho, u) at t = 0 and the exported moments match the oracle."""
    lbm = lbm_mod()
    D, dims = 3, (8, 6, 5)
    rho, u = inputs.random_state(D, dims, seed=3, u_max=0.3)
    lat = lbm.Lattice(lbm.D3Q27, dims, 0.7, lbm.ENTROPIC, 0, lbm.F64)
    lat.init_fields(rho, u)
    assert max_rel(lat.get_populations(), core.init(D, dims, core.EQ_ENTROPIC, rho, u)) <= 1e-13
    r, v = lat.moments()
    np.testing.assert_allclose(r, rho, rtol=1e-14)
    np.testing.assert_allclose(v, u, rtol=1e-12, atol=1e-15)
    lat.close()


# --------------------------------------------------------------------- reduced precision

@pytest.mark.parametrize("prec,tol", [(1, 1e-4), (2, 1e-3)])
def test_reduced_precision_taylor_green_2d(prec, tol):
    """D2Q9 64^2 Taylor-Green, 500 steps: relative L2 velocity error against FP64."""
    n, tau, steps = 64, 0.8, 500
    rho, u = inputs.taylor_green_2d(n, u0=0.05)
    got, _ = run_gpu(2, (n, n, 1), core.EQ_ENTROPIC, 0, tau, prec, rho, u, steps)
    ref = run_oracle(2, (n, n, 1), core.EQ_ENTROPIC, 0, tau, rho, u, steps)
    _, ug = core.moments(2, (n, n, 1), got)
    _, ur = core.moments(2, (n, n, 1), ref)
    err = rel_l2(ug, ur)
    print(f"D2Q9 TGV {n}^2 prec={prec} steps={steps}: rel-L2 velocity error {err:.3e}")
    assert err <= tol, f"rel-L2 velocity error {err:.3e} > {tol}"


@pytest.mark.parametrize("prec,tol", [(1, 1e-4), (2, 1e-3)])
@pytest.mark.parametrize("bulk", [0, 1])
def test_reduced_precision_taylor_green_3d(prec, tol, bulk):
    """D3Q27 32^3 Taylor-Green at Re = 1600 (u0 = 0.1, nu = u0 (N / 2 pi) / Re), four
    convective times N / (2 pi u0): relative L2 velocity error against FP64."""
    n, u0 = 32, 0.1
    nu = u0 * (n / (2 * math.pi)) / 1600.0
    tau = 0.5 + 3 * nu
    steps = int(round(4 * n / (2 * math.pi * u0)))
    rho, u = inputs.taylor_green_3d(n, u0=u0)
    dims = (n, n, n)
    got, _ = run_gpu(3, dims, core.EQ_ENTROPIC, bulk, tau, prec, rho, u, steps)
    ref = run_oracle(3, dims, core.EQ_ENTROPIC, bulk, tau, rho, u, steps)
    _, ug = core.moments(3, dims, got)
    _, ur = core.moments(3, dims, ref)
    err = rel_l2(ug, ur)
    print(f"D3Q27 TGV {n}^3 prec={prec} bulk={bulk} steps={steps}: rel-L2 velocity error {err:.3e}")
    assert err <= tol, f"rel-L2 velocity error {err:.3e} > {tol}"


# ----------------------------------------------------------------------- diagnostics

def test_fused_diagnostics_match_oracle():
    lbm = lbm_mod()
    n, tau = 48, 0.7
    rho, u = inputs.taylor_green_2d(n, u0=0.08)
    lat = lbm.Lattice(lbm.D2Q9, (n, n, 1), tau, lbm.ENTROPIC, 1, lbm.F64)
    lat.set_option(lbm.OPT_DIAG_EVERY, 5)
    lat.init_fields(rho, u)
    lat.step(23)
    hist = lat.diag_history()
    assert [h["step"] for h in hist] == [0, 5, 10, 15, 20]
    f = core.init(2, (n, n, 1), core.EQ_ENTROPIC, rho, u)
    t = 0
    for h in hist:
        f = core.step(2, (n, n, 1), core.EQ_ENTROPIC, 1, tau, h["step"] - t, f)
        t = h["step"]
        d = core.diagnostics(2, (n, n, 1), f)
        assert abs(h["mass"] - d["mass"]) <= 1e-12 * d["mass"]
        np.testing.assert_allclose(h["momentum"], d["momentum"], atol=1e-12 * d["mass"])
        assert abs(h["kinetic"] - d["kinetic"]) <= 1e-11 * d["kinetic"]
        assert abs(h["max_u"] - d["max_u"]) <= 1e-13
        assert h["nonfinite"] == 0
    now = lat.diagnostics()
    f = core.step(2, (n, n, 1), core.EQ_ENTROPIC, 1, tau, 23 - t, f)
    d = core.diagnostics(2, (n, n, 1), f)
    assert now["step"] == 23
    assert abs(now["kinetic"] - d["kinetic"]) <= 1e-11 * d["kinetic"]
    lat.close()


DIAG_CASES = [
    (2, (64, 64, 1), None),
    (2, (64, 64, 1), (1, 256)),
    (3, (24, 20, 12), None),
    (3, (24, 20, 12), (2, 128, 2, 2, 24, 2048)),
    (3, (24, 20, 12), (1, 128)),
]


@pytest.mark.parametrize("D,dims,shape", DIAG_CASES)
@pytest.mark.parametrize("prec", [1, 2])
def test_fused_diagnostics_reduced_precision(D, dims, shape, prec):
    """Fused diagnostics of the FP32 and binary16 paths (every kernel, the paired binary16
    body included) against the oracle's compensated sums over the same state (exported as
    FP64 at the step the record describes): mass and momentum (the conservation
    constraints of Sec. II), kinetic energy, max |u_a|.  The kernels form each cell's
    moments in FP32 from its Q stored values (up to Q roundings of terms bounded by
    S_c = sum_i |f_i - w_i rho0|) and add at most 128 cells in FP32 before an FP64 sum, so
    |sum_gpu - sum_ref| <= 2^-24 (Q + 128) sum_c S_c for mass and momentum; the kinetic
    energy gets 2^-24 [(Q + 138) E + Q sum_c |u_c| S_c] (the FP32 u = j / rho and the
    products), max |u| 2^-24 Q max_c S_c / rho + 4 ulp; everything twice for safety.  A
    missed or doubled cell changes the mass by about rho, far outside these bounds."""
    lbm = lbm_mod()
    Q = 3 ** D
    if D == 2:
        rho, u = inputs.taylor_green_2d(dims[0], u0=0.08)
    else:
        rho, u = inputs.random_state(3, dims, seed=41 + prec, rho_range=(0.9, 1.1), u_max=0.1)
    lat = lbm.Lattice(lbm.D2Q9 if D == 2 else lbm.D3Q27, dims, 0.6, lbm.ENTROPIC, 1, prec)
    if shape is not None:
        lat.set_launch_shape(*shape)
    lat.set_option(lbm.OPT_DIAG_EVERY, 3)
    lat.init_fields(rho, u)
    f0 = lat.get_populations()
    lat.step(6)
    f6 = lat.get_populations()
    lat.step(1)
    hist = lat.diag_history()
    assert [h["step"] for h in hist] == [0, 3, 6]
    _, w = core.lattice(D)
    eps = 2.0 ** -24
    for h, f in ((hist[0], f0), (hist[2], f6)):
        d = core.diagnostics(D, dims, f)
        S = np.abs(f - w[:, None]).sum(axis=0)
        r, v = core.moments(D, dims, f)
        speed = np.sqrt((v ** 2).sum(axis=0))
        tol_m = 2 * eps * (Q + 128) * S.sum() + 1e-13 * d["mass"]
        tol_e = 2 * eps * ((Q + 138) * d["kinetic"] + Q * (speed * S).sum())
        tol_u = 2 * eps * Q * (S / r).max() + 4 * eps * d["max_u"]
        assert h["nonfinite"] == 0
        assert abs(h["mass"] - d["mass"]) <= tol_m, (h["mass"], d["mass"], tol_m)
        assert np.all(np.abs(h["momentum"] - d["momentum"]) <= tol_m), (h["momentum"], d["momentum"], tol_m)
        assert abs(h["kinetic"] - d["kinetic"]) <= tol_e, (h["kinetic"], d["kinetic"], tol_e)
        assert abs(h["max_u"] - d["max_u"]) <= tol_u, (h["max_u"], d["max_u"], tol_u)
    lat.close()


def test_nonfinite_state_is_reported():
    """A NaN population (fault injected on the host through lbm_set_populations) makes
    the next fused diagnostics return LBM_ENONFINITE; the object stays usable."""
    lbm = lbm_mod()
    n = 16
    rho, u = inputs.taylor_green_2d(n, u0=0.05)
    lat = lbm.Lattice(lbm.D2Q9, (n, n, 1), 0.8, lbm.ENTROPIC, 0, lbm.F32)
    lat.set_option(lbm.OPT_DIAG_EVERY, 1)
    lat.init_fields(rho, u)
    lat.step(3)
    f = lat.get_populations()
    f[4, 37] = np.nan
    lat.set_populations(f)
    with pytest.raises(lbm.LBMError) as e:
        lat.step(2)
    assert e.value.status == lbm.ENONFINITE
    assert lat.diagnostics()["nonfinite"] >= 1
    lat.close()


# ------------------------------------------------------------ checkpoint, graph, self test

@pytest.mark.parametrize("prec", [0, 1, 2])
def test_checkpoint_resume_is_bitwise(prec):
    lbm = lbm_mod()
    D, dims, tau = 3, (16, 12, 10), 0.6
    rho, u = inputs.taylor_green_3d(16, u0=0.1)
    rho, u = rho[: 16 * 12 * 10], u[:, : 16 * 12 * 10]
    a = lbm.Lattice(lbm.D3Q27, dims, tau, lbm.ENTROPIC, 1, prec)
    a.init_fields(rho, u)
    a.step(14)
    full = a.get_populations()
    b = lbm.Lattice(lbm.D3Q27, dims, tau, lbm.ENTROPIC, 1, prec)
    b.init_fields(rho, u)
    b.step(7)
    ck, t = b.get_populations("storage"), b.step_count
    c = lbm.Lattice(lbm.D3Q27, dims, tau, lbm.ENTROPIC, 1, prec)
    c.set_step_count(t)
    c.set_populations(ck, "storage")
    c.step(7)
    np.testing.assert_array_equal(c.get_populations(), full)
    np.testing.assert_array_equal(c.get_populations("storage"), a.get_populations("storage"))
    for x in (a, b, c):
        x.close()


def test_graph_replay_equals_launches():
    lbm = lbm_mod()
    n = 64
    rho, u = inputs.taylor_green_2d(n, u0=0.05)
    f1, _ = run_gpu(2, (n, n, 1), 0, 0, 0.8, 1, rho, u, 41)
    f2, _ = run_gpu(2, (n, n, 1), 0, 0, 0.8, 1, rho, u, 41, graph=True)
    np.testing.assert_array_equal(f1, f2)


def test_bounded_wait_times_out():
    """A kernel waiting on a shared-memory barrier nothing arrives on returns
    LBM_ETIMEOUT after its limit (1 ms) instead of hanging."""
    lbm = lbm_mod()
    assert lbm.selftest_bounded_wait(1_000_000) == lbm.ETIMEOUT


def test_invalid_launch_shape_is_rejected():
    lbm = lbm_mod()
    lat = lbm.Lattice(lbm.D2Q9, (40, 8, 1), 0.8, lbm.ENTROPIC, 0, lbm.F32)
    with pytest.raises(lbm.LBMError):
        lat.set_launch_shape(2, 256, 3, 1, 6, 1024)  # segment not a multiple of 4 floats
    with pytest.raises(lbm.LBMError):
        lat.set_launch_shape(2, 256, 9, 1, 40, 1024)  # too many stages
    lat.close()
    lat = lbm.Lattice(lbm.D2Q9, (40, 8, 1), 0.8, lbm.ENTROPIC, 0, lbm.F32)
    before = lat.launch_info()
    bad = [(2, 256, 3, 1, 0, 1024),            # empty segment
           (2, 256, 3, 1, -8, 1024),           # negative segment
           (2, 512, 3, 1, 40, 1024),           # 512 threads: binary16 D2Q9 only
           (2, 2 ** 32 + 64, 3, 1, 40, 1024),  # would wrap to 64 in 32 bits
           (2, 256, 2 ** 32 + 3, 1, 40, 1024),
           (1, 2 ** 32 + 128)]
    for shape in bad:
        with pytest.raises(lbm.LBMError) as e:
            lat.set_launch_shape(*shape)
        assert e.value.status == lbm.EINVAL, shape
    assert lat.launch_info() == before
    lat.close()
    lat = lbm.Lattice(lbm.D2Q9, (13, 8, 1), 0.8, lbm.ENTROPIC, 0, lbm.F32)
    assert lat.launch_info()["kernel"] == lbm.KERNEL_GENERIC  # 52-byte rows: no TMA
    with pytest.raises(lbm.LBMError):
        lat.set_launch_shape(2, 256, 3, 1, 13, 1024)
    lat.close()


def test_512_thread_shape_d2q9_binary16():
    """D2Q9 with binary16 storage accepts up to 512 colliding threads per block (the
    tuner's candidates); the state equals the one-cell kernel's bit for bit."""
    lbm = lbm_mod()
    dims = (256, 40, 1)
    rho, u = inputs.random_state(2, dims, seed=88, u_max=0.1)
    lats = []
    for shape in ((2, 512, 2, 4, 256, 2048), (1, 256)):
        lat = lbm.Lattice(lbm.D2Q9, dims, 0.57, lbm.ENTROPIC, 1, lbm.F16S)
        lat.set_launch_shape(*shape)
        lat.init_fields(rho, u)
        lats.append(lat)
    assert lats[0].launch_info()["threads"] == 512
    for n in (1, 2):
        for lat in lats:
            lat.step(1)
        a, b = (lat.get_populations("storage") for lat in lats)
        assert np.array_equal(a.view(np.uint16), b.view(np.uint16)), f"differ after {n} steps"
    for lat in lats:
        lat.close()


_TUNE_CACHE_CHILD = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2303_08163_gb300 import lbm, inputs
lbm.load()
dims = (24, 10, 6)
lat = lbm.Lattice(lbm.D3Q27, dims, 0.57, lbm.ENTROPIC, 0, lbm.F16S)
info = lat.launch_info()
ref = lbm.Lattice(lbm.D3Q27, dims, 0.57, lbm.ENTROPIC, 0, lbm.F16S)
ref.set_launch_shape(1, 128)
rho, u = inputs.random_state(3, dims, seed=5, u_max=0.1)
for x in (lat, ref):
    x.init_fields(rho, u)
    x.step(3)
same = np.array_equal(lat.get_populations("storage").view(np.uint16), ref.get_populations("storage").view(np.uint16))
print("RESULT", info["kernel"], info["stages"], info["smem_bytes"], int(same))
"""


def test_bad_tune_cache_entries_are_rejected(tmp_path):
    """Launch shapes remembered in the LBM_TUNE_CACHE file are checked against the lattice
    and the device before use: an entry with too many stages, or whose shared-memory size
    does not match its shape, is ignored (the default shape is used instead), so an edited
    or stale file cannot make a kernel overrun its shared memory."""
    import os
    import subprocess
    import sys
    import torch
    lbm = lbm_mod()
    ver = lbm.load().lbm_version()
    name = torch.cuda.get_device_name(0).replace(" ", "_")
    key = f"v{ver}|{name}|D3|P2|E0|B0|24x10x6"
    for rec in ("2 256 152 20 1 24 1024 552960",   # 20 stages: past the barrier arrays
                "2 256 152 3 3 24 1024 9999",      # shared memory does not match the shape
                "2 256 152 3 1 6 1024 82944"):     # 6-cell segments: not whole 16-byte units
        path = tmp_path / "tune.txt"
        path.write_text(f"{key} {rec}\n")
        root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
        env = dict(os.environ, LBM_TUNE_CACHE=str(path))
        r = subprocess.run([sys.executable, "-c", _TUNE_CACHE_CHILD, root], capture_output=True, text=True,
                           env=env, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        line = [x for x in r.stdout.splitlines() if x.startswith("RESULT")][-1].split()
        kernel, stages, smem, same = (int(v) for v in line[1:])
        assert (stages, smem) not in ((20, 552960), (3, 9999), (3, 82944)), line
        assert same == 1


# ------------------------------------------------------------------------------- batch

def test_batch_parity_and_probes():
    """Batched FP64 instances of ragged sizes and per-instance tau: populations after an
    odd number of steps and the probe series equal the oracle's instance by instance."""
    lbm = lbm_mod()
    table = inputs.linear_mode_batch(count=12, seed=7, nmin=5, nmax=40)
    dims = np.stack([table["nx"], table["ny"], np.ones(12, dtype=np.int32)], axis=1)
    fields = [inputs.linear_mode_fields(table, k) for k in range(12)]
    rho = np.concatenate([f[0] for f in fields])
    u = np.concatenate([f[1].reshape(-1) for f in fields])
    kvec = np.stack([table["nmode"], np.zeros(12, dtype=np.int32), np.zeros(12, dtype=np.int32)], axis=1)
    for eq, bulk in ((core.EQ_ENTROPIC, 0), (core.EQ_POLY2, 1)):
        b = lbm.Batch(lbm.D2Q9, dims, table["tau"], eq, bulk)
        b.init_fields(rho, u)
        b.set_probe(kvec, 3)
        b.step(20)
        b.step(11)
        series = b.probe_series()
        pops = b.get_populations()
        assert series.shape == (12, 11, 4)
        assert np.all(b.status() == 0)
        for k in range(12):
            d3 = (int(dims[k, 0]), int(dims[k, 1]), 1)
            f0 = core.init(2, d3, eq, fields[k][0], fields[k][1])
            fk, sk = core.run_probed(2, d3, eq, bulk, float(table["tau"][k]), 31, 3, tuple(kvec[k]), f0)
            c0, c1 = b.cell_start[k], b.cell_start[k + 1]
            gk = pops[9 * c0: 9 * c1].reshape(9, -1)
            assert max_rel(gk, fk) <= 1e-12
            # each projection sums ncell terms of order one: absolute floor ncell * 1e-13
            ncell = int(c1 - c0)
            assert np.all(np.abs(series[k] - sk) <= 1e-12 * np.abs(sk) + 1e-13 * ncell)
        b.close()


def test_batch_d3q27_parity_and_probes():
    """Batched FP64 D3Q27 instances of ragged 3-D sizes, random fields and per-instance tau,
    all three equilibria with and without the bulk correction: populations after an odd
    number of steps and the probe series equal the oracle's instance by instance."""
    lbm = lbm_mod()
    rng = np.random.default_rng(44)
    count = 6
    dims = rng.integers(3, 9, size=(count, 3)).astype(np.int32)
    taus = 0.5 + rng.uniform(0.05, 0.6, count)
    states = [inputs.random_state(3, tuple(int(v) for v in d), seed=500 + k, u_max=0.1)
              for k, d in enumerate(dims)]
    rho = np.concatenate([s[0] for s in states])
    u = np.concatenate([s[1].reshape(-1) for s in states])
    kvec = np.stack([np.ones(count, np.int32), rng.integers(0, 2, count).astype(np.int32),
                     np.ones(count, np.int32)], axis=1)
    for eq, bulk in ((core.EQ_ENTROPIC, 0), (core.EQ_POLY2, 1), (core.EQ_PRODUCT, 1)):
        b = lbm.Batch(lbm.D3Q27, dims, taus, eq, bulk)
        b.init_fields(rho, u)
        b.set_probe(kvec, 2)
        b.step(7)
        series = b.probe_series()
        pops = b.get_populations()
        assert np.all(b.status() == 0)
        for k in range(count):
            d3 = tuple(int(v) for v in dims[k])
            f0 = core.init(3, d3, eq, states[k][0], states[k][1])
            fk, sk = core.run_probed(3, d3, eq, bulk, float(taus[k]), 7, 2, tuple(kvec[k]), f0)
            c0, c1 = b.cell_start[k], b.cell_start[k + 1]
            gk = pops[27 * c0: 27 * c1].reshape(27, -1)
            assert max_rel(gk, fk) <= 1e-12
            ncell = int(c1 - c0)
            assert np.all(np.abs(series[k] - sk) <= 1e-12 * np.abs(sk) + 1e-13 * ncell)
        b.close()


def test_batch_autotune_keeps_state_and_parity():
    """lbm_batch_autotune changes only the launch shape: the populations, the step counter,
    the status and the recorded probe samples are unchanged, and stepping on with the
    chosen shape still matches the oracle (populations and probes to 1e-12).  Invalid
    shapes are rejected."""
    lbm = lbm_mod()
    table = inputs.linear_mode_batch(count=40, seed=21, nmin=6, nmax=48)
    count = len(table["nx"])
    dims = np.stack([table["nx"], table["ny"], np.ones(count, dtype=np.int32)], axis=1)
    fields = [inputs.linear_mode_fields(table, k) for k in range(count)]
    rho = np.concatenate([f[0] for f in fields])
    u = np.concatenate([f[1].reshape(-1) for f in fields])
    kvec = np.stack([table["nmode"], np.zeros(count, np.int32), np.zeros(count, np.int32)], axis=1)
    b = lbm.Batch(lbm.D2Q9, dims, table["tau"], core.EQ_ENTROPIC, 1)
    b.init_fields(rho, u)
    b.set_probe(kvec, 4)
    b.step(9)
    before, series0, st0 = b.get_populations(), b.probe_series(), b.status()
    b.autotune(steps=6)
    info = b.launch_info()
    assert info["threads"] in (64, 128, 256) and 1 <= info["blocks"] <= count
    assert b.info()["step"] == 9
    assert np.array_equal(b.get_populations(), before)
    assert np.array_equal(b.probe_series(), series0) and np.array_equal(b.status(), st0)
    b.step(14)
    series, pops = b.probe_series(), b.get_populations()
    for k in range(count):
        d3 = (int(dims[k, 0]), int(dims[k, 1]), 1)
        f0 = core.init(2, d3, core.EQ_ENTROPIC, fields[k][0], fields[k][1])
        fk, sk = core.run_probed(2, d3, core.EQ_ENTROPIC, 1, float(table["tau"][k]), 23, 4, tuple(kvec[k]), f0)
        c0, c1 = b.cell_start[k], b.cell_start[k + 1]
        assert max_rel(pops[9 * c0: 9 * c1].reshape(9, -1), fk) <= 1e-12
        assert np.all(np.abs(series[k] - sk) <= 1e-12 * np.abs(sk) + 1e-13 * int(c1 - c0))
    for threads, blocks in ((48, 4), (512, 4), (128, 0), (128, count + 1)):
        with pytest.raises(lbm.LBMError) as e:
            b.set_launch_shape(threads, blocks)
        assert e.value.status == lbm.EINVAL
    b.set_launch_shape(64, count)  # one instance per block
    assert b.launch_info()["blocks"] == count
    b.close()


# ------------------------------------------------------------------- degenerate states

TINY = [(2, (1, 1, 1)), (2, (1, 5, 1)), (2, (3, 1, 1)), (2, (2, 2, 1)), (3, (1, 1, 1)), (3, (2, 1, 3)),
        (3, (1, 4, 1))]


@pytest.mark.parametrize("D,dims", TINY)
@pytest.mark.parametrize("eq", [core.EQ_ENTROPIC, core.EQ_POLY2, core.EQ_PRODUCT])
def test_tiny_periodic_lattices_fp64(D, dims, eq):
    """Lattices so small that a cell is its own neighbour along an axis (periodic wrap onto
    itself) or has a single neighbour: FP64, bulk correction on, 57 steps, against the
    oracle to 1e-12; the same lattices as instances of one batch."""
    lbm = lbm_mod()
    rho, u = inputs.random_state(D, dims, seed=900 + 3 * eq + D, u_max=0.1)
    tau = 0.58
    got, _ = run_gpu(D, dims, eq, 1, tau, 0, rho, u, 57)
    ref = run_oracle(D, dims, eq, 1, tau, rho, u, 57)
    assert max_rel(got, ref) <= 1e-12


def test_tiny_instances_in_a_batch():
    """A batch of degenerate instances (1 x 1, 1 x 7, 2 x 1, 3 x 3 cells) beside a larger one:
    populations and probe series after 41 steps equal the oracle's instance by instance."""
    lbm = lbm_mod()
    dims = np.array([[1, 1, 1], [1, 7, 1], [2, 1, 1], [3, 3, 1], [16, 9, 1]], dtype=np.int32)
    count = len(dims)
    taus = np.array([0.6, 0.75, 0.52, 1.3, 0.9])
    states = [inputs.random_state(2, tuple(int(v) for v in d), seed=60 + k, u_max=0.1) for k, d in enumerate(dims)]
    rho = np.concatenate([st[0] for st in states])
    u = np.concatenate([st[1].reshape(-1) for st in states])
    kvec = np.array([[0, 0, 0], [0, 1, 0], [1, 0, 0], [1, 1, 0], [2, 1, 0]], dtype=np.int32)
    b = lbm.Batch(lbm.D2Q9, dims, taus, core.EQ_ENTROPIC, 1)
    b.init_fields(rho, u)
    b.set_probe(kvec, 4)
    b.step(41)
    series, pops = b.probe_series(), b.get_populations()
    assert np.all(b.status() == 0)
    for k in range(count):
        d3 = tuple(int(v) for v in dims[k])
        f0 = core.init(2, d3, core.EQ_ENTROPIC, states[k][0], states[k][1])
        fk, sk = core.run_probed(2, d3, core.EQ_ENTROPIC, 1, float(taus[k]), 41, 4, tuple(kvec[k]), f0)
        c0, c1 = b.cell_start[k], b.cell_start[k + 1]
        assert max_rel(pops[9 * c0: 9 * c1].reshape(9, -1), fk) <= 1e-12
        assert np.all(np.abs(series[k] - sk) <= 1e-12 * np.abs(sk) + 1e-13 * int(c1 - c0))
    b.close()

@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("shape", [(1, 128), (2, 128, 2, 2, 16, 1024)])
def test_rest_state_is_a_fixed_point(prec, shape):
    """rho = rho0, u = 0: every shifted population is exactly 0, and the collision and the
    streaming keep it exactly 0 (a fixed point of the scheme, in every precision and
    kernel path, with the bulk correction on)."""
    lbm = lbm_mod()
    dims = (16, 6, 4)
    lat = lbm.Lattice(lbm.D3Q27, dims, 0.56, lbm.ENTROPIC, 1, prec)
    lat.set_launch_shape(*shape)
    n = int(np.prod(dims))
    lat.init_fields(np.ones(n), np.zeros((3, n)))
    lat.step(5)
    raw = lat.get_populations("storage")
    assert np.all(raw == 0)
    lat.close()


@pytest.mark.parametrize("eq,u0", [(core.EQ_ENTROPIC, (0.9, -0.6, 0.3)), (core.EQ_POLY2, (0.3, -0.2, 0.1)),
                                   (core.EQ_PRODUCT, (0.4, 0.3, -0.2))])
def test_uniform_flow_is_a_fixed_point(eq, u0):
    """A uniform flow f = f^eq(rho, U) streams onto itself and collides to itself, so it
    is invariant; at |U| up to 0.9 per axis for the entropic equilibrium (close to its
    limit |u| < 1) the GPU FP64 state stays at the oracle's over 7 steps.  Tolerance:
    1e-12 relative, plus an absolute 1e-14 w_i, because the GPU stores f - w rho0 and at
    this speed some f_i are ~1e-4 of w_i, so the rounding of the stored value (2^-53 of
    about w_i per step) is no longer small against f_i itself."""
    lbm = lbm_mod()
    dims = (8, 5, 3)
    n = int(np.prod(dims))
    rho = np.full(n, 1.05)
    u = np.tile(np.array(u0)[:, None], (1, n))
    lat = lbm.Lattice(lbm.D3Q27, dims, 0.53, eq, 1, lbm.F64)
    lat.init_fields(rho, u)
    lat.step(7)
    got = lat.get_populations()
    f0 = core.init(3, dims, eq, rho, u)
    ref = core.step(3, dims, eq, 1, 0.53, 7, f0)
    _, w = core.lattice(3)
    tol = 1e-12 * np.abs(ref) + 1e-14 * w[:, None]
    assert np.all(np.abs(got - ref) <= tol)
    assert np.all(np.abs(got - f0) <= tol)
    lat.close()
