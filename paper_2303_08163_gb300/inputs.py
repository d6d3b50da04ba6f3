"""Seeded synthetic inputs: initial density and velocity fields, batch instance tables.

This module is shared by the CUDA path's tests and benchmark and by the oracle's tests.
It holds none of the lattice-BGK arithmetic: only the flow fields that the runs start
from (Taylor-Green vortices, a double shear layer, a random solenoidal field with a
prescribed spectrum, and small-amplitude plane waves), all from fixed seeds
(NumPy PCG64).

Array conventions match the library: dims = (Nx, Ny, Nz), cell index x + Nx (y + Ny z);
rho has shape (ncell,), u has shape (D, ncell).
"""
import math

import numpy as np


def _grid(dims, scale):
    nx, ny, nz = dims
    x = np.arange(nx, dtype=np.float64) * scale[0]
    y = np.arange(ny, dtype=np.float64) * scale[1]
    z = np.arange(nz, dtype=np.float64) * scale[2]
    return x, y, z


def taylor_green_2d(n, u0=0.05, rho0=1.0):
    """2-D Taylor-Green vortex on an n x n periodic lattice, x = 2 pi i / n:
    u = (u0 sin x cos y, -u0 cos x sin y), rho = rho0."""
    x, y, _ = _grid((n, n, 1), (2 * math.pi / n,) * 3)
    X = x[None, :]
    Y = y[:, None]
    ux = u0 * np.sin(X) * np.cos(Y)
    uy = -u0 * np.cos(X) * np.sin(Y)
    rho = np.full(n * n, rho0)
    return rho, np.stack([ux.reshape(-1), uy.reshape(-1)])


def taylor_green_3d_fields(n, u0=0.1, rho0=1.0, cs2=1.0 / 3.0):
    """Field functions of the 3-D Taylor-Green vortex on an n^3 lattice, x = 2 pi i / n:
    u = u0 (sin x cos y cos z, -cos x sin y cos z, 0),
    rho = rho0 + (rho0 u0^2 / (16 cs2)) (cos 2x + cos 2y) (cos 2z + 2).

    Returns (rho_fn, u_fn) taking integer index arrays (ix, iy, iz), so a caller can
    evaluate any subset of cells without building the full grid.
    """
    h = 2 * math.pi / n

    def rho_fn(ix, iy, iz):
        X, Y, Z = ix * h, iy * h, iz * h
        return rho0 + rho0 * u0 * u0 / (16 * cs2) * (np.cos(2 * X) + np.cos(2 * Y)) * (
            np.cos(2 * Z) + 2)

    def u_fn(ix, iy, iz):
        X, Y, Z = ix * h, iy * h, iz * h
        ux = u0 * np.sin(X) * np.cos(Y) * np.cos(Z)
        uy = -u0 * np.cos(X) * np.sin(Y) * np.cos(Z)
        return np.stack([ux, uy, np.zeros_like(ux)])

    return rho_fn, u_fn


def taylor_green_3d_torch(n, u0=0.1, rho0=1.0, device="cuda", slab=64):
    """The 3-D Taylor-Green fields of `taylor_green_3d_fields` as float32 device tensors
    (rho flat, u of shape (3, n^3), x fastest), built one slab of z-planes at a time in
    float64 so that lattices of billions of cells need no host copy and no full-size
    float64 temporaries."""
    import torch
    h = 2 * math.pi / n
    t = torch.arange(n, device=device, dtype=torch.float64) * h
    s, c, c2 = torch.sin(t), torch.cos(t), torch.cos(2 * t)
    rho = torch.empty(n ** 3, device=device, dtype=torch.float32)
    u = torch.zeros(3, n ** 3, device=device, dtype=torch.float32)
    plane = n * n
    for z0 in range(0, n, slab):
        z1 = min(n, z0 + slab)
        cz, c2z = c[z0:z1, None, None], c2[z0:z1, None, None]
        sl = slice(z0 * plane, z1 * plane)
        u[0, sl] = (u0 * cz * c[None, :, None] * s[None, None, :]).reshape(-1)
        u[1, sl] = (-u0 * cz * s[None, :, None] * c[None, None, :]).reshape(-1)
        rho[sl] = (rho0 + rho0 * u0 * u0 * 3.0 / 16.0 * (c2[None, None, :] + c2[None, :, None])
                   * (c2z + 2.0)).reshape(-1)
    return rho, u


def taylor_green_3d(n, u0=0.1, rho0=1.0, dtype=np.float64):
    """Full 3-D Taylor-Green fields as flat arrays (separable evaluation)."""
    h = 2 * math.pi / n
    t = np.arange(n) * h
    s, c = np.sin(t), np.cos(t)
    c2 = np.cos(2 * t)
    ux = (u0 * c[:, None, None] * c[None, :, None] * s[None, None, :]).astype(dtype)
    uy = (-u0 * c[:, None, None] * s[None, :, None] * c[None, None, :]).astype(dtype)
    uz = np.zeros_like(ux)
    rho = (rho0 + rho0 * u0 * u0 * 3.0 / 16.0 * (c2[None, :, None] + c2[None, None, :])
           * (c2[:, None, None] + 2.0)).astype(dtype)
    return rho.reshape(-1), np.stack([ux.reshape(-1), uy.reshape(-1), uz.reshape(-1)])


def double_shear_layer_fields(n, u0=0.1, kappa=80.0, delta=0.05):
    """Field functions of the periodic double shear layer on an n x n lattice,
    x = i / n, y = j / n: u_x = u0 tanh(kappa (y - 1/4)) for y <= 1/2 and
    u0 tanh(kappa (3/4 - y)) otherwise; u_y = delta u0 sin(2 pi (x + 1/4)); rho = 1."""

    def rho_fn(ix, iy, iz):
        return np.ones(np.broadcast(ix, iy, iz).shape)

    def u_fn(ix, iy, iz):
        X = ix / n
        Y = iy / n
        ux = np.where(Y <= 0.5, u0 * np.tanh(kappa * (Y - 0.25)), u0 * np.tanh(kappa * (0.75 - Y)))
        uy = delta * u0 * np.sin(2 * math.pi * (X + 0.25))
        ux, uy = np.broadcast_arrays(ux, uy)
        return np.stack([ux, uy])

    return rho_fn, u_fn


def double_shear_layer(n, u0=0.1, kappa=80.0, delta=0.05, dtype=np.float64):
    """Full double-shear-layer fields as flat arrays."""
    y = np.arange(n) / n
    x = np.arange(n) / n
    ux_y = np.where(y <= 0.5, u0 * np.tanh(kappa * (y - 0.25)), u0 * np.tanh(kappa * (0.75 - y)))
    uy_x = delta * u0 * np.sin(2 * math.pi * (x + 0.25))
    ux = np.broadcast_to(ux_y[:, None], (n, n)).astype(dtype)
    uy = np.broadcast_to(uy_x[None, :], (n, n)).astype(dtype)
    rho = np.ones(n * n, dtype=dtype)
    return rho, np.stack([ux.reshape(-1), uy.reshape(-1)])


def random_solenoidal(dims, u_rms=0.05, k_peak=8.0, seed=2303):
    """Random-phase solenoidal velocity on a periodic box of dims = (Nx, Ny, Nz) cells.

    The box is [0, 2 pi Nx / Ny) x [0, 2 pi)^2 (so unit wavenumber spacing along y and z);
    the energy spectrum is E(k) ~ k^4 exp(-2 (k / k_peak)^2).  Each Fourier mode gets a
    complex Gaussian amplitude scaled by sqrt(E(k) / (4 pi k^2)), is projected
    perpendicular to k, and the field is scaled to the given rms of one component.
    Returns rho = 1 and u with shape (3, ncell), float64.
    """
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    kx = np.fft.fftfreq(nx, d=1.0 / nx) * (ny / nx)
    ky = np.fft.fftfreq(ny, d=1.0 / ny)
    kz = np.fft.rfftfreq(nz, d=1.0 / nz)
    KX, KY, KZ = np.meshgrid(kx, ky, kz, indexing="ij")
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    k = np.sqrt(k2)
    with np.errstate(divide="ignore", invalid="ignore"):
        amp = np.sqrt(k ** 4 * np.exp(-2.0 * (k / k_peak) ** 2) / (4 * math.pi * np.where(k2 > 0, k2, 1.0)))
    amp[k2 == 0] = 0.0
    comps = []
    for _ in range(3):
        re = rng.standard_normal(KX.shape)
        im = rng.standard_normal(KX.shape)
        comps.append(amp * (re + 1j * im))
    kdotv = (KX * comps[0] + KY * comps[1] + KZ * comps[2]) / np.where(k2 > 0, k2, 1.0)
    comps = [comps[0] - KX * kdotv, comps[1] - KY * kdotv, comps[2] - KZ * kdotv]
    # arrays are indexed [x, y, z]; the library wants x fastest (z, y, x order)
    u = [np.fft.irfftn(cv, s=(nx, ny, nz), axes=(0, 1, 2)).transpose(2, 1, 0).reshape(-1) for cv in comps]
    u = np.stack(u)
    scale = u_rms / np.sqrt(np.mean(u * u))
    u *= scale
    rho = np.ones(nx * ny * nz)
    return rho, u


def random_solenoidal_torch(dims, u_rms=0.05, k_peak=8.0, seed=2303, device="cuda"):
    """The field of random_solenoidal, generated with torch (on a GPU for the full-size
    1024 x 512 x 512 box) from a seeded torch generator.  Returns float32 tensors rho
    (ncell,) and u (3, ncell) on `device`, x fastest."""
    import torch
    nx, ny, nz = dims
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    f64 = torch.float64
    kx = torch.fft.fftfreq(nx, d=1.0 / nx, device=device, dtype=f64) * (ny / nx)
    ky = torch.fft.fftfreq(ny, d=1.0 / ny, device=device, dtype=f64)
    kz = torch.fft.rfftfreq(nz, d=1.0 / nz, device=device, dtype=f64)
    KX, KY, KZ = torch.meshgrid(kx, ky, kz, indexing="ij")
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    safe = torch.where(k2 > 0, k2, torch.ones_like(k2))
    amp = torch.sqrt(k2 * k2 * torch.exp(-2.0 * k2 / (k_peak * k_peak)) / (4 * math.pi * safe))
    amp[k2 == 0] = 0.0
    comps = []
    for _ in range(3):
        re = torch.randn(KX.shape, generator=gen, device=device, dtype=f64)
        im = torch.randn(KX.shape, generator=gen, device=device, dtype=f64)
        comps.append(amp * torch.complex(re, im))
    del re, im, amp
    kdotv = (KX * comps[0] + KY * comps[1] + KZ * comps[2]) / safe
    comps = [comps[0] - KX * kdotv, comps[1] - KY * kdotv, comps[2] - KZ * kdotv]
    del kdotv, KX, KY, KZ, k2, safe
    u = torch.empty((3, nx * ny * nz), device=device, dtype=torch.float32)
    sq = 0.0
    for a in range(3):
        ua = torch.fft.irfftn(comps[a], s=(nx, ny, nz))  # indexed [x, y, z]
        comps[a] = None
        ua = ua.permute(2, 1, 0).contiguous().reshape(-1)  # x fastest
        sq += float(torch.sum(ua * ua))
        u[a] = ua.float()
        del ua
    scale = u_rms / math.sqrt(sq / (3 * nx * ny * nz))
    u *= scale
    rho = torch.ones(nx * ny * nz, device=device, dtype=torch.float32)
    return rho, u


def linear_mode_batch(count=4096, seed=2303, nmin=16, nmax=256, amp=1e-4, u0max=0.3,
                      tau_minus_half=(5e-4, 1.0), kmax=8):
    """Instance table of the batched linear-mode sweep.

    Per instance: N_x, N_y independently log-uniform in [nmin, nmax]; integer wavenumber
    n uniform in 1 .. min(kmax, N_x // 4) along x; background U0 uniform in [0, u0max]
    along x; tau - 1/2 log-uniform in the given range; kind 0 = shear wave
    (u_y = amp sin(k x)), kind 1 = acoustic wave (rho = 1 + amp sin(k x)).
    """
    rng = np.random.default_rng(seed)
    lo, hi = math.log(nmin), math.log(nmax + 1)
    nx = np.floor(np.exp(rng.uniform(lo, hi, count))).astype(np.int32)
    ny = np.floor(np.exp(rng.uniform(lo, hi, count))).astype(np.int32)
    nx = np.clip(nx, nmin, nmax)
    ny = np.clip(ny, nmin, nmax)
    nmode = np.array([rng.integers(1, min(kmax, int(a) // 4) + 1) for a in nx], dtype=np.int32)
    U0 = rng.uniform(0.0, u0max, count)
    tl, th = math.log(tau_minus_half[0]), math.log(tau_minus_half[1])
    tau = 0.5 + np.exp(rng.uniform(tl, th, count))
    kind = rng.integers(0, 2, count).astype(np.int32)
    return {"nx": nx, "ny": ny, "nmode": nmode, "U0": U0, "tau": tau, "kind": kind,
            "amp": amp}


def linear_mode_fields(table, k):
    """rho (ncell,), u (2, ncell) of instance k of a linear_mode_batch table."""
    nx, ny = int(table["nx"][k]), int(table["ny"][k])
    n = int(table["nmode"][k])
    a = table["amp"]
    x = np.arange(nx, dtype=np.float64)
    wave = np.sin(2 * math.pi * n * x / nx)
    rho = np.ones((ny, nx))
    ux = np.full((ny, nx), float(table["U0"][k]))
    uy = np.zeros((ny, nx))
    if int(table["kind"][k]) == 0:
        uy += a * wave[None, :]
    else:
        rho += a * wave[None, :]
    return rho.reshape(-1), np.stack([ux.reshape(-1), uy.reshape(-1)])


def acoustic_wave_1d(nx, U0, drho=1e-3, rho0=1.0, ny=1):
    """rho = rho0 + drho sin(2 pi x / N_x), u = (U0, 0) on an N_x x ny lattice."""
    x = np.arange(nx, dtype=np.float64)
    rho = np.broadcast_to(rho0 + drho * np.sin(2 * math.pi * x / nx), (ny, nx)).reshape(-1)
    ux = np.full(nx * ny, float(U0))
    return rho.copy(), np.stack([ux, np.zeros(nx * ny)])


def random_state_torch(D, dims, seed, rho_range=(0.8, 1.2), u_max=0.2, device="cuda"):
    """Uniform random rho and u drawn independently for every cell, as float32 tensors on
    `device` (rho (ncell,), u (D, ncell), x fastest), from a seeded torch generator: the
    non-smooth field of the full-size parity checks, built without a host copy."""
    import torch
    n = int(np.prod(dims))
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    rho = torch.rand(n, generator=gen, device=device, dtype=torch.float32)
    rho.mul_(rho_range[1] - rho_range[0]).add_(rho_range[0])
    u = torch.rand(D, n, generator=gen, device=device, dtype=torch.float32)
    u.mul_(2 * u_max).sub_(u_max)
    return rho, u


def random_state(D, dims, seed, rho_range=(0.8, 1.2), u_max=0.2):
    """Smooth-free random fields (uniform per cell) for parity tests."""
    n = int(np.prod(dims))
    rng = np.random.default_rng(seed)
    rho = rng.uniform(rho_range[0], rho_range[1], n)
    u = rng.uniform(-u_max, u_max, (D, n))
    return rho, u
