"""The full-size sampled-cell checks of tests/test_gpu_fullsize.py can fail.

A data-movement mistake is planted in the oracle's result, on the CPU: every direction's
population at cell x is taken from the neighbour x + e_x instead (a wrong-neighbour read
or write, the typical indexing error of a streaming kernel).  On a field that varies from
cell to cell (uniform random rho and u per cell, as in the non-smooth full-size check)
the planted error exceeds the rounding bound of the binary16 and FP32 checks for nearly
every population of every direction.  On the smooth 512^3 Taylor-Green vortex it stays
inside the binary16 bound everywhere: there a wrong neighbour changes a population by
only about w_i |grad u|, which is why the binary16 layouts are also compared bit for bit
with the one-cell kernel at full size.
"""
import math

import numpy as np

from fullsize_bounds import sampled_tolerance
from oracle import core
from paper_2303_08163_gb300 import inputs

N, U0 = 512, 0.1
TAU = 0.5 + 3 * U0 * (N / (2 * math.pi)) / 1600.0  # the Re = 1600 vortex at 512^3


def test_wrong_neighbour_is_caught_on_a_nonsmooth_field():
    dims = (16, 16, 16)
    rho, u = inputs.random_state(3, dims, seed=5, rho_range=(0.9, 1.1), u_max=0.1)
    f0 = core.init(3, dims, core.EQ_ENTROPIC, rho, u)
    _, w = core.lattice(3)
    for nsteps in (1, 2):
        f = core.step(3, dims, core.EQ_ENTROPIC, 0, TAU, nsteps, f0)
        planted = np.roll(f.reshape(27, 16, 16, 16), -1, axis=3).reshape(27, -1)
        for prec in (2, 1):
            tol = sampled_tolerance(f.T, w, 3, TAU, prec, nsteps, 0.12, rho_min=0.85).T
            caught = np.abs(planted - f) > tol
            per_dir = caught.mean(axis=1)
            print(f"steps={nsteps} prec={prec}: caught {caught.mean():.3f}, worst direction {per_dir.min():.3f}")
            assert per_dir.min() >= 0.8


def test_wrong_neighbour_hides_in_the_binary16_bound_on_the_smooth_vortex():
    rho_fn, u_fn = inputs.taylor_green_3d_fields(N, u0=U0)
    rng = np.random.default_rng(3)
    cells = np.array([[int(rng.integers(0, N)) for _ in range(3)] for _ in range(8)])
    nb = cells.copy()
    nb[:, 0] = (nb[:, 0] + 1) % N
    _, w = core.lattice(3)
    ref = core.local_populations(3, (N, N, N), core.EQ_ENTROPIC, 0, TAU, 1, rho_fn, u_fn, cells)
    wrong = core.local_populations(3, (N, N, N), core.EQ_ENTROPIC, 0, TAU, 1, rho_fn, u_fn, nb)
    ratio = np.abs(wrong - ref) / sampled_tolerance(ref, w, 3, TAU, 2, 1, U0)
    print(f"smooth vortex, binary16: largest planted error / bound = {ratio.max():.3f}")
    assert ratio.max() < 1.0
