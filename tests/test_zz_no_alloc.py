"""lbm_diagnostics_noalloc: diagnostics of populations the caller already owns, with no
device allocation by the library.  It serves callers that cannot call cudaMalloc
(inside another framework's memory pool, with all device memory reserved up front, or
inside a stream capture).  Its result must equal lbm_diagnostics of the same state, on
two calls in a row (the calls share one static scratch array).

This file sorts last so that a run stopping at the first failure has already run every
other test; it also passes alone in a fresh process.

Tolerance: lbm_diagnostics forms each cell's moments in the collision precision of the
state (FP64 for FP64 storage, FP32 otherwise) before the FP64 sums; this entry point reads
FP64 populations.  So the two agree to 1e-12 (relative) for an FP64 state and to the FP32
rounding of the per-cell moments, 1e-6, for an FP32 state.
"""
import ctypes

import numpy as np
import pytest

from paper_2303_08163_gb300 import inputs

pytestmark = pytest.mark.gpu


def _state(lbm, lattice, dims, prec, steps):
    D = 2 if lattice == lbm.D2Q9 else 3
    rho, u = inputs.random_state(D, dims, seed=17 + D, u_max=0.1)
    lat = lbm.Lattice(lattice, dims, 0.62, lbm.ENTROPIC, 1, prec)
    lat.init_fields(rho, u)
    lat.step(steps)
    return lat


@pytest.mark.parametrize("lattice,dims,prec", [(1, (24, 20, 18), 0), (0, (70, 33, 1), 1)])
def test_noalloc_diagnostics_match_existing_entry_point(lattice, dims, prec):
    import torch
    from paper_2303_08163_gb300 import build, lbm
    build.build()
    lbm.load()
    lat = _state(lbm, lattice, dims, prec, steps=7)
    ref = lat.diagnostics()
    Q, ncell = lat.Q, lat.ncell
    f = torch.empty((Q, ncell), dtype=torch.float64, device="cuda")
    rc = lbm.load().lbm_get_populations(lat._h, ctypes.c_void_p(f.data_ptr()), lbm.DT_F64, 1)
    assert rc == 0
    torch.cuda.synchronize()
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    tol = 1e-12 if prec == 0 else 1e-6
    for call in range(2):
        out.fill_(np.nan)
        lbm.diagnostics_noalloc(lattice, dims, f, out, blocks=64 + 37 * call)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert abs(o[0] - ref["mass"]) <= tol * ref["mass"]
        np.testing.assert_allclose(o[1:4], ref["momentum"], rtol=0, atol=tol * ref["mass"])
        assert abs(o[4] - ref["kinetic"]) <= tol * ref["kinetic"]
        assert abs(o[5] - ref["max_u"]) <= tol * ref["max_u"]
        assert o[6] == 0 and o[7] == 0
    # the limit of the static scratch is enforced
    with pytest.raises(lbm.LBMError) as e:
        lbm.diagnostics_noalloc(lattice, dims, f, out, blocks=1025)
    assert e.value.status == lbm.EINVAL
    # sizes beyond lbm_create's limits (a dimension above 2^30, or a cell count that
    # overflows 64 bits) are rejected before anything is launched
    for bad in ((1 << 31, 4, 4), (1 << 30, 1 << 30, 1 << 30)):
        with pytest.raises(lbm.LBMError) as e:
            lbm.diagnostics_noalloc(lbm.D3Q27, bad, f, out, blocks=64)
        assert e.value.status == lbm.EINVAL
    lat.close()
