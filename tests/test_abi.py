"""The C-ABI library builds, loads and exports every symbol include/lbm.h declares; the
argument checks that run before any CUDA call reject bad input (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2303_08163_gb300 import build, lbm
    build.build()
    return lbm.load()


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ["lbm_create", "lbm_init_fields", "lbm_step", "lbm_moments", "lbm_diagnostics",
                     "lbm_get_populations", "lbm_set_populations", "lbm_batch_create",
                     "lbm_batch_init_fields", "lbm_batch_set_probe", "lbm_batch_step",
                     "lbm_batch_probe_series", "lbm_batch_status", "lbm_batch_moments",
                     "lbm_sync", "lbm_last_error", "lbm_destroy", "lbm_batch_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2303_08163_gb300 import lbm
    names = header_functions()
    assert names, "no declarations parsed"
    for name in names:
        assert hasattr(lib, name), f"{name} declared in lbm.h but not exported"
        assert name in lbm.SIGNATURES, f"{name} has no binding signature"


def test_version_and_error_string(lib):
    assert lib.lbm_version() >= 10000
    assert isinstance(lib.lbm_last_error(), bytes)


def _create(lib, lattice=0, dims=(8, 8, 1), tau=0.8, eq=0, bulk=0, prec=0, rho0=1.0):
    h = ctypes.c_void_p()
    d = (ctypes.c_int64 * 3)(*dims)
    return lib.lbm_create(ctypes.byref(h), lattice, d, tau, eq, bulk, prec, rho0, None)


@pytest.mark.parametrize("kw,why", [
    (dict(tau=0.5), "tau"), (dict(tau=0.3), "tau"), (dict(tau=float("nan")), "tau"),
    (dict(lattice=2), "lattice"), (dict(eq=3), "eq_kind"), (dict(bulk=2), "bulk"),
    (dict(prec=3), "precision"), (dict(dims=(0, 8, 1)), "dims"), (dict(dims=(8, 8, 2)), "D2Q9"),
    (dict(rho0=0.0), "rho0"),
])
def test_create_rejects_bad_arguments(lib, kw, why):
    from paper_2303_08163_gb300 import lbm
    assert _create(lib, **kw) == lbm.EINVAL
    assert lib.lbm_last_error()


def test_batch_create_rejects_bad_arguments(lib):
    from paper_2303_08163_gb300 import lbm
    import numpy as np
    h = ctypes.c_void_p()
    dims = np.array([[8, 8, 1], [9, 7, 1]], dtype=np.int32)
    tau = np.array([0.8, 0.5])
    rc = lib.lbm_batch_create(ctypes.byref(h), 0, 2, dims.ctypes.data_as(lbm._pi32),
                              tau.ctypes.data_as(lbm._pdbl), 0, 0, 0, 1.0, None)
    assert rc == lbm.EINVAL
    tau = np.array([0.8, 0.9])
    rc = lib.lbm_batch_create(ctypes.byref(h), 0, 2, dims.ctypes.data_as(lbm._pi32),
                              tau.ctypes.data_as(lbm._pdbl), 0, 0, 1, 1.0, None)
    assert rc == lbm.EINVAL  # the batched path stores FP64 only


def test_null_object_calls_fail_cleanly(lib):
    from paper_2303_08163_gb300 import lbm
    assert lib.lbm_step(None, 1) == lbm.EINVAL
    assert lib.lbm_sync(None) == lbm.EINVAL
    lib.lbm_destroy(None)
    lib.lbm_batch_destroy(None)


def test_status_codes_match_the_header():
    """Every enumerator of enum lbm_status in lbm.h has the same value in the binding."""
    import re
    from paper_2303_08163_gb300 import lbm
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    body = text[text.index("enum lbm_status"):]
    body = body[:body.index("};")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    codes = {m.group(1): int(m.group(2)) for m in re.finditer(r"(LBM_[A-Z]+)\s*=\s*(-?\d+)", body)}
    assert codes["LBM_ECHECK"] == lbm.ECHECK == -7
    for name, value in codes.items():
        assert lbm.STATUS_NAMES[value] == name
