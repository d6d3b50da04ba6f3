"""Thin ctypes binding of the C ABI in include/lbm.h (argument marshalling only).

Every step of the method runs in the CUDA kernels of liblbm.so; this module converts
NumPy arrays / torch tensors to pointers and raises LBMError on a non-zero status.  It
has no fallback: if the shared library is missing or cannot be loaded, every call
raises.

Names follow the C ABI: ``Lattice`` wraps ``lbm_ctx`` (lbm_create, lbm_init_fields,
lbm_step, lbm_moments, ...), ``Batch`` wraps ``lbm_batch`` (lbm_batch_*).
"""
import ctypes
import os

import numpy as np

from . import build as _build

D2Q9, D3Q27 = 0, 1
ENTROPIC, POLY2, PRODUCT = 0, 1, 2
F64, F32, F16S = 0, 1, 2
DT_F64, DT_F32, DT_STORAGE = 0, 1, 2
STORAGE_NUMPY = {0: np.float64, 1: np.float32, 2: np.float16}
OPT_DIAG_EVERY, OPT_KERNEL, OPT_USE_GRAPH, OPT_TUNE = 0, 1, 2, 3
KERNEL_AUTO, KERNEL_GENERIC, KERNEL_TMA = 0, 1, 2

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, ESTATE, ECHECK = 0, -1, -2, -3, -4, -5, -6, -7
STATUS_NAMES = {0: "LBM_OK", -1: "LBM_EINVAL", -2: "LBM_ENOMEM", -3: "LBM_ECUDA",
                -4: "LBM_ENONFINITE", -5: "LBM_ETIMEOUT", -6: "LBM_ESTATE", -7: "LBM_ECHECK"}

# Every symbol the header declares, with (restype, argtypes).
_vp, _i, _i64, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
_p64 = ctypes.POINTER(ctypes.c_int64)
_pdbl = ctypes.POINTER(ctypes.c_double)
_pi32 = ctypes.POINTER(ctypes.c_int32)


class lbm_diag(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("momentum", ctypes.c_double * 3),
                ("kinetic", ctypes.c_double), ("max_u", ctypes.c_double),
                ("step", ctypes.c_int64), ("nonfinite", ctypes.c_int64)]


SIGNATURES = {
    "lbm_create": (_i, [ctypes.POINTER(_vp), _i, _p64, _d, _i, _i, _i, _d, _vp]),
    "lbm_set_option": (_i, [_vp, _i, _i64]),
    "lbm_init_fields": (_i, [_vp, _vp, _vp, _i, _i]),
    "lbm_step": (_i, [_vp, _i64]),
    "lbm_moments": (_i, [_vp, _vp, _vp, _i, _i]),
    "lbm_diagnostics": (_i, [_vp, ctypes.POINTER(lbm_diag)]),
    "lbm_diag_history": (_i, [_vp, ctypes.POINTER(lbm_diag), _i64, _p64]),
    "lbm_get_populations": (_i, [_vp, _vp, _i, _i]),
    "lbm_set_populations": (_i, [_vp, _vp, _i, _i]),
    "lbm_set_step_count": (_i, [_vp, _i64]),
    "lbm_sample_populations": (_i, [_vp, _p64, _i64, _pdbl]),
    "lbm_step_count": (_i, [_vp, _p64]),
    "lbm_launch_info": (_i, [_vp, _p64]),
    "lbm_set_launch_shape": (_i, [_vp, _p64]),
    "lbm_sync": (_i, [_vp]),
    "lbm_destroy": (None, [_vp]),
    "lbm_batch_create": (_i, [ctypes.POINTER(_vp), _i, _i64, _pi32, _pdbl, _i, _i, _i, _d, _vp]),
    "lbm_batch_init_fields": (_i, [_vp, _vp, _vp, _i, _i]),
    "lbm_batch_set_probe": (_i, [_vp, _pi32, _i64]),
    "lbm_batch_step": (_i, [_vp, _i64]),
    "lbm_batch_probe_series": (_i, [_vp, _pdbl, _i64, _p64]),
    "lbm_batch_status": (_i, [_vp, _pi32]),
    "lbm_batch_moments": (_i, [_vp, _vp, _vp, _i, _i]),
    "lbm_batch_get_populations": (_i, [_vp, _vp, _i, _i]),
    "lbm_batch_info": (_i, [_vp, _p64, _p64]),
    "lbm_batch_launch_info": (_i, [_vp, _p64]),
    "lbm_batch_set_launch_shape": (_i, [_vp, _i, _i64]),
    "lbm_batch_autotune": (_i, [_vp, _i64]),
    "lbm_batch_sync": (_i, [_vp]),
    "lbm_batch_destroy": (None, [_vp]),
    "lbm_last_error": (ctypes.c_char_p, []),
    "lbm_version": (_i, []),
    "lbm_selftest_bounded_wait": (_i, [_vp, _i64, _pi32]),
    "lbm_diagnostics_noalloc": (_i, [_i, _p64, _vp, _i64, _vp, _vp]),
    "lbm_vn_eigenvalues": (_i, [_i, _i, _i64, _pdbl, _pdbl, _vp]),
    "lbm_vn_stability_limit": (_i, [_i, _i64, _pdbl, _pdbl, _i, _d, _i, _d, _pdbl, _vp]),
}

_lib = None


class LBMError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def library_path():
    """The in-tree liblbm.so; LBM_LIBRARY names another in-tree build (the checked one)."""
    return os.environ.get("LBM_LIBRARY") or _build.LIB


def load():
    """Load liblbm.so (built in-tree by build.build()); raise if it is missing."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"the CUDA library {path} is not built; run "
                               "paper_2303_08163_gb300.build.build() (or __graft_entry__.build())")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(rc):
    if rc != 0:
        raise LBMError(rc, load().lbm_last_error().decode())
    return rc


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _buffer(arr, dtype):
    """(pointer, on_device, keepalive) of a NumPy array or torch tensor of `dtype`
    (np.float64 / np.float32), C-contiguous."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(arr, torch.Tensor):
        want = torch.float64 if dtype == np.float64 else torch.float32
        if arr.dtype != want or not arr.is_contiguous():
            arr = arr.to(want).contiguous()
        return ctypes.c_void_p(arr.data_ptr()), int(arr.is_cuda), arr
    a = np.ascontiguousarray(arr, dtype=dtype)
    return ctypes.c_void_p(a.ctypes.data), 0, a


def _dt(dtype):
    return DT_F64 if np.dtype(dtype) == np.float64 else DT_F32


class Lattice:
    """One periodic D2Q9 or D3Q27 lattice (lbm_create ... lbm_destroy)."""

    def __init__(self, lattice, dims, tau, eq_kind=ENTROPIC, bulk_corr=0, precision=F64,
                 rho0=1.0, stream=None):
        lib = load()
        d = (list(dims) + [1, 1, 1])[:3]
        self.dims = tuple(int(v) for v in d)
        self.D = 2 if lattice == D2Q9 else 3
        self.Q = 3 ** self.D
        self.ncell = int(np.prod(self.dims))
        self.lattice, self.tau, self.eq_kind = lattice, tau, eq_kind
        self.bulk_corr, self.precision, self.rho0 = bulk_corr, precision, rho0
        self._h = ctypes.c_void_p()
        self._stream = _stream_handle(stream)
        dims_c = (ctypes.c_int64 * 3)(*self.dims)
        _check(lib.lbm_create(ctypes.byref(self._h), int(lattice), dims_c, float(tau), int(eq_kind),
                              int(bulk_corr), int(precision), float(rho0), self._stream))

    def close(self):
        if self._h:
            load().lbm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_option(self, option, value):
        _check(load().lbm_set_option(self._h, int(option), int(value)))

    def init_fields(self, rho, u, dtype=np.float64):
        pr, dev_r, kr = _buffer(rho, dtype)
        pu, dev_u, ku = _buffer(u, dtype)
        if dev_r != dev_u:
            raise ValueError("rho and u must both be host or both be device buffers")
        _check(load().lbm_init_fields(self._h, pr, pu, _dt(dtype), dev_r))

    def step(self, n=1):
        _check(load().lbm_step(self._h, int(n)))

    def moments(self, dtype=np.float64, out=None):
        """rho (ncell,) and u (D, ncell) as NumPy arrays, or into torch tensors `out`."""
        if out is not None:
            rho, u = out
            _check(load().lbm_moments(self._h, ctypes.c_void_p(rho.data_ptr()),
                                      ctypes.c_void_p(u.data_ptr()), _dt(dtype), int(rho.is_cuda)))
            return rho, u
        rho = np.empty(self.ncell, dtype=dtype)
        u = np.empty((self.D, self.ncell), dtype=dtype)
        _check(load().lbm_moments(self._h, ctypes.c_void_p(rho.ctypes.data),
                                  ctypes.c_void_p(u.ctypes.data), _dt(dtype), 0))
        return rho, u

    def diagnostics(self):
        d = lbm_diag()
        _check(load().lbm_diagnostics(self._h, ctypes.byref(d)))
        return _diag_dict(d)

    def diag_history(self, max_records=65536):
        cnt = ctypes.c_int64()
        arr = (lbm_diag * max(int(max_records), 1))()
        _check(load().lbm_diag_history(self._h, arr, int(max_records), ctypes.byref(cnt)))
        return [_diag_dict(arr[i]) for i in range(min(cnt.value, max_records))]

    def get_populations(self, dtype=np.float64, out=None):
        """Canonical populations (Q, ncell); dtype="storage" returns the stored shifted
        values f - w rho0 in the storage type, bit for bit.  With `out` (a contiguous torch
        tensor of Q * ncell elements on the lattice's device, of the storage type's size for
        "storage"), the populations are written there without a host copy."""
        if out is not None:
            dt = DT_STORAGE if isinstance(dtype, str) and dtype == "storage" else _dt(dtype)
            want = {DT_STORAGE: np.dtype(STORAGE_NUMPY[self.precision]).itemsize, DT_F64: 8, DT_F32: 4}[dt]
            if (not out.is_cuda or not out.is_contiguous() or out.element_size() != want
                    or out.numel() != self.Q * self.ncell):
                raise ValueError("out must be a contiguous device tensor of Q * ncell elements of the requested type")
            _check(load().lbm_get_populations(self._h, ctypes.c_void_p(out.data_ptr()), dt, 1))
            return out
        if isinstance(dtype, str) and dtype == "storage":
            f = np.empty((self.Q, self.ncell), dtype=STORAGE_NUMPY[self.precision])
            _check(load().lbm_get_populations(self._h, ctypes.c_void_p(f.ctypes.data), DT_STORAGE, 0))
            return f
        f = np.empty((self.Q, self.ncell), dtype=dtype)
        _check(load().lbm_get_populations(self._h, ctypes.c_void_p(f.ctypes.data), _dt(dtype), 0))
        return f

    def set_populations(self, f, dtype=np.float64):
        if isinstance(dtype, str) and dtype == "storage":
            a = np.ascontiguousarray(f, dtype=STORAGE_NUMPY[self.precision])
            _check(load().lbm_set_populations(self._h, ctypes.c_void_p(a.ctypes.data), DT_STORAGE, 0))
            return
        p, dev, keep = _buffer(f, dtype)
        _check(load().lbm_set_populations(self._h, p, _dt(dtype), dev))

    def set_step_count(self, step):
        _check(load().lbm_set_step_count(self._h, int(step)))

    def sample_populations(self, cells):
        c = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.empty((len(c), self.Q))
        _check(load().lbm_sample_populations(self._h, c.ctypes.data_as(_p64), len(c),
                                             out.ctypes.data_as(_pdbl)))
        return out

    @property
    def step_count(self):
        v = ctypes.c_int64()
        _check(load().lbm_step_count(self._h, ctypes.byref(v)))
        return v.value

    def launch_info(self):
        out = (ctypes.c_int64 * 8)()
        _check(load().lbm_launch_info(self._h, out))
        keys = ["kernel", "threads", "blocks", "stages", "rows", "seg", "smem_bytes", "storage_bytes"]
        return dict(zip(keys, list(out)))

    def set_launch_shape(self, kernel, threads=256, stages=4, rows=1, seg=1 << 30, cap=2048):
        shape = (ctypes.c_int64 * 6)(kernel, threads, stages, rows, seg, cap)
        _check(load().lbm_set_launch_shape(self._h, shape))

    def sync(self):
        _check(load().lbm_sync(self._h))


def _diag_dict(d):
    return {"mass": d.mass, "momentum": np.array(d.momentum[:]), "kinetic": d.kinetic,
            "max_u": d.max_u, "step": d.step, "nonfinite": d.nonfinite}


class Batch:
    """Many independent periodic lattices advanced together (lbm_batch_*)."""

    def __init__(self, lattice, dims, tau, eq_kind=ENTROPIC, bulk_corr=0, rho0=1.0,
                 stream=None):
        lib = load()
        dims = np.ascontiguousarray(dims, dtype=np.int32).reshape(-1, 3)
        self.dims = dims
        self.count = len(dims)
        self.D = 2 if lattice == D2Q9 else 3
        self.Q = 3 ** self.D
        self.ncells = dims.prod(axis=1).astype(np.int64)
        self.cell_start = np.concatenate([[0], np.cumsum(self.ncells)])
        tau = np.ascontiguousarray(tau, dtype=np.float64)
        self._h = ctypes.c_void_p()
        self._stream = _stream_handle(stream)
        _check(lib.lbm_batch_create(ctypes.byref(self._h), int(lattice), self.count,
                                    dims.ctypes.data_as(_pi32), tau.ctypes.data_as(_pdbl),
                                    int(eq_kind), int(bulk_corr), F64, float(rho0), self._stream))

    def close(self):
        if self._h:
            load().lbm_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_fields(self, rho, u, dtype=np.float64):
        pr, dev_r, kr = _buffer(rho, dtype)
        pu, dev_u, ku = _buffer(u, dtype)
        _check(load().lbm_batch_init_fields(self._h, pr, pu, _dt(dtype), dev_r))

    def set_probe(self, kvec, every_k):
        k = np.ascontiguousarray(kvec, dtype=np.int32).reshape(-1, 3)
        _check(load().lbm_batch_set_probe(self._h, k.ctypes.data_as(_pi32), int(every_k)))

    def step(self, n):
        _check(load().lbm_batch_step(self._h, int(n)))

    def probe_series(self):
        """Complex array (count, samples, 4): projections of rho, j_x, j_y, j_z."""
        ns = ctypes.c_int64()
        _check(load().lbm_batch_probe_series(self._h, None, 0, ctypes.byref(ns)))
        n = ns.value
        out = np.zeros((self.count, max(n, 1), 8))
        _check(load().lbm_batch_probe_series(self._h, out.ctypes.data_as(_pdbl), max(n, 1),
                                             ctypes.byref(ns)))
        out = out[:, :n]
        return out[..., 0::2] + 1j * out[..., 1::2]

    def status(self):
        s = np.zeros(self.count, dtype=np.int32)
        _check(load().lbm_batch_status(self._h, s.ctypes.data_as(_pi32)))
        return s

    def moments(self, dtype=np.float64, out=None):
        """rho (total,) and u (per instance [D][cells], packed) as NumPy arrays, or into
        the torch tensors `out` (host or device)."""
        if out is not None:
            rho, u = out
            _check(load().lbm_batch_moments(self._h, ctypes.c_void_p(rho.data_ptr()),
                                            ctypes.c_void_p(u.data_ptr()), _dt(dtype), int(rho.is_cuda)))
            return rho, u
        total = int(self.cell_start[-1])
        rho = np.empty(total, dtype=dtype)
        u = np.empty(total * self.D, dtype=dtype)
        _check(load().lbm_batch_moments(self._h, ctypes.c_void_p(rho.ctypes.data),
                                        ctypes.c_void_p(u.ctypes.data), _dt(dtype), 0))
        return rho, u

    def get_populations(self, dtype=np.float64):
        total = int(self.cell_start[-1])
        f = np.empty(total * self.Q, dtype=dtype)
        _check(load().lbm_batch_get_populations(self._h, ctypes.c_void_p(f.ctypes.data), _dt(dtype), 0))
        return f

    def info(self):
        t, s = ctypes.c_int64(), ctypes.c_int64()
        _check(load().lbm_batch_info(self._h, ctypes.byref(t), ctypes.byref(s)))
        return {"total_cells": t.value, "step": s.value}

    def launch_info(self):
        out = (ctypes.c_int64 * 4)()
        _check(load().lbm_batch_launch_info(self._h, out))
        return dict(zip(["threads", "blocks", "max_load", "mean_load"], list(out)))

    def set_launch_shape(self, threads, blocks):
        _check(load().lbm_batch_set_launch_shape(self._h, int(threads), int(blocks)))

    def autotune(self, steps=10):
        """lbm_batch_autotune: keep the fastest launch shape (the state is unchanged)."""
        _check(load().lbm_batch_autotune(self._h, int(steps)))

    def sync(self):
        _check(load().lbm_batch_sync(self._h))


def diagnostics_noalloc(lattice, dims, f, out, blocks=256, stream=None):
    """lbm_diagnostics_noalloc on device tensors: f (Q, ncell) float64 canonical
    populations, out (8,) float64; nothing is allocated and nothing synchronised."""
    d = (ctypes.c_int64 * 3)(*(list(dims) + [1, 1, 1])[:3])
    _check(load().lbm_diagnostics_noalloc(int(lattice), d, ctypes.c_void_p(f.data_ptr()), int(blocks),
                                          ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))


def vn_eigenvalues(eq_kind, bulk_corr, params, stream=None):
    """Eigenvalues (count, 9) complex of M = E (delta + J) for params (count, 6) =
    (tau, rho, u_x, u_y, k_x, k_y), sorted by decreasing modulus (lbm_vn_eigenvalues)."""
    p = np.ascontiguousarray(params, dtype=np.float64).reshape(-1, 6)
    out = np.zeros((len(p), 9, 2))
    _check(load().lbm_vn_eigenvalues(int(eq_kind), int(bulk_corr), len(p), p.ctypes.data_as(_pdbl),
                                     out.ctypes.data_as(_pdbl), _stream_handle(stream)))
    return out[..., 0] + 1j * out[..., 1]


def vn_stability_limit(eq_kind, nu, theta, nk=33, u_hi=0.999, iterations=20, tol=1e-10, stream=None):
    """Largest linearly stable |u| per (nu, theta) pair (lbm_vn_stability_limit)."""
    nu = np.ascontiguousarray(nu, dtype=np.float64).reshape(-1)
    theta = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1)
    out = np.zeros(len(nu))
    _check(load().lbm_vn_stability_limit(int(eq_kind), len(nu), nu.ctypes.data_as(_pdbl),
                                         theta.ctypes.data_as(_pdbl), int(nk), float(u_hi),
                                         int(iterations), float(tol), out.ctypes.data_as(_pdbl),
                                         _stream_handle(stream)))
    return out


def selftest_bounded_wait(timeout_ns=1_000_000, stream=None):
    """Run the bounded-wait self test; returns the status the kernel wrote."""
    st = ctypes.c_int32(12345)
    _check(load().lbm_selftest_bounded_wait(_stream_handle(stream), int(timeout_ns), ctypes.byref(st)))
    return st.value
