"""Thin ctypes binding of libehdlb (include/ehdlb.h), same names as the C ABI.

Only argument marshalling happens here: every step of the solver runs in the
CUDA kernels of the library.  If the library cannot be loaded the import
fails; there is no other implementation behind these functions.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

FIELDS = ["phi", "ux", "uy", "p", "psi", "Ex", "Ey", "cp", "cm", "q"]
FP64, FP32, FP16S = 0, 1, 2
OK, WNOTCONV, EINVAL, ENOMEM, ECUDA, EUNSTABLE, ESTATE, EFULL = 0, 1, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "OK", 1: "WNOTCONV", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA",
                -4: "EUNSTABLE", -5: "ESTATE", -6: "EFULL"}

_PARAM_FIELDS = [
    ("size", C.c_size_t),
    ("tau_f", C.c_double), ("rho_ratio", C.c_double), ("eta_ratio", C.c_double),
    ("sigma", C.c_double), ("W", C.c_double), ("W_init", C.c_double),
    ("M_phi", C.c_double), ("nhat_eps", C.c_double),
    ("xc", C.c_double), ("yc", C.c_double), ("R", C.c_double),
    ("init_shape", C.c_int),
    ("D", C.c_double), ("mu_v", C.c_double), ("mu_r", C.c_double),
    ("m", C.c_double), ("k_d", C.c_double), ("k_r", C.c_double),
    ("onsager_cb", C.c_double),
    ("onsager_form", C.c_int), ("ion_bc", C.c_int), ("einstein_D", C.c_int),
    ("ion_L_term", C.c_int),
    ("c_init_scale", C.c_double), ("c0", C.c_double),
    ("eps_r", C.c_double), ("Kq", C.c_double), ("vartheta", C.c_double),
    ("psi_src_literal", C.c_int),
    ("psi_anode", C.c_double), ("psi_cathode", C.c_double),
    ("sweeps_min", C.c_int), ("sweeps_max", C.c_int),
    ("sweep_tol", C.c_double),
    ("init_sweeps_max", C.c_int), ("init_sweeps_fixed", C.c_int),
    ("init_psi_zero", C.c_int),
    ("freeze_E", C.c_int), ("E_frozen_x", C.c_double), ("E_frozen_y", C.c_double),
    ("s_free", C.c_double), ("bgk", C.c_int),
    ("ion_lattice", C.c_int), ("side_walls", C.c_int),
]


class ehdlb_params(C.Structure):
    _fields_ = _PARAM_FIELDS


class ehdlb_stats(C.Structure):
    _fields_ = [
        ("steps", C.c_longlong), ("t", C.c_longlong), ("sweeps_total", C.c_longlong),
        ("sweeps_max", C.c_int), ("not_converged", C.c_int),
        ("last_residual", C.c_double), ("sum_phi", C.c_double), ("sum_q", C.c_double),
        ("seconds", C.c_double), ("mlups", C.c_double),
        ("ms_prep", C.c_double), ("ms_sweeps", C.c_double), ("ms_main", C.c_double),
        ("launches", C.c_longlong), ("sweep_launches", C.c_longlong),
        ("sweeps_per_launch", C.c_int), ("tile_shape", C.c_int), ("deformation", C.c_double),
    ]


class ehdlb_batch_stats(C.Structure):
    _fields_ = [
        ("steps", C.c_longlong), ("cases", C.c_int), ("unstable_cases", C.c_int),
        ("seconds", C.c_double), ("device_ms", C.c_double), ("mlups", C.c_double),
        ("launches", C.c_longlong), ("sweeps_per_launch", C.c_int), ("tile_shape", C.c_int),
    ]


class EhdlbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load libehdlb.so (building it in-tree with nvcc if it is out of date)."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise ImportError(f"libehdlb.so missing at {path}")
        L = C.CDLL(path)
        vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
        L.ehdlb_version.restype = C.c_int
        L.ehdlb_params_default.argtypes = [C.POINTER(ehdlb_params)]
        L.ehdlb_params_from_physical.argtypes = [C.POINTER(ehdlb_params), C.c_int, C.c_int,
                                                 C.c_double, C.c_double, C.c_double, C.c_double]
        L.ehdlb_create.argtypes = [C.POINTER(vp), C.c_int, C.c_int, C.c_int, vp]
        L.ehdlb_set_params.argtypes = [vp, C.POINTER(ehdlb_params)]
        L.ehdlb_set_sweep_schedule.argtypes = [vp, ip, C.c_int]
        L.ehdlb_step.argtypes = [vp, C.c_int, C.POINTER(ehdlb_stats)]
        L.ehdlb_test_stall_copies.argtypes = [vp]
        L.ehdlb_get_fields.argtypes = [vp, C.c_uint, dp, C.c_size_t]
        L.ehdlb_get_sweep_counts.argtypes = [vp, ip, C.c_int]
        L.ehdlb_state_len.argtypes = [vp]
        L.ehdlb_state_len.restype = C.c_size_t
        L.ehdlb_get_state.argtypes = [vp, dp, C.c_size_t]
        L.ehdlb_set_state.argtypes = [vp, dp, C.c_size_t]
        L.ehdlb_set_timing.argtypes = [vp, C.c_int]
        L.ehdlb_set_tuning.argtypes = [vp, C.c_int, C.c_int, C.c_int]
        L.ehdlb_set_reporting.argtypes = [vp, C.c_uint, C.c_int]
        L.ehdlb_potential_noalloc.argtypes = [C.c_int, C.c_int, C.POINTER(ehdlb_params), vp, vp,
                                              C.c_int, vp, vp, vp, dp, vp]
        L.ehdlb_deformation.argtypes = [vp, dp]
        L.ehdlb_batch_create.argtypes = [C.POINTER(vp), C.c_int, C.c_size_t, C.c_int, vp]
        L.ehdlb_batch_footprint.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_size_t)]
        L.ehdlb_batch_add.argtypes = [vp, C.c_int, C.c_int, C.POINTER(ehdlb_params), ip]
        L.ehdlb_batch_remove.argtypes = [vp, C.c_int]
        L.ehdlb_batch_step.argtypes = [vp, C.c_int, C.POINTER(ehdlb_batch_stats)]
        L.ehdlb_batch_get_fields.argtypes = [vp, C.c_int, C.c_uint, dp, C.c_size_t]
        L.ehdlb_batch_get_state.argtypes = [vp, C.c_int, dp, C.c_size_t]
        L.ehdlb_batch_deformation.argtypes = [vp, C.c_int, ip, dp]
        L.ehdlb_batch_set_tuning.argtypes = [vp, C.c_int, C.c_int, C.c_int]
        L.ehdlb_batch_autotune.argtypes = [vp, C.c_int, ip, ip, dp]
        L.ehdlb_batch_info.argtypes = [vp, ip, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]
        L.ehdlb_batch_last_error.argtypes = [vp]
        L.ehdlb_batch_last_error.restype = C.c_char_p
        L.ehdlb_batch_destroy.argtypes = [vp]
        L.ehdlb_batch_destroy.restype = None
        L.ehdlb_destroy.argtypes = [vp]
        L.ehdlb_destroy.restype = None
        L.ehdlb_last_error.argtypes = [vp]
        L.ehdlb_last_error.restype = C.c_char_p
        if L.ehdlb_version() != 5:
            raise ImportError("libehdlb ABI version mismatch")
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _check(ctx, status, what):
    if status < 0:
        msg = lib().ehdlb_last_error(ctx).decode() if ctx else ""
        raise EhdlbError(status, f"{what}: {msg}")
    return status


# ---- the C functions, one to one ---------------------------------------------

def ehdlb_version() -> int:
    return lib().ehdlb_version()


def ehdlb_params_default(overrides: dict | None = None) -> ehdlb_params:
    p = ehdlb_params()
    _check(None, lib().ehdlb_params_default(C.byref(p)), "ehdlb_params_default")
    return _apply(p, overrides)


def ehdlb_params_from_physical(nx, ny, d_mm, dpsi_kV, eps_r, mu_r,
                               overrides: dict | None = None) -> ehdlb_params:
    p = ehdlb_params()
    _check(None, lib().ehdlb_params_from_physical(C.byref(p), nx, ny, d_mm, dpsi_kV, eps_r, mu_r),
           "ehdlb_params_from_physical")
    return _apply(p, overrides)


def _apply(p, overrides):
    if overrides:
        names = {n for n, _ in _PARAM_FIELDS}
        bad = set(overrides) - names
        if bad:
            raise KeyError(f"unknown parameters: {sorted(bad)}")
        for k, v in overrides.items():
            setattr(p, k, v)
    return p


def params_dict(p: ehdlb_params) -> dict:
    return {n: getattr(p, n) for n, _ in _PARAM_FIELDS if n != "size"}


def ehdlb_create(nx: int, ny: int, precision: int = FP32, cuda_stream: int | None = None):
    h = C.c_void_p()
    _check(None, lib().ehdlb_create(C.byref(h), nx, ny, precision,
                                    C.c_void_p(cuda_stream) if cuda_stream else None),
           "ehdlb_create")
    return h


def ehdlb_set_params(ctx, p: ehdlb_params):
    return _check(ctx, lib().ehdlb_set_params(ctx, C.byref(p)), "ehdlb_set_params")


def ehdlb_set_sweep_schedule(ctx, counts):
    a = np.ascontiguousarray(np.asarray(counts, dtype=np.int32))
    return _check(ctx, lib().ehdlb_set_sweep_schedule(
        ctx, a.ctypes.data_as(C.POINTER(C.c_int)), int(a.size)), "ehdlb_set_sweep_schedule")


def ehdlb_test_stall_copies(ctx):
    return _check(ctx, lib().ehdlb_test_stall_copies(ctx), "ehdlb_test_stall_copies")


def ehdlb_step(ctx, nsteps: int):
    st = ehdlb_stats()
    status = _check(ctx, lib().ehdlb_step(ctx, nsteps, C.byref(st)), "ehdlb_step")
    return status, st


def ehdlb_get_fields(ctx, mask: int, dst: np.ndarray):
    assert dst.dtype == np.float64 and dst.flags.c_contiguous
    return _check(ctx, lib().ehdlb_get_fields(ctx, mask, _dp(dst), dst.size), "ehdlb_get_fields")


def ehdlb_get_sweep_counts(ctx, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.int32)
    _check(ctx, lib().ehdlb_get_sweep_counts(ctx, out.ctypes.data_as(C.POINTER(C.c_int)), n),
           "ehdlb_get_sweep_counts")
    return out


def ehdlb_state_len(ctx) -> int:
    return lib().ehdlb_state_len(ctx)


def ehdlb_get_state(ctx, dst: np.ndarray):
    assert dst.dtype == np.float64 and dst.flags.c_contiguous
    return _check(ctx, lib().ehdlb_get_state(ctx, _dp(dst), dst.size), "ehdlb_get_state")


def ehdlb_set_state(ctx, src: np.ndarray):
    src = np.ascontiguousarray(src, dtype=np.float64)
    return _check(ctx, lib().ehdlb_set_state(ctx, _dp(src), src.size), "ehdlb_set_state")


def ehdlb_set_timing(ctx, every):
    """every: True / False, or record every n-th step (n >= 1; 0 off)."""
    n = (1 if every else 0) if isinstance(every, bool) else int(every)
    return _check(ctx, lib().ehdlb_set_timing(ctx, n), "ehdlb_set_timing")


def ehdlb_potential_noalloc(nx, ny, p: ehdlb_params, phi_dev: int, q_dev: int, nsweeps: int,
                            psi_dev: int, ex_dev: int, ey_dev: int, cuda_stream: int | None = None):
    """Potential solve that allocates nothing; arrays are device addresses.
    Returns (status, residual of the last sweep)."""
    r = C.c_double(float("nan"))
    status = lib().ehdlb_potential_noalloc(
        nx, ny, C.byref(p), C.c_void_p(phi_dev), C.c_void_p(q_dev), nsweeps,
        C.c_void_p(psi_dev), C.c_void_p(ex_dev), C.c_void_p(ey_dev), C.byref(r),
        C.c_void_p(cuda_stream) if cuda_stream else None)
    return status, r.value


def ehdlb_set_reporting(ctx, snapshot_mask: int, deformation: int = 0):
    return _check(ctx, lib().ehdlb_set_reporting(ctx, snapshot_mask, deformation), "ehdlb_set_reporting")


def ehdlb_set_tuning(ctx, sweeps_per_launch: int = -1, tile_shape: int = -1, main_staging: int = -1):
    return _check(ctx, lib().ehdlb_set_tuning(ctx, sweeps_per_launch, tile_shape, main_staging),
                  "ehdlb_set_tuning")


def ehdlb_deformation(ctx) -> float:
    d = C.c_double()
    _check(ctx, lib().ehdlb_deformation(ctx, C.byref(d)), "ehdlb_deformation")
    return d.value


def ehdlb_destroy(ctx):
    lib().ehdlb_destroy(ctx)


# ---- batches ---------------------------------------------------------------------

def _bcheck(b, status, what):
    if status < 0:
        msg = lib().ehdlb_batch_last_error(b).decode() if b else ""
        raise EhdlbError(status, f"{what}: {msg}")
    return status


def ehdlb_batch_create(precision: int, budget_bytes: int, sweeps: int, cuda_stream: int | None = None):
    h = C.c_void_p()
    _bcheck(None, lib().ehdlb_batch_create(C.byref(h), precision, budget_bytes, sweeps,
                                           C.c_void_p(cuda_stream) if cuda_stream else None),
            "ehdlb_batch_create")
    return h


def ehdlb_batch_footprint(precision: int, nx: int, ny: int) -> int:
    b = C.c_size_t()
    _bcheck(None, lib().ehdlb_batch_footprint(precision, nx, ny, C.byref(b)), "ehdlb_batch_footprint")
    return b.value


def ehdlb_batch_add(b, nx: int, ny: int, p: ehdlb_params):
    """Returns (status, id); status EFULL (no room) is returned, not raised."""
    i = C.c_int(-1)
    st = lib().ehdlb_batch_add(b, nx, ny, C.byref(p), C.byref(i))
    if st != EFULL:
        _bcheck(b, st, "ehdlb_batch_add")
    return st, i.value


def ehdlb_batch_remove(b, case_id: int):
    return _bcheck(b, lib().ehdlb_batch_remove(b, case_id), "ehdlb_batch_remove")


def ehdlb_batch_step(b, nsteps: int):
    st = ehdlb_batch_stats()
    status = _bcheck(b, lib().ehdlb_batch_step(b, nsteps, C.byref(st)), "ehdlb_batch_step")
    return status, st


def ehdlb_batch_get_fields(b, case_id: int, mask: int, out: np.ndarray):
    assert out.dtype == np.float64 and out.flags["C_CONTIGUOUS"]
    return _bcheck(b, lib().ehdlb_batch_get_fields(b, case_id, mask, _dp(out), out.size),
                   "ehdlb_batch_get_fields")


def ehdlb_batch_get_state(b, case_id: int, out: np.ndarray):
    assert out.dtype == np.float64 and out.flags["C_CONTIGUOUS"]
    return _bcheck(b, lib().ehdlb_batch_get_state(b, case_id, _dp(out), out.size), "ehdlb_batch_get_state")


def ehdlb_batch_deformation(b, ids) -> np.ndarray:
    ids = np.ascontiguousarray(np.asarray(ids, dtype=np.int32))
    out = np.zeros(ids.size)
    _bcheck(b, lib().ehdlb_batch_deformation(b, ids.size, ids.ctypes.data_as(C.POINTER(C.c_int)), _dp(out)),
            "ehdlb_batch_deformation")
    return out


def ehdlb_batch_set_tuning(b, sweeps_per_launch=-1, tile_shape=-1, use_graphs=-1):
    return _bcheck(b, lib().ehdlb_batch_set_tuning(b, sweeps_per_launch, tile_shape, use_graphs),
                   "ehdlb_batch_set_tuning")


def ehdlb_batch_autotune(b, steps: int):
    spl, shape, ms = C.c_int(), C.c_int(), C.c_double()
    _bcheck(b, lib().ehdlb_batch_autotune(b, steps, C.byref(spl), C.byref(shape), C.byref(ms)),
            "ehdlb_batch_autotune")
    return spl.value, shape.value, ms.value


def ehdlb_batch_info(b):
    n, used, cap = C.c_int(), C.c_size_t(), C.c_size_t()
    _bcheck(b, lib().ehdlb_batch_info(b, C.byref(n), C.byref(used), C.byref(cap)), "ehdlb_batch_info")
    return n.value, used.value, cap.value


def ehdlb_batch_destroy(b):
    lib().ehdlb_batch_destroy(b)


def ehdlb_last_error(ctx) -> str:
    return lib().ehdlb_last_error(ctx).decode()


# ---- convenience wrapper -------------------------------------------------------

class Lattice:
    """One solver context: create + set_params, then step / fields / state."""

    def __init__(self, nx, ny, params: dict | ehdlb_params | None = None, precision=FP32,
                 cuda_stream=None, schedule=None):
        self.nx, self.ny, self.precision = nx, ny, precision
        self.ctx = ehdlb_create(nx, ny, precision, cuda_stream)
        if schedule is not None:
            ehdlb_set_sweep_schedule(self.ctx, schedule)
        p = params if isinstance(params, ehdlb_params) else ehdlb_params_default(params)
        self.params = p
        ehdlb_set_params(self.ctx, p)

    def step(self, nsteps: int):
        status, st = ehdlb_step(self.ctx, nsteps)
        return status, st

    def fields(self, names=None) -> dict:
        names = FIELDS if names is None else list(names)
        idx = sorted(FIELDS.index(n) for n in names)
        mask = sum(1 << i for i in idx)
        out = np.zeros((len(idx), self.ny, self.nx))
        ehdlb_get_fields(self.ctx, mask, out)
        return {FIELDS[i]: out[j] for j, i in enumerate(idx)}

    def sweep_counts(self, n):
        return ehdlb_get_sweep_counts(self.ctx, n)

    def state(self) -> np.ndarray:
        spn = lib().ehdlb_state_len(self.ctx) // (self.nx * self.ny)
        out = np.zeros((self.ny, self.nx, spn))
        ehdlb_get_state(self.ctx, out)
        return out

    def set_state(self, s):
        spn = lib().ehdlb_state_len(self.ctx) // (self.nx * self.ny)
        ehdlb_set_state(self.ctx, np.asarray(s, dtype=np.float64).reshape(self.ny, self.nx, spn))

    def deformation(self) -> float:
        return ehdlb_deformation(self.ctx)

    def close(self):
        if self.ctx:
            ehdlb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many lattices stepped together (see ehdlb_batch_create)."""

    def __init__(self, budget_bytes: int, sweeps: int = 20, precision=FP32, cuda_stream=None):
        self.precision = precision
        self.b = ehdlb_batch_create(precision, budget_bytes, sweeps, cuda_stream)
        self.sizes = {}

    def add(self, nx, ny, params: dict | ehdlb_params):
        """Case id, or None if the budget has no room."""
        p = params if isinstance(params, ehdlb_params) else ehdlb_params_default(params)
        st, cid = ehdlb_batch_add(self.b, nx, ny, p)
        if st == EFULL:
            return None
        self.sizes[cid] = (nx, ny)
        return cid

    def remove(self, cid):
        ehdlb_batch_remove(self.b, cid)
        del self.sizes[cid]

    def step(self, nsteps: int):
        return ehdlb_batch_step(self.b, nsteps)

    def fields(self, cid, names=None) -> dict:
        nx, ny = self.sizes[cid]
        names = FIELDS if names is None else list(names)
        idx = sorted(FIELDS.index(n) for n in names)
        out = np.zeros((len(idx), ny, nx))
        ehdlb_batch_get_fields(self.b, cid, sum(1 << i for i in idx), out)
        return {FIELDS[i]: out[j] for j, i in enumerate(idx)}

    def state(self, cid) -> np.ndarray:
        nx, ny = self.sizes[cid]
        out = np.zeros((ny, nx, 35))
        ehdlb_batch_get_state(self.b, cid, out)
        return out

    def deformation(self, ids) -> np.ndarray:
        return ehdlb_batch_deformation(self.b, ids)

    def set_tuning(self, sweeps_per_launch=-1, tile_shape=-1, use_graphs=-1):
        ehdlb_batch_set_tuning(self.b, sweeps_per_launch, tile_shape, use_graphs)

    def autotune(self, steps: int):
        return ehdlb_batch_autotune(self.b, steps)

    def info(self):
        return ehdlb_batch_info(self.b)

    def close(self):
        if self.b:
            ehdlb_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
