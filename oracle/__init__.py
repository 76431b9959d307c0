"""ctypes binding of the FP64 CPU oracle (ehd_oracle.c).

TEST INFRASTRUCTURE ONLY.  The oracle is the yardstick for the CUDA library:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the product.

Parameters are passed as a plain dict whose keys are the field names of
``orc_params`` (see ``ehd_oracle.h``); missing keys keep the defaults below,
which are the lattice values of the plain 64x64 droplet case.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ehd_oracle.c")
LIB = os.path.join(HERE, "libehd_oracle.so")

FIELDS = ["phi", "ux", "uy", "p", "psi", "Ex", "Ey", "cp", "cm", "q"]
STATE_PER_NODE = 35  # f9 h9 p5 n5 g5 phiu2 (43 with ions on D2Q9: p9 n9)

_PARAM_FIELDS = [
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


class OrcParams(C.Structure):
    _fields_ = _PARAM_FIELDS


DEFAULTS = dict(
    tau_f=0.8, rho_ratio=1.0, eta_ratio=1.0, sigma=0.01, W=4.0, W_init=0.0,
    M_phi=0.02, nhat_eps=1e-3, xc=31.5, yc=31.5, R=12.0, init_shape=0, D=0.01, mu_v=1.0,
    mu_r=1.0, m=1.0, k_d=1.0, k_r=1.0, onsager_cb=1.0, onsager_form=0,
    ion_bc=0, einstein_D=1, ion_L_term=1, c_init_scale=1.0, c0=1.0, eps_r=2.0,
    Kq=5.6893 / 64**2, vartheta=0.3, psi_src_literal=0, psi_anode=1.0, psi_cathode=0.0,
    sweeps_min=1, sweeps_max=200, sweep_tol=1e-8, init_sweeps_max=100000,
    init_sweeps_fixed=-1, init_psi_zero=0, freeze_E=0, E_frozen_x=0.0,
    E_frozen_y=0.0, s_free=1.0, bgk=0, ion_lattice=5, side_walls=0,
)


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/libehd_oracle.so with gcc (C11)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "ehd_oracle.h"))
    ):
        cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-ffp-contract=off",
               "-fPIC", "-shared", "-o", LIB, SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.c_int, C.c_int, C.POINTER(OrcParams)]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_init.argtypes = [C.c_void_p]
        L.orc_init.restype = C.c_int
        L.orc_step.argtypes = [C.c_void_p, C.c_int, ip, ip, dp]
        L.orc_step.restype = C.c_int
        L.orc_get_fields.argtypes = [C.c_void_p, dp]
        L.orc_get_state.argtypes = [C.c_void_p, dp]
        L.orc_set_state.argtypes = [C.c_void_p, dp]
        L.orc_sum_phi.argtypes = [C.c_void_p]
        L.orc_sum_phi.restype = C.c_double
        L.orc_time.argtypes = [C.c_void_p]
        L.orc_time.restype = C.c_long
        L.orc_matrices.argtypes = [dp, dp, dp, dp]
        L.orc_feq.argtypes = [C.c_double] * 4 + [dp]
        L.orc_forcing_f.argtypes = [C.c_double] * 6 + [dp]
        L.orc_heq.argtypes = [C.c_double] * 3 + [dp]
        L.orc_pressure.argtypes = [dp] + [C.c_double] * 5
        L.orc_pressure.restype = C.c_double
        L.orc_ion_src.argtypes = [C.c_int] + [C.c_double] * 4 + [C.c_int, dp]
        L.orc_Hsrc.argtypes = [C.c_double] * 7 + [dp]
        L.orc_ion_eq.argtypes = [C.c_double] * 3 + [dp]
        L.orc_ion_eq9.argtypes = [C.c_double] * 3 + [dp]
        L.orc_state_per_node.argtypes = [C.c_void_p]
        L.orc_state_per_node.restype = C.c_int
        L.orc_geq.argtypes = [C.c_double, dp]
        L.orc_mrt.argtypes = [C.c_int, dp, dp, dp, dp, dp]
        L.orc_onsager.argtypes = [C.c_double, C.c_int]
        L.orc_onsager.restype = C.c_double
        L.orc_reaction.argtypes = [C.c_double] * 5 + [dp, dp, dp]
        L.orc_stencil.argtypes = [C.c_int, C.c_int, dp, dp, dp, dp]
        L.orc_stencil_walls.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, dp, dp]
        L.orc_params_from_physical.argtypes = [C.POINTER(OrcParams), C.c_int,
                                               C.c_int] + [C.c_double] * 4
        L.orc_sample.argtypes = [C.c_int, C.c_int, dp, C.c_double, C.c_double]
        L.orc_sample.restype = C.c_double
        L.orc_deformation.argtypes = [C.c_int, C.c_int, dp]
        L.orc_deformation.restype = C.c_double
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def make_params(overrides: dict | None = None) -> OrcParams:
    d = dict(DEFAULTS)
    if overrides:
        unknown = set(overrides) - set(d)
        if unknown:
            raise KeyError(f"unknown oracle parameters: {sorted(unknown)}")
        d.update(overrides)
    P = OrcParams()
    for name, _ in _PARAM_FIELDS:
        setattr(P, name, d[name])
    return P


def params_from_physical(nx, ny, d_mm, dpsi_kV, eps_r, mu_r) -> dict:
    P = OrcParams()
    lib().orc_params_from_physical(C.byref(P), nx, ny, d_mm, dpsi_kV, eps_r, mu_r)
    return {name: getattr(P, name) for name, _ in _PARAM_FIELDS}


class Oracle:
    """One lattice advanced by the oracle."""

    def __init__(self, nx: int, ny: int, params: dict | None = None):
        self.nx, self.ny = nx, ny
        self._P = make_params(params)
        self._h = lib().orc_create(nx, ny, C.byref(self._P))
        if not self._h:
            raise ValueError("orc_create rejected the lattice")
        self.init_sweeps = lib().orc_init(self._h)

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, nsteps: int, forced=None):
        """Advance; returns (sweep counts, last residuals, not-converged)."""
        counts = np.zeros(nsteps, dtype=np.int32)
        res = np.zeros(nsteps, dtype=np.float64)
        fp = None
        if forced is not None:
            fa = np.ascontiguousarray(np.asarray(forced, dtype=np.int32))
            assert fa.size >= nsteps
            fp = _ip(fa)
        nc = lib().orc_step(self._h, nsteps, fp, _ip(counts), _dp(res))
        return counts, res, nc

    def fields(self) -> dict:
        out = np.zeros((len(FIELDS), self.ny, self.nx))
        lib().orc_get_fields(self._h, _dp(out))
        return {k: out[i] for i, k in enumerate(FIELDS)}

    def state(self) -> np.ndarray:
        out = np.zeros((self.ny, self.nx, lib().orc_state_per_node(self._h)))
        lib().orc_get_state(self._h, _dp(out))
        return out

    def set_state(self, s: np.ndarray):
        s = np.ascontiguousarray(s, dtype=np.float64)
        assert s.shape == (self.ny, self.nx, lib().orc_state_per_node(self._h))
        lib().orc_set_state(self._h, _dp(s))

    def sum_phi(self) -> float:
        return lib().orc_sum_phi(self._h)

    @property
    def t(self) -> int:
        return lib().orc_time(self._h)


# ---- per-node building blocks ------------------------------------------------

def matrices():
    M = np.zeros((9, 9)); Mi = np.zeros((9, 9)); N = np.zeros((5, 5)); Ni = np.zeros((5, 5))
    lib().orc_matrices(_dp(M), _dp(Mi), _dp(N), _dp(Ni))
    return M, Mi, N, Ni


def feq(p, rho, ux, uy):
    o = np.zeros(9); lib().orc_feq(p, rho, ux, uy, _dp(o)); return o


def forcing_f(ux, uy, Fx, Fy, grx, gry):
    o = np.zeros(9); lib().orc_forcing_f(ux, uy, Fx, Fy, grx, gry, _dp(o)); return o


def pressure(f, rho, ux, uy, grx, gry):
    f = np.ascontiguousarray(f, dtype=np.float64)
    return lib().orc_pressure(_dp(f), rho, ux, uy, grx, gry)


def ion_src(R, c, Fx, Fy, L_term=1, q=5):
    o = np.zeros(q); lib().orc_ion_src(q, R, c, Fx, Fy, L_term, _dp(o)); return o


def heq(phi, ux, uy):
    o = np.zeros(9); lib().orc_heq(phi, ux, uy, _dp(o)); return o


def Hsrc(phi, W, dpux, dpuy, gx, gy, eps=0.0):
    o = np.zeros(9); lib().orc_Hsrc(phi, W, dpux, dpuy, gx, gy, eps, _dp(o)); return o


def ion_eq(c, ux, uy, q=5):
    o = np.zeros(q)
    (lib().orc_ion_eq9 if q == 9 else lib().orc_ion_eq)(c, ux, uy, _dp(o))
    return o


def geq(psi):
    o = np.zeros(5); lib().orc_geq(psi, _dp(o)); return o


def mrt(s, x, xeq, src):
    s = np.ascontiguousarray(s, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    xeq = np.ascontiguousarray(xeq, dtype=np.float64)
    src = np.ascontiguousarray(src, dtype=np.float64)
    o = np.zeros(x.size)
    lib().orc_mrt(x.size, _dp(s), _dp(x), _dp(xeq), _dp(src), _dp(o))
    return o


def onsager(b, form=0):
    return lib().orc_onsager(b, form)


def reaction(sum_p, sum_n, k_d, k_r, F):
    cp = C.c_double(); cm = C.c_double(); R = C.c_double()
    lib().orc_reaction(sum_p, sum_n, k_d, k_r, F, C.byref(cp), C.byref(cm), C.byref(R))
    return cp.value, cm.value, R.value


def stencil(chi: np.ndarray, side_walls: int = 0):
    chi = np.ascontiguousarray(chi, dtype=np.float64)
    ny, nx = chi.shape
    gx = np.zeros_like(chi); gy = np.zeros_like(chi); lap = np.zeros_like(chi)
    if side_walls:
        lib().orc_stencil_walls(nx, ny, 1, _dp(chi), _dp(gx), _dp(gy), _dp(lap))
    else:
        lib().orc_stencil(nx, ny, _dp(chi), _dp(gx), _dp(gy), _dp(lap))
    return gx, gy, lap


def sample(phi, x, y):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    ny, nx = phi.shape
    return lib().orc_sample(nx, ny, _dp(phi), x, y)


def deformation(phi: np.ndarray) -> float:
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    ny, nx = phi.shape
    return lib().orc_deformation(nx, ny, _dp(phi))
