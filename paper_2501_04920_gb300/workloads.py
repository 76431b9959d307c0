"""Lattice parameters of the standard synthetic droplet-in-field cases.

Plain data only (parameter dictionaries keyed by the ehdlb_params field names,
which the oracle's parameter block shares); no arithmetic of the method lives
here.  Cases:

* ``droplet64``: the plain 64x64 case in FP64 -- centred droplet R = 12 with
  a tanh profile of width 4 (phi = 1 inside), electrodes psi = 1 below row 0
  and psi = 0 above row 63, periodic x; tau_f = 0.8, density and viscosity
  ratio 1, sigma = 0.01, M_phi = 0.02; D = 0.01, mu_r = 1, k_d = k_r = 1,
  b = sqrt(|E|); eps_r = 2, Kq = W0 / 64^2 with W0 = 5.6893 (d = 2 mm,
  1 kV); potential swept to a relative change of 1e-8 (cap 200) every step,
  the initial potential solved to the same tolerance; 2000 steps.
* ``uneven_cases()``: 96 physical cases of uneven size for the batch engine.
* ``arrivals()``: a Poisson stream of cases for the serving loop.
* ``droplet(n)``: the plain FP32 case on an n x n lattice (n = 2048 for the
  throughput case, n = 256 for its oracle-sized copy): R = n / 8, eps_r = 4,
  mu_r = 2, dpsi = 2, b = 0.5 sqrt(|E|), Kq = 5.6893 / n^2 (W0 at d = 2 mm,
  2 kV, times dpsi), exactly 20 sweeps per step, initial potential linear
  (no initial sweeps); 20000 steps at 2048^2.
"""
from __future__ import annotations

W0_2MM_1KV = 5.6893  # conduction number printed with Fig. 10 (d = 2 mm, 1 kV)


def droplet64() -> dict:
    n = 64
    return dict(
        tau_f=0.8, rho_ratio=1.0, eta_ratio=1.0, sigma=0.01, W=4.0, W_init=0.0,
        M_phi=0.02, nhat_eps=1e-3, xc=(n - 1) / 2, yc=(n - 1) / 2, R=12.0, init_shape=0,
        D=0.01, mu_v=1.0, mu_r=1.0, m=1.0, k_d=1.0, k_r=1.0, onsager_cb=1.0,
        onsager_form=0, ion_bc=0, einstein_D=1, ion_L_term=1, c_init_scale=1.0,
        c0=1.0, eps_r=2.0, Kq=W0_2MM_1KV / n**2, vartheta=0.3, psi_src_literal=0,
        psi_anode=1.0, psi_cathode=0.0, sweeps_min=1, sweeps_max=200,
        sweep_tol=1e-8, init_sweeps_max=100000, init_sweeps_fixed=-1,
        init_psi_zero=0, freeze_E=0, E_frozen_x=0.0, E_frozen_y=0.0,
        s_free=1.0, bgk=0)


def droplet(n: int = 2048) -> dict:
    d = droplet64()
    d.update(xc=(n - 1) / 2, yc=(n - 1) / 2, R=n / 8, eps_r=4.0, mu_r=2.0,
             psi_anode=2.0, psi_cathode=0.0, onsager_cb=0.5,
             Kq=(W0_2MM_1KV / 2) * 2.0 / n**2,
             sweeps_min=20, sweeps_max=20, init_sweeps_fixed=0, init_sweeps_max=0)
    return d


def uneven_cases(n: int = 96, seed: int = 20250109) -> list[dict]:
    """The uneven batch: n physical cases drawn with numpy's default_rng(seed).
    nx from {128, 192, ..., 768}; ny uniform over the multiples of 64 in
    [nx, 2 nx]; electrode gap d ~ U[0.5, 2] mm; dpsi ~ U[0.5, 4] kV; eps_r from
    {0.5, 1, 2, 4}; mu_r from {0.5, 1, 2}.  Each entry holds the arguments of
    ehdlb_params_from_physical (R = nx / 5 there); 10000 steps each."""
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nx = int(rng.choice(np.arange(128, 769, 64)))
        ny = int(rng.choice(np.arange(nx, 2 * nx + 1, 64)))
        out.append(dict(nx=nx, ny=ny, d_mm=float(rng.uniform(0.5, 2.0)),
                        dpsi_kV=float(rng.uniform(0.5, 4.0)),
                        eps_r=float(rng.choice([0.5, 1.0, 2.0, 4.0])),
                        mu_r=float(rng.choice([0.5, 1.0, 2.0]))))
    return out


def arrivals(n: int = 1000, rate_per_s: float = 1.0, seed: int = 20250109,
             side_min: int = 128, side_max_factor: float = 8.0) -> list[dict]:
    """A stream of served cases: Poisson arrival times at rate_per_s, square
    lattices of side side_min * side_max_factor^U (U ~ U[0, 1]) rounded to a
    multiple of 64, physical parameters drawn as in uneven_cases."""
    import numpy as np
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
    out = []
    for i in range(n):
        side = int(max(64, round(side_min * side_max_factor ** rng.uniform() / 64) * 64))
        out.append(dict(t=float(t[i]), nx=side, ny=side, d_mm=float(rng.uniform(0.5, 2.0)),
                        dpsi_kV=float(rng.uniform(0.5, 4.0)),
                        eps_r=float(rng.choice([0.5, 1.0, 2.0, 4.0])),
                        mu_r=float(rng.choice([0.5, 1.0, 2.0]))))
    return out


STEPS = {"droplet64": 2000, "droplet2048": 20000, "uneven": 10000}
