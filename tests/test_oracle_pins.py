"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test names the part of the oracle it pins and the source of the expected
value (an equation of arXiv 2501.04920, a printed number under tests/golden/, a
closed form or an independent library routine).  None of them recomputes the
oracle's own formula; each is chosen so that a dropped term, a wrong sign or a
transposed operand in that part fails it.
"""
import os

import numpy as np
import pytest
from scipy import integrate, special

import oracle as O

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

CX9 = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY9 = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
CX5 = CX9[:5]
CY5 = CY9[:5]
W5 = np.array([1 / 3] + [1 / 6] * 4)
CS2 = 1.0 / 3.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "printed_values.txt")

# a quiet lattice: no droplet, no ions, no field (used by several pins)
QUIET = dict(R=-100.0, k_d=0.0, k_r=0.0, c0=0.0, onsager_form=2, Kq=0.0,
             eps_r=1.0, psi_anode=0.0, psi_cathode=0.0, freeze_E=1,
             sweeps_min=0, sweeps_max=0, init_sweeps_fixed=0)


# ---- P1: moment matrices (Eq. 28, Eq. 46) ---------------------------------

def _inv1d(c):
    # 1D basis {1, c, c^2} on velocities {0, 1, -1}: rows of the inverse
    return {0: (1.0, 0.0, -1.0), 1: (0.0, 0.5, 0.5), -1: (0.0, -0.5, 0.5)}[c]


def test_p1_matrices_are_the_natural_moment_basis_and_invert():
    M, Mi, N, Ni = O.matrices()
    mono9 = [(0, 0), (1, 0), (0, 1), (2, 0), (0, 2), (1, 1), (1, 2), (2, 1), (2, 2)]
    Mt = np.array([[cx**a * cy**b for cx, cy in zip(CX9, CY9)] for a, b in mono9], float)
    assert np.array_equal(M, Mt)
    # tensor-product closed form of the inverse: Minv[i, (a,b)] = psi_a(cx_i) psi_b(cy_i)
    Mit = np.array([[_inv1d(cx)[a] * _inv1d(cy)[b] for (a, b) in mono9]
                    for cx, cy in zip(CX9, CY9)])
    np.testing.assert_allclose(Mi, Mit, rtol=0, atol=1e-15)
    np.testing.assert_allclose(M @ Mi, np.eye(9), rtol=0, atol=1e-15)
    mono5 = [(0, 0), (1, 0), (0, 1), (2, 0), (0, 2)]
    Nt = np.array([[cx**a * cy**b for cx, cy in zip(CX5, CY5)] for a, b in mono5], float)
    assert np.array_equal(N, Nt)
    # D2Q5: g0 = m0 - m3 - m4, g(+-1,0) = (m3 +- m1)/2, g(0,+-1) = (m4 +- m2)/2
    Nit = np.array([[1, 0, 0, -1, -1], [0, .5, 0, .5, 0], [0, 0, .5, 0, .5],
                    [0, -.5, 0, .5, 0], [0, 0, -.5, 0, .5]])
    np.testing.assert_allclose(Ni, Nit, rtol=0, atol=1e-15)


# ---- P2: equilibria (Eq. 31, 38, 45, 52-53, 57) ----------------------------

def test_p2_equilibrium_moments():
    rng = np.random.default_rng(2)
    for _ in range(25):
        p, rho = rng.uniform(-1e-2, 1e-2), rng.uniform(0.5, 2.0)
        ux, uy = rng.uniform(-0.1, 0.1, 2)
        fe = O.feq(p, rho, ux, uy)
        # zero-mass incompressible form: sum f_eq = 0, first moment rho u,
        # momentum flux p I + rho u u
        assert abs(fe.sum()) < 1e-15
        np.testing.assert_allclose([CX9 @ fe, CY9 @ fe], [rho * ux, rho * uy], atol=1e-15)
        np.testing.assert_allclose(
            [(CX9**2) @ fe, (CY9**2) @ fe, (CX9 * CY9) @ fe],
            [p + rho * ux * ux, p + rho * uy * uy, rho * ux * uy], atol=1e-15)
        # Eq. 57 returns p from f_eq (grad rho = 0): sum_{i>0} f_eq = (1-w0) p/cs2 - rho r_0
        r0 = -W9[0] * (ux * ux + uy * uy) / (2 * CS2)
        p_back = CS2 / (1 - W9[0]) * (fe[1:].sum() + rho * r0)
        assert abs(p_back - p) < 1e-15
        phi = rng.uniform(0, 1)
        he = O.heq(phi, ux, uy)
        np.testing.assert_allclose(
            [he.sum(), CX9 @ he, CY9 @ he, (CX9**2) @ he, (CX9 * CY9) @ he],
            [phi, phi * ux, phi * uy, phi * CS2, 0.0], atol=1e-15)
        c = rng.uniform(0, 2)
        ie = O.ion_eq(c, ux, uy)
        np.testing.assert_allclose([ie.sum(), CX5 @ ie, CY5 @ ie],
                                   [c, c * ux, c * uy], atol=1e-15)
        psi = rng.uniform(-2, 2)
        ge = O.geq(psi)
        assert abs(ge.sum()) < 1e-15
        assert abs(ge[1:].sum() / (1 - W5[0]) - psi) < 1e-15   # Eq. 49


# ---- P3: MRT with one rate is BGK -------------------------------------------

def test_p3_uniform_rates_reduce_to_bgk():
    rng = np.random.default_rng(3)
    for Q in (9, 5):
        for _ in range(20):
            tau = rng.uniform(0.51, 2.0)
            x, xeq, src = (rng.normal(size=Q) for _ in range(3))
            out = O.mrt(np.full(Q, 1 / tau), x, xeq, src)
            ref = x - (x - xeq) / tau + (1 - 1 / (2 * tau)) * src
            np.testing.assert_allclose(out, ref, rtol=0, atol=1e-14)


# ---- P4: conserved-moment sources, independent of the free rates -------------

def test_p4_momentum_and_ion_sources_exact_for_any_rates():
    rng = np.random.default_rng(4)
    for _ in range(25):
        f = rng.normal(scale=1e-2, size=9)
        F = rng.normal(scale=1e-3, size=2)
        gr = rng.normal(scale=1e-2, size=2)
        rho, p = rng.uniform(0.5, 2), rng.normal(scale=1e-3)
        ux, uy = (np.array([CX9 @ f, CY9 @ f]) + 0.5 * F) / rho    # Eq. 56
        fe = O.feq(p, rho, ux, uy)
        Fi = O.forcing_f(ux, uy, F[0], F[1], gr[0], gr[1])
        # the forcing term carries exactly the force in its first moment
        np.testing.assert_allclose([CX9 @ Fi, CY9 @ Fi], F, atol=1e-16)
        # zeroth and second moments of Eq. 54 in closed form (isotropy of the
        # weights): sum F_i = u.grad rho, sum c_a c_b F_i = cs2 [(u.grad rho)
        # delta_ab + u_a d_b rho + u_b d_a rho]
        ugr = ux * gr[0] + uy * gr[1]
        cs2 = 1.0 / 3.0
        assert abs(Fi.sum() - ugr) < 1e-17
        np.testing.assert_allclose([CX9 * CX9 @ Fi, CY9 * CY9 @ Fi, CX9 * CY9 @ Fi],
                                   [cs2 * (ugr + 2 * ux * gr[0]), cs2 * (ugr + 2 * uy * gr[1]),
                                    cs2 * (ux * gr[1] + uy * gr[0])], atol=1e-17)
        out = O.mrt(rng.uniform(0.2, 1.9, 9), f, fe, Fi)
        np.testing.assert_allclose([CX9 @ out, CY9 @ out],
                                   [CX9 @ f + F[0], CY9 @ f + F[1]], atol=1e-15)
        # ions: with c = sum p + R/2 (Eq. 41) the zeroth moment gains exactly R
        pp = rng.uniform(0, 0.5, 5)
        R = rng.normal(scale=0.1)
        c = pp.sum() + 0.5 * R
        out5 = O.mrt(rng.uniform(0.2, 1.9, 5), pp, O.ion_eq(c, ux, uy), W5 * R)
        assert abs(out5.sum() - (pp.sum() + R)) < 1e-15
        # Allen-Cahn: phi = sum h is conserved by the collision
        h = rng.uniform(0, 0.3, 9)
        phi = h.sum()
        Hs = O.Hsrc(phi, 4.0, *rng.normal(scale=1e-3, size=2), *rng.normal(size=2))
        outh = O.mrt(rng.uniform(0.2, 1.9, 9), h, O.heq(phi, ux, uy), Hs)
        assert abs(outh.sum() - phi) < 1e-15


def test_p14_pressure_of_eq57_round_trips_with_forcing():
    # f = f_eq(p, rho, u) - F_i / 2 are the populations whose Eq. 56 velocity
    # is u; Eq. 57 must return p for any grad rho (its 1/2 u.grad rho term
    # cancels the half forcing of the non-rest populations)
    rng = np.random.default_rng(14)
    for _ in range(25):
        p, rho = rng.normal(scale=1e-3), rng.uniform(0.5, 2)
        ux, uy = rng.normal(scale=1e-2, size=2)
        Fx, Fy = rng.normal(scale=1e-3, size=2)
        grx, gry = rng.normal(scale=1e-1, size=2)
        f = O.feq(p, rho, ux, uy) - 0.5 * O.forcing_f(ux, uy, Fx, Fy, grx, gry)
        np.testing.assert_allclose((np.array([CX9 @ f, CY9 @ f]) + 0.5 * np.array([Fx, Fy])) / rho,
                                   [ux, uy], atol=1e-16)
        assert abs(O.pressure(f, rho, ux, uy, grx, gry) - p) < 1e-16


@pytest.mark.parametrize("q", [5, 9])
def test_p15_ion_sources_carry_R_and_c_F(q):
    # Eq. 39 and the reaction term: sum_i = R, sum_i c_i = c F (L term on),
    # 0 (L term off), on D2Q5 and D2Q9
    cx, cy = (CX9, CY9) if q == 9 else (CX9[:5], CY9[:5])
    rng = np.random.default_rng(15)
    for _ in range(25):
        R, c = rng.normal(scale=1e-2), rng.uniform(0.1, 2)
        Fx, Fy = rng.normal(scale=1e-3, size=2)
        on, off = O.ion_src(R, c, Fx, Fy, 1, q), O.ion_src(R, c, Fx, Fy, 0, q)
        assert abs(on.sum() - R) < 1e-17 and abs(off.sum() - R) < 1e-17
        np.testing.assert_allclose([cx @ on, cy @ on], [c * Fx, c * Fy], atol=1e-18)
        np.testing.assert_allclose([cx @ off, cy @ off], [0.0, 0.0], atol=1e-18)


# ---- P5: isotropic stencils (Eq. 59 and the Laplacian) ---------------------

def test_p5_stencil_exact_on_low_degree_polynomials():
    ny, nx = 10, 12
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    inner = (slice(1, ny - 1), slice(1, nx - 1))
    rng = np.random.default_rng(5)
    a = rng.normal(size=10)
    chi = (a[0] + a[1] * x + a[2] * y + a[3] * x * x + a[4] * x * y + a[5] * y * y)
    gx, gy, lap = O.stencil(chi)
    np.testing.assert_allclose(gx[inner], (a[1] + 2 * a[3] * x + a[4] * y)[inner], atol=1e-11)
    np.testing.assert_allclose(gy[inner], (a[2] + a[4] * x + 2 * a[5] * y)[inner], atol=1e-11)
    np.testing.assert_allclose(lap[inner], np.full((ny - 2, nx - 2), 2 * a[3] + 2 * a[5]), atol=1e-10)
    cub = a[6] * x**3 + a[7] * x * x * y + a[8] * x * y * y + a[9] * y**3
    _, _, lap3 = O.stencil(cub)
    ref3 = 6 * a[6] * x + 2 * a[7] * y + 2 * a[8] * x + 6 * a[9] * y
    np.testing.assert_allclose(lap3[inner], ref3[inner], atol=1e-9)


def test_p5_stencil_periodic_x_and_mirror_rows():
    ny, nx = 6, 16
    k = 2 * np.pi / nx
    x = np.arange(nx)
    chi = np.tile(np.sin(k * x), (ny, 1))
    gx, gy, _ = O.stencil(chi)
    # on a Fourier mode the gradient stencil returns sin(k) cos(kx) at every x,
    # including the periodic wrap
    np.testing.assert_allclose(gx, np.tile(np.sin(k) * np.cos(k * x), (ny, 1)), atol=1e-14)
    np.testing.assert_allclose(gy, 0.0, atol=1e-15)
    # a field linear in y: the ghost row below y = 0 mirrors row 0, so the
    # one-sided gradient there is half the slope
    chi = np.tile(np.arange(ny, dtype=float)[:, None], (1, nx))
    _, gy, _ = O.stencil(chi)
    np.testing.assert_allclose(gy[0], 0.5, atol=1e-15)
    np.testing.assert_allclose(gy[ny - 1], 0.5, atol=1e-15)
    np.testing.assert_allclose(gy[1:-1], 1.0, atol=1e-14)


# ---- P6: Onsager function -------------------------------------------------------

def test_p6_onsager_full_form_matches_bessel_i1():
    for b in np.logspace(-6, 1.3, 60):
        ref = special.i1(4 * b) / (2 * b)
        assert abs(O.onsager(b, 0) - ref) <= 1e-14 * ref, b
    assert O.onsager(0.0, 0) == 1.0
    for b in (1e-4, 1e-3):
        assert abs(O.onsager(b, 0) - (1 + 2 * b * b + 4 / 3 * b**4)) < 1e-15
    # the linear form of Eq. 6 is the first two series terms
    for b in (0.0, 0.3, 1.7):
        assert O.onsager(b, 1) == 1 + 2 * b * b


# ---- P7: implicit reaction (Eq. 41-43) --------------------------------------

def test_p7_reaction_satisfies_eq41_with_eq5():
    rng = np.random.default_rng(7)
    cases = [(rng.uniform(0, 3), rng.uniform(0, 3), rng.uniform(0.1, 5),
              rng.uniform(0.1, 5), rng.uniform(1, 3)) for _ in range(200)]
    cases += [(10.0, 0.0, 1.0, 1.0, 1.0), (0.0, 10.0, 1.0, 2.0, 1.5)]  # both branches
    for sp, sn, kd, kr, F in cases:
        cp, cm, R = O.reaction(sp, sn, kd, kr, F)
        assert cp >= 0.0 and cm >= 0.0
        # Eq. 41 with R = k_d F - k_r c+ c- (Eq. 5): the system the quadratic solves
        assert abs(R - (kd * F - kr * cp * cm)) <= 1e-14 * max(1.0, kd * F)
        assert abs(cp - (sp + 0.5 * R)) <= 1e-14 * max(1.0, cp)
        assert abs(cm - (sn + 0.5 * R)) <= 1e-14 * max(1.0, cm)
    # uniform n_eq = sqrt(k_d F / k_r) is a fixed point (R = 0)
    kd, kr, F = 1.3, 0.7, 1.9
    neq = np.sqrt(kd * F / kr)
    cp, cm, R = O.reaction(neq, neq, kd, kr, F)
    assert abs(cp - neq) < 1e-15 and abs(cm - neq) < 1e-15 and abs(R) < 1e-14


# ---- mapping of Sec. 3 pinned by the printed numbers ------------------------

def _golden():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        kv = dict(p.split("=") for p in parts[1:] if "=" in p)
        val = float([p for p in parts[1:] if "=" not in p][0])
        rows.append((parts[0], {k: float(v) for k, v in kv.items()}, val))
    return rows


def test_mapping_reproduces_printed_W0_and_beta():
    ny = 128
    for name, cond, val in _golden():
        d = cond["d_mm"]
        P = O.params_from_physical(128, ny, d, cond.get("dpsi_kV", 1.0), 0.5, 5.0)
        dpsi = cond.get("dpsi_kV", 1.0)
        if name == "W0":
            W0 = P["Kq"] * ny * ny / dpsi
            assert abs(W0 / val - 1) < 2e-5, (d, W0, val)
        else:
            beta = np.sqrt(P["onsager_cb"] ** 2 * P["Kq"] * ny)  # beta^2 = O W0
            assert abs(beta / val - 1) < 2e-4, (d, beta, val)


# ---- P8: conservation of sum phi --------------------------------------------

def test_p8_sum_phi_conserved_with_electrodes_and_walls():
    o = O.Oracle(32, 32, dict(xc=15.5, yc=15.5, R=8.0, Kq=5.6893 / 32**2,
                              sweeps_max=30, init_sweeps_max=20000))
    s0 = o.sum_phi()
    o.step(120)
    assert abs(o.sum_phi() - s0) <= 1e-13 * s0
    f = o.fields()
    # charge layers of the right sign: anions at the anode (bottom), cations
    # at the cathode (top)
    assert f["q"][0].mean() < -0.05 and f["q"][-1].mean() > 0.05


# ---- P9, P10: potential (Eq. 44-50) --------------------------------------------

def test_p9_linear_potential_between_electrodes():
    ny = 32
    o = O.Oracle(4, ny, dict(QUIET, freeze_E=0, psi_anode=1.0, psi_cathode=0.0,
                             init_psi_zero=1, init_sweeps_fixed=-1,
                             init_sweeps_max=400000, sweep_tol=1e-13))
    f = o.fields()
    j = np.arange(ny)
    ref = 1.0 - (j + 0.5) / ny
    np.testing.assert_allclose(f["psi"], np.tile(ref[:, None], (1, 4)), atol=1e-9)
    np.testing.assert_allclose(f["Ey"], 1.0 / ny, atol=1e-9)
    np.testing.assert_allclose(f["Ex"], 0.0, atol=1e-12)


def test_p9_initial_linear_potential_is_exact_at_t0_and_a_fixed_point():
    # The initial potential of the 2048^2 case (no initial sweeps): g at the
    # equilibrium of Eq. 45 for the linear psi between the electrodes plus the
    # first-order non-equilibrium part.  With that part Eq. 49 must return
    # psi_lin and Eq. 50 E = -grad psi_lin exactly at t = 0, before any sweep;
    # with q = 0 and a uniform eps the linear profile is the steady state of
    # Eq. 44 with the electrode anti-bounce-back, so sweeps must leave it
    # unchanged.  A wrong sign or factor of the non-equilibrium part gives a
    # wrong E at t = 0 and a state that the first sweep moves.
    nx, ny, pa, pc = 6, 20, 1.7, -0.3
    o = O.Oracle(nx, ny, dict(QUIET, freeze_E=0, eps_r=1.0, Kq=0.0, psi_anode=pa, psi_cathode=pc,
                              init_psi_zero=0, init_sweeps_fixed=0, sweeps_min=1, sweeps_max=1))
    lin = np.tile((pa + (pc - pa) * (np.arange(ny) + 0.5) / ny)[:, None], (1, nx))
    for steps in (0, 1, 5):
        o.step(steps)
        f = o.fields()
        np.testing.assert_allclose(f["psi"], lin, rtol=0, atol=1e-13)
        np.testing.assert_allclose(f["Ey"], (pa - pc) / ny, rtol=0, atol=1e-14)
        np.testing.assert_allclose(f["Ex"], 0.0, rtol=0, atol=1e-14)


def test_p9_field_is_minus_grad_psi_for_a_charge_wave():
    # q = cos(2 pi x / nx) between grounded electrodes: E from the populations
    # (Eq. 50) against the central differences of the same psi (Eq. 49); both
    # components nonzero, agreement to the second-order error of the lattice
    nx, ny, kq = 64, 24, 1e-3
    o = O.Oracle(nx, ny, dict(QUIET, freeze_E=0, Kq=kq, psi_anode=0.0, psi_cathode=0.0,
                              sweeps_min=1, sweeps_max=4000000, sweep_tol=1e-15))
    s = o.state()
    wave = np.cos(2 * np.pi * np.arange(nx) / nx)[None, :, None]
    s[:, :, 18:23] = W5 * (1.0 + 0.5 * wave)     # cations
    s[:, :, 23:28] = W5 * (1.0 - 0.5 * wave)     # anions: q = cos(k x)
    o.set_state(s)
    o.step(1)
    f = o.fields()
    psi, Ex, Ey = f["psi"], f["Ex"], f["Ey"]
    dx = -(np.roll(psi, -1, axis=1) - np.roll(psi, 1, axis=1)) / 2
    dy = -(psi[2:, :] - psi[:-2, :]) / 2
    inner = slice(2, ny - 2)
    assert np.max(np.abs(Ex)) > 0.1 * np.max(np.abs(Ey)) > 0
    assert np.max(np.abs(Ex[inner] - dx[inner])) < 2e-2 * np.max(np.abs(Ex))
    assert np.max(np.abs(Ey[inner] - dy[1:-1][:ny - 4])) < 2e-2 * np.max(np.abs(Ey))


def _parabola_error(ny, kq):
    o = O.Oracle(4, ny, dict(QUIET, freeze_E=0, Kq=kq, sweeps_min=1,
                             sweeps_max=4000000, sweep_tol=1e-14))
    s = o.state()
    s[:, :, 18:23] = W5          # cations with sum p = 1, no anions: q = 1
    o.set_state(s)
    o.step(1)
    f = o.fields()
    y = np.arange(ny)
    ref = 0.5 * kq * (y + 0.5) * (ny - 0.5 - y)
    Eref = kq * (y - (ny - 1) / 2)
    return (np.max(np.abs(f["psi"][:, 0] - ref)) / ref.max(),
            np.max(np.abs(f["Ey"][:, 0] - Eref)) / Eref.max())


def test_p9_uniform_charge_gives_the_poisson_parabola():
    # lap psi = -Kq q (Eq. 7 with eps = 1) between grounded half-way electrodes:
    # psi = Kq q (y + 1/2)(ny - 1/2 - y) / 2 and E = -psi'.  The source of
    # Eq. 44 carries the 1/(1 - w0) that makes its steady state this equation
    # (without it the parabola comes out 2/3 as high); the scheme is second
    # order, so the relative error must fall 4x per doubling of ny.
    e32, E32 = _parabola_error(32, 1e-3)
    e64, E64 = _parabola_error(64, 2.5e-4)
    assert e32 < 5e-3 and E32 < 1e-6, (e32, E32)
    assert e64 < e32 / 3.5, (e32, e64)


def _two_layer_error(ny, W, R, eps_r):
    yc = (ny - 1) / 2
    o = O.Oracle(4, ny, dict(QUIET, freeze_E=0, init_shape=1, W=W, R=R, yc=yc,
                             eps_r=eps_r, psi_anode=1.0, psi_cathode=0.0,
                             init_sweeps_fixed=-1, init_sweeps_max=2000000,
                             sweep_tol=1e-13))
    psi = o.fields()["psi"][:, 0]
    eps = lambda y: 1 + (eps_r - 1) * 0.5 * (1 + np.tanh(2 * (R - abs(y - yc)) / W))
    yy = np.linspace(-0.5, ny - 0.5, 200 * ny + 1)
    inv = 1.0 / eps(yy)
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (inv[1:] + inv[:-1]) * np.diff(yy))])
    ref = 1.0 - np.interp(np.arange(ny), yy, cum) / cum[-1]
    # bulk field ratio of the series capacitor: E_outside / E_inside = eps_r
    f = o.fields()
    Ey = f["Ey"][:, 0]
    return np.max(np.abs(psi - ref)), Ey[2] / Ey[int(yc)]


@pytest.mark.slow
def test_p10_two_layer_potential_converges_second_order():
    e1, ratio = _two_layer_error(64, 4.0, 16.0, 4.0)
    e2, _ = _two_layer_error(128, 8.0, 32.0, 4.0)
    assert e1 < 3e-3, e1
    assert e2 < e1 / 3.0, (e1, e2)
    assert abs(ratio - 4.0) < 0.1, ratio


# ---- P11: flat interface relaxes to the tanh profile (Eq. 1-2) -----------------

def _flat_interface_error(ny, W, R, steps):
    yc = (ny - 1) / 2
    o = O.Oracle(4, ny, dict(QUIET, init_shape=1, W=W, W_init=2 * W, R=R, yc=yc,
                             M_phi=0.05))
    o.step(steps)
    phi = o.fields()["phi"][:, 0]
    y = np.arange(ny)
    ref = 0.5 * (1 + np.tanh(2 * (R - np.abs(y - yc)) / W))
    return np.max(np.abs(phi - ref))


@pytest.mark.slow
def test_p11_flat_interface_relaxes_to_tanh():
    e1 = _flat_interface_error(48, 4.0, 12.0, 3000)
    e2 = _flat_interface_error(96, 8.0, 24.0, 9000)
    assert e1 < 1e-2, e1
    assert e2 < e1 / 3.0, (e1, e2)


def test_flat_interface_at_rest_has_no_pressure_bump():
    # With beta = 12 sigma / W and kappa = 3 sigma W / 2 (Eq. 13) the tanh
    # profile of width W makes mu of Eq. 12 vanish, so across a flat interface
    # at rest the pressure (Eq. 56-57) stays flat.  A mismatched pair leaves
    # p = f(phi) - kappa phi'^2 / 2 inside the interface, (beta / 16 -
    # 3 sigma / (4 W)) at phi = 1/2; the lattice's own residue is ~0.05 sigma / W.
    ny, W, sigma = 64, 6.0, 0.01
    o = O.Oracle(4, ny, dict(QUIET, sigma=sigma, W=W, init_shape=1, yc=(ny - 1) / 2, R=ny / 4, xc=1.5))
    o.step(400)
    f = o.fields()
    p, phi = f["p"][:, 0], f["phi"][:, 0]
    bulk = np.where(phi > 0.5, np.median(p[phi > 0.99]), np.median(p[phi < 0.01]))
    assert np.max(np.abs(p - bulk)) < 0.1 * sigma / W


# ---- P12: Laplace law (Eq. 12-13, 56-57) ---------------------------------------

@pytest.mark.slow
def test_p12_static_droplet_obeys_laplace_law():
    n, sigma = 48, 0.01
    invR, dp = [], []
    for R in (8.0, 10.0, 12.0, 14.0):
        o = O.Oracle(n, n, dict(QUIET, R=R, xc=(n - 1) / 2, yc=(n - 1) / 2, sigma=sigma))
        o.step(1500)
        f = o.fields()
        c = n // 2
        dp.append(f["p"][c - 1:c + 1, c - 1:c + 1].mean() - f["p"][n // 2, 1:3].mean())
        invR.append(1.0 / R)
        umax = np.max(np.hypot(f["ux"], f["uy"]))
        assert umax < 1e-4, umax
    slope = np.polyfit(invR, dp, 1)[0]
    assert abs(slope / sigma - 1) < 0.05, slope


# ---- P13: dissociation-recombination equilibrium (Eq. 5) ---------------------

@pytest.mark.parametrize("scale", [0.0, 2.0])
def test_p13_uniform_field_reaches_n_eq(scale):
    E0, cb = 0.3, 1.0
    o = O.Oracle(8, 8, dict(QUIET, onsager_form=0, k_d=1.0, k_r=1.0, onsager_cb=cb,
                            ion_bc=2, E_frozen_x=E0, c_init_scale=scale))
    o.step(200)
    f = o.fields()
    neq = np.sqrt(special.i1(4 * cb * np.sqrt(E0)) / (2 * cb * np.sqrt(E0)))
    np.testing.assert_allclose(f["cp"], neq, rtol=1e-12)
    np.testing.assert_allclose(f["cm"], neq, rtol=1e-12)


# ---- ion drift (Eq. 34-35, 40): sign and speed -------------------------------

def test_ion_drift_moves_the_centroid_at_mobility_times_field():
    nx, ny, E0, mu, m = 64, 4, 0.02, 1.0, 0.5
    o = O.Oracle(nx, ny, dict(QUIET, ion_bc=2, E_frozen_x=E0, mu_v=mu, m=m,
                              einstein_D=0))
    s = o.state()
    x = np.arange(nx)
    bump = np.exp(-0.5 * ((x - 24.0) / 3.0) ** 2)
    s[:, :, 18:23] += W5[None, None, :] * bump[None, :, None]   # cations
    s[:, :, 23:28] += W5[None, None, :] * bump[None, :, None]   # anions
    o.set_state(s)
    N = 200
    o.step(N)
    st = o.state()
    cp = st[:, :, 18:23].sum(-1).sum(0)
    cm = st[:, :, 23:28].sum(-1).sum(0)
    x0 = (bump * x).sum() / bump.sum()
    s_p = 1 / (0.5 + 0.01 / CS2)           # first-moment rate, Eq. 37
    lag = (1 - s_p) * (1 - (1 - s_p) ** N) / s_p
    assert abs((cp * x).sum() / cp.sum() - x0 - mu * E0 * (N - lag)) < 1e-8
    assert abs((cm * x).sum() / cm.sum() - x0 + m * mu * E0 * (N - lag)) < 1e-8


# ---- viscosity (Eq. 51, 55 and the viscous rates) ------------------------------

def test_shear_wave_decays_at_the_viscosity_of_tau_f():
    ny, tau = 32, 0.8
    o = O.Oracle(4, ny, dict(QUIET, tau_f=tau))
    s = o.state()
    y = np.arange(ny)
    k = np.pi / ny
    mode = np.cos(k * (y + 0.5 - ny / 2))     # zero at the half-way walls
    for j in range(ny):
        fe = O.feq(0.0, 1.0, 1e-3 * mode[j], 0.0)
        s[j, :, 0:9] = fe
    o.set_state(s)
    amp = []
    for n in (100, 400):
        o.step(n - o.t)
        ux = o.fields()["ux"][:, 0]
        amp.append(ux @ mode / (mode @ mode))
    nu = CS2 * (tau - 0.5)
    rate = -np.log(amp[1] / amp[0]) / 300
    assert abs(rate / (nu * k * k) - 1) < 0.01, (rate, nu * k * k)


def test_shear_wave_inside_the_drop_phase_decays_at_eta_over_rho():
    # phi = 1 everywhere with rho_r = 2, eta_r = 3 (Eq. 61): the local tau_f
    # of Eq. 55 gives the kinematic viscosity eta_v eta_r / rho_r
    ny, tau, rr, er = 32, 0.8, 2.0, 3.0
    o = O.Oracle(4, ny, dict(QUIET, tau_f=tau, rho_ratio=rr, eta_ratio=er))
    s = o.state()
    y = np.arange(ny)
    k = np.pi / ny
    mode = np.cos(k * (y + 0.5 - ny / 2))
    for j in range(ny):
        s[j, :, 0:9] = O.feq(0.0, rr, 1e-3 * mode[j], 0.0)
    s[:, :, 9:18] = W9                            # h at rest with phi = 1
    o.set_state(s)
    amp = []
    for n in (100, 400):
        o.step(n - o.t)
        ux = o.fields()["ux"][:, 0]
        amp.append(ux @ mode / (mode @ mode))
    nu = CS2 * (tau - 0.5) * er / rr
    rate = -np.log(amp[1] / amp[0]) / 300
    assert abs(rate / (nu * k * k) - 1) < 0.01, (rate, nu * k * k)


def test_flat_interface_translates_with_a_uniform_flow_along_it():
    # u = (U, 0), p = 0 and a flat layer phi(y) solve Eq. 10-11 exactly for any
    # rho(phi): the u grad(rho) terms of Eq. 54 keep the lattice on it.  The
    # no-slip electrodes slow the flow only within a few sqrt(nu t) of the
    # walls, so the middle half of the channel is checked after 20 steps.
    nx, ny, U, rr, W = 4, 64, 0.02, 2.0, 8.0
    o = O.Oracle(nx, ny, dict(QUIET, tau_f=0.8, rho_ratio=rr, eta_ratio=3.0, W=W))
    s = o.state()
    y = np.arange(ny)
    phi = 0.5 * (1.0 + np.tanh(2.0 * (y - (ny - 1) / 2) / W))
    for j in range(ny):
        s[j, :, 0:9] = O.feq(0.0, 1.0 + (rr - 1.0) * phi[j], U, 0.0)
        s[j, :, 9:18] = O.heq(phi[j], U, 0.0)
        s[j, :, 33] = phi[j] * U                  # (phi u) of the previous step
        s[j, :, 34] = 0.0
    s[:, :, 18:28] = 0.0
    o.set_state(s)
    o.step(20)
    ux = o.fields()["ux"][ny // 4:3 * ny // 4]
    assert np.max(np.abs(ux - U)) < 5e-3 * U


# ---- polarization force (Eq. 14) on a flat dielectric layer ---------------------

@pytest.mark.slow
def test_polarization_force_sets_the_pressure_jump():
    # sign and factor 1/2 of the polarization force: at rest, dp/dy balances
    # -1/2 E^2 deps/dy with E = D / eps, so the pressure inside a dielectric
    # layer differs from outside by D^2 (1/eps_r - 1) / 2 (no surface tension;
    # tau_f = 2 damps the acoustic sloshing of the 1D column)
    ny, eps_r = 64, 4.0
    yc = (ny - 1) / 2
    o = O.Oracle(4, ny, dict(QUIET, freeze_E=0, init_shape=1, R=16.0, W=4.0, yc=yc,
                             sigma=0.0, tau_f=2.0, eps_r=eps_r, psi_anode=1.0,
                             init_sweeps_fixed=-1, init_sweeps_max=4000000,
                             sweep_tol=1e-13))
    o.step(4000)
    f = o.fields()
    psi = f["psi"][:, 0]
    D = (psi[2] - psi[6]) / 4.0       # displacement from the outer potential drop
    p = f["p"][:, 0]
    jump = p[int(yc)] - 0.5 * (p[4] + p[ny - 5])
    ref = 0.5 * D * D * (1 / eps_r - 1)
    assert abs(jump / ref - 1) < 0.03, (jump, ref)
    assert np.max(np.abs(f["uy"])) < 1e-6


def test_polarization_force_across_a_tangential_field():
    # the x part of -1/2 |E|^2 grad eps: a dielectric slab |x - xc| < R in a
    # frozen field E0 along y (tangential to its faces) comes to rest with a
    # pressure inside lower by E0^2 (eps_r - 1) / 2 (no surface tension, no
    # charge force; tau_f = 2 damps the acoustic sloshing)
    nx, ny, eps_r, E0, R = 64, 4, 4.0, 0.1, 16.0
    xc = (nx - 1) / 2
    o = O.Oracle(nx, ny, dict(QUIET, freeze_E=1, E_frozen_x=0.0, E_frozen_y=E0, sigma=0.0, tau_f=2.0,
                              eps_r=eps_r, Kq=0.0, W=6.0))
    s = o.state()
    x = np.arange(nx)
    phi = 0.5 * (1.0 + np.tanh(2.0 * (R - np.abs(x - xc)) / 6.0))
    s[:, :, 9:18] = W9[None, None, :] * phi[None, :, None]     # h at rest: w_i phi
    s[:, :, 0:9] = 0.0
    s[:, :, 33:35] = 0.0
    o.set_state(s)
    o.step(4000)
    f = o.fields()
    pr = f["p"][ny // 2]
    jump = pr[int(xc)] - 0.5 * (pr[4] + pr[nx - 5])
    ref = -0.5 * E0 * E0 * (eps_r - 1.0)
    assert abs(jump / ref - 1) < 0.03, (jump, ref)
    assert np.max(np.abs(f["ux"])) < 1e-6


# ---- Coulomb force (Eq. 14) in a 1D column with heterocharge layers ----------

@pytest.mark.slow
def test_coulomb_force_balances_the_pressure_gradient():
    # no droplet, uniform eps: once the ions have formed their layers at the
    # electrodes the column is at rest and dp/dy = Kq q E_y (Eq. 11, 14)
    ny = 32
    kq = 4 * 5.6893 / ny**2
    o = O.Oracle(4, ny, dict(R=-100.0, Kq=kq, eps_r=1.0, tau_f=2.0, sweeps_min=1,
                             sweeps_max=100, sweep_tol=1e-11, init_sweeps_max=400000))
    o.step(1000)
    f = o.fields()
    p = f["p"][:, 0]
    F = kq * f["q"][:, 0] * f["Ey"][:, 0]
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (F[1:] + F[:-1]))])
    assert np.max(np.abs(cum)) > 1e-4          # the layers carry a real force
    err = np.max(np.abs((p - p[0]) - cum)) / np.max(np.abs(cum))
    assert err < 2e-3, err


# ---- the interface normal of Eq. 32 and the conditioning of the step -----------

def test_regularised_normal_is_the_unit_normal_away_from_flat_regions():
    # with n = grad phi / sqrt(|grad phi|^2 + eps^2) the source of Eq. 32 differs
    # from the printed unit normal by the factor |g| / sqrt(|g|^2 + eps^2)
    rng = np.random.default_rng(11)
    eps = 1e-3
    for _ in range(20):
        g = rng.normal(size=2) * 0.2
        phi = rng.uniform(0.05, 0.95)
        a = O.Hsrc(phi, 4.0, 0.0, 0.0, g[0], g[1], 0.0)
        b = O.Hsrc(phi, 4.0, 0.0, 0.0, g[0], g[1], eps)
        m = np.hypot(*g)
        np.testing.assert_allclose(b, a * m / np.sqrt(m * m + eps * eps), rtol=1e-14, atol=1e-18)
    # flat region: the source vanishes with the gradient instead of keeping |lambda|
    b = O.Hsrc(1.0001, 4.0, 0.0, 0.0, 1e-10, -2e-10, eps)
    assert np.max(np.abs(b)) < 1e-10


@pytest.mark.slow
def test_step_is_well_conditioned_with_the_regularised_normal():
    # a 1e-16 relative perturbation of h must stay at round-off over 300 steps
    # of the 64x64 droplet (with the printed normal it grows ~e-fold every 10
    # steps inside the droplet, where phi overshoots 1 and grad phi ~ 0)
    from paper_2501_04920_gb300 import workloads
    prm = workloads.droplet64()
    growth = {}
    for eps in (1e-3, 0.0):
        prm["nhat_eps"] = eps
        a, b = O.Oracle(64, 64, prm), O.Oracle(64, 64, prm)
        s = b.state()
        rng = np.random.default_rng(0)
        s[:, :, 9:18] *= 1 + 1e-16 * rng.standard_normal(s[:, :, 9:18].shape)
        b.set_state(s)
        counts, _, _ = a.step(300)
        b.step(300, forced=counts)
        growth[eps] = np.max(np.abs(a.fields()["phi"] - b.fields()["phi"]))
    assert growth[1e-3] < 1e-13, growth
    assert growth[0.0] > 1e3 * growth[1e-3], growth


# ---- deformation factor (Eq. 63) ------------------------------------------------

def test_deformation_sampler_is_exact_for_bilinear_fields():
    # the extents of Eq. 63 sample phi by bilinear interpolation: exact for
    # a + b x + c y + d x y at any interior point (x, y not on the periodic seam)
    ny, nx = 24, 32
    yy, xx = np.mgrid[0:ny, 0:nx].astype(float)
    rng = np.random.default_rng(63)
    a, b, c, d = rng.normal(size=4)
    phi = a + b * xx + c * yy + d * xx * yy
    for _ in range(50):
        x, y = rng.uniform(0, nx - 1), rng.uniform(0, ny - 1)
        assert abs(O.sample(phi, x, y) - (a + b * x + c * y + d * x * y)) < 1e-12


def test_deformation_factor_of_ellipses():
    n = 96
    y, x = np.mgrid[0:n, 0:n].astype(float)
    for a, b in ((20.0, 20.0), (24.0, 16.0), (15.0, 22.0)):   # a along y, b along x
        r = np.sqrt(((x - 47.5) / b) ** 2 + ((y - 47.5) / a) ** 2)
        phi = 0.5 * (1 + np.tanh(2 * (1 - r) * min(a, b) / 4.0))
        assert abs(O.deformation(phi) - (a - b) / (a + b)) < 2e-3


# ---- side walls (Eq. 64, "the other boundaries") ------------------------------------

def test_side_wall_stencil_mirrors_the_ghost_columns():
    # Eq. 59 with ghost columns equal to the first / last column: exact at a
    # wall for a quadratic that is even about that wall (x = -1/2, nx - 1/2)
    nx, ny = 12, 6
    x = np.arange(nx)[None, :] * np.ones((ny, 1))
    for chi, col, d1, d2 in (((x + 0.5) ** 2, 0, 1.0, 2.0),
                             ((x - nx + 0.5) ** 2, nx - 1, -1.0, 2.0)):
        gx, gy, lap = O.stencil(chi, side_walls=1)
        np.testing.assert_allclose(gx[:, col], d1, atol=1e-12)
        np.testing.assert_allclose(lap[:, col], d2, atol=1e-12)
        np.testing.assert_allclose(gy, 0.0, atol=1e-12)
    # the periodic stencil sees the other side of the lattice instead
    gx, _, _ = O.stencil((x + 0.5) ** 2, side_walls=0)
    assert abs(gx[0, 0] - 1.0) > 1.0


def test_side_walls_potential_equals_the_mirrored_periodic_lattice():
    # D2Q5 bounce-back at a side wall is a mirror for the potential: a
    # droplet centred on the right wall of an nx-wide walled lattice has the
    # initial potential of the 2 nx-wide periodic lattice whose droplet sits
    # at the same place (it is even about x = -1/2 and x = nx - 1/2)
    nx, ny = 12, 16
    base = dict(QUIET, freeze_E=0, psi_anode=1.0, psi_cathode=0.0, eps_r=4.0,
                R=5.0, yc=(ny - 1) / 2, xc=nx - 0.5, init_sweeps_fixed=400)
    walled = O.Oracle(nx, ny, dict(base, side_walls=1)).fields()
    periodic = O.Oracle(2 * nx, ny, dict(base, side_walls=0)).fields()
    for k in ("psi", "Ex", "Ey", "phi"):
        np.testing.assert_allclose(walled[k], periodic[k][:, :nx], rtol=0, atol=1e-13, err_msg=k)
    # and it is not the periodic nx-wide answer
    per_nx = O.Oracle(nx, ny, dict(base, side_walls=0)).fields()
    assert np.max(np.abs(per_nx["Ex"] - walled["Ex"])) > 1e-4


def test_side_walls_and_electrode_walls_act_alike_on_the_fluid():
    # with no field and no ions, f and h see four bounce-back walls: a
    # droplet on the diagonal of a square box evolves symmetric under x <-> y
    n = 24
    o = O.Oracle(n, n, dict(QUIET, side_walls=1, xc=8.3, yc=8.3, R=5.0, sigma=0.02))
    o.step(60)
    f = o.fields()
    scale = np.max(np.hypot(f["ux"], f["uy"]))
    assert scale > 1e-6                         # the droplet does move
    np.testing.assert_allclose(f["phi"], f["phi"].T, rtol=0, atol=1e-13)
    np.testing.assert_allclose(f["ux"], f["uy"].T, rtol=0, atol=1e-13 * max(1.0, scale))
    np.testing.assert_allclose(f["p"], f["p"].T, rtol=0, atol=1e-13)


def test_side_walls_keep_a_centred_case_mirror_symmetric_and_conserve_phi():
    nx, ny = 20, 24
    prm = dict(side_walls=1, xc=(nx - 1) / 2, yc=9.0, R=5.0, Kq=5.6893 / ny**2,
               eps_r=3.0, mu_r=2.0, sweeps_min=40, sweeps_max=40, init_sweeps_fixed=300)
    o = O.Oracle(nx, ny, prm)
    s0 = o.sum_phi()
    o.step(80)
    f = o.fields()
    assert abs(o.sum_phi() - s0) <= 1e-13 * s0
    for k, sign in (("phi", 1), ("psi", 1), ("q", 1), ("cp", 1), ("uy", 1), ("Ey", 1),
                    ("ux", -1), ("Ex", -1)):
        a = f[k]
        np.testing.assert_allclose(a, sign * a[:, ::-1], rtol=0,
                                   atol=1e-12 * max(1e-12, np.max(np.abs(a))), err_msg=k)
    # no flux through the side walls: the wall columns do not leak ions
    assert np.max(np.abs(f["ux"])) > 0


# ---- ions on D2Q9 (Eq. 34-38 as printed, ion_lattice = 9) -------------------------------

def _ion_slices(q):
    return slice(18, 18 + q), slice(18 + q, 18 + 2 * q)


def _ion_state(o, q, cp_y, cm_y):
    # ions at rest in equilibrium, w_i c(y) for both species (p then n)
    s = o.state()
    w = W9 if q == 9 else W5
    s[:, :, 18:18 + q] = w[None, None, :] * cp_y[:, None, None]
    s[:, :, 18 + q:18 + 2 * q] = w[None, None, :] * cm_y[:, None, None]
    return s


@pytest.mark.parametrize("q", [5, 9])
def test_ions_decay_in_the_slowest_mode_between_absorbing_electrodes(q):
    # c = 0 at both half-way electrode walls (anti-bounce-back of Eq. 64):
    # sin(pi (y + 1/2) / ny) decays as exp(-D (pi / ny)^2 t), on D2Q5 and D2Q9
    nx, ny, steps, D = 4, 32, 4001, 0.01
    o = O.Oracle(nx, ny, dict(QUIET, ion_bc=1, ion_lattice=q, D=D))
    mode = np.sin(np.pi * (np.arange(ny) + 0.5) / ny)
    o.set_state(_ion_state(o, q, mode, 0.5 * mode))
    o.step(steps)
    t = steps - 1                      # the snapshot precedes the last streaming
    decay = np.exp(-D * (np.pi / ny) ** 2 * t)
    f = o.fields()
    np.testing.assert_allclose(f["cp"][:, 0] / mode, decay, rtol=3e-3)
    np.testing.assert_allclose(f["cm"][:, 0] / (0.5 * mode), decay, rtol=3e-3)


def test_ion_diffusivities_follow_the_mobilities_inside_the_drop_phase():
    # einstein_D (Sec. 2.2): D+ = D mu+ / mu_v and D- = D m mu+ / mu_v with
    # mu+ = mu_v (1 + (mu_r - 1) phi) (Eq. 61); in a uniform phi = 1 medium
    # with mu_r = 2, m = 1.5 the slowest mode between absorbing electrodes
    # decays at 2 D (pi/ny)^2 for cations and 3 D (pi/ny)^2 for anions
    nx, ny, steps, D = 4, 32, 2001, 0.01
    o = O.Oracle(nx, ny, dict(QUIET, ion_bc=1, D=D, mu_r=2.0, m=1.5, einstein_D=1))
    mode = np.sin(np.pi * (np.arange(ny) + 0.5) / ny)
    s = _ion_state(o, 5, mode, mode)
    s[:, :, 9:18] = W9[None, None, :]            # h at rest with phi = 1
    o.set_state(s)
    o.step(steps)
    t = steps - 1
    f = o.fields()
    np.testing.assert_allclose(f["phi"], 1.0, atol=1e-12)
    for key, scale in (("cp", 2.0), ("cm", 3.0)):
        decay = np.exp(-scale * D * (np.pi / ny) ** 2 * t)
        np.testing.assert_allclose(f[key][:, 0] / mode, decay, rtol=3e-3)


@pytest.mark.parametrize("q", [5, 9])
def test_uniform_ions_stay_uniform_at_zero_gradient_electrodes_and_side_walls(q):
    # Eq. 64: the attracted species takes the node's own value at its
    # electrode (anions at the anode below, cations at the cathode above) and
    # every species bounces back at the side walls; a uniform concentration
    # at rest is then stationary there, on D2Q5 and D2Q9 (populations move one
    # node per step, so after 5 streamings the repelled species' absorption at
    # the other electrode has not reached the rows checked)
    nx, ny, steps, c0 = 8, 24, 6, 0.7
    o = O.Oracle(nx, ny, dict(QUIET, ion_bc=0, ion_lattice=q, side_walls=1))
    o.set_state(_ion_state(o, q, np.full(ny, c0), np.full(ny, c0)))
    o.step(steps)
    f = o.fields()
    np.testing.assert_allclose(f["cm"][:ny - 8], c0, rtol=1e-13)
    np.testing.assert_allclose(f["cp"][8:], c0, rtol=1e-13)


def test_d2q9_ion_equilibrium_moments():
    c, ux, uy = 1.3, 0.02, -0.01
    e = O.ion_eq(c, ux, uy, q=9)
    assert abs(e.sum() - c) < 1e-15
    assert abs((CX9 * e).sum() - c * ux) < 1e-15 and abs((CY9 * e).sum() - c * uy) < 1e-15
    # the second moments of Eq. 38 on D2Q9 are those of D2Q5: c cs^2 along
    # each axis, no cross term
    assert abs((CX9**2 * e).sum() - c * CS2) < 1e-15 and abs((CX9 * CY9 * e).sum()) < 1e-15
    assert np.allclose(W9, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


@pytest.mark.parametrize("scale", [0.0, 2.0])
def test_d2q9_ions_reach_n_eq_in_a_uniform_field(scale):
    E0, cb = 0.3, 1.0
    o = O.Oracle(8, 8, dict(QUIET, ion_lattice=9, onsager_form=0, k_d=1.0, k_r=1.0, onsager_cb=cb,
                            ion_bc=2, E_frozen_x=E0, c_init_scale=scale))
    o.step(200)
    f = o.fields()
    neq = np.sqrt(special.i1(4 * cb * np.sqrt(E0)) / (2 * cb * np.sqrt(E0)))
    np.testing.assert_allclose(f["cp"], neq, rtol=1e-12)
    np.testing.assert_allclose(f["cm"], neq, rtol=1e-12)


def test_d2q9_and_d2q5_ions_share_centroid_and_spread_of_a_drifting_blob():
    # for a profile that varies along y only (x periodic), the cy moments of
    # Eq. 34-37 up to second order are the same on both lattices, and the
    # electrode bounce-back maps the cy = +1 group to the cy = -1 group on
    # both, so the mean and the variance of the blob evolve identically
    # (the mean at mu E, Eq. 40)
    nx, ny, E0 = 4, 64, 0.02
    y = np.arange(ny)
    bump = np.exp(-0.5 * ((y - 24.0) / 3.0) ** 2)
    moments = {}
    for q, w in ((5, W5), (9, W9)):
        o = O.Oracle(nx, ny, dict(QUIET, ion_lattice=q, ion_bc=2, E_frozen_y=E0, einstein_D=0))
        s = o.state()
        sp, sn = _ion_slices(q)
        s[:, :, sp] += w[None, None, :] * bump[:, None, None]
        o.set_state(s)
        o.step(150)
        st = o.state()
        cp = st[:, :, sp].sum(-1).sum(1)
        m0 = cp.sum()
        m1 = (cp * y).sum() / m0
        m2 = (cp * (y - m1) ** 2).sum() / m0
        moments[q] = (m0, m1, m2)
    for a, b in zip(moments[5], moments[9]):
        assert abs(a - b) <= 1e-11 * max(1.0, abs(a))
    assert moments[9][2] > 9.0 + 2 * 0.01 * 100      # it does spread (D = 0.01)


def test_d2q9_ions_conserved_between_zero_flux_electrodes():
    # ion_bc = 2 (bounce-back at both electrodes), no reaction: every
    # population, diagonal ones included, comes back at the wall
    o = O.Oracle(16, 12, dict(QUIET, ion_lattice=9, ion_bc=2, freeze_E=1, E_frozen_y=0.05,
                              E_frozen_x=0.01, k_d=0.0, k_r=0.0, c0=1.0, onsager_form=2))
    sp, sn = _ion_slices(9)
    s0 = o.state()
    m0 = s0[:, :, sp].sum()
    o.step(300)
    s1 = o.state()
    assert abs(s1[:, :, sp].sum() - m0) <= 1e-12 * m0
    f = o.fields()
    assert f["cp"][-1].mean() > f["cp"][0].mean()   # cations pile up downfield (E_y > 0)
