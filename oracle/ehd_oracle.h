/*
 * ehd_oracle.h -- plain FP64 CPU oracle of the phase-field lattice Boltzmann
 * method for two-phase EHD flow with Onsager-Wien dissociation (Zheng, Wang,
 * Xiong, Huang, Luo, arXiv 2501.04920).
 *
 * TEST INFRASTRUCTURE ONLY.  This header and ehd_oracle.c are the yardstick the
 * CUDA library is measured against.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load the oracle; the product library
 * neither includes, links nor calls anything here, and this file shares no code
 * with it.
 *
 * Lattice units throughout (dx = dt = 1, c = 1, cs^2 = 1/3).  Node (x, y),
 * x in [0, nx) periodic, y in [0, ny); the walls/electrodes sit half-way
 * between nodes: y = -1/2 is the anode (psi_anode), y = ny - 1/2 the cathode
 * (psi_cathode).
 *
 * Parity unpinned: the coupled long-run trajectory of the five equations has
 * no closed form; it is pinned only piecewise (tests/test_oracle_pins.py).
 */
#ifndef EHD_ORACLE_H
#define EHD_ORACLE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Problem parameters (lattice units).  Field meanings follow Sec. 2-4. */
typedef struct orc_params {
    /* incompressible NS, Eq. 51-57 and Eq. 61 */
    double tau_f;        /* relaxation time of the outer phase (phi = 0), Eq. 55 */
    double rho_ratio;    /* rho_l / rho_v, rho_v = 1 (Eq. 60) */
    double eta_ratio;    /* eta_l / eta_v (Eq. 60) */
    /* interface, Eq. 1-2, 12-13, 27-33 */
    double sigma;        /* surface tension zeta (Eq. 13) */
    double W;            /* interface thickness */
    double W_init;       /* width of the initial tanh profile (<= 0: W) */
    double M_phi;        /* Allen-Cahn mobility (Eq. 30) */
    double nhat_eps;     /* regularisation of the normal in Eq. 32 (0: none) */
    /* initial droplet / slab */
    double xc, yc, R;    /* centre and radius (slab: half-width) */
    int init_shape;      /* 0 disc, 1 horizontal slab |y - yc| < R */
    /* ions, Eq. 3-6 and 34-43 */
    double D;            /* ion diffusivity in the outer phase (Eq. 37) */
    double mu_v;         /* cation mobility in the outer phase */
    double mu_r;         /* mobility ratio mu_l / mu_v (Eq. 60) */
    double m;            /* mu_- / mu_+ (Eq. 23) */
    double k_d;          /* dissociation prefactor delta*c0^2 (Eq. 5) */
    double k_r;          /* recombination constant delta (Eq. 5) */
    double onsager_cb;   /* b = onsager_cb * sqrt(|E|) */
    int onsager_form;    /* 0: F = I1(4b)/(2b); 1: F = 1 + 2 b^2 (Eq. 6); 2: R = 0 */
    int ion_bc;          /* 0: Eq. 64; 1: c = 0 at both electrodes; 2: zero flux */
    int einstein_D;      /* 1: D_pm = D mu_pm / mu_v (Sec. 2.2) */
    int ion_L_term;      /* 1: keep the L_i source of Eq. 39 */
    double c_init_scale; /* initial c_pm = scale * n_eq */
    double c0;           /* initial c_pm when k_r = 0 or R = 0 */
    /* potential, Eq. 7-9 and 44-50 */
    double eps_r;        /* permittivity ratio eps_l / eps_v (Eq. 60) */
    double Kq;           /* charge coupling e0 c0 / eps_v in lattice units */
    double vartheta;     /* artificial diffusion of the potential LB (Eq. 47) */
    int psi_src_literal; /* 1: Eq. 44 source as printed; 0: divided by 1 - w0 */
    double psi_anode, psi_cathode;
    int sweeps_min, sweeps_max;   /* pseudo-time sweeps per step */
    double sweep_tol;             /* relative L2 change of psi per sweep */
    int init_sweeps_max;          /* cap of the initial potential solve */
    int init_sweeps_fixed;        /* >= 0: exactly this many initial sweeps */
    int init_psi_zero;            /* 1: start the potential from psi = 0 */
    int freeze_E;                 /* 1: skip the potential, use E_frozen */
    double E_frozen_x, E_frozen_y;
    /* collision */
    double s_free;       /* the free relaxation rates (1.0 in Sec. 6) */
    int bgk;             /* 1: every rate equals the hydrodynamic one */
    /* geometry */
    int ion_lattice;     /* 5: ions on D2Q5 with N (Eq. 46) and the weights of
                            Eq. 26 (the reading used by default); 9: on D2Q9
                            with M (Eq. 28) and the weights of Eq. 25, as
                            Eq. 34-36 print them */
    int side_walls;      /* 0: periodic x; 1: solid walls half-way left of
                            x = 0 and right of x = nx - 1 with the "other
                            boundaries" rules of Eq. 64: u = 0, zero normal
                            gradient of c+-, psi and phi (bounce-back of f, h,
                            p, n and g; mirrored ghost columns in Eq. 59) */
} orc_params;

/* Snapshot fields, row-major [field][ny][nx]. */
enum { ORC_PHI = 0, ORC_UX, ORC_UY, ORC_P, ORC_PSI, ORC_EX, ORC_EY,
       ORC_CP, ORC_CM, ORC_Q, ORC_NFIELDS };

typedef struct orc_ctx orc_ctx;

/* Lattice-wide driver.  orc_create returns NULL on invalid input. */
orc_ctx *orc_create(int nx, int ny, const orc_params *P);
void orc_destroy(orc_ctx *c);
/* Initial state (droplet, linear potential, potential solve, n_eq ions);
 * returns the number of initial sweeps taken. */
int orc_init(orc_ctx *c);
/* Advance nsteps; counts (nullable) receives the sweeps each step used,
 * resid (nullable) the last sweep residual of each step.  forced (nullable)
 * replays given sweep counts.  Returns the number of steps that hit the cap
 * without reaching sweep_tol. */
int orc_step(orc_ctx *c, int nsteps, const int *forced, int *counts, double *resid);
/* Copy the snapshot of the last step (time t of that step) into
 * out[ORC_NFIELDS * ny * nx]. */
void orc_get_fields(const orc_ctx *c, double *out);
/* Raw populations: f[9], h[9], p[5], n[5], g[5], phiu_prev[2] per node. */
/* State per node: f9 h9 p[Q] n[Q] g5 (phi u)2, Q = ion_lattice: 35 doubles
 * (Q = 5) or 43 (Q = 9). */
int orc_state_per_node(const orc_ctx *c);
void orc_get_state(const orc_ctx *c, double *out);
void orc_set_state(orc_ctx *c, const double *in);
double orc_sum_phi(const orc_ctx *c);   /* sum of phi = sum h over all nodes */
long orc_time(const orc_ctx *c);

/* Per-node building blocks, exported so that each can be pinned alone. */
void orc_matrices(double *M, double *Minv, double *N, double *Ninv);
void orc_feq(double p, double rho, double ux, double uy, double *out9);
void orc_forcing_f(double ux, double uy, double Fx, double Fy,
                   double grx, double gry, double *out9);
/* Eq. 57: pressure from the populations f9 (f0 unused), rho, u, grad rho. */
double orc_pressure(const double *f9, double rho, double ux, double uy, double grx, double gry);
/* Source of Eq. 34-35 on the Q-lattice (5 or 9): w_i R plus, with L_term,
 * L_i = w_i (c_i . F) c / cs2 of Eq. 39. */
void orc_ion_src(int Q, double R, double c, double Fx, double Fy, int L_term, double *outQ);
void orc_heq(double phi, double ux, double uy, double *out9);
void orc_Hsrc(double phi, double W, double dphiux, double dphiuy,
              double gx, double gy, double eps, double *out9);
void orc_ion_eq(double c, double ux, double uy, double *out5);
/* Eq. 38 on D2Q9 (weights of Eq. 25). */
void orc_ion_eq9(double c, double ux, double uy, double *out9);
void orc_geq(double psi, double *out5);
/* One MRT collision x* = x - Minv S M (x - xeq) + Minv (I - S/2) M src,
 * Q = 9 (matrix of Eq. 28) or 5 (Eq. 46). */
void orc_mrt(int Q, const double *s, const double *x, const double *xeq,
             const double *src, double *out);
double orc_onsager(double b, int form);
void orc_reaction(double sum_p, double sum_n, double k_d, double k_r, double F,
                  double *cp, double *cm, double *R);
/* Isotropic gradient and Laplacian (Eq. 59), mirrored ghost rows, x periodic. */
void orc_stencil(int nx, int ny, const double *chi, double *gx, double *gy,
                 double *lap);
/* The same with side walls (side_walls = 1): ghost columns mirror the
 * first and last column, as the ghost rows do. */
void orc_stencil_walls(int nx, int ny, int side_walls, const double *chi, double *gx,
                       double *gy, double *lap);
/* Physical -> lattice mapping of Sec. 3 (see the definition for the steps). */
void orc_params_from_physical(orc_params *P, int nx, int ny, double d_mm,
                              double dpsi_kV, double eps_r, double mu_r);
/* Deformation factor of Eq. 63 from a phi field [ny][nx]. */
/* phi at (x, y) by bilinear interpolation of the nodes (x periodic, rows
 * clamped at the walls), as Eq. 63's extents sample it. */
double orc_sample(int nx, int ny, const double *phi, double x, double y);
double orc_deformation(int nx, int ny, const double *phi);

#ifdef __cplusplus
}
#endif
#endif
