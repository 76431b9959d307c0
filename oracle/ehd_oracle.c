/*
 * ehd_oracle.c -- plain FP64 CPU oracle of the phase-field lattice Boltzmann
 * EHD method of arXiv 2501.04920 (Sec. 4): conservative Allen-Cahn (h, D2Q9),
 * cation/anion Nernst-Planck with Onsager-Wien dissociation (p, n, D2Q5),
 * Poisson potential in pseudo-time (g, D2Q5) and incompressible NS (f, D2Q9).
 *
 * TEST INFRASTRUCTURE ONLY: the yardstick for the CUDA library.  Only tests,
 * the smoke check and the CPU-baseline leg of the benchmark load it.  It is
 * slow on purpose: dense moment matrices as printed in Eq. 28 and Eq. 46,
 * every equation applied literally, one node at a time, in the order below.
 * The only parallelism is an optional OpenMP split of independent per-node
 * loops; every reduction is serial.
 *
 * One time step t -> t+1 (the paper lists the equations but not their order;
 * this is the order used here and by the GPU library):
 *   O1  phi = sum h (Eq. 33); properties by Eq. 61.
 *   O2  grad phi, lap phi (Eq. 59 and the Laplacian after it).
 *   O3  q = sum p - sum n (= c+ - c-, the R/2 terms of Eq. 41 cancel).
 *   O4  potential sweeps (Eq. 44-50) until the stop rule; then psi, E (Eq. 49-50).
 *   O5  Onsager F, implicit reaction (Eq. 42-43), R (Eq. 5).
 *   O6  forces (Eq. 12-14).   O7  u, p (Eq. 56-57) -> snapshot.
 *   O8  f collision (Eq. 51-55).  O9  h collision (Eq. 27-32, Eq. 58).
 *   O10 p, n collisions (Eq. 34-40).  O11 streaming with wall rules (Eq. 64).
 *
 * Readings of points the paper leaves open (all shared with the GPU library):
 *  - ions on D2Q5 with the matrix N of Eq. 46 and weights of Eq. 26
 *    (ion_lattice = 9: on D2Q9 with M and the weights of Eq. 25, as printed);
 *  - NS: the viscous rates are those of the second-order moments (rows 3-5 of
 *    Eq. 28) besides the s1 = s2 of Eq. 55; every other rate is s_free;
 *  - variable permittivity: the potential source is
 *    (Kq q - grad(eps) . E) / eps, i.e. Eq. 7 expanded, E from Eq. 50;
 *  - the source of Eq. 44 is divided by (1 - w0): as printed, Eq. 44 with
 *    psi from Eq. 49 relaxes to lap psi = -(1 - w0) rho_e / eps, a factor 2/3
 *    off Eq. 7 (psi_src_literal = 1 keeps the printed form);
 *  - G_i of Eq. 40 is w_i c_i . (mu c grad psi) / cs^2 for both species;
 *  - walls half-way between nodes; f, h bounce back; g anti-bounce-back to the
 *    electrode potential; ions: the species an electrode repels has c = 0
 *    there, the one it attracts has zero gradient (Eq. 64) -- both by
 *    anti-bounce-back, the latter with the wall value taken from the node;
 *  - sweep residual: ||psi^k - psi^(k-1)||_2 / ||psi^k||_2 over all nodes;
 *  - the normal of Eq. 32 is grad phi / sqrt(|grad phi|^2 + nhat_eps^2):
 *    printed as grad phi / |grad phi|, it has unbounded gain where phi
 *    overshoots 1 (lambda != 0) yet |grad phi| ~ 0, which makes the step
 *    chaotic at round-off level; nhat_eps = 0 keeps the printed form (with
 *    n_hat = 0 where |grad phi| < 1e-12);
 *  - (phi u)(t - 1) = 0 at t = 0.
 */
#include "ehd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* D2Q9 velocities and weights, Eq. 25 */
static const int cx9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int cy9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double w9[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                             1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int opp9[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
/* D2Q5 velocities and weights, Eq. 26 */
static const int cx5[5] = {0, 1, 0, -1, 0};
static const int cy5[5] = {0, 0, 1, 0, -1};
static const double w5[5] = {1.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0,
                             1.0 / 6.0};
static const int opp5[5] = {0, 3, 4, 1, 2};
static const double cs2 = 1.0 / 3.0;

/* Eq. 28, as printed */
static const double M9[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1}, {0, 1, 0, 1, 0, 1, 1, 1, 1},
    {0, 0, 1, 0, 1, 1, 1, 1, 1},    {0, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, 0, 0, 1, -1, -1, 1},  {0, 0, 0, 0, 0, 1, 1, -1, -1},
    {0, 0, 0, 0, 0, 1, 1, 1, 1}};
/* Eq. 46, as printed */
static const double N5[5][5] = {{1, 1, 1, 1, 1},
                                {0, 1, 0, -1, 0},
                                {0, 0, 1, 0, -1},
                                {0, 1, 0, 1, 0},
                                {0, 0, 1, 0, 1}};
static double M9inv[9][9];
static double N5inv[5][5];
static int inverses_ready = 0;

/* Gauss-Jordan inversion with partial pivoting of an n x n matrix. */
static void invert(int n, const double *A, double *Ainv)
{
    double a[9][18];
    for (int r = 0; r < n; ++r)
        for (int col = 0; col < 2 * n; ++col)
            a[r][col] = col < n ? A[r * n + col] : (col - n == r ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (piv != col)
            for (int k = 0; k < 2 * n; ++k) {
                double t = a[col][k];
                a[col][k] = a[piv][k];
                a[piv][k] = t;
            }
        double d = a[col][col];
        for (int k = 0; k < 2 * n; ++k) a[col][k] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double fct = a[r][col];
            for (int k = 0; k < 2 * n; ++k) a[r][k] -= fct * a[col][k];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int col = 0; col < n; ++col) Ainv[r * n + col] = a[r][n + col];
}

static void ensure_inverses(void)
{
    if (inverses_ready) return;
    invert(9, &M9[0][0], &M9inv[0][0]);
    invert(5, &N5[0][0], &N5inv[0][0]);
    inverses_ready = 1;
}

static const double *mat(int Q) { return Q == 9 ? &M9[0][0] : &N5[0][0]; }
static const double *matinv(int Q)
{
    return Q == 9 ? &M9inv[0][0] : &N5inv[0][0];
}

static void matvec(int Q, const double *A, const double *v, double *y)
{
    for (int r = 0; r < Q; ++r) {
        double s = 0.0;
        for (int col = 0; col < Q; ++col) s += A[r * Q + col] * v[col];
        y[r] = s;
    }
}

/* y = Minv diag(s) M v : the relaxation operator of Eq. 27/34/44/51 */
static void msm(int Q, const double *s, const double *v, double *y)
{
    double m[9];
    matvec(Q, mat(Q), v, m);
    for (int k = 0; k < Q; ++k) m[k] *= s[k];
    matvec(Q, matinv(Q), m, y);
}

/* y = Minv (I - diag(s)/2) M v : the source operator of Eq. 27/34/51 */
static void msm_half(int Q, const double *s, const double *v, double *y)
{
    double m[9];
    matvec(Q, mat(Q), v, m);
    for (int k = 0; k < Q; ++k) m[k] *= (1.0 - 0.5 * s[k]);
    matvec(Q, matinv(Q), m, y);
}

void orc_matrices(double *M, double *Minv, double *N, double *Ninv)
{
    ensure_inverses();
    memcpy(M, M9, sizeof M9);
    memcpy(Minv, M9inv, sizeof M9inv);
    memcpy(N, N5, sizeof N5);
    memcpy(Ninv, N5inv, sizeof N5inv);
}

void orc_mrt(int Q, const double *s, const double *x, const double *xeq,
             const double *src, double *out)
{
    ensure_inverses();
    double d[9], a[9], b[9];
    for (int i = 0; i < Q; ++i) d[i] = x[i] - xeq[i];
    msm(Q, s, d, a);
    msm_half(Q, s, src, b);
    for (int i = 0; i < Q; ++i) out[i] = x[i] - a[i] + b[i];
}

/* ---- equilibria and sources ------------------------------------------- */

/* r_i(u) of Eq. 53 */
static double r_u(int i, double ux, double uy)
{
    double cu = cx9[i] * ux + cy9[i] * uy;
    double uu = ux * ux + uy * uy;
    return w9[i] * (cu / cs2 + cu * cu / (2.0 * cs2 * cs2) - uu / (2.0 * cs2));
}

/* Eq. 52 */
void orc_feq(double p, double rho, double ux, double uy, double *out)
{
    for (int i = 0; i < 9; ++i) {
        double a = (i == 0) ? (w9[0] - 1.0) * p / cs2 : w9[i] * p / cs2;
        out[i] = a + rho * r_u(i, ux, uy);
    }
}

/* Eq. 54; (grx, gry) = grad rho */
void orc_forcing_f(double ux, double uy, double Fx, double Fy, double grx,
                   double gry, double *out)
{
    double ugr = ux * grx + uy * gry;
    for (int i = 0; i < 9; ++i) {
        double cF = cx9[i] * Fx + cy9[i] * Fy;
        double uc = ux * cx9[i] + uy * cy9[i];
        double gc = grx * cx9[i] + gry * cy9[i];
        /* u grad(rho) : (c c - cs2 I) = (u.c)(c.grad rho) - cs2 u.grad rho */
        double tens = uc * gc - cs2 * ugr;
        out[i] = w9[i] * (ugr + cF / cs2 + tens / cs2);
    }
}

/* Eq. 57: the pressure from the populations f (f0 not used), rho, u and
 * grad rho */
double orc_pressure(const double *f, double rho, double ux, double uy, double grx, double gry)
{
    double s_ne0 = 0.0;
    for (int i = 1; i < 9; ++i) s_ne0 += f[i];
    return cs2 / (1.0 - w9[0]) * (s_ne0 + 0.5 * (ux * grx + uy * gry) + rho * r_u(0, ux, uy));
}

/* Eq. 39 and the reaction source of Eq. 34-35 on the Q-lattice (5 or 9):
 * w_i R plus, with L_term, L_i = w_i (c_i . F) c / cs2 */
void orc_ion_src(int Q, double R, double c, double Fx, double Fy, int L_term, double *out)
{
    const int *cxq = Q == 9 ? cx9 : cx5, *cyq = Q == 9 ? cy9 : cy5;
    const double *wq = Q == 9 ? w9 : w5;
    for (int i = 0; i < Q; ++i) {
        double cF = cxq[i] * Fx + cyq[i] * Fy;
        out[i] = wq[i] * R + (L_term ? wq[i] * cF * c / cs2 : 0.0);
    }
}

/* Eq. 31 */
void orc_heq(double phi, double ux, double uy, double *out)
{
    for (int i = 0; i < 9; ++i)
        out[i] = w9[i] * phi * (1.0 + (cx9[i] * ux + cy9[i] * uy) / cs2);
}

/* Eq. 32 with lambda of Eq. 2; (gx, gy) = grad phi.  eps > 0: the normal is
 * grad phi / sqrt(|grad phi|^2 + eps^2); eps = 0: grad phi / |grad phi|, and
 * 0 where |grad phi| < 1e-12. */
void orc_Hsrc(double phi, double W, double dphiux, double dphiuy, double gx,
              double gy, double eps, double *out)
{
    double mag = sqrt(gx * gx + gy * gy);
    double nx = 0.0, ny = 0.0;
    if (eps > 0.0) {
        double den = sqrt(gx * gx + gy * gy + eps * eps);
        nx = gx / den;
        ny = gy / den;
    } else if (mag >= 1e-12) {
        nx = gx / mag;
        ny = gy / mag;
    }
    double lam = 4.0 * phi * (1.0 - phi) / W;
    double vx = dphiux + cs2 * lam * nx;
    double vy = dphiuy + cs2 * lam * ny;
    for (int i = 0; i < 9; ++i)
        out[i] = w9[i] * (cx9[i] * vx + cy9[i] * vy) / cs2;
}

/* Eq. 38 on D2Q5 */
void orc_ion_eq(double c, double ux, double uy, double *out)
{
    for (int i = 0; i < 5; ++i)
        out[i] = w5[i] * c * (1.0 + (cx5[i] * ux + cy5[i] * uy) / cs2);
}

void orc_ion_eq9(double c, double ux, double uy, double *out)
{
    for (int i = 0; i < 9; ++i)
        out[i] = w9[i] * c * (1.0 + (cx9[i] * ux + cy9[i] * uy) / cs2);
}

/* Eq. 38 on the ion lattice of the context (Q = 5 or 9). */
static void ion_eq(int Q, double c, double ux, double uy, double *out)
{
    if (Q == 9) orc_ion_eq9(c, ux, uy, out);
    else orc_ion_eq(c, ux, uy, out);
}

/* Eq. 45 */
void orc_geq(double psi, double *out)
{
    for (int i = 0; i < 5; ++i)
        out[i] = (i == 0) ? (w5[0] - 1.0) * psi : w5[i] * psi;
}

/* Onsager function.  Form 0: F(b) = I1(4b) / (2b) written out as the power
 * series of I1, I1(z) = sum_k (z/2)^(2k+1) / (k! (k+1)!), so that
 * F(b) = sum_k (4 b^2)^k / (k! (k+1)!), F(0) = 1.  Form 1: the linear Eq. 6
 * with b^2 standing for gamma E.  Form 2 (R = 0): 0. */
double orc_onsager(double b, int form)
{
    if (form == 1) return 1.0 + 2.0 * b * b;
    if (form == 2) return 0.0;
    double y = 4.0 * b * b;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 500; ++k) {
        term *= y / ((double)k * (double)(k + 1));
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return sum;
}

/* Eq. 42-43 with lambda0 = k_r / 2 (dt = 1) and delta c0^2 F = k_d F.  The
 * positive root of lambda0 c^2 + B c - cbar_+ = 0, B = 1 - lambda0 cbar_+ +
 * lambda0 cbar_-, taken in the form that does not cancel. */
void orc_reaction(double sum_p, double sum_n, double k_d, double k_r, double F,
                  double *cp, double *cm, double *R)
{
    double cbp = sum_p + 0.5 * k_d * F;
    double cbm = sum_n + 0.5 * k_d * F;
    double lam0 = 0.5 * k_r;
    double B = 1.0 - lam0 * cbp + lam0 * cbm;
    double disc = sqrt(B * B + 4.0 * lam0 * cbp);
    double c;
    if (B >= 0.0)
        c = (B + disc > 0.0) ? 2.0 * cbp / (B + disc) : 0.0;
    else
        c = (-B + disc) / (2.0 * lam0);
    *cp = c;
    *cm = c - cbp + cbm;
    *R = k_d * F - k_r * (*cp) * (*cm);
}

/* ---- lattice context ---------------------------------------------------- */

struct orc_ctx {
    int nx, ny;
    long nn;
    orc_params P;
    double tau_g;
    int qi;                         /* ion lattice: 5 or 9 */
    double *f, *h, *p, *n, *g;      /* post-streaming populations */
    double *fs, *hs, *ps, *ns, *gs; /* post-collision populations */
    double *phiu_prev;              /* (phi u)(t - 1), 2 per node */
    double *phi, *gpx, *gpy, *lap, *q, *psi_prev;
    double *cwb, *cwt;              /* wall values, per x */
    double *snap;                   /* ORC_NFIELDS x nn */
    long t;
};

static long idx(const orc_ctx *c, int x, int y) { return (long)y * c->nx + x; }
static int wrapx(const orc_ctx *c, int x)
{
    return (x % c->nx + c->nx) % c->nx;
}

void orc_stencil(int nx, int ny, const double *chi, double *gx, double *gy,
                 double *lap)
{
    orc_stencil_walls(nx, ny, 0, chi, gx, gy, lap);
}

void orc_stencil_walls(int nx, int ny, int side_walls, const double *chi, double *gx,
                       double *gy, double *lap)
{
#pragma omp parallel for
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double c0 = chi[(long)y * nx + x];
            double sx = 0.0, sy = 0.0, sl = 0.0;
            for (int i = 1; i < 9; ++i) {
                int xn = ((x + cx9[i]) % nx + nx) % nx;
                if (side_walls) {            /* mirror ghost column */
                    xn = x + cx9[i];
                    if (xn < 0) xn = 0;
                    if (xn >= nx) xn = nx - 1;
                }
                int yn = y + cy9[i];
                if (yn < 0) yn = 0;          /* mirror ghost row: zero normal */
                if (yn >= ny) yn = ny - 1;   /* gradient at the half-way wall  */
                double v = chi[(long)yn * nx + xn];
                sx += w9[i] * cx9[i] * v;
                sy += w9[i] * cy9[i] * v;
                sl += 2.0 * w9[i] * (v - c0);
            }
            gx[(long)y * nx + x] = sx / cs2;
            gy[(long)y * nx + x] = sy / cs2;
            lap[(long)y * nx + x] = sl / cs2;
        }
}

static double *alloc(long n)
{
    double *a = (double *)calloc((size_t)n, sizeof(double));
    return a;
}

orc_ctx *orc_create(int nx, int ny, const orc_params *P)
{
    if (nx < 4 || ny < 4 || !P) return NULL;
    ensure_inverses();
    orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
    if (!c) return NULL;
    c->nx = nx;
    c->ny = ny;
    c->nn = (long)nx * ny;
    c->P = *P;
    c->tau_g = 0.5 + P->vartheta / cs2; /* Eq. 47 */
    long nn = c->nn;
    c->f = alloc(9 * nn);
    c->h = alloc(9 * nn);
    c->qi = P->ion_lattice == 9 ? 9 : 5;
    c->p = alloc(9 * nn);
    c->n = alloc(9 * nn);
    c->g = alloc(5 * nn);
    c->fs = alloc(9 * nn);
    c->hs = alloc(9 * nn);
    c->ps = alloc(9 * nn);
    c->ns = alloc(9 * nn);
    c->gs = alloc(5 * nn);
    c->phiu_prev = alloc(2 * nn);
    c->phi = alloc(nn);
    c->gpx = alloc(nn);
    c->gpy = alloc(nn);
    c->lap = alloc(nn);
    c->q = alloc(nn);
    c->psi_prev = alloc(nn);
    c->cwb = alloc(nx);
    c->cwt = alloc(nx);
    c->snap = alloc(ORC_NFIELDS * nn);
    if (!c->f || !c->h || !c->p || !c->n || !c->g || !c->fs || !c->hs ||
        !c->ps || !c->ns || !c->gs || !c->phiu_prev || !c->phi || !c->gpx ||
        !c->gpy || !c->lap || !c->q || !c->psi_prev || !c->cwb || !c->cwt ||
        !c->snap) {
        orc_destroy(c);
        return NULL;
    }
    return c;
}

void orc_destroy(orc_ctx *c)
{
    if (!c) return;
    free(c->f); free(c->h); free(c->p); free(c->n); free(c->g);
    free(c->fs); free(c->hs); free(c->ps); free(c->ns); free(c->gs);
    free(c->phiu_prev); free(c->phi); free(c->gpx); free(c->gpy);
    free(c->lap); free(c->q); free(c->psi_prev); free(c->cwb); free(c->cwt);
    free(c->snap);
    free(c);
}

/* ---- streaming ----------------------------------------------------------- */

/* Pull-stream a D2Q9 field; a link that crosses a wall bounces back. */
static void stream9_bounce(const orc_ctx *c, const double *post, double *out)
{
    const int walls = c->P.side_walls;
#pragma omp parallel for
    for (int y = 0; y < c->ny; ++y)
        for (int x = 0; x < c->nx; ++x) {
            long k = idx(c, x, y);
            for (int i = 0; i < 9; ++i) {
                int sy = y - cy9[i], sx = x - cx9[i];
                if (sy < 0 || sy >= c->ny || (walls && (sx < 0 || sx >= c->nx)))
                    out[k * 9 + i] = post[k * 9 + opp9[i]];
                else
                    out[k * 9 + i] = post[idx(c, wrapx(c, x - cx9[i]), sy) * 9 + i];
            }
        }
}

/* Pull-stream a D2Q5 field.  A link crossing the bottom (top) wall takes
 * anti-bounce-back  out_i = -post_opp(i) + 2 w_i v_wall  when mode = 0, or
 * plain bounce-back out_i = post_opp(i) when mode = 1.  A link crossing a
 * side wall bounces back (zero normal gradient, Eq. 64). */
static void stream5(const orc_ctx *c, const double *post, double *out,
                    int mode_bot, const double *vbot, int mode_top,
                    const double *vtop)
{
    const int walls = c->P.side_walls;
#pragma omp parallel for
    for (int y = 0; y < c->ny; ++y)
        for (int x = 0; x < c->nx; ++x) {
            long k = idx(c, x, y);
            for (int i = 0; i < 5; ++i) {
                int sy = y - cy5[i], sx = x - cx5[i];
                if (walls && (sx < 0 || sx >= c->nx)) {
                    out[k * 5 + i] = post[k * 5 + opp5[i]];
                } else if (sy < 0 || sy >= c->ny) {
                    int bottom = sy < 0;
                    int mode = bottom ? mode_bot : mode_top;
                    double v = bottom ? vbot[x] : vtop[x];
                    double a = post[k * 5 + opp5[i]];
                    out[k * 5 + i] = mode == 0 ? -a + 2.0 * w5[i] * v : a;
                } else {
                    out[k * 5 + i] =
                        post[idx(c, wrapx(c, x - cx5[i]), sy) * 5 + i];
                }
            }
        }
}

/* Pull-stream a D2Q9 ion field: a link crossing the bottom (top) wall takes
 * anti-bounce-back out_i = -post_opp(i) + 2 w_i v_wall (mode 0) or
 * bounce-back (mode 1), as stream5 does; a link that crosses only a side
 * wall bounces back; a diagonal link through a corner takes the electrode's
 * rule. */
static void stream9_ion(const orc_ctx *c, const double *post, double *out,
                        int mode_bot, const double *vbot, int mode_top,
                        const double *vtop)
{
    const int walls = c->P.side_walls;
#pragma omp parallel for
    for (int y = 0; y < c->ny; ++y)
        for (int x = 0; x < c->nx; ++x) {
            long k = idx(c, x, y);
            for (int i = 0; i < 9; ++i) {
                int sy = y - cy9[i], sx = x - cx9[i];
                if (sy < 0 || sy >= c->ny) {
                    int bottom = sy < 0;
                    int mode = bottom ? mode_bot : mode_top;
                    double v = bottom ? vbot[x] : vtop[x];
                    double a = post[k * 9 + opp9[i]];
                    out[k * 9 + i] = mode == 0 ? -a + 2.0 * w9[i] * v : a;
                } else if (walls && (sx < 0 || sx >= c->nx)) {
                    out[k * 9 + i] = post[k * 9 + opp9[i]];
                } else {
                    out[k * 9 + i] = post[idx(c, wrapx(c, sx), sy) * 9 + i];
                }
            }
        }
}

/* Ion streaming on the context's lattice. */
static void stream_ion(const orc_ctx *c, const double *post, double *out,
                       int mode_bot, const double *vbot, int mode_top,
                       const double *vtop)
{
    if (c->qi == 9) stream9_ion(c, post, out, mode_bot, vbot, mode_top, vtop);
    else stream5(c, post, out, mode_bot, vbot, mode_top, vtop);
}

/* ---- potential (Eq. 44-50) --------------------------------------------- */

static double psi_of(const double *g) /* Eq. 49 */
{
    double s = 0.0;
    for (int i = 1; i < 5; ++i) s += g[i];
    return s / (1.0 - w5[0]);
}

static void E_of(const double *g, double tau_g, double *Ex, double *Ey) /* Eq. 50 */
{
    double sx = 0.0, sy = 0.0;
    for (int i = 0; i < 5; ++i) {
        sx += cx5[i] * g[i];
        sy += cy5[i] * g[i];
    }
    *Ex = sx / (cs2 * tau_g);
    *Ey = sy / (cs2 * tau_g);
}

static void rates5(const orc_params *P, double tau, double *s)
{
    for (int k = 0; k < 5; ++k) s[k] = P->bgk ? 1.0 / tau : P->s_free;
    s[1] = s[2] = 1.0 / tau;
}

/* Ion rates of Eq. 36-37 on Q = 5 or 9: the first moments (rows 1, 2 of N or
 * M) relax at 1/tau, the others at s_free (all at 1/tau with bgk). */
static void rates_ion(const orc_params *P, int Q, double tau, double *s)
{
    for (int k = 0; k < Q; ++k) s[k] = P->bgk ? 1.0 / tau : P->s_free;
    s[1] = s[2] = 1.0 / tau;
}

/* One pseudo-time sweep: collide every node (Eq. 44) then stream with
 * anti-bounce-back to the electrode potentials. */
static void potential_sweep(orc_ctx *c)
{
    const orc_params *P = &c->P;
    double s[5];
    rates5(P, c->tau_g, s);
#pragma omp parallel for
    for (long k = 0; k < c->nn; ++k) {
        const double *g = c->g + 5 * k;
        double phi = c->phi[k];
        double eps = 1.0 + (P->eps_r - 1.0) * phi;        /* Eq. 61 */
        double dex = (P->eps_r - 1.0) * c->gpx[k];
        double dey = (P->eps_r - 1.0) * c->gpy[k];
        double psi = psi_of(g);
        double Ex, Ey;
        E_of(g, c->tau_g, &Ex, &Ey);
        double rho_t = (P->Kq * c->q[k] - (dex * Ex + dey * Ey)) / eps;
        double geq[5], d[5], a[5];
        orc_geq(psi, geq);
        for (int i = 0; i < 5; ++i) d[i] = g[i] - geq[i];
        msm(5, s, d, a);
        /* Eq. 44 source; divided by (1 - w0) unless psi_src_literal, so that
         * the steady state of Eq. 44 with psi from Eq. 49 is Eq. 7 (summing
         * Eq. 44 over i != 0 leaves lap psi = -(1 - w0) * source / vartheta) */
        double norm = P->psi_src_literal ? 1.0 : 1.0 / (1.0 - w5[0]);
        for (int i = 0; i < 5; ++i)
            c->gs[5 * k + i] = g[i] - a[i] + w5[i] * rho_t * P->vartheta * norm;
    }
    for (int x = 0; x < c->nx; ++x) {
        c->cwb[x] = P->psi_anode;
        c->cwt[x] = P->psi_cathode;
    }
    stream5(c, c->gs, c->g, 0, c->cwb, 0, c->cwt);
}

/* Sweep until the stop rule: k >= kmin and (r_k < tol or k = kmax).  Returns
 * the number of sweeps; *resid receives r of the last sweep (NaN if none). */
static int potential_solve(orc_ctx *c, int kmin, int kmax, double tol,
                           double *resid)
{
    for (long k = 0; k < c->nn; ++k) c->psi_prev[k] = psi_of(c->g + 5 * k);
    double r = NAN;
    int it = 0;
    while (it < kmax) {
        potential_sweep(c);
        ++it;
        double sd = 0.0, sp = 0.0;
        for (long k = 0; k < c->nn; ++k) {
            double ps = psi_of(c->g + 5 * k);
            double d = ps - c->psi_prev[k];
            sd += d * d;
            sp += ps * ps;
            c->psi_prev[k] = ps;
        }
        r = sp > 0.0 ? sqrt(sd / sp) : sqrt(sd);
        if (it >= kmin && (r < tol || it >= kmax)) break;
    }
    if (resid) *resid = r;
    return it;
}

/* ---- initial state ------------------------------------------------------ */

static void macro_phi_q(orc_ctx *c)
{
#pragma omp parallel for
    for (long k = 0; k < c->nn; ++k) {
        double s = 0.0;
        for (int i = 0; i < 9; ++i) s += c->h[9 * k + i]; /* Eq. 33 */
        c->phi[k] = s;
        double sp = 0.0, sn = 0.0;
        for (int i = 0; i < c->qi; ++i) {
            sp += c->p[c->qi * k + i];
            sn += c->n[c->qi * k + i];
        }
        c->q[k] = sp - sn;
    }
    orc_stencil_walls(c->nx, c->ny, c->P.side_walls, c->phi, c->gpx, c->gpy, c->lap);
}

static double n_eq_of(const orc_params *P, double Emag)
{
    if (P->k_r > 0.0 && P->onsager_form != 2) {
        double b = P->onsager_cb * sqrt(Emag);
        return sqrt(P->k_d * orc_onsager(b, P->onsager_form) / P->k_r);
    }
    return P->c0;
}

int orc_init(orc_ctx *c)
{
    const orc_params *P = &c->P;
    double Wi = P->W_init > 0.0 ? P->W_init : P->W;
    double feq[9];
    orc_feq(0.0, 1.0, 0.0, 0.0, feq);
    for (int y = 0; y < c->ny; ++y)
        for (int x = 0; x < c->nx; ++x) {
            long k = idx(c, x, y);
            double r = P->init_shape == 1
                           ? fabs(y - P->yc)
                           : sqrt((x - P->xc) * (x - P->xc) +
                                  (y - P->yc) * (y - P->yc));
            double phi0 = 0.5 * (1.0 + tanh(2.0 * (P->R - r) / Wi));
            orc_heq(phi0, 0.0, 0.0, c->h + 9 * k);
            double rho = 1.0 + (P->rho_ratio - 1.0) * phi0;
            orc_feq(0.0, rho, 0.0, 0.0, c->f + 9 * k);
            for (int i = 0; i < c->qi; ++i) c->p[c->qi * k + i] = c->n[c->qi * k + i] = 0.0;
            c->phiu_prev[2 * k] = c->phiu_prev[2 * k + 1] = 0.0;
            /* potential: linear profile between the half-way electrodes with
             * the first-order non-equilibrium part that makes Eq. 50 return
             * E = -grad psi */
            double dpsi = (P->psi_cathode - P->psi_anode) / c->ny;
            double psil = P->psi_anode + dpsi * (y + 0.5);
            double *g = c->g + 5 * k;
            if (P->init_psi_zero) {
                for (int i = 0; i < 5; ++i) g[i] = 0.0;
            } else {
                orc_geq(psil, g);
                for (int i = 1; i < 5; ++i)
                    g[i] -= c->tau_g * w5[i] * cy5[i] * dpsi;
            }
        }
    macro_phi_q(c); /* phi = sum h; q = 0 */
    int sweeps = 0;
    if (!P->freeze_E) {
        if (P->init_sweeps_fixed >= 0)
            sweeps = potential_solve(c, P->init_sweeps_fixed,
                                     P->init_sweeps_fixed, P->sweep_tol, NULL);
        else
            sweeps = potential_solve(c, 0, P->init_sweeps_max, P->sweep_tol,
                                     NULL);
    }
    for (long k = 0; k < c->nn; ++k) {
        double Ex, Ey;
        if (P->freeze_E) {
            Ex = P->E_frozen_x;
            Ey = P->E_frozen_y;
        } else {
            E_of(c->g + 5 * k, c->tau_g, &Ex, &Ey);
        }
        double ceq = P->c_init_scale * n_eq_of(P, sqrt(Ex * Ex + Ey * Ey));
        ion_eq(c->qi, ceq, 0.0, 0.0, c->p + c->qi * k);
        ion_eq(c->qi, ceq, 0.0, 0.0, c->n + c->qi * k);
        double sp = 0.0, sn = 0.0;
        for (int i = 0; i < c->qi; ++i) {
            sp += c->p[c->qi * k + i];
            sn += c->n[c->qi * k + i];
        }
        c->snap[ORC_PHI * c->nn + k] = c->phi[k];
        c->snap[ORC_UX * c->nn + k] = 0.0;
        c->snap[ORC_UY * c->nn + k] = 0.0;
        c->snap[ORC_P * c->nn + k] = 0.0;
        c->snap[ORC_PSI * c->nn + k] = psi_of(c->g + 5 * k);
        c->snap[ORC_EX * c->nn + k] = Ex;
        c->snap[ORC_EY * c->nn + k] = Ey;
        c->snap[ORC_CP * c->nn + k] = sp;
        c->snap[ORC_CM * c->nn + k] = sn;
        c->snap[ORC_Q * c->nn + k] = sp - sn;
    }
    c->t = 0;
    return sweeps;
}

/* ---- one time step ------------------------------------------------------ */

static int step_once(orc_ctx *c, int forced, int *used, double *resid)
{
    const orc_params *P = &c->P;
    const long nn = c->nn;
    const double beta = 12.0 * P->sigma / P->W;   /* Eq. 13 */
    const double kappa = 1.5 * P->sigma * P->W;
    const double eta_v = cs2 * (P->tau_f - 0.5);  /* Eq. 55 with rho_v = 1 */

    /* O1-O3 */
    macro_phi_q(c);

    /* O4 */
    int nsw = 0;
    double r = NAN;
    int notconv = 0;
    if (!P->freeze_E) {
        if (forced >= 0) {
            nsw = potential_solve(c, forced, forced, P->sweep_tol, &r);
        } else {
            nsw = potential_solve(c, P->sweeps_min, P->sweeps_max,
                                  P->sweep_tol, &r);
            if (nsw > 0 && !(r < P->sweep_tol) && P->sweeps_max > P->sweeps_min)
                notconv = 1;
        }
    }
    if (used) *used = nsw;
    if (resid) *resid = r;

#pragma omp parallel for
    for (long k = 0; k < nn; ++k) {
        const double *f = c->f + 9 * k, *h = c->h + 9 * k;
        const int Q = c->qi;
        const double *pp = c->p + Q * k, *np = c->n + Q * k;
        double phi = c->phi[k];
        double gx = c->gpx[k], gy = c->gpy[k], lap = c->lap[k];

        /* O1: properties, Eq. 61 */
        double rho = 1.0 + (P->rho_ratio - 1.0) * phi;
        double eta = eta_v * (1.0 + (P->eta_ratio - 1.0) * phi);
        double tau_f = 0.5 + eta / (rho * cs2);
        double mup = P->mu_v * (1.0 + (P->mu_r - 1.0) * phi);
        double mum = P->m * mup;
        double Dp = P->einstein_D ? P->D * mup / P->mu_v : P->D;
        double Dm = P->einstein_D ? P->D * mum / P->mu_v : P->D;
        double grx = (P->rho_ratio - 1.0) * gx, gry = (P->rho_ratio - 1.0) * gy;
        double dex = (P->eps_r - 1.0) * gx, dey = (P->eps_r - 1.0) * gy;

        /* O4 result: psi and E, Eq. 49-50 */
        double psi = psi_of(c->g + 5 * k);
        double Ex, Ey;
        if (P->freeze_E) {
            Ex = P->E_frozen_x;
            Ey = P->E_frozen_y;
        } else {
            E_of(c->g + 5 * k, c->tau_g, &Ex, &Ey);
        }

        /* O5: Onsager F and the implicit reaction, Eq. 5, 42-43 */
        double sp = 0.0, sn = 0.0;
        for (int i = 0; i < Q; ++i) {
            sp += pp[i];
            sn += np[i];
        }
        double q = sp - sn;
        double cp, cm, R;
        if (P->onsager_form == 2) {
            cp = sp;
            cm = sn;
            R = 0.0;
        } else {
            double b = P->onsager_cb * sqrt(sqrt(Ex * Ex + Ey * Ey));
            double F = orc_onsager(b, P->onsager_form);
            orc_reaction(sp, sn, P->k_d, P->k_r, F, &cp, &cm, &R);
        }

        /* O6: forces, Eq. 12-14 */
        double mu_phi = 4.0 * beta * phi * (phi - 1.0) * (phi - 0.5) - kappa * lap;
        double E2 = Ex * Ex + Ey * Ey;
        double Fx = mu_phi * gx + P->Kq * q * Ex - 0.5 * E2 * dex;
        double Fy = mu_phi * gy + P->Kq * q * Ey - 0.5 * E2 * dey;

        /* O7: velocity and pressure, Eq. 56-57 */
        double jx = 0.0, jy = 0.0;
        for (int i = 0; i < 9; ++i) {
            jx += cx9[i] * f[i];
            jy += cy9[i] * f[i];
        }
        double ux = (jx + 0.5 * Fx) / rho;
        double uy = (jy + 0.5 * Fy) / rho;
        double pr = orc_pressure(f, rho, ux, uy, grx, gry);

        /* O8: f, Eq. 51 */
        double sf[9];
        for (int kk = 0; kk < 9; ++kk) sf[kk] = P->bgk ? 1.0 / tau_f : P->s_free;
        sf[1] = sf[2] = sf[3] = sf[4] = sf[5] = 1.0 / tau_f;
        double feq[9], Fi[9], d9[9], a9[9], b9[9];
        orc_feq(pr, rho, ux, uy, feq);
        orc_forcing_f(ux, uy, Fx, Fy, grx, gry, Fi);
        for (int i = 0; i < 9; ++i) d9[i] = f[i] - feq[i];
        msm(9, sf, d9, a9);
        msm_half(9, sf, Fi, b9);
        for (int i = 0; i < 9; ++i) c->fs[9 * k + i] = f[i] - a9[i] + b9[i];

        /* O9: h, Eq. 27 with Eq. 31-32 and the Euler derivative Eq. 58 */
        double tau_h = 0.5 + P->M_phi / cs2; /* Eq. 30 */
        double sh[9];
        for (int kk = 0; kk < 9; ++kk) sh[kk] = P->bgk ? 1.0 / tau_h : P->s_free;
        sh[1] = sh[2] = 1.0 / tau_h;
        double dpux = phi * ux - c->phiu_prev[2 * k];
        double dpuy = phi * uy - c->phiu_prev[2 * k + 1];
        double heq[9], Hi[9];
        orc_heq(phi, ux, uy, heq);
        orc_Hsrc(phi, P->W, dpux, dpuy, gx, gy, P->nhat_eps, Hi);
        for (int i = 0; i < 9; ++i) d9[i] = h[i] - heq[i];
        msm(9, sh, d9, a9);
        msm_half(9, sh, Hi, b9);
        for (int i = 0; i < 9; ++i) c->hs[9 * k + i] = h[i] - a9[i] + b9[i];
        c->phiu_prev[2 * k] = phi * ux;
        c->phiu_prev[2 * k + 1] = phi * uy;

        /* O10: ions, Eq. 34-40 (G of Eq. 40 with grad psi = -E), on the
         * D2Q5 lattice (N of Eq. 46, weights of Eq. 26) or, ion_lattice = 9,
         * on D2Q9 (M of Eq. 28, weights of Eq. 25); s1 = s2 = 1/tau (Eq. 37) */
        const int *cxq = Q == 9 ? cx9 : cx5, *cyq = Q == 9 ? cy9 : cy5;
        const double *wq = Q == 9 ? w9 : w5;
        double gpsx = -Ex, gpsy = -Ey;
        double sqp[9], sqn[9];
        rates_ion(P, Q, 0.5 + Dp / cs2, sqp);
        rates_ion(P, Q, 0.5 + Dm / cs2, sqn);
        double eqq[9], Gq[9], RL[9], dq[9], aq[9], bq[9], cq[9];
        ion_eq(Q, cp, ux, uy, eqq);
        orc_ion_src(Q, R, cp, Fx, Fy, P->ion_L_term, RL);
        for (int i = 0; i < Q; ++i) {
            double cg = cxq[i] * gpsx + cyq[i] * gpsy;
            Gq[i] = wq[i] * cg * mup * cp / cs2;
            dq[i] = pp[i] - eqq[i];
        }
        msm(Q, sqp, dq, aq);
        msm_half(Q, sqp, RL, bq);
        msm(Q, sqp, Gq, cq);
        for (int i = 0; i < Q; ++i)
            c->ps[Q * k + i] = pp[i] - aq[i] + bq[i] - cq[i];   /* Eq. 34 */
        ion_eq(Q, cm, ux, uy, eqq);
        orc_ion_src(Q, R, cm, Fx, Fy, P->ion_L_term, RL);
        for (int i = 0; i < Q; ++i) {
            double cg = cxq[i] * gpsx + cyq[i] * gpsy;
            Gq[i] = wq[i] * cg * mum * cm / cs2;
            dq[i] = np[i] - eqq[i];
        }
        msm(Q, sqn, dq, aq);
        msm_half(Q, sqn, RL, bq);
        msm(Q, sqn, Gq, cq);
        for (int i = 0; i < Q; ++i)
            c->ns[Q * k + i] = np[i] - aq[i] + bq[i] + cq[i];   /* Eq. 35 */

        /* snapshot of time t */
        c->snap[ORC_PHI * nn + k] = phi;
        c->snap[ORC_UX * nn + k] = ux;
        c->snap[ORC_UY * nn + k] = uy;
        c->snap[ORC_P * nn + k] = pr;
        c->snap[ORC_PSI * nn + k] = psi;
        c->snap[ORC_EX * nn + k] = Ex;
        c->snap[ORC_EY * nn + k] = Ey;
        c->snap[ORC_CP * nn + k] = cp;
        c->snap[ORC_CM * nn + k] = cm;
        c->snap[ORC_Q * nn + k] = q;
    }

    /* O11: streaming with the wall rules */
    stream9_bounce(c, c->fs, c->f);
    stream9_bounce(c, c->hs, c->h);
    const double *cpf = c->snap + ORC_CP * nn, *cmf = c->snap + ORC_CM * nn;
    double *zero = c->cwb, *zero2 = c->cwt;
    double *tmp_b = (double *)malloc(sizeof(double) * c->nx);
    double *tmp_t = (double *)malloc(sizeof(double) * c->nx);
    for (int x = 0; x < c->nx; ++x) zero[x] = zero2[x] = 0.0;
    if (P->ion_bc == 2) {
        stream_ion(c, c->ps, c->p, 1, zero, 1, zero2);
        stream_ion(c, c->ns, c->n, 1, zero, 1, zero2);
    } else if (P->ion_bc == 1) {
        stream_ion(c, c->ps, c->p, 0, zero, 0, zero2);
        stream_ion(c, c->ns, c->n, 0, zero, 0, zero2);
    } else {
        /* cations: repelled by the anode (c = 0), attracted by the cathode
         * (zero gradient, wall value from the node) */
        for (int x = 0; x < c->nx; ++x)
            tmp_t[x] = cpf[idx(c, x, c->ny - 1)];
        stream_ion(c, c->ps, c->p, 0, zero, 0, tmp_t);
        /* anions: attracted by the anode, repelled by the cathode */
        for (int x = 0; x < c->nx; ++x) tmp_b[x] = cmf[idx(c, x, 0)];
        stream_ion(c, c->ns, c->n, 0, tmp_b, 0, zero2);
    }
    free(tmp_b);
    free(tmp_t);
    c->t += 1;
    return notconv;
}

int orc_step(orc_ctx *c, int nsteps, const int *forced, int *counts,
             double *resid)
{
    int notconv = 0;
    for (int s = 0; s < nsteps; ++s) {
        int used = 0;
        double r = NAN;
        notconv += step_once(c, forced ? forced[s] : -1, &used, &r);
        if (counts) counts[s] = used;
        if (resid) resid[s] = r;
    }
    return notconv;
}

void orc_get_fields(const orc_ctx *c, double *out)
{
    memcpy(out, c->snap, sizeof(double) * ORC_NFIELDS * c->nn);
}

int orc_state_per_node(const orc_ctx *c) { return 25 + 2 * c->qi; }

void orc_get_state(const orc_ctx *c, double *out)
{
    const int Q = c->qi, S = 25 + 2 * Q;
    for (long k = 0; k < c->nn; ++k) {
        double *o = out + S * k;
        memcpy(o, c->f + 9 * k, 9 * sizeof(double));
        memcpy(o + 9, c->h + 9 * k, 9 * sizeof(double));
        memcpy(o + 18, c->p + Q * k, Q * sizeof(double));
        memcpy(o + 18 + Q, c->n + Q * k, Q * sizeof(double));
        memcpy(o + 18 + 2 * Q, c->g + 5 * k, 5 * sizeof(double));
        memcpy(o + 23 + 2 * Q, c->phiu_prev + 2 * k, 2 * sizeof(double));
    }
}

void orc_set_state(orc_ctx *c, const double *in)
{
    const int Q = c->qi, S = 25 + 2 * Q;
    for (long k = 0; k < c->nn; ++k) {
        const double *o = in + S * k;
        memcpy(c->f + 9 * k, o, 9 * sizeof(double));
        memcpy(c->h + 9 * k, o + 9, 9 * sizeof(double));
        memcpy(c->p + Q * k, o + 18, Q * sizeof(double));
        memcpy(c->n + Q * k, o + 18 + Q, Q * sizeof(double));
        memcpy(c->g + 5 * k, o + 18 + 2 * Q, 5 * sizeof(double));
        memcpy(c->phiu_prev + 2 * k, o + 23 + 2 * Q, 2 * sizeof(double));
    }
}

double orc_sum_phi(const orc_ctx *c)
{
    double s = 0.0;
    for (long k = 0; k < 9 * c->nn; ++k) s += c->h[k];
    return s;
}

long orc_time(const orc_ctx *c) { return c->t; }

/* ---- physical -> lattice mapping (Sec. 3) -------------------------------- *
 * Fixed lattice values are those of the plain droplet case (tau_f = 0.8,
 * sigma = 0.01, W = 4, M_phi = 0.02, D = 0.01, k_d = k_r = 1, vartheta = 0.3).
 *   W0    = 1.42233 d^2 / dpsi        (Eq. 23, W0 ~ d^2 / dpsi; value at
 *                                      d = 1 mm, dpsi = 1 kV from Sec. 6)
 *   beta  = 0.5643 sqrt(d / 2)        (Eq. 24, beta ~ d^(1/2); Sec. 6)
 *   O     = beta^2 / W0               (Eq. 24)
 *   Kq    = W0 dpsi_lat / ny^2        (Eq. 20 with x* = y / ny, psi* = psi /
 *                                      dpsi_lat; dpsi_lat = dpsi in kV)
 *   cb    = sqrt(O ny / dpsi_lat)     (b^2 = O |E*|, E* = E ny / dpsi_lat)
 *   R     = nx / 5, centred.                                               */
void orc_params_from_physical(orc_params *P, int nx, int ny, double d_mm,
                              double dpsi_kV, double eps_r, double mu_r)
{
    memset(P, 0, sizeof *P);
    P->tau_f = 0.8; P->rho_ratio = 1.0; P->eta_ratio = 1.0;
    P->sigma = 0.01; P->W = 4.0; P->W_init = 0.0; P->M_phi = 0.02; P->nhat_eps = 1e-3;
    P->xc = 0.5 * (nx - 1); P->yc = 0.5 * (ny - 1); P->R = nx / 5.0;
    P->D = 0.01; P->mu_v = 1.0; P->mu_r = mu_r; P->m = 1.0;
    P->k_d = 1.0; P->k_r = 1.0;
    double W0 = 1.42233 * d_mm * d_mm / dpsi_kV;
    double beta = 0.5643 * sqrt(d_mm / 2.0);
    double O = beta * beta / W0;
    P->onsager_cb = sqrt(O * ny / dpsi_kV);
    P->onsager_form = 0; P->ion_bc = 0; P->einstein_D = 1; P->ion_L_term = 1;
    P->c_init_scale = 1.0; P->c0 = 1.0;
    P->eps_r = eps_r;
    P->Kq = W0 * dpsi_kV / ((double)ny * ny);
    P->vartheta = 0.3;
    P->psi_anode = dpsi_kV; P->psi_cathode = 0.0;
    P->sweeps_min = 20; P->sweeps_max = 20; P->sweep_tol = 1e-8;
    P->init_sweeps_max = 0; P->init_sweeps_fixed = 0; P->init_psi_zero = 0;
    P->freeze_E = 0;
    P->s_free = 1.0; P->bgk = 0;
    P->ion_lattice = 5; P->side_walls = 0;
}

/* ---- deformation factor, Eq. 63 ------------------------------------------ *
 * L: extent of phi >= 1/2 along the field (y) through the phi-weighted
 * centroid, H: the same across it (x); crossings by linear interpolation
 * along the line, the line itself sampled by linear interpolation. */
double orc_sample(int nx, int ny, const double *phi, double x, double y)
{
    int x0 = (int)floor(x), y0 = (int)floor(y);
    double fx = x - x0, fy = y - y0;
    int x1 = x0 + 1, y1 = y0 + 1;
    x0 = ((x0 % nx) + nx) % nx;
    x1 = ((x1 % nx) + nx) % nx;
    if (y0 < 0) y0 = 0;
    if (y1 > ny - 1) y1 = ny - 1;
    if (y0 > ny - 1) y0 = ny - 1;
    double a = phi[(long)y0 * nx + x0] * (1 - fx) + phi[(long)y0 * nx + x1] * fx;
    double b = phi[(long)y1 * nx + x0] * (1 - fx) + phi[(long)y1 * nx + x1] * fx;
    return a * (1 - fy) + b * fy;
}

static double extent(int nx, int ny, const double *phi, double xc, double yc,
                     int along_y)
{
    int lim = along_y ? ny : nx;
    double ends[2];
    for (int dir = 0; dir < 2; ++dir) {
        double sgn = dir ? 1.0 : -1.0;
        double prev_t = 0.0;
        double prev_v = along_y ? orc_sample(nx, ny, phi, xc, yc)
                                : orc_sample(nx, ny, phi, xc, yc);
        double end = sgn * lim;
        for (int s = 1; s < lim; ++s) {
            double tt = sgn * s;
            double v = along_y ? orc_sample(nx, ny, phi, xc, yc + tt)
                               : orc_sample(nx, ny, phi, xc + tt, yc);
            if (prev_v >= 0.5 && v < 0.5) {
                end = prev_t + (tt - prev_t) * (prev_v - 0.5) / (prev_v - v);
                break;
            }
            prev_t = tt;
            prev_v = v;
        }
        ends[dir] = end;
    }
    return ends[1] - ends[0];
}

double orc_deformation(int nx, int ny, const double *phi)
{
    double s = 0.0, sx = 0.0, sy = 0.0;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double v = phi[(long)y * nx + x];
            s += v;
            sx += v * x;
            sy += v * y;
        }
    if (s <= 0.0) return 0.0;
    double xc = sx / s, yc = sy / s;
    double L = extent(nx, ny, phi, xc, yc, 1);
    double H = extent(nx, ny, phi, xc, yc, 0);
    return (L - H) / (L + H);
}
