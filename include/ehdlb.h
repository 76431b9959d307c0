/*
 * ehdlb.h -- C ABI of the GB300 (sm_103a) solver for the phase-field lattice
 * Boltzmann method for two-phase electrohydrodynamic flow driven by the
 * Onsager-Wien effect (Zheng, Wang, Xiong, Huang, Luo, arXiv 2501.04920).
 *
 * One time step advances five coupled lattice Boltzmann equations on a 2D
 * lattice (Sec. 4): the conservative Allen-Cahn equation (D2Q9, Eq. 27-33),
 * the cation and anion Nernst-Planck equations with field-enhanced
 * dissociation and recombination (D2Q5, Eq. 34-43), the electric potential
 * in pseudo-time (D2Q5, Eq. 44-50, swept inside every step) and the
 * incompressible Navier-Stokes equations with surface-tension and electric
 * forces (D2Q9, Eq. 51-57).  All compute runs in CUDA kernels; there is no
 * CPU path behind this interface.
 *
 * Conventions for every entry point:
 *  - Lattice units (dx = dt = 1).  Node (x, y), x in [0, nx) periodic,
 *    y in [0, ny).  The anode (psi_anode) lies half a spacing below row 0,
 *    the cathode (psi_cathode) half a spacing above row ny - 1 (Eq. 64).
 *  - Host arrays are row-major [ny][nx] (x fastest), FP64, caller-owned and
 *    only borrowed for the duration of the call.  The context owns all device
 *    memory; nothing returned points into it.
 *  - Every call returns an ehdlb_status; none aborts the process.  On an
 *    error, ehdlb_last_error() describes it.  A context is used by one host
 *    thread at a time.
 */
#ifndef EHDLB_H
#define EHDLB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EHDLB_ABI_VERSION 5

typedef struct ehdlb_ctx ehdlb_ctx;

typedef enum ehdlb_status {
    EHDLB_OK = 0,
    EHDLB_WNOTCONV = 1,   /* warning: a step hit sweeps_max above sweep_tol */
    EHDLB_EINVAL = -1,    /* invalid argument or parameter */
    EHDLB_ENOMEM = -2,    /* device or host allocation failed */
    EHDLB_ECUDA = -3,     /* a CUDA call failed */
    EHDLB_EUNSTABLE = -4, /* NaN or Inf in the fields */
    EHDLB_ESTATE = -5,    /* call out of order (e.g. step before set_params) */
    EHDLB_EFULL = -6      /* a batch's device-memory budget has no room for the case */
} ehdlb_status;

typedef enum ehdlb_precision {
    EHDLB_FP64 = 0,       /* populations and arithmetic in double */
    EHDLB_FP32 = 1,       /* populations and arithmetic in float; residual and
                             global sums in double */
    EHDLB_FP16S = 2       /* populations stored in FP16 as scaled deviations
                             from rest states (h from w_i phi_ref, g from
                             w_i psi_lin, p and n from w_i c_ref), arithmetic
                             in float, residual and sums in double; the storage
                             form that halves the memory traffic of the state
                             (a design choice with no counterpart in the paper) */
} ehdlb_precision;

/* Snapshot fields (bit i of a field mask selects field i). */
typedef enum ehdlb_field {
    EHDLB_PHI = 0,  /* order parameter, Eq. 33 */
    EHDLB_UX,       /* velocity, Eq. 56 */
    EHDLB_UY,
    EHDLB_P,        /* hydrodynamic pressure, Eq. 57 */
    EHDLB_PSI,      /* electric potential, Eq. 49 */
    EHDLB_EX,       /* electric field, Eq. 50 */
    EHDLB_EY,
    EHDLB_CP,       /* cation concentration, Eq. 42 */
    EHDLB_CM,       /* anion concentration, Eq. 42 */
    EHDLB_Q,        /* net charge c+ - c- */
    EHDLB_NFIELDS
} ehdlb_field;

/* Problem statement in lattice units.  Fill with ehdlb_params_default() or
 * ehdlb_params_from_physical(), then edit; size must equal
 * sizeof(ehdlb_params). */
typedef struct ehdlb_params {
    size_t size;
    /* incompressible NS (Eq. 51-57, 60-61) */
    double tau_f;        /* relaxation time of the outer phase (phi = 0), > 0.5 */
    double rho_ratio;    /* rho_l / rho_v, rho_v = 1 */
    double eta_ratio;    /* eta_l / eta_v */
    /* interface (Eq. 1-2, 12-13, 27-33) */
    double sigma;        /* surface tension */
    double W;            /* interface thickness, > 0 */
    double W_init;       /* thickness of the initial profile (<= 0: W) */
    double M_phi;        /* Allen-Cahn mobility, > 0 */
    double nhat_eps;     /* interface normal of Eq. 32 taken as grad phi /
                            sqrt(|grad phi|^2 + nhat_eps^2); 0: the printed
                            grad phi / |grad phi| (0 below |grad phi| 1e-12) */
    /* initial droplet: phi = (1 + tanh(2 (R - r) / W_init)) / 2 */
    double xc, yc, R;    /* centre and radius; for the slab, half-width */
    int init_shape;      /* 0 disc, 1 horizontal slab |y - yc| < R */
    /* ions (Eq. 3-6, 34-43) */
    double D;            /* ion diffusivity in the outer phase, > 0 */
    double mu_v;         /* cation mobility in the outer phase, > 0 */
    double mu_r;         /* mobility ratio mu_l / mu_v */
    double m;            /* anion / cation mobility ratio */
    double k_d;          /* dissociation rate delta c0^2 (Eq. 5), >= 0 */
    double k_r;          /* recombination rate delta (Eq. 5), >= 0 */
    double onsager_cb;   /* b = onsager_cb * sqrt(|E|) */
    int onsager_form;    /* 0: F = I1(4b) / (2b); 1: F = 1 + 2 b^2 (Eq. 6);
                            2: no reaction, R = 0 (Sec. 5.2) */
    int ion_bc;          /* 0: Eq. 64 (repelled species c = 0, attracted
                            species zero gradient); 1: c = 0 at both
                            electrodes; 2: zero flux */
    int einstein_D;      /* 1: D_pm = D mu_pm / mu_v (Sec. 2.2) */
    int ion_L_term;      /* 1: keep the source L_i of Eq. 39 */
    double c_init_scale; /* initial c_pm = c_init_scale * n_eq(E) */
    double c0;           /* initial c_pm when k_r = 0 or onsager_form = 2 */
    /* potential (Eq. 7-9, 44-50) */
    double eps_r;        /* permittivity ratio eps_l / eps_v, > 0 */
    double Kq;           /* charge coupling: lap psi = -Kq (c+ - c-) / eps */
    double vartheta;     /* artificial diffusion (Eq. 47), > 0 */
    int psi_src_literal; /* 1: Eq. 44 source as printed; 0 (default): divided
                            by (1 - w0) so that the steady state is Eq. 7 */
    double psi_anode, psi_cathode;
    int sweeps_min, sweeps_max;  /* pseudo-time sweeps per step, min <= max */
    double sweep_tol;            /* stop on ||psi^k - psi^(k-1)|| / ||psi^k|| */
    int init_sweeps_max;         /* cap of the initial potential solve */
    int init_sweeps_fixed;       /* >= 0: exactly this many initial sweeps */
    int init_psi_zero;           /* 1: start the potential from psi = 0 */
    int freeze_E;                /* 1: no potential sweeps, E = E_frozen */
    double E_frozen_x, E_frozen_y;
    /* collision */
    double s_free;       /* the free MRT rates, in (0, 2); 1.0 in Sec. 6 */
    int bgk;             /* 1: all rates equal the hydrodynamic one */
    /* ion lattice */
    int ion_lattice;     /* 5 (default): ions on D2Q5 with N (Eq. 46) and the
                            weights of Eq. 26; 9: on D2Q9 with M (Eq. 28) and
                            the weights of Eq. 25, as Eq. 34-36 print them
                            (s1 = s2 = 1/tau, Eq. 37, other rates free; a link
                            through an electrode, corners included, takes the
                            electrode's rule).  The state then holds 43 doubles
                            per node instead of 35. */
    /* geometry */
    int side_walls;      /* 0: periodic x (default); 1: solid walls half-way
                            left of x = 0 and right of x = nx - 1 with the
                            "other boundaries" rules of Eq. 64 (u = 0, zero
                            normal gradient of c+-, psi and phi): bounce-back
                            of f, h, p, n and g, mirrored ghost columns in
                            Eq. 59.  Potential sweeps then run one per launch. */
} ehdlb_params;

/* Counters of one ehdlb_step() call. */
typedef struct ehdlb_stats {
    long long steps;          /* steps advanced by the call */
    long long t;              /* time steps since set_params */
    long long sweeps_total;   /* potential sweeps in the call */
    int sweeps_max;           /* most sweeps in one step */
    int not_converged;        /* steps that hit sweeps_max above sweep_tol */
    double last_residual;     /* residual of the last sweep (NaN: none) */
    double sum_phi, sum_q;    /* FP64 sums of phi and q of the last snapshot */
    double seconds;           /* wall time of the call */
    double mlups;             /* nx ny steps / seconds / 1e6 */
    double ms_prep, ms_sweeps, ms_main;  /* device time per kernel class when
                                            timing is on (ehdlb_set_timing),
                                            over all steps of the call */
    long long launches;       /* kernels launched by the call */
    long long sweep_launches; /* of which potential-sweep kernels */
    int sweeps_per_launch;    /* fused sweeps per launch (0: one sweep per launch) */
    int tile_shape;           /* tile shape of the fused sweep kernel (ehdlb_set_tuning) */
    double deformation;       /* D (Eq. 63) of the last step when ehdlb_set_reporting asked
                                 for it, else NaN */
} ehdlb_stats;

/* Counters of one ehdlb_batch_step() call. */
typedef struct ehdlb_batch_stats {
    long long steps;          /* batch steps (every case advances by this many) */
    int cases;                /* cases stepped */
    int unstable_cases;       /* cases with NaN or Inf in their fields */
    double seconds;           /* wall time of the call */
    double device_ms;         /* device time of the call (CUDA events) */
    double mlups;             /* sum over cases of nx ny, times steps, / device time / 1e6 */
    long long launches;       /* kernels (graph nodes included) launched by the call */
    int sweeps_per_launch;    /* fused potential sweeps per launch used */
    int tile_shape;           /* tile shape of the fused sweep kernel used (0, 1, 2) */
} ehdlb_batch_stats;

/* ABI version of the loaded library (EHDLB_ABI_VERSION). */
int ehdlb_version(void);

/* Lattice values of the plain 64x64 droplet case: tau_f 0.8, sigma 0.01,
 * W 4, M_phi 0.02, R 12, D 0.01, k_d = k_r = 1, eps_r 2, vartheta 0.3 (Sec. 4.2),
 * Kq = 5.6893 / 64^2, sweeps 1..200 to 1e-8.  Returns EHDLB_EINVAL on NULL. */
int ehdlb_params_default(ehdlb_params *p);

/* Physical problem of Sec. 6 -> lattice values (Sec. 3): reference length
 * d_mm (electrode gap), applied voltage dpsi_kV, eps_r and mu_r.
 *   W0 = 1.42233 d^2 / dpsi (Eq. 23, value printed with Fig. 10),
 *   beta = 0.5643 (d / 2)^(1/2) (Eq. 24, values printed in Sec. 6),
 *   O = beta^2 / W0, Kq = W0 dpsi / ny^2 (Eq. 20), onsager_cb = (O ny / dpsi)^(1/2)
 *   (b^2 = O |E*|, Eq. 17), psi_anode = dpsi, R = nx / 5; other values as
 * ehdlb_params_default, 20 sweeps per step, no initial solve. */
int ehdlb_params_from_physical(ehdlb_params *p, int nx, int ny, double d_mm,
                               double dpsi_kV, double eps_r, double mu_r);

/* Allocate a solver for an nx x ny lattice (nx, ny >= 4) in the given
 * precision.  cuda_stream: a cudaStream_t to launch on, or NULL for a stream
 * the context creates.  The device is the current one.  *out receives the
 * context; EHDLB_ENOMEM if device memory runs out. */
int ehdlb_create(ehdlb_ctx **out, int nx, int ny, int precision,
                 void *cuda_stream);

/* Validate p and (re)initialise the lattice at t = 0 (Sec. 6 set-up): the
 * droplet profile, u = p = 0, the linear potential with its initial solve
 * (q = 0), ions at n_eq of the resulting field, populations at equilibrium.
 * EHDLB_EINVAL on a relaxation time <= 0.5 or any other invalid value. */
int ehdlb_set_params(ehdlb_ctx *c, const ehdlb_params *p);

/* Replay given sweep counts: step t (counted from the last set_params)
 * takes exactly counts[t] sweeps for t < n; later steps follow the stop rule.
 * n = 0 clears the schedule.  Used to compare with a run whose sweep counts
 * were decided elsewhere. */
int ehdlb_set_sweep_schedule(ehdlb_ctx *c, const int *counts, int n);

/* Test hook of the failure detection; the paper has no counterpart.  The
 * next ehdlb_step call runs its step kernel with copies that never complete
 * (each block waits for 16 bytes more than its tensor-memory-accelerator
 * boxes deliver): the bounded wait of every block runs out (about 70 ms), the
 * block leaves without computing, and the call returns EHDLB_ECUDA with
 * ehdlb_last_error naming the late copies.  Nothing faults; the context stays
 * usable, but the lattice's state is then undefined until ehdlb_set_params
 * or ehdlb_set_state.  EHDLB_ESTATE when the step kernel does not take staged
 * copies on this lattice (FP64, ions on D2Q9, side walls, rows that are not
 * a multiple of 16 bytes, or staging chosen otherwise with ehdlb_set_tuning). */
int ehdlb_test_stall_copies(ehdlb_ctx *c);

/* Advance nsteps time steps.  Blocks until the device has finished.  out
 * (nullable) receives the counters.  Returns EHDLB_WNOTCONV if a step hit
 * sweeps_max above sweep_tol, EHDLB_EUNSTABLE on NaN/Inf. */
int ehdlb_step(ehdlb_ctx *c, int nsteps, ehdlb_stats *out);

/* Copy snapshot fields to the host: the fields of the last step, at the
 * time t of that step (before its collision), with psi and E after its
 * sweeps; before any step, the initial fields.  mask selects fields (bit
 * EHDLB_PHI ...); they are written in increasing field order, each
 * [ny][nx], into dst of dst_len doubles (>= popcount(mask) nx ny). */
int ehdlb_get_fields(ehdlb_ctx *c, unsigned mask, double *dst,
                     size_t dst_len);

/* What the last step of every ehdlb_step call reports.  snapshot_mask
 * (bits EHDLB_PHI ...) selects the fields its snapshot captures for
 * ehdlb_get_fields (default: all); asking ehdlb_get_fields for a field
 * outside the last capture returns EHDLB_ESTATE.  deformation = 1 makes every
 * call also compute the deformation factor D of Eq. 63 from that snapshot
 * (phi is then captured whatever the mask) and return it in
 * ehdlb_stats.deformation, read back with the call's counters.  The initial
 * fields after ehdlb_set_params are always captured whole.  EINVAL for a
 * mask with bits at or above EHDLB_NFIELDS or deformation outside 0, 1. */
int ehdlb_set_reporting(ehdlb_ctx *c, unsigned snapshot_mask, int deformation);

/* Sweep counts of the steps of the last ehdlb_step call, n <= its nsteps. */
int ehdlb_get_sweep_counts(ehdlb_ctx *c, int *dst, int n);

/* Raw state as S doubles per node, node-major [ny][nx][S]: f0..f8, h0..h8,
 * the ion populations p and n (Eq. 25-26 order), g0..g4, (phi u)(t-1) x and
 * y; S = 35 with ions on D2Q5 (p0..p4, n0..n4) and 43 on D2Q9 (p0..p8,
 * n0..n8); ehdlb_state_len gives S nx ny for the ion lattice of the last
 * ehdlb_set_params.  The library does not store f0 and g0 (no other quantity
 * depends on them): get_state writes 0 there and set_state ignores them.
 * len in doubles. */
size_t ehdlb_state_len(const ehdlb_ctx *c);
int ehdlb_get_state(ehdlb_ctx *c, double *dst, size_t len);
int ehdlb_set_state(ehdlb_ctx *c, const double *src, size_t len);

/* Device time per kernel class in ehdlb_stats (ms_prep, ms_sweeps, ms_main):
 * every > 0 records CUDA events around the kernel classes of every every-th
 * step of a call (its first step, then every every-th) and scales their sums
 * to all the call's steps; 0 records none (the default).  A recorded step
 * runs a few microseconds longer: its events stand between kernels that
 * otherwise start as programmatic dependents of their predecessors.
 * EINVAL if every < 0. */
int ehdlb_set_timing(ehdlb_ctx *c, int every);

/* Performance knobs; none changes the result beyond round-off.
 *   sweeps_per_launch: potential sweeps the fused sweep kernel computes in
 *     shared memory per launch when a step takes a fixed number of sweeps,
 *     1..5 (the double-precision solver uses at most 2), 0 for one sweep per
 *     launch; default 5 (float) / 2 (double);
 *   tile_shape: blocks of the fused sweep kernel, 0: 64 x 32 region per
 *     block (512 threads; the double solver's only shape), 1: 64 x 32 (256
 *     threads), 2: clusters of 2 x 4 blocks of 64 x 32 that exchange
 *     populations through distributed shared memory every sweep, 3: 64 x 64
 *     (512 threads), 4: 64 x 32 and 5: 64 x 40 (persistent blocks of 256
 *     threads, each thread holding the populations of 2 x 4 or 2 x 5 nodes
 *     in registers; populations cross lanes by warp shuffles and warps
 *     through shared memory; 5 is the default for float), 6: shape 5 with
 *     the pass that forms phi, grad phi and q fused into the first sweep
 *     launch of a step (float storage, D2Q5 ions, no side walls and a fixed
 *     sweep count; else shape 5), 7: shape 5 with each block walking its
 *     tiles down a column strip and keeping the upward flux of the row
 *     under a region in shared memory; 1 to 7 float only;
 *   main_staging: how the step kernel copies its block's populations to
 *     shared memory, 0: one asynchronous copy per node and plane, 1: 16-byte
 *     copies of row segments (used only when nx times the element size is a
 *     multiple of 16 bytes, else 0; default for double), 2: tensor-memory-
 *     accelerator loads of the block's tile behind one mbarrier, one tile
 *     per block (default for float), 3: the same in persistent blocks with
 *     two stages; 2 and 3 need float compute, D2Q5 ions, no side walls and
 *     nx times the element size a multiple of 16 bytes, else 1.
 * -1 keeps a setting.  EINVAL outside these ranges. */
int ehdlb_set_tuning(ehdlb_ctx *c, int sweeps_per_launch, int tile_shape, int main_staging);

/* Largest lattice, in nodes nx * ny, that ehdlb_potential_noalloc accepts. */
#define EHDLB_NOALLOC_MAX_NODES 65536

/* Potential solve that allocates no device memory.  The paper has no
 * counterpart; this entry point exists for callers that cannot call
 * cudaMalloc: code inside an allocator or memory-pool callback, a process
 * whose device memory is entirely held and budgeted by another runtime, or a
 * latency-critical loop that must not risk the implicit device
 * synchronisation of an allocation.
 *
 * Runs nsweeps pseudo-time sweeps of the potential equation (Eq. 44-50) in
 * FP64 on an nx x ny lattice (nx ny <= EHDLB_NOALLOC_MAX_NODES, nx, ny >= 4),
 * starting from the initial potential of ehdlb_set_params (linear between the
 * electrodes, or zero if p->init_psi_zero), with the source from phi (eps,
 * Eq. 61) and q (net charge), and writes psi (Eq. 49) and E (Eq. 50).  With
 * q = 0 the result is the initial potential ehdlb_set_params computes with
 * p->init_sweeps_fixed = nsweeps.  Only the potential fields of p are read.
 *   phi, q     : caller-owned DEVICE arrays [ny][nx] of double (inputs)
 *   psi, Ex, Ey: caller-owned DEVICE arrays [ny][nx] of double (outputs)
 *   residual   : host pointer or NULL; receives ||psi^K - psi^(K-1)|| /
 *                ||psi^K|| of the last sweep (NaN for nsweeps = 0); when it is
 *                not NULL the call waits for the stream
 *   cuda_stream: cudaStream_t to launch on, or NULL for the default stream
 * Every intermediate lives in one file-scope device array of about 5.6 MB
 * that each GPU loading this library reserves until the process exits; the
 * call makes no allocation.  All calls share that array and it keeps the last
 * call's contents (the call resets what must start at zero), so calls whose
 * work overlaps on the GPU -- on different streams, or from different host
 * threads -- race and must be serialised by the caller.  The first call on a
 * device looks up the array's device address (with that device current), and
 * so does the first call after the device's context was replaced (by
 * cudaDeviceReset, for instance); make that first call before any stream
 * capture begins.
 * Returns EHDLB_EINVAL for a lattice above the maximum, nx or ny < 4, NULL
 * arrays, p->size != sizeof(ehdlb_params) or invalid potential parameters;
 * EHDLB_ECUDA if a launch or copy fails. */
int ehdlb_potential_noalloc(int nx, int ny, const ehdlb_params *p, const double *phi,
                            const double *q, int nsweeps, double *psi, double *Ex,
                            double *Ey, double *residual, void *cuda_stream);

/* Deformation factor D = (L - H) / (L + H) of Eq. 63 from the phi field of the
 * last snapshot (the last step of the last ehdlb_step call): L is the extent
 * of phi >= 1/2 along the field (y) on the line through the phi-weighted
 * centroid, H the same across it (x); the line is sampled by bilinear
 * interpolation of the nodes and each end is the crossing of 1/2 interpolated
 * linearly between unit-spaced samples.  Computed on the device (one block).
 * EHDLB_EINVAL on NULL, EHDLB_ESTATE before set_params. */
int ehdlb_deformation(ehdlb_ctx *c, double *D);

/* Free all device memory of the context (NULL is a no-op). */
void ehdlb_destroy(ehdlb_ctx *c);

/* Text of the last error on c (empty if none); valid until the next call. */
const char *ehdlb_last_error(const ehdlb_ctx *c);

/* ---- batches: many lattices stepped together -------------------------------------
 * A batch owns one device arena of budget_bytes from which every case's
 * buffers are carved (first fit); ehdlb_batch_add admits a case only if its
 * footprint (ehdlb_batch_footprint) fits.  ehdlb_batch_step advances every
 * case by nsteps time steps with one launch per kernel kind and step: the
 * persistent kernels walk a device work-list of (case, tile) items and run
 * the per-block code of the single-lattice kernels, so a case's fields are
 * bit for bit those of the same case stepped alone with the same sweeps per
 * launch and tile shape.  The steps of a call but the last replay a captured
 * CUDA graph of one batch step.  All cases take the batch's fixed number of
 * potential sweeps per step (params.sweeps_min = sweeps_max = sweeps); batch
 * cases need nx a multiple of 8, periodic x (side_walls = 0), freeze_E = 0 and
 * init_sweeps_fixed >= 0.  precision: EHDLB_FP32 or EHDLB_FP16S.  One host
 * thread at a time per batch.  (A design of this build; the paper steps one
 * lattice.) */
typedef struct ehdlb_batch ehdlb_batch;

/* Create a batch; cuda_stream: cudaStream_t or NULL (the batch makes one).
 * EHDLB_EINVAL for a bad precision, sweeps < 1 or budget 0; EHDLB_ENOMEM if
 * the arena cannot be allocated. */
int ehdlb_batch_create(ehdlb_batch **out, int precision, size_t budget_bytes, int sweeps,
                       void *cuda_stream);

/* Device bytes one case of nx x ny nodes takes in a batch of that precision. */
int ehdlb_batch_footprint(int precision, int nx, int ny, size_t *bytes);

/* Add a case (set up as by ehdlb_set_params, state at t = 0); *id identifies
 * it.  EHDLB_EFULL if the arena has no room; EHDLB_EINVAL for parameters a
 * batch does not take (see above) or that ehdlb_set_params rejects. */
int ehdlb_batch_add(ehdlb_batch *b, int nx, int ny, const ehdlb_params *p, int *id);

/* Remove a case and return its memory to the arena. */
int ehdlb_batch_remove(ehdlb_batch *b, int id);

/* Advance every case by nsteps steps; the last step writes each case's
 * snapshot.  st may be NULL.  EHDLB_EUNSTABLE if a case's fields hold NaN or
 * Inf, EHDLB_ESTATE for an empty batch. */
int ehdlb_batch_step(ehdlb_batch *b, int nsteps, ehdlb_batch_stats *st);

/* Snapshot fields of case id, as ehdlb_get_fields (dst: host, FP64,
 * [field][ny][nx] for the fields of mask in order). */
int ehdlb_batch_get_fields(ehdlb_batch *b, int id, unsigned mask, double *dst, size_t dst_len);

/* State of case id as ehdlb_get_state (35 doubles per node: batch cases
 * have ions on D2Q5). */
int ehdlb_batch_get_state(ehdlb_batch *b, int id, double *dst, size_t len);

/* D of Eq. 63 (as ehdlb_deformation) of n cases from their last snapshots,
 * all computed on the device in one launch. */
int ehdlb_batch_deformation(ehdlb_batch *b, int n, const int *ids, double *D);

/* Sweeps fused per launch (1..5; default 5), tile shape of the fused sweep
 * kernel (0: 64 x 32 regions in shared memory, 512 threads; 1: the same with
 * 256 threads; 2: 64 x 40 regions in registers, as tile shape 5 of
 * ehdlb_set_tuning, default) and whether steps replay a captured graph (default 1);
 * -1 keeps a setting; EINVAL outside these ranges. */
int ehdlb_batch_set_tuning(ehdlb_batch *b, int sweeps_per_launch, int tile_shape, int use_graphs);

/* Autotuner: time `steps` batch steps of the current cases for every sweeps
 * per launch in 3..5 and the three tile shapes, keep the fastest and report
 * it.  The timed steps are real steps: the cases advance by 9 (steps + 1). */
int ehdlb_batch_autotune(ehdlb_batch *b, int steps, int *sweeps_per_launch, int *tile_shape,
                         double *ms_per_step);

/* Number of cases, arena bytes in use and arena capacity (any may be NULL). */
int ehdlb_batch_info(const ehdlb_batch *b, int *cases, size_t *bytes_in_use, size_t *capacity);

const char *ehdlb_batch_last_error(const ehdlb_batch *b);

/* Free the batch and all its device memory (NULL is a no-op). */
void ehdlb_batch_destroy(ehdlb_batch *b);

#ifdef __cplusplus
}
#endif
#endif
