// ehdlb_api.cu -- the extern "C" boundary declared in include/ehdlb.h:
// argument checks, parameter validation, error codes and messages.  All
// compute is delegated to the CUDA solver; there is no host fallback.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "ehdlb.h"
#include "ehdlb_solver_base.h"

struct ehdlb_ctx {
    ehdlb::SolverBase *solver = nullptr;
    int nx = 0, ny = 0, precision = 0;
    bool has_params = false;
    std::string err;
};

struct ehdlb_batch {
    ehdlb::BatchBase *batch = nullptr;
    int precision = 0;
    std::string err;
};

namespace {

int fail(ehdlb_ctx *c, int status, const std::string &msg)
{
    if (c) c->err = msg;
    return status;
}

bool finite_all(const ehdlb_params *p)
{
    const double v[] = {p->tau_f, p->rho_ratio, p->eta_ratio, p->sigma, p->W, p->W_init, p->M_phi, p->nhat_eps,
                        p->xc, p->yc, p->R, p->D, p->mu_v, p->mu_r, p->m, p->k_d, p->k_r,
                        p->onsager_cb, p->c_init_scale, p->c0, p->eps_r, p->Kq, p->vartheta,
                        p->psi_anode, p->psi_cathode, p->sweep_tol, p->E_frozen_x, p->E_frozen_y,
                        p->s_free};
    for (double x : v)
        if (!std::isfinite(x)) return false;
    return true;
}

// Returns an empty string if p is acceptable for an nx x ny lattice.
std::string validate(const ehdlb_params *p)
{
    if (p->size != sizeof(ehdlb_params)) return "params.size != sizeof(ehdlb_params)";
    if (!finite_all(p)) return "a parameter is NaN or Inf";
    if (!(p->tau_f > 0.5)) return "tau_f must be > 0.5";
    if (!(p->rho_ratio > 0.0) || !(p->eta_ratio > 0.0)) return "rho_ratio and eta_ratio must be > 0";
    // the local NS relaxation time (Eq. 55 with Eq. 61) must stay > 0.5 in both phases
    if (!(p->eta_ratio / p->rho_ratio * (p->tau_f - 0.5) > 0.0)) return "tau_f of the inner phase <= 0.5";
    if (!(p->W > 0.0)) return "W must be > 0";
    if (!(p->M_phi > 0.0)) return "M_phi must be > 0 (tau_h > 0.5)";
    if (!(p->sigma >= 0.0)) return "sigma must be >= 0";
    if (!(p->nhat_eps >= 0.0)) return "nhat_eps must be >= 0";
    if (!(p->D > 0.0)) return "D must be > 0 (ion tau > 0.5)";
    if (!(p->mu_v > 0.0) || !(p->mu_r > 0.0) || !(p->m > 0.0)) return "mobilities must be > 0";
    if (!(p->k_d >= 0.0) || !(p->k_r >= 0.0)) return "k_d and k_r must be >= 0";
    if (!(p->onsager_cb >= 0.0)) return "onsager_cb must be >= 0";
    if (p->onsager_form < 0 || p->onsager_form > 2) return "onsager_form must be 0, 1 or 2";
    if (p->ion_bc < 0 || p->ion_bc > 2) return "ion_bc must be 0, 1 or 2";
    if (!(p->eps_r > 0.0)) return "eps_r must be > 0";
    if (!(p->vartheta > 0.0)) return "vartheta must be > 0 (tau_g > 0.5)";
    if (p->sweeps_min < 0 || p->sweeps_max < p->sweeps_min) return "need 0 <= sweeps_min <= sweeps_max";
    if (p->sweeps_max > 1000000) return "sweeps_max above 1e6";
    if (!(p->sweep_tol >= 0.0)) return "sweep_tol must be >= 0";
    if (p->init_sweeps_max < 0 || p->init_sweeps_max > 100000000) return "init_sweeps_max out of range";
    if (p->init_sweeps_fixed > 100000000) return "init_sweeps_fixed out of range";
    if (!(p->s_free > 0.0 && p->s_free < 2.0)) return "s_free must lie in (0, 2)";
    if (!(p->c_init_scale >= 0.0) || !(p->c0 >= 0.0)) return "initial concentrations must be >= 0";
    if (p->side_walls != 0 && p->side_walls != 1) return "side_walls must be 0 or 1";
    if (p->ion_lattice != 5 && p->ion_lattice != 9) return "ion_lattice must be 5 or 9";
    return "";
}

}  // namespace

extern "C" {

int ehdlb_version(void) { return EHDLB_ABI_VERSION; }

int ehdlb_params_default(ehdlb_params *p)
{
    if (!p) return EHDLB_EINVAL;
    std::memset(p, 0, sizeof *p);
    p->size = sizeof *p;
    p->tau_f = 0.8; p->rho_ratio = 1.0; p->eta_ratio = 1.0;
    p->sigma = 0.01; p->W = 4.0; p->W_init = 0.0; p->M_phi = 0.02; p->nhat_eps = 1e-3;
    p->xc = 31.5; p->yc = 31.5; p->R = 12.0; p->init_shape = 0;
    p->D = 0.01; p->mu_v = 1.0; p->mu_r = 1.0; p->m = 1.0;
    p->k_d = 1.0; p->k_r = 1.0; p->onsager_cb = 1.0;
    p->onsager_form = 0; p->ion_bc = 0; p->einstein_D = 1; p->ion_L_term = 1;
    p->c_init_scale = 1.0; p->c0 = 1.0;
    p->eps_r = 2.0; p->Kq = 5.6893 / (64.0 * 64.0); p->vartheta = 0.3; p->psi_src_literal = 0;
    p->psi_anode = 1.0; p->psi_cathode = 0.0;
    p->sweeps_min = 1; p->sweeps_max = 200; p->sweep_tol = 1e-8;
    p->init_sweeps_max = 100000; p->init_sweeps_fixed = -1; p->init_psi_zero = 0;
    p->freeze_E = 0; p->E_frozen_x = 0.0; p->E_frozen_y = 0.0;
    p->s_free = 1.0; p->bgk = 0;
    p->side_walls = 0;
    p->ion_lattice = 5;
    return EHDLB_OK;
}

int ehdlb_params_from_physical(ehdlb_params *p, int nx, int ny, double d_mm, double dpsi_kV,
                               double eps_r, double mu_r)
{
    if (!p || nx < 4 || ny < 4 || !(d_mm > 0.0) || !(dpsi_kV > 0.0) || !(eps_r > 0.0) || !(mu_r > 0.0))
        return EHDLB_EINVAL;
    ehdlb_params_default(p);
    const double W0 = 1.42233 * d_mm * d_mm / dpsi_kV;   // Eq. 23, Fig. 10 caption
    const double beta = 0.5643 * std::sqrt(d_mm / 2.0);  // Eq. 24, Sec. 6
    const double O = beta * beta / W0;                   // Eq. 24
    p->xc = 0.5 * (nx - 1);
    p->yc = 0.5 * (ny - 1);
    p->R = nx / 5.0;
    p->mu_r = mu_r;
    p->eps_r = eps_r;
    p->Kq = W0 * dpsi_kV / ((double)ny * ny);            // Eq. 20
    p->onsager_cb = std::sqrt(O * ny / dpsi_kV);         // b^2 = O |E*| (Eq. 17)
    p->psi_anode = dpsi_kV;
    p->psi_cathode = 0.0;
    p->sweeps_min = 20;
    p->sweeps_max = 20;
    p->init_sweeps_max = 0;
    p->init_sweeps_fixed = 0;
    return EHDLB_OK;
}

int ehdlb_create(ehdlb_ctx **out, int nx, int ny, int precision, void *cuda_stream)
{
    if (!out) return EHDLB_EINVAL;
    *out = nullptr;
    if (nx < 4 || ny < 4) return EHDLB_EINVAL;
    if ((long long)nx * ny > (1LL << 31)) return EHDLB_EINVAL;
    if (precision != EHDLB_FP64 && precision != EHDLB_FP32 && precision != EHDLB_FP16S) return EHDLB_EINVAL;
    ehdlb_ctx *c = new (std::nothrow) ehdlb_ctx;
    if (!c) return EHDLB_ENOMEM;
    c->nx = nx;
    c->ny = ny;
    c->precision = precision;
    int status = EHDLB_OK;
    std::string err;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    c->solver = precision == EHDLB_FP64   ? ehdlb::make_solver_fp64(nx, ny, s, &status, err)
                : precision == EHDLB_FP16S ? ehdlb::make_solver_fp16s(nx, ny, s, &status, err)
                                           : ehdlb::make_solver_fp32(nx, ny, s, &status, err);
    if (!c->solver) {
        delete c;
        return status != EHDLB_OK ? status : EHDLB_ENOMEM;
    }
    *out = c;
    return EHDLB_OK;
}

int ehdlb_set_params(ehdlb_ctx *c, const ehdlb_params *p)
{
    if (!c) return EHDLB_EINVAL;
    if (!p) return fail(c, EHDLB_EINVAL, "params is NULL");
    const std::string why = validate(p);
    if (!why.empty()) return fail(c, EHDLB_EINVAL, why);
    c->has_params = false;
    const int st = c->solver->set_params(*p, c->err);
    if (st == EHDLB_OK) c->has_params = true;
    return st;
}

int ehdlb_set_sweep_schedule(ehdlb_ctx *c, const int *counts, int n)
{
    if (!c) return EHDLB_EINVAL;
    if (n < 0 || (n > 0 && !counts)) return fail(c, EHDLB_EINVAL, "bad schedule");
    for (int i = 0; i < n; ++i)
        if (counts[i] < 0 || counts[i] > 1000000) return fail(c, EHDLB_EINVAL, "schedule entry out of range");
    c->solver->set_schedule(counts, n);
    return EHDLB_OK;
}

int ehdlb_test_stall_copies(ehdlb_ctx *c)
{
    if (!c) return EHDLB_EINVAL;
    if (!c->has_params) return fail(c, EHDLB_ESTATE, "ehdlb_set_params must come first");
    const int st = c->solver->stall_next_copies();
    if (st != EHDLB_OK) return fail(c, st, "the step kernel does not take staged copies on this lattice");
    return EHDLB_OK;
}

int ehdlb_step(ehdlb_ctx *c, int nsteps, ehdlb_stats *out)
{
    if (!c) return EHDLB_EINVAL;
    if (!c->has_params) return fail(c, EHDLB_ESTATE, "ehdlb_set_params must come before ehdlb_step");
    if (nsteps < 0) return fail(c, EHDLB_EINVAL, "nsteps < 0");
    if (out) std::memset(out, 0, sizeof *out);
    if (nsteps == 0) return EHDLB_OK;
    return c->solver->step(nsteps, out, c->err);
}

int ehdlb_get_fields(ehdlb_ctx *c, unsigned mask, double *dst, size_t dst_len)
{
    if (!c) return EHDLB_EINVAL;
    if (!c->has_params) return fail(c, EHDLB_ESTATE, "no fields before ehdlb_set_params");
    if (mask == 0 || (mask >> EHDLB_NFIELDS) != 0) return fail(c, EHDLB_EINVAL, "bad field mask");
    int nf = 0;
    for (int f = 0; f < EHDLB_NFIELDS; ++f) nf += (mask >> f) & 1;
    if (!dst || dst_len < (size_t)nf * c->nx * c->ny) return fail(c, EHDLB_EINVAL, "dst too small");
    return c->solver->get_fields(mask, dst, c->err);
}

int ehdlb_get_sweep_counts(ehdlb_ctx *c, int *dst, int n)
{
    if (!c) return EHDLB_EINVAL;
    if (n < 0 || n > c->solver->last_nsteps || (n > 0 && !dst))
        return fail(c, EHDLB_EINVAL, "n exceeds the steps of the last call");
    return c->solver->get_counts(dst, n, c->err);
}

size_t ehdlb_state_len(const ehdlb_ctx *c)
{
    return c ? (size_t)c->solver->state_per_node() * c->nx * c->ny : 0;
}

int ehdlb_get_state(ehdlb_ctx *c, double *dst, size_t len)
{
    if (!c) return EHDLB_EINVAL;
    if (!c->has_params) return fail(c, EHDLB_ESTATE, "no state before ehdlb_set_params");
    if (!dst || len < ehdlb_state_len(c)) return fail(c, EHDLB_EINVAL, "dst too small");
    return c->solver->get_state(dst, c->err);
}

int ehdlb_set_state(ehdlb_ctx *c, const double *src, size_t len)
{
    if (!c) return EHDLB_EINVAL;
    if (!c->has_params) return fail(c, EHDLB_ESTATE, "ehdlb_set_params must come before ehdlb_set_state");
    if (!src || len < ehdlb_state_len(c)) return fail(c, EHDLB_EINVAL, "src too small");
    return c->solver->set_state(src, c->err);
}

int ehdlb_set_timing(ehdlb_ctx *c, int every)
{
    if (!c) return EHDLB_EINVAL;
    if (every < 0) return fail(c, EHDLB_EINVAL, "timing stride must be >= 0");
    c->solver->set_timing(every);
    return EHDLB_OK;
}

int ehdlb_set_reporting(ehdlb_ctx *c, unsigned snapshot_mask, int deformation)
{
    if (!c) return EHDLB_EINVAL;
    if (snapshot_mask >> EHDLB_NFIELDS) return fail(c, EHDLB_EINVAL, "snapshot_mask has bits beyond the fields");
    if (deformation != 0 && deformation != 1) return fail(c, EHDLB_EINVAL, "deformation must be 0 or 1");
    c->solver->set_reporting(snapshot_mask, deformation);
    return EHDLB_OK;
}

int ehdlb_set_tuning(ehdlb_ctx *c, int sweeps_per_launch, int tile_shape, int main_staging)
{
    if (!c) return EHDLB_EINVAL;
    if (sweeps_per_launch < -1 || sweeps_per_launch > 5)
        return fail(c, EHDLB_EINVAL, "sweeps_per_launch must lie in -1..5");
    if (tile_shape < -1 || tile_shape > 7) return fail(c, EHDLB_EINVAL, "tile_shape must lie in -1..7");
    if (main_staging < -1 || main_staging > 3) return fail(c, EHDLB_EINVAL, "main_staging must lie in -1..3");
    c->solver->set_tuning(sweeps_per_launch, tile_shape, main_staging);
    return EHDLB_OK;
}

void ehdlb_destroy(ehdlb_ctx *c)
{
    if (!c) return;
    delete c->solver;
    delete c;
}

const char *ehdlb_last_error(const ehdlb_ctx *c) { return c ? c->err.c_str() : "null context"; }

int ehdlb_deformation(ehdlb_ctx *c, double *D)
{
    if (!c || !D) return EHDLB_EINVAL;
    if (!c->has_params) return fail(c, EHDLB_ESTATE, "ehdlb_set_params first");
    return c->solver->deformation(D, c->err);
}

// ---- batches ----------------------------------------------------------------

static int bfail(ehdlb_batch *b, int status, const std::string &msg)
{
    if (b) b->err = msg;
    return status;
}

int ehdlb_batch_create(ehdlb_batch **out, int precision, size_t budget_bytes, int sweeps, void *cuda_stream)
{
    if (!out) return EHDLB_EINVAL;
    *out = nullptr;
    if (precision != EHDLB_FP32 && precision != EHDLB_FP16S) return EHDLB_EINVAL;
    if (sweeps < 1 || sweeps > 1000000 || budget_bytes == 0) return EHDLB_EINVAL;
    ehdlb_batch *b = new (std::nothrow) ehdlb_batch;
    if (!b) return EHDLB_ENOMEM;
    b->precision = precision;
    int status = EHDLB_OK;
    std::string err;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    b->batch = precision == EHDLB_FP16S ? ehdlb::make_batch_fp16s(budget_bytes, sweeps, s, &status, err)
                                        : ehdlb::make_batch_fp32(budget_bytes, sweeps, s, &status, err);
    if (!b->batch) {
        delete b;
        return status != EHDLB_OK ? status : EHDLB_ENOMEM;
    }
    *out = b;
    return EHDLB_OK;
}

int ehdlb_batch_footprint(int precision, int nx, int ny, size_t *bytes)
{
    if (!bytes || nx < 4 || ny < 4) return EHDLB_EINVAL;
    if (precision == EHDLB_FP32) *bytes = ehdlb::footprint_fp32(nx, ny);
    else if (precision == EHDLB_FP16S) *bytes = ehdlb::footprint_fp16s(nx, ny);
    else return EHDLB_EINVAL;
    return EHDLB_OK;
}

int ehdlb_batch_add(ehdlb_batch *b, int nx, int ny, const ehdlb_params *p, int *id)
{
    if (!b || !p || !id) return EHDLB_EINVAL;
    if (nx < 4 || ny < 4 || (long long)nx * ny + 4LL * nx >= (1LL << 31)) return bfail(b, EHDLB_EINVAL, "bad lattice size");
    const std::string why = validate(p);
    if (!why.empty()) return bfail(b, EHDLB_EINVAL, why);
    return b->batch->add(nx, ny, *p, id, b->err);
}

int ehdlb_batch_remove(ehdlb_batch *b, int id)
{
    if (!b) return EHDLB_EINVAL;
    return b->batch->remove(id, b->err);
}

int ehdlb_batch_step(ehdlb_batch *b, int nsteps, ehdlb_batch_stats *st)
{
    if (!b || nsteps < 0) return EHDLB_EINVAL;
    if (nsteps == 0) return EHDLB_OK;
    return b->batch->step(nsteps, st, b->err);
}

int ehdlb_batch_get_fields(ehdlb_batch *b, int id, unsigned mask, double *dst, size_t dst_len)
{
    if (!b || !dst) return EHDLB_EINVAL;
    int nx = 0, ny = 0;
    if (b->batch->case_size(id, &nx, &ny) != EHDLB_OK) return bfail(b, EHDLB_EINVAL, "no such case");
    if (mask == 0 || (mask >> EHDLB_NFIELDS) != 0) return bfail(b, EHDLB_EINVAL, "bad field mask");
    int nf = 0;
    for (int f = 0; f < EHDLB_NFIELDS; ++f) nf += (mask >> f) & 1;
    if (dst_len < (size_t)nf * nx * ny) return bfail(b, EHDLB_EINVAL, "dst too small");
    return b->batch->get_fields(id, mask, dst, b->err);
}

int ehdlb_batch_get_state(ehdlb_batch *b, int id, double *dst, size_t len)
{
    if (!b || !dst) return EHDLB_EINVAL;
    int nx = 0, ny = 0;
    if (b->batch->case_size(id, &nx, &ny) != EHDLB_OK) return bfail(b, EHDLB_EINVAL, "no such case");
    if (len < (size_t)35 * nx * ny) return bfail(b, EHDLB_EINVAL, "dst too small");
    return b->batch->get_state(id, dst, b->err);
}

int ehdlb_batch_deformation(ehdlb_batch *b, int n, const int *ids, double *D)
{
    if (!b || n < 0 || (n > 0 && (!ids || !D))) return EHDLB_EINVAL;
    if (n == 0) return EHDLB_OK;
    return b->batch->deformation(n, ids, D, b->err);
}

int ehdlb_batch_set_tuning(ehdlb_batch *b, int sweeps_per_launch, int tile_shape, int use_graphs)
{
    if (!b) return EHDLB_EINVAL;
    if (sweeps_per_launch < -1 || sweeps_per_launch == 0 || sweeps_per_launch > 5)
        return bfail(b, EHDLB_EINVAL, "sweeps_per_launch must lie in 1..5 (or -1)");
    if (tile_shape < -1 || tile_shape > 2) return bfail(b, EHDLB_EINVAL, "tile_shape must lie in -1..2");
    if (use_graphs < -1 || use_graphs > 1) return bfail(b, EHDLB_EINVAL, "use_graphs must lie in -1..1");
    return b->batch->set_tuning(sweeps_per_launch, tile_shape, use_graphs);
}

int ehdlb_batch_autotune(ehdlb_batch *b, int steps, int *sweeps_per_launch, int *tile_shape, double *ms_per_step)
{
    if (!b || steps < 1) return EHDLB_EINVAL;
    return b->batch->autotune(steps, sweeps_per_launch, tile_shape, ms_per_step, b->err);
}

int ehdlb_batch_info(const ehdlb_batch *b, int *cases, size_t *bytes_in_use, size_t *capacity)
{
    if (!b) return EHDLB_EINVAL;
    b->batch->info(cases, bytes_in_use, capacity);
    return EHDLB_OK;
}

const char *ehdlb_batch_last_error(const ehdlb_batch *b) { return b ? b->err.c_str() : "null batch"; }

void ehdlb_batch_destroy(ehdlb_batch *b)
{
    if (!b) return;
    delete b->batch;
    delete b;
}

}  // extern "C"
