// ehdlb_noalloc.cu -- ehdlb_potential_noalloc: the potential solve for callers
// that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: code inside an allocator or
// memory-pool callback (an allocation there re-enters the allocator), a host
// process whose device memory is owned and budgeted by another runtime that
// forbids foreign allocations, or a latency-critical loop that must not risk
// the implicit device synchronisation of an allocation.  For them this entry
// point runs the pseudo-time sweeps of the potential equation with every
// intermediate (the swept populations, phi with its ghost rows, psi of the
// previous sweep, the block partial sums of the residual and the sweep
// parity) in one file-scope device array of fixed size.  Every GPU that loads
// this library reserves that array until the process exits.  The caller
// provides the inputs (phi, q) and the outputs (psi, E) in its own device
// memory.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "ehdlb.h"
#include "ehdlb_kernels.cuh"

namespace {

using ehdlb::Control;
using ehdlb::DevP;

constexpr long long kMaxNodes = EHDLB_NOALLOC_MAX_NODES;
constexpr int kBX = 64, kBY = 4;
// Largest block grid of a (64, 4) launch over nx * ny <= kMaxNodes with
// nx, ny >= 4: ceil(nx/64) ceil(ny/4) <= nx ny / 256 + nx / 64 + ny / 4 + 1.
constexpr long long kMaxBlocks = kMaxNodes / 256 + kMaxNodes / 256 + kMaxNodes / 16 + 1;
// Layout in doubles: control block, g (2 buffers x 4 planes), phi with two
// ghost rows, psi of the previous sweep, residual partials (2 per block),
// the final residual.
constexpr long long kCtlDoubles = 32;
constexpr long long kScratchDoubles =
    kCtlDoubles + 8 * kMaxNodes + (kMaxNodes + 2 * (kMaxNodes / 4)) + kMaxNodes + 2 * kMaxBlocks + 8;
static_assert(sizeof(Control) <= kCtlDoubles * sizeof(double), "control block does not fit");

// The scratch array.  Host code must not use this name as an address: it
// obtains the device address with cudaGetSymbolAddress (see scratch_ptr).
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// Cache of the scratch array's device address, one entry per device.  The
// address belongs to the device's current context: a context created anew
// (after cudaDeviceReset, say) loads the module again, possibly elsewhere, so
// each entry also records the unique id of the context it was looked up in,
// read through the driver's cuCtxGetCurrent and cuCtxGetId.  If those two
// cannot be resolved, the entry is keyed by the device alone.
constexpr int kMaxDevices = 64;
struct ScratchEntry {
    double *addr = nullptr;
    unsigned long long ctx_id = 0;
};
ScratchEntry g_scratch[kMaxDevices];
std::mutex g_scratch_mu;

typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);

// Unique id of the calling thread's current context; 0 if no context is
// current.  *known is false if the driver functions could not be resolved.
unsigned long long current_ctx_id(bool *known)
{
    static CtxGetCurrentFn get_cur = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool resolved = false;
    if (!resolved) {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
            qb == cudaDriverEntryPointSuccess) {
            get_cur = reinterpret_cast<CtxGetCurrentFn>(a);
            get_id = reinterpret_cast<CtxGetIdFn>(b);
        }
        resolved = true;
    }
    *known = get_cur && get_id;
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (!*known || get_cur(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

// Address of the scratch array on the current device.  The set-up step: the
// first call on a device (and the first after its context was replaced)
// looks it up with cudaGetSymbolAddress, with that device current; later
// calls reuse it.
cudaError_t scratch_ptr(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    bool known = false;
    const unsigned long long id = current_ctx_id(&known);
    ScratchEntry &ent = g_scratch[dev];
    if (!ent.addr || (known && (id == 0 || ent.ctx_id != id))) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);   // creates the context if none was current
        if (e != cudaSuccess) return e;
        ent.addr = static_cast<double *>(p);
        ent.ctx_id = current_ctx_id(&known);
    }
    *out = ent.addr;
    return cudaSuccess;
}

// phi [ny][nx] -> phi with one mirrored ghost row below and above.
__global__ void k_noalloc_phig(const double *__restrict__ phi, double *__restrict__ phig, int nx, int ny)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const double v = phi[(long long)y * nx + x];
    phig[(long long)(y + 1) * nx + x] = v;
    if (y == 0) phig[x] = v;
    if (y == ny - 1) phig[(long long)(ny + 1) * nx + x] = v;
}

// The initial potential of ehdlb_set_params: the linear profile between the
// electrodes with the non-equilibrium part that makes Eq. 50 give E = -grad
// psi (or psi = 0), stored relative to w_i psi_lin(y).
__global__ void k_noalloc_init_g(const DevP<double> P, double *__restrict__ g, int psi_zero)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const long long nn = P.nn, k = (long long)y * P.nx + x;
    const double w = 1.0 / 6.0;
    if (psi_zero) {
        const double v = -w * ehdlb::psi_lin(P, y);
        for (int i = 0; i < 4; ++i) g[i * nn + k] = v;
    } else {
        g[k] = 0.0;
        g[nn + k] = -P.tau_g * w * P.G;
        g[2 * nn + k] = 0.0;
        g[3 * nn + k] = P.tau_g * w * P.G;
    }
}

// psi and E from the final populations (Eq. 49-50) and the residual
// partials of the last sweep against psi of the sweep before.
__global__ void __launch_bounds__(256) k_noalloc_finish(const DevP<double> P, const double *__restrict__ g,
                                                        const double *__restrict__ psi_prev, int resid,
                                                        double *__restrict__ psi, double *__restrict__ Ex,
                                                        double *__restrict__ Ey, double *__restrict__ part)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    double red[2] = {0.0, 0.0};
    if (x < P.nx && y < P.ny) {
        const long long nn = P.nn, k = (long long)y * P.nx + x;
        const double g1 = g[k], g2 = g[nn + k], g3 = g[2 * nn + k], g4 = g[3 * nn + k];
        const double psit = 1.5 * ((g1 + g3) + (g2 + g4));
        const double ps = psit + ehdlb::psi_lin(P, y);
        psi[k] = ps;
        Ex[k] = 3.0 * (g1 - g3) / P.tau_g;
        Ey[k] = 3.0 * (g2 - g4) / P.tau_g;
        if (resid) {
            const double d = psit - psi_prev[k];
            red[0] = d * d;
            red[1] = ps * ps;
        }
    }
    ehdlb::block_sum_store<double, 2>(red, part);
}

__global__ void __launch_bounds__(256) k_noalloc_residual(const double *__restrict__ part, long long nb,
                                                          double *__restrict__ out)
{
    double tot[2];
    ehdlb::sum_partials<2>(part, nb, tot);
    if (threadIdx.x == 0) *out = tot[1] > 0.0 ? sqrt(tot[0] / tot[1]) : sqrt(tot[0]);
}

}  // namespace

extern "C" int ehdlb_potential_noalloc(int nx, int ny, const ehdlb_params *p, const double *phi,
                                       const double *q, int nsweeps, double *psi, double *Ex, double *Ey,
                                       double *residual, void *cuda_stream)
{
    if (nx < 4 || ny < 4 || (long long)nx * ny > kMaxNodes) return EHDLB_EINVAL;
    if (!p || p->size != sizeof(ehdlb_params) || !phi || !q || !psi || !Ex || !Ey) return EHDLB_EINVAL;
    if (nsweeps < 0 || nsweeps > 100000000) return EHDLB_EINVAL;
    if (!(p->vartheta > 0.0) || !(p->eps_r > 0.0) || !(p->s_free > 0.0 && p->s_free < 2.0)) return EHDLB_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    double *base = nullptr;
    if (scratch_ptr(&base) != cudaSuccess) return EHDLB_ECUDA;

    const long long nn = (long long)nx * ny;
    Control *ctl = reinterpret_cast<Control *>(base);
    double *gbuf[2] = {base + kCtlDoubles, base + kCtlDoubles + 4 * nn};
    double *phig = base + kCtlDoubles + 8 * nn;
    double *psi_prev = phig + nn + 2 * (long long)nx;
    double *part = psi_prev + nn;
    const dim3 blk(kBX, kBY), grid((nx + kBX - 1) / kBX, (ny + kBY - 1) / kBY);
    const long long nb = (long long)grid.x * grid.y;
    double *rout = part + 2 * nb;

    // lattice coefficients of the potential sweep (Eq. 44-50), as the context solver sets them
    DevP<double> d;
    std::memset(&d, 0, sizeof d);
    d.nx = nx;
    d.ny = ny;
    d.nn = nn;
    d.bgk = p->bgk;
    d.side_walls = p->side_walls;
    const double tau_g = 0.5 + 3.0 * p->vartheta;
    d.tau_g = tau_g;
    d.s_g = 1.0 / tau_g;
    d.s_free_g = p->bgk ? 1.0 / tau_g : p->s_free;
    d.src_norm = p->vartheta * (p->psi_src_literal ? 1.0 : 1.5);
    d.Kq = p->Kq;
    d.er1 = p->eps_r - 1.0;
    d.src_a = d.src_norm * p->Kq / 3.0;
    d.src_b = d.src_norm * (p->eps_r - 1.0) / tau_g;
    d.psi_a = p->psi_anode;
    d.psi_c = p->psi_cathode;
    d.G = (p->psi_cathode - p->psi_anode) / ny;
    d.wG = (p->psi_cathode - p->psi_anode) / ny / 6.0;

    // the scratch keeps the previous call's contents: the control block (sweep
    // parity) starts at zero, every other region is written before it is read
    if (cudaMemsetAsync(ctl, 0, sizeof(Control), s) != cudaSuccess) return EHDLB_ECUDA;
    k_noalloc_phig<<<grid, blk, 0, s>>>(phi, phig, nx, ny);
    k_noalloc_init_g<<<grid, blk, 0, s>>>(d, gbuf[0], p->init_psi_zero);
    for (int j = 1; j <= nsweeps; ++j) {
        if (j == nsweeps)
            ehdlb::k_sweep<double, double, true, false, false>
                <<<grid, blk, 0, s>>>(d, gbuf[0], gbuf[1], phig, q, psi_prev, part, ctl, j);
        else
            ehdlb::k_sweep<double, double, false, false, false>
                <<<grid, blk, 0, s>>>(d, gbuf[0], gbuf[1], phig, q, psi_prev, part, ctl, j);
    }
    k_noalloc_finish<<<grid, blk, 0, s>>>(d, gbuf[nsweeps & 1], psi_prev, nsweeps >= 1 ? 1 : 0, psi, Ex, Ey,
                                          part);
    k_noalloc_residual<<<1, 256, 0, s>>>(part, nb, rout);
    if (cudaGetLastError() != cudaSuccess) return EHDLB_ECUDA;
    if (residual) {
        double r = 0.0;
        if (cudaMemcpyAsync(&r, rout, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return EHDLB_ECUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return EHDLB_ECUDA;
        *residual = nsweeps >= 1 ? r : NAN;
    }
    return EHDLB_OK;
}
