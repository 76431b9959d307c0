// ehdlb_kernels.cuh -- sm_103a kernels of one time step of the phase-field
// lattice Boltzmann EHD method (arXiv 2501.04920, Sec. 4).
//
// Storage (structure of arrays, one plane of nx*ny values per population):
//   f  : 8 planes, f1..f8 of Eq. 25.  f0 is never stored: with the zero-mass
//        equilibrium of Eq. 52 the rest population only feeds the zeroth moment
//        sum f, and neither u (Eq. 56), p (Eq. 57) nor any other population
//        depends on that moment (the moment basis of Eq. 28 is a tensor product
//        of {1, c, c^2}, so only f0 reads m00).
//   h  : 9 planes (Eq. 27) stored as h_i - w_i phi_ref: the deviation from the
//        rest state of a fixed reference field phi_ref (the initial profile).
//        phi = phi_ref + dphi with dphi = sum of the stored values, and the
//        reference's gradient and chemical potential are evaluated once, in
//        double; near equilibrium the chemical potential of Eq. 13 is a small
//        residual of O(1) terms, which float cannot resolve from phi ~ 1 itself.
//   p, n : 5 planes each (Eq. 34-35, D2Q5), or 9 each on D2Q9 (QI = 9).
//   g  : 4 planes, g1..g4 of Eq. 44, stored as g_i - w_i psi_lin(y) where
//        psi_lin is the linear profile between the electrodes; g0 is not
//        stored (psi (Eq. 49) and E (Eq. 50) do not read it, and the diagonal
//        relaxation of N (Eq. 46) keeps the other moments free of it).  The
//        shift keeps the small first moment that carries E (Eq. 50) from
//        drowning in the rounding of psi ~ 1.
//   f, h, p, n are double-buffered by time step and g by sweep; every
//   kernel reads its node's own populations and pushes post-collision values
//   to the neighbours (x periodic, walls half-way below row 0 and above row
//   ny - 1).
// Storage type S of the populations f, h, p, n and of (phi u)(t-1) is T
// itself or, with T = float, __half: each value is then stored as its
// deviation from a rest state (h as above, p and n as w_i c_ref) times a
// power-of-two scale per field that keeps it in the normal range of FP16;
// the arithmetic stays in T.  g and every other plane are T: the potential
// is relaxed by a few sweeps per step, and rounding g to FP16 at every
// sweep would feed its slowest modes faster than the sweeps damp them.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace ehdlb {

// ---- lattice constants (Eq. 25, Eq. 26) -----------------------------------

__host__ __device__ constexpr int cx9(int i)
{
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy9(int i)
{
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp9(int i)
{
    return i == 0 ? 0 : (i < 5 ? ((i + 1) % 4) + 1 : ((i - 5 + 2) % 4) + 5);
}
template <typename T> __host__ __device__ constexpr T w9(int i)
{
    return i == 0 ? T(4) / T(9) : (i < 5 ? T(1) / T(9) : T(1) / T(36));
}

// Device-side problem constants, derived once on the host (kernel argument).
template <typename T> struct DevP {
    int nx, ny;
    long long nn;
    int onsager_form, ion_bc, einstein_D, ion_L_term, bgk, freeze_E;
    int side_walls;                // 1: walls left of x = 0 and right of x = nx - 1 (Eq. 64)
    T tau_g, s_g, s_free_g;        // potential rates
    T src_norm;                    // vartheta (Eq. 44) times 1 or 1/(1 - w0)
    T Kq, er1;                     // Kq, eps_r - 1
    T psi_a, psi_c, G, wG;         // electrodes; G = (psi_c - psi_a) / ny, wG = G / 6
    T rho1, eta_v, eta1;           // rho_r - 1, eta_v, eta_r - 1
    T beta, kappa, W, tau_h;       // Eq. 13, Eq. 30
    T nhat_eps2;                   // regularisation of the normal of Eq. 32 (squared)
    T mu_v, mu1, m, D;             // ions
    T k_d, k_r, cb;
    T s_free;
    T Ex_frozen, Ey_frozen;
    // derived constants of the main kernel
    T s_h, sfree_h;                // Allen-Cahn rates (Eq. 30) and the free rate
    T s_f0;                        // 1/tau_f when rho and eta are uniform, else 0
    T s_p0, s_n0;                  // ion rates (Eq. 37) when D is uniform, else 0
    T inv_mu_v, three_over_tau_g, inv_W;
    T src_a, src_b;                // fused sweeps: src_norm Kq / 3, src_norm (eps_r - 1) / tau_g
    unsigned snap_mask;            // fields the step kernel's snapshot writes (bit f: field f)
    unsigned tx_extra;             // test hook: bytes the staged step kernel waits for beyond its copies
    // storage scales (value x sc is stored, stored x isc is the value) and
    // the rest concentration of the stored p, n; 1, 1 and 0 unless S != T
    T sc_f, isc_f, sc_h, isc_h, sc_c, isc_c, sc_g, isc_g, sc_u, isc_u;  // sc_g: g stored as S
    T cref;
};

// Per-run control block in device memory (all kernels of a step read it).
struct Control {
    int cur0;          // g buffer that holds the state at the start of the step
    int done;          // converge mode: no further sweeps this step
    int K;             // sweeps taken by this step
    int flips;         // g buffer swaps of this step (state after it: cur0 + flips)
    int kmin, kmax;
    int early;         // stopped on the residual; r_last already set
    int unstable;      // NaN or Inf seen
    int notconv;       // steps of the current call that hit kmax above tol
    int sweeps_max;    // most sweeps in one step of the current call
    int converge;      // 1: stop rule active
    long long t;       // steps since set_params
    long long tloc;    // step index within the current call
    long long sweeps_total;
    double tol;
    double r_last;
    double r_step;     // residual of the last finished step
    double sum_phi, sum_q;
    int tpar;          // f, h, p, n buffer that holds the state (flipped by k_step_end;
                       // read by the batched kernels, the single-lattice host tracks its own)
    int fault;         // a staged copy did not arrive in time (k_main_tma)
};

// Programmatic dependent launch: a kernel launched as a dependent of the
// previous kernel in its stream may be scheduled before that one finishes; it
// waits here for it (and all its memory operations) before touching memory,
// then lets its own dependents be scheduled.  In a kernel launched without
// that attribute both instructions have no effect.
__device__ __forceinline__ void griddep_begin()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Host: launch kernel k on stream st; dep: as a programmatic dependent of the
// previous kernel in the stream (k must call griddep_begin first), so that it
// may be scheduled while that one drains.  Captured into a graph, the
// dependency becomes a programmatic edge.
template <typename... P, typename... A>
inline cudaError_t launch_k(cudaStream_t st, void (*k)(P...), dim3 grid, dim3 block, size_t smem, bool dep,
                            A &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = dep ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}

// Opens an ehdlb_step call: zeroes its per-call counters (launch: 1 thread).
static __global__ void k_open_call(Control *c)
{
    c->tloc = 0;
    c->sweeps_total = 0;
    c->sweeps_max = 0;
    c->notconv = 0;
    c->unstable = 0;
}

// One allocation of 17 + 2 QI planes (QI = 5 or 9 ion populations): f at +0,
// h at +8 nn, p at +17 nn, n at +(17 + QI) nn.
template <typename S> struct Pops {
    S *f;   // 8 planes
    S *h;   // 9 planes (h_i - w_i phi_ref)
    S *p;   // 5 planes
    S *n;   // 5 planes
};

// ---- storage conversion --------------------------------------------------------

template <typename S, typename T> constexpr bool kSame = std::is_same<S, T>::value;

// Stored value -> T (times the field's isc when S != T).
template <typename S, typename T> __device__ __forceinline__ T lds(const S *p, T isc)
{
    if constexpr (kSame<S, T>) return *p;
    else return __half2float(*p) * isc;
}
// T -> stored value (times the field's sc when S != T, rounded to nearest).
template <typename S, typename T> __device__ __forceinline__ void sts(S *p, T v, T sc)
{
    if constexpr (kSame<S, T>) *p = v;
    else *p = __float2half_rn(v * sc);
}
// Stochastic rounding of the FP16 stores of f, h, p and n.  Rounding to
// nearest makes the error of a quasi-steady population the same at every
// step, so it accumulates linearly over the run; rounding up with
// probability equal to the discarded fraction makes it a zero-mean random
// walk.  The random bits come from a counter-based generator: the 32-bit
// finaliser of MurmurHash3 (Appleby) over (node, step, stream), advanced per
// store by the linear congruential step of Numerical Recipes (1664525,
// 1013904223), whose high bits are used.
__device__ __forceinline__ uint32_t mix32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x85ebca6bu;
    x ^= x >> 13;
    x *= 0xc2b2ae35u;
    x ^= x >> 16;
    return x;
}

struct SRng {
    uint32_t s;
    __device__ __forceinline__ SRng(long long node, long long step, uint32_t stream)
        : s(mix32((uint32_t)node * 0x9e3779b1u ^ mix32((uint32_t)step * 0x632be5abu + stream)))
    {
    }
    __device__ __forceinline__ uint32_t next()
    {
        s = s * 1664525u + 1013904223u;
        return s;
    }
};

// float -> FP16, rounded up in magnitude with probability equal to the
// discarded fraction (r: 32 random bits): 13 random bits are added below the
// 10 mantissa bits that FP16 keeps and the rest is cut off.  Below the normal
// range of FP16 (2^-14) the final conversion rounds the partly randomised
// value to nearest; the storage scales keep typical values above that range.
__device__ __forceinline__ __half f2h_sr(float v, uint32_t r)
{
    const uint32_t b = (__float_as_uint(v) + (r >> 19)) & ~0x1fffu;
    return __float2half_rn(__uint_as_float(b));
}

// T -> stored value as sts, stochastically rounded when S != T.
template <typename S, typename T> __device__ __forceinline__ void sts_sr(S *p, T v, T sc, SRng &rng)
{
    if constexpr (kSame<S, T>) *p = v;
    else *p = f2h_sr(v * sc, rng.next());
}

// Raw stored value -> T without scaling (for sums scaled once).
template <typename S, typename T> __device__ __forceinline__ T raw(S v)
{
    if constexpr (kSame<S, T>) return v;
    else return __half2float(v);
}

// The reference field of the stored h and its derived planes.
template <typename T> struct PhiRef {
    T *phir;   // phi_ref with a mirrored ghost row below and above [(ny+2)][nx]
    T *gxr;    // grad phi_ref by Eq. 59 [ny][nx]
    T *gyr;
    T *mur;    // chemical potential of phi_ref, Eq. 13 [ny][nx]
    T *dphig;  // dphi = phi - phi_ref of the current step, with ghost rows
};

// ---- small helpers ------------------------------------------------------------

template <typename T> __device__ __forceinline__ T dsqrt(T v);
template <> __device__ __forceinline__ double dsqrt<double>(double v) { return sqrt(v); }
template <> __device__ __forceinline__ float dsqrt<float>(float v) { return sqrtf(v); }

template <typename T> __device__ __forceinline__ T bessel_i1(T v);
template <> __device__ __forceinline__ double bessel_i1<double>(double v) { return cyl_bessel_i1(v); }
template <> __device__ __forceinline__ float bessel_i1<float>(float v) { return cyl_bessel_i1f(v); }

// Onsager function F(b) = I1(4b) / (2b) with F(0) = 1 (north of b = 1e-4 the
// CUDA Bessel function, below it the series 1 + 2 b^2, whose next term
// (4/3) b^4 is under 2e-16); form 1 is Eq. 6 with b^2 = gamma E.
template <typename T> __device__ __forceinline__ T onsager(T b, int form)
{
    if (form == 1) return T(1) + T(2) * b * b;
    if (b < T(1e-4)) return T(1) + T(2) * b * b;
    return bessel_i1<T>(T(4) * b) / (T(2) * b);
}

__device__ __forceinline__ int wrapx(int x, int nx)
{
    return x < 0 ? x + nx : (x >= nx ? x - nx : x);
}

// Column of the x neighbour at x + dx (|dx| = 1) for the stencils of
// Eq. 59: periodic, or with side walls the mirrored ghost column (the node
// itself).
__device__ __forceinline__ int nbx(int x, int dx, int nx, int walls)
{
    const int v = x + dx;
    if (walls) return v < 0 ? 0 : (v >= nx ? nx - 1 : v);
    return v < 0 ? v + nx : (v >= nx ? v - nx : v);
}

template <typename T> __device__ __forceinline__ T psi_lin(const DevP<T> &P, int y)
{
    return P.psi_a + P.G * (T(y) + T(0.5));
}

// Deterministic block sum of NV values (fixed tree order), written by thread
// 0 to out[NV * slot].  Each warp sums in T; the warp sums are added in
// double.  blockDim must be a multiple of 32, <= 1024.
template <typename T, int NV> __device__ __forceinline__ void block_sum_store_at(T (&v)[NV], double *out, long long slot)
{
    __shared__ double red[32][NV];
    const int lane = (threadIdx.x + threadIdx.y * blockDim.x) & 31;
    const int warp = (threadIdx.x + threadIdx.y * blockDim.x) >> 5;
    const int nwarp = (blockDim.x * blockDim.y) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        T s = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) red[warp][k] = (double)s;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = lane < nwarp ? red[lane][k] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) out[(size_t)NV * (size_t)slot + k] = s;
        }
    }
}

// The same into the slot of this block of the grid.
template <typename T, int NV> __device__ __forceinline__ void block_sum_store(T (&v)[NV], double *out)
{
    block_sum_store_at<T, NV>(v, out, blockIdx.x + (long long)blockIdx.y * gridDim.x);
}

// Sum NV-wide partials of nb blocks in a fixed order (one block of 256).
template <int NV> __device__ __forceinline__ void sum_partials(const double *part, long long nb,
                                                              double (&tot)[NV])
{
    __shared__ double red[256][NV];
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
    for (long long b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] += part[NV * b + k];
#pragma unroll
    for (int k = 0; k < NV; ++k) red[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
#pragma unroll
            for (int k = 0; k < NV; ++k) red[threadIdx.x][k] += red[threadIdx.x + s][k];
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) tot[k] = red[0][k];
}

// ---- D2Q9 natural moments (Eq. 28) by the tensor product of {1, c, c^2} ------
// Moment order as the rows of Eq. 28: m00 m10 m01 m20 m02 m11 m12 m21 m22
// (first index: power of cx).

template <typename T> __device__ __forceinline__ void moments9(const T (&v)[9], T (&m)[9])
{
    // x-transform of the rows cy = 0, +1, -1
    T a0 = v[3] + v[0] + v[1], a1 = v[1] - v[3], a2 = v[1] + v[3];
    T b0 = v[6] + v[2] + v[5], b1 = v[5] - v[6], b2 = v[5] + v[6];
    T c0 = v[7] + v[4] + v[8], c1 = v[8] - v[7], c2 = v[8] + v[7];
    m[0] = a0 + b0 + c0;
    m[1] = a1 + b1 + c1;
    m[2] = b0 - c0;
    m[3] = a2 + b2 + c2;
    m[4] = b0 + c0;
    m[5] = b1 - c1;
    m[6] = b1 + c1;
    m[7] = b2 - c2;
    m[8] = b2 + c2;
}

template <typename T> __device__ __forceinline__ void inverse9(const T (&m)[9], T (&v)[9])
{
    // y-inverse for each x-moment k: row cy=+1 (b), cy=-1 (c), cy=0 (a)
    const T h = T(0.5);
    T b0 = h * (m[2] + m[4]), c0 = h * (m[4] - m[2]), a0 = m[0] - m[4];
    T b1 = h * (m[5] + m[6]), c1 = h * (m[6] - m[5]), a1 = m[1] - m[6];
    T b2 = h * (m[7] + m[8]), c2 = h * (m[8] - m[7]), a2 = m[3] - m[8];
    v[0] = a0 - a2; v[1] = h * (a1 + a2); v[3] = h * (a2 - a1);
    v[2] = b0 - b2; v[5] = h * (b1 + b2); v[6] = h * (b2 - b1);
    v[4] = c0 - c2; v[8] = h * (c1 + c2); v[7] = h * (c2 - c1);
}

// Asynchronous 4- or 8-byte global -> shared copy (no register staging).
template <typename T> __device__ __forceinline__ void cp_async(T *smem, const T *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
// Asynchronous 16-byte global -> shared copy; both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
// Asynchronous copy of two consecutive elements; both addresses aligned to
// twice the element size.
template <typename T> __device__ __forceinline__ void cp_async_pair(T *smem, const T *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ---- kernels -----------------------------------------------------------------

// phi = sum h (Eq. 33) with mirrored ghost rows, q = sum p - sum n.  The
// stored h are deviations from w_i phi_ref: dphi = their sum, phi = phi_ref
// + dphi; both are written (phi for the potential, dphi for the stencils of
// the main kernel).  With init_ctl the first thread also opens the step in
// the control block.
// VN consecutive values from an address aligned to VN elements, as one load.
template <int VN, typename V> struct alignas(sizeof(V) * VN) VecN { V v[VN]; };
template <int VN, typename V> __device__ __forceinline__ void ld_n(const V *a, V (&o)[VN])
{
    const VecN<VN, V> u = *reinterpret_cast<const VecN<VN, V> *>(a);
#pragma unroll
    for (int j = 0; j < VN; ++j) o[j] = u.v[j];
}
template <int VN, typename V> __device__ __forceinline__ void st_n(V *a, const V (&o)[VN])
{
    VecN<VN, V> u;
#pragma unroll
    for (int j = 0; j < VN; ++j) u.v[j] = o[j];
    *reinterpret_cast<VecN<VN, V> *>(a) = u;
}

// Body of k_prep for the block at (bx, by) of the lattice's grid: each
// thread takes VN consecutive nodes of a row (VN > 1 needs nx % VN == 0, so
// every plane offset is aligned to VN elements), each node computed alone.
template <typename T, typename S, int QI = 5, int VN = 1>
__device__ __forceinline__ void prep_body(const DevP<T> &P, const S *__restrict__ h, const S *__restrict__ p,
                                          const S *__restrict__ n, const PhiRef<T> &R, T *__restrict__ phig,
                                          T *__restrict__ q, Control *ctl, int fixedK, int kmin, int kmax,
                                          int flips, int bx, int by)
{
    const int x = (bx * blockDim.x + threadIdx.x) * VN;
    const int y = by * blockDim.y + threadIdx.y;
    if (bx == 0 && by == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        if (fixedK >= 0) {
            ctl->K = fixedK; ctl->flips = flips; ctl->done = 1; ctl->converge = 0;
        } else {
            ctl->K = 0; ctl->flips = 0; ctl->done = (kmax <= 0); ctl->converge = 1;
        }
        ctl->kmin = kmin; ctl->kmax = kmax; ctl->early = 0; ctl->r_last = nan("");
    }
    if (x >= P.nx || y >= P.ny) return;
    const long long nn = P.nn, k = (long long)y * P.nx + x;
    S hv[9][VN], pv[QI][VN], nv[QI][VN];
#pragma unroll
    for (int i = 0; i < 9; ++i) ld_n<VN>(h + i * nn + k, hv[i]);
#pragma unroll
    for (int i = 0; i < QI; ++i) {
        ld_n<VN>(p + i * nn + k, pv[i]);
        ld_n<VN>(n + i * nn + k, nv[i]);
    }
    const long long gk = (long long)(y + 1) * P.nx + x;
    T pr[VN], ph[VN], dd[VN], qq[VN];
    ld_n<VN>(R.phir + gk, pr);
#pragma unroll
    for (int j = 0; j < VN; ++j) {
        // pairwise: rest, axis pairs, diagonal pairs
        T d = raw<S, T>(hv[0][j]) +
              ((((raw<S, T>(hv[1][j]) + raw<S, T>(hv[3][j])) + (raw<S, T>(hv[2][j]) + raw<S, T>(hv[4][j])))) +
               ((raw<S, T>(hv[5][j]) + raw<S, T>(hv[7][j])) + (raw<S, T>(hv[6][j]) + raw<S, T>(hv[8][j]))));
        T sp = T(0), sn = T(0);
#pragma unroll
        for (int i = 0; i < QI; ++i) { sp += raw<S, T>(pv[i][j]); sn += raw<S, T>(nv[i][j]); }
        T qv = sp - sn;   // the rest concentrations of stored p and n cancel
        if constexpr (!kSame<S, T>) { d *= P.isc_h; qv *= P.isc_c; }
        dd[j] = d;
        ph[j] = pr[j] + d;
        qq[j] = qv;
    }
    st_n<VN>(phig + gk, ph);
    st_n<VN>(R.dphig + gk, dd);
    if (y == 0) {
        st_n<VN>(phig + x, ph);
        st_n<VN>(R.dphig + x, dd);
    }
    if (y == P.ny - 1) {
        st_n<VN>(phig + (long long)(P.ny + 1) * P.nx + x, ph);
        st_n<VN>(R.dphig + (long long)(P.ny + 1) * P.nx + x, dd);
    }
    st_n<VN>(q + k, qq);
}

// Launch: blockDim (64, 4) over the lattice, VN nodes per thread along x.
template <typename T, typename S, int QI = 5, int VN = 1>
__global__ void __launch_bounds__(256) k_prep(const DevP<T> P, const S *__restrict__ h,
                                              const S *__restrict__ p, const S *__restrict__ n,
                                              const PhiRef<T> R, T *__restrict__ phig, T *__restrict__ q,
                                              Control *ctl, int fixedK, int kmin, int kmax, int flips)
{
    griddep_begin();
    prep_body<T, S, QI, VN>(P, h, p, n, R, phig, q, ctl, fixedK, kmin, kmax, flips, blockIdx.x, blockIdx.y);
}

// One pseudo-time sweep of the potential (Eq. 44-50) at every node: E and
// psi from the node's own populations, the variable-permittivity source
// (Kq q - grad eps . E) / eps, MRT collision with N (Eq. 46), push to the
// neighbours with anti-bounce-back to the electrode potentials.
//   WRITE_PSI: store psi (shifted) for the residual of the next sweep/main.
//   RESID    : partial sums of (psi - psi_prev)^2 and psi^2 (FP64).
//   CTRL     : converge mode; skip if the step is done, parity from K.
template <typename T, typename S, bool WRITE_PSI, bool RESID, bool CTRL>
__global__ void __launch_bounds__(256) k_sweep(const DevP<T> P, S *__restrict__ gA,
                                               S *__restrict__ gB, const T *__restrict__ phig,
                                               const T *__restrict__ q, T *__restrict__ psi_prev,
                                               double *__restrict__ part, const Control *__restrict__ ctl,
                                               int j)
{
    if (CTRL && ctl->done) return;
    const int par = (ctl->cur0 + j - 1) & 1;
    const S *__restrict__ src = par ? gB : gA;
    S *__restrict__ dst = par ? gA : gB;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    double red[2] = {0.0, 0.0};
    if (x < P.nx && y < P.ny) {
        const int nx = P.nx;
        const long long nn = P.nn, k = (long long)y * nx + x;
        const T g1 = lds(src + k, P.isc_g), g2 = lds(src + nn + k, P.isc_g), g3 = lds(src + 2 * nn + k, P.isc_g),
                g4 = lds(src + 3 * nn + k, P.isc_g);
        const T psit = T(1.5) * ((g1 + g3) + (g2 + g4));      // Eq. 49, minus psi_lin
        if (RESID) {
            const double d = (double)psit - (double)psi_prev[k];
            const double ps = (double)psit + (double)psi_lin(P, y);
            red[0] = d * d;
            red[1] = ps * ps;
        }
        if (WRITE_PSI) psi_prev[k] = psit;
        // grad phi by Eq. 59 (only grad eps enters the potential)
        const int xm = nbx(x, -1, nx, P.side_walls), xp = nbx(x, 1, nx, P.side_walls);
        const T *r0 = phig + (long long)y * nx, *r1 = r0 + nx, *r2 = r1 + nx;
        const T phi = r1[x];
        const T gx = (r1[xp] - r1[xm]) * T(1.0 / 3.0) +
                     ((r2[xp] - r2[xm]) + (r0[xp] - r0[xm])) * T(1.0 / 12.0);
        const T gy = (r2[x] - r0[x]) * T(1.0 / 3.0) +
                     ((r2[xp] + r2[xm]) - (r0[xp] + r0[xm])) * T(1.0 / 12.0);
        const T m1 = g1 - g3, m2 = g2 - g4;
        const T Ex = T(3) * m1 / P.tau_g, Ey = T(3) * m2 / P.tau_g;  // Eq. 50
        const T eps = T(1) + P.er1 * phi;
        const T rt = (P.Kq * q[k] - P.er1 * (gx * Ex + gy * Ey)) / eps;
        const T X3 = P.src_norm * rt * T(1.0 / 3.0);                // w_i source, 2nd moments
        const T eq = psit * T(1.0 / 3.0);
        const T m3 = g1 + g3, m4 = g2 + g4;
        const T n1 = (T(1) - P.s_g) * m1, n2 = (T(1) - P.s_g) * m2;
        const T n3 = m3 - P.s_free_g * (m3 - eq) + X3;
        const T n4 = m4 - P.s_free_g * (m4 - eq) + X3;
        const T o1 = T(0.5) * (n3 + n1), o3 = T(0.5) * (n3 - n1);
        const T o2 = T(0.5) * (n4 + n2), o4 = T(0.5) * (n4 - n2);
        // side walls: bounce-back (zero normal gradient of psi, Eq. 64)
        if (P.side_walls && x == nx - 1) sts(dst + 2 * nn + k, o1, P.sc_g);
        else sts(dst + (long long)y * nx + wrapx(x + 1, nx), o1, P.sc_g);
        if (P.side_walls && x == 0) sts(dst + k, o3, P.sc_g);
        else sts(dst + 2 * nn + (long long)y * nx + wrapx(x - 1, nx), o3, P.sc_g);
        if (y + 1 < P.ny) sts(dst + nn + k + nx, o2 - P.wG, P.sc_g);
        else sts(dst + 3 * nn + k, -o2 + P.wG, P.sc_g);          // cathode: ABB to psi_c
        if (y > 0) sts(dst + 3 * nn + k - nx, o4 + P.wG, P.sc_g);
        else sts(dst + nn + k, -o4 - P.wG, P.sc_g);              // anode: ABB to psi_a
    }
    if (RESID) block_sum_store<double, 2>(red, part);
}


// NSW potential sweeps (Eq. 44-50) fused in shared memory.  A block holds an
// RW x RH region of the lattice: its output tile of (RW - 2 NSW) x
// (RH - 2 NSW) nodes plus a halo NSW nodes wide (x periodic; rows outside the
// lattice stay empty, the electrode rules act on the wall links).  Every
// sweep collides and pushes the whole region; values at distance < s from
// the region edge are incomplete after sweep s, so after NSW sweeps the
// output tile is exact.  The four population planes are stored in a moving
// frame: after s sweeps the population g_i of node (lx, ly) sits at
// (lx, ly) - s c_i, so the value a node pushes to its neighbour lands in the
// cell the node itself has just read.  Every thread therefore reads and
// writes the same four cells per node and a sweep needs one block barrier;
// the planes moving along x are NSW cells wider, those moving along y NSW
// cells taller.  An electrode link writes the bounced value into the node's
// own cell of the opposite plane for the next sweep.  The source
// coefficients of each node stay in registers: X/3 = A - Bx m1 - By m2 with
// m1, m2 the first moments (E = 3 m / tau_g), A = th Kq q / (3 eps),
// B = th (eps_r - 1) grad phi / (tau_g eps), th = vartheta (times 1/(1 - w0)).
//   FIRST: first launch of the step; the coefficients come from phi (with
//          its ring of neighbours) and q, and the output tile's are written
//          to coef (three planes A, Bx, By) for the later launches, which
//          load them instead.
//   RESID: the last sweep of the step; residual partials of the output tile.
// Launch: blockDim (32, BY), dynamic shared memory
// tb_smem_bytes<T, RW, RH>(FIRST) (sized for up to TB_NSW_MAX sweeps).
// Source coefficients of Eq. 44 at a node for the fused sweeps, from phi,
// q and grad phi (Eq. 59): A = th Kq q / (3 eps), (Bx, By) = th (eps_r - 1)
// grad phi / (tau_g eps), eps = 1 + (eps_r - 1) phi.
template <typename T>
__device__ __forceinline__ void src_coefs(const DevP<T> &P, T phi, T q, T gx, T gy, T &A, T &Bx, T &By)
{
    const T inv = T(1) / (T(1) + P.er1 * phi);
    const T bb = P.src_b * inv;
    A = P.src_a * q * inv;
    Bx = bb * gx;
    By = bb * gy;
}

constexpr int TB_NSW_MAX = 5;
template <typename T, int RW, int RH> __host__ __device__ constexpr size_t tb_smem_bytes(bool first)
{
    return sizeof(T) * ((size_t)2 * RH * (RW + TB_NSW_MAX) + (size_t)2 * (RH + TB_NSW_MAX) * RW +
                        (first ? (size_t)(RH + 2) * (RW + 2) + (size_t)RH * RW : 0));
}

// x mod nx for x within one lattice width of [0, nx) (wide == true) or any x.
__device__ __forceinline__ int wrap_x(int x, int nx, bool wide)
{
    if (wide) return x < 0 ? x + nx : (x >= nx ? x - nx : x);
    return ((x % nx) + nx) % nx;
}

// Body of k_sweep_tb for the block at (bx, by) of the lattice's tile grid;
// slot: its residual partials.
template <typename T, typename S, int NSW, int RW, int RH, int BY, bool FIRST, bool RESID>
__device__ __forceinline__ void tb_body(const DevP<T> &P, S *__restrict__ gA, S *__restrict__ gB,
                                        const T *__restrict__ phig, const T *__restrict__ q, T *__restrict__ coef,
                                        double *__restrict__ part, const Control *__restrict__ ctl, int m, int bx,
                                        int by, long long slot)
{
    constexpr int H = NSW, TX = RW - 2 * H, TY = RH - 2 * H;
    constexpr int W1 = RW + H;                    // width of the planes moving along x
    constexpr int P1 = RH * W1, P2 = (RH + H) * RW;
    constexpr int FW = RW + 2;                    // phi with its one-node ring
    constexpr int NB = RW / 32, NA = RH / BY;
    static_assert(RW % 32 == 0 && RH % BY == 0, "region must tile the block");
    static_assert(TX > 0 && TY > 0 && NA >= 1 && H <= TB_NSW_MAX, "tile too small for NSW");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // planes g1 (+x), g3 (-x), g2 (+y), g4 (-y); then (FIRST) phi ring and q
    T *const s1 = reinterpret_cast<T *>(smem_raw);
    T *const s3 = s1 + P1, *const s2 = s1 + 2 * P1, *const s4 = s2 + P2;
    T *const sphi = s4 + P2, *const sq = sphi + (RH + 2) * FW;
    const int par = (ctl->cur0 + m) & 1;
    const S *__restrict__ src = par ? gB : gA;
    S *__restrict__ dst = par ? gA : gB;
    const int nx = P.nx, ny = P.ny;
    const long long nn = P.nn;
    const int x0 = bx * TX, y0 = by * TY;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const bool wide = nx >= RW + 2;

    int gxs[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) gxs[b] = wrap_x(x0 - H + tx + 32 * b, nx, wide);

    // ---- load the region: g (async) into the frame of sweep 0; the
    // coefficients from coef into registers, or (FIRST) phi with a one-node
    // ring and q (async) ----
    T cA[NA][NB], cBx[NA][NB], cBy[NA][NB];
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const int ly = ty + BY * a, gy = y0 - H + ly;
#pragma unroll
        for (int b = 0; b < NB; ++b) cA[a][b] = cBx[a][b] = cBy[a][b] = T(0);
        if (FIRST && gy >= -1 && gy <= ny) {   // phi of this node (the ghost rows included)
#pragma unroll
            for (int b = 0; b < NB; ++b)
                cp_async(sphi + (ly + 1) * FW + tx + 32 * b + 1, phig + (long long)(gy + 1) * nx + gxs[b]);
        }
        if (gy < 0 || gy >= ny) continue;
        const long long row = (long long)gy * nx;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int lx = tx + 32 * b;
            const long long k = row + gxs[b];
            T *c1 = s1 + ly * W1 + lx + H, *c3 = s3 + ly * W1 + lx, *c2 = s2 + (ly + H) * RW + lx,
              *c4 = s4 + ly * RW + lx;
            if constexpr (kSame<S, T>) {
                cp_async(c1, src + k);
                cp_async(c2, src + nn + k);
                cp_async(c3, src + 2 * nn + k);
                cp_async(c4, src + 3 * nn + k);
            } else {
                *c1 = lds(src + k, P.isc_g);
                *c2 = lds(src + nn + k, P.isc_g);
                *c3 = lds(src + 2 * nn + k, P.isc_g);
                *c4 = lds(src + 3 * nn + k, P.isc_g);
            }
            if (FIRST) {
                cp_async(sq + ly * RW + lx, q + k);
            } else {
                cA[a][b] = coef[k];
                cBx[a][b] = coef[nn + k];
                cBy[a][b] = coef[2 * nn + k];
            }
        }
    }
    if (FIRST) {
        // the ring of phi around the region: the rows below and above it
        // (2 FW cells), then its left and right columns (2 RH cells); phig
        // holds the rows -1 .. ny
        constexpr int NR = 2 * FW + 2 * RH;
        for (int e = tx + 32 * ty; e < NR; e += 32 * BY) {
            int py, px;
            if (e < 2 * FW) {
                py = e < FW ? 0 : RH + 1;
                px = e < FW ? e : e - FW;
            } else {
                const int c = e - 2 * FW;
                py = 1 + (c < RH ? c : c - RH);
                px = c < RH ? 0 : RW + 1;
            }
            const int gy = y0 - H - 1 + py;
            if (gy < -1 || gy > ny) continue;
            const int gx = wrap_x(x0 - H - 1 + px, nx, wide);
            cp_async(sphi + py * FW + px, phig + (long long)(gy + 1) * nx + gx);
        }
    }
    cp_async_wait_all();
    // every thread reads the cells of sweep 0 it copied itself; the ring of
    // phi was copied by all threads
    if (FIRST) {
        __syncthreads();
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            const int ly = ty + BY * a, gy = y0 - H + ly;
            if (gy < 0 || gy >= ny) continue;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int lx = tx + 32 * b;
                const T *r1 = sphi + (ly + 1) * FW + lx + 1, *r0 = r1 - FW, *r2 = r1 + FW;
                const T phi = r1[0];
                const T gxs_ = (r1[1] - r1[-1]) * T(1.0 / 3.0) +
                               ((r2[1] - r2[-1]) + (r0[1] - r0[-1])) * T(1.0 / 12.0);
                const T gys_ = (r2[0] - r0[0]) * T(1.0 / 3.0) +
                               ((r2[1] + r2[-1]) - (r0[1] + r0[-1])) * T(1.0 / 12.0);
                src_coefs(P, phi, sq[ly * RW + lx], gxs_, gys_, cA[a][b], cBx[a][b], cBy[a][b]);
            }
        }
    }

    T psi_before[NA][NB];
    // half of the collision constants: o = 0.5 (n3 +- n1) etc.
    const T k1 = T(0.5) * (T(1) - P.s_g);            // first moments
    const T kf = T(0.5) * (T(1) - P.s_free_g);       // second moments
    const T ke = T(0.25) * P.s_free_g;               // their equilibrium psi/3, psi = 1.5 (m3 + m4)
    const T wG = P.wG;
    const bool interior = y0 - H >= 0 && y0 - H + RH <= ny;
#pragma unroll
    for (int s = 0; s < NSW; ++s) {
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            const int ly = ty + BY * a, gy = y0 - H + ly;
            if (!interior && (gy < 0 || gy >= ny)) continue;
            const bool top = !interior && gy + 1 >= ny, bot = !interior && gy == 0;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int lx = tx + 32 * b;
                // this node's cells after s sweeps
                T *c1 = s1 + ly * W1 + lx - s + H, *c3 = s3 + ly * W1 + lx + s;
                T *c2 = s2 + (ly - s + H) * RW + lx, *c4 = s4 + (ly + s) * RW + lx;
                const T g1 = *c1, g2 = *c2, g3 = *c3, g4 = *c4;
                const T m1 = g1 - g3, m2 = g2 - g4, m3 = g1 + g3, m4 = g2 + g4;
                if (RESID) psi_before[a][b] = T(1.5) * (m3 + m4);
                const T X6 = T(0.5) * (cA[a][b] - cBx[a][b] * m1 - cBy[a][b] * m2);
                const T e = ke * (m3 + m4) + X6;                 // half of s psi/3 + X/3
                const T h3 = kf * m3 + e, h4 = kf * m4 + e;      // half of n3, n4
                const T h1 = k1 * m1, h2 = k1 * m2;              // half of n1, n2
                const T p2 = h4 + h2, p4 = h4 - h2;
                *c1 = h3 + h1;
                *c3 = h3 - h1;
                if (top) c4[RW] = -p2 + wG;         // cathode: ABB to psi_c, this node's g4 next sweep
                else *c2 = p2 - wG;
                if (bot) c2[-RW] = -p4 - wG;        // anode: ABB to psi_a, this node's g2 next sweep
                else *c4 = p4 + wG;
            }
        }
        __syncthreads();
    }

    // ---- store the output tile (and, FIRST, its coefficients) ----
    T red[2] = {T(0), T(0)};
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const int ly = ty + BY * a, gy = y0 - H + ly;
        if (ly < H || ly >= H + TY || gy >= ny) continue;
        const long long row = (long long)gy * nx;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int lx = tx + 32 * b, gx = x0 - H + lx;
            if (lx < H || lx >= H + TX || gx >= nx) continue;
            const long long k = row + gx;
            // cells after NSW = H sweeps
            const T g1 = s1[ly * W1 + lx], g3 = s3[ly * W1 + lx + H];
            const T g2 = s2[ly * RW + lx], g4 = s4[(ly + H) * RW + lx];
            sts(dst + k, g1, P.sc_g);
            sts(dst + nn + k, g2, P.sc_g);
            sts(dst + 2 * nn + k, g3, P.sc_g);
            sts(dst + 3 * nn + k, g4, P.sc_g);
            if (FIRST) {
                coef[k] = cA[a][b];
                coef[nn + k] = cBx[a][b];
                coef[2 * nn + k] = cBy[a][b];
            }
            if (RESID) {
                const T psit = T(1.5) * ((g1 + g3) + (g2 + g4));
                const T d = psit - psi_before[a][b];
                const T ps = psit + psi_lin(P, gy);
                red[0] += d * d;
                red[1] += ps * ps;
            }
        }
    }
    if (RESID) block_sum_store_at<T, 2>(red, part, slot);
}

template <typename T, typename S, int NSW, int RW, int RH, int BY, int MINB, bool FIRST, bool RESID>
__global__ void __launch_bounds__(32 * BY, MINB)
    k_sweep_tb(const DevP<T> P, S *__restrict__ gA, S *__restrict__ gB, const T *__restrict__ phig,
               const T *__restrict__ q, T *__restrict__ coef, double *__restrict__ part,
               const Control *__restrict__ ctl, int m)
{
    tb_body<T, S, NSW, RW, RH, BY, FIRST, RESID>(P, gA, gB, phig, q, coef, part, ctl, m, blockIdx.x, blockIdx.y,
                                                 blockIdx.x + (long long)blockIdx.y * gridDim.x);
}

// a * b + c rounded once.
template <typename T> __device__ __forceinline__ T fma_t(T a, T b, T c)
{
    if constexpr (sizeof(T) == 4) return __fmaf_rn(a, b, c);
    else return __fma_rn(a, b, c);
}

// (a0 + c, a1 + c), each rounded once; one packed instruction on FP32.
template <typename T> __device__ __forceinline__ void add_pair(T &d0, T &d1, T a0, T a1, T c)
{
    if constexpr (sizeof(T) == 4) {
        const float2 v = __fadd2_rn(make_float2(a0, a1), make_float2(c, c));
        d0 = v.x;
        d1 = v.y;
    } else {
        d0 = a0 + c;
        d1 = a1 + c;
    }
}

// ---- register-blocked fused sweeps ----------------------------------------------

// The NSW fused sweeps of tb_body on 64 x 8R regions, computed in registers
// by a persistent block (blockDim (32, NW)) that walks the tiles of the grid:
// lane l of warp w holds the nodes 2l and 2l + 1 of the region rows
// wR .. wR + R - 1, their four populations and their source coefficients.
// After each collision the populations moving along x cross lanes by one
// warp shuffle per node (lane 0's left and lane 31's right neighbours are
// outside the region: those cells are incomplete, as is every cell at
// distance < s from the region edge after s sweeps); those moving along y
// stay in the thread between its own rows and cross to the warps above and
// below through shared memory, one row per band edge, double buffered by
// sweep parity, so a sweep needs one block barrier.  While a tile is swept,
// the next one is copied to shared memory (cp.async), each thread copying
// the cells it will read itself.  Collision, electrode links, FIRST and
// RESID as in tb_body (except that the coefficient planes hold halves of A,
// Bx, By here); the residual partials go to the tile's slot.  The
// region's left and right halos are HL = NSW rounded up to even nodes, so a
// lane's two nodes sit at an even lattice column: for even nx they are one
// aligned 8-byte pair in every plane, copied and stored as one.
template <typename T> struct Vec2T;
template <> struct Vec2T<float> { using type = float2; };
template <> struct Vec2T<double> { using type = double2; };

__host__ __device__ constexpr int tbr_halo_x(int nsw) { return nsw + (nsw & 1); }

// Planes of one staged tile (NW warps, bands of R rows): g1..g4 and A, Bx,
// By, or (FIRST) g1..g4, q and phi with its one-node ring.
// phi with its ring is kept in rows of 68: region column lx at lx + 2, so a
// lane's node pair is 8-byte aligned there too.
constexpr int TBR_FW = 68;
template <typename T, int R, int NW> __host__ __device__ constexpr size_t tbr_smem_bytes(bool first)
{
    return sizeof(T) * (first ? (size_t)5 * NW * R * 64 + (size_t)(NW * R + 2) * TBR_FW : (size_t)7 * NW * R * 64);
}

// One tile of the register-blocked sweeps: its lattice (constants, g buffer
// read and written, phi with ghost rows, q, the coefficient planes, the
// residual partials and the tile's slot in them) and its first output node.
template <typename T> struct TbrTile {
    const DevP<T> *P;
    const T *src;
    T *dst;
    const T *phig, *q;
    T *coef;
    double *part;
    long long slot;
    int x0, y0;
    // fused prep (the first launch computes phi and q itself): the h, p, n
    // planes of the time level, phi_ref and dphi (both with ghost rows)
    const T *h, *pp, *pn, *phir;
    T *dphig;
    int ry0;   // lattice row of the region's first row
    int oy1;   // end of the output rows [y0, oy1)
    int carry; // walk: the row below the region was the previous tile's (its upward flux is carried)
    int strip; // walk: the tile's strip of columns
};

// Rows of tile row ty of a lattice of ny rows for regions of RH rows and H
// sweeps.  An edge of a region that lies on an electrode wall needs no halo
// (the wall links are exact inside the region), so the first tile row takes
// the region [0, RH) and outputs [0, RH - H), the last [ny - RH, ny) and
// outputs its last rows, and the rows between take TY = RH - 2 H rows of
// output from regions with H rows of halo on both sides; a lattice of at
// most RH rows is one region.  Returns the region's first row and sets the
// output rows [*oy0, *oy1).
__host__ __device__ inline int tbr_rows(int ty, int ny, int RH, int H, int *oy0, int *oy1)
{
    const int TY = RH - 2 * H;
    if (ny <= RH) {
        *oy0 = 0;
        *oy1 = ny;
        return 0;
    }
    const int edge = RH - H, mid = ny - 2 * edge > 0 ? (ny - 2 * edge + TY - 1) / TY : 0;
    if (ty == 0) {
        *oy0 = 0;
        *oy1 = edge;
        return 0;
    }
    if (ty <= mid) {
        *oy0 = edge + (ty - 1) * TY;
        *oy1 = *oy0 + TY;
        return *oy0 - H;
    }
    *oy0 = edge + mid * TY;
    *oy1 = ny;
    return ny - RH;
}
// Tile rows of that partition.
__host__ __device__ inline int tbr_tile_rows(int ny, int RH, int H)
{
    const int TY = RH - 2 * H, edge = RH - H;
    if (ny <= RH) return 1;
    return 2 + (ny - 2 * edge > 0 ? (ny - 2 * edge + TY - 1) / TY : 0);
}

// Walking order of the register-blocked sweeps: the lattice is cut into
// strips of TX output columns, and the strips, bottom to top and one after
// another, form one sequence of nstrips x ny rows, of which block b of G
// takes the rows [b T / G, (b + 1) T / G).  A block walks its rows upward in
// regions of RH rows.  Potential populations cross a row upward only through
// g2 (Eq. 44-50, D2Q5), so a region that starts right above the rows the
// previous region output needs no halo below: the post-collision g2 of the
// row under it, at every sweep, is the one the previous region computed
// there (valid at every sweep, H rows below that region's top), carried in
// shared memory.  Such a region outputs its RH - H lowest rows; a region
// that starts at the electrode wall needs no halo below either; a block's
// first region elsewhere takes a halo of H rows below and outputs RH - 2 H
// rows; a region that reaches the top wall outputs up to it.  Each tile
// reports its partials of the residual into the block's slot.
template <typename T> struct TbrWalkTiles {
    const DevP<T> *P;
    const T *src;
    T *dst;
    const T *phig, *q;
    T *coef;
    double *part;
    int nstrips;
    int RH, H, TX;
    int p1;   // end of this block's rows in the sequence (nstrips ny < 2^31)
    __device__ void at(TbrTile<T> &t, int strip, int row, bool carry) const
    {
        t = TbrTile<T>{P, src, dst, phig, q, coef, part, (long long)blockIdx.x, strip * TX, row};
        const int ny = P->ny;
        t.carry = carry;
        t.strip = strip;
        t.ry0 = carry ? row : (row > H ? row - H : 0);   // at most H rows from the wall: start at it
        int oy1 = t.ry0 + RH >= ny ? ny : t.ry0 + RH - H;
        const int pend = p1 - strip * ny;   // the block's end in this strip's rows
        if (pend < oy1) oy1 = pend;
        t.oy1 = oy1;
    }
    __device__ bool begin(TbrTile<T> &t)
    {
        const int ny = P->ny;
        const long long T_ = (long long)nstrips * ny;
        const int p0 = (int)(T_ * blockIdx.x / gridDim.x);
        p1 = (int)(T_ * (blockIdx.x + 1) / gridDim.x);
        if (p0 >= p1) return false;
        const int strip = p0 / ny;
        at(t, strip, p0 - strip * ny, false);
        return true;
    }
    // the tile after t (which it overwrites); false at the block's end
    __device__ bool next(TbrTile<T> &t) const
    {
        const int ny = P->ny;
        if (t.strip * ny + t.oy1 >= p1) return false;
        if (t.oy1 >= ny) at(t, t.strip + 1, 0, false);
        else at(t, t.strip, t.oy1, true);
        return true;
    }
};

// The tiles of one lattice, tiles_x per row, row by row; src / dst: the g
// buffers the launch reads and writes.
template <typename T> struct TbrLatticeTiles {
    const DevP<T> *P;
    const T *src;
    T *dst;
    const T *phig, *q;
    T *coef;
    double *part;
    int tiles_x, ntiles;
    const T *h = nullptr, *pp = nullptr, *pn = nullptr, *phir = nullptr;
    T *dphig = nullptr;
    __device__ int count() const { return ntiles; }
    __device__ TbrTile<T> tile(int t, int TX, int TY, int H) const
    {
        int oy0, oy1;
        const int ry0 = tbr_rows(t / tiles_x, P->ny, TY + 2 * H, H, &oy0, &oy1);
        return TbrTile<T>{P, src, dst,  phig, q,     coef, part, t,   (t % tiles_x) * TX, oy0,
                          h, pp,  pn,   phir, dphig, ry0,  oy1};
    }
};

// The persistent loop over the tiles J gives (count(), tile(i, TX, TY)).
// Launch: blockDim (32, NW), dynamic shared memory tbr_smem_bytes<T, R, NW>(FIRST),
// grid = min(tiles, resident blocks).
// FPREP (with FIRST): the launch also does the prep pass of the step for its
// tiles: phi = phi_ref + sum h (Eq. 33) and q = sum p - sum n of every region
// node and of the one-node ring from the populations, in the order prep_body
// sums them (so the coefficients are the same bits), and writes dphi of its
// output nodes (with the mirrored ghost rows).
template <typename T, int NSW, int R, int NW, bool FIRST, bool RESID, bool FPREP = false, bool WALK = false,
          typename Tiles>
__device__ __forceinline__ void tbr_run(Tiles &J)
{
    using V2 = typename Vec2T<T>::type;
    constexpr int H = NSW, HL = tbr_halo_x(NSW), RW = 64, RH = NW * R, TX = RW - 2 * HL,
                  TY = RH - 2 * H;
    constexpr int FW = TBR_FW, PL = RH * RW;
    static_assert(TX > 0 && TY > 0 && H <= TB_NSW_MAX, "region too small for NSW");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *const stg = reinterpret_cast<T *>(smem_raw);           // planes of the staged tile
    T *const sphi = stg + 5 * PL;                               // FIRST: phi with its ring
    __shared__ __align__(16) T xup[2][NW][RW];   // p2 of each warp's top row, for the warp above
    __shared__ __align__(16) T xdn[2][NW][RW];   // p4 of each warp's bottom row, for the warp below
    // walk: p2 of the carried row (local row RH - H - 1) at each sweep, by tile parity
    __shared__ __align__(16) T carry[WALK ? 2 : 1][WALK ? NSW : 1][RW];
    constexpr int CW = (RH - H - 1) / R, CR = (RH - H - 1) % R;   // its warp and row in the warp
    const int lane = threadIdx.x, w = threadIdx.y;
    const int lx0 = 2 * lane, ly0 = w * R;
    static_assert(!FPREP || FIRST, "the prep pass is fused into the first launch of a step");
    constexpr int NPL = FIRST ? (FPREP ? 4 : 5) : 7;

    // copy tile tl to the stage: this thread's own cells (zeros outside the
    // lattice rows), and (FIRST) a share of phi with its ring
    auto issue = [&](const TbrTile<T> &tl) {
        const int nx = tl.P->nx, ny = tl.P->ny;
        const long long nn = tl.P->nn;
        const bool wide = nx >= RW + 2;
        const bool pairs = (nx & 1) == 0;   // a lane's two nodes are one aligned pair
        const T *__restrict__ phig = tl.phig;
        // plane pl of the staged inputs: g1..g4, then q or A, Bx, By
        auto plane = [&](int pl) -> const T * {
            return pl < 4 ? tl.src + pl * nn : (FIRST ? tl.q : tl.coef + (pl - 4) * nn);
        };
        const int x0 = tl.x0, ry = tl.ry0;
        const int gx = wrap_x(x0 - HL + lx0, nx, wide);
        const int gx1 = pairs ? gx + 1 : wrap_x(x0 - HL + lx0 + 1, nx, wide);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int gy = ry + ly0 + r;
            T *c = stg + (ly0 + r) * RW + lx0;
            if (gy < 0 || gy >= ny) {
#pragma unroll
                for (int pl = 0; pl < NPL; ++pl) *reinterpret_cast<V2 *>(c + pl * PL) = V2{T(0), T(0)};
                continue;
            }
            const int k = gy * nx + gx, k1 = gy * nx + gx1;   // < nn <= 2^31
            if (pairs) {
#pragma unroll
                for (int pl = 0; pl < NPL; ++pl) cp_async_pair(c + pl * PL, plane(pl) + k);
            } else {
#pragma unroll
                for (int pl = 0; pl < NPL; ++pl) {
                    cp_async(c + pl * PL, plane(pl) + k);
                    cp_async(c + pl * PL + 1, plane(pl) + k1);
                }
            }
        }
        if (FIRST && !FPREP) {
            // phi (phig holds the rows -1 .. ny): this thread's node pairs,
            // then the ring (rows -1 and RH, columns -1 and 64) by all
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int gy = ry + ly0 + r;
                T *c = sphi + (ly0 + r + 1) * FW + lx0 + 2;
                if (gy < -1 || gy > ny) {
                    *reinterpret_cast<V2 *>(c) = V2{T(0), T(0)};
                    continue;
                }
                const T *row = phig + (long long)(gy + 1) * nx;
                if (pairs) {
                    cp_async_pair(c, row + gx);
                } else {
                    cp_async(c, row + gx);
                    cp_async(c + 1, row + gx1);
                }
            }
            constexpr int NRING = 2 * (RW + 2) + 2 * RH;
            for (int e = lane + 32 * w; e < NRING; e += 32 * NW) {
                int ly, lx;
                if (e < 2 * (RW + 2)) {
                    ly = e < RW + 2 ? -1 : RH;
                    lx = (e < RW + 2 ? e : e - (RW + 2)) - 1;
                } else {
                    const int c = e - 2 * (RW + 2);
                    ly = c < RH ? c : c - RH;
                    lx = c < RH ? -1 : RW;
                }
                const int gy = ry + ly;
                T *d = sphi + (ly + 1) * FW + lx + 2;
                if (gy >= -1 && gy <= ny)
                    cp_async(d, phig + (long long)(gy + 1) * nx + wrap_x(x0 - HL + lx, nx, wide));
                else
                    *d = T(0);
            }
        }
    };

    T k1, kf, ke, wG;   // collision constants of the current tile's lattice
    int ny;
    int sw = 0;         // sweeps done by this block: parity of the exchange rows

    // NSW sweeps of the tile in registers; EDGE: the region reaches an
    // electrode row (block-uniform), which adds the wall links.  ch = half of
    // the coefficients A, Bx, By (exact), so X/6 = chA - chBx m1 - chBy m2.
    auto sweeps = [&](auto edge, int gy0, T (&g1)[R][2], T (&g2)[R][2], T (&g3)[R][2], T (&g4)[R][2],
                      const T (&chA)[R][2], const T (&chBx)[R][2], const T (&chBy)[R][2], T (&psi_before)[R][2],
                      bool carry_in, int cpar) {
        constexpr bool EDGE = decltype(edge)::value;
#pragma unroll
        for (int s = 0; s < NSW; ++s, ++sw) {
            T o1[R][2], o3[R][2], p2[R][2], p4[R][2];
            if constexpr (sizeof(T) == 4) {
                // The same collision on the lane's node pair with packed FP32
                // operations (each element rounded once, as by the scalar
                // form).  The signs sit on exact operands: n1 = g3 - g1 and
                // n2 = g4 - g2 are -m1 and -m2 bit for bit, so every product
                // and sum below equals its scalar counterpart.
                const float2 K1 = make_float2(k1, k1), NK1 = make_float2(-k1, -k1);
                const float2 KF = make_float2(kf, kf), KE = make_float2(ke, ke);
                const float2 N1 = make_float2(-1.f, -1.f);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float2 G1 = make_float2(g1[r][0], g1[r][1]), G2 = make_float2(g2[r][0], g2[r][1]);
                    const float2 G3 = make_float2(g3[r][0], g3[r][1]), G4 = make_float2(g4[r][0], g4[r][1]);
                    const float2 n1 = __ffma2_rn(G1, N1, G3), n2 = __ffma2_rn(G2, N1, G4);
                    const float2 m3 = __fadd2_rn(G1, G3), m4 = __fadd2_rn(G2, G4);
                    const float2 m34 = __fadd2_rn(m3, m4);
                    if (RESID) {
                        const float2 pb = __fmul2_rn(make_float2(1.5f, 1.5f), m34);
                        psi_before[r][0] = pb.x;
                        psi_before[r][1] = pb.y;
                    }
                    const float2 X6 = __ffma2_rn(make_float2(chBy[r][0], chBy[r][1]), n2,
                                                 __ffma2_rn(make_float2(chBx[r][0], chBx[r][1]), n1,
                                                            make_float2(chA[r][0], chA[r][1])));
                    const float2 e = __ffma2_rn(KE, m34, X6);
                    const float2 h3 = __ffma2_rn(KF, m3, e), h4 = __ffma2_rn(KF, m4, e);
                    const float2 O1 = __ffma2_rn(NK1, n1, h3), O3 = __ffma2_rn(K1, n1, h3);
                    const float2 P2 = __ffma2_rn(NK1, n2, h4), P4 = __ffma2_rn(K1, n2, h4);
                    o1[r][0] = O1.x;
                    o1[r][1] = O1.y;
                    o3[r][0] = O3.x;
                    o3[r][1] = O3.y;
                    p2[r][0] = P2.x;
                    p2[r][1] = P2.y;
                    p4[r][0] = P4.x;
                    p4[r][1] = P4.y;
                }
            } else {
#pragma unroll
            for (int r = 0; r < R; ++r) {
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const T m1 = g1[r][j] - g3[r][j], m2 = g2[r][j] - g4[r][j];
                    const T m3 = g1[r][j] + g3[r][j], m4 = g2[r][j] + g4[r][j];
                    const T m34 = m3 + m4;
                    if (RESID) psi_before[r][j] = T(1.5) * m34;
                    const T X6 = fma_t(-chBy[r][j], m2, fma_t(-chBx[r][j], m1, chA[r][j]));
                    const T e = fma_t(ke, m34, X6);
                    const T h3 = fma_t(kf, m3, e), h4 = fma_t(kf, m4, e);   // halves of n3, n4
                    o1[r][j] = fma_t(k1, m1, h3);
                    o3[r][j] = fma_t(-k1, m1, h3);
                    p2[r][j] = fma_t(k1, m2, h4);
                    p4[r][j] = fma_t(-k1, m2, h4);
                }
            }
            }
            const int b = sw & 1;
            *reinterpret_cast<V2 *>(&xup[b][w][lx0]) = V2{p2[R - 1][0], p2[R - 1][1]};
            if constexpr (WALK) {
                if (w == CW) *reinterpret_cast<V2 *>(&carry[cpar][s][lx0]) = V2{p2[CR][0], p2[CR][1]};
            }
            *reinterpret_cast<V2 *>(&xdn[b][w][lx0]) = V2{p4[0][0], p4[0][1]};
#pragma unroll
            for (int r = 0; r < R; ++r) {
                g1[r][1] = o1[r][0];
                g1[r][0] = __shfl_up_sync(0xffffffffu, o1[r][1], 1);
                g3[r][0] = o3[r][1];
                g3[r][1] = __shfl_down_sync(0xffffffffu, o3[r][0], 1);
                if (r > 0) add_pair(g2[r][0], g2[r][1], p2[r - 1][0], p2[r - 1][1], -wG);
                if (r < R - 1) add_pair(g4[r][0], g4[r][1], p4[r + 1][0], p4[r + 1][1], wG);
            }
            __syncthreads();
            if (w > 0) {
                const V2 v = *reinterpret_cast<const V2 *>(&xup[b][w - 1][lx0]);
                add_pair(g2[0][0], g2[0][1], v.x, v.y, -wG);
            } else if (WALK && carry_in) {   // the previous tile's row below, at this sweep
                const V2 v = *reinterpret_cast<const V2 *>(&carry[cpar ^ 1][s][lx0]);
                add_pair(g2[0][0], g2[0][1], v.x, v.y, -wG);
            } else {
                g2[0][0] = g2[0][1] = T(0);   // below the region
            }
            if (w < NW - 1) {
                const V2 v = *reinterpret_cast<const V2 *>(&xdn[b][w + 1][lx0]);
                add_pair(g4[R - 1][0], g4[R - 1][1], v.x, v.y, wG);
            } else {
                g4[R - 1][0] = g4[R - 1][1] = T(0);   // above the region
            }
            if (EDGE) {
                // electrodes: ABB of the wall links into the node's own cell
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int gy = gy0 + r;
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        if (gy == 0) g2[r][j] = -p4[r][j] - wG;        // anode, psi_a
                        if (gy == ny - 1) g4[r][j] = -p2[r][j] + wG;   // cathode, psi_c
                    }
                }
            }
        }
    };

    TbrTile<T> cur;
    bool have;
    int t = blockIdx.x, ntiles = 0;
    if constexpr (WALK) {
        have = J.begin(cur);
    } else {
        ntiles = J.count();
        have = t < ntiles;
        if (have) cur = J.tile(t, TX, TY, H);
    }
    if (have) issue(cur);
    T racc[2] = {T(0), T(0)};   // walk: the block's residual partials over its tiles
    for (int ck = 0; have; ++ck) {
        const DevP<T> &P = *cur.P;
        const int nx = P.nx;
        const long long nn = P.nn;
        const bool pairs = (nx & 1) == 0;
        ny = P.ny;
        k1 = T(0.5) * (T(1) - P.s_g);
        kf = T(0.5) * (T(1) - P.s_free_g);
        ke = T(0.25) * P.s_free_g;
        wG = P.wG;
        const int x0 = cur.x0, ry = cur.ry0, oy0 = cur.y0, oy1 = cur.oy1;
        const int gy0 = ry + ly0;   // lattice row of this thread's row 0
        cp_async_wait_all();
        T g1[R][2], g2[R][2], g3[R][2], g4[R][2], cA[R][2], cBx[R][2], cBy[R][2];
        if constexpr (FPREP) {
            // phi of the region and its ring from the populations
            const bool wide = nx >= RW + 2;
            auto node = [&](int gy, int gx, T &d, T &qv) {
                const long long kk = (long long)gy * nx + gx;
                const T *hp = cur.h + kk;
                d = hp[0] + ((((hp[nn] + hp[3 * nn]) + (hp[2 * nn] + hp[4 * nn]))) +
                             ((hp[5 * nn] + hp[7 * nn]) + (hp[6 * nn] + hp[8 * nn])));
                T sp = T(0), sn = T(0);
#pragma unroll
                for (int i = 0; i < 5; ++i) { sp += cur.pp[i * nn + kk]; sn += cur.pn[i * nn + kk]; }
                qv = sp - sn;
            };
            const int gxA = wrap_x(x0 - HL + lx0, nx, wide);
            const int gxB = pairs ? gxA + 1 : wrap_x(x0 - HL + lx0 + 1, nx, wide);
            const int gxo = x0 - HL + lx0;
            const bool xout = lx0 >= HL && lx0 < HL + TX && gxo < nx;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int gy = gy0 + r, ly = ly0 + r;
                T *c = sphi + (ly + 1) * TBR_FW + lx0 + 2;
                T qA = T(0), qB = T(0);
                if (gy >= -1 && gy <= ny) {
                    const int ry = gy < 0 ? 0 : (gy >= ny ? ny - 1 : gy);   // the ghost rows mirror
                    T dA, dB, qa, qb;
                    node(ry, gxA, dA, qa);
                    node(ry, gxB, dB, qb);
                    const T *pr = cur.phir + (long long)(gy + 1) * nx;
                    c[0] = pr[gxA] + dA;
                    c[1] = pr[gxB] + dB;
                    if (gy >= 0 && gy < ny) {
                        qA = qa;
                        qB = qb;
                        if (xout && gy >= oy0 && gy < oy1) {
                            // dphi of the output nodes and of the ghost rows they mirror into
                            T *drow = cur.dphig + (long long)(gy + 1) * nx;
                            drow[gxo] = dA;
                            if (gxo + 1 < nx) drow[gxo + 1] = dB;
                            if (gy == 0) {
                                cur.dphig[gxo] = dA;
                                if (gxo + 1 < nx) cur.dphig[gxo + 1] = dB;
                            }
                            if (gy == ny - 1) {
                                T *top = cur.dphig + (long long)(ny + 1) * nx;
                                top[gxo] = dA;
                                if (gxo + 1 < nx) top[gxo + 1] = dB;
                            }
                        }
                    }
                } else {
                    c[0] = T(0);
                    c[1] = T(0);
                }
                cA[r][0] = qA;
                cA[r][1] = qB;
            }
            constexpr int NRING = 2 * (RW + 2) + 2 * RH;
            for (int e = lane + 32 * w; e < NRING; e += 32 * NW) {
                int ly, lx;
                if (e < 2 * (RW + 2)) {
                    ly = e < RW + 2 ? -1 : RH;
                    lx = (e < RW + 2 ? e : e - (RW + 2)) - 1;
                } else {
                    const int c = e - 2 * (RW + 2);
                    ly = c < RH ? c : c - RH;
                    lx = c < RH ? -1 : RW;
                }
                const int gy = ry + ly;
                T *dd = sphi + (ly + 1) * TBR_FW + lx + 2;
                if (gy >= -1 && gy <= ny) {
                    const int ry = gy < 0 ? 0 : (gy >= ny ? ny - 1 : gy);
                    const int gx = wrap_x(x0 - HL + lx, nx, wide);
                    T d, qv;
                    node(ry, gx, d, qv);
                    *dd = cur.phir[(long long)(gy + 1) * nx + gx] + d;
                } else {
                    *dd = T(0);
                }
            }
            __syncthreads();      // phi of the region and ring written by all
        } else if (FIRST) {
            __syncthreads();      // phi was copied by all threads
        }

#pragma unroll
        for (int r = 0; r < R; ++r) {
            const T *c = stg + (ly0 + r) * RW + lx0;
            auto ld2 = [&](int pl, T(&v)[R][2]) {
                const V2 u = *reinterpret_cast<const V2 *>(c + pl * PL);
                v[r][0] = u.x;
                v[r][1] = u.y;
            };
            ld2(0, g1);
            ld2(1, g2);
            ld2(2, g3);
            ld2(3, g4);
            if (FIRST) {
                if (!FPREP) ld2(4, cA);   // q until the coefficients are formed
            } else {
                ld2(4, cA);
                ld2(5, cBx);
                ld2(6, cBy);
            }
        }
        if (FIRST) {
            // the coefficients from phi: columns lx0 - 1 .. lx0 + 2 of the
            // rows around each of this thread's rows, read once per row
            T win[3][4];
            auto ldrow = [&](int ly, T(&v)[4]) {
                const T *c = sphi + (ly + 1) * FW + lx0 + 1;
                const V2 u = *reinterpret_cast<const V2 *>(c + 1);
                v[0] = c[0];
                v[1] = u.x;
                v[2] = u.y;
                v[3] = c[3];
            };
            ldrow(ly0 - 1, win[0]);
            ldrow(ly0, win[1]);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                ldrow(ly0 + r + 1, win[(r + 2) % 3]);
                const T(&w0)[4] = win[r % 3];
                const T(&w1)[4] = win[(r + 1) % 3];
                const T(&w2)[4] = win[(r + 2) % 3];
                const int gy = gy0 + r;
                const bool in = gy >= 0 && gy < ny;
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    // r0, r1, r2: the rows below, at and above; [j + 1] is the node
                    const T phi = w1[j + 1];
                    const T gxs_ = (w1[j + 2] - w1[j]) * T(1.0 / 3.0) +
                                   ((w2[j + 2] - w2[j]) + (w0[j + 2] - w0[j])) * T(1.0 / 12.0);
                    const T gys_ = (w2[j + 1] - w0[j + 1]) * T(1.0 / 3.0) +
                                   ((w2[j + 2] + w2[j]) - (w0[j + 2] + w0[j])) * T(1.0 / 12.0);
                    T a, bx, by;
                    src_coefs(P, phi, cA[r][j], gxs_, gys_, a, bx, by);
                    cA[r][j] = in ? a : T(0);
                    cBx[r][j] = in ? bx : T(0);
                    cBy[r][j] = in ? by : T(0);
                }
            }
            __syncthreads();      // phi read by all before it is refilled
        }
        TbrTile<T> nxt = cur;
        bool more;
        if constexpr (WALK) {
            more = J.next(nxt);
        } else {
            more = t + (int)gridDim.x < ntiles;
            if (more) nxt = J.tile(t + gridDim.x, TX, TY, H);
        }
        if (more) issue(nxt);

        // halves of the coefficients (exact); the first launch stores them
        // so that the later ones load halves
        T chA[R][2], chBx[R][2], chBy[R][2], psi_before[R][2];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const T f = FIRST ? T(0.5) : T(1);
                chA[r][j] = f * cA[r][j];
                chBx[r][j] = f * cBx[r][j];
                chBy[r][j] = f * cBy[r][j];
            }
        const bool cin = WALK && cur.carry;
        if (ry <= 0 || ry + RH >= ny)
            sweeps(std::true_type{}, gy0, g1, g2, g3, g4, chA, chBx, chBy, psi_before, cin, ck & 1);
        else
            sweeps(std::false_type{}, gy0, g1, g2, g3, g4, chA, chBx, chBy, psi_before, cin, ck & 1);

        // ---- the output tile (and, FIRST, its coefficients); lx0 and HL
        // are even, so a lane's two nodes are both in the tile or both out ----
        T red[2] = {T(0), T(0)};
        const int gxo = x0 - HL + lx0;
        const bool xin = lx0 >= HL && lx0 < HL + TX && gxo < nx;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int ly = ly0 + r, gy = gy0 + r;
            if (!xin || gy < oy0 || gy >= oy1 || gy >= ny) continue;
            const int k = gy * nx + gxo;
            auto st2 = [&](T *base, const T(&v)[R][2]) {
                if (pairs) {
                    *reinterpret_cast<V2 *>(base + k) = V2{v[r][0], v[r][1]};
                } else {
                    base[k] = v[r][0];
                    if (gxo + 1 < nx) base[k + 1] = v[r][1];
                }
            };
            st2(cur.dst, g1);
            st2(cur.dst + nn, g2);
            st2(cur.dst + 2 * nn, g3);
            st2(cur.dst + 3 * nn, g4);
            if (FIRST) {
                st2(cur.coef, chA);
                st2(cur.coef + nn, chBx);
                st2(cur.coef + 2 * nn, chBy);
            }
            if (RESID) {
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    if (j == 1 && gxo + 1 >= nx) continue;
                    const T psit = T(1.5) * ((g1[r][j] + g3[r][j]) + (g2[r][j] + g4[r][j]));
                    const T d = psit - psi_before[r][j];
                    const T ps = psit + psi_lin(P, gy);
                    red[0] += d * d;
                    red[1] += ps * ps;
                }
            }
        }
        if constexpr (RESID) {
            if constexpr (WALK) {
                racc[0] += red[0];
                racc[1] += red[1];
            } else {
                block_sum_store_at<T, 2>(red, cur.part, cur.slot);
            }
        }
        cur = nxt;
        have = more;
        t += gridDim.x;
    }
    if constexpr (WALK && RESID) block_sum_store_at<T, 2>(racc, J.part, (long long)blockIdx.x);
    cp_async_wait_all();
}

template <typename T, int NSW, int R, int NW, int MINB, bool FIRST, bool RESID>
__global__ void __launch_bounds__(32 * NW, MINB)
    k_sweep_tbr(const __grid_constant__ DevP<T> P, T *__restrict__ gA, T *__restrict__ gB,
                const T *__restrict__ phig, const T *__restrict__ q, T *__restrict__ coef,
                double *__restrict__ part, const Control *__restrict__ ctl, int m, int tiles_x, int ntiles)
{
    griddep_begin();
    const int par = (ctl->cur0 + m) & 1;
    TbrLatticeTiles<T> J{&P, par ? gB : gA, par ? gA : gB, phig, q, coef, part, tiles_x, ntiles};
    tbr_run<T, NSW, R, NW, FIRST, RESID>(J);
}

// The register-blocked sweeps in the walking order (TbrWalkTiles): grid =
// resident blocks, each walking its share of the strip rows; residual
// partials in one slot per block.
template <typename T, int NSW, int R, int NW, int MINB, bool FIRST, bool RESID>
__global__ void __launch_bounds__(32 * NW, MINB)
    k_sweep_tbw(const __grid_constant__ DevP<T> P, T *__restrict__ gA, T *__restrict__ gB,
                const T *__restrict__ phig, const T *__restrict__ q, T *__restrict__ coef,
                double *__restrict__ part, const Control *__restrict__ ctl, int m, int nstrips)
{
    const int par = (ctl->cur0 + m) & 1;
    constexpr int H = NSW, HL = tbr_halo_x(NSW), RH = NW * R;
    TbrWalkTiles<T> J{&P, par ? gB : gA, par ? gA : gB, phig, q, coef, part, nstrips, RH, H, 64 - 2 * HL, 0};
    tbr_run<T, NSW, R, NW, FIRST, RESID, false, true>(J);
}

// The first sweep launch of a step with the prep pass fused (tbr_run FPREP):
// reads h, p, n of the step's time level instead of the prep kernel's phi
// and q, writes dphi for the step kernel, and opens the step in the control
// block (fixed sweep count K, flips g buffer swaps) as the prep kernel does.
template <typename T, int NSW, int R, int NW, int MINB, bool RESID>
__global__ void __launch_bounds__(32 * NW, MINB)
    k_sweep_tbr_fp(const __grid_constant__ DevP<T> P, T *__restrict__ gA, T *__restrict__ gB,
                   const T *__restrict__ h, const T *__restrict__ pp, const T *__restrict__ pn,
                   const T *__restrict__ phir, T *__restrict__ dphig, T *__restrict__ coef,
                   double *__restrict__ part, Control *__restrict__ ctl, int tiles_x, int ntiles, int fixedK,
                   int flips)
{
    griddep_begin();
    const int par = ctl->cur0 & 1;   // the first launch of the step (m = 0)
    if (blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        ctl->K = fixedK; ctl->flips = flips; ctl->done = 1; ctl->converge = 0;
        ctl->kmin = fixedK; ctl->kmax = fixedK; ctl->early = 0; ctl->r_last = nan("");
    }
    TbrLatticeTiles<T> J{&P, par ? gB : gA, par ? gA : gB, nullptr, nullptr, coef, part, tiles_x, ntiles};
    J.h = h;
    J.pp = pp;
    J.pn = pn;
    J.phir = phir;
    J.dphig = dphig;
    tbr_run<T, NSW, R, NW, true, RESID, true>(J);
}

// ---- thread-block clusters -------------------------------------------------------

__device__ __forceinline__ unsigned cluster_ctaid_x()
{
    unsigned v;
    asm volatile("mov.u32 %0, %%cluster_ctaid.x;" : "=r"(v));
    return v;
}
__device__ __forceinline__ unsigned cluster_ctaid_y()
{
    unsigned v;
    asm volatile("mov.u32 %0, %%cluster_ctaid.y;" : "=r"(v));
    return v;
}
__device__ __forceinline__ unsigned cluster_ctarank()
{
    unsigned v;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(v));
    return v;
}
// All threads of all CTAs of the cluster; shared-memory writes before it
// (local or remote) are visible to every CTA after it.
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Shared-memory address of the same offset in CTA `rank` of the cluster.
__device__ __forceinline__ unsigned map_shared(unsigned local, unsigned rank)
{
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_cluster(unsigned addr, float v)
{
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void st_cluster(unsigned addr, double v)
{
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}

// NSW potential sweeps (Eq. 44-50) by a cluster of CX x CY CTAs that
// together hold a (CX 64) x (CY 32) region of the lattice, each CTA a 64 x 32
// part of it.  Populations that cross from one CTA's part into another's are
// written straight into the neighbour's shared memory, and the cluster
// synchronises once per sweep, so only the cluster region needs a halo: NSW
// nodes at its outer edge, after which its output tile of
// (CX 64 - 2 NSW) x (CY 32 - 2 NSW) nodes is exact.  Two buffers of four
// planes: sweep s reads buffer s mod 2 and writes the other one, so that the
// barrier after sweep s also orders every read of the buffer that sweep s + 1
// writes.  The other rules (empty rows outside the lattice, electrode links,
// periodic x, coefficients in registers, FIRST and RESID) are those of
// k_sweep_tb.
// Launch: grid (CX ceil(nx / TX), CY ceil(ny / TY)) with TX = CX 64 - 2 NSW,
// TY = CY 32 - 2 NSW, blockDim (32, BY), cluster (CX, CY), dynamic shared
// memory tb_cl_smem_bytes<T>().
template <typename T> __host__ __device__ constexpr size_t tb_cl_smem_bytes()
{
    return sizeof(T) * 8 * (size_t)(32 + 2) * (64 + 2);
}

template <typename T, int NSW, int CX, int CY, int BY, bool FIRST, bool RESID>
__global__ void __cluster_dims__(CX, CY, 1) __launch_bounds__(32 * BY, 3)
    k_sweep_cl(const DevP<T> P, T *__restrict__ gA, T *__restrict__ gB, const T *__restrict__ phig,
               const T *__restrict__ q, T *__restrict__ coef, double *__restrict__ part,
               const Control *__restrict__ ctl, int m)
{
    constexpr int RW = 64, RH = 32, H = NSW;
    constexpr int CW = CX * RW, CH = CY * RH, TX = CW - 2 * H, TY = CH - 2 * H;
    constexpr int PW = RW + 2, PH = RH + 2, PL = PW * PH;
    constexpr int NB = RW / 32, NA = RH / BY;
    static_assert(RH % BY == 0 && TX > 0 && TY > 0, "cluster too small for NSW");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *sg = reinterpret_cast<T *>(smem_raw);   // [2][4][PH][PW]
    const int par = (ctl->cur0 + m) & 1;
    const T *__restrict__ src = par ? gB : gA;
    T *__restrict__ dst = par ? gA : gB;
    const int nx = P.nx, ny = P.ny;
    const long long nn = P.nn;
    const int cx = (int)cluster_ctaid_x(), cy = (int)cluster_ctaid_y();
    const unsigned rank = cluster_ctarank();
    const int X0 = (blockIdx.x / CX) * TX - H, Y0 = (blockIdx.y / CY) * TY - H;   // cluster region origin
    const int x0 = X0 + cx * RW, y0 = Y0 + cy * RH;                               // this CTA's part
    const int tx = threadIdx.x, ty = threadIdx.y;
    const bool wide = nx >= CW + 2;
    // neighbours in the cluster (rank x-fastest); a missing one maps to itself
    const unsigned sbase = (unsigned)__cvta_generic_to_shared(sg);
    const bool has_r = cx < CX - 1, has_l = cx > 0, has_u = cy < CY - 1, has_d = cy > 0;
    const unsigned base_r = map_shared(sbase, has_r ? rank + 1 : rank);
    const unsigned base_l = map_shared(sbase, has_l ? rank - 1 : rank);
    const unsigned base_u = map_shared(sbase, has_u ? rank + CX : rank);
    const unsigned base_d = map_shared(sbase, has_d ? rank - CX : rank);

    int gxs[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) gxs[b] = wrap_x(x0 + tx + 32 * b, nx, wide);

    // ---- load this CTA's part: g into buffer 0, coefficients or (FIRST)
    // phi with its ring and q into planes 0 and 1 of buffer 1 ----
    T cA[NA][NB], cBx[NA][NB], cBy[NA][NB];
    T *const sphi = sg + 4 * PL, *const sq = sg + 5 * PL;
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const int ly = ty + BY * a, gy = y0 + ly;
#pragma unroll
        for (int b = 0; b < NB; ++b) cA[a][b] = cBx[a][b] = cBy[a][b] = T(0);
        if (gy < 0 || gy >= ny) continue;
        const long long row = (long long)gy * nx;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const long long k = row + gxs[b];
            const int li = (ly + 1) * PW + tx + 32 * b + 1;
#pragma unroll
            for (int i = 0; i < 4; ++i) cp_async(sg + i * PL + li, src + i * nn + k);
            if (FIRST) {
                cp_async(sq + li, q + k);
            } else {
                cA[a][b] = coef[k];
                cBx[a][b] = coef[nn + k];
                cBy[a][b] = coef[2 * nn + k];
            }
        }
    }
    if (FIRST) {
        for (int e = tx + 32 * ty; e < PL; e += 32 * BY) {
            const int py = e / PW, px = e - py * PW;
            const int gy = y0 - 1 + py;
            if (gy < -1 || gy > ny) continue;
            const int gx = wrap_x(x0 - 1 + px, nx, wide);
            cp_async(sphi + e, phig + (long long)(gy + 1) * nx + gx);
        }
    }
    cp_async_wait_all();
    __syncthreads();
    if (FIRST) {
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            const int ly = ty + BY * a, gy = y0 + ly;
            if (gy < 0 || gy >= ny) continue;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int li = (ly + 1) * PW + tx + 32 * b + 1;
                const T *r1 = sphi + li, *r0 = r1 - PW, *r2 = r1 + PW;
                const T phi = r1[0];
                const T gxs_ = (r1[1] - r1[-1]) * T(1.0 / 3.0) +
                               ((r2[1] - r2[-1]) + (r0[1] - r0[-1])) * T(1.0 / 12.0);
                const T gys_ = (r2[0] - r0[0]) * T(1.0 / 3.0) +
                               ((r2[1] + r2[-1]) - (r0[1] + r0[-1])) * T(1.0 / 12.0);
                src_coefs(P, phi, sq[li], gxs_, gys_, cA[a][b], cBx[a][b], cBy[a][b]);
            }
        }
    }
    // every CTA has loaded (and read its staging) before any sweep writes into it
    cluster_sync();

    T psi_before[NA][NB];
    const T k1 = T(0.5) * (T(1) - P.s_g);
    const T kf = T(0.5) * (T(1) - P.s_free_g);
    const T ke = T(0.25) * P.s_free_g;
    const T wG = P.wG;
    const bool interior = y0 >= 0 && y0 + RH <= ny;
    int li[NA][NB];
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b) li[a][b] = (ty + BY * a + 1) * PW + tx + 32 * b + 1;
    // pad cells that hold populations leaving this CTA's part, and where they
    // land in the neighbour: column RW of g1 -> column 0 of the right one,
    // column -1 of g3 -> column RW - 1 of the left one, row RH of g2 -> row 0
    // of the upper one, row -1 of g4 -> row RH - 1 of the lower one
    const int tid = tx + 32 * ty;
#pragma unroll 1
    for (int s = 0; s < NSW; ++s) {
        const T *gc = sg + (s & 1) * 4 * PL;
        T *gn = sg + ((s + 1) & 1) * 4 * PL;
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            const int gy = y0 + ty + BY * a;
            if (!interior && (gy < 0 || gy >= ny)) continue;
            const bool top = !interior && gy + 1 >= ny, bot = !interior && gy == 0;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int l = li[a][b];
                const T g1 = gc[l], g2 = gc[PL + l], g3 = gc[2 * PL + l], g4 = gc[3 * PL + l];
                const T m1 = g1 - g3, m2 = g2 - g4, m3 = g1 + g3, m4 = g2 + g4;
                if (RESID) psi_before[a][b] = T(1.5) * (m3 + m4);
                const T X6 = T(0.5) * (cA[a][b] - cBx[a][b] * m1 - cBy[a][b] * m2);
                const T e = ke * (m3 + m4) + X6;
                const T h3 = kf * m3 + e, h4 = kf * m4 + e;
                const T h1 = k1 * m1, h2 = k1 * m2;
                const T p2 = h4 + h2, p4 = h4 - h2;
                gn[l + 1] = h3 + h1;
                gn[2 * PL + l - 1] = h3 - h1;
                if (top) gn[3 * PL + l] = -p2 + wG;     // cathode: ABB to psi_c
                else gn[PL + l + PW] = p2 - wG;
                if (bot) gn[PL + l] = -p4 - wG;         // anode: ABB to psi_a
                else gn[3 * PL + l - PW] = p4 + wG;
            }
        }
        __syncthreads();
        // hand the pad cells to the neighbours (their copies of these cells
        // are not written by their own pushes)
        const unsigned nb_off = (unsigned)(((s + 1) & 1) * 4 * PL * (int)sizeof(T));
        if (tid < RW) {
            const int c = tid + 1;
            if (has_u) st_cluster(base_u + nb_off + (unsigned)((PL + PW + c) * (int)sizeof(T)), gn[PL + (RH + 1) * PW + c]);
            if (has_d) st_cluster(base_d + nb_off + (unsigned)((3 * PL + RH * PW + c) * (int)sizeof(T)), gn[3 * PL + c]);
        } else if (tid < RW + RH) {
            const int r = tid - RW + 1;
            if (has_r) st_cluster(base_r + nb_off + (unsigned)((r * PW + 1) * (int)sizeof(T)), gn[r * PW + RW + 1]);
            if (has_l) st_cluster(base_l + nb_off + (unsigned)((2 * PL + r * PW + RW) * (int)sizeof(T)), gn[2 * PL + r * PW]);
        }
        cluster_sync();
    }

    // ---- store the output tile (and, FIRST, its coefficients) ----
    const T *gf = sg + (NSW & 1) * 4 * PL;
    T red[2] = {T(0), T(0)};
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const int ly = ty + BY * a, gy = y0 + ly, Y = cy * RH + ly;
        if (Y < H || Y >= CH - H || gy >= ny) continue;
        const long long row = (long long)gy * nx;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int lx = tx + 32 * b, gx = x0 + lx, X = cx * RW + lx;
            if (X < H || X >= CW - H || gx >= nx) continue;
            const int l = (ly + 1) * PW + lx + 1;
            const long long k = row + gx;
            const T g1 = gf[l], g2 = gf[PL + l], g3 = gf[2 * PL + l], g4 = gf[3 * PL + l];
            dst[k] = g1;
            dst[nn + k] = g2;
            dst[2 * nn + k] = g3;
            dst[3 * nn + k] = g4;
            if (FIRST) {
                coef[k] = cA[a][b];
                coef[nn + k] = cBx[a][b];
                coef[2 * nn + k] = cBy[a][b];
            }
            if (RESID) {
                const T psit = T(1.5) * ((g1 + g3) + (g2 + g4));
                const T d = psit - psi_before[a][b];
                const T ps = psit + psi_lin(P, gy);
                red[0] += d * d;
                red[1] += ps * ps;
            }
        }
    }
    if (RESID) block_sum_store<T, 2>(red, part);
}

// Converge mode, after sweep j (one block of 256): r_{j-1} from the partials
// of sweep j, then the stop rule k >= kmin and (r_k < tol or k = kmax).
static __global__ void __launch_bounds__(256) k_sweep_decide(const double *__restrict__ part, long long nb,
                                                      Control *ctl, int j)
{
    if (ctl->done) return;
    double tot[2] = {0.0, 0.0};
    if (j >= 2) sum_partials<2>(part, nb, tot);
    if (threadIdx.x != 0) return;
    if (j >= 2) {
        const double r = tot[1] > 0.0 ? sqrt(tot[0] / tot[1]) : sqrt(tot[0]);
        if (j - 1 >= ctl->kmin && r < ctl->tol) {
            ctl->K = j - 1; ctl->flips = j - 1; ctl->done = 1; ctl->early = 1; ctl->r_last = r;
            return;
        }
    }
    ctl->K = j;
    ctl->flips = j;
    if (j >= ctl->kmax) ctl->done = 1;
}

// Planes k_main stages per node: f1..f8, h0..h8, the QI planes of p and of
// n (one allocation of 17 + 2 QI planes) and (phi u)(t-1) x, y of type S,
// then g1..g4 of type T.  With FP16 storage it also stages the chemical
// potential of phi_ref (a fifth plane of type T) and phi_ref on the block's
// 64 x 4 nodes with a one-node ring (6 x 66), which the h push reads; with
// S = T those two come from global memory after the staging (measured at
// 2048^2: staging them costs FP32 0.031 ms per step and saves FP16
// storage 0.008 ms).
template <int QI> __host__ __device__ constexpr int main_splanes() { return 17 + 2 * QI + 2; }

// ---- the step kernel's inputs staged by the tensor memory accelerator -----
// One stage holds a 64 x 4 tile's inputs, each part at a 128-byte boundary:
// the 27 population planes (f, h, p, n) and the 2 planes of (phi u)(t-1) as
// S (one run, as the cp.async staging lays them out), then as T the 4 g
// planes, mu_ref, grad phi_ref (x, y) and psi_prev, then dphi and phi_ref over
// the tile's rows -1 .. 4 and columns -4 .. 67 (a box of 72 x 6 starting at a
// 16-byte boundary; the columns outside the lattice read zero and the
// periodic neighbours of the first and last column come from global memory).
constexpr int TMA_HW = 72, TMA_HH = 6, TMA_HX = 4;
__host__ __device__ constexpr size_t tma_align(size_t b) { return (b + 127) & ~(size_t)127; }
template <typename T, typename S> struct TmaLayout {
    static constexpr size_t pops = 0;                                     // 27 + 2 planes of S
    static constexpr size_t tpl = tma_align(sizeof(S) * 29 * 256);       // g1..g4, mu_ref, gxr, gyr, psi_prev
    static constexpr size_t dphi = tma_align(tpl + sizeof(T) * 8 * 256);
    static constexpr size_t phir = tma_align(dphi + sizeof(T) * TMA_HW * TMA_HH);
    static constexpr size_t stage = tma_align(phir + sizeof(T) * TMA_HW * TMA_HH);
    // bytes the loads of one stage deliver (psi_prev only with the residual)
    __host__ __device__ static constexpr unsigned tx(bool resid)
    {
        return (unsigned)(sizeof(S) * 29 * 256 + sizeof(T) * (resid ? 8 : 7) * 256 +
                          2 * sizeof(T) * TMA_HW * TMA_HH);
    }
};
// Pointers into the stage of the tile being computed.
template <typename T, typename S> struct TmaView {
    const S *pops;    // [29][256]
    const T *tpl;     // [8][256]: g1..g4, mu_ref, gxr, gyr, psi_prev
    const T *dphi;    // [6][72]
    const T *phir;    // [6][72]
};
// Tensor maps of the step kernel's inputs (cuTensorMapEncodeTiled on the host).
struct MainMaps {
    CUtensorMap pops;     // 3D (nx, ny, 27), box (64, 4, 27): the source time level
    CUtensorMap phiu;     // 3D (nx, ny, 2), box (64, 4, 2)
    CUtensorMap g[2];     // 3D (nx, ny, 4), box (64, 4, 4): the two g buffers
    CUtensorMap mur, gxr, gyr, psi;   // 2D (nx, ny), box (64, 4)
    CUtensorMap dphi, phir;           // 2D (nx, ny + 2) with ghost rows, box (72, 6)
};
// Blocks of 256 per SM the step kernel's registers are sized for: 4 in float
// (64 registers; measured 9 % faster at 2048^2 than 3 blocks at 80 registers,
// though a few bytes spill), 3 in double.
template <typename T> constexpr int MAIN_MINB = sizeof(T) == 4 ? 4 : 3;
template <typename T, typename S> constexpr bool MAIN_STAGE_REF = !std::is_same<S, T>::value;
template <typename T, typename S> constexpr int MAIN_TPLANES = MAIN_STAGE_REF<T, S> ? 5 : 4;
constexpr int MAIN_RING_W = 66, MAIN_RING = 6 * MAIN_RING_W;
template <typename T, typename S, int QI = 5> __host__ __device__ constexpr size_t main_smem_bytes()
{
    return (sizeof(S) * main_splanes<QI>() + sizeof(T) * MAIN_TPLANES<T, S>) * 256 +
           (MAIN_STAGE_REF<T, S> ? sizeof(T) * MAIN_RING : 0);
}

// Copy NPL planes of the block's 64 x 4 nodes (x0, y0) to st[plane][256]
// asynchronously; plane(i) gives the base of plane i.  VEC: 16-byte copies
// of row segments shared by all threads (needs nx * sizeof(E) to be a
// multiple of 16); else one copy per node.
template <typename E, int NPL, bool VEC, typename PlaneF>
__device__ __forceinline__ void stage_planes(E *st, PlaneF plane, int nx, int ny, int x0, int y0, int tid,
                                             bool inside, long long k)
{
    if constexpr (VEC) {
        // a plane's 4 rows of 64 take PER 16-byte chunks; 256 / PER planes per
        // pass of the block, so each thread keeps its row and chunk and steps
        // through the planes
        constexpr int NE = 16 / (int)sizeof(E), CH = 64 / NE, PER = 4 * CH, STEP = 256 / PER;
        static_assert(256 % PER == 0, "staging pass");
        const int r = tid % PER, row = r / CH, ch = r - row * CH;
        const int y = y0 + row, x = x0 + ch * NE;
        if (y < ny && x < nx) {
            const long long off = (long long)y * nx + x;
            E *d = st + row * 64 + ch * NE;
#pragma unroll
            for (int j = 0; j < (NPL + STEP - 1) / STEP; ++j) {
                const int pl = tid / PER + j * STEP;
                if (pl < NPL) cp_async16(d + pl * 256, plane(pl) + off);
            }
        }
    } else {
        if (!inside) return;
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            if constexpr (sizeof(E) >= 4) cp_async(st + i * 256 + tid, plane(i) + k);
            else st[i * 256 + tid] = plane(i)[k];
        }
    }
}

// The rest of the step at every node (O5-O11): reaction (Eq. 42-43), forces
// (Eq. 12-14), u and p (Eq. 56-57), MRT collisions of f (Eq. 51), h (Eq. 27),
// p and n (Eq. 34-35), push with the wall rules (Eq. 64).  The block's
// populations are copied to shared memory asynchronously first, so that all
// of them are in flight at once.  The equilibria and sources of f and h
// enter directly as their moments in the basis of Eq. 28:
//   M f_eq = (0, rho u, p + rho ux^2, p + rho uy^2, rho ux uy, rho ux/3,
//             rho uy/3, p/3 + rho u^2/3)          (rows 1..8, Eq. 52-53)
//   M F    = (F, ux gx + uy gy/3, uy gy + ux gx/3, (ux gy + uy gx)/3, Fx/3,
//             Fy/3, u.g/3),  g = grad rho           (Eq. 54)
//   M h_eq = (phi, phi u, phi/3, phi/3, 0, phi ux/3, phi uy/3, phi/9) (Eq. 31)
//   M H    = (0, V, 0, 0, 0, Vx/3, Vy/3, 0), V = d(phi u)/dt + cs^2 lambda n (Eq. 32)
//   SNAP  : write the macroscopic snapshot and its sums of phi and q.
//   FROZEN: E from DevP.
//   RESID : residual of the last sweep against psi_prev.
//   VEC   : 16-byte staging (stage_planes).
// NaN or Inf in the macroscopic fields raises *unstable.
// Launch: blockDim (64, 4), dynamic shared memory main_smem_bytes<T, S>().
// Body of k_main for the block at (bx, by) of the lattice's grid; slot: its
// partials.
//   TMA   : the inputs were staged by the caller (k_main_tma) into tv.
template <typename T, typename S, bool SNAP, bool FROZEN, bool RESID, bool VEC, int QI = 5, bool TMA = false>
__device__ __forceinline__ void main_body(const DevP<T> &P, const Pops<S> &src, const Pops<S> &dst,
                                          const T *__restrict__ gA, const T *__restrict__ gB,
                                          const Control *__restrict__ ctl, const PhiRef<T> &Rf,
                                          S *__restrict__ phiu, const T *__restrict__ psi_prev, T *__restrict__ snap,
                                          double *__restrict__ part, int *__restrict__ unstable, int bx, int by,
                                          long long slot, const TmaView<T, S> *tv = nullptr)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int NSP = main_splanes<QI>(), NPOP = 17 + 2 * QI;
    static_assert(!TMA || QI == 5, "the staged step kernel takes ions on D2Q5");
    const S *st;
    const T *stg;
    if constexpr (TMA) {
        st = tv->pops;
        stg = tv->tpl;
    } else {
        st = reinterpret_cast<S *>(smem_raw);
        stg = reinterpret_cast<T *>(smem_raw + sizeof(S) * NSP * 256);
    }
    // the legacy staging writes these buffers
    S *st_w = reinterpret_cast<S *>(smem_raw);
    T *stg_w = reinterpret_cast<T *>(smem_raw + sizeof(S) * NSP * 256);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int x = bx * blockDim.x + threadIdx.x;
    const int y = by * blockDim.y + threadIdx.y;
    const bool inside = x < P.nx && y < P.ny;
    const long long nn = P.nn, k = (long long)y * P.nx + x;
    T red[4] = {T(0), T(0), T(0), T(0)};
    if constexpr (!TMA) {
        const T *__restrict__ g = ((ctl->cur0 + ctl->flips) & 1) ? gB : gA;
        const S *pops = src.f, *pu = phiu;
        const int x0 = bx * blockDim.x, y0 = by * blockDim.y;
        stage_planes<S, NSP, VEC>(
            st_w, [=](int i) { return i < NPOP ? pops + i * nn : pu + (i - NPOP) * nn; }, P.nx, P.ny, x0, y0, tid,
            inside, k);
        const T *mur = Rf.mur;
        stage_planes<T, MAIN_TPLANES<T, S>, VEC>(stg_w, [=](int i) { return i < 4 ? g + i * nn : mur; }, P.nx,
                                                 P.ny, x0, y0, tid, inside, k);
        // phi_ref of rows y0 - 1 .. y0 + 4 (phir holds the rows -1 .. ny),
        // columns x0 - 1 .. x0 + 64 (periodic); rows above ny are never read
        T *ring = stg_w + MAIN_TPLANES<T, S> * 256;
        for (int e = tid; MAIN_STAGE_REF<T, S> && e < MAIN_RING; e += 256) {
            const int ry = e / MAIN_RING_W, rx = e - ry * MAIN_RING_W;
            const int gy = y0 - 1 + ry;
            int gx = x0 - 1 + rx;
            gx = gx < 0 ? gx + P.nx : (gx >= P.nx ? gx % P.nx : gx);
            if (gy <= P.ny) cp_async(ring + e, Rf.phir + (long long)(gy + 1) * P.nx + gx);
        }
    }
    const T pprev = (RESID && inside) ? (TMA ? stg[7 * 256 + tid] : psi_prev[k]) : T(0);
    const int nx = P.nx, ny = P.ny;
    const T third = T(1.0 / 3.0);
    // ---- O1-O2: phi, properties (Eq. 61), stencils (Eq. 59) ----
    // phi = phi_ref + dphi; the stencils act on dphi and add the
    // reference's gradient; differences first (exact for neighbours)
    int xm = 0, xp = 0;
    T dphi = T(0), phir = T(0), phi = T(0), gx = T(0), gy = T(0), lapd = T(0);
    if (inside) {
        xm = nbx(x, -1, nx, P.side_walls);
        xp = nbx(x, 1, nx, P.side_walls);
        const int ki = y * nx + x;   // in-plane index (nx ny < 2^31)
        const T *r1 = Rf.dphig + nx + ki, *r0 = r1 - nx, *r2 = r1 + nx;
        xm -= x;   // column offsets from here on
        xp -= x;
        T vc, vE, vW, vN, vS, vNE, vNW, vSW, vSE, gxr, gyr;
        if constexpr (TMA) {
            // the staged box; the periodic neighbours of the first and last
            // column from global memory
            const T *h1 = tv->dphi + (threadIdx.y + 1) * TMA_HW + threadIdx.x + TMA_HX;
            vc = h1[0]; vN = h1[TMA_HW]; vS = h1[-TMA_HW];
            if (x == 0 || x == nx - 1) {
                vE = r1[xp]; vW = r1[xm]; vNE = r2[xp]; vNW = r2[xm]; vSW = r0[xm]; vSE = r0[xp];
            } else {
                vE = h1[1]; vW = h1[-1]; vNE = h1[TMA_HW + 1]; vNW = h1[TMA_HW - 1];
                vSW = h1[-TMA_HW - 1]; vSE = h1[-TMA_HW + 1];
            }
            phir = tv->phir[(threadIdx.y + 1) * TMA_HW + threadIdx.x + TMA_HX];
            gxr = stg[5 * 256 + tid];
            gyr = stg[6 * 256 + tid];
        } else {
            vc = r1[0]; vE = r1[xp]; vW = r1[xm]; vN = r2[0]; vS = r0[0];
            vNE = r2[xp]; vNW = r2[xm]; vSW = r0[xm]; vSE = r0[xp];
            phir = Rf.phir[nx + ki];
            gxr = Rf.gxr[ki];
            gyr = Rf.gyr[ki];
        }
        dphi = vc;
        const T dE = vE - dphi, dW = vW - dphi, dN = vN - dphi, dS = vS - dphi;
        const T dNE = vNE - dphi, dNW = vNW - dphi, dSW = vSW - dphi, dSE = vSE - dphi;
        phi = phir + dphi;
        gx = gxr + ((dE - dW) * third + ((dNE - dNW) + (dSE - dSW)) * T(1.0 / 12.0));
        gy = gyr + ((dN - dS) * third + ((dNE + dNW) - (dSE + dSW)) * T(1.0 / 12.0));
        lapd = T(2.0 / 3.0) * ((dE + dW) + (dN + dS)) + T(1.0 / 6.0) * ((dNE + dSW) + (dNW + dSE));
    }
    if constexpr (!TMA) {
        cp_async_wait_all();
        if constexpr (VEC || MAIN_STAGE_REF<T, S>) __syncthreads();   // copies of all threads
    }
    if (inside) {
        SRng rng(k, kSame<S, T> ? 0 : ctl->t, 0x1b873593u);
        // in-plane offsets of the push targets: rows below / at / above, the
        // columns left / at / right; a link through a wall bounces back to
        // the node itself
        const bool top = y + 1 >= ny, bot = y == 0;
        const bool lwall = P.side_walls && x == 0, rwall = P.side_walls && x == nx - 1;
        const int rowC = y * nx + x, rowN = top ? rowC : rowC + nx, rowS = bot ? rowC : rowC - nx;
        auto dest = [&](int cx, int cy) -> int {
            const int col = cx < 0 ? xm : (cx > 0 ? xp : 0);
            return cy > 0 ? rowN + col : (cy < 0 ? rowS + col : rowC + col);
        };
        auto bounced = [&](int cx, int cy) -> bool {
            return (cy > 0 && top) || (cy < 0 && bot) || (cx > 0 && rwall) || (cx < 0 && lwall);
        };
        const T rho = T(1) + P.rho1 * phi;
        const T inv_rho = T(1) / rho;
        const T mup = P.mu_v * (T(1) + P.mu1 * phi);
        const T mum = P.m * mup;
        const T grx = P.rho1 * gx, gry = P.rho1 * gy;
        const T dex = P.er1 * gx, dey = P.er1 * gy;

        // ---- O4 result: psi, E from the last sweep (Eq. 49-50) ----
        const T g1 = stg[tid], g2 = stg[256 + tid], g3 = stg[2 * 256 + tid], g4 = stg[3 * 256 + tid];
        const T psit = T(1.5) * ((g1 + g3) + (g2 + g4));
        const T psi = psit + psi_lin(P, y);
        T Ex, Ey;
        if (FROZEN) { Ex = P.Ex_frozen; Ey = P.Ey_frozen; }
        else { Ex = P.three_over_tau_g * (g1 - g3); Ey = P.three_over_tau_g * (g2 - g4); }
        if (RESID) {
            const T d = psit - pprev;
            red[2] = d * d;
            red[3] = psi * psi;
        }

        // ---- O5: Onsager dissociation and the implicit reaction (Eq. 5, 42-43) ----
        T pv[QI], nv[QI];
#pragma unroll
        for (int i = 0; i < QI; ++i) {
            pv[i] = lds(st + (17 + i) * 256 + tid, P.isc_c);
            nv[i] = lds(st + (17 + QI + i) * 256 + tid, P.isc_c);
            if constexpr (!kSame<S, T>) {
                const T wc = (QI == 9 ? w9<T>(i) : (i == 0 ? T(1.0 / 3.0) : T(1.0 / 6.0))) * P.cref;
                pv[i] += wc;
                nv[i] += wc;
            }
        }
        T sp, sn;
        if constexpr (QI == 5) {
            sp = (((pv[0] + pv[1]) + pv[2]) + pv[3]) + pv[4];
            sn = (((nv[0] + nv[1]) + nv[2]) + nv[3]) + nv[4];
        } else {
            sp = T(0);
            sn = T(0);
#pragma unroll
            for (int i = 0; i < QI; ++i) { sp += pv[i]; sn += nv[i]; }
        }
        const T q = sp - sn;
        T cp, cm, R;
        if (P.onsager_form == 2) {
            cp = sp; cm = sn; R = T(0);
        } else {
            const T b = P.cb * dsqrt<T>(dsqrt<T>(Ex * Ex + Ey * Ey));
            const T F = onsager<T>(b, P.onsager_form);
            const T cbp = sp + T(0.5) * P.k_d * F, cbm = sn + T(0.5) * P.k_d * F;
            const T lam0 = T(0.5) * P.k_r;
            const T B = T(1) - lam0 * cbp + lam0 * cbm;
            const T disc = dsqrt<T>(B * B + T(4) * lam0 * cbp);
            if (B >= T(0)) cp = (B + disc > T(0)) ? T(2) * cbp / (B + disc) : T(0);
            else cp = (-B + disc) / (T(2) * lam0);
            cm = cp - cbp + cbm;
            R = P.k_d * F - P.k_r * cp * cm;
        }

        // ---- O6: forces (Eq. 12-14) ----
        // mu_phi - mu_ref: the cubic of Eq. 13 as (phi - phi_ref) times
        // (phi^2 + phi phi_ref + phi_ref^2 - 1.5 (phi + phi_ref) + 0.5)
        const T mu_phi = ((MAIN_STAGE_REF<T, S> || TMA) ? stg[4 * 256 + tid] : Rf.mur[rowC]) +
                         T(4) * P.beta * dphi * ((phi * phi + phi * phir + phir * phir) - T(1.5) * (phi + phir) + T(0.5)) -
                         P.kappa * lapd;
        const T E2 = Ex * Ex + Ey * Ey;
        const T Fx = mu_phi * gx + P.Kq * q * Ex - T(0.5) * E2 * dex;
        const T Fy = mu_phi * gy + P.Kq * q * Ey - T(0.5) * E2 * dey;

        // ---- O7: u and p (Eq. 56-57), moments of f ----
        T fv[9];
        fv[0] = T(0);
#pragma unroll
        for (int i = 1; i < 9; ++i) fv[i] = lds(st + (i - 1) * 256 + tid, P.isc_f);
        T mf[9];
        moments9<T>(fv, mf);     // mf[0] is not used (f0 is not stored)
        const T ux = (mf[1] + T(0.5) * Fx) * inv_rho;
        const T uy = (mf[2] + T(0.5) * Fy) * inv_rho;
        const T uu = ux * ux + uy * uy;
        const T sne0 = mf[3] + mf[4] - mf[8];           // sum of f1..f8
        const T ugr = ux * grx + uy * gry;
        const T pr = T(0.6) * (sne0 + T(0.5) * ugr - rho * T(2.0 / 3.0) * uu);

        // ---- O8: f collision (Eq. 51-55) in moment space ----
        {
            const T sv = P.s_f0 > T(0) ? P.s_f0 : T(1) / (T(0.5) + T(3) * P.eta_v * (T(1) + P.eta1 * phi) * inv_rho);
            const T sfree = P.bgk ? sv : P.s_free;
            const T ru = rho * ux, rv = rho * uy;
            T d[9], mF[9];
            d[0] = T(0);
            d[1] = mf[1] - ru;
            d[2] = mf[2] - rv;
            d[3] = mf[3] - (pr + ru * ux);
            d[4] = mf[4] - (pr + rv * uy);
            d[5] = mf[5] - ru * uy;
            d[6] = mf[6] - ru * third;
            d[7] = mf[7] - rv * third;
            d[8] = mf[8] - (pr + rho * uu) * third;
            mF[0] = T(0);
            mF[1] = Fx;
            mF[2] = Fy;
            mF[3] = ux * grx + uy * gry * third;
            mF[4] = uy * gry + ux * grx * third;
            mF[5] = (ux * gry + uy * grx) * third;
            mF[6] = Fx * third;
            mF[7] = Fy * third;
            mF[8] = ugr * third;
            T mc[9], dl[9];
#pragma unroll
            for (int kk = 0; kk < 9; ++kk) {
                const T s = (kk >= 1 && kk <= 5) ? sv : sfree;
                mc[kk] = s * d[kk] - (T(1) - T(0.5) * s) * mF[kk];
            }
            inverse9<T>(mc, dl);
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const T v = fv[i] - dl[i];
                if (bounced(cx9(i), cy9(i))) sts_sr(dst.f + (opp9(i) - 1) * nn + rowC, v, P.sc_f, rng);
                else sts_sr(dst.f + (i - 1) * nn + dest(cx9(i), cy9(i)), v, P.sc_f, rng);
            }
        }

        // ---- O9: h collision (Eq. 27-33, Eq. 58) in moment space ----
        {
            T hv[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) hv[i] = lds(st + (8 + i) * 256 + tid, P.isc_h);
            const T pux = phi * ux, puy = phi * uy;
            const T dpx = pux - lds(st + NPOP * 256 + tid, P.isc_u), dpy = puy - lds(st + (NPOP + 1) * 256 + tid, P.isc_u);
            sts(phiu + k, pux, P.sc_u);
            sts(phiu + nn + k, puy, P.sc_u);
            // normal of Eq. 32, regularised: grad phi / sqrt(|grad phi|^2 + eps^2)
            const T g2s = gx * gx + gy * gy;
            T nhx = T(0), nhy = T(0);
            if (P.nhat_eps2 > T(0)) {
                const T inv = T(1) / dsqrt<T>(g2s + P.nhat_eps2);
                nhx = gx * inv; nhy = gy * inv;
            } else {
                const T mag = dsqrt<T>(g2s);
                if (mag >= T(1e-12)) { nhx = gx / mag; nhy = gy / mag; }
            }
            const T lam = T(4) * phi * (T(1) - phi) * P.inv_W;
            const T Vx = dpx + third * lam * nhx, Vy = dpy + third * lam * nhy;
            // moments of the stored deviations; the reference part cancels
            // against phi M w of the equilibrium, leaving dphi M w
            T mh[9];
            moments9<T>(hv, mh);
            T d[9];
            d[0] = mh[0] - dphi;
            d[1] = mh[1] - pux;
            d[2] = mh[2] - puy;
            d[3] = mh[3] - dphi * third;
            d[4] = mh[4] - dphi * third;
            d[5] = mh[5];
            d[6] = mh[6] - pux * third;
            d[7] = mh[7] - puy * third;
            d[8] = mh[8] - dphi * T(1.0 / 9.0);
            const T sv = P.s_h, sfree = P.sfree_h;
            const T hv_ = T(1) - T(0.5) * sv;
            T mc[9], dl[9];
            mc[0] = sfree * d[0];
            mc[1] = sv * d[1] - hv_ * Vx;
            mc[2] = sv * d[2] - hv_ * Vy;
            mc[3] = sfree * d[3];
            mc[4] = sfree * d[4];
            mc[5] = sfree * d[5];
            mc[6] = sfree * d[6] - (T(1) - T(0.5) * sfree) * Vx * third;
            mc[7] = sfree * d[7] - (T(1) - T(0.5) * sfree) * Vy * third;
            mc[8] = sfree * d[8];
            inverse9<T>(mc, dl);
            // push, re-based on the destination's reference:
            // + w_i (phi_ref(x) - phi_ref(x + c_i)); a bounced population stays
            const T *qr = MAIN_STAGE_REF<T, S>
                              ? stg + MAIN_TPLANES<T, S> * 256 + (threadIdx.y + 1) * MAIN_RING_W + threadIdx.x + 1
                              : Rf.phir + nx;   // phi_ref without its ghost row
            // phi_ref of the push target in direction i (in-plane offset o)
            auto qphi = [&](int i, int o) -> T {
                if constexpr (TMA) {
                    if ((x == 0 && cx9(i) < 0) || (x == nx - 1 && cx9(i) > 0)) return Rf.phir[nx + o];
                    return tv->phir[(threadIdx.y + 1 + cy9(i)) * TMA_HW + threadIdx.x + TMA_HX + cx9(i)];
                } else {
                    return qr[MAIN_STAGE_REF<T, S> ? cy9(i) * MAIN_RING_W + cx9(i) : o];
                }
            };
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const T v = hv[i] - dl[i];
                if (bounced(cx9(i), cy9(i))) {
                    sts_sr(dst.h + opp9(i) * nn + rowC, v, P.sc_h, rng);
                } else {
                    const int o = dest(cx9(i), cy9(i));
                    const T shift = i == 0 ? T(0) : w9<T>(i) * (phir - qphi(i, o));
                    sts_sr(dst.h + i * nn + o, v + shift, P.sc_h, rng);
                }
            }
        }

        // ---- O10-O11: ions (Eq. 34-40) on D2Q5, push with Eq. 64 ----
        if constexpr (QI == 5) {
            T sv_p = P.s_p0, sv_n = P.s_n0;
            if (!(sv_p > T(0))) {
                const T Dp = P.einstein_D ? P.D * mup * P.inv_mu_v : P.D;
                const T Dm = P.einstein_D ? P.D * mum * P.inv_mu_v : P.D;
                sv_p = T(1) / (T(0.5) + T(3) * Dp);
                sv_n = T(1) / (T(0.5) + T(3) * Dm);
            }
            const T fp = P.bgk ? sv_p : P.s_free, fn = P.bgk ? sv_n : P.s_free;
            const T Lx = P.ion_L_term ? Fx : T(0), Ly = P.ion_L_term ? Fy : T(0);
            // cations: moments of (p - p_eq) + G and of R_i + L_i
            T mc0 = fp * (sp - cp) - (T(1) - T(0.5) * fp) * R;
            T mc1 = sv_p * ((pv[1] - pv[3]) - cp * ux - mup * cp * Ex) - (T(1) - T(0.5) * sv_p) * cp * Lx;
            T mc2 = sv_p * ((pv[2] - pv[4]) - cp * uy - mup * cp * Ey) - (T(1) - T(0.5) * sv_p) * cp * Ly;
            T mc3 = fp * ((pv[1] + pv[3]) - cp * third) - (T(1) - T(0.5) * fp) * R * third;
            T mc4 = fp * ((pv[2] + pv[4]) - cp * third) - (T(1) - T(0.5) * fp) * R * third;
            T po[5];
            po[0] = pv[0] - (mc0 - mc3 - mc4);
            po[1] = pv[1] - T(0.5) * (mc3 + mc1);
            po[3] = pv[3] - T(0.5) * (mc3 - mc1);
            po[2] = pv[2] - T(0.5) * (mc4 + mc2);
            po[4] = pv[4] - T(0.5) * (mc4 - mc2);
            // anions: (n - n_eq) - G_bar
            mc0 = fn * (sn - cm) - (T(1) - T(0.5) * fn) * R;
            mc1 = sv_n * ((nv[1] - nv[3]) - cm * ux + mum * cm * Ex) - (T(1) - T(0.5) * sv_n) * cm * Lx;
            mc2 = sv_n * ((nv[2] - nv[4]) - cm * uy + mum * cm * Ey) - (T(1) - T(0.5) * sv_n) * cm * Ly;
            mc3 = fn * ((nv[1] + nv[3]) - cm * third) - (T(1) - T(0.5) * fn) * R * third;
            mc4 = fn * ((nv[2] + nv[4]) - cm * third) - (T(1) - T(0.5) * fn) * R * third;
            T no[5];
            no[0] = nv[0] - (mc0 - mc3 - mc4);
            no[1] = nv[1] - T(0.5) * (mc3 + mc1);
            no[3] = nv[3] - T(0.5) * (mc3 - mc1);
            no[2] = nv[2] - T(0.5) * (mc4 + mc2);
            no[4] = nv[4] - T(0.5) * (mc4 - mc2);

            const T w = T(1) / T(6);
            T bp2, bn2, bp4, bn4;     // pushed or bounced values of directions 2 and 4
            if (y + 1 < ny) {
                bp2 = po[2];
                bn2 = no[2];
            } else {  // cathode: attracts cations (zero gradient), repels anions
                const T cwp = P.ion_bc == 0 ? cp : T(0);
                bp2 = P.ion_bc == 2 ? po[2] : -po[2] + T(2) * w * cwp;
                bn2 = P.ion_bc == 2 ? no[2] : -no[2];
            }
            if (y > 0) {
                bp4 = po[4];
                bn4 = no[4];
            } else {  // anode: repels cations, attracts anions
                const T cwm = P.ion_bc == 0 ? cm : T(0);
                bp4 = P.ion_bc == 2 ? po[4] : -po[4];
                bn4 = P.ion_bc == 2 ? no[4] : -no[4] + T(2) * w * cwm;
            }
            if constexpr (!kSame<S, T>) {   // stored relative to w_i c_ref
                const T c0 = P.cref * T(1.0 / 3.0), c1 = P.cref * w;
                po[0] -= c0; no[0] -= c0;
                po[1] -= c1; no[1] -= c1;
                po[3] -= c1; no[3] -= c1;
                bp2 -= c1; bn2 -= c1;
                bp4 -= c1; bn4 -= c1;
            }
            sts_sr(dst.p + rowC, po[0], P.sc_c, rng);
            sts_sr(dst.n + rowC, no[0], P.sc_c, rng);
            // directions 1 and 3 bounce back at the side walls (zero gradient)
            const long long o1 = rwall ? 3 * nn + rowC : nn + rowC + xp;
            const long long o3 = lwall ? nn + rowC : 3 * nn + rowC + xm;
            sts_sr(dst.p + o1, po[1], P.sc_c, rng);
            sts_sr(dst.n + o1, no[1], P.sc_c, rng);
            sts_sr(dst.p + o3, po[3], P.sc_c, rng);
            sts_sr(dst.n + o3, no[3], P.sc_c, rng);
            // direction 2 lands in plane 2 of the row above or, bounced, in plane 4 here
            const long long o2 = top ? 4 * nn + rowC : 2 * nn + rowN;
            const long long o4 = bot ? 2 * nn + rowC : 4 * nn + rowS;
            sts_sr(dst.p + o2, bp2, P.sc_c, rng);
            sts_sr(dst.n + o2, bn2, P.sc_c, rng);
            sts_sr(dst.p + o4, bp4, P.sc_c, rng);
            sts_sr(dst.n + o4, bn4, P.sc_c, rng);
        } else {
            // ---- ions on D2Q9 as Eq. 34-38 print them: M of Eq. 28, the
            // weights of Eq. 25, s1 = s2 = 1/tau (Eq. 37), the other rates free.
            // In the basis of Eq. 28 the moments of p_eq, of the drift G and of
            // R_i + L_i are (with a = mu c grad psi, the drift of Eq. 40):
            //   M p_eq  = c (1, ux, uy, 1/3, 1/3, 0, ux/3, uy/3, 1/9)
            //   M G     = (0, ax, ay, 0, 0, 0, ax/3, ay/3, 0)
            //   M (R+L) = (R, c Lx, c Ly, R/3, R/3, 0, c Lx/3, c Ly/3, R/9)
            T sv_p = P.s_p0, sv_n = P.s_n0;
            if (!(sv_p > T(0))) {
                const T Dp = P.einstein_D ? P.D * mup * P.inv_mu_v : P.D;
                const T Dm = P.einstein_D ? P.D * mum * P.inv_mu_v : P.D;
                sv_p = T(1) / (T(0.5) + T(3) * Dp);
                sv_n = T(1) / (T(0.5) + T(3) * Dm);
            }
            const T Lx = P.ion_L_term ? Fx : T(0), Ly = P.ion_L_term ? Fy : T(0);
            const T ninth = T(1.0 / 9.0);
            // post-collision populations; the drift enters as m - m_eq + a with
            // a = -mu+ c+ E for cations (Eq. 34) and a = +mu- c- E for anions
            // (Eq. 35, the sign of its G term)
            auto collide = [&](const T (&v)[9], T c, T ax, T ay, T sv, T (&o)[9]) {
                const T fr = P.bgk ? sv : P.s_free;
                const T hf = T(1) - T(0.5) * fr, hv = T(1) - T(0.5) * sv;
                T m[9], dm[9], dl[9];
                moments9<T>(v, m);
                const T cLx = c * Lx, cLy = c * Ly;
                dm[0] = fr * (m[0] - c) - hf * R;
                dm[1] = sv * ((m[1] - c * ux) + ax) - hv * cLx;
                dm[2] = sv * ((m[2] - c * uy) + ay) - hv * cLy;
                dm[3] = fr * (m[3] - c * third) - hf * R * third;
                dm[4] = fr * (m[4] - c * third) - hf * R * third;
                dm[5] = fr * m[5];
                dm[6] = fr * ((m[6] - c * ux * third) + ax * third) - hf * cLx * third;
                dm[7] = fr * ((m[7] - c * uy * third) + ay * third) - hf * cLy * third;
                dm[8] = fr * (m[8] - c * ninth) - hf * R * ninth;
                inverse9<T>(dm, dl);
#pragma unroll
                for (int i = 0; i < 9; ++i) o[i] = v[i] - dl[i];
            };
            T po[9], no[9];
            collide(pv, cp, -mup * cp * Ex, -mup * cp * Ey, sv_p, po);
            collide(nv, cm, mum * cm * Ex, mum * cm * Ey, sv_n, no);
            // push; an electrode link (which also decides a corner link) takes
            // anti-bounce-back to the wall value (the attracted species keeps
            // the node's concentration, the repelled one 0; ion_bc 1: 0 for
            // both, 2: bounce-back), a side-wall link bounces back
            auto push = [&](S *base, T (&o)[9], bool cation) {
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const int cx = cx9(i), cy = cy9(i);
                    T v = o[i];
                    long long off;
                    if ((cy > 0 && top) || (cy < 0 && bot)) {
                        const bool attracted = cation ? (cy > 0) : (cy < 0);
                        const T cw = (P.ion_bc == 0 && attracted) ? (cation ? cp : cm) : T(0);
                        if (P.ion_bc != 2) v = -v + T(2) * w9<T>(i) * cw;
                        off = opp9(i) * nn + rowC;
                    } else if ((cx > 0 && rwall) || (cx < 0 && lwall)) {
                        off = opp9(i) * nn + rowC;
                    } else {
                        off = i * nn + dest(cx, cy);
                    }
                    if constexpr (!kSame<S, T>) v -= w9<T>(i) * P.cref;   // stored relative to w_i c_ref
                    sts_sr(base + off, v, P.sc_c, rng);
                }
            };
            push(dst.p, po, true);
            push(dst.n, no, false);
        }

        if (SNAP) {
            const unsigned sm = P.snap_mask;   // block-uniform
            if (sm & 1u) snap[k] = phi;
            if (sm & 2u) snap[nn + k] = ux;
            if (sm & 4u) snap[2 * nn + k] = uy;
            if (sm & 8u) snap[3 * nn + k] = pr;
            if (sm & 16u) snap[4 * nn + k] = psi;
            if (sm & 32u) snap[5 * nn + k] = Ex;
            if (sm & 64u) snap[6 * nn + k] = Ey;
            if (sm & 128u) snap[7 * nn + k] = cp;
            if (sm & 256u) snap[8 * nn + k] = cm;
            if (sm & 512u) snap[9 * nn + k] = q;
            red[0] = phi;
            red[1] = q;
        }
        const T chk = ux + uy + pr + psi + cp + cm;
        if (!isfinite(chk)) *unstable = 1;
    }
    if (SNAP || RESID) block_sum_store_at<T, 4>(red, part, slot);
}

template <typename T, typename S, bool SNAP, bool FROZEN, bool RESID, bool VEC, int QI = 5>
__global__ void __launch_bounds__(256, MAIN_MINB<T>) k_main(const DevP<T> P, const Pops<S> src, const Pops<S> dst,
                                                 const T *__restrict__ gA, const T *__restrict__ gB,
                                                 const Control *__restrict__ ctl, const PhiRef<T> Rf,
                                                 S *__restrict__ phiu, const T *__restrict__ psi_prev,
                                                 T *__restrict__ snap, double *__restrict__ part,
                                                 int *__restrict__ unstable)
{
    main_body<T, S, SNAP, FROZEN, RESID, VEC, QI>(P, src, dst, gA, gB, ctl, Rf, phiu, psi_prev, snap, part, unstable,
                                              blockIdx.x, blockIdx.y, blockIdx.x + (long long)blockIdx.y * gridDim.x);
}

// ---- tensor memory accelerator and mbarrier (inline PTX) --------------------------

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for the phase of the given parity, at most about 70 ms (2^20 tries,
// spaced by 64 ns after the first 64); false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity)
{
    for (unsigned i = 0; i < (1u << 20); ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i >= 64) __nanosleep(64);
    }
    return false;
}
// Orders this thread's earlier generic-proxy accesses of shared memory before
// its later asynchronous-proxy ones (a stage is refilled after it was read).
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];\n" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];\n" ::"r"(smem_u32(dst)),
        "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// The step kernel on inputs staged by the tensor memory accelerator:
// persistent blocks of 64 x 4 threads walk the 64 x 4 tiles of the lattice;
// thread 0 loads the next tile's inputs (MainMaps: one box of the 27
// population planes, one of (phi u)(t-1), one of the g buffer the sweeps
// left, mu_ref, grad phi_ref, psi_prev with the residual, and the 72 x 6 boxes
// of dphi and phi_ref) into the other of two stages while the block computes
// the current tile with main_body.  Needs D2Q5 ions, periodic x and rows of
// 16-byte multiples.  A stage that does not arrive within about 70 ms sets
// *fault, the block waits (bounded) for its copies and returns.
// Launch: blockDim (64, 4), grid min(tiles, resident blocks), dynamic shared
// memory 2 TmaLayout<T, S>::stage.
template <typename T, typename S, bool SNAP, bool FROZEN, bool RESID>
__global__ void __launch_bounds__(256, sizeof(S) == 4 ? 2 : 3)
    k_main_tma(const __grid_constant__ DevP<T> P, const __grid_constant__ MainMaps M, const Pops<S> src,
               const Pops<S> dst, const T *__restrict__ gA, const T *__restrict__ gB,
               const Control *__restrict__ ctl, const PhiRef<T> Rf, S *__restrict__ phiu,
               const T *__restrict__ psi_prev, T *__restrict__ snap, double *__restrict__ part,
               int *__restrict__ unstable, int *__restrict__ fault, int tiles_x, int ntiles)
{
    using L = TmaLayout<T, S>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    const int tid = threadIdx.x + threadIdx.y * 64;
    const int gsel = (ctl->cur0 + ctl->flips) & 1;
    // the copies need 128-byte aligned destinations (block-uniform check)
    if (smem_u32(smem_raw) & 127u) {
        if (tid == 0) atomicExch(fault, 2);
        return;
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    auto issue = [&](int t, int sidx) {
        unsigned char *base = smem_raw + (size_t)sidx * L::stage;
        const int x0 = (t % tiles_x) * 64, y0 = (t / tiles_x) * 4;
        mbar_expect_tx(&bar[sidx], L::tx(RESID) + P.tx_extra);
        tma_load_3d(base + L::pops, &M.pops, &bar[sidx], x0, y0, 0);
        tma_load_3d(base + L::pops + sizeof(S) * 27 * 256, &M.phiu, &bar[sidx], x0, y0, 0);
        tma_load_3d(base + L::tpl, gsel ? &M.g[1] : &M.g[0], &bar[sidx], x0, y0, 0);
        tma_load_2d(base + L::tpl + sizeof(T) * 4 * 256, &M.mur, &bar[sidx], x0, y0);
        tma_load_2d(base + L::tpl + sizeof(T) * 5 * 256, &M.gxr, &bar[sidx], x0, y0);
        tma_load_2d(base + L::tpl + sizeof(T) * 6 * 256, &M.gyr, &bar[sidx], x0, y0);
        if (RESID) tma_load_2d(base + L::tpl + sizeof(T) * 7 * 256, &M.psi, &bar[sidx], x0, y0);
        // rows y0 - 1 .. y0 + 4 are rows y0 .. y0 + 5 of the ghost-row arrays
        tma_load_2d(base + L::dphi, &M.dphi, &bar[sidx], x0 - TMA_HX, y0);
        tma_load_2d(base + L::phir, &M.phir, &bar[sidx], x0 - TMA_HX, y0);
    };
    if (tid == 0 && (int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
    int k = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
        const int sidx = k & 1;
        const bool late = !mbar_wait_bounded(&bar[sidx], (k >> 1) & 1);
        if (__syncthreads_or(late)) {   // every thread of the block leaves together
            if (tid == 0) atomicExch(fault, 1);
            mbar_wait_bounded(&bar[sidx], (k >> 1) & 1);   // the copies in flight
            return;
        }
        if (tid == 0 && t + (int)gridDim.x < ntiles) {
            fence_proxy_async();
            issue(t + gridDim.x, sidx ^ 1);
        }
        const unsigned char *base = smem_raw + (size_t)sidx * L::stage;
        const TmaView<T, S> tv{reinterpret_cast<const S *>(base + L::pops), reinterpret_cast<const T *>(base + L::tpl),
                               reinterpret_cast<const T *>(base + L::dphi), reinterpret_cast<const T *>(base + L::phir)};
        main_body<T, S, SNAP, FROZEN, RESID, false, 5, true>(P, src, dst, gA, gB, ctl, Rf, phiu, psi_prev, snap, part,
                                                             unstable, t % tiles_x, t / tiles_x, t, &tv);
    }
}

// The same with one tile per block and one stage (grid: every tile), sized
// for 4 resident blocks per SM in float: the blocks of an SM overlap one
// another's copies with their arithmetic instead of a block prefetching its
// next tile.  Dynamic shared memory TmaLayout<T, S>::stage.
template <typename T, typename S, bool SNAP, bool FROZEN, bool RESID>
__global__ void __launch_bounds__(256, MAIN_MINB<T>)
    k_main_tma1(const __grid_constant__ DevP<T> P, const __grid_constant__ MainMaps M, const Pops<S> src,
                const Pops<S> dst, const T *__restrict__ gA, const T *__restrict__ gB,
                const Control *__restrict__ ctl, const PhiRef<T> Rf, S *__restrict__ phiu,
                const T *__restrict__ psi_prev, T *__restrict__ snap, double *__restrict__ part,
                int *__restrict__ unstable, int *__restrict__ fault)
{
    griddep_begin();
    using L = TmaLayout<T, S>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    const int tid = threadIdx.x + threadIdx.y * 64;
    if (smem_u32(smem_raw) & 127u) {
        if (tid == 0) atomicExch(fault, 2);
        return;
    }
    const int x0 = blockIdx.x * 64, y0 = blockIdx.y * 4;
    if (tid == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
        const int gsel = (ctl->cur0 + ctl->flips) & 1;
        mbar_expect_tx(&bar, L::tx(RESID) + P.tx_extra);
        tma_load_3d(smem_raw + L::pops, &M.pops, &bar, x0, y0, 0);
        tma_load_3d(smem_raw + L::pops + sizeof(S) * 27 * 256, &M.phiu, &bar, x0, y0, 0);
        tma_load_3d(smem_raw + L::tpl, gsel ? &M.g[1] : &M.g[0], &bar, x0, y0, 0);
        tma_load_2d(smem_raw + L::tpl + sizeof(T) * 4 * 256, &M.mur, &bar, x0, y0);
        tma_load_2d(smem_raw + L::tpl + sizeof(T) * 5 * 256, &M.gxr, &bar, x0, y0);
        tma_load_2d(smem_raw + L::tpl + sizeof(T) * 6 * 256, &M.gyr, &bar, x0, y0);
        if (RESID) tma_load_2d(smem_raw + L::tpl + sizeof(T) * 7 * 256, &M.psi, &bar, x0, y0);
        tma_load_2d(smem_raw + L::dphi, &M.dphi, &bar, x0 - TMA_HX, y0);
        tma_load_2d(smem_raw + L::phir, &M.phir, &bar, x0 - TMA_HX, y0);
    }
    __syncthreads();   // the barrier is initialised before anyone waits on it
    const bool late = !mbar_wait_bounded(&bar, 0);
    if (__syncthreads_or(late)) {
        if (tid == 0) atomicExch(fault, 1);
        mbar_wait_bounded(&bar, 0);
        return;
    }
    const TmaView<T, S> tv{reinterpret_cast<const S *>(smem_raw + L::pops),
                           reinterpret_cast<const T *>(smem_raw + L::tpl),
                           reinterpret_cast<const T *>(smem_raw + L::dphi),
                           reinterpret_cast<const T *>(smem_raw + L::phir)};
    main_body<T, S, SNAP, FROZEN, RESID, false, 5, true>(P, src, dst, gA, gB, ctl, Rf, phiu, psi_prev, snap, part,
                                                         unstable, blockIdx.x, blockIdx.y,
                                                         blockIdx.x + (long long)blockIdx.y * gridDim.x, &tv);
}

// End of step (one block of 256): global sums of the main kernel (when it
// reduced), the step's residual, counters, the next step's g parity.
//   resid: 0 none; 1 from the main kernel's partials (columns 2, 3 of 4);
//          2 from the fused sweep kernel's partials (2 per block in part2).
// First stage of a two-stage sum of NV-wide block partials in a fixed order:
// thread t of block b adds the partials b * 256 + t + k * 256 G (G = gridDim.x),
// the block's tree sum goes to out[NV * b].  The end of step then sums the G
// results in one block.
template <int NV>
__global__ void __launch_bounds__(256) k_partials(const double *__restrict__ part, long long nb, double *out)
{
    griddep_begin();
    __shared__ double red[256][NV];
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < nb; i += 256LL * gridDim.x)
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] += part[NV * i + k];
#pragma unroll
    for (int k = 0; k < NV; ++k) red[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
#pragma unroll
            for (int k = 0; k < NV; ++k) red[threadIdx.x][k] += red[threadIdx.x + s][k];
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) out[NV * blockIdx.x + k] = red[0][k];
}

__device__ __forceinline__ void step_end_body(const double *__restrict__ part, long long nb,
                                              const double *__restrict__ part2, long long nb2, Control *ctl,
                                              int *counts, int resid, int sums)
{
    double tot[4] = {0.0, 0.0, 0.0, 0.0};
    if (resid == 1 || sums) sum_partials<4>(part, nb, tot);
    if (resid == 2) {
        __syncthreads();
        double t2[2];
        sum_partials<2>(part2, nb2, t2);
        tot[2] = t2[0];
        tot[3] = t2[1];
    }
    if (threadIdx.x == 0) {
        const int K = ctl->K;
        double r = ctl->r_last;
        if (!ctl->early) {
            if (resid && K >= 1) r = tot[3] > 0.0 ? sqrt(tot[2] / tot[3]) : sqrt(tot[2]);
            else r = nan("");
        }
        ctl->r_step = r;
        if (sums) {
            ctl->sum_phi = tot[0];
            ctl->sum_q = tot[1];
        }
        if (counts) counts[ctl->tloc] = K;
        ctl->sweeps_total += K;
        if (K > ctl->sweeps_max) ctl->sweeps_max = K;
        if (ctl->converge && ctl->kmax > ctl->kmin && K >= ctl->kmax && !(r < ctl->tol)) ctl->notconv += 1;
        ctl->cur0 = (ctl->cur0 + ctl->flips) & 1;
        ctl->t += 1;
        ctl->tloc += 1;
        ctl->tpar ^= 1;
    }
}

static __global__ void __launch_bounds__(256) k_step_end(const double *__restrict__ part, long long nb,
                                                         const double *__restrict__ part2, long long nb2,
                                                         Control *ctl, int *counts, int resid, int sums)
{
    griddep_begin();
    step_end_body(part, nb, part2, nb2, ctl, counts, resid, sums);
}

// ---- initial state (Sec. 6 set-up) ------------------------------------------------

template <typename T, typename S, int QI = 5>
__global__ void __launch_bounds__(256) k_init_state(const DevP<T> P, Pops<S> pops, T *__restrict__ g,
                                                    S *__restrict__ phiu, PhiRef<T> Rf, double xc, double yc,
                                                    double R, double Wi, int shape, int psi_zero)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const long long nn = P.nn, k = (long long)y * P.nx + x;
    const double r = shape == 1 ? fabs(y - yc) : sqrt((x - xc) * (x - xc) + (y - yc) * (y - yc));
    const T phi0 = (T)(0.5 * (1.0 + tanh(2.0 * (R - r) / Wi)));
    // h = w_i phi0 at rest is exactly the reference state: deviations 0
#pragma unroll
    for (int i = 0; i < 9; ++i) sts(pops.h + i * nn + k, T(0), P.sc_h);
    const long long gk = (long long)(y + 1) * P.nx + x;
    Rf.phir[gk] = phi0;
    if (y == 0) Rf.phir[x] = phi0;
    if (y == P.ny - 1) Rf.phir[(long long)(P.ny + 1) * P.nx + x] = phi0;
#pragma unroll
    for (int i = 0; i < 8; ++i) sts(pops.f + i * nn + k, T(0), P.sc_f);
    // p, n are set by k_init_ions
#pragma unroll
    for (int i = 0; i < QI; ++i) { sts(pops.p + i * nn + k, T(0), P.sc_c); sts(pops.n + i * nn + k, T(0), P.sc_c); }
    sts(phiu + k, T(0), P.sc_u);
    sts(phiu + nn + k, T(0), P.sc_u);
    const T w = T(1) / T(6);
    if (psi_zero) {
        const T v = -w * psi_lin(P, y);
#pragma unroll
        for (int i = 0; i < 4; ++i) g[i * nn + k] = v;
    } else {  // linear profile with the non-equilibrium part giving E = -grad psi
        g[k] = T(0);
        g[nn + k] = -P.tau_g * w * P.G;
        g[2 * nn + k] = T(0);
        g[3 * nn + k] = P.tau_g * w * P.G;
    }
}

// Gradient (Eq. 59) and chemical potential (Eq. 13) of the stored reference
// field, evaluated in double from its stored values.
template <typename T>
__global__ void __launch_bounds__(256) k_init_ref(const DevP<T> P, PhiRef<T> Rf, double beta, double kappa)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const int nx = P.nx;
    const long long k = (long long)y * nx + x;
    const int xm = nbx(x, -1, nx, P.side_walls), xp = nbx(x, 1, nx, P.side_walls);
    const T *r0 = Rf.phir + (long long)y * nx, *r1 = r0 + nx, *r2 = r1 + nx;
    const double c = r1[x];
    const double E = r1[xp], W = r1[xm], N = r2[x], S = r0[x];
    const double NE = r2[xp], NW = r2[xm], SW = r0[xm], SE = r0[xp];
    const double gx = (E - W) / 3.0 + ((NE - NW) + (SE - SW)) / 12.0;
    const double gy = (N - S) / 3.0 + ((NE + NW) - (SE + SW)) / 12.0;
    const double lap = 2.0 / 3.0 * (((E - c) + (W - c)) + ((N - c) + (S - c))) +
                       1.0 / 6.0 * (((NE - c) + (SW - c)) + ((NW - c) + (SE - c)));
    Rf.gxr[k] = (T)gx;
    Rf.gyr[k] = (T)gy;
    Rf.mur[k] = (T)(4.0 * beta * c * (c - 1.0) * (c - 0.5) - kappa * lap);
}

template <typename T, typename S, int QI = 5>
__global__ void __launch_bounds__(256) k_init_ions(const DevP<T> P, Pops<S> pops, const T *__restrict__ gA,
                                                   const T *__restrict__ gB, const Control *__restrict__ ctl,
                                                   const T *__restrict__ phig, T *__restrict__ snap,
                                                   double c_scale, double c0)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const long long nn = P.nn, k = (long long)y * P.nx + x;
    const T *__restrict__ g = ((ctl->cur0 + ctl->flips) & 1) ? gB : gA;
    const T g1 = g[k], g2 = g[nn + k], g3 = g[2 * nn + k], g4 = g[3 * nn + k];
    const T psi = T(1.5) * ((g1 + g3) + (g2 + g4)) + psi_lin(P, y);
    T Ex, Ey;
    if (P.freeze_E) { Ex = P.Ex_frozen; Ey = P.Ey_frozen; }
    else { Ex = T(3) * (g1 - g3) / P.tau_g; Ey = T(3) * (g2 - g4) / P.tau_g; }
    T ceq;
    if (P.k_r > T(0) && P.onsager_form != 2) {
        const T b = P.cb * dsqrt<T>(dsqrt<T>(Ex * Ex + Ey * Ey));
        ceq = dsqrt<T>(P.k_d * onsager<T>(b, P.onsager_form) / P.k_r);
    } else {
        ceq = (T)c0;
    }
    ceq = (T)c_scale * ceq;
    T sp = T(0), sn = T(0);
#pragma unroll
    for (int i = 0; i < QI; ++i) {
        const T wi = QI == 9 ? w9<T>(i) : (i == 0 ? T(1) / T(3) : T(1) / T(6));
        const T v = wi * ceq;
        const T vs = kSame<S, T> ? v : v - wi * P.cref;
        sts(pops.p + i * nn + k, vs, P.sc_c);
        sts(pops.n + i * nn + k, vs, P.sc_c);
        sp += v;
        sn += v;
    }
    const T phi = phig[(long long)(y + 1) * P.nx + x];
    snap[k] = phi;
    snap[nn + k] = T(0);
    snap[2 * nn + k] = T(0);
    snap[3 * nn + k] = T(0);
    snap[4 * nn + k] = psi;
    snap[5 * nn + k] = Ex;
    snap[6 * nn + k] = Ey;
    snap[7 * nn + k] = sp;
    snap[8 * nn + k] = sn;
    snap[9 * nn + k] = sp - sn;
}

// ---- state transfer (checkpoint / test hook) ---------------------------------------
// Packs rows [y0, y0 + rows) of the state into 25 + 2 QI doubles per node:
// f0..f8, h0..h8, p (QI), n (QI), g0..g4, (phi u)(t-1) x, y.
template <typename T, typename S, int QI = 5>
__global__ void k_pack_state(const DevP<T> P, const Pops<S> pops, const T *__restrict__ g,
                             const S *__restrict__ phiu, const T *__restrict__ phir, double *__restrict__ out,
                             int y0, int rows)
{
    constexpr int SPN = 25 + 2 * QI, G0 = 18 + 2 * QI;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long cnt = (long long)rows * P.nx;
    if (i >= cnt) return;
    const int y = y0 + (int)(i / P.nx);
    const long long nn = P.nn, k = (long long)y0 * P.nx + i;
    double *o = out + SPN * i;
    o[0] = 0.0;
    for (int q = 1; q < 9; ++q) o[q] = (double)lds(pops.f + (q - 1) * nn + k, P.isc_f);
    const double pr = (double)phir[(long long)(y + 1) * P.nx + (k - (long long)y * P.nx)];
    for (int q = 0; q < 9; ++q) o[9 + q] = (double)lds(pops.h + q * nn + k, P.isc_h) + (double)w9<T>(q) * pr;
    const double cr = (double)P.cref;
    for (int q = 0; q < QI; ++q) {
        const double wq = QI == 9 ? (double)w9<double>(q) : (q == 0 ? 1.0 / 3.0 : 1.0 / 6.0);
        o[18 + q] = (double)lds(pops.p + q * nn + k, P.isc_c) + wq * cr;
        o[18 + QI + q] = (double)lds(pops.n + q * nn + k, P.isc_c) + wq * cr;
    }
    const double pl = (double)psi_lin(P, y);
    o[G0] = 0.0;
    for (int q = 0; q < 4; ++q) o[G0 + 1 + q] = (double)g[q * nn + k] + pl / 6.0;
    o[G0 + 5] = (double)lds(phiu + k, P.isc_u);
    o[G0 + 6] = (double)lds(phiu + nn + k, P.isc_u);
}

template <typename T, typename S, int QI = 5>
__global__ void k_unpack_state(const DevP<T> P, Pops<S> pops, T *__restrict__ g, S *__restrict__ phiu,
                               const T *__restrict__ phir, const double *__restrict__ in, int y0, int rows)
{
    constexpr int SPN = 25 + 2 * QI, G0 = 18 + 2 * QI;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long cnt = (long long)rows * P.nx;
    if (i >= cnt) return;
    const int y = y0 + (int)(i / P.nx);
    const long long nn = P.nn, k = (long long)y0 * P.nx + i;
    const double *o = in + SPN * i;
    for (int q = 1; q < 9; ++q) sts(pops.f + (q - 1) * nn + k, (T)o[q], P.sc_f);
    const double pr = (double)phir[(long long)(y + 1) * P.nx + (k - (long long)y * P.nx)];
    for (int q = 0; q < 9; ++q) sts(pops.h + q * nn + k, (T)(o[9 + q] - (double)w9<T>(q) * pr), P.sc_h);
    const double cr = (double)P.cref;
    for (int q = 0; q < QI; ++q) {
        const double wq = QI == 9 ? (double)w9<double>(q) : (q == 0 ? 1.0 / 3.0 : 1.0 / 6.0);
        sts(pops.p + q * nn + k, (T)(o[18 + q] - wq * cr), P.sc_c);
        sts(pops.n + q * nn + k, (T)(o[18 + QI + q] - wq * cr), P.sc_c);
    }
    const double pl = (double)psi_lin(P, y);
    for (int q = 0; q < 4; ++q) g[q * nn + k] = (T)(o[G0 + 1 + q] - pl / 6.0);
    sts(phiu + k, (T)o[G0 + 5], P.sc_u);
    sts(phiu + nn + k, (T)o[G0 + 6], P.sc_u);
}

template <typename T>
__global__ void k_to_double(const T *__restrict__ a, double *__restrict__ out, long long n)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)a[i];
}

// ---- deformation factor (Eq. 63) ------------------------------------------------

// Deformation factor D = (L - H) / (L + H) (Eq. 63) of the phi field (the
// first plane of a snapshot): L is the extent of phi >= 1/2 along the field
// (y) through the phi-weighted centroid, H the same across it (x); the line
// is sampled by bilinear interpolation of the nodes (x periodic, rows clamped
// at the walls) and each end is the crossing of 1/2 interpolated linearly
// between consecutive samples.
template <typename T>
__device__ __forceinline__ double phi_sample(const T *phi, int nx, int ny, double x, double y)
{
    int x0 = (int)floor(x), y0 = (int)floor(y);
    const double fx = x - x0, fy = y - y0;
    int x1 = x0 + 1, y1 = y0 + 1;
    x0 = ((x0 % nx) + nx) % nx;
    x1 = ((x1 % nx) + nx) % nx;
    y0 = min(max(y0, 0), ny - 1);
    y1 = min(max(y1, 0), ny - 1);
    // every product and sum rounded on its own, so that all kernels that
    // sample a line (one lattice, a batch) give the same bits
    const double gx = 1.0 - fx, gy = 1.0 - fy;
    const double a = __dadd_rn(__dmul_rn((double)phi[(long long)y0 * nx + x0], gx),
                               __dmul_rn((double)phi[(long long)y0 * nx + x1], fx));
    const double b = __dadd_rn(__dmul_rn((double)phi[(long long)y1 * nx + x0], gx),
                               __dmul_rn((double)phi[(long long)y1 * nx + x1], fx));
    return __dadd_rn(__dmul_rn(a, gy), __dmul_rn(b, fy));
}

// The phi-weighted sums of the centroid are taken over slices of the nodes in
// row-major order, deform_slices(nx, ny) of them of (near) equal size, each
// reduced by one block in a fixed order, so one lattice and the same lattice
// inside a batch give the same bits.
constexpr int DEF_MAX_SLICES = 1024;
constexpr int DEF_SLICE_NODES = 4096;

__host__ __device__ inline int deform_slices(int nx, int ny)
{
    const long long s = (long long)nx * ny / DEF_SLICE_NODES;
    return (int)(s < 1 ? 1 : (s > DEF_MAX_SLICES ? DEF_MAX_SLICES : s));
}

// Error-free sum of two floats (Knuth's TwoSum): returns s = fl(a + b) and
// sets e with s + e == a + b exactly.
__device__ __forceinline__ float two_sum(float a, float b, float &e)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

// (sum phi, sum phi x, sum phi y) over slice j of nsl (one block of 256);
// thread 0 writes the three sums to dst.
template <typename T>
__device__ __forceinline__ void deform_slice_sums(const T *__restrict__ phi, int nx, int ny, int j, int nsl,
                                                  double (*red)[3], double *dst)
{
    const long long nn = (long long)nx * ny;
    const long long k0 = j * nn / nsl, k1 = (j + 1) * nn / nsl;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    // (every product and sum is rounded on its own: the slice sums of one
    // lattice and of a batch come from different kernels and must agree)
    // FP32 fields: each thread keeps its sums as unevaluated float pairs
    // (hi + lo; exact products by fmaf, TwoSum additions), about 48 bits, and
    // hands them to double per row (sum phi, sum phi y) and at the end (sum
    // phi x): the FP32 pipe does the per-node work.
    float h1 = 0.f, l1 = 0.f;
    int y = (int)(k0 / nx);
    for (long long rowk = (long long)y * nx; rowk < k1; ++y, rowk += nx) {
        const int xs = (int)(k0 > rowk ? k0 - rowk : 0), xe = (int)(k1 - rowk < nx ? k1 - rowk : nx);
        const T *row = phi + rowk;
        const double fy = (double)y;
        if constexpr (sizeof(T) == 4) {
            const int x0 = xs + (int)threadIdx.x;
            if (x0 >= xe) continue;   // no node of this row for this thread
            float rh = 0.f, rl = 0.f;
            float xf = (float)x0;   // exact: x < 2^24
#pragma unroll 4
            for (int x = x0; x < xe; x += 256, xf = __fadd_rn(xf, 256.f)) {
                const float v = (float)row[x];
                float e;
                rh = two_sum(rh, v, e);
                rl = __fadd_rn(rl, e);
                const float p = __fmul_rn(v, xf), pe = __fmaf_rn(v, xf, -p);
                h1 = two_sum(h1, p, e);
                l1 = __fadd_rn(l1, __fadd_rn(e, pe));
            }
            const double r = __dadd_rn((double)rh, (double)rl);
            a0 = __dadd_rn(a0, r);
            a2 = __dadd_rn(a2, __dmul_rn(r, fy));
        } else {
#pragma unroll 4
            for (int x = xs + (int)threadIdx.x; x < xe; x += 256) {
                const double v = (double)row[x];
                a0 = __dadd_rn(a0, v);
                a1 = __dadd_rn(a1, __dmul_rn(v, (double)x));
                a2 = __dadd_rn(a2, __dmul_rn(v, fy));
            }
        }
    }
    a1 = __dadd_rn(a1, __dadd_rn((double)h1, (double)l1));
    red[threadIdx.x][0] = a0;
    red[threadIdx.x][1] = a1;
    red[threadIdx.x][2] = a2;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int i = 0; i < 3; ++i) red[threadIdx.x][i] += red[threadIdx.x + s][i];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int i = 0; i < 3; ++i) dst[i] = red[0][i];
    __syncthreads();
}

// End of the phi >= 1/2 run through (xc, yc) in direction sgn along y or x,
// searched by one warp 32 samples at a time: the first s = 1 .. lim-1 whose
// sample drops below 1/2 after one at or above it, interpolated linearly
// between the two; sgn * lim when there is none.
template <typename T>
__device__ __forceinline__ double phi_run_end(const T *phi, int nx, int ny, double xc, double yc, bool along_y,
                                              double sgn)
{
    const int lane = threadIdx.x & 31, lim = along_y ? ny : nx;
    double carry = phi_sample(phi, nx, ny, xc, yc);
    for (int base = 1; base < lim; base += 32) {
        const int s = base + lane;
        const double tt = sgn * (double)s;
        double v = 0.0;
        if (s < lim) v = along_y ? phi_sample(phi, nx, ny, xc, yc + tt) : phi_sample(phi, nx, ny, xc + tt, yc);
        double pv = __shfl_up_sync(0xffffffffu, v, 1);
        if (lane == 0) pv = carry;
        const bool hit = s < lim && pv >= 0.5 && v < 0.5;
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (m) {
            const int first = __ffs(m) - 1;
            double end = 0.0;
            if (lane == first) {
                const double pt = s == 1 ? 0.0 : sgn * (double)(s - 1);
                end = pt + (tt - pt) * (pv - 0.5) / (pv - v);
            }
            return __shfl_sync(0xffffffffu, end, first);
        }
        carry = __shfl_sync(0xffffffffu, v, 31);
    }
    return sgn * lim;
}

// D = (L - H) / (L + H) from the deform_slices(nx, ny) slice sums at parts
// (one block of 256; four warps search the four ends of the two axes).
template <typename T>
__device__ __forceinline__ void deform_finish(const T *__restrict__ phi, int nx, int ny, const double *parts,
                                              double (*red)[3], double *out)
{
    __shared__ double ends[4];
    const int nsl = deform_slices(nx, ny);
    for (int i = 0; i < 3; ++i) {
        double acc = 0.0;
        for (int j = threadIdx.x; j < nsl; j += 256) acc += parts[3 * j + i];
        red[threadIdx.x][i] = acc;
    }
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int i = 0; i < 3; ++i) red[threadIdx.x][i] += red[threadIdx.x + s][i];
        __syncthreads();
    }
    const double sphi = red[0][0];
    if (!(sphi > 0.0)) {
        if (threadIdx.x == 0) *out = 0.0;
        __syncthreads();
        return;
    }
    const double xc = red[0][1] / sphi, yc = red[0][2] / sphi;
    const int w = threadIdx.x >> 5;
    if (w < 4) {
        const double e = phi_run_end(phi, nx, ny, xc, yc, w >= 2, (w & 1) ? 1.0 : -1.0);
        if ((threadIdx.x & 31) == 0) ends[w] = e;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double L = ends[3] - ends[2], H = ends[1] - ends[0];
        *out = (L - H) / (L + H);
    }
    __syncthreads();
}

// Slice sums of one lattice (launch: deform_slices(nx, ny) blocks of 256).
template <typename T>
__global__ void __launch_bounds__(256) k_deform_sums(const T *__restrict__ phi, int nx, int ny, double *parts)
{
    griddep_begin();
    __shared__ double red[256][3];
    deform_slice_sums(phi, nx, ny, blockIdx.x, gridDim.x, red, parts + 3 * blockIdx.x);
}

// D of one lattice from its slice sums (launch: 1 block of 256).
template <typename T>
__global__ void __launch_bounds__(256) k_deform_finish(const T *__restrict__ phi, int nx, int ny,
                                                       const double *__restrict__ parts, double *out)
{
    griddep_begin();
    __shared__ double red[256][3];
    deform_finish(phi, nx, ny, parts, red, out);
}

}  // namespace ehdlb
