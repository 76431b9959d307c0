// ehdlb_solver.cuh -- host side of one lattice: device buffers, the initial
// state, the kernel sequence of a time step, transfers.  Instantiated with
// arithmetic type T and population storage type S: (float, float) in
// solver_fp32.cu, (double, double) in solver_fp64.cu and (float, __half) in
// solver_fp16s.cu.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "ehdlb.h"
#include "ehdlb_kernels.cuh"
#include "ehdlb_solver_base.h"

namespace ehdlb {

// cuTensorMapEncodeTiled of the driver, resolved through the runtime (no
// link against the driver library); nullptr if unavailable.
using TensorMapEncodeFn = decltype(&cuTensorMapEncodeTiled);
inline TensorMapEncodeFn tensor_map_encoder()
{
    static TensorMapEncodeFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (TensorMapEncodeFn) nullptr;
        return reinterpret_cast<TensorMapEncodeFn>(p);
    }();
    return fn;
}

// A tiled map of `planes` planes of an nx x rows array of E (planes > 1:
// rank 3, planes nn elements apart), box (bw, bh, planes).
template <typename E>
bool encode_tiles(CUtensorMap *m, const void *base, int nx, int rows, int planes, long long nn, int bw, int bh)
{
    TensorMapEncodeFn enc = tensor_map_encoder();
    if (!enc) return false;
    const CUtensorMapDataType dt = sizeof(E) == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)rows, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * sizeof(E), (cuuint64_t)nn * sizeof(E)};
    const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, (cuuint32_t)planes};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, dt, planes > 1 ? 3 : 2, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

#define EHDLB_CK(call)                                                              \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            err = std::string(#call) + ": " + cudaGetErrorString(e_);               \
            return e_ == cudaErrorMemoryAllocation ? EHDLB_ENOMEM : EHDLB_ECUDA;    \
        }                                                                           \
    } while (0)

template <typename T, typename S = T> class Solver : public SolverBase {
  public:
    static constexpr int BX = 64, BY = 4;

    Solver(int nx, int ny, cudaStream_t s, DevArena *arena = nullptr)
        : nx_(nx), ny_(ny), nn_((long long)nx * ny), stream_(s), arena_(arena)
    {
    }

    ~Solver() override
    {
        for (void *p : allocs_) {
            if (arena_) arena_->release(p);
            else cudaFree(p);
        }
        for (cudaEvent_t e : events_) cudaEventDestroy(e);
        if (pin_) cudaFreeHost(pin_);
        if (own_stream_) cudaStreamDestroy(stream_);
    }

    int allocate(std::string &err)
    {
        if (!stream_) {
            EHDLB_CK(cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking));
            own_stream_ = true;
        }
        grid_ = dim3((nx_ + BX - 1) / BX, (ny_ + BY - 1) / BY);
        nb_ = (long long)grid_.x * grid_.y;
        {
            int dev = 0;
            EHDLB_CK(cudaGetDevice(&dev));
            EHDLB_CK(cudaDeviceGetAttribute(&sms_, cudaDevAttrMultiProcessorCount, dev));
        }
        const size_t plane = sizeof(T) * (size_t)nn_, splane = sizeof(S) * (size_t)nn_;
        for (int b = 0; b < 2; ++b) {
            EHDLB_CK(alloc_pops(b, 5));
            EHDLB_CK(alloc((void **)&g_[b], plane * 4));
        }
        // 16-byte staging of the main kernel: every row starts on a 16-byte boundary
        vec_ok_ = ((size_t)nx_ * sizeof(S)) % 16 == 0 && ((size_t)nx_ * sizeof(T)) % 16 == 0;
        EHDLB_CK(alloc((void **)&phig_, sizeof(T) * (size_t)(ny_ + 2) * nx_));
        EHDLB_CK(alloc((void **)&ref_.phir, sizeof(T) * (size_t)(ny_ + 2) * nx_));
        EHDLB_CK(alloc((void **)&ref_.dphig, sizeof(T) * (size_t)(ny_ + 2) * nx_));
        EHDLB_CK(alloc((void **)&ref_.gxr, plane));
        EHDLB_CK(alloc((void **)&ref_.gyr, plane));
        EHDLB_CK(alloc((void **)&ref_.mur, plane));
        EHDLB_CK(alloc((void **)&q_, plane));
        EHDLB_CK(alloc((void **)&coef_, plane * 3));
        EHDLB_CK(alloc((void **)&phiu_, splane * 2));
        EHDLB_CK(alloc((void **)&psi_prev_, plane));
        EHDLB_CK(alloc((void **)&snap_, plane * EHDLB_NFIELDS));
        EHDLB_CK(alloc((void **)&part_, sizeof(double) * 4 * (size_t)nb_));
        EHDLB_CK(alloc((void **)&ctl_, sizeof(Control)));
        {
            long long nbmax = 0;
            for (int nsw = 1; nsw <= TB_MAX; ++nsw)
                for (int sh = 0; sh < TB_NSHAPES; ++sh) {
                    const dim3 g = tb_grid(nsw, sh, nx_, ny_);
                    nbmax = std::max(nbmax, (long long)g.x * g.y);
                }
            EHDLB_CK(alloc((void **)&part2_, sizeof(double) * 2 * (size_t)nbmax));
        }
        EHDLB_CK((main_attr<true, true, false>()));
        EHDLB_CK((main_attr<true, false, true>()));
        EHDLB_CK((main_attr<true, false, false>()));
        EHDLB_CK((main_attr<false, true, false>()));
        EHDLB_CK((main_attr<false, false, true>()));
        EHDLB_CK((main_attr<false, false, false>()));
        if constexpr (kTmaMain) {
            EHDLB_CK((tma_attr<true, true, false>()));
            EHDLB_CK((tma_attr<true, false, true>()));
            EHDLB_CK((tma_attr<true, false, false>()));
            EHDLB_CK((tma_attr<false, true, false>()));
            EHDLB_CK((tma_attr<false, false, true>()));
            EHDLB_CK((tma_attr<false, false, false>()));
        }
        EHDLB_CK(tb_attr<1>());
        EHDLB_CK(tb_attr<2>());
        if constexpr (TB_MAX >= 5) {
            EHDLB_CK(tb_attr<3>());
            EHDLB_CK(tb_attr<4>());
            EHDLB_CK(tb_attr<5>());
        }
        EHDLB_CK(alloc((void **)&stage_, sizeof(double) * (size_t)nn_));
        EHDLB_CK(alloc((void **)&red_, sizeof(double) * (6 * PSUM + 3 * DEF_MAX_SLICES)));
        EHDLB_CK(cudaMemsetAsync(snap_, 0, plane * EHDLB_NFIELDS, stream_));
        EHDLB_CK(cudaStreamSynchronize(stream_));
        encode_main_maps();
        return EHDLB_OK;
    }

    int set_params(const ehdlb_params &p, std::string &err) override
    {
        P_ = p;
        make_devp();
        snap_valid_ = (1u << EHDLB_NFIELDS) - 1;   // the initial fields are captured whole
        const int qi = p.ion_lattice == 9 ? 9 : 5;
        if (qi != qi_) {   // the ion lattice sets the size of the population blocks
            EHDLB_CK(cudaStreamSynchronize(stream_));
            EHDLB_CK(alloc_pops(0, qi));
            EHDLB_CK(alloc_pops(1, qi));
            encode_main_maps();
        }
        Control c{};
        c.cur0 = 0;
        c.tol = p.sweep_tol;
        c.r_last = NAN;
        c.r_step = NAN;
        ctl_h_ = c;
        EHDLB_CK(cudaMemcpyAsync(ctl_, &ctl_h_, sizeof(Control), cudaMemcpyHostToDevice, stream_));
        const double Wi = p.W_init > 0.0 ? p.W_init : p.W;
        if (qi_ == 9)
            k_init_state<T, S, 9><<<grid_, dim3(BX, BY), 0, stream_>>>(dp_, pops_[0], g_[0], phiu_, ref_, p.xc, p.yc,
                                                                      p.R, Wi, p.init_shape, p.init_psi_zero);
        else
            k_init_state<T, S, 5><<<grid_, dim3(BX, BY), 0, stream_>>>(dp_, pops_[0], g_[0], phiu_, ref_, p.xc, p.yc,
                                                                      p.R, Wi, p.init_shape, p.init_psi_zero);
        EHDLB_CK(cudaGetLastError());
        k_init_ref<T><<<grid_, dim3(BX, BY), 0, stream_>>>(dp_, ref_, 12.0 * p.sigma / p.W, 1.5 * p.sigma * p.W);
        EHDLB_CK(cudaGetLastError());
        // initial potential solve with q = 0 (p = n = 0 at this point)
        if (p.freeze_E) {
            launch_prep(0, 0, 0, 0, 0);
        } else if (p.init_sweeps_fixed >= 0) {
            launch_prep(0, p.init_sweeps_fixed, p.init_sweeps_fixed, p.init_sweeps_fixed, p.init_sweeps_fixed);
            for (int j = 1; j <= p.init_sweeps_fixed; ++j) launch_sweep(j, false, false, false);
        } else {
            launch_prep(0, -1, 0, p.init_sweeps_max, 0);
            const int chunk = 256;
            for (int j0 = 1; j0 <= p.init_sweeps_max; j0 += chunk) {
                const int j1 = std::min(p.init_sweeps_max, j0 + chunk - 1);
                for (int j = j0; j <= j1; ++j) {
                    launch_sweep(j, true, j >= 2, true);
                    k_sweep_decide<<<1, 256, 0, stream_>>>(part_, nb_, ctl_, j);
                }
                EHDLB_CK(cudaGetLastError());
                EHDLB_CK(cudaMemcpyAsync(&ctl_h_, ctl_, sizeof(Control), cudaMemcpyDeviceToHost, stream_));
                EHDLB_CK(cudaStreamSynchronize(stream_));
                if (ctl_h_.done) break;
            }
        }
        EHDLB_CK(cudaGetLastError());
        if (qi_ == 9)
            k_init_ions<T, S, 9><<<grid_, dim3(BX, BY), 0, stream_>>>(dp_, pops_[0], g_[0], g_[1], ctl_, phig_, snap_,
                                                                     p.c_init_scale, p.c0);
        else
            k_init_ions<T, S, 5><<<grid_, dim3(BX, BY), 0, stream_>>>(dp_, pops_[0], g_[0], g_[1], ctl_, phig_, snap_,
                                                                     p.c_init_scale, p.c0);
        EHDLB_CK(cudaGetLastError());
        EHDLB_CK(cudaMemcpyAsync(&ctl_h_, ctl_, sizeof(Control), cudaMemcpyDeviceToHost, stream_));
        EHDLB_CK(cudaStreamSynchronize(stream_));
        init_sweeps_ = ctl_h_.K;
        c = Control{};
        c.cur0 = (ctl_h_.cur0 + ctl_h_.flips) & 1;
        c.tol = p.sweep_tol;
        c.r_last = NAN;
        c.r_step = NAN;
        ctl_h_ = c;
        EHDLB_CK(cudaMemcpyAsync(ctl_, &ctl_h_, sizeof(Control), cudaMemcpyHostToDevice, stream_));
        EHDLB_CK(cudaStreamSynchronize(stream_));
        tpar_ = 0;
        t_ = 0;
        return EHDLB_OK;
    }

    void set_schedule(const int *c, int n) override { sched_.assign(c, c + n); }
    // the tensor maps of the staged step kernel for the two time levels
    // (false if this lattice cannot take it)
    bool main_maps(MainMaps (&m)[2]) const
    {
        if (!(kTmaMain && tma_ok_ && qi_ == 5 && !P_.side_walls)) return false;
        m[0] = maps_[0];
        m[1] = maps_[1];
        return true;
    }
    int stall_next_copies() override
    {
        if (!(kTmaMain && tma_ && tma_ok_ && qi_ == 5 && !P_.side_walls)) return EHDLB_ESTATE;
        stall_ = true;
        return EHDLB_OK;
    }
    void set_timing(int every) override { timing_ = every > 0 ? every : 0; }
    void set_tuning(int sweeps_per_launch, int shape, int vec_staging) override
    {
        if (sweeps_per_launch >= 0) tb_chunk_ = sweeps_per_launch;
        if (shape >= 0) tb_shape_ = shape < TB_NSHAPES ? shape : 0;
        if (vec_staging >= 0) {
            vec_ = vec_staging != 0;
            tma_ = vec_staging >= 2;
            tma_persist_ = vec_staging == 3;
        }
    }

    int step(int nsteps, ehdlb_stats *st, std::string &err) override
    {
        const auto t0 = std::chrono::steady_clock::now();
        if (nsteps > counts_cap_) {
            int *nc;
            EHDLB_CK(alloc((void **)&nc, sizeof(int) * (size_t)nsteps));
            counts_ = nc;
            counts_cap_ = nsteps;
        }
        EHDLB_CK(pinned());
        if (timing_ && (int)events_.size() < 4 * nsteps) {
            while ((int)events_.size() < 4 * nsteps) {
                cudaEvent_t e;
                EHDLB_CK(cudaEventCreate(&e));
                events_.push_back(e);
            }
        }
        launches_ = 0;
        sweep_launches_ = 0;
        dp_.tx_extra = stall_ ? 16u : 0u;   // test hook: one call whose staged copies never complete
        stall_ = false;
        // open the call: per-call counters
        k_open_call<<<1, 1, 0, stream_>>>(ctl_);
        ++launches_;
        for (int s = 0; s < nsteps; ++s) {
            enqueue_step(s, s == nsteps - 1);
            EHDLB_CK(cudaGetLastError());
        }
        if (deform_each_) {   // D of the last step, read back with the control block
            EHDLB_CK(enqueue_deformation());
            launches_ += 2;
        }
        EHDLB_CK(cudaMemcpyAsync(&pin_->c, ctl_, sizeof(Control), cudaMemcpyDeviceToHost, stream_));
        EHDLB_CK(cudaStreamSynchronize(stream_));
        EHDLB_CK(cudaGetLastError());
        ctl_h_ = pin_->c;
        if (nsteps > 0) snap_valid_ = snap_mask_;
        last_nsteps = nsteps;
        const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (st) {
            st->steps = nsteps;
            st->t = ctl_h_.t;
            st->sweeps_total = ctl_h_.sweeps_total;
            st->sweeps_max = ctl_h_.sweeps_max;
            st->not_converged = ctl_h_.notconv;
            st->last_residual = ctl_h_.r_step;
            st->sum_phi = ctl_h_.sum_phi;
            st->sum_q = ctl_h_.sum_q;
            st->seconds = secs;
            st->mlups = secs > 0 ? (double)nn_ * nsteps / secs / 1e6 : 0.0;
            st->ms_prep = st->ms_sweeps = st->ms_main = 0.0;
            if (timing_) {
                // the recorded steps, scaled to all steps of the call
                int nrec = 0;
                for (int s = 0; s < nsteps; s += timing_) {
                    float a = 0, b = 0, c = 0;
                    cudaEventElapsedTime(&a, events_[4 * s], events_[4 * s + 1]);
                    cudaEventElapsedTime(&b, events_[4 * s + 1], events_[4 * s + 2]);
                    cudaEventElapsedTime(&c, events_[4 * s + 2], events_[4 * s + 3]);
                    st->ms_prep += a;
                    st->ms_sweeps += b;
                    st->ms_main += c;
                    ++nrec;
                }
                if (nrec > 0) {
                    const double f = (double)nsteps / nrec;
                    st->ms_prep *= f;
                    st->ms_sweeps *= f;
                    st->ms_main *= f;
                }
            }
            st->launches = launches_;
            st->sweep_launches = sweep_launches_;
            st->sweeps_per_launch = tb_chunk();
            st->tile_shape = tb_shape_;
            st->deformation = deform_each_ && nsteps > 0 ? pin_->D : NAN;
        }
        if (ctl_h_.fault) {
            err = "a staged copy of the step kernel did not arrive in time";
            return EHDLB_ECUDA;
        }
        if (ctl_h_.unstable) {
            err = "NaN or Inf in the fields";
            return EHDLB_EUNSTABLE;
        }
        return ctl_h_.notconv > 0 ? EHDLB_WNOTCONV : EHDLB_OK;
    }

    int get_fields(unsigned mask, double *dst, std::string &err) override
    {
        if (mask & ~snap_valid_) {
            err = "a requested field was not captured by the last step (ehdlb_set_reporting)";
            return EHDLB_ESTATE;
        }
        size_t off = 0;
        const int nthr = 256;
        const unsigned nblk = (unsigned)((nn_ + nthr - 1) / nthr);
        for (int f = 0; f < EHDLB_NFIELDS; ++f) {
            if (!(mask & (1u << f))) continue;
            k_to_double<T><<<nblk, nthr, 0, stream_>>>(snap_ + (size_t)f * nn_, stage_, nn_);
            EHDLB_CK(cudaGetLastError());
            EHDLB_CK(cudaMemcpyAsync(dst + off, stage_, sizeof(double) * (size_t)nn_, cudaMemcpyDeviceToHost,
                                     stream_));
            off += (size_t)nn_;
        }
        EHDLB_CK(cudaStreamSynchronize(stream_));
        return EHDLB_OK;
    }

    int get_counts(int *dst, int n, std::string &err) override
    {
        if (n <= 0) return EHDLB_OK;
        EHDLB_CK(cudaMemcpyAsync(dst, counts_, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost, stream_));
        EHDLB_CK(cudaStreamSynchronize(stream_));
        return EHDLB_OK;
    }

    int get_state(double *dst, std::string &err) override { return transfer_state(dst, nullptr, err); }

    // D of Eq. 63 from the phi of the last snapshot
    int deformation(double *out, std::string &err) override
    {
        if (!(snap_valid_ & 1u)) {
            err = "phi was not captured by the last step (ehdlb_set_reporting)";
            return EHDLB_ESTATE;
        }
        EHDLB_CK(pinned());
        EHDLB_CK(enqueue_deformation());
        EHDLB_CK(cudaStreamSynchronize(stream_));
        *out = pin_->D;
        return EHDLB_OK;
    }

    void set_reporting(unsigned snap_mask, int deformation) override
    {
        deform_each_ = deformation != 0;
        snap_mask_ = (snap_mask & ((1u << EHDLB_NFIELDS) - 1)) | (deform_each_ ? 1u : 0u);
        dp_.snap_mask = snap_mask_;
    }
    int set_state(const double *src, std::string &err) override { return transfer_state(nullptr, src, err); }

  private:
    // D of Eq. 63 from the snapshot's phi into the page-locked mirror (on
    // the stream; the caller synchronises)
    cudaError_t enqueue_deformation()
    {
        double *parts = red_ + 6 * PSUM;
        launch_k(k_deform_sums<T>, dim3(deform_slices(nx_, ny_)), dim3(256), 0, true, snap_, nx_, ny_, parts);
        launch_k(k_deform_finish<T>, dim3(1), dim3(256), 0, true, snap_, nx_, ny_, parts, stage_);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&pin_->D, stage_, sizeof(double), cudaMemcpyDeviceToHost, stream_);
        return e;
    }

    // page-locked host copy of the control block and D, read back by every
    // step call and deformation (allocated on first use: cases of a batch
    // never need it)
    cudaError_t pinned()
    {
        return pin_ ? cudaSuccess : cudaHostAlloc((void **)&pin_, sizeof(HostMirror), cudaHostAllocDefault);
    }

    cudaError_t alloc(void **p, size_t bytes)
    {
        cudaError_t e = arena_ ? arena_->alloc(p, bytes) : cudaMalloc(p, bytes);
        if (e == cudaSuccess) allocs_.push_back(*p);
        return e;
    }

    // f, h, p, n of time level b for QI ion populations per species (the
    // previous block, if any, is released first)
    cudaError_t alloc_pops(int b, int qi)
    {
        if (pops_[b].f) {
            void *old = pops_[b].f;
            for (auto it = allocs_.begin(); it != allocs_.end(); ++it)
                if (*it == old) { allocs_.erase(it); break; }
            if (arena_) arena_->release(old);
            else cudaFree(old);
            pops_[b] = Pops<S>{};
        }
        S *base;
        const cudaError_t e = alloc((void **)&base, sizeof(S) * (size_t)nn_ * (17 + 2 * qi));
        if (e != cudaSuccess) return e;
        pops_[b].f = base;
        pops_[b].h = base + 8 * nn_;
        pops_[b].p = base + 17 * nn_;
        pops_[b].n = base + (17 + qi) * nn_;
        qi_ = qi;
        return cudaSuccess;
    }

  public:
    int state_per_node() const override { return 25 + 2 * qi_; }

    // Device bytes of one lattice of nx x ny nodes (what allocate() takes,
    // rounded up to 256-byte blocks; the per-call counters excluded).
    static size_t footprint(int nx, int ny)
    {
        const size_t nn = (size_t)nx * ny, t = sizeof(T), s = sizeof(S);
        const size_t gx = (size_t)(nx + BX - 1) / BX, gy = (size_t)(ny + BY - 1) / BY;
        size_t nbmax = 0;
        for (int nsw = 1; nsw <= TB_MAX; ++nsw)
            for (int sh = 0; sh < TB_NSHAPES; ++sh) {
                const dim3 g = tb_grid(nsw, sh, nx, ny);
                nbmax = std::max(nbmax, (size_t)g.x * g.y);
            }
        const size_t planes_row = (size_t)(ny + 2) * nx;
        // one entry per allocation of allocate(), in its order
        const size_t b[] = {27 * nn * s, 4 * nn * t, 27 * nn * s, 4 * nn * t,
                            planes_row * t, planes_row * t, planes_row * t,
                            nn * t, nn * t, nn * t, nn * t, 3 * nn * t, 2 * nn * s, nn * t,
                            EHDLB_NFIELDS * nn * t, 4 * gx * gy * 8, sizeof(Control), 2 * nbmax * 8, nn * 8,
                            (size_t)(6 * PSUM + 3 * DEF_MAX_SLICES) * 8};
        size_t tot = 0;
        for (size_t v : b) tot += (v + 255) / 256 * 256;
        return tot;
    }

    // Pointers and constants of this lattice for the batched kernels.
    void describe(DevP<T> &P, Pops<S> (&pops)[2], T *(&g)[2], S *&phiu, T *&phig, T *&q, T *&coef,
                  T *&psi_prev, T *&snap, PhiRef<T> &ref, double *&part, double *&part2, Control *&ctl) const
    {
        P = dp_;
        pops[0] = pops_[0];
        pops[1] = pops_[1];
        g[0] = g_[0];
        g[1] = g_[1];
        phiu = phiu_;
        phig = phig_;
        q = q_;
        coef = coef_;
        psi_prev = psi_prev_;
        snap = snap_;
        ref = ref_;
        part = part_;
        part2 = part2_;
        ctl = ctl_;
    }
    int nx() const { return nx_; }
    int ny() const { return ny_; }
    const ehdlb_params &params() const { return P_; }

  private:

    void make_devp()
    {
        const ehdlb_params &p = P_;
        DevP<T> d{};
        d.nx = nx_;
        d.ny = ny_;
        d.nn = nn_;
        d.onsager_form = p.onsager_form;
        d.ion_bc = p.ion_bc;
        d.einstein_D = p.einstein_D;
        d.ion_L_term = p.ion_L_term;
        d.bgk = p.bgk;
        d.freeze_E = p.freeze_E;
        d.side_walls = p.side_walls;
        const double tau_g = 0.5 + 3.0 * p.vartheta;  // Eq. 47
        d.tau_g = (T)tau_g;
        d.s_g = (T)(1.0 / tau_g);
        d.s_free_g = (T)(p.bgk ? 1.0 / tau_g : p.s_free);
        const double src_norm = p.vartheta * (p.psi_src_literal ? 1.0 : 1.5);
        d.src_norm = (T)src_norm;
        d.Kq = (T)p.Kq;
        d.er1 = (T)(p.eps_r - 1.0);
        d.snap_mask = snap_mask_;
        d.src_a = (T)(src_norm * p.Kq / 3.0);
        d.src_b = (T)(src_norm * (p.eps_r - 1.0) / tau_g);
        d.psi_a = (T)p.psi_anode;
        d.psi_c = (T)p.psi_cathode;
        d.G = (T)((p.psi_cathode - p.psi_anode) / ny_);
        d.wG = (T)((p.psi_cathode - p.psi_anode) / ny_ / 6.0);
        d.rho1 = (T)(p.rho_ratio - 1.0);
        d.eta_v = (T)((p.tau_f - 0.5) / 3.0);
        d.eta1 = (T)(p.eta_ratio - 1.0);
        d.beta = (T)(12.0 * p.sigma / p.W);
        d.kappa = (T)(1.5 * p.sigma * p.W);
        d.W = (T)p.W;
        d.tau_h = (T)(0.5 + 3.0 * p.M_phi);
        d.nhat_eps2 = (T)(p.nhat_eps * p.nhat_eps);
        d.s_h = (T)(1.0 / (0.5 + 3.0 * p.M_phi));
        d.sfree_h = (T)(p.bgk ? 1.0 / (0.5 + 3.0 * p.M_phi) : p.s_free);
        d.s_f0 = (T)((p.rho_ratio == 1.0 && p.eta_ratio == 1.0) ? 1.0 / p.tau_f : 0.0);
        const bool uniform_D = !p.einstein_D || p.mu_r == 1.0;
        d.s_p0 = (T)(uniform_D ? 1.0 / (0.5 + 3.0 * (p.einstein_D ? p.D : p.D)) : 0.0);
        d.s_n0 = (T)(uniform_D ? 1.0 / (0.5 + 3.0 * (p.einstein_D ? p.D * p.m : p.D)) : 0.0);
        d.inv_mu_v = (T)(1.0 / p.mu_v);
        d.three_over_tau_g = (T)(3.0 / (0.5 + 3.0 * p.vartheta));
        d.inv_W = (T)(1.0 / p.W);
        d.mu_v = (T)p.mu_v;
        d.mu1 = (T)(p.mu_r - 1.0);
        d.m = (T)p.m;
        d.D = (T)p.D;
        d.k_d = (T)p.k_d;
        d.k_r = (T)p.k_r;
        d.cb = (T)p.onsager_cb;
        d.s_free = (T)p.s_free;
        d.Ex_frozen = (T)p.E_frozen_x;
        d.Ey_frozen = (T)p.E_frozen_y;
        // FP16 storage: power-of-two scales that lift the fields' typical
        // deviations (f ~ 1e-4, h ~ 1e-2, p and n ~ 0.1, phi u ~ 1e-4) to
        // 1..100 and keep deviations down to ~1e-7 above the subnormal range,
        // with room to 16 (f, phi u) or 255 (h, p, n) below the FP16 maximum;
        // the rest concentration is that of the initial state in a uniform
        // field (Eq. 43 with F = 1); g stays in T
        const bool half = !kSame<S, T>;
        const double sf = half ? 4096.0 : 1.0, sh = half ? 256.0 : 1.0, sc = half ? 256.0 : 1.0, sg = 1.0,
                     su = half ? 4096.0 : 1.0;
        d.sc_f = (T)sf; d.isc_f = (T)(1.0 / sf);
        d.sc_h = (T)sh; d.isc_h = (T)(1.0 / sh);
        d.sc_c = (T)sc; d.isc_c = (T)(1.0 / sc);
        d.sc_g = (T)sg; d.isc_g = (T)(1.0 / sg);
        d.sc_u = (T)su; d.isc_u = (T)(1.0 / su);
        double cref = 0.0;
        if (half) cref = p.c_init_scale * ((p.k_r > 0.0 && p.onsager_form != 2) ? std::sqrt(p.k_d / p.k_r) : p.c0);
        d.cref = (T)cref;
        dp_ = d;
    }

    // launch kernel k on the solver's stream (dep: as a programmatic dependent)
    template <typename... P, typename... A>
    void launch_k(void (*k)(P...), dim3 grid, dim3 block, size_t smem, bool dep, A &&...args)
    {
        (void)ehdlb::launch_k(stream_, k, grid, block, smem, dep, std::forward<A>(args)...);
    }

    void launch_prep(int par, int fixedK, int kmin, int kmax, int flips)
    {
        // four nodes per thread (one vector load per plane) when rows split
        // into aligned fours
        const bool v4 = nx_ % 4 == 0;
        const dim3 g = v4 ? dim3((nx_ / 4 + BX - 1) / BX, grid_.y) : grid_;
        const Pops<S> &pp = pops_[par];
        const dim3 b(BX, BY);
        if (qi_ == 9) {
            if (v4) launch_k(k_prep<T, S, 9, 4>, g, b, 0, true, dp_, pp.h, pp.p, pp.n, ref_, phig_, q_, ctl_, fixedK, kmin, kmax, flips);
            else launch_k(k_prep<T, S, 9, 1>, g, b, 0, true, dp_, pp.h, pp.p, pp.n, ref_, phig_, q_, ctl_, fixedK, kmin, kmax, flips);
        } else {
            if (v4) launch_k(k_prep<T, S, 5, 4>, g, b, 0, true, dp_, pp.h, pp.p, pp.n, ref_, phig_, q_, ctl_, fixedK, kmin, kmax, flips);
            else launch_k(k_prep<T, S, 5, 1>, g, b, 0, true, dp_, pp.h, pp.p, pp.n, ref_, phig_, q_, ctl_, fixedK, kmin, kmax, flips);
        }
        ++launches_;
    }

    // Fused sweep kernel: region shapes (width, height, threads per column,
    // blocks per SM the registers are sized for) and the largest number of
    // sweeps one launch fuses.
    // r: rows per thread of the register-blocked kernel (k_sweep_tbr), 0 for
    // the shared-memory one (k_sweep_tb).
    struct TbShape { int rw, rh, by, minb, r; };
    // float: shape 2 is the cluster kernel (k_sweep_cl), 2 x 4 CTAs of 64 x 32;
    // shapes 4 and 5 are register-blocked (by = warps, r = rows per warp),
    // 64 x 32 and 64 x 40
    static constexpr int TB_NSHAPES = sizeof(T) == 4 ? 8 : 1;
    static constexpr int CL_X = 2, CL_Y = 4, CL_BY = 16;
    static constexpr TbShape tb_shape(int i)
    {
        if (sizeof(T) != 4) return TbShape{64, 16, 16, 2, 0};
        switch (i) {
        case 1: return TbShape{64, 32, 8, 4, 0};
        case 3: return TbShape{64, 64, 16, 2, 0};
        case 4: return TbShape{64, 32, 8, 2, 4};
        case 5: return TbShape{64, 40, 8, 2, 5};
        case 6: return TbShape{64, 40, 8, 2, 5};   // shape 5 with the prep pass in its first launch
        case 7: return TbShape{64, 40, 8, 2, 5};   // shape 5 in the walking order (TbrWalkTiles)
        default: return TbShape{64, 32, 16, 3, 0};
        }
    }
    static constexpr int TB_MAX = sizeof(T) == 4 ? 5 : 2;

    static dim3 tb_grid(int nsw, int shape, int nx, int ny)
    {
        if (sizeof(T) == 4 && shape == 2) {
            const int tx = CL_X * 64 - 2 * nsw, ty = CL_Y * 32 - 2 * nsw;
            return dim3(CL_X * ((nx + tx - 1) / tx), CL_Y * ((ny + ty - 1) / ty));
        }
        const TbShape sh = tb_shape(shape);
        const int tx = sh.rw - 2 * (sh.r ? tbr_halo_x(nsw) : nsw), ty = sh.rh - 2 * nsw;
        // register-blocked regions need no halo at the electrode walls (tbr_rows)
        return dim3((nx + tx - 1) / tx, sh.r ? tbr_tile_rows(ny, sh.rh, nsw) : (ny + ty - 1) / ty);
    }

    // The staged step kernel runs for float arithmetic on float or FP16
    // storage; FP64 keeps the cp.async staging.
    static constexpr bool kTmaMain = std::is_same<T, float>::value;

    template <bool SN, bool F, bool R> cudaError_t tma_attr()
    {
        if constexpr (kTmaMain) {
            auto kern = k_main_tma<T, S, SN, F, R>;
            const int smem = (int)(2 * TmaLayout<T, S>::stage);
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            int per = 0;
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, smem);
            if (e == cudaSuccess) tma_per_sm_ = std::max(1, std::min(tma_per_sm_, per));
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_main_tma1<T, S, SN, F, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)TmaLayout<T, S>::stage);
            return e;
        }
        return cudaSuccess;
    }

    // Tensor maps of the staged step kernel; tma_ok_ records whether the
    // lattice can take it (rows of 16-byte multiples, maps encoded).
    void encode_main_maps()
    {
        tma_ok_ = false;
        if constexpr (kTmaMain) {
            if (((size_t)nx_ * sizeof(S)) % 16 != 0 || qi_ != 5) return;
            bool ok = true;
            for (int b = 0; b < 2; ++b) {
                MainMaps &m = maps_[b];
                ok = ok && encode_tiles<S>(&m.pops, pops_[b].f, nx_, ny_, 27, nn_, 64, 4);
                ok = ok && encode_tiles<S>(&m.phiu, phiu_, nx_, ny_, 2, nn_, 64, 4);
                ok = ok && encode_tiles<T>(&m.g[0], g_[0], nx_, ny_, 4, nn_, 64, 4);
                ok = ok && encode_tiles<T>(&m.g[1], g_[1], nx_, ny_, 4, nn_, 64, 4);
                ok = ok && encode_tiles<T>(&m.mur, ref_.mur, nx_, ny_, 1, nn_, 64, 4);
                ok = ok && encode_tiles<T>(&m.gxr, ref_.gxr, nx_, ny_, 1, nn_, 64, 4);
                ok = ok && encode_tiles<T>(&m.gyr, ref_.gyr, nx_, ny_, 1, nn_, 64, 4);
                ok = ok && encode_tiles<T>(&m.psi, psi_prev_, nx_, ny_, 1, nn_, 64, 4);
                ok = ok && encode_tiles<T>(&m.dphi, ref_.dphig, nx_, ny_ + 2, 1, nn_, TMA_HW, TMA_HH);
                ok = ok && encode_tiles<T>(&m.phir, ref_.phir, nx_, ny_ + 2, 1, nn_, TMA_HW, TMA_HH);
            }
            tma_ok_ = ok;
        }
    }

    template <bool SN, bool F, bool R> cudaError_t main_attr()
    {
        cudaError_t e = cudaSuccess;
        for (cudaError_t x :
             {cudaFuncSetAttribute(k_main<T, S, SN, F, R, true, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)main_smem_bytes<T, S, 5>()),
              cudaFuncSetAttribute(k_main<T, S, SN, F, R, false, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)main_smem_bytes<T, S, 5>()),
              cudaFuncSetAttribute(k_main<T, S, SN, F, R, true, 9>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)main_smem_bytes<T, S, 9>()),
              cudaFuncSetAttribute(k_main<T, S, SN, F, R, false, 9>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)main_smem_bytes<T, S, 9>())})
            if (x != cudaSuccess) e = x;
        return e;
    }

    template <int NSW, int SH, bool FIRST, bool RESID> cudaError_t tb_attr2()
    {
        constexpr TbShape sh = tb_shape(SH);
        return cudaFuncSetAttribute(k_sweep_tb<T, T, NSW, sh.rw, sh.rh, sh.by, sh.minb, FIRST, RESID>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)tb_smem_bytes<T, sh.rw, sh.rh>(FIRST));
    }

    template <int NSW, int SH> cudaError_t tb_attr1()
    {
        cudaError_t e = tb_attr2<NSW, SH, false, false>();
        if (e == cudaSuccess) e = tb_attr2<NSW, SH, false, true>();
        if (e == cudaSuccess) e = tb_attr2<NSW, SH, true, false>();
        if (e == cudaSuccess) e = tb_attr2<NSW, SH, true, true>();
        return e;
    }

    template <int NSW, bool FIRST, bool RESID> cudaError_t cl_attr2()
    {
        return cudaFuncSetAttribute(k_sweep_cl<T, NSW, CL_X, CL_Y, CL_BY, FIRST, RESID>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tb_cl_smem_bytes<T>());
    }

    template <int NSW> cudaError_t tb_attr()
    {
        cudaError_t e = tb_attr1<NSW, 0>();
        if constexpr (TB_NSHAPES > 1) {
            if (e == cudaSuccess) e = tb_attr1<NSW, 1>();
            if (e == cudaSuccess) e = tb_attr1<NSW, 3>();
            if (e == cudaSuccess) e = tbr_attr1<NSW, 4>();
            if (e == cudaSuccess) e = tbr_attr1<NSW, 5>();
            if (e == cudaSuccess) e = tbw_attr2<NSW, false, false>();
            if (e == cudaSuccess) e = tbw_attr2<NSW, false, true>();
            if (e == cudaSuccess) e = tbw_attr2<NSW, true, false>();
            if (e == cudaSuccess) e = tbw_attr2<NSW, true, true>();
            if (e == cudaSuccess) e = tbr_fp_attr<NSW, false>();
            if (e == cudaSuccess) e = tbr_fp_attr<NSW, true>();
            if (e == cudaSuccess) e = cl_attr2<NSW, false, false>();
            if (e == cudaSuccess) e = cl_attr2<NSW, false, true>();
            if (e == cudaSuccess) e = cl_attr2<NSW, true, false>();
            if (e == cudaSuccess) e = cl_attr2<NSW, true, true>();
        }
        return e;
    }

    template <int NSW, bool FIRST, bool RESID> void cl_launch2()
    {
        const dim3 g = tb_grid(NSW, 2, nx_, ny_);
        k_sweep_cl<T, NSW, CL_X, CL_Y, CL_BY, FIRST, RESID>
            <<<g, dim3(32, CL_BY), tb_cl_smem_bytes<T>(), stream_>>>(dp_, g_[0], g_[1], phig_, q_, coef_, part2_,
                                                                     ctl_, tb_m_);
    }

    template <int NSW, int SH, bool FIRST, bool RESID> void tb_launch2()
    {
        constexpr TbShape sh = tb_shape(SH);
        constexpr int TXo = sh.rw - 2 * NSW, TYo = sh.rh - 2 * NSW;
        const dim3 g((nx_ + TXo - 1) / TXo, (ny_ + TYo - 1) / TYo);
        k_sweep_tb<T, T, NSW, sh.rw, sh.rh, sh.by, sh.minb, FIRST, RESID>
            <<<g, dim3(32, sh.by), tb_smem_bytes<T, sh.rw, sh.rh>(FIRST), stream_>>>(
                dp_, g_[0], g_[1], phig_, q_, coef_, part2_, ctl_, tb_m_);
    }

    template <int NSW, int SH, bool FIRST, bool RESID> cudaError_t tbr_attr2()
    {
        constexpr TbShape sh = tb_shape(SH);
        const size_t smem = tbr_smem_bytes<T, sh.r, sh.by>(FIRST);
        auto kern = k_sweep_tbr<T, NSW, sh.r, sh.by, sh.minb, FIRST, RESID>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 32 * sh.by, smem);
        // persistent grid: the fewest resident blocks per SM of any variant
        if (e == cudaSuccess) tbr_per_sm_[SH - 4] = std::max(1, std::min(tbr_per_sm_[SH - 4], per));
        return e;
    }

    // the first launch with the prep pass fused (shape 6, float storage)
    template <int NSW, bool RESID> cudaError_t tbr_fp_attr()
    {
        if constexpr (kSame<S, T>) {
            constexpr TbShape sh = tb_shape(6);
            const size_t smem = tbr_smem_bytes<T, sh.r, sh.by>(true);
            auto kern = k_sweep_tbr_fp<T, NSW, sh.r, sh.by, sh.minb, RESID>;
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            int per = 0;
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 32 * sh.by, smem);
            if (e == cudaSuccess) tbr_per_sm_[1] = std::max(1, std::min(tbr_per_sm_[1], per));
            return e;
        }
        return cudaSuccess;
    }

    // the walking order (shape 7)
    template <int NSW, bool FIRST, bool RESID> cudaError_t tbw_attr2()
    {
        if constexpr (TB_NSHAPES > 7) {
            constexpr TbShape sh = tb_shape(7);
            const size_t smem = tbr_smem_bytes<T, sh.r, sh.by>(FIRST);
            auto kern = k_sweep_tbw<T, NSW, sh.r, sh.by, sh.minb, FIRST, RESID>;
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            int per = 0;
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 32 * sh.by, smem);
            if (e == cudaSuccess) tbr_per_sm_[1] = std::max(1, std::min(tbr_per_sm_[1], per));
            return e;
        }
        return cudaSuccess;
    }

    // blocks of a walking launch of nsw sweeps: the resident blocks, at most
    // the tiles of shape 5 (whose partial slots are allocated)
    int tbw_blocks(int nsw) const
    {
        const dim3 g = tb_grid(nsw, 5, nx_, ny_);
        return std::max(1, std::min((int)(g.x * g.y), tbr_per_sm_[1] * sms_));
    }

    template <int NSW, bool FIRST, bool RESID> void tbw_launch2()
    {
        if constexpr (TB_NSHAPES > 7) {
            constexpr TbShape sh = tb_shape(7);
            const int tx = 64 - 2 * tbr_halo_x(NSW);
            k_sweep_tbw<T, NSW, sh.r, sh.by, sh.minb, FIRST, RESID>
                <<<tbw_blocks(NSW), dim3(32, sh.by), tbr_smem_bytes<T, sh.r, sh.by>(FIRST), stream_>>>(
                    dp_, g_[0], g_[1], phig_, q_, coef_, part2_, ctl_, tb_m_, (nx_ + tx - 1) / tx);
        }
    }

    // prep fused into the first sweep launch of a fixed-count step
    bool fprep() const
    {
        return kSame<S, T> && sizeof(T) == 4 && tb_shape_ == 6 && qi_ == 5 && !P_.side_walls;
    }

    template <int NSW, bool RESID> void tbr_fp_launch(int fixedK, int flips)
    {
        if constexpr (kSame<S, T> && TB_NSHAPES > 6) {
            constexpr TbShape sh = tb_shape(6);
            const dim3 g = tb_grid(NSW, 6, nx_, ny_);
            const int ntiles = (int)(g.x * g.y);
            const int grid = std::min(ntiles, tbr_per_sm_[1] * sms_);
            const Pops<S> &pp = pops_[tpar_];
            launch_k(k_sweep_tbr_fp<T, NSW, sh.r, sh.by, sh.minb, RESID>, dim3(grid), dim3(32, sh.by),
                     tbr_smem_bytes<T, sh.r, sh.by>(true), true, dp_, g_[0], g_[1], pp.h, pp.p, pp.n, ref_.phir,
                     ref_.dphig, coef_, part2_, ctl_, (int)g.x, ntiles, fixedK, flips);
        }
    }

    template <int NSW, int SH> cudaError_t tbr_attr1()
    {
        cudaError_t e = tbr_attr2<NSW, SH, false, false>();
        if (e == cudaSuccess) e = tbr_attr2<NSW, SH, false, true>();
        if (e == cudaSuccess) e = tbr_attr2<NSW, SH, true, false>();
        if (e == cudaSuccess) e = tbr_attr2<NSW, SH, true, true>();
        return e;
    }

    template <int NSW, int SH, bool FIRST, bool RESID> void tbr_launch2()
    {
        constexpr TbShape sh = tb_shape(SH);
        const dim3 g = tb_grid(NSW, SH, nx_, ny_);
        const int ntiles = (int)(g.x * g.y);
        const int grid = std::min(ntiles, tbr_per_sm_[SH - 4] * sms_);
        launch_k(k_sweep_tbr<T, NSW, sh.r, sh.by, sh.minb, FIRST, RESID>, dim3(grid), dim3(32, sh.by),
                 tbr_smem_bytes<T, sh.r, sh.by>(FIRST), true, dp_, g_[0], g_[1], phig_, q_, coef_, part2_, ctl_,
                 tb_m_, (int)g.x, ntiles);
    }

    template <int NSW, int SH> void tbr_launch1(bool first, bool resid)
    {
        if (first) {
            if (resid) tbr_launch2<NSW, SH, true, true>();
            else tbr_launch2<NSW, SH, true, false>();
        } else {
            if (resid) tbr_launch2<NSW, SH, false, true>();
            else tbr_launch2<NSW, SH, false, false>();
        }
    }

    template <int NSW, int SH> void tb_launch1(bool first, bool resid)
    {
        if (first) {
            if (resid) tb_launch2<NSW, SH, true, true>();
            else tb_launch2<NSW, SH, true, false>();
        } else {
            if (resid) tb_launch2<NSW, SH, false, true>();
            else tb_launch2<NSW, SH, false, false>();
        }
    }

    template <int NSW> void tb_launch(int m, bool resid)
    {
        tb_m_ = m;
        const bool first = m == 0;
        if constexpr (TB_NSHAPES > 1) {
            if (tb_shape_ == 2) {
                if (first) {
                    if (resid) cl_launch2<NSW, true, true>();
                    else cl_launch2<NSW, true, false>();
                } else {
                    if (resid) cl_launch2<NSW, false, true>();
                    else cl_launch2<NSW, false, false>();
                }
            } else if (tb_shape_ == 1) {
                tb_launch1<NSW, 1>(first, resid);
            } else if (tb_shape_ == 3) {
                tb_launch1<NSW, 3>(first, resid);
            } else if (tb_shape_ == 4) {
                tbr_launch1<NSW, 4>(first, resid);
            } else if (tb_shape_ == 7) {
                if (first) {
                    if (resid) tbw_launch2<NSW, true, true>();
                    else tbw_launch2<NSW, true, false>();
                } else {
                    if (resid) tbw_launch2<NSW, false, true>();
                    else tbw_launch2<NSW, false, false>();
                }
            } else if (tb_shape_ == 5 || tb_shape_ == 6) {
                if (first && fprep()) {
                    if (resid) tbr_fp_launch<NSW, true>(fp_fixedK_, fp_flips_);
                    else tbr_fp_launch<NSW, false>(fp_fixedK_, fp_flips_);
                } else {
                    tbr_launch1<NSW, 5>(first, resid);
                }

            } else {
                tb_launch1<NSW, 0>(first, resid);
            }
        } else {
            tb_launch1<NSW, 0>(first, resid);
        }
        ++launches_;
        ++sweep_launches_;
    }

    void launch_sweep_tb(int nsw, int m, bool resid)
    {
        switch (nsw) {
        case 1: tb_launch<1>(m, resid); break;
        case 2: tb_launch<2>(m, resid); break;
        case 3: if constexpr (TB_MAX >= 3) tb_launch<3>(m, resid); break;
        case 4: if constexpr (TB_MAX >= 4) tb_launch<4>(m, resid); break;
        default: if constexpr (TB_MAX >= 5) tb_launch<5>(m, resid); break;
        }
    }

    int tb_chunk() const { return tb_chunk_ > 0 ? std::min(tb_chunk_, TB_MAX) : 0; }

    void launch_sweep(int j, bool write_psi, bool resid, bool ctrl)
    {
        const dim3 b(BX, BY);
#define EHDLB_SWEEP(W, R, C)                                                                            \
    k_sweep<T, T, W, R, C><<<grid_, b, 0, stream_>>>(dp_, g_[0], g_[1], phig_, q_, psi_prev_, part_, ctl_, j)
        if (ctrl) {
            if (resid) EHDLB_SWEEP(true, true, true);
            else EHDLB_SWEEP(true, false, true);
        } else {
            if (write_psi) EHDLB_SWEEP(true, false, false);
            else EHDLB_SWEEP(false, false, false);
        }
#undef EHDLB_SWEEP
        ++launches_;
        ++sweep_launches_;
    }

    // Kernel sequence of one time step; s is the step index within the call,
    // last marks the final step (snapshot, sums and residual reported).
    void enqueue_step(int s, bool last)
    {
        const int par = tpar_;
        const bool frozen = P_.freeze_E != 0;
        int fixedK = -1, kmin = P_.sweeps_min, kmax = P_.sweeps_max;
        if (frozen) fixedK = 0;
        else if (t_ < (long long)sched_.size()) fixedK = sched_[(size_t)t_];
        else if (P_.sweeps_min == P_.sweeps_max) fixedK = P_.sweeps_max;
        const bool converge = fixedK < 0;
        if (!converge) kmin = kmax = fixedK;
        const int chunk = tb_chunk();
        // the fused sweep kernels implement the periodic x of the benchmark
        // cases; with side walls every sweep is its own launch
        const bool fused = !converge && fixedK > 0 && chunk > 0 && !P_.side_walls;
        const int nk = fused ? (fixedK + chunk - 1) / chunk : (converge ? 0 : fixedK);
        const bool tev = timing_ > 0 && s % timing_ == 0;   // this step's kernel classes are timed
        if (tev) cudaEventRecord(events_[4 * s], stream_);
        const bool fp = fused && fprep();
        if (fp) {
            fp_fixedK_ = fixedK;   // the first sweep launch does the prep pass
            fp_flips_ = nk;
        } else {
            launch_prep(par, fixedK, kmin, kmax, nk);
        }
        if (tev) cudaEventRecord(events_[4 * s + 1], stream_);
        if (fused) {
            for (int m = 0, done = 0; m < nk; ++m) {
                const int nsw = std::min(chunk, fixedK - done);
                launch_sweep_tb(nsw, m, last && m == nk - 1);
                done += nsw;
            }
        } else if (!converge) {
            for (int j = 1; j <= fixedK; ++j) launch_sweep(j, last && j == fixedK, false, false);
        } else {
            for (int j = 1; j <= kmax; ++j) {
                launch_sweep(j, true, j >= 2, true);
                k_sweep_decide<<<1, 256, 0, stream_>>>(part_, nb_, ctl_, j);
                ++launches_;
            }
        }
        if (tev) cudaEventRecord(events_[4 * s + 2], stream_);
        const bool main_resid = !frozen && !fused && kmax >= 1 && (converge || last);
        const int resid_mode = main_resid ? 1 : ((fused && last) ? 2 : 0);
        const dim3 b(BX, BY);
        int *unstable = &ctl_->unstable;
#define EHDLB_MAIN1(SN, F, R, V, Q)                                                                      \
    k_main<T, S, SN, F, R, V, Q><<<grid_, b, main_smem_bytes<T, S, Q>(), stream_>>>(                       \
        dp_, pops_[par], pops_[par ^ 1], g_[0], g_[1], ctl_, ref_, phiu_, psi_prev_, snap_, part_, unstable)
#define EHDLB_MAIN(SN, F, R)                                                                             \
    do {                                                                                                 \
        const bool v_ = vec_ok_ && vec_;                                                                 \
        if (qi_ == 9) {                                                                                  \
            if (v_) EHDLB_MAIN1(SN, F, R, true, 9);                                                      \
            else EHDLB_MAIN1(SN, F, R, false, 9);                                                        \
        } else {                                                                                         \
            if (v_) EHDLB_MAIN1(SN, F, R, true, 5);                                                      \
            else EHDLB_MAIN1(SN, F, R, false, 5);                                                        \
        }                                                                                                \
    } while (0)
        const bool staged = kTmaMain && tma_ && tma_ok_ && qi_ == 5 && !P_.side_walls;
#define EHDLB_MAIN_TMA(SN, F, R)                                                                         \
    do {                                                                                                 \
        if constexpr (kTmaMain) {                                                                        \
            const int ntiles = (int)(grid_.x * grid_.y);                                                 \
            if (tma_persist_)                                                                            \
                k_main_tma<T, S, SN, F, R><<<std::min(ntiles, tma_per_sm_ * sms_), b,                    \
                                             2 * TmaLayout<T, S>::stage, stream_>>>(                     \
                    dp_, maps_[par], pops_[par], pops_[par ^ 1], g_[0], g_[1], ctl_, ref_, phiu_, psi_prev_, \
                    snap_, part_, unstable, &ctl_->fault, (int)grid_.x, ntiles);                         \
            else                                                                                         \
                launch_k(k_main_tma1<T, S, SN, F, R>, grid_, b, TmaLayout<T, S>::stage, true, dp_, maps_[par], \
                         pops_[par], pops_[par ^ 1], g_[0], g_[1], ctl_, ref_, phiu_, psi_prev_, snap_, part_,   \
                         unstable, &ctl_->fault);                                                        \
        }                                                                                                \
    } while (0)
        if (staged) {
            if (last) {
                if (frozen) EHDLB_MAIN_TMA(true, true, false);
                else if (main_resid) EHDLB_MAIN_TMA(true, false, true);
                else EHDLB_MAIN_TMA(true, false, false);
            } else {
                if (frozen) EHDLB_MAIN_TMA(false, true, false);
                else if (main_resid) EHDLB_MAIN_TMA(false, false, true);
                else EHDLB_MAIN_TMA(false, false, false);
            }
        } else if (last) {
            if (frozen) EHDLB_MAIN(true, true, false);
            else if (main_resid) EHDLB_MAIN(true, false, true);
            else EHDLB_MAIN(true, false, false);
        } else {
            if (frozen) EHDLB_MAIN(false, true, false);
            else if (main_resid) EHDLB_MAIN(false, false, true);
            else EHDLB_MAIN(false, false, false);
        }
#undef EHDLB_MAIN_TMA
#undef EHDLB_MAIN
#undef EHDLB_MAIN1
        long long nb2 = 0;
        if (resid_mode == 2) {
            const int nsw = std::min(chunk, fixedK - (nk - 1) * chunk);
            const dim3 g = tb_grid(nsw, tb_shape_, nx_, ny_);
            nb2 = tb_shape_ == 7 ? tbw_blocks(nsw) : (long long)g.x * g.y;
        }
        // sums of the block partials in two stages (PSUM blocks, then one)
        const double *p4 = part_, *p2 = part2_;
        long long n4 = nb_, n2 = nb2;
        if ((resid_mode == 1 || last) && nb_ > PSUM) {
            launch_k(k_partials<4>, dim3(PSUM), dim3(256), 0, true, part_, nb_, red_);
            p4 = red_;
            n4 = PSUM;
            ++launches_;
        }
        if (resid_mode == 2 && nb2 > PSUM) {
            launch_k(k_partials<2>, dim3(PSUM), dim3(256), 0, true, part2_, nb2, red_ + 4 * PSUM);
            p2 = red_ + 4 * PSUM;
            n2 = PSUM;
            ++launches_;
        }
        launch_k(k_step_end, dim3(1), dim3(256), 0, true, p4, n4, p2, n2, ctl_, counts_, resid_mode, last ? 1 : 0);
        launches_ += 2;
        if (tev) cudaEventRecord(events_[4 * s + 3], stream_);
        tpar_ ^= 1;
        ++t_;
    }

        int transfer_state(double *dst, const double *src, std::string &err)
    {
        EHDLB_CK(cudaMemcpyAsync(&ctl_h_, ctl_, sizeof(Control), cudaMemcpyDeviceToHost, stream_));
        EHDLB_CK(cudaStreamSynchronize(stream_));
        const int cur = ctl_h_.cur0;
        // rows of the state per chunk through the solver's staging buffer
        // (nn doubles); the chunks follow one another on the stream, which
        // is synchronised once at the end
        const size_t per_row = (size_t)state_per_node() * nx_;
        const int rows = (int)std::min<size_t>((size_t)ny_, ((size_t)nn_) / per_row);
        double *stage = stage_;
        int status = EHDLB_OK;
        if (rows < 1) {   // a row of the state exceeds the staging buffer (nn < per_row)
            EHDLB_CK(cudaMalloc((void **)&stage, sizeof(double) * per_row));
        }
        const int crows = std::max(1, rows);
        for (int y0 = 0; y0 < ny_ && status == EHDLB_OK; y0 += crows) {
            const int r = std::min(crows, ny_ - y0);
            const long long cnt = (long long)r * nx_;
            const unsigned nblk = (unsigned)((cnt + 255) / 256);
            cudaError_t e = cudaSuccess;
            if (dst) {
                if (qi_ == 9)
                    k_pack_state<T, S, 9><<<nblk, 256, 0, stream_>>>(dp_, pops_[ctl_h_.tpar & 1], g_[cur], phiu_,
                                                                     ref_.phir, stage, y0, r);
                else
                    k_pack_state<T, S, 5><<<nblk, 256, 0, stream_>>>(dp_, pops_[ctl_h_.tpar & 1], g_[cur], phiu_,
                                                                     ref_.phir, stage, y0, r);
                e = cudaGetLastError();
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(dst + per_row * y0, stage, sizeof(double) * per_row * r,
                                        cudaMemcpyDeviceToHost, stream_);
            } else {
                e = cudaMemcpyAsync(stage, src + per_row * y0, sizeof(double) * per_row * r,
                                    cudaMemcpyHostToDevice, stream_);
                if (e == cudaSuccess)
                {
                    if (qi_ == 9)
                        k_unpack_state<T, S, 9><<<nblk, 256, 0, stream_>>>(dp_, pops_[ctl_h_.tpar & 1], g_[cur],
                                                                           phiu_, ref_.phir, stage, y0, r);
                    else
                        k_unpack_state<T, S, 5><<<nblk, 256, 0, stream_>>>(dp_, pops_[ctl_h_.tpar & 1], g_[cur],
                                                                           phiu_, ref_.phir, stage, y0, r);
                }
                if (e == cudaSuccess) e = cudaGetLastError();
            }
            if (e != cudaSuccess) {
                err = std::string("state transfer: ") + cudaGetErrorString(e);
                status = EHDLB_ECUDA;
            }
        }
        const cudaError_t e = cudaStreamSynchronize(stream_);
        if (e != cudaSuccess && status == EHDLB_OK) {
            err = std::string("state transfer: ") + cudaGetErrorString(e);
            status = EHDLB_ECUDA;
        }
        if (stage != stage_) cudaFree(stage);
        return status;
    }

    int nx_, ny_;
    long long nn_;
    cudaStream_t stream_;
    DevArena *arena_ = nullptr;
    bool own_stream_ = false;
    dim3 grid_;
    long long nb_ = 0;
    Pops<S> pops_[2]{};
    T *g_[2]{};
    S *phiu_ = nullptr;
    bool vec_ok_ = false;                     // 16-byte staging possible
    bool vec_ = true;                         // and chosen (tuning)
    bool tma_ = true;                         // staged step kernel chosen (tuning main_staging 2, 3; default 2)
    bool tma_persist_ = false;                // its persistent two-stage form (main_staging 3)
    bool stall_ = false;                      // test hook armed for the next step call
    int fp_fixedK_ = 0, fp_flips_ = 0;        // the step the fused prep pass opens
    bool tma_ok_ = false;                     // and possible for this lattice
    int tma_per_sm_ = 1 << 20;                // resident blocks per SM of the staged step kernel
    MainMaps maps_[2]{};                      // its tensor maps, by the time level of the source
    T *phig_ = nullptr, *q_ = nullptr, *psi_prev_ = nullptr, *snap_ = nullptr;
    PhiRef<T> ref_{};
    double *part_ = nullptr, *part2_ = nullptr, *stage_ = nullptr;
    int tb_chunk_ = sizeof(T) == 4 ? 5 : 2;  // sweeps fused per launch (0: one per launch)
    int tb_shape_ = sizeof(T) == 4 ? 5 : 0;   // region shape of the fused sweep kernel
    int tbr_per_sm_[2] = {1 << 20, 1 << 20};  // resident blocks per SM of the register-blocked shapes
    unsigned snap_mask_ = (1u << EHDLB_NFIELDS) - 1;   // fields the reporting step captures
    unsigned snap_valid_ = (1u << EHDLB_NFIELDS) - 1;  // fields the snapshot holds now
    bool deform_each_ = false;                        // every step call also computes D
    int sms_ = 1;                             // SMs of the device
    int tb_m_ = 0;                            // launch index within the step
    int qi_ = 0;                              // ion populations per species (5 or 9) of pops_
    static constexpr int PSUM = 64;           // blocks of the first stage of the partial sums
    double *red_ = nullptr;                   // their results: 4 PSUM, then 2 PSUM doubles, then the
                                              // slice sums of the deformation factor
    T *coef_ = nullptr;                       // source coefficients A, Bx, By of the step
    Control *ctl_ = nullptr;
    struct HostMirror {
        Control c;
        double D;
    } *pin_ = nullptr;
    Control ctl_h_{};
    int *counts_ = nullptr;
    int counts_cap_ = 0;
    std::vector<void *> allocs_;
    std::vector<cudaEvent_t> events_;
    std::vector<int> sched_;
    ehdlb_params P_{};
    DevP<T> dp_{};
    int tpar_ = 0;
    long long t_ = 0;
    int init_sweeps_ = 0;
    int timing_ = 0;   // record the kernel classes of every timing_-th step (0: none)
    long long launches_ = 0;
    long long sweep_launches_ = 0;
};

}  // namespace ehdlb
