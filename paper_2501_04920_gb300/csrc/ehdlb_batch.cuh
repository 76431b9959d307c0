// ehdlb_batch.cuh -- many lattices (cases) stepped together by persistent
// kernels over one work-list of tiles.
//
// Each case is a Solver whose buffers come from one device arena (first fit,
// 256-byte blocks); a case is admitted only if its footprint fits in what the
// arena has left.  A batch step runs the kernel sequence of one time step of
// every case with one launch per kernel kind: the persistent kernels take
// work items (case, block column, block row, partials slot) from device
// arrays, copy the case's descriptor (constants and buffer pointers) to
// shared memory and run the same per-block bodies as the single-lattice
// kernels, so a case steps bit for bit as it does alone.  The time parity of
// each case's f, h, p, n buffers lives in its control block and the
// work-lists in device memory; the steps of a call but the last replay one
// captured CUDA graph of a batch step, captured again after the set of cases
// changes.  All cases of a batch take the same fixed number of potential
// sweeps per step.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "ehdlb_solver.cuh"

namespace ehdlb {

// ---- device arena -------------------------------------------------------------------

class Arena : public DevArena {
  public:
    ~Arena() override
    {
        if (base_) cudaFree(base_);
    }
    cudaError_t init(size_t bytes)
    {
        bytes = (bytes + 255) / 256 * 256;
        cudaError_t e = cudaMalloc(&base_, bytes);
        if (e != cudaSuccess) {
            base_ = nullptr;
            return e;
        }
        cap_ = bytes;
        free_[0] = bytes;
        return cudaSuccess;
    }
    cudaError_t alloc(void **p, size_t bytes) override
    {
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > bytes) free_[off + bytes] = len - bytes;
            used_[off] = bytes;
            in_use_ += bytes;
            *p = static_cast<char *>(base_) + off;
            return cudaSuccess;
        }
        return cudaErrorMemoryAllocation;
    }
    void release(void *p) override
    {
        const size_t off = (size_t)(static_cast<char *>(p) - static_cast<char *>(base_));
        auto u = used_.find(off);
        if (u == used_.end()) return;
        size_t start = off, len = u->second;
        in_use_ -= len;
        used_.erase(u);
        auto nx = free_.lower_bound(start);
        if (nx != free_.end() && nx->first == start + len) {   // merge with the next block
            len += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {                               // and the previous one
            auto pv = std::prev(nx);
            if (pv->first + pv->second == start) {
                start = pv->first;
                len += pv->second;
                free_.erase(pv);
            }
        }
        free_[start] = len;
    }
    size_t capacity() const { return cap_; }
    size_t in_use() const { return in_use_; }
    size_t largest_free() const
    {
        size_t m = 0;
        for (auto &f : free_) m = std::max(m, f.second);
        return m;
    }

  private:
    void *base_ = nullptr;
    size_t cap_ = 0, in_use_ = 0;
    std::map<size_t, size_t> free_, used_;   // offset -> length
};

// ---- case descriptors and work items --------------------------------------------------

template <typename T, typename S> struct CaseDev {
    DevP<T> P;
    Pops<S> pops[2];
    T *g[2];
    S *phiu;
    T *phig, *q, *coef, *psi_prev, *snap;
    PhiRef<T> ref;
    double *part, *part2;
    Control *ctl;
    long long nb_main;       // partial slots of the step kernel
    long long nb_tb;         // partial slots of the last sweep launch
    int gxm, gym;            // grid of 64 x 4 blocks of the step kernel
    int pad_[2];
};

// Block rows of the step and prep kernels one work item covers (one
// descriptor load per item).
constexpr int KB_ROWS = 4;

// x: case index, y, z: block column and row in the case's grid, w: partials
// slot (step and prep kernels: z is the first of KB_ROWS block rows and the
// slot follows from the row)
using WorkItem = int4;

// Copy the descriptor of case c to shared memory (all threads; no barrier).
template <typename T, typename S>
__device__ __forceinline__ void load_case(CaseDev<T, S> &dst, const CaseDev<T, S> *__restrict__ cases, int c)
{
    static_assert(sizeof(CaseDev<T, S>) % 4 == 0, "descriptor size");
    const unsigned *src = reinterpret_cast<const unsigned *>(cases + c);
    unsigned *d = reinterpret_cast<unsigned *>(&dst);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x, nt = blockDim.x * blockDim.y;
    for (int i = tid; i < (int)(sizeof(CaseDev<T, S>) / 4); i += nt) d[i] = src[i];
}

// ---- kernels of a batch step -----------------------------------------------------------------

// O1-O3 of every case, one 64 x 4 tile per block: block (i, r) takes block
// row z + r of work item i (grid: items x KB_ROWS; blockDim (64, 4)).
template <typename T, typename S>
__global__ void __launch_bounds__(256) kb_prep(const CaseDev<T, S> *__restrict__ cases,
                                               const WorkItem *__restrict__ items, const int *__restrict__ nitems,
                                               int fixedK, int flips)
{
    griddep_begin();
    __shared__ CaseDev<T, S> C;
    if ((int)blockIdx.x >= *nitems) return;
    const WorkItem w = items[blockIdx.x];
    load_case(C, cases, w.x);
    __syncthreads();
    const int by = w.z + (int)blockIdx.y;
    if (by >= min(w.z + KB_ROWS, C.gym)) return;
    const Pops<S> &cur = C.pops[C.ctl->tpar & 1];
    prep_body<T, S>(C.P, cur.h, cur.p, cur.n, C.ref, C.phig, C.q, C.ctl, fixedK, fixedK, fixedK, flips, w.y, by);
}

// Sweep launch m of every case (NSW sweeps fused).  blockDim (32, BY).
template <typename T, typename S, int NSW, int BY, int MINB, bool FIRST>
__global__ void __launch_bounds__(32 * BY, MINB) kb_sweep(const CaseDev<T, S> *__restrict__ cases,
                                                           const WorkItem *__restrict__ items,
                                                           const int *__restrict__ nitems, int m)
{
    griddep_begin();
    __shared__ CaseDev<T, S> C;
    const int n = *nitems;
    for (int it = blockIdx.x; it < n; it += gridDim.x) {
        const WorkItem w = items[it];
        load_case(C, cases, w.x);
        __syncthreads();
        tb_body<T, T, NSW, 64, 32, BY, FIRST, false>(C.P, C.g[0], C.g[1], C.phig, C.q, C.coef, C.part2, C.ctl, m,
                                                     w.y, w.z, w.w);
        __syncthreads();
    }
}

// The tiles of a batch's register-blocked sweep launch m: item (case, tile
// column, tile row, index) of the case's grid of tiles.
template <typename T, typename S> struct TbrBatchTiles {
    const CaseDev<T, S> *cases;
    const WorkItem *items;
    int n, m;
    __device__ int count() const { return n; }
    __device__ TbrTile<T> tile(int i, int TX, int TY, int H) const
    {
        const WorkItem w = items[i];
        const CaseDev<T, S> &C = cases[w.x];
        const int par = (C.ctl->cur0 + m) & 1;
        TbrTile<T> t{&C.P, C.g[par], C.g[par ^ 1], C.phig, C.q, C.coef, C.part2, w.w, w.y * TX, w.z * TY};
        t.ry0 = t.y0 - H;   // regions with a halo on both sides
        t.oy1 = min(t.y0 + TY, C.P.ny);
        return t;
    }
};

// Sweep launch m of every case, register-blocked (k_sweep_tbr's tiles of
// 64 x 8R).  blockDim (32, 8), dynamic shared memory tbr_smem_bytes<T, R, 8>(FIRST).
template <typename T, typename S, int NSW, int R, bool FIRST>
__global__ void __launch_bounds__(256, 2) kb_sweep_r(const CaseDev<T, S> *__restrict__ cases,
                                                     const WorkItem *__restrict__ items,
                                                     const int *__restrict__ nitems, int m)
{
    griddep_begin();
    TbrBatchTiles<T, S> J{cases, items, *nitems, m};
    tbr_run<T, NSW, R, 8, FIRST, false>(J);
}

// O5-O11 of every case, one 64 x 4 tile per block: block (i, r) takes block
// row z + r of work item i (grid: items x KB_ROWS; blockDim (64, 4), dynamic
// shared memory main_smem_bytes<T, S>()), so that many blocks per SM hide the
// latency of each one's staged copies (a persistent loop over the items
// moved the same bytes at 0.61 of the copy bandwidth).
template <typename T, typename S, bool SNAP>
__global__ void __launch_bounds__(256, MAIN_MINB<T>) kb_main(const CaseDev<T, S> *__restrict__ cases,
                                                   const WorkItem *__restrict__ items, const int *__restrict__ nitems)
{
    griddep_begin();
    __shared__ CaseDev<T, S> C;
    if ((int)blockIdx.x >= *nitems) return;
    const WorkItem w = items[blockIdx.x];
    load_case(C, cases, w.x);
    __syncthreads();
    const int by = w.z + (int)blockIdx.y;
    if (by >= min(w.z + KB_ROWS, C.gym)) return;
    const int par = C.ctl->tpar & 1;
    main_body<T, S, SNAP, false, false, true>(C.P, C.pops[par], C.pops[par ^ 1], C.g[0], C.g[1], C.ctl, C.ref,
                                              C.phiu, C.psi_prev, C.snap, C.part, &C.ctl->unstable, w.y, by,
                                              (long long)by * C.gxm + w.y);
}

// The same with the tile staged by the tensor memory accelerator through the
// case's tensor maps (maps[2 c + parity], in device memory; every case's
// rows a multiple of 16 bytes): one thread issues the nine loads of the
// single-lattice staged kernel behind one mbarrier and the block waits for
// them (bounded: a late copy sets the case's Control::fault and the block
// returns).  Dynamic shared memory TmaLayout<T, S>::stage.
template <typename T, typename S, bool SNAP>
__global__ void __launch_bounds__(256, MAIN_MINB<T>) kb_main_tma(const CaseDev<T, S> *__restrict__ cases,
                                                      const MainMaps *__restrict__ maps,
                                                      const WorkItem *__restrict__ items,
                                                      const int *__restrict__ nitems)
{
    griddep_begin();
    using L = TmaLayout<T, S>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ CaseDev<T, S> C;
    const int tid = threadIdx.x + threadIdx.y * 64;
    if ((int)blockIdx.x >= *nitems) return;
    const WorkItem w = items[blockIdx.x];
    load_case(C, cases, w.x);
    __syncthreads();
    const int by = w.z + (int)blockIdx.y;
    if (by >= min(w.z + KB_ROWS, C.gym)) return;
    if (smem_u32(smem_raw) & 127u) {
        if (tid == 0) atomicExch(&C.ctl->fault, 2);
        return;
    }
    const int par = C.ctl->tpar & 1;
    const MainMaps *M = maps + 2 * w.x + par;
    const int x0 = w.y * 64, y0 = by * 4;
    if (tid == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
        const int gsel = (C.ctl->cur0 + C.ctl->flips) & 1;
        mbar_expect_tx(&bar, L::tx(false) + C.P.tx_extra);
        tma_load_3d(smem_raw + L::pops, &M->pops, &bar, x0, y0, 0);
        tma_load_3d(smem_raw + L::pops + sizeof(S) * 27 * 256, &M->phiu, &bar, x0, y0, 0);
        tma_load_3d(smem_raw + L::tpl, gsel ? &M->g[1] : &M->g[0], &bar, x0, y0, 0);
        tma_load_2d(smem_raw + L::tpl + sizeof(T) * 4 * 256, &M->mur, &bar, x0, y0);
        tma_load_2d(smem_raw + L::tpl + sizeof(T) * 5 * 256, &M->gxr, &bar, x0, y0);
        tma_load_2d(smem_raw + L::tpl + sizeof(T) * 6 * 256, &M->gyr, &bar, x0, y0);
        tma_load_2d(smem_raw + L::dphi, &M->dphi, &bar, x0 - TMA_HX, y0);
        tma_load_2d(smem_raw + L::phir, &M->phir, &bar, x0 - TMA_HX, y0);
    }
    __syncthreads();   // the barrier is initialised before anyone waits on it
    const bool late = !mbar_wait_bounded(&bar, 0);
    if (__syncthreads_or(late)) {
        if (tid == 0) atomicExch(&C.ctl->fault, 1);
        mbar_wait_bounded(&bar, 0);
        return;
    }
    const TmaView<T, S> tv{reinterpret_cast<const S *>(smem_raw + L::pops),
                           reinterpret_cast<const T *>(smem_raw + L::tpl),
                           reinterpret_cast<const T *>(smem_raw + L::dphi),
                           reinterpret_cast<const T *>(smem_raw + L::phir)};
    main_body<T, S, SNAP, false, false, false, 5, true>(C.P, C.pops[par], C.pops[par ^ 1], C.g[0], C.g[1], C.ctl,
                                                        C.ref, C.phiu, C.psi_prev, C.snap, C.part,
                                                        &C.ctl->unstable, w.y, by, (long long)by * C.gxm + w.y, &tv);
}

// End of step of every case (one block of 256 per case at a time).
template <typename T, typename S>
__global__ void __launch_bounds__(256) kb_step_end(const CaseDev<T, S> *__restrict__ cases, const int *__restrict__ ncases,
                                                   int sums)
{
    griddep_begin();
    const int n = *ncases;
    for (int c = blockIdx.x; c < n; c += gridDim.x) {
        const CaseDev<T, S> *C = cases + c;
        step_end_body(C->part, C->nb_main, C->part2, C->nb_tb, C->ctl, nullptr, 0, sums);
        __syncthreads();
    }
}

// Slice sums of every case of a batch, item (case, slice) at parts[3 * item]
// with DEF_MAX_SLICES items per case
// (launch: any number of blocks of 256).
template <typename T, typename S>
__global__ void __launch_bounds__(256) kb_deform_sums(const CaseDev<T, S> *__restrict__ cases,
                                                      const int *__restrict__ ncases, double *parts)
{
    __shared__ double red[256][3];
    const long long n = (long long)*ncases * DEF_MAX_SLICES;
    for (long long i = blockIdx.x; i < n; i += gridDim.x) {
        const CaseDev<T, S> *C = cases + i / DEF_MAX_SLICES;
        const int j = (int)(i % DEF_MAX_SLICES), nsl = deform_slices(C->P.nx, C->P.ny);
        if (j < nsl) deform_slice_sums(C->snap, C->P.nx, C->P.ny, j, nsl, red, parts + 3 * i);
    }
}

// D of every case of a batch from its slice sums (launch: any number of blocks of 256).
template <typename T, typename S>
__global__ void __launch_bounds__(256) kb_deform_finish(const CaseDev<T, S> *__restrict__ cases,
                                                        const int *__restrict__ ncases,
                                                        const double *__restrict__ parts, double *out)
{
    __shared__ double red[256][3];
    const int n = *ncases;
    for (int c = blockIdx.x; c < n; c += gridDim.x)
        deform_finish(cases[c].snap, cases[c].P.nx, cases[c].P.ny, parts + (long long)3 * DEF_MAX_SLICES * c, red,
                      out + c);
}

}  // namespace ehdlb

namespace ehdlb {

// Zero the per-call counters of every case (one thread per case).
template <typename T, typename S>
__global__ void kb_open(const CaseDev<T, S> *__restrict__ cases, const int *__restrict__ ncases)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= *ncases) return;
    Control *ctl = cases[c].ctl;
    ctl->unstable = 0;
    ctl->tloc = 0;
    ctl->sweeps_total = 0;
    ctl->sweeps_max = 0;
    ctl->notconv = 0;
}

template <typename T, typename S> class Batch : public BatchBase {
  public:
    static constexpr int TBMAX = 5;
    static constexpr int TBR_R = 5;   // rows per thread of the register-blocked sweeps (64 x 40 regions)
    using Sv = Solver<T, S>;

    Batch(int sweeps, cudaStream_t s) : S_(sweeps), stream_(s) {}

    ~Batch() override
    {
        if (gexec_) cudaGraphExecDestroy(gexec_);
        cases_.clear();   // solvers release their arena blocks before the arena goes
        for (void *p : dev_) cudaFree(p);
        if (ev0_) cudaEventDestroy(ev0_);
        if (ev1_) cudaEventDestroy(ev1_);
        if (own_stream_) cudaStreamDestroy(stream_);
    }

    int init(size_t budget, std::string &err)
    {
        if (!stream_) {
            EHDLB_CK(cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking));
            own_stream_ = true;
        }
        EHDLB_CK(arena_.init(budget));
        EHDLB_CK(cudaEventCreate(&ev0_));
        EHDLB_CK(cudaEventCreate(&ev1_));
        EHDLB_CK(dalloc((void **)&d_nitems_, sizeof(host_nitems_)));
        int dev = 0;
        EHDLB_CK(cudaGetDevice(&dev));
        EHDLB_CK(cudaDeviceGetAttribute(&sms_, cudaDevAttrMultiProcessorCount, dev));
        EHDLB_CK(cudaFuncSetAttribute(kb_main<T, S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)main_smem_bytes<T, S>()));
        EHDLB_CK(cudaFuncSetAttribute(kb_main<T, S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)main_smem_bytes<T, S>()));
        EHDLB_CK(cudaFuncSetAttribute(kb_main_tma<T, S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)TmaLayout<T, S>::stage));
        EHDLB_CK(cudaFuncSetAttribute(kb_main_tma<T, S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)TmaLayout<T, S>::stage));
        EHDLB_CK(sweep_attr<1>());
        EHDLB_CK(sweep_attr<2>());
        EHDLB_CK(sweep_attr<3>());
        EHDLB_CK(sweep_attr<4>());
        EHDLB_CK(sweep_attr<5>());
        return EHDLB_OK;
    }

    int add(int nx, int ny, const ehdlb_params &p, int *id, std::string &err) override
    {
        if (nx % 8 != 0) { err = "batch lattices need nx to be a multiple of 8"; return EHDLB_EINVAL; }
        if (p.sweeps_min != S_ || p.sweeps_max != S_) {
            err = "batch cases take the batch's fixed sweeps per step (sweeps_min = sweeps_max)";
            return EHDLB_EINVAL;
        }
        if (p.freeze_E || p.side_walls || p.init_sweeps_fixed < 0 || p.ion_lattice == 9) {
            err = "batch cases need freeze_E = 0, side_walls = 0, ions on D2Q5 and init_sweeps_fixed >= 0";
            return EHDLB_EINVAL;
        }
        if (Sv::footprint(nx, ny) > arena_.largest_free()) {
            err = "not enough free device memory in the batch's budget";
            return EHDLB_EFULL;
        }
        std::unique_ptr<Sv> sv(new Sv(nx, ny, stream_, &arena_));
        int st = sv->allocate(err);
        if (st == EHDLB_OK) st = sv->set_params(p, err);
        if (st != EHDLB_OK) {
            if (st == EHDLB_ENOMEM) st = EHDLB_EFULL;
            return st;
        }
        const int k = next_id_++;
        cases_[k] = std::move(sv);
        *id = k;
        dirty_ = true;
        return EHDLB_OK;
    }

    int remove(int id, std::string &err) override
    {
        auto it = cases_.find(id);
        if (it == cases_.end()) { err = "no such case"; return EHDLB_EINVAL; }
        EHDLB_CK(cudaStreamSynchronize(stream_));
        cases_.erase(it);
        dirty_ = true;
        return EHDLB_OK;
    }

    int step(int nsteps, ehdlb_batch_stats *st, std::string &err) override
    {
        if (cases_.empty()) { err = "the batch has no case"; return EHDLB_ESTATE; }
        if (dirty_) {
            const int r = rebuild(err);
            if (r != EHDLB_OK) return r;
        }
        const auto t0 = std::chrono::steady_clock::now();
        launches_ = 0;
        kb_open<T, S><<<(ncases_ + 127) / 128, 128, 0, stream_>>>(d_cases_, d_nitems_ + 6);
        ++launches_;
        EHDLB_CK(cudaGetLastError());
        EHDLB_CK(cudaEventRecord(ev0_, stream_));
        for (int s = 0; s < nsteps; ++s) {
            const bool last = s == nsteps - 1;
            if (graphs_ && !last) {
                if (!gexec_) {
                    const int r = capture(err);
                    if (r != EHDLB_OK) return r;
                }
                EHDLB_CK(cudaGraphLaunch(gexec_, stream_));
                launches_ += per_step_launches();
            } else {
                enqueue_step(last);
            }
            EHDLB_CK(cudaGetLastError());
        }
        EHDLB_CK(cudaEventRecord(ev1_, stream_));
        EHDLB_CK(cudaStreamSynchronize(stream_));
        float ms = 0.f;
        EHDLB_CK(cudaEventElapsedTime(&ms, ev0_, ev1_));
        const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        // per-case control blocks: instability
        int unstable = 0, fault = 0;
        std::vector<Control> ctl(ncases_);
        for (int c = 0; c < ncases_; ++c)
            EHDLB_CK(cudaMemcpyAsync(&ctl[c], host_cases_[c].ctl, sizeof(Control), cudaMemcpyDeviceToHost, stream_));
        EHDLB_CK(cudaStreamSynchronize(stream_));
        for (int c = 0; c < ncases_; ++c) {
            unstable += ctl[c].unstable != 0;
            fault += ctl[c].fault != 0;
        }
        if (st) {
            st->steps = nsteps;
            st->cases = ncases_;
            st->seconds = secs;
            st->device_ms = ms;
            st->mlups = ms > 0 ? (double)nodes_ * nsteps / (ms * 1e-3) / 1e6 : 0.0;
            st->launches = launches_;
            st->unstable_cases = unstable;
            st->sweeps_per_launch = chunk_;
            st->tile_shape = shape_;
        }
        if (fault) { err = "a staged copy of the step kernel did not arrive in time"; return EHDLB_ECUDA; }
        if (unstable) { err = "NaN or Inf in a case"; return EHDLB_EUNSTABLE; }
        return EHDLB_OK;
    }

    int get_fields(int id, unsigned mask, double *dst, std::string &err) override
    {
        auto it = cases_.find(id);
        if (it == cases_.end()) { err = "no such case"; return EHDLB_EINVAL; }
        return it->second->get_fields(mask, dst, err);
    }

    int get_state(int id, double *dst, std::string &err) override
    {
        auto it = cases_.find(id);
        if (it == cases_.end()) { err = "no such case"; return EHDLB_EINVAL; }
        return it->second->get_state(dst, err);
    }

    int case_size(int id, int *nx, int *ny) const override
    {
        auto it = cases_.find(id);
        if (it == cases_.end()) return EHDLB_EINVAL;
        *nx = it->second->nx();
        *ny = it->second->ny();
        return EHDLB_OK;
    }

    int deformation(int n, const int *ids, double *out, std::string &err) override
    {
        if (cases_.empty()) { err = "the batch has no case"; return EHDLB_ESTATE; }
        if (dirty_) {
            const int r = rebuild(err);
            if (r != EHDLB_OK) return r;
        }
        kb_deform_sums<T, S><<<(int)std::min<long long>((long long)ncases_ * DEF_MAX_SLICES, 8LL * sms_), 256, 0,
                               stream_>>>(d_cases_, d_nitems_ + 6, d_Dpart_);
        kb_deform_finish<T, S><<<std::min(ncases_, 4 * sms_), 256, 0, stream_>>>(d_cases_, d_nitems_ + 6, d_Dpart_,
                                                                                 d_D_);
        EHDLB_CK(cudaGetLastError());
        std::vector<double> all(ncases_);
        EHDLB_CK(cudaMemcpyAsync(all.data(), d_D_, sizeof(double) * ncases_, cudaMemcpyDeviceToHost, stream_));
        EHDLB_CK(cudaStreamSynchronize(stream_));
        for (int i = 0; i < n; ++i) {
            auto pos = index_of_.find(ids[i]);
            if (pos == index_of_.end()) { err = "no such case"; return EHDLB_EINVAL; }
            out[i] = all[pos->second];
        }
        return EHDLB_OK;
    }

    int set_tuning(int sweeps_per_launch, int shape, int use_graphs) override
    {
        if (sweeps_per_launch >= 1) chunk_ = std::min(TBMAX, sweeps_per_launch);
        if (shape >= 0) shape_ = std::min(shape, 2);
        if (use_graphs >= 0) graphs_ = use_graphs != 0;
        drop_graph();
        return EHDLB_OK;
    }

    int autotune(int steps, int *best_chunk, int *best_shape, double *best_ms, std::string &err) override
    {
        // every configuration runs `steps` batch steps of the current cases
        // (they advance); the fastest per step is kept
        double best = 1e300;
        int bc = chunk_, bs = shape_;
        for (int sh = 0; sh < 3; ++sh)
            for (int ch = 3; ch <= TBMAX; ++ch) {
                set_tuning(ch, sh, -1);
                ehdlb_batch_stats st{};
                int r = step(1, &st, err);   // warm-up (and graph capture)
                if (r == EHDLB_OK) r = step(steps, &st, err);
                if (r != EHDLB_OK) return r;
                const double per = st.device_ms / steps;
                if (per < best) { best = per; bc = ch; bs = sh; }
            }
        set_tuning(bc, bs, -1);
        if (best_chunk) *best_chunk = bc;
        if (best_shape) *best_shape = bs;
        if (best_ms) *best_ms = best;
        return EHDLB_OK;
    }

    void info(int *cases, size_t *in_use, size_t *capacity) const override
    {
        if (cases) *cases = (int)cases_.size();
        if (in_use) *in_use = arena_.in_use();
        if (capacity) *capacity = arena_.capacity();
    }

  private:
    cudaError_t dalloc(void **p, size_t bytes)
    {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) dev_.push_back(*p);
        return e;
    }

    template <int NSW> cudaError_t sweep_attr()
    {
        cudaError_t e = cudaSuccess;
        for (cudaError_t x : {cudaFuncSetAttribute(kb_sweep_r<T, S, NSW, TBR_R, true>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)tbr_smem_bytes<T, TBR_R, 8>(true)),
                              cudaFuncSetAttribute(kb_sweep_r<T, S, NSW, TBR_R, false>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)tbr_smem_bytes<T, TBR_R, 8>(false))})
            if (x != cudaSuccess) e = x;
        const int sm = (int)tb_smem_bytes<T, 64, 32>(true);
        for (cudaError_t x : {cudaFuncSetAttribute(kb_sweep<T, S, NSW, 16, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm),
                              cudaFuncSetAttribute(kb_sweep<T, S, NSW, 16, 3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm),
                              cudaFuncSetAttribute(kb_sweep<T, S, NSW, 8, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm),
                              cudaFuncSetAttribute(kb_sweep<T, S, NSW, 8, 4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)})
            if (x != cudaSuccess) e = x;
        return e;
    }

    // blocks of a persistent launch: resident blocks per SM x SMs
    template <typename K> int pgrid(K kernel, int threads, size_t smem, int items)
    {
        int per = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess || per < 1) per = 1;
        return std::max(1, std::min(items, per * sms_));
    }

    int per_step_launches() const { return 3 + (S_ + chunk_ - 1) / chunk_; }

    template <int NSW, int BY, int MINB> void sweep_launch(int m)
    {
        const size_t sm = tb_smem_bytes<T, 64, 32>(m == 0);
        const int items = host_nitems_[NSW];
        if (m == 0) {
            const int g = pgrid(kb_sweep<T, S, NSW, BY, MINB, true>, 32 * BY, sm, items);
            launch_k(stream_, kb_sweep<T, S, NSW, BY, MINB, true>, dim3(g), dim3(32, BY), sm, true, d_cases_,
                     d_items_tb_[NSW], d_nitems_ + NSW, m);
        } else {
            const int g = pgrid(kb_sweep<T, S, NSW, BY, MINB, false>, 32 * BY, sm, items);
            launch_k(stream_, kb_sweep<T, S, NSW, BY, MINB, false>, dim3(g), dim3(32, BY), sm, true, d_cases_,
                     d_items_tb_[NSW], d_nitems_ + NSW, m);
        }
    }

    template <int NSW> void sweep_launch_r(int m)
    {
        const size_t sm = tbr_smem_bytes<T, TBR_R, 8>(m == 0);
        const int items = host_nitems_[8 + NSW];
        if (m == 0) {
            const int g = pgrid(kb_sweep_r<T, S, NSW, TBR_R, true>, 256, sm, items);
            launch_k(stream_, kb_sweep_r<T, S, NSW, TBR_R, true>, dim3(g), dim3(32, 8), sm, true, d_cases_,
                     d_items_tbr_[NSW], d_nitems_ + 8 + NSW, m);
        } else {
            const int g = pgrid(kb_sweep_r<T, S, NSW, TBR_R, false>, 256, sm, items);
            launch_k(stream_, kb_sweep_r<T, S, NSW, TBR_R, false>, dim3(g), dim3(32, 8), sm, true, d_cases_,
                     d_items_tbr_[NSW], d_nitems_ + 8 + NSW, m);
        }
    }

    template <int NSW> void sweep_launch_shape(int m)
    {
        if (shape_ == 2) sweep_launch_r<NSW>(m);
        else if (shape_ == 1) sweep_launch<NSW, 8, 4>(m);
        else sweep_launch<NSW, 16, 3>(m);
    }

    void enqueue_step(bool last)
    {
        const int nk = (S_ + chunk_ - 1) / chunk_;
        const int items = host_nitems_[0];
        launch_k(stream_, kb_prep<T, S>, dim3(std::max(1, items), KB_ROWS), dim3(64, 4), 0, true, d_cases_,
                 d_items_node_, d_nitems_, S_, nk);
        for (int m = 0, done = 0; m < nk; ++m) {
            const int nsw = std::min(chunk_, S_ - done);
            switch (nsw) {
            case 1: sweep_launch_shape<1>(m); break;
            case 2: sweep_launch_shape<2>(m); break;
            case 3: sweep_launch_shape<3>(m); break;
            case 4: sweep_launch_shape<4>(m); break;
            default: sweep_launch_shape<5>(m); break;
            }
            done += nsw;
        }
        const size_t msm = main_smem_bytes<T, S>();
        const dim3 mg(std::max(1, items), KB_ROWS), mb(64, 4);
        if (tma_) {   // every case's tile staged through its tensor maps
            const size_t tsm = TmaLayout<T, S>::stage;
            if (last)
                launch_k(stream_, kb_main_tma<T, S, true>, mg, mb, tsm, true, d_cases_, d_maps_, d_items_node_,
                         d_nitems_);
            else
                launch_k(stream_, kb_main_tma<T, S, false>, mg, mb, tsm, true, d_cases_, d_maps_, d_items_node_,
                         d_nitems_);
        } else if (last) {
            launch_k(stream_, kb_main<T, S, true>, mg, mb, msm, true, d_cases_, d_items_node_, d_nitems_);
        } else {
            launch_k(stream_, kb_main<T, S, false>, mg, mb, msm, true, d_cases_, d_items_node_, d_nitems_);
        }
        launch_k(stream_, kb_step_end<T, S>, dim3(std::min(ncases_, 4 * sms_)), dim3(256), 0, true, d_cases_,
                 d_nitems_ + 6, last ? 1 : 0);
        launches_ += per_step_launches();
    }

    int capture(std::string &err)
    {
        cudaGraph_t g = nullptr;
        EHDLB_CK(cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal));
        enqueue_step(false);
        launches_ -= per_step_launches();
        EHDLB_CK(cudaStreamEndCapture(stream_, &g));
        const cudaError_t e = cudaGraphInstantiate(&gexec_, g, 0);
        cudaGraphDestroy(g);
        EHDLB_CK(e);
        return EHDLB_OK;
    }

    void drop_graph()
    {
        if (gexec_) cudaGraphExecDestroy(gexec_);
        gexec_ = nullptr;
    }

    // growable device array; a new allocation invalidates the captured graph
    template <typename E> cudaError_t ensure(E *&ptr, size_t &cap, size_t n)
    {
        if (n <= cap && ptr) return cudaSuccess;
        const size_t want = std::max<size_t>(n, cap * 2 + 64);
        E *p = nullptr;
        cudaError_t e = dalloc((void **)&p, sizeof(E) * want);
        if (e != cudaSuccess) return e;
        ptr = p;   // the old block stays allocated until the batch is destroyed
        cap = want;
        drop_graph();
        return cudaSuccess;
    }

    // descriptors and work-lists of the current cases
    int rebuild(std::string &err)
    {
        EHDLB_CK(cudaStreamSynchronize(stream_));
        host_cases_.clear();
        index_of_.clear();
        std::vector<WorkItem> node;
        std::vector<WorkItem> tb[TBMAX + 1], tbr[TBMAX + 1];
        std::vector<MainMaps> maps;   // two per case: its time levels
        bool all_maps = true;
        nodes_ = 0;
        int c = 0;
        for (auto &kv : cases_) {
            const Sv &sv = *kv.second;
            CaseDev<T, S> d{};
            sv.describe(d.P, d.pops, d.g, d.phiu, d.phig, d.q, d.coef, d.psi_prev, d.snap, d.ref, d.part, d.part2,
                        d.ctl);
            const int nx = sv.nx(), ny = sv.ny();
            const int gx = (nx + 63) / 64, gy = (ny + 3) / 4;
            d.nb_main = (long long)gx * gy;
            d.nb_tb = 0;
            d.gxm = gx;
            d.gym = gy;
            host_cases_.push_back(d);
            MainMaps m[2] = {};
            all_maps = sv.main_maps(m) && all_maps;
            maps.push_back(m[0]);
            maps.push_back(m[1]);
            index_of_[kv.first] = c;
            for (int by = 0; by < gy; by += KB_ROWS)
                for (int bx = 0; bx < gx; ++bx) node.push_back(make_int4(c, bx, by, by * gx + bx));
            for (int nsw = 1; nsw <= TBMAX; ++nsw) {
                const int tx = 64 - 2 * nsw, ty = 32 - 2 * nsw;
                const int tgx = (nx + tx - 1) / tx, tgy = (ny + ty - 1) / ty;
                for (int by = 0; by < tgy; ++by)
                    for (int bx = 0; bx < tgx; ++bx) tb[nsw].push_back(make_int4(c, bx, by, by * tgx + bx));
                const int rx = 64 - 2 * tbr_halo_x(nsw), ry = 8 * TBR_R - 2 * nsw;
                const int rgx = (nx + rx - 1) / rx, rgy = (ny + ry - 1) / ry;
                for (int by = 0; by < rgy; ++by)
                    for (int bx = 0; bx < rgx; ++bx) tbr[nsw].push_back(make_int4(c, bx, by, by * rgx + bx));
            }
            nodes_ += (long long)nx * ny;
            ++c;
        }
        ncases_ = c;
        EHDLB_CK(ensure(d_cases_, cap_cases_, host_cases_.size()));
        EHDLB_CK(ensure(d_D_, cap_D_, host_cases_.size()));
        EHDLB_CK(ensure(d_Dpart_, cap_Dpart_, host_cases_.size() * 3 * DEF_MAX_SLICES));
        EHDLB_CK(ensure(d_items_node_, cap_node_, node.size()));
        EHDLB_CK(ensure(d_maps_, cap_maps_, maps.size()));
        tma_ = all_maps && !maps.empty();
        for (int nsw = 1; nsw <= TBMAX; ++nsw) {
            EHDLB_CK(ensure(d_items_tb_[nsw], cap_tb_[nsw], tb[nsw].size()));
            EHDLB_CK(ensure(d_items_tbr_[nsw], cap_tbr_[nsw], tbr[nsw].size()));
        }
        EHDLB_CK(cudaMemcpyAsync(d_cases_, host_cases_.data(), sizeof(CaseDev<T, S>) * host_cases_.size(),
                                 cudaMemcpyHostToDevice, stream_));
        EHDLB_CK(cudaMemcpyAsync(d_items_node_, node.data(), sizeof(WorkItem) * node.size(), cudaMemcpyHostToDevice,
                                 stream_));
        if (!maps.empty())
            EHDLB_CK(cudaMemcpyAsync(d_maps_, maps.data(), sizeof(MainMaps) * maps.size(), cudaMemcpyHostToDevice,
                                     stream_));
        for (int nsw = 1; nsw <= TBMAX; ++nsw)
            EHDLB_CK(cudaMemcpyAsync(d_items_tbr_[nsw], tbr[nsw].data(), sizeof(WorkItem) * tbr[nsw].size(),
                                     cudaMemcpyHostToDevice, stream_));
        for (int nsw = 1; nsw <= TBMAX; ++nsw)
            EHDLB_CK(cudaMemcpyAsync(d_items_tb_[nsw], tb[nsw].data(), sizeof(WorkItem) * tb[nsw].size(),
                                     cudaMemcpyHostToDevice, stream_));
        host_nitems_[0] = (int)node.size();
        for (int nsw = 1; nsw <= TBMAX; ++nsw) {
            host_nitems_[nsw] = (int)tb[nsw].size();
            host_nitems_[8 + nsw] = (int)tbr[nsw].size();
        }
        host_nitems_[6] = ncases_;
        host_nitems_[7] = 0;
        EHDLB_CK(cudaMemcpyAsync(d_nitems_, host_nitems_, sizeof(host_nitems_), cudaMemcpyHostToDevice, stream_));
        EHDLB_CK(cudaStreamSynchronize(stream_));
        // the grids of a captured step depend on the item counts
        drop_graph();
        dirty_ = false;
        return EHDLB_OK;
    }

    int S_;
    cudaStream_t stream_;
    bool own_stream_ = false;
    Arena arena_;
    std::map<int, std::unique_ptr<Sv>> cases_;
    std::map<int, int> index_of_;
    std::vector<CaseDev<T, S>> host_cases_;
    int next_id_ = 0;
    int ncases_ = 0;
    long long nodes_ = 0;
    bool dirty_ = true;
    int chunk_ = 5, shape_ = 2;
    bool graphs_ = true;
    int sms_ = 1;
    long long launches_ = 0;
    std::vector<void *> dev_;
    CaseDev<T, S> *d_cases_ = nullptr;
    double *d_D_ = nullptr;
    double *d_Dpart_ = nullptr;   // slice sums of the deformation factor
    WorkItem *d_items_node_ = nullptr;
    MainMaps *d_maps_ = nullptr;   // tensor maps of the staged step kernel, two per case
    size_t cap_maps_ = 0;
    bool tma_ = false;             // every case takes the staged step kernel (kb_main_tma)
    WorkItem *d_items_tb_[TBMAX + 1] = {};
    WorkItem *d_items_tbr_[TBMAX + 1] = {};   // tiles of the register-blocked sweeps
    int *d_nitems_ = nullptr;   // [0] node items, [1..5] sweep items by NSW, [6] cases, [9..13] register-blocked sweep items
    int host_nitems_[16] = {};
    size_t cap_cases_ = 0, cap_D_ = 0, cap_Dpart_ = 0, cap_node_ = 0, cap_tb_[TBMAX + 1] = {}, cap_tbr_[TBMAX + 1] = {};
    cudaGraphExec_t gexec_ = nullptr;
    cudaEvent_t ev0_ = nullptr, ev1_ = nullptr;
};

}  // namespace ehdlb
