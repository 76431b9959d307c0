// ehdlb_solver_base.h -- interface between the C-ABI layer and the
// precision-specific CUDA solvers (float: solver_fp32.cu, double:
// solver_fp64.cu, float with FP16 storage: solver_fp16s.cu).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "ehdlb.h"

namespace ehdlb {

// Device memory source of a solver: cudaMalloc by default, or an arena of
// the batch engine.
class DevArena {
  public:
    virtual ~DevArena() {}
    virtual cudaError_t alloc(void **p, size_t bytes) = 0;
    virtual void release(void *p) = 0;
};

class SolverBase {
  public:
    virtual ~SolverBase() {}
    virtual int set_params(const ehdlb_params &p, std::string &err) = 0;
    virtual int step(int nsteps, ehdlb_stats *st, std::string &err) = 0;
    virtual int get_fields(unsigned mask, double *dst, std::string &err) = 0;
    virtual int get_counts(int *dst, int n, std::string &err) = 0;
    virtual int get_state(double *dst, std::string &err) = 0;
    virtual int set_state(const double *src, std::string &err) = 0;
    virtual void set_schedule(const int *c, int n) = 0;
    virtual void set_timing(int every) = 0;
    virtual void set_tuning(int sweeps_per_launch, int shape, int vec_staging) = 0;
    virtual int deformation(double *out, std::string &err) = 0;
    // fields the last step of each call captures, and whether each call
    // also computes D of Eq. 63 (stats->deformation)
    virtual void set_reporting(unsigned snap_mask, int deformation) = 0;
    virtual int state_per_node() const = 0;   // doubles per node of get_state / set_state
    virtual int stall_next_copies() = 0;      // test hook (ehdlb_test_stall_copies)
    int last_nsteps = 0;
};

// A set of lattices stepped together (ehdlb_batch.cuh).
class BatchBase {
  public:
    virtual ~BatchBase() {}
    virtual int add(int nx, int ny, const ehdlb_params &p, int *id, std::string &err) = 0;
    virtual int remove(int id, std::string &err) = 0;
    virtual int step(int nsteps, ehdlb_batch_stats *st, std::string &err) = 0;
    virtual int get_fields(int id, unsigned mask, double *dst, std::string &err) = 0;
    virtual int get_state(int id, double *dst, std::string &err) = 0;
    virtual int case_size(int id, int *nx, int *ny) const = 0;
    virtual int deformation(int n, const int *ids, double *out, std::string &err) = 0;
    virtual int set_tuning(int sweeps_per_launch, int shape, int use_graphs) = 0;
    virtual int autotune(int steps, int *best_chunk, int *best_shape, double *best_ms, std::string &err) = 0;
    virtual void info(int *cases, size_t *in_use, size_t *capacity) const = 0;
};

BatchBase *make_batch_fp32(size_t budget, int sweeps, cudaStream_t s, int *status, std::string &err);
BatchBase *make_batch_fp16s(size_t budget, int sweeps, cudaStream_t s, int *status, std::string &err);
size_t footprint_fp32(int nx, int ny);
size_t footprint_fp16s(int nx, int ny);

SolverBase *make_solver_fp32(int nx, int ny, cudaStream_t s, int *status, std::string &err);
SolverBase *make_solver_fp64(int nx, int ny, cudaStream_t s, int *status, std::string &err);
SolverBase *make_solver_fp16s(int nx, int ny, cudaStream_t s, int *status, std::string &err);

}  // namespace ehdlb
