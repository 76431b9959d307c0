// ehdlb_solver_base.h -- interface between the C-ABI layer and the
// precision-specific CUDA solvers (float: solver_fp32.cu, double:
// solver_fp64.cu, float with FP16 storage: solver_fp16s.cu).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "ehdlb.h"

namespace ehdlb {

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
    virtual void set_timing(int on) = 0;
    virtual void set_tuning(int sweeps_per_launch, int shape, int vec_staging) = 0;
    int last_nsteps = 0;
};

SolverBase *make_solver_fp32(int nx, int ny, cudaStream_t s, int *status, std::string &err);
SolverBase *make_solver_fp64(int nx, int ny, cudaStream_t s, int *status, std::string &err);
SolverBase *make_solver_fp16s(int nx, int ny, cudaStream_t s, int *status, std::string &err);

}  // namespace ehdlb
