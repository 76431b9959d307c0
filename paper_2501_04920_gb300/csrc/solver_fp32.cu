// solver_fp32.cu -- the lattice solver with float populations and arithmetic.
#include "ehdlb_solver.cuh"

namespace ehdlb {

SolverBase *make_solver_fp32(int nx, int ny, cudaStream_t s, int *status, std::string &err)
{
    Solver<float> *sv = new Solver<float>(nx, ny, s);
    *status = sv->allocate(err);
    if (*status != EHDLB_OK) {
        delete sv;
        return nullptr;
    }
    return sv;
}

}  // namespace ehdlb
