// solver_fp64.cu -- the lattice solver with double populations and arithmetic.
#include "ehdlb_solver.cuh"

namespace ehdlb {

SolverBase *make_solver_fp64(int nx, int ny, cudaStream_t s, int *status, std::string &err)
{
    Solver<double> *sv = new Solver<double>(nx, ny, s);
    *status = sv->allocate(err);
    if (*status != EHDLB_OK) {
        delete sv;
        return nullptr;
    }
    return sv;
}

}  // namespace ehdlb
