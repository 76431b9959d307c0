// solver_fp16s.cu -- the lattice solver with FP16 population storage (scaled
// deviations from rest states) and float arithmetic.
#include "ehdlb_solver.cuh"

namespace ehdlb {

SolverBase *make_solver_fp16s(int nx, int ny, cudaStream_t s, int *status, std::string &err)
{
    Solver<float, __half> *sv = new Solver<float, __half>(nx, ny, s);
    *status = sv->allocate(err);
    if (*status != EHDLB_OK) {
        delete sv;
        return nullptr;
    }
    return sv;
}

}  // namespace ehdlb
