// batch_fp32.cu -- batches of float lattices (float storage and FP16 storage).
#include "ehdlb_batch.cuh"

namespace ehdlb {

template <typename T, typename S>
static BatchBase *make_batch(size_t budget, int sweeps, cudaStream_t s, int *status, std::string &err)
{
    Batch<T, S> *b = new Batch<T, S>(sweeps, s);
    *status = b->init(budget, err);
    if (*status != EHDLB_OK) {
        delete b;
        return nullptr;
    }
    return b;
}

BatchBase *make_batch_fp32(size_t budget, int sweeps, cudaStream_t s, int *status, std::string &err)
{
    return make_batch<float, float>(budget, sweeps, s, status, err);
}

BatchBase *make_batch_fp16s(size_t budget, int sweeps, cudaStream_t s, int *status, std::string &err)
{
    return make_batch<float, __half>(budget, sweeps, s, status, err);
}

size_t footprint_fp32(int nx, int ny) { return Solver<float, float>::footprint(nx, ny); }
size_t footprint_fp16s(int nx, int ny) { return Solver<float, __half>::footprint(nx, ny); }

}  // namespace ehdlb
