// Kernel instantiations for values of type float with x / y / accumulation in float.
#include "spmv_kernels.cuh"

namespace spmv {

cudaError_t exec_f32(const DevPlan &P, const void *x, void *y, cudaStream_t s)
{
    return launch_exec<float, float>(P, x, y, s);
}

}  // namespace spmv
