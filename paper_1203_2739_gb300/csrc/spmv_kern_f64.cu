// Kernel instantiations for values of type double with x / y / accumulation in double.
#include "spmv_kernels.cuh"

namespace spmv {

cudaError_t exec_f64(const DevPlan &P, const void *x, void *y, cudaStream_t s)
{
    return launch_exec<double, double>(P, x, y, s);
}

}  // namespace spmv
