// Kernel instantiations for values of type __nv_bfloat16 with x / y / accumulation in float.
#include "spmv_kernels.cuh"

namespace spmv {

cudaError_t exec_bf16(const DevPlan &P, const void *x, void *y, cudaStream_t s)
{
    return launch_exec<__nv_bfloat16, float>(P, x, y, s);
}

}  // namespace spmv
