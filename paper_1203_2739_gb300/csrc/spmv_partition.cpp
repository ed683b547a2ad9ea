// placeholder, replaced by the recursive hypergraph bisection
#include "spmv_internal.h"
extern "C" spmv_status spmv_partition(const spmv_csr *, const spmv_partition_opts *, spmv_partition_out *out)
{
    if (out) *out = spmv_partition_out{};
    spmv::set_error("not built yet");
    return SPMV_E_UNSUPPORTED;
}
extern "C" void spmv_partition_free(spmv_partition_out *) {}
