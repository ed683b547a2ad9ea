// The plan object behind the C ABI's opaque spmv_plan (spmv_capi.cu owns its
// life cycle; spmv_cg.cu drives two plans in its solver).
#pragma once

#include "spmv_device.h"

struct spmv_plan {
    spmv::HostPlan hp;            // metadata only after upload
    spmv::DevPlan dp;
    spmv_plan_info info{};
    void *arena = nullptr;
    size_t arena_bytes = 0;
    void *(*alloc)(size_t, void *) = nullptr;
    void (*release)(void *, void *) = nullptr;
    void *ctx = nullptr;
    int device = 0;
    const int32_t *d_row_perm = nullptr;
    const int32_t *d_col_perm = nullptr;
    bool same_perm = true;        // square, and row_perm == col_perm (both may be NULL)
    void *io_x = nullptr, *io_y = nullptr;
    int32_t *h_status = nullptr;  // pinned copy of the device status word
    size_t xbytes = 0, ybytes = 0;
};

namespace spmv {

// Device memory through the plan's allocator (cudaMalloc when it has none).
void *plan_alloc(spmv_plan *p, size_t bytes);
void plan_free(spmv_plan *p, void *ptr);

// y_hat <- A_hat x_hat with the plan's kernels on stream s (no checks).
cudaError_t plan_run(const spmv_plan *p, const void *x, void *y, cudaStream_t s);

}  // namespace spmv
