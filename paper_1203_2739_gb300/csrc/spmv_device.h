// Device-side view of a plan and the per-precision launchers.  Included by the
// CUDA translation units only.
#pragma once

#include <cuda_runtime.h>

#include "spmv_internal.h"

namespace spmv {

struct DevPlan {
    int32_t m = 0, n = 0, nrhs = 1, lanes = 8, long_thresh = 0;
    bool use_k1 = true;
    const int32_t *rowptr = nullptr;   // K1: m+1; tiles: plan rows + 1
    const int32_t *col32 = nullptr;
    const uint16_t *col16 = nullptr;
    const void *val = nullptr;
    const int32_t *long_rows = nullptr;
    int32_t n_long = 0;
    const Tile *tiles = nullptr;
    int32_t n_tiles = 0;
    const int32_t *chunk_off = nullptr;
    const int32_t *chunk_mix = nullptr;
    const int32_t *slot_dst = nullptr;
    const int32_t *slot_len = nullptr;
    const VRow *vrows = nullptr;
    const int32_t *xlist = nullptr;
    void *partial = nullptr;
    const Fixup *fixups = nullptr;
    int32_t n_fixups = 0;
    int32_t smem_bytes = 0;            // staged x entries
    // SM-affine schedule (nq = 0: one CTA per tile in tile order)
    const int32_t *qbeg = nullptr;     // nq + 1
    int32_t *qcount = nullptr;         // nq + 1 counters, zero between launches
    int32_t nq = 0;
    int32_t *status = nullptr;         // 1 after a bounded device wait gave up
    uint32_t wait_limit = 1u << 22;    // polls of the first wait on a staging copy
    // persistent schedule (ctr = NULL: one CTA per tile)
    int32_t *ctr = nullptr;            // next-tile counter, finished-CTA counter
    int32_t n_sm = 0;
    int32_t cta_threads = 256;         // 256, 512 (two per SM) or 1024 (one per SM)
};

cudaError_t exec_f64(const DevPlan &P, const void *x, void *y, cudaStream_t s);
cudaError_t exec_f32(const DevPlan &P, const void *x, void *y, cudaStream_t s);
cudaError_t exec_bf16(const DevPlan &P, const void *x, void *y, cudaStream_t s);

// dst[i*r + c] = src[perm[i]*r + c] (gather) or dst[perm[i]*r + c] = src[i*r + c]
// (scatter), elements of elem_bytes (4 or 8).
cudaError_t permute_vector(int elem_bytes, int32_t count, int32_t r, const int32_t *perm,
                           const void *src, void *dst, bool scatter, cudaStream_t s);

}  // namespace spmv
