// Internal declarations shared by the host plan builder (spmv_plan.cpp), the
// partitioner (spmv_partition.cpp), the kernels (spmv_kern_*.cu) and the C ABI
// (spmv_capi.cu).  Not installed; the public interface is include/spmv.h.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "spmv.h"

namespace spmv {

// ---------------------------------------------------------------- errors --
void set_error(const char *fmt, ...);
void clear_error();

// ----------------------------------------------------------------- tiles --
// A tile is the unit of work of one CTA in the tiled kernel.  It plays the
// part the paper gives to a submatrix that "fits into the cache" (Sec. 3):
// its whole x working set is staged in the CTA's shared memory.
enum TileKind : int32_t {
    TILE_STAGED = 0,   // rows [r0,r1), x entries staged in shared memory
    TILE_GLOBAL = 1,   // rows [r0,r1), x gathered from global memory (L2)
    TILE_CHUNK = 2     // nonzeros [r0,r1) of one long row -> partial slot y0
};

struct Tile {          // 32 bytes, copied to the device as is
    int32_t kind;
    int32_t r0, r1;    // plan rows (STAGED/GLOBAL) or nonzero range (CHUNK)
    int32_t y0;        // >= 0: plan row r writes y[y0 + r - r0]; -1: via dst[r];
                       // CHUNK: the partial slot it writes
    int32_t run0, runlen;   // STAGED: x_hat[run0 + i] -> smem[i]
    int32_t list0, listlen; // STAGED: x_hat[xlist[list0 + i]] -> smem[runlen + i]
};
static_assert(sizeof(Tile) == 32, "Tile layout");

struct Fixup {         // y[row] = sum of partial[slot0 .. slot0+count) in order
    int32_t row, slot0, count, pad;
};
static_assert(sizeof(Fixup) == 16, "Fixup layout");

// Host image of a plan: every array the device needs, in device layout.
struct HostPlan {
    int32_t m = 0, n = 0;
    int64_t nnz = 0;
    int32_t form = SPMV_NATURAL, K = 0, dtype = SPMV_F64, nrhs = 1;
    int32_t lanes = 8, tile_cols = 0, long_thresh = 0;
    int32_t flags = 0;
    bool use_k1 = true;            // natural form: vector-per-row kernel

    std::vector<int32_t> rowptr;   // K1: m+1; tiles: plan rows + 1
    std::vector<int32_t> col32;    // global column (x_hat index) per nonzero
    std::vector<uint16_t> col16;   // local shared-memory index (staged tiles)
    std::vector<double> val;       // FP64 master values in plan order
    std::vector<int32_t> long_rows;  // K1: rows reduced by a whole CTA

    std::vector<Tile> tiles;
    std::vector<int32_t> xlist;
    std::vector<int32_t> dst;      // per plan row: y row, or -(slot+1)
    std::vector<Fixup> fixups;
    int64_t partial_slots = 0;
    int32_t n_chunk_tiles = 0, n_staged_tiles = 0, n_global_tiles = 0;
    int64_t staged_entries = 0, list_entries = 0;

    std::vector<int32_t> row_perm, col_perm;  // empty = identity
};

// Build the host image (validation, P_r A P_c, split, tiling).
spmv_status build_host_plan(const spmv_csr *A, const spmv_perm *perm,
                            const spmv_splits *splits, const spmv_opts *opts,
                            HostPlan *out);

// Round-to-nearest-even FP64 -> BF16 bits.
uint16_t bf16_rne(double v);

// Form derivation (also behind spmv_form_from_labels).
spmv_status form_from_labels(const spmv_csr *A, int32_t form, int32_t K,
                             const int32_t *labels, int32_t *row_perm,
                             int32_t *col_perm, int32_t *row_part_ptr,
                             int32_t *col_part_ptr);

// Validate a host CSR (sorted unique columns, monotone rowptr).
spmv_status validate_csr(const spmv_csr *A);

int hardware_threads();

}  // namespace spmv
