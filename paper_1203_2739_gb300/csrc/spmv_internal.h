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
// when the plan stages, the x entries it reuses are copied once into the
// CTA's shared memory and the others are gathered through L1 / L2; otherwise
// every x entry is gathered.
//
// Inside a tile the rows are sorted by length and cut into chunks of 32; a
// chunk is stored column-major (element k of the chunk's 32 rows are 32
// consecutive entries), so a warp handles 32 rows with one lane per row,
// coalesced loads and one full-width FMA per stored element.  GB300 executes
// two FP64 FMAs per SM per clock: an FP64 SpMV only keeps up with HBM when no
// FP64 instruction runs with idle lanes and no shuffle reductions are needed.
enum TileKind : int32_t {
    TILE_NARROW = 0,   // every nonzero reads staged x: 16-bit local indices (col16)
    TILE_MIXED = 1,    // col32 >= 0: staged index; col32 < 0: ~global x index
    TILE_GLOBAL = 2,   // col32 = global x index, nothing staged
    TILE_CHUNK = 3,    // elements [e0, e1) of one long row -> partial slot
    TILE_DELTA = 4     // nothing staged; chunks whose chunk_mix (the base
                       // column) is >= 0 store 16-bit column increments in
                       // col16, the others col32 as in GLOBAL tiles
};

// Column increments (the colDiff of ICSR, Sec. 2.1, kept per lane): in a
// chunk of a DELTA tile with base column B, lane i's running column starts at
// B and element k adds col16 at delta_pos(off, L, k, i); padding elements add
// 0.  Slots come in pairs, so that a lane reads the increments of two slots
// with one 32-bit load: slots 2p and 2p+1 of lane i sit at off + 64 p + 2 i
// and the next entry; when L is odd the last slot keeps the plain layout
// (off + 32 (L - 1) + i).  off is even.
inline int64_t delta_pos(int64_t off, int32_t L, int32_t k, int32_t i)
{
    if (k < L - (L & 1)) return off + 64 * (int64_t)(k >> 1) + 2 * i + (k & 1);
    return off + 32 * (int64_t)k + i;
}

// The staged window of a tile is up to two contiguous runs of x_hat and a
// gathered list, back to back in shared memory:
//   smem[0 .. runlen)                   = x_hat[run0 .. run0 + runlen)
//   smem[run2_at .. run2_at + run2len)  = x_hat[run2_0 .. run2_0 + run2len)
//   smem[run2_at + run2len + i]         = x_hat[xlist[list0 + i]]
// Each run starts on a 16-byte boundary of x_hat and of shared memory (its
// bulk copy needs both); run2_at rounds the first run's length up to that.
struct Tile {          // 64 bytes, copied to the device as is
    int32_t kind;
    int32_t chunk0, nchunks;  // chunks of 32 rows (not CHUNK tiles)
    int32_t slot;             // CHUNK: the partial slot it writes
    int32_t run0, runlen;     // first staged run
    int32_t run2_0, run2len;  // second staged run
    int32_t list0, listlen;   // gathered list
    int32_t e0, e1;           // CHUNK: element range (contiguous, global indices)
    int32_t vrow0, nvrows;    // rows too long for one lane: vrows[vrow0 ..]
    int32_t run2_at;          // shared-memory entry where the second run starts
                              // (the first run's length rounded up to 16 bytes)
    int32_t pad;
};
static_assert(sizeof(Tile) == 64, "Tile layout");

// A row of a tile reduced by a whole warp: elements [e0, e0 + len) stored
// contiguously with the tile's index encoding; dst as slot_dst.
struct VRow {
    int32_t e0, len, dst, pad;
};
static_assert(sizeof(VRow) == 16, "VRow layout");

struct Fixup {         // y[row] = sum of partial[slot0 .. slot0+count) in order
    int32_t row, slot0, count, pad;
};
static_assert(sizeof(Fixup) == 16, "Fixup layout");

// slot_dst encoding: >= 0 y row; -1 empty slot; <= -2 partial slot -(d + 2)
inline int32_t dst_partial(int32_t slot) { return -(slot + 2); }

// Host image of a plan: every array the device needs, in device layout.
struct HostPlan {
    int32_t m = 0, n = 0;
    int64_t nnz = 0;
    int32_t form = SPMV_NATURAL, K = 0, dtype = SPMV_F64, nrhs = 1;
    int32_t lanes = 8, tile_cols = 0, long_thresh = 0;
    int32_t flags = 0;
    int32_t cta_threads = 256;     // tiled kernel CTA size (1024: one per SM)
    bool use_k1 = true;            // natural form: vector-per-row kernel

    // K1: CSR.  Tiled forms: elements in chunk order, then the long rows.
    std::vector<int32_t> rowptr;   // K1 only
    std::vector<int32_t> col32;    // K1 / GLOBAL / CHUNK: x index; MIXED: signed
    std::vector<uint16_t> col16;   // NARROW tiles: shared-memory index; DELTA
                                   // tiles: column increments
    std::vector<double> val;       // FP64 master values in element order
    std::vector<int32_t> long_rows;  // K1: rows reduced by a whole CTA

    std::vector<Tile> tiles;
    std::vector<int32_t> chunk_off;  // element offset of each chunk
    // MIXED tiles: per chunk, the number of leading element slots that may
    // read x from global memory; every lane's elements from that slot on
    // are staged (each row stores its gathered elements first).  DELTA
    // tiles: the chunk's base column, or -1 for a chunk stored in col32.
    // Other tiles: 0.
    std::vector<int32_t> chunk_mix;
    std::vector<int32_t> slot_dst;   // 32 per chunk
    std::vector<int32_t> slot_len;   // 32 per chunk (row length, 0 if empty)
    std::vector<VRow> vrows;
    std::vector<int32_t> xlist;
    std::vector<Fixup> fixups;
    int64_t partial_slots = 0;
    int32_t n_chunk_tiles = 0, n_staged_tiles = 0, n_global_tiles = 0;
    int64_t staged_entries = 0, list_entries = 0, direct_nnz = 0, narrow_nnz = 0;
    int64_t delta_nnz = 0;         // nonzeros stored as column increments
    int32_t max_staged = 0;        // most x entries one tile stages
    int64_t padded_elems = 0;      // stored elements (with padding) in chunks
    int64_t fma_slots = 0;         // FMA lanes issued: 32 * (longest row) per chunk,
                                   // 32 * ceil(len / 32) per warp row
    int64_t mixed_slots = 0;       // element slots of MIXED chunks that load x
                                   // from both global and shared memory

    std::vector<int32_t> row_perm, col_perm;  // empty = identity
};

// Build the host image (validation, P_r A P_c, split, tiling).  n_sm: the
// device's SM count, which sets the default tile size (0 = 152, GB300).
spmv_status build_host_plan(const spmv_csr *A, const spmv_perm *perm,
                            const spmv_splits *splits, const spmv_opts *opts,
                            int32_t n_sm, HostPlan *out);

// Resident 256-thread CTAs per SM the tiled kernel is sized for (its
// register budget asks for at least this many), by right-hand-side count.
#ifndef SPMV_TILE_MINBLOCKS
#define SPMV_TILE_MINBLOCKS 6
#endif
inline int32_t tile_ctas_per_sm_for(int32_t r)
{
    return r <= 2 ? SPMV_TILE_MINBLOCKS : (r == 4 ? 4 : 3);
}

// Round-to-nearest-even FP64 -> BF16 bits.
uint16_t bf16_rne(double v);

// Form derivation (also behind spmv_form_from_labels).
spmv_status form_from_labels(const spmv_csr *A, int32_t form, int32_t K,
                             const int32_t *labels, int32_t *row_perm,
                             int32_t *col_perm, int32_t *row_part_ptr,
                             int32_t *col_part_ptr);

// Row / column orders of the comparison methods (spmv_reorder).
spmv_status reorder(const spmv_csr *A, int32_t method, int32_t K, const int32_t *labels,
                    int32_t *row_perm, int32_t *col_perm);

// Validate a host CSR (sorted unique columns, monotone rowptr).
spmv_status validate_csr(const spmv_csr *A);

int hardware_threads();

}  // namespace spmv
