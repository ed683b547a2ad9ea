// SpMV kernels for sm_103a.  SpMV is a gather-and-reduce with about 0.17
// flop per byte in FP64, so these kernels are built around the memory system,
// not the tensor cores:
//
//  * k_csr_vector  -- plain natural-order CSR (Sec. 2.1): LANES threads per row,
//                     coalesced streaming of values and column indices
//                     (evict-first), x gathered through the read-only path,
//                     warp-shuffle reduction; rows longer than a threshold get
//                     a whole CTA each.  This is the baseline.
//  * k_tiles       -- one CTA per tile of consecutive rows of the SB / DB
//                     form or of a split (Sec. 3, Sec. 4).  When the plan says
//                     so, the tile first copies the x window it reuses into
//                     shared memory -- the "cache" the partition was sized
//                     for -- with one bulk copy for the contiguous run of home
//                     columns and a gather for the listed others.  Then each
//                     warp takes chunks of 32 length-sorted rows stored
//                     column-major: one lane per row, coalesced loads, one FMA
//                     chain per row.  No FP64 instruction runs with idle lanes
//                     for want of work and no shuffle reduction is needed,
//                     which matters on GB300 where FP64 issues at two FMAs per
//                     SM per clock.  Columns not staged are gathered through
//                     L1 / L2.  Chunk tiles reduce a slice of one long row
//                     into a partial sum.  256-thread CTAs (several per SM)
//                     or 1024-thread CTAs (one per SM, large windows).
//  * k_fixup       -- rows with several contributions (split rows shared by
//                     parts, chunked long rows) are summed from their partial
//                     sums in part order: y <- y + A^k x accumulated on the fly
//                     (Sec. 4), deterministically.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <utility>

#include "spmv_device.h"

namespace spmv {

constexpr int kThreads = 256;
constexpr int kMidThreads = 512;
constexpr int kWideThreads = 1024;

// Tuning knobs (compile-time):
//   SPMV_STREAM_HINT  how the matrix stream (values, indices) is loaded:
//                     0 = ld.global.cs (evict-first), 1 = ld.global.nc with
//                     L1::no_allocate (keeps L1 for x), 2 = ld.global.nc
//   SPMV_TILE_MINBLOCKS  minimum resident CTAs per SM asked of the compiler
//                     for the tiled kernel (register budget)
#ifndef SPMV_STREAM_HINT
#define SPMV_STREAM_HINT 0
#endif
#ifndef SPMV_TILE_MINBLOCKS
#define SPMV_TILE_MINBLOCKS 6
#endif
//   SPMV_WIDE_U       elements per lane in flight per batch in the wide CTAs
#ifndef SPMV_WIDE_U
#define SPMV_WIDE_U 8
#endif
//   SPMV_U256         elements per lane in flight per batch in the 256-thread
//                     CTAs (one right-hand side; a power of two up to 16)
#ifndef SPMV_U256
#define SPMV_U256 8
#endif
//   SPMV_PRED_PAD     1 = with FP64 values, a lane whose row has ended issues
//                     no load, gather or FMA for the chunk's remaining slots;
//                     0 (and FP32 / BF16 values) = every lane loads every
//                     slot up to the chunk's longest row and discards the
//                     padding's products
#ifndef SPMV_PRED_PAD
#define SPMV_PRED_PAD 1
#endif
//   SPMV_L1_PREF      1 = ask for the largest L1 carveout for the tile kernels
#ifndef SPMV_L1_PREF
#define SPMV_L1_PREF 0
#endif
// resident 256-thread tile CTAs per SM the register budget is sized for:
// fewer for many right-hand sides, which hold r accumulators per lane
constexpr int tile_ctas_per_sm(int r)
{
    return r <= 2 ? SPMV_TILE_MINBLOCKS : (r == 4 ? 4 : 3);
}

// loads of the matrix stream, read exactly once per SpMV
__device__ __forceinline__ double ld_stream(const double *p)
{
#if SPMV_STREAM_HINT == 1
    double v;
    asm volatile("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
#elif SPMV_STREAM_HINT == 2
    return __ldg(p);
#else
    return __ldcs(p);
#endif
}
__device__ __forceinline__ float ld_stream(const float *p)
{
#if SPMV_STREAM_HINT == 1
    float v;
    asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
#elif SPMV_STREAM_HINT == 2
    return __ldg(p);
#else
    return __ldcs(p);
#endif
}
__device__ __forceinline__ int32_t ld_stream(const int32_t *p)
{
#if SPMV_STREAM_HINT == 1
    int32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
#elif SPMV_STREAM_HINT == 2
    return __ldg(p);
#else
    return __ldcs(p);
#endif
}
__device__ __forceinline__ uint32_t ld_stream(const uint32_t *p)
{
#if SPMV_STREAM_HINT == 1
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
#elif SPMV_STREAM_HINT == 2
    return __ldg(p);
#else
    return __ldcs(p);
#endif
}
__device__ __forceinline__ uint16_t ld_stream(const uint16_t *p)
{
#if SPMV_STREAM_HINT == 1
    uint16_t v;
    asm volatile("ld.global.nc.L1::no_allocate.u16 %0, [%1];" : "=h"(v) : "l"(p));
    return v;
#elif SPMV_STREAM_HINT == 2
    return __ldg(p);
#else
    return __ldcs(p);
#endif
}

__device__ __forceinline__ double load_val(const double *p) { return ld_stream(p); }
__device__ __forceinline__ float load_val(const float *p) { return ld_stream(p); }
__device__ __forceinline__ float load_val(const __nv_bfloat16 *p)
{
    const uint16_t u = ld_stream(reinterpret_cast<const uint16_t *>(p));
    return __uint_as_float(static_cast<unsigned>(u) << 16);
}

template <int LANES, typename T>
__device__ __forceinline__ T group_sum(T v)
{
#pragma unroll
    for (int off = LANES / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off, LANES);
    return v;
}

// Sum s[] over the CTA; the result is valid in thread 0.  Every thread of the
// CTA must call it.
template <int R, typename T, int NT = kThreads>
__device__ __forceinline__ void block_sum(T (&s)[R])
{
    __shared__ T red[R][NT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < R; ++c) {
        T v = group_sum<32>(s[c]);
        if (lane == 0) red[c][warp] = v;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int c = 0; c < R; ++c) {
            T v = lane < NT / 32 ? red[c][lane] : T(0);
            s[c] = group_sum<32>(v);
        }
    }
}

// ------------------------------------------- bulk copies into shared memory --
// The staged run of a tile is one contiguous range of x_hat: one thread
// hands it to the TMA engine as a single bulk copy (cp.async.bulk) that
// signals an mbarrier, instead of every thread loading and storing entries.
// Waits are bounded: after kWaitLimit polls the CTA gives up, raises a flag
// the host reads (SPMV_E_TIMEOUT) and skips the tile.
constexpr uint32_t kWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// One arrival that expects `bytes` of asynchronous copies on the barrier.
__device__ __forceinline__ void mbar_expect(uint64_t *bar, uint32_t bytes)
{
    // order earlier generic-proxy reads of the destination (a previous tile)
    // before the async-proxy writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// A bulk copy global -> shared memory completing on the barrier (both
// addresses 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}
// Poll the barrier's phase at most `limit` times.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t phase, uint32_t limit)
{
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok) : "r"(smem_addr(bar)), "r"(phase) : "memory");
        if (ok) return true;
    }
    return false;
}

// The R entries of one column index in a row-major n x R block of vectors
// (global memory when GLOBAL, else shared memory): 16-byte loads where the
// R entries fill whole 16-byte words, one 8-byte load for two FP32 entries,
// scalar loads otherwise (R = 1).  x_hat and the staged window start on 16
// bytes and a column's block is R entries long, so every such load is
// aligned.
template <int R, typename XT, bool GLOBAL>
__device__ __forceinline__ void load_xrow(const XT *p, XT (&o)[R])
{
    constexpr int B = R * (int)sizeof(XT);
    if constexpr (B >= 16 && B % 16 == 0) {
        using V = typename std::conditional<sizeof(XT) == 8, double2, float4>::type;
        constexpr int per = 16 / (int)sizeof(XT);
#pragma unroll
        for (int c = 0; c < R; c += per) {
            const V *q = reinterpret_cast<const V *>(p + c);
            const V t = GLOBAL ? __ldg(q) : *q;
            const XT *e = reinterpret_cast<const XT *>(&t);
#pragma unroll
            for (int k = 0; k < per; ++k) o[c + k] = e[k];
        }
    } else if constexpr (B == 8 && sizeof(XT) == 4) {
        const float2 *q = reinterpret_cast<const float2 *>(p);
        const float2 t = GLOBAL ? __ldg(q) : *q;
        o[0] = t.x;
        o[1] = t.y;
    } else {
#pragma unroll
        for (int c = 0; c < R; ++c) o[c] = GLOBAL ? __ldg(p + c) : p[c];
    }
}

// ------------------------------------------------ plain CSR, vector per row --
template <int LANES, int R, typename VT, typename XT>
__global__ void __launch_bounds__(kThreads)
k_csr_vector(const int32_t m, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
             const VT *__restrict__ val, const XT *__restrict__ x, XT *__restrict__ y,
             const int32_t *__restrict__ long_rows, const int32_t n_long, const int32_t long_thresh)
{
    if ((int32_t)blockIdx.x < n_long) {
        // one whole CTA for a long row
        const int32_t row = long_rows[blockIdx.x];
        const int32_t p0 = rowptr[row], p1 = rowptr[row + 1];
        XT s[R];
#pragma unroll
        for (int c = 0; c < R; ++c) s[c] = XT(0);
        for (int32_t p = p0 + (int32_t)threadIdx.x; p < p1; p += kThreads) {
            const XT v = (XT)load_val(val + p);
            const int64_t xc = (int64_t)ld_stream(col + p) * R;
            XT xo[R];
            load_xrow<R, XT, true>(x + xc, xo);
#pragma unroll
            for (int c = 0; c < R; ++c) s[c] = fma(v, xo[c], s[c]);
        }
        block_sum<R>(s);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int c = 0; c < R; ++c) y[(int64_t)row * R + c] = s[c];
        }
        return;
    }
    const int64_t gt = (int64_t)(blockIdx.x - n_long) * kThreads + threadIdx.x;
    const int32_t row = (int32_t)(gt / LANES);
    const int lane = threadIdx.x & (LANES - 1);
    const bool valid = row < m;
    int32_t p0 = 0, p1 = 0;
    bool is_long = false;
    if (valid) {
        p0 = rowptr[row];
        p1 = rowptr[row + 1];
        is_long = (p1 - p0) > long_thresh;
        if (is_long) p1 = p0;      // reduced by its own CTA
    }
    XT s[R];
#pragma unroll
    for (int c = 0; c < R; ++c) s[c] = XT(0);
    for (int32_t p = p0 + lane; p < p1; p += LANES) {
        const XT v = (XT)load_val(val + p);
        const int64_t xc = (int64_t)ld_stream(col + p) * R;
        XT xo[R];
        load_xrow<R, XT, true>(x + xc, xo);
#pragma unroll
        for (int c = 0; c < R; ++c) s[c] = fma(v, xo[c], s[c]);
    }
#pragma unroll
    for (int c = 0; c < R; ++c) s[c] = group_sum<LANES>(s[c]);
    if (valid && !is_long && lane == 0) {
#pragma unroll
        for (int c = 0; c < R; ++c) y[(int64_t)row * R + c] = s[c];
    }
}

// ----------------------------------------------------------- tiled kernel --
template <typename VT, typename XT>
struct TileArgs {
    const Tile *tiles;
    const int32_t *chunk_off, *chunk_mix, *slot_dst, *slot_len;
    const VRow *vrows;
    const uint16_t *c16;
    const int32_t *c32;
    const VT *val;
    const int32_t *xlist;
    const XT *x;
    XT *y, *partial;
    // SM-affine schedule: tiles of queue q are qbeg[q] .. qbeg[q+1]-1
    const int32_t *qbeg;
    int32_t *qcount;        // nq claim counters, then one finished-CTA counter
    int32_t nq;
    int32_t *status;        // set to 1 when a bounded wait gives up
    uint32_t wait_limit;    // polls of the first wait on a tile's staging copy
};

// How one stored element finds its x entries.
enum : int {
    FX_GLOBAL = 0,   // col32 is an x_hat index: gathered through L1 / L2
    FX_MIXED = 1,    // col32 >= 0: staged entry; col32 < 0: x_hat[~col32].  Both
                     // loads are issued (the unused one reads entry 0) and one
                     // is selected, so a batch has no branch
    FX_SMEM32 = 2,   // col32 is a staged entry
    FX_SMEM16 = 3,   // col16 is a staged entry (narrow tiles)
    FX_DELTA = 4     // col16 holds column increments along the lane's row
                     // (DELTA tiles): the running column is the x_hat index
};

template <int FX, int R, typename XT>
__device__ __forceinline__ void fetch_x(int32_t ci, const XT *seg, const XT *__restrict__ x,
                                        XT (&o)[R])
{
    if constexpr (FX == FX_SMEM16 || FX == FX_SMEM32) {
        load_xrow<R, XT, false>(seg + ci * R, o);
    } else if constexpr (FX == FX_GLOBAL || FX == FX_DELTA) {
        load_xrow<R, XT, true>(x + (int64_t)ci * R, o);
    } else {
        const bool g = ci < 0;
        const int64_t gi = g ? (int64_t)(~ci) : 0;
        const int32_t si = g ? 0 : ci;
        XT a[R], b[R];
        load_xrow<R, XT, true>(x + gi * R, a);
        load_xrow<R, XT, false>(seg + si * R, b);
#pragma unroll
        for (int c = 0; c < R; ++c) o[c] = g ? a[c] : b[c];
    }
}

template <int FX>
__device__ __forceinline__ int32_t load_col(const int32_t *__restrict__ c32,
                                            const uint16_t *__restrict__ c16, int64_t e)
{
    if constexpr (FX == FX_SMEM16) return (int32_t)ld_stream(c16 + e);
    else return ld_stream(c32 + e);
}

// Element slots [k0, k0 + UB) of a chunk (k0 + UB <= the chunk's longest
// row, so every slot exists for the warp): element k of lane i is at
// off + 32 k + i.  All UB value / index loads are issued before the UB
// gathers, and all gathers before the FMAs, so UB gathers per lane are in
// flight together.  A lane whose row has ended issues no load and no gather
// for the slot (per-lane predicates, no branch): rows are sorted longest
// first, so the padding of a slot is its top lanes and whole sectors of the
// stream are never requested.  Padding slots hold index 0 all the same: the
// mixed path (two loads per slot) keeps every lane's loads and selects its
// sums, which fits the 256-thread register budget, and so do FP32 / BF16
// values (measured faster that way).
//
// FX_DELTA: cc is the lane's running column.  The increments of slots 2p
// and 2p + 1 sit side by side (chunk start + 64 p + 2 lane), one 32-bit load
// for both; UB >= 2 batches start on an even slot (the batches of a chunk
// are U, ..., 4, 2, 1 slots long, U even), and a batch of 1 is the odd last
// slot, stored plainly.  Padding increments are 0, so a finished lane's
// column stays on its last entry.
template <int FX, int UB, int R, typename VT, typename XT>
__device__ __forceinline__ void chunk_batch(int32_t k0, int64_t off, int32_t len,
                                            const VT *__restrict__ val,
                                            const int32_t *__restrict__ c32,
                                            const uint16_t *__restrict__ c16, const XT *seg,
                                            const XT *__restrict__ x, XT (&s)[R], int32_t &cc)
{
    // padding lanes skip their loads with FP64 values only: with FP32 /
    // BF16 values the predicated form timed 3-7% slower
    constexpr bool PRED = SPMV_PRED_PAD && FX != FX_MIXED && std::is_same<VT, double>::value;
    XT v[UB];
    int32_t ci[UB];
#pragma unroll
    for (int u = 0; u < UB; ++u) {
        const int64_t e = off + (int64_t)(k0 + u) * 32;
        v[u] = XT(0);
        ci[u] = 0;
        if (!PRED || k0 + u < len) {
            v[u] = (XT)load_val(val + e);
            if constexpr (FX != FX_DELTA) ci[u] = load_col<FX>(c32, c16, e);
        }
    }
    if constexpr (FX == FX_DELTA) {
        if constexpr (UB == 1) {
            if (!PRED || k0 < len) ci[0] = (int32_t)ld_stream(c16 + off + (int64_t)k0 * 32);
        } else {
            static_assert(UB % 2 == 0, "increment pairs");
            // off = chunk start + lane; the pair word of lane i is at
            // chunk start + 32 k + 2 i
            const uint32_t *pw = reinterpret_cast<const uint32_t *>(
                c16 + off + (threadIdx.x & 31) + (int64_t)k0 * 32);
#pragma unroll
            for (int j = 0; j < UB / 2; ++j) {
                uint32_t w = 0;       // a pair past the row's end adds 0
                if (!PRED || k0 + 2 * j < len) w = ld_stream(pw + 32 * j);
                ci[2 * j] = (int32_t)(w & 0xffffu);
                ci[2 * j + 1] = (int32_t)(w >> 16);
            }
        }
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            cc += ci[u];
            ci[u] = cc;
        }
    }
#pragma unroll
    for (int u = 0; u < UB; ++u) {
        const bool on = k0 + u < len;
        if constexpr (!PRED) {
            XT xo[R];
            fetch_x<FX, R, XT>(ci[u], seg, x, xo);
#pragma unroll
            for (int c = 0; c < R; ++c) {
                const XT f = fma(v[u], xo[c], s[c]);
                s[c] = on ? f : s[c];
            }
        } else if (on) {
            XT xo[R];
            fetch_x<FX, R, XT>(ci[u], seg, x, xo);
#pragma unroll
            for (int c = 0; c < R; ++c) s[c] = fma(v[u], xo[c], s[c]);
        }
    }
}

// Slots [kb, ke) of a chunk: full batches of U, then the remainder in
// batches of 4, 2 and 1 (ke is the same for the whole warp, so these
// branches do not diverge).  Exactly ke - kb FMAs per lane are issued: on
// GB300, which runs two FP64 FMAs per SM per clock, a padded batch would
// cost as much as a useful one.
template <int FX, int U, int R, typename VT, typename XT>
__device__ __forceinline__ void chunk_span(int32_t kb, int32_t ke, int64_t off, int32_t len,
                                           const VT *__restrict__ val,
                                           const int32_t *__restrict__ c32,
                                           const uint16_t *__restrict__ c16, const XT *seg,
                                           const XT *__restrict__ x, XT (&s)[R], int32_t &cc)
{
    static_assert(FX != FX_DELTA || U % 2 == 0, "increment pairs need even batches");
    int32_t k0 = kb;
    for (; k0 + U <= ke; k0 += U)
        chunk_batch<FX, U, R, VT, XT>(k0, off, len, val, c32, c16, seg, x, s, cc);
    if constexpr (U > 8) {
        if ((ke - k0) & 8) {
            chunk_batch<FX, 8, R, VT, XT>(k0, off, len, val, c32, c16, seg, x, s, cc);
            k0 += 8;
        }
    }
    if constexpr (U > 4) {
        if ((ke - k0) & 4) {
            chunk_batch<FX, 4, R, VT, XT>(k0, off, len, val, c32, c16, seg, x, s, cc);
            k0 += 4;
        }
    }
    if constexpr (U > 2) {
        if ((ke - k0) & 2) {
            chunk_batch<FX, 2, R, VT, XT>(k0, off, len, val, c32, c16, seg, x, s, cc);
            k0 += 2;
        }
    }
    if constexpr (U > 1) {
        if ((ke - k0) & 1)
            chunk_batch<FX, 1, R, VT, XT>(k0, off, len, val, c32, c16, seg, x, s, cc);
    } else {
        static_assert(FX != FX_DELTA, "increment pairs need even batches");
    }
}

// A row reduced by a whole warp: batches of U elements per lane (slots past
// the row's end read the row's first element and are discarded), then a
// shuffle sum.
template <int FX, int U, int R, typename VT, typename XT>
__device__ __forceinline__ void warp_row(const VRow &row, const VT *__restrict__ val,
                                         const int32_t *__restrict__ c32,
                                         const uint16_t *__restrict__ c16, const XT *seg,
                                         const XT *__restrict__ x, XT (&s)[R])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < R; ++c) s[c] = XT(0);
    for (int32_t k0 = 0; k0 < row.len; k0 += 32 * U) {
        XT v[U];
        int32_t ci[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int32_t k = k0 + u * 32 + lane;
            const int64_t e = row.e0 + (k < row.len ? k : 0);
            v[u] = (XT)load_val(val + e);
            ci[u] = load_col<FX>(c32, c16, e);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            XT xo[R];
            fetch_x<FX, R, XT>(ci[u], seg, x, xo);
            const bool on = k0 + u * 32 + lane < row.len;
#pragma unroll
            for (int c = 0; c < R; ++c) {
                const XT f = fma(v[u], xo[c], s[c]);
                s[c] = on ? f : s[c];
            }
        }
    }
#pragma unroll
    for (int c = 0; c < R; ++c) s[c] = group_sum<32>(s[c]);
}

// The rows of a tile after staging, as a sequence of items: the warp rows
// (longest first), then the chunks of 32 rows (longest first).  Warp w
// starts with item w; with `claim` (a shared-memory counter at zero) each
// warp then claims its next item from the counter as it starts the current
// one, so the warps of the CTA finish together however the row lengths
// vary (longest-first claiming); without it, warp w takes items w + k NT/32.
// A chunk's metadata (row lengths, destinations, offset, mixed prefix) is
// loaded when the chunk is claimed, one item ahead, so a chunk costs two
// dependent trips to memory (its stream, then its gathers).
struct ChunkMeta {
    int32_t len, dst, off, mix;
};

template <int KIND, int R, typename VT, typename XT, int NT>
__device__ __forceinline__ void rows_work(const Tile &t, const TileArgs<VT, XT> &A,
                                          const XT *seg, int32_t *claim)
{
    const int32_t *__restrict__ chunk_off = A.chunk_off;
    const int32_t *__restrict__ chunk_mix = A.chunk_mix;
    const int32_t *__restrict__ slot_dst = A.slot_dst;
    const int32_t *__restrict__ slot_len = A.slot_len;
    const VRow *__restrict__ vrows = A.vrows;
    const uint16_t *__restrict__ c16 = A.c16;
    const int32_t *__restrict__ c32 = A.c32;
    const VT *__restrict__ val = A.val;
    const XT *__restrict__ x = A.x;
    XT *__restrict__ y = A.y;
    XT *__restrict__ partial = A.partial;
    constexpr int NW = NT / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    auto store = [&](int32_t d, const XT (&s)[R]) {
        if (d >= 0) {
#pragma unroll
            for (int c = 0; c < R; ++c) y[(int64_t)d * R + c] = s[c];
        } else if (d <= -2) {
            const int64_t ps = (int64_t)(-d - 2) * R;
#pragma unroll
            for (int c = 0; c < R; ++c) partial[ps + c] = s[c];
        }
    };
    // elements per lane in flight per batch (the wider CTAs have the larger
    // register budget)
    constexpr int U = (R == 1 ? (NT == kThreads ? SPMV_U256 : SPMV_WIDE_U) : (R == 2 ? 4 : 2));
    constexpr int FXW = KIND == TILE_NARROW ? FX_SMEM16 : (KIND == TILE_MIXED ? FX_MIXED : FX_GLOBAL);
    int32_t cc = 0;

    const int32_t nv = t.nvrows, nitems = t.nvrows + t.nchunks;
    auto meta = [&](int32_t item) {
        ChunkMeta mt{0, -1, 0, 0};
        if (item >= nv && item < nitems) {
            const int32_t ch = t.chunk0 + (item - nv);
            mt.len = __ldg(slot_len + ch * 32 + lane);
            mt.dst = __ldg(slot_dst + ch * 32 + lane);
            mt.off = __ldg(chunk_off + ch);
            if (KIND == TILE_MIXED || KIND == TILE_DELTA) mt.mix = __ldg(chunk_mix + ch);
        }
        return mt;
    };
    int32_t cur = warp;
    ChunkMeta mc = meta(cur);
    while (cur < nitems) {
        int32_t nxt;
        if (claim) {
            int32_t v = 0;
            if (lane == 0) v = atomicAdd(claim, 1);
            nxt = __shfl_sync(0xffffffffu, v, 0) + NW;
        } else {
            nxt = cur + NW;
        }
        const ChunkMeta mn = meta(nxt);
        XT s[R];
        if (cur < nv) {
            // a row too long for one lane: the whole warp
            const VRow row = vrows[t.vrow0 + cur];
            warp_row<FXW, U, R, VT, XT>(row, val, c32, c16, seg, x, s);
            if (lane == 0) store(row.dst, s);
        } else {
            // a chunk of 32 rows, one lane per row
            const int64_t off = (int64_t)mc.off + lane;
            const int32_t L = __shfl_sync(0xffffffffu, mc.len, 0);   // lane 0 is longest
#pragma unroll
            for (int c = 0; c < R; ++c) s[c] = XT(0);
            if constexpr (KIND == TILE_MIXED) {
                // rows store their gathered elements first: slots [0, G) may
                // gather, slots [G, L) read shared memory only
                chunk_span<FX_MIXED, U, R, VT, XT>(0, mc.mix, off, mc.len, val, c32, c16, seg, x, s,
                                                   cc);
                chunk_span<FX_SMEM32, U, R, VT, XT>(mc.mix, L, off, mc.len, val, c32, c16, seg, x,
                                                    s, cc);
            } else if constexpr (KIND == TILE_NARROW) {
                chunk_span<FX_SMEM16, U, R, VT, XT>(0, L, off, mc.len, val, c32, c16, seg, x, s,
                                                    cc);
            } else if constexpr (KIND == TILE_DELTA) {
                // chunk_mix: the base column (same for the whole warp), or
                // -1 for a chunk of 32-bit indices
                if (mc.mix >= 0) {
                    cc = mc.mix;
                    chunk_span<FX_DELTA, U, R, VT, XT>(0, L, off, mc.len, val, c32, c16, seg, x,
                                                       s, cc);
                } else {
                    chunk_span<FX_GLOBAL, U, R, VT, XT>(0, L, off, mc.len, val, c32, c16, seg, x,
                                                        s, cc);
                }
            } else {
                chunk_span<FX_GLOBAL, U, R, VT, XT>(0, L, off, mc.len, val, c32, c16, seg, x, s,
                                                    cc);
            }
            store(mc.dst, s);
        }
        cur = nxt;
        mc = mn;
    }
}

// Returns false when the staging copy did not complete within the wait limit
// (the tile is then skipped and A.status raised).  `bar` is the CTA's
// mbarrier, `phase` its current parity.
template <int R, typename VT, typename XT, int NT = kThreads>
__device__ __forceinline__ bool tile_work(const Tile &t, const TileArgs<VT, XT> &A,
                                          uint64_t *bar, uint32_t &phase,
                                          int32_t *claim = nullptr)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    XT *seg = reinterpret_cast<XT *>(smem_raw);
    const VT *__restrict__ val = A.val;
    const int32_t *__restrict__ c32 = A.c32;
    const int32_t *__restrict__ xlist = A.xlist;
    const XT *__restrict__ x = A.x;
    XT *__restrict__ partial = A.partial;

    if (t.kind == TILE_CHUNK) {
        XT s[R];
#pragma unroll
        for (int c = 0; c < R; ++c) s[c] = XT(0);
        for (int32_t e = t.e0 + (int32_t)threadIdx.x; e < t.e1; e += NT) {
            const XT v = (XT)load_val(val + e);
            const int64_t xc = (int64_t)ld_stream(c32 + e) * R;
            XT xo[R];
            load_xrow<R, XT, true>(x + xc, xo);
#pragma unroll
            for (int c = 0; c < R; ++c) s[c] = fma(v, xo[c], s[c]);
        }
        block_sum<R, XT, NT>(s);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int c = 0; c < R; ++c) partial[(int64_t)t.slot * R + c] = s[c];
        }
        return true;
    }

    const int kind = t.kind;
    if (kind == TILE_NARROW || kind == TILE_MIXED) {
        // stage the window: the 16-byte bodies of the two runs by bulk copy
        // (one elected thread, one mbarrier for both), their tails and the
        // gathered list by the CTA's threads
        const int32_t n1 = t.runlen * R, n2 = t.run2len * R, at2 = t.run2_at * R;
        const uint32_t body1 = (uint32_t)(n1 * (int32_t)sizeof(XT)) & ~15u;
        const uint32_t body2 = (uint32_t)(n2 * (int32_t)sizeof(XT)) & ~15u;
        const bool copy = body1 + body2 > 0;
        if (threadIdx.x == 0 && copy) {
            mbar_expect(bar, body1 + body2);
            if (body1) bulk_g2s(seg, x + (int64_t)t.run0 * R, body1, bar);
            if (body2) bulk_g2s(seg + at2, x + (int64_t)t.run2_0 * R, body2, bar);
        }
        for (int32_t i = (int32_t)(body1 / sizeof(XT)) + threadIdx.x; i < n1; i += NT)
            seg[i] = __ldg(x + (int64_t)t.run0 * R + i);
        for (int32_t i = (int32_t)(body2 / sizeof(XT)) + threadIdx.x; i < n2; i += NT)
            seg[at2 + i] = __ldg(x + (int64_t)t.run2_0 * R + i);
        // list: batches of entries per thread, every index load issued
        // before the gathers that depend on them
        const int32_t lat = at2 + n2;
        constexpr int LB = R == 1 ? 8 : (R == 2 ? 4 : (R == 4 ? 2 : 1));
        for (int32_t i0 = 0; i0 < t.listlen; i0 += LB * NT) {
            int32_t src[LB];
#pragma unroll
            for (int u = 0; u < LB; ++u) {
                const int32_t i = i0 + u * NT + (int32_t)threadIdx.x;
                src[u] = i < t.listlen ? __ldg(xlist + t.list0 + i) : -1;
            }
            XT v[LB][R];
#pragma unroll
            for (int u = 0; u < LB; ++u)
#pragma unroll
                for (int c = 0; c < R; ++c)
                    v[u][c] = src[u] >= 0 ? __ldg(x + (int64_t)src[u] * R + c) : XT(0);
#pragma unroll
            for (int u = 0; u < LB; ++u) {
                const int32_t i = i0 + u * NT + (int32_t)threadIdx.x;
                if (i < t.listlen) {
#pragma unroll
                    for (int c = 0; c < R; ++c) seg[lat + i * R + c] = v[u][c];
                }
            }
        }
        bool ok = true;
        if (copy) ok = mbar_wait(bar, phase, A.wait_limit);
        ok = __syncthreads_and(ok);
        if (copy) phase ^= 1u;
        if (!ok) {
            // the copy is still owed to this barrier: wait once more (bounded)
            // before the CTA leaves, then report
            if (threadIdx.x == 0) {
                atomicExch(A.status, 1);
                mbar_wait(bar, phase ^ 1u, kWaitLimit);
            }
            return false;
        }
    }

    switch (kind) {
    case TILE_NARROW: rows_work<TILE_NARROW, R, VT, XT, NT>(t, A, seg, claim); break;
    case TILE_MIXED: rows_work<TILE_MIXED, R, VT, XT, NT>(t, A, seg, claim); break;
    case TILE_DELTA: rows_work<TILE_DELTA, R, VT, XT, NT>(t, A, seg, claim); break;
    default: rows_work<TILE_GLOBAL, R, VT, XT, NT>(t, A, seg, claim); break;
    }
    return true;
}

// One CTA per tile, in tile order.  NT = kThreads: several CTAs per SM;
// NT = kMidThreads: two CTAs per SM, each with about half of the SM's shared
// memory for its window; NT = kWideThreads: one wide CTA per SM with a large
// staging window.
template <int R, typename VT, typename XT, int NT>
__global__ void __launch_bounds__(NT, NT == kThreads ? tile_ctas_per_sm(R)
                                                     : (NT == kMidThreads ? 2 : 1))
k_tiles(const TileArgs<VT, XT> A)
{
    __shared__ __align__(8) uint64_t bar;
    __shared__ int32_t claim;          // next item of the tile to hand out
    if (threadIdx.x == 0) {
        mbar_init(&bar);
        claim = 0;
    }
    __syncthreads();
    uint32_t phase = 0;
    const Tile t = A.tiles[blockIdx.x];
    tile_work<R, VT, XT, NT>(t, A, &bar, phase, &claim);
}

// Persistent CTAs, one per resident slot, claiming tiles in tile order from
// one counter.  The first tile of CTA b is tile b; each further claim is an
// atomic issued at the start of the current tile, so its latency hides
// behind the tile's work.  No CTA waits for another.  The last CTA out resets
// the counters for the next launch.
template <int R, typename VT, typename XT>
__global__ void __launch_bounds__(kThreads, SPMV_TILE_MINBLOCKS)
k_tiles_persist(const TileArgs<VT, XT> A, const int32_t n_tiles, int32_t *ctr)
{
    __shared__ int32_t claim;
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar);
    __syncthreads();
    uint32_t phase = 0;
    int32_t cur = (int32_t)blockIdx.x;
    while (cur < n_tiles) {
        int32_t nxt = 0;
        if (threadIdx.x == 0) nxt = (int32_t)gridDim.x + atomicAdd(ctr, 1);
        if (!tile_work<R, VT, XT>(A.tiles[cur], A, &bar, phase)) break;
        __syncthreads();                // every warp is done with this tile
        if (threadIdx.x == 0) claim = nxt;
        __syncthreads();
        cur = claim;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const int32_t done = atomicAdd(ctr + 1, 1);
        if (done == (int32_t)(gridDim.x - 1)) {
            ctr[0] = 0;
            ctr[1] = 0;
            __threadfence();
        }
    }
}

__device__ __forceinline__ uint32_t sm_id()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t sm_id_count()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%nsmid;" : "=r"(r));
    return r;
}

// Persistent CTAs with an SM-affine schedule.  The plan cuts the tile
// sequence (tiles of a part are consecutive) into one queue per SM; a CTA
// first drains the queue of the SM it runs on, so every CTA on that SM works
// on the same part and the part's x window stays in the SM's L1 -- the
// per-SM cache the partition was sized for.  Then it helps the other queues:
// the whole CTA reads every queue's counter at once and claims from the
// queue with the most tiles left, so all tiles are done however the CTAs were
// placed, at one round trip per steal.  Claims are atomic counters (no
// waiting); the last CTA to finish resets them for the next call.
template <int R, typename VT, typename XT>
__global__ void __launch_bounds__(kThreads, SPMV_TILE_MINBLOCKS)
k_tiles_affine(const TileArgs<VT, XT> A)
{
    __shared__ int32_t claim, claim_q;
    __shared__ int32_t best_left[kThreads / 32], best_q[kThreads / 32];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar);
    uint32_t phase = 0;
    const int32_t nq = A.nq;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t q = (int32_t)(((uint64_t)sm_id() * (uint64_t)nq) / max(1u, sm_id_count()));
    for (;;) {
        __syncthreads();                // the previous tile is done with shared memory
        if (threadIdx.x == 0) {
            const int32_t b = __ldg(A.qbeg + q), len = __ldg(A.qbeg + q + 1) - b;
            const int32_t i = atomicAdd(A.qcount + q, 1);
            claim = i < len ? b + i : -1;
        }
        __syncthreads();
        const int32_t ti = claim;
        if (ti >= 0) {
            if (!tile_work<R, VT, XT>(A.tiles[ti], A, &bar, phase)) break;
            continue;
        }
        // this queue is drained: find the one with the most unclaimed tiles
        int32_t left = 0, lq = -1;
        for (int32_t k = threadIdx.x; k < nq; k += kThreads) {
            const int32_t len = __ldg(A.qbeg + k + 1) - __ldg(A.qbeg + k);
            const int32_t l = len - *((volatile int32_t *)(A.qcount + k));
            if (l > left) {
                left = l;
                lq = k;
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const int32_t l2 = __shfl_xor_sync(0xffffffffu, left, off);
            const int32_t q2 = __shfl_xor_sync(0xffffffffu, lq, off);
            if (l2 > left || (l2 == left && q2 > lq)) {
                left = l2;
                lq = q2;
            }
        }
        if (lane == 0) {
            best_left[warp] = left;
            best_q[warp] = lq;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t bl = 0, bq = -1;
            for (int w = 0; w < kThreads / 32; ++w)
                if (best_left[w] > bl) {
                    bl = best_left[w];
                    bq = best_q[w];
                }
            claim_q = bq;
        }
        __syncthreads();
        if (claim_q < 0) break;         // every queue is drained
        q = claim_q;
    }
    // the last CTA out resets the claim counters for the next launch
    if (threadIdx.x == 0) {
        __threadfence();
        const int32_t done = atomicAdd(A.qcount + nq, 1);
        if (done == (int32_t)(gridDim.x - 1)) {
            for (int32_t k = 0; k < nq; ++k) A.qcount[k] = 0;
            A.qcount[nq] = 0;
            __threadfence();
        }
    }
}

// ------------------------------------------------------------------ fix-up --
template <int R, typename XT>
__global__ void __launch_bounds__(kThreads)
k_fixup(const Fixup *__restrict__ f, const int32_t nf, const XT *__restrict__ partial,
        XT *__restrict__ y)
{
    const int32_t i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= nf) return;
    const Fixup e = f[i];
#pragma unroll
    for (int c = 0; c < R; ++c) {
        XT s = XT(0);
        for (int32_t t = 0; t < e.count; ++t) s += partial[(int64_t)(e.slot0 + t) * R + c];
        y[(int64_t)e.row * R + c] = s;
    }
}

// ---------------------------------------------------------------- launcher --
// Raise the dynamic shared memory limit of a kernel once per device (the
// kernels also hold a little static shared memory, so the opt-in is needed
// below 48 KB of dynamic memory too).
template <class Kern>
inline cudaError_t ensure_smem(Kern k, int bytes)
{
#if SPMV_L1_PREF
    {
        // prefer the largest L1 (a hint; launches that need more shared
        // memory still get it)
        static std::mutex mu1;
        static std::map<std::pair<const void *, int>, bool> pref;
        int dev1 = 0;
        cudaError_t e1 = cudaGetDevice(&dev1);
        if (e1 != cudaSuccess) return e1;
        std::lock_guard<std::mutex> g1(mu1);
        const auto key1 = std::make_pair(reinterpret_cast<const void *>(k), dev1);
        if (!pref.count(key1)) {
            e1 = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
            if (e1 != cudaSuccess) return e1;
            pref[key1] = true;
        }
    }
#endif
    if (bytes <= 0) return cudaSuccess;
    // one cache per kernel instance (the template is shared by every kernel
    // with the same signature, so the key is the kernel's address)
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const auto key = std::make_pair(reinterpret_cast<const void *>(k), dev);
    std::lock_guard<std::mutex> g(mu);
    auto it = done.find(key);
    if (it != done.end() && it->second >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done[key] = bytes;
    return e;
}

// CTAs of a kernel resident per SM at a given dynamic shared memory size,
// cached per (kernel, device, size).
template <class Kern>
inline cudaError_t resident_ctas(Kern k, int smem, int *out)
{
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, int>, int> cache;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const auto key = std::make_tuple(reinterpret_cast<const void *>(k), dev, smem);
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kThreads, smem);
    if (e != cudaSuccess) return e;
    cache[key] = n;
    *out = n;
    return cudaSuccess;
}

template <int LANES, int R, typename VT, typename XT>
cudaError_t launch_k1(const DevPlan &P, const XT *x, XT *y, cudaStream_t s)
{
    constexpr int rows_per_block = kThreads / LANES;
    const int64_t nb = ((int64_t)P.m + rows_per_block - 1) / rows_per_block + P.n_long;
    if (nb > 0)
        k_csr_vector<LANES, R, VT, XT><<<(unsigned)nb, kThreads, 0, s>>>(
            P.m, P.rowptr, P.col32, static_cast<const VT *>(P.val), x, y, P.long_rows, P.n_long,
            P.long_thresh);
    return cudaGetLastError();
}

template <int R, typename VT, typename XT>
cudaError_t launch_tiled(const DevPlan &P0, const XT *x, XT *y, cudaStream_t s)
{
#ifdef SPMV_FORCE_SMEM
    DevPlan P = P0;     // experiment: reserve shared memory the tiles do not use
    P.smem_bytes = std::max(P.smem_bytes, (int32_t)SPMV_FORCE_SMEM);
#else
    const DevPlan &P = P0;
#endif
    if (P.n_tiles > 0) {
        TileArgs<VT, XT> A;
        A.tiles = P.tiles;
        A.chunk_off = P.chunk_off;
        A.chunk_mix = P.chunk_mix;
        A.slot_dst = P.slot_dst;
        A.slot_len = P.slot_len;
        A.vrows = P.vrows;
        A.c16 = P.col16;
        A.c32 = P.col32;
        A.val = static_cast<const VT *>(P.val);
        A.xlist = P.xlist;
        A.x = x;
        A.y = y;
        A.partial = static_cast<XT *>(P.partial);
        A.qbeg = P.qbeg;
        A.qcount = P.qcount;
        A.nq = P.nq;
        A.status = P.status;
        A.wait_limit = P.wait_limit;
        cudaError_t e;
        if (P.nq > 0) {
            auto kern = k_tiles_affine<R, VT, XT>;
            e = ensure_smem(kern, P.smem_bytes);
            if (e != cudaSuccess) return e;
            int per_sm = 0;
            e = resident_ctas(kern, P.smem_bytes, &per_sm);
            if (e != cudaSuccess) return e;
            const int64_t grid = std::min<int64_t>((int64_t)P.nq * std::max(per_sm, 1),
                                                   (int64_t)P.n_tiles);
            kern<<<(unsigned)grid, kThreads, P.smem_bytes, s>>>(A);
        } else if (P.ctr != nullptr) {
            auto kern = k_tiles_persist<R, VT, XT>;
            e = ensure_smem(kern, P.smem_bytes);
            if (e != cudaSuccess) return e;
            int per_sm = 0;
            e = resident_ctas(kern, P.smem_bytes, &per_sm);
            if (e != cudaSuccess) return e;
            const int64_t grid = std::min<int64_t>((int64_t)P.n_sm * std::max(per_sm, 1),
                                                   (int64_t)P.n_tiles);
            kern<<<(unsigned)grid, kThreads, P.smem_bytes, s>>>(A, P.n_tiles, P.ctr);
        } else if (P.cta_threads == kWideThreads) {
            auto kern = k_tiles<R, VT, XT, kWideThreads>;
            e = ensure_smem(kern, P.smem_bytes);
            if (e != cudaSuccess) return e;
            kern<<<(unsigned)P.n_tiles, kWideThreads, P.smem_bytes, s>>>(A);
        } else if (P.cta_threads == kMidThreads) {
            auto kern = k_tiles<R, VT, XT, kMidThreads>;
            e = ensure_smem(kern, P.smem_bytes);
            if (e != cudaSuccess) return e;
            kern<<<(unsigned)P.n_tiles, kMidThreads, P.smem_bytes, s>>>(A);
        } else {
            auto kern = k_tiles<R, VT, XT, kThreads>;
            e = ensure_smem(kern, P.smem_bytes);
            if (e != cudaSuccess) return e;
            kern<<<(unsigned)P.n_tiles, kThreads, P.smem_bytes, s>>>(A);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (P.n_fixups > 0) {
        k_fixup<R, XT><<<(unsigned)((P.n_fixups + kThreads - 1) / kThreads), kThreads, 0, s>>>(
            P.fixups, P.n_fixups, static_cast<const XT *>(P.partial), y);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

template <int R, typename VT, typename XT>
cudaError_t launch_r(const DevPlan &P, const XT *x, XT *y, cudaStream_t s)
{
    if (!P.use_k1) return launch_tiled<R, VT, XT>(P, x, y, s);
    switch (P.lanes) {
    case 1: return launch_k1<1, R, VT, XT>(P, x, y, s);
    case 2: return launch_k1<2, R, VT, XT>(P, x, y, s);
    case 4: return launch_k1<4, R, VT, XT>(P, x, y, s);
    case 8: return launch_k1<8, R, VT, XT>(P, x, y, s);
    case 16: return launch_k1<16, R, VT, XT>(P, x, y, s);
    case 32: return launch_k1<32, R, VT, XT>(P, x, y, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename VT, typename XT>
cudaError_t launch_exec(const DevPlan &P, const void *xv, void *yv, cudaStream_t s)
{
    const XT *x = static_cast<const XT *>(xv);
    XT *y = static_cast<XT *>(yv);
    if (P.m == 0) return cudaSuccess;
    switch (P.nrhs) {
    case 1: return launch_r<1, VT, XT>(P, x, y, s);
    case 2: return launch_r<2, VT, XT>(P, x, y, s);
    case 4: return launch_r<4, VT, XT>(P, x, y, s);
    case 8: return launch_r<8, VT, XT>(P, x, y, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace spmv
