// SpMV kernels for sm_103a.  SpMV is a gather-and-reduce with about 0.17
// flop per byte in FP64, so these kernels are built around the memory system,
// not the tensor cores:
//
//  * k_csr_vector  -- plain natural-order CSR (Sec. 2.1): LANES threads per row,
//                     coalesced streaming of values and column indices
//                     (evict-first), x gathered through the read-only path,
//                     warp-shuffle reduction; rows longer than a threshold get
//                     a whole CTA each.  This is the baseline.
//  * k_tiles       -- one CTA per tile of a part of the SB / DB form or of a
//                     split (Sec. 3, Sec. 4).  The tile first copies the x
//                     entries it reuses into shared memory -- the "cache" the
//                     partition was sized for -- then each warp takes chunks of
//                     32 length-sorted rows stored column-major: one lane per
//                     row, coalesced loads, one FMA chain per row.  No FP64
//                     instruction runs with idle lanes for want of work and no
//                     shuffle reduction is needed, which matters on GB300 where
//                     FP64 issues at two FMAs per SM per clock.  Columns used
//                     once by the tile are gathered from L2 directly.  Chunk
//                     tiles reduce a slice of one long row into a partial sum.
//  * k_fixup       -- rows with several contributions (split rows shared by
//                     parts, chunked long rows) are summed from their partial
//                     sums in part order: y <- y + A^k x accumulated on the fly
//                     (Sec. 4), deterministically.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>

#include "spmv_device.h"

namespace spmv {

constexpr int kThreads = 256;

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
template <int R, typename T>
__device__ __forceinline__ void block_sum(T (&s)[R])
{
    __shared__ T red[R][kThreads / 32];
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
            T v = lane < kThreads / 32 ? red[c][lane] : T(0);
            s[c] = group_sum<32>(v);
        }
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
#pragma unroll
            for (int c = 0; c < R; ++c) s[c] = fma(v, __ldg(x + xc + c), s[c]);
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
#pragma unroll
        for (int c = 0; c < R; ++c) s[c] = fma(v, __ldg(x + xc + c), s[c]);
    }
#pragma unroll
    for (int c = 0; c < R; ++c) s[c] = group_sum<LANES>(s[c]);
    if (valid && !is_long && lane == 0) {
#pragma unroll
        for (int c = 0; c < R; ++c) y[(int64_t)row * R + c] = s[c];
    }
}

// ----------------------------------------------------------- tiled kernel --
// One CTA per tile.  After staging, warp w takes chunks w, w+8, ...; lane i
// owns row i of the chunk and runs one FMA chain over its row: element k of
// the chunk's rows sits at chunk_off + 32 k + i, so every load is coalesced
// and every FP64 FMA runs with the lanes of all rows still going.
template <int R, typename VT, typename XT>
__global__ void __launch_bounds__(kThreads, SPMV_TILE_MINBLOCKS)
k_tiles(const Tile *__restrict__ tiles, const int32_t *__restrict__ chunk_off,
        const int32_t *__restrict__ slot_dst, const int32_t *__restrict__ slot_len,
        const VRow *__restrict__ vrows, const uint16_t *__restrict__ c16,
        const int32_t *__restrict__ c32,
        const VT *__restrict__ val, const int32_t *__restrict__ xlist,
        const XT *__restrict__ x, XT *__restrict__ y, XT *__restrict__ partial)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    XT *seg = reinterpret_cast<XT *>(smem_raw);
    const Tile t = tiles[blockIdx.x];

    if (t.kind == TILE_CHUNK) {
        XT s[R];
#pragma unroll
        for (int c = 0; c < R; ++c) s[c] = XT(0);
        for (int32_t e = t.e0 + (int32_t)threadIdx.x; e < t.e1; e += kThreads) {
            const XT v = (XT)load_val(val + e);
            const int64_t xc = (int64_t)ld_stream(c32 + e) * R;
#pragma unroll
            for (int c = 0; c < R; ++c) s[c] = fma(v, __ldg(x + xc + c), s[c]);
        }
        block_sum<R>(s);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int c = 0; c < R; ++c) partial[(int64_t)t.slot * R + c] = s[c];
        }
        return;
    }

    const int kind = t.kind;
    if (kind != TILE_GLOBAL) {
        // stage the reused x entries: the contiguous run, then the list
        for (int32_t i = threadIdx.x; i < t.runlen; i += kThreads) {
            const int64_t src = (int64_t)(t.run0 + i) * R;
#pragma unroll
            for (int c = 0; c < R; ++c) seg[i * R + c] = __ldg(x + src + c);
        }
        for (int32_t i = threadIdx.x; i < t.listlen; i += kThreads) {
            const int64_t src = (int64_t)__ldg(xlist + t.list0 + i) * R;
            const int32_t d = (t.runlen + i) * R;
#pragma unroll
            for (int c = 0; c < R; ++c) seg[d + c] = __ldg(x + src + c);
        }
        __syncthreads();
    }

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the x entry of element e for right-hand side c
    auto xat = [&](int32_t ci, int c) -> XT {
        if (kind == TILE_GLOBAL) return __ldg(x + (int64_t)ci * R + c);
        if (ci >= 0) return seg[ci * R + c];
        return __ldg(x + (int64_t)(~ci) * R + c);
    };
    auto colat = [&](int64_t e) -> int32_t {
        return kind == TILE_NARROW ? (int32_t)ld_stream(c16 + e) : ld_stream(c32 + e);
    };
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
    constexpr int U = R == 1 ? 8 : (R == 2 ? 4 : 2);

    // rows too long for one lane: a warp each, batches of U loads per lane
    for (int32_t vr = t.vrow0 + warp; vr < t.vrow0 + t.nvrows; vr += kThreads / 32) {
        const VRow row = vrows[vr];
        XT s[R];
#pragma unroll
        for (int c = 0; c < R; ++c) s[c] = XT(0);
        for (int32_t k0 = 0; k0 < row.len; k0 += 32 * U) {
            XT v[U];
            int32_t ci[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int32_t k = k0 + u * 32 + lane;
                const bool on = k < row.len;
                v[u] = on ? (XT)load_val(val + row.e0 + k) : XT(0);
                ci[u] = on ? colat(row.e0 + k) : 0;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (k0 + u * 32 + lane < row.len) {
#pragma unroll
                    for (int c = 0; c < R; ++c) s[c] = fma(v[u], xat(ci[u], c), s[c]);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < R; ++c) s[c] = group_sum<32>(s[c]);
        if (lane == 0) store(row.dst, s);
    }

    // chunks of 32 rows, one lane per row, batches of U elements per lane
    for (int32_t ch = t.chunk0 + warp; ch < t.chunk0 + t.nchunks; ch += kThreads / 32) {
        const int32_t slot = ch * 32 + lane;
        const int32_t len = __ldg(slot_len + slot);
        const int32_t L = __shfl_sync(0xffffffffu, len, 0);   // rows sorted: lane 0 is longest
        const int64_t off = __ldg(chunk_off + ch) + lane;
        XT s[R];
#pragma unroll
        for (int c = 0; c < R; ++c) s[c] = XT(0);
        for (int32_t k0 = 0; k0 < L; k0 += U) {
            XT v[U];
            int32_t ci[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool on = k0 + u < len;
                const int64_t e = off + (int64_t)(k0 + u) * 32;
                v[u] = on ? (XT)load_val(val + e) : XT(0);
                ci[u] = on ? colat(e) : 0;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (k0 + u < len) {
#pragma unroll
                    for (int c = 0; c < R; ++c) s[c] = fma(v[u], xat(ci[u], c), s[c]);
                }
            }
        }
        store(__ldg(slot_dst + slot), s);
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
cudaError_t launch_tiled(const DevPlan &P, const XT *x, XT *y, cudaStream_t s)
{
    if (P.n_tiles > 0) {
        auto kern = k_tiles<R, VT, XT>;
        cudaError_t e = ensure_smem(kern, P.smem_bytes);
        if (e != cudaSuccess) return e;
        kern<<<(unsigned)P.n_tiles, kThreads, P.smem_bytes, s>>>(
            P.tiles, P.chunk_off, P.slot_dst, P.slot_len, P.vrows, P.col16, P.col32,
            static_cast<const VT *>(P.val), P.xlist, x, y, static_cast<XT *>(P.partial));
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
