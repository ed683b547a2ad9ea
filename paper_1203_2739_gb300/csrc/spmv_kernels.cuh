// SpMV kernels for sm_103a.  SpMV is a gather-and-reduce with about 0.17
// flop per byte in FP64, so these kernels are built around the memory system,
// not the tensor cores:
//
//  * k_csr_vector  -- plain natural-order CSR (Sec. 2.1): LANES threads per row,
//                     coalesced streaming of values and column indices
//                     (evict-first), x gathered through the read-only path,
//                     warp-shuffle reduction; rows longer than a threshold get
//                     a whole CTA each.
//  * k_tiles       -- one CTA per tile of a part of the SB / DB form or of a
//                     split (Sec. 3, Sec. 4).  A staged tile first copies its x
//                     working set (a contiguous run of x plus an index list)
//                     into shared memory, which is the "cache" the partition
//                     was sized for, then reduces its rows against shared
//                     memory with 16-bit local column indices.  Global tiles
//                     (the DB row border R_B, tiles with no reuse) gather x
//                     from L2.  Chunk tiles reduce a slice of one long row into
//                     a partial sum.
//  * k_fixup       -- rows with several contributions (split rows shared by
//                     parts, chunked long rows) are summed from their partial
//                     sums in part order: y <- y + A^k x accumulated on the fly
//                     (Sec. 4), deterministically.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "spmv_device.h"

namespace spmv {

constexpr int kThreads = 256;

// value load, streamed with evict-first so the matrix does not push x out of L2
__device__ __forceinline__ double load_val(const double *p) { return __ldcs(p); }
__device__ __forceinline__ float load_val(const float *p) { return __ldcs(p); }
__device__ __forceinline__ float load_val(const __nv_bfloat16 *p)
{
    unsigned short u = __ldcs(reinterpret_cast<const unsigned short *>(p));
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
            const int64_t xc = (int64_t)__ldcs(col + p) * R;
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
        const int64_t xc = (int64_t)__ldcs(col + p) * R;
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
template <int LANES, int R, typename VT, typename XT>
__global__ void __launch_bounds__(kThreads)
k_tiles(const Tile *__restrict__ tiles, const int32_t *__restrict__ prp,
        const uint16_t *__restrict__ c16, const int32_t *__restrict__ c32,
        const VT *__restrict__ val, const int32_t *__restrict__ xlist,
        const int32_t *__restrict__ dst, const XT *__restrict__ x, XT *__restrict__ y,
        XT *__restrict__ partial)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    XT *seg = reinterpret_cast<XT *>(smem_raw);
    const Tile t = tiles[blockIdx.x];

    if (t.kind == TILE_CHUNK) {
        XT s[R];
#pragma unroll
        for (int c = 0; c < R; ++c) s[c] = XT(0);
        for (int32_t p = t.r0 + (int32_t)threadIdx.x; p < t.r1; p += kThreads) {
            const XT v = (XT)load_val(val + p);
            const int64_t xc = (int64_t)__ldcs(c32 + p) * R;
#pragma unroll
            for (int c = 0; c < R; ++c) s[c] = fma(v, __ldg(x + xc + c), s[c]);
        }
        block_sum<R>(s);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int c = 0; c < R; ++c) partial[(int64_t)t.y0 * R + c] = s[c];
        }
        return;
    }

    const bool staged = (t.kind == TILE_STAGED);
    if (staged) {
        // stage the tile's x working set: the contiguous run, then the list
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

    constexpr int NG = kThreads / LANES;
    const int g = threadIdx.x / LANES, lane = threadIdx.x & (LANES - 1);
    for (int32_t rb = t.r0; rb < t.r1; rb += NG) {
        const int32_t r = rb + g;
        const bool valid = r < t.r1;
        int32_t p0 = 0, p1 = 0;
        if (valid) {
            p0 = prp[r];
            p1 = prp[r + 1];
        }
        XT s[R];
#pragma unroll
        for (int c = 0; c < R; ++c) s[c] = XT(0);
        if (staged) {
            for (int32_t p = p0 + lane; p < p1; p += LANES) {
                const XT v = (XT)load_val(val + p);
                const int32_t l = (int32_t)__ldcs(c16 + p) * R;
#pragma unroll
                for (int c = 0; c < R; ++c) s[c] = fma(v, seg[l + c], s[c]);
            }
        } else {
            for (int32_t p = p0 + lane; p < p1; p += LANES) {
                const XT v = (XT)load_val(val + p);
                const int64_t xc = (int64_t)__ldcs(c32 + p) * R;
#pragma unroll
                for (int c = 0; c < R; ++c) s[c] = fma(v, __ldg(x + xc + c), s[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < R; ++c) s[c] = group_sum<LANES>(s[c]);
        if (valid && lane == 0) {
            XT *out;
            if (t.y0 >= 0) {
                out = y + (int64_t)(t.y0 + (r - t.r0)) * R;
            } else {
                const int32_t d = dst[r];
                out = d >= 0 ? y + (int64_t)d * R : partial + (int64_t)(-d - 1) * R;
            }
#pragma unroll
            for (int c = 0; c < R; ++c) out[c] = s[c];
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
// Raise the dynamic shared memory limit of a kernel once per device.
template <class Kern>
inline cudaError_t ensure_smem(Kern k, int bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    static int done_bytes[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 64 && done_bytes[dev] >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && dev < 64) done_bytes[dev] = bytes;
    return e;
}

template <int LANES, int R, typename VT, typename XT>
cudaError_t launch_fixed(const DevPlan &P, const XT *x, XT *y, cudaStream_t s)
{
    if (P.use_k1) {
        constexpr int rows_per_block = kThreads / LANES;
        const int64_t nb = ((int64_t)P.m + rows_per_block - 1) / rows_per_block + P.n_long;
        if (nb > 0)
            k_csr_vector<LANES, R, VT, XT><<<(unsigned)nb, kThreads, 0, s>>>(
                P.m, P.rowptr, P.col32, static_cast<const VT *>(P.val), x, y, P.long_rows,
                P.n_long, P.long_thresh);
        return cudaGetLastError();
    }
    if (P.n_tiles > 0) {
        auto kern = k_tiles<LANES, R, VT, XT>;
        cudaError_t e = ensure_smem(kern, P.smem_bytes);
        if (e != cudaSuccess) return e;
        kern<<<(unsigned)P.n_tiles, kThreads, P.smem_bytes, s>>>(
            P.tiles, P.rowptr, P.col16, P.col32, static_cast<const VT *>(P.val), P.xlist, P.dst,
            x, y, static_cast<XT *>(P.partial));
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

template <int LANES, typename VT, typename XT>
cudaError_t launch_r(const DevPlan &P, const XT *x, XT *y, cudaStream_t s)
{
    switch (P.nrhs) {
    case 1: return launch_fixed<LANES, 1, VT, XT>(P, x, y, s);
    case 2: return launch_fixed<LANES, 2, VT, XT>(P, x, y, s);
    case 4: return launch_fixed<LANES, 4, VT, XT>(P, x, y, s);
    case 8: return launch_fixed<LANES, 8, VT, XT>(P, x, y, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename VT, typename XT>
cudaError_t launch_exec(const DevPlan &P, const void *xv, void *yv, cudaStream_t s)
{
    const XT *x = static_cast<const XT *>(xv);
    XT *y = static_cast<XT *>(yv);
    if (P.m == 0) return cudaSuccess;
    switch (P.lanes) {
    case 2: return launch_r<2, VT, XT>(P, x, y, s);
    case 4: return launch_r<4, VT, XT>(P, x, y, s);
    case 8: return launch_r<8, VT, XT>(P, x, y, s);
    case 16: return launch_r<16, VT, XT>(P, x, y, s);
    case 32: return launch_r<32, VT, XT>(P, x, y, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace spmv
