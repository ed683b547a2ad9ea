// spmv_csr_exec_noalloc: y = A x for a CSR matrix already on the device,
// without allocating anything.
//
// Some callers cannot allocate device memory at the point where they need a
// product: code running inside a memory pool they do not own, a plugin
// handed only its input and output buffers, or a step that must not change
// the allocator's state.  They can call this entry point: every nonzero range
// of CHUNK elements is reduced by one CTA, and the partial sums of rows that
// cross chunk boundaries go to a fixed scratch array declared in this file
// (static device memory, part of the loaded module) instead of memory from
// cudaMalloc.  A second kernel adds those partial sums, in chunk order, into
// y.  The result has the same meaning as spmv_exec on a natural-order FP64
// plan; the summation order differs.
#include <cuda_runtime.h>

#include <mutex>

#include "spmv_device.h"

namespace spmv {
namespace {

constexpr int kNoallocThreads = 256;
constexpr int64_t kChunk = 4096;     // nonzeros per CTA
// SPMV_NOALLOC_MAX_NNZ / kChunk chunks, two partial sums each (4 MiB)
constexpr int64_t kMaxChunks = SPMV_NOALLOC_MAX_NNZ / kChunk;

// head[b]: chunk b's share of the row that started before the chunk;
// tail[b]: chunk b's share of a row that starts in it and runs past its end.
// Every call writes every entry the fix-up kernel then reads, so nothing has
// to start at zero; concurrent calls share the array and race.
static __device__ __align__(256) double g_noalloc_scratch[2 * kMaxChunks];

__device__ __forceinline__ int32_t lower_bound_dev(const int32_t *a, int32_t n, int64_t v)
{
    // first index i in [0, n] with a[i] >= v (a is nondecreasing)
    int32_t lo = 0, hi = n;
    while (lo < hi) {
        const int32_t mid = lo + (hi - lo) / 2;
        if ((int64_t)__ldg(a + mid) < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// One CTA per chunk of kChunk nonzeros.  Rows that start inside the chunk
// and end inside it are written to y; the row running in from the previous
// chunk goes to head[b]; a row starting here and running out goes to tail[b].
// Empty rows are written (as 0) by the chunk holding their start position.
__global__ void __launch_bounds__(kNoallocThreads)
k_noalloc_chunks(int32_t m, int64_t nnz, const int32_t *__restrict__ rowptr,
                 const int32_t *__restrict__ col, const double *__restrict__ val,
                 const double *__restrict__ x, double *__restrict__ y,
                 double *__restrict__ scratch, int64_t nchunks)
{
    const int64_t b = blockIdx.x;
    const int64_t c0 = b * kChunk, c1 = min(nnz, c0 + kChunk);
    double *head = scratch, *tail = scratch + nchunks;
    // rows starting in [c0, c1); the last chunk also owns rows starting at nnz
    const int32_t r_lo = lower_bound_dev(rowptr, m, c0);
    const int32_t r_hi = (b == nchunks - 1) ? m : lower_bound_dev(rowptr, m, c1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kWarps = kNoallocThreads / 32;
    // row -1 stands for the row running in from before the chunk
    const bool has_head = r_lo > 0 && (int64_t)__ldg(rowptr + r_lo) > c0;
    for (int32_t q = (has_head ? -1 : 0) + warp; q < r_hi - r_lo; q += kWarps) {
        const int32_t r = q < 0 ? r_lo - 1 : r_lo + q;
        const int64_t a = max((int64_t)__ldg(rowptr + r), c0);
        const int64_t e = (int64_t)__ldg(rowptr + r + 1);
        const int64_t z = min(e, c1);
        double s = 0.0;
        for (int64_t p = a + lane; p < z; p += 32) s = fma(__ldg(val + p), __ldg(x + __ldg(col + p)), s);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) {
            if (q < 0) head[b] = s;
            else if (e > c1) tail[b] = s;
            else y[r] = s;
        }
    }
}

// One thread per chunk: if a row starts in chunk b and runs past it, add its
// pieces in chunk order and write y.
__global__ void __launch_bounds__(kNoallocThreads)
k_noalloc_fixup(int32_t m, int64_t nnz, const int32_t *__restrict__ rowptr,
                double *__restrict__ y, const double *__restrict__ scratch, int64_t nchunks)
{
    const int64_t b = (int64_t)blockIdx.x * kNoallocThreads + threadIdx.x;
    if (b >= nchunks) return;
    const double *head = scratch, *tail = scratch + nchunks;
    const int64_t c0 = b * kChunk, c1 = min(nnz, c0 + kChunk);
    const int32_t r_lo = lower_bound_dev(rowptr, m, c0);
    const int32_t r_hi = (b == nchunks - 1) ? m : lower_bound_dev(rowptr, m, c1);
    if (r_hi <= r_lo) return;
    const int32_t r = r_hi - 1;                      // last row starting in the chunk
    const int64_t e = (int64_t)__ldg(rowptr + r + 1);
    if (e <= c1) return;                             // complete: already written
    double s = tail[b];
    for (int64_t b2 = b + 1; b2 < nchunks && b2 * kChunk < e; ++b2) s += head[b2];
    y[r] = s;
}

__global__ void k_noalloc_zero(int32_t m, double *__restrict__ y)
{
    const int64_t i = (int64_t)blockIdx.x * kNoallocThreads + threadIdx.x;
    if (i < m) y[i] = 0.0;
}

// Device address of the scratch array, looked up once per device with that
// device current (in host code the array's name is only a host-side handle).
// CUDA loads modules lazily by default: the lookup loads this file's module
// (and with it the scratch array) onto the device, and cudaFuncGetAttributes
// loads each kernel's code, so that no later call has to allocate for them.
std::mutex g_mu;
double *g_scratch_ptr[128] = {nullptr};

spmv_status scratch_for_current_device(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error("cudaGetDevice: %s", cudaGetErrorString(e));
        return SPMV_E_CUDA;
    }
    if (dev < 0 || dev >= 128) {
        set_error("device index %d out of range", dev);
        return SPMV_E_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            set_error("cudaGetSymbolAddress of the scratch array: %s", cudaGetErrorString(e));
            return SPMV_E_CUDA;
        }
        const void *kernels[] = {reinterpret_cast<const void *>(k_noalloc_chunks),
                                 reinterpret_cast<const void *>(k_noalloc_fixup),
                                 reinterpret_cast<const void *>(k_noalloc_zero)};
        for (const void *k : kernels) {
            cudaFuncAttributes fa;
            e = cudaFuncGetAttributes(&fa, k);
            if (e != cudaSuccess) {
                set_error("loading the kernels of this entry point: %s", cudaGetErrorString(e));
                return SPMV_E_CUDA;
            }
        }
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return SPMV_OK;
}

}  // namespace
}  // namespace spmv

using namespace spmv;

extern "C" spmv_status spmv_csr_exec_noalloc(int32_t m, int32_t n, int64_t nnz,
                                             const int32_t *rowptr_dev,
                                             const int32_t *colidx_dev,
                                             const double *vals_dev, const double *x_dev,
                                             double *y_dev, void *stream)
{
    clear_error();
    if (m < 0 || n < 0 || nnz < 0) {
        set_error("negative size m=%d n=%d nnz=%lld", m, n, (long long)nnz);
        return SPMV_E_INVALID;
    }
    if (nnz > SPMV_NOALLOC_MAX_NNZ) {
        set_error("nnz=%lld exceeds the scratch limit of this entry point (%lld nonzeros)",
                  (long long)nnz, (long long)SPMV_NOALLOC_MAX_NNZ);
        return SPMV_E_UNSUPPORTED;
    }
    // set-up first: a call with m = 0 does only this (see the header)
    double *scratch = nullptr;
    spmv_status st = scratch_for_current_device(&scratch);
    if (st != SPMV_OK) return st;
    if (m == 0) return SPMV_OK;
    if (!rowptr_dev || !y_dev || (nnz > 0 && (!colidx_dev || !vals_dev || !x_dev))) {
        set_error("NULL argument");
        return SPMV_E_INVALID;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (nnz == 0) {
        k_noalloc_zero<<<(unsigned)((m + kNoallocThreads - 1) / kNoallocThreads), kNoallocThreads,
                         0, s>>>(m, y_dev);
    } else {
        const int64_t nchunks = (nnz + kChunk - 1) / kChunk;
        k_noalloc_chunks<<<(unsigned)nchunks, kNoallocThreads, 0, s>>>(
            m, nnz, rowptr_dev, colidx_dev, vals_dev, x_dev, y_dev, scratch, nchunks);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_error("chunk kernel launch: %s", cudaGetErrorString(e));
            return SPMV_E_CUDA;
        }
        k_noalloc_fixup<<<(unsigned)((nchunks + kNoallocThreads - 1) / kNoallocThreads),
                          kNoallocThreads, 0, s>>>(m, nnz, rowptr_dev, y_dev, scratch, nchunks);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("kernel launch: %s", cudaGetErrorString(e));
        return SPMV_E_CUDA;
    }
    return SPMV_OK;
}
