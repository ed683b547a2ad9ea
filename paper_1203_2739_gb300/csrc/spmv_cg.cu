// Mixed-precision conjugate gradients with iterative refinement on two plans
// of the same matrix (the precision extension; the paper itself computes in
// FP64 throughout, Sec. 5.2).
//
// The outer loop computes the residual r = b - A x with the FP64 plan, in
// FP64, and stops when ||r|| <= tol ||b||.  Each outer step solves A d = r/||r||
// approximately with plain CG whose matrix-vector products use the low
// plan (FP32 or BF16 values, FP32 vectors and accumulation; or FP64), then
// updates x <- x + ||r|| d in FP64.  CG needs a symmetric operator, so the
// solver works in the plan's column space x_hat = x P_c: the product
// y_hat = A_hat x_hat lands in row space and is moved to column space with
// the composed permutation q[j'] = y_hat[rowpos(col_perm[j'])] (skipped when
// the row and column permutations are equal).
//
// The CG scalars live on the device: a dot product is one kernel of block
// partial sums plus a one-block kernel that adds them in a fixed order (so a
// solve is deterministic) and updates alpha or beta.  Once the inner
// iteration converges, a device flag turns the remaining vector kernels of
// the batch into no-ops.  A batch of kInnerBatch iterations is captured once
// in a CUDA graph and replayed; the host reads the flag after each replay.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "spmv_plan_obj.h"

using namespace spmv;

namespace {

constexpr int kT = 256;              // threads per block
constexpr int kMaxBlocks = 1024;     // blocks of the vector kernels (partials)
constexpr int kInnerBatch = 8;       // inner iterations per graph replay

struct Scalars {
    double rr;        // r.r of the inner iteration
    double rr0;       // r.r at its start
    double pq;        // p.q
    double alpha, beta;
    double norm;      // ||b - A x|| of the current outer step
    int32_t done;     // 1: converged / iteration limit; 2: breakdown (p.q <= 0)
    int32_t iters;    // inner iterations done in this outer step
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block; valid in thread 0.
__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double w[kT / 32];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = threadIdx.x < kT / 32 ? w[threadIdx.x] : 0.0;
        s = warp_sum(s);
    }
    return s;
}

// Sum of nb partials in a fixed order (one block).
__device__ __forceinline__ double sum_partials(const double *part, int nb)
{
    double v = 0.0;
    for (int i = threadIdx.x; i < nb; i += kT) v += part[i];
    return block_sum(v);
}

template <typename T>
__global__ void __launch_bounds__(kT) k_dot(const T *__restrict__ a, const T *__restrict__ b,
                                            int32_t n, double *__restrict__ part,
                                            const Scalars *S)
{
    if (S && S->done) return;
    double v = 0.0;
    for (int32_t i = blockIdx.x * kT + threadIdx.x; i < n; i += gridDim.x * kT)
        v += (double)a[i] * (double)b[i];
    v = block_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
}

// alpha = rr / (p.q)
__global__ void __launch_bounds__(kT) k_alpha(const double *__restrict__ part, int nb, Scalars *S)
{
    if (S->done) return;
    const double pq = sum_partials(part, nb);
    if (threadIdx.x == 0) {
        S->pq = pq;
        if (!(pq > 0.0)) {
            S->done = 2;
            S->alpha = 0.0;
        } else {
            S->alpha = S->rr / pq;
        }
    }
}

// d += alpha p; r -= alpha q; partials of r.r
template <typename T>
__global__ void __launch_bounds__(kT) k_step(T *__restrict__ d, T *__restrict__ r,
                                             const T *__restrict__ p, const T *__restrict__ q,
                                             int32_t n, double *__restrict__ part,
                                             const Scalars *S)
{
    if (S->done) return;
    const T alpha = (T)S->alpha;
    double v = 0.0;
    for (int32_t i = blockIdx.x * kT + threadIdx.x; i < n; i += gridDim.x * kT) {
        d[i] = fma(alpha, p[i], d[i]);
        const T ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        v += (double)ri * (double)ri;
    }
    v = block_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
}

// beta = rr_new / rr; convergence test of the inner iteration
__global__ void __launch_bounds__(kT) k_beta(const double *__restrict__ part, int nb, Scalars *S,
                                             double tol2, int32_t max_inner)
{
    if (S->done) return;
    const double rr = sum_partials(part, nb);
    if (threadIdx.x == 0) {
        S->beta = rr / S->rr;
        S->rr = rr;
        S->iters += 1;
        if (rr <= tol2 * S->rr0 || S->iters >= max_inner) S->done = 1;
    }
}

// p = r + beta p
template <typename T>
__global__ void __launch_bounds__(kT) k_direction(T *__restrict__ p, const T *__restrict__ r,
                                                  int32_t n, const Scalars *S)
{
    if (S->done) return;
    const T beta = (T)S->beta;
    for (int32_t i = blockIdx.x * kT + threadIdx.x; i < n; i += gridDim.x * kT)
        p[i] = fma(beta, p[i], r[i]);
}

// r64 = b - t; partials of r64.r64
__global__ void __launch_bounds__(kT) k_residual(const double *__restrict__ b,
                                                 const double *__restrict__ t, int32_t n,
                                                 double *__restrict__ r, double *__restrict__ part)
{
    double v = 0.0;
    for (int32_t i = blockIdx.x * kT + threadIdx.x; i < n; i += gridDim.x * kT) {
        const double ri = b[i] - t[i];
        r[i] = ri;
        v += ri * ri;
    }
    v = block_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
}

// norm = sqrt(sum of partials); start of an inner solve
__global__ void __launch_bounds__(kT) k_norm(const double *__restrict__ part, int nb, Scalars *S,
                                             double *out)
{
    const double s = sum_partials(part, nb);
    if (threadIdx.x == 0) {
        S->norm = sqrt(s);
        *out = s;
        S->done = 0;
        S->iters = 0;
    }
}

// r = r64 / norm (in T); p = r; d = 0; partials of r.r
template <typename T>
__global__ void __launch_bounds__(kT) k_inner_start(const double *__restrict__ r64, T *__restrict__ r,
                                                    T *__restrict__ p, T *__restrict__ d,
                                                    int32_t n, double *__restrict__ part,
                                                    const Scalars *S)
{
    const double inv = S->norm > 0.0 ? 1.0 / S->norm : 0.0;
    double v = 0.0;
    for (int32_t i = blockIdx.x * kT + threadIdx.x; i < n; i += gridDim.x * kT) {
        const T ri = (T)(r64[i] * inv);
        r[i] = ri;
        p[i] = ri;
        d[i] = T(0);
        v += (double)ri * (double)ri;
    }
    v = block_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
}

__global__ void __launch_bounds__(kT) k_rr0(const double *__restrict__ part, int nb, Scalars *S)
{
    const double s = sum_partials(part, nb);
    if (threadIdx.x == 0) {
        S->rr = s;
        S->rr0 = s;
        if (!(s > 0.0)) S->done = 1;
    }
}

// x += norm * d (FP64)
template <typename T>
__global__ void __launch_bounds__(kT) k_update_x(double *__restrict__ x, const T *__restrict__ d,
                                                 int32_t n, const Scalars *S)
{
    const double s = S->norm;
    for (int32_t i = blockIdx.x * kT + threadIdx.x; i < n; i += gridDim.x * kT)
        x[i] = fma(s, (double)d[i], x[i]);
}

// rinv[row_perm[i]] = i
__global__ void k_inverse(const int32_t *__restrict__ perm, int32_t n, int32_t *__restrict__ inv)
{
    const int32_t i = blockIdx.x * kT + threadIdx.x;
    if (i < n) inv[perm[i]] = i;
}

// q[j] = rinv[col_perm[j]] (NULL perms are the identity)
__global__ void k_compose(const int32_t *__restrict__ rinv, const int32_t *__restrict__ col_perm,
                          int32_t n, int32_t *__restrict__ q)
{
    const int32_t j = blockIdx.x * kT + threadIdx.x;
    if (j >= n) return;
    const int32_t c = col_perm ? col_perm[j] : j;
    q[j] = rinv ? rinv[c] : c;
}

template <typename T>
__global__ void __launch_bounds__(kT) k_gather(const T *__restrict__ src, const int32_t *__restrict__ idx,
                                               int32_t n, T *__restrict__ dst, const Scalars *S)
{
    if (S && S->done) return;
    for (int32_t i = blockIdx.x * kT + threadIdx.x; i < n; i += gridDim.x * kT) dst[i] = src[idx[i]];
}

// x_hat[j] = x[col_perm[j]] (gather) or x[col_perm[j]] = x_hat[j] (scatter)
__global__ void k_perm64(const double *__restrict__ src, const int32_t *__restrict__ perm, int32_t n,
                         double *__restrict__ dst, bool scatter)
{
    const int32_t j = blockIdx.x * kT + threadIdx.x;
    if (j >= n) return;
    const int32_t c = perm ? perm[j] : j;
    if (scatter) dst[c] = src[j];
    else dst[j] = src[c];
}

struct Work {
    spmv_plan *owner = nullptr;
    std::vector<void *> bufs;
    void *get(size_t bytes)
    {
        void *p = plan_alloc(owner, bytes);
        if (p) bufs.push_back(p);
        return p;
    }
    ~Work()
    {
        for (void *p : bufs) plan_free(owner, p);
    }
};

spmv_status fail(cudaError_t e, const char *what)
{
    set_error("%s: %s", what, cudaGetErrorString(e));
    return SPMV_E_CUDA;
}

template <typename T>
spmv_status solve(spmv_plan *low, spmv_plan *f64, const double *b, double *x,
                  const spmv_cg_opts &o, spmv_cg_info *info, cudaStream_t user)
{
    const int32_t n = low->info.n;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(kMaxBlocks, (n + kT - 1) / kT));
    const unsigned pgrid = (unsigned)((n + kT - 1) / kT);
    Work w;
    w.owner = low;
    double *bh = (double *)w.get((size_t)n * 8), *xh = (double *)w.get((size_t)n * 8);
    double *t_y = (double *)w.get((size_t)n * 8), *t_x = (double *)w.get((size_t)n * 8);
    double *r64 = (double *)w.get((size_t)n * 8);
    T *r = (T *)w.get((size_t)n * sizeof(T)), *p = (T *)w.get((size_t)n * sizeof(T));
    T *q_y = (T *)w.get((size_t)n * sizeof(T)), *q = (T *)w.get((size_t)n * sizeof(T));
    T *d = (T *)w.get((size_t)n * sizeof(T));
    double *part = (double *)w.get(kMaxBlocks * 8);
    Scalars *S = (Scalars *)w.get(sizeof(Scalars));
    double *nrm = (double *)w.get(8);
    int32_t *qidx = nullptr, *rinv = nullptr;
    const bool same = low->same_perm;
    if (!same) {
        qidx = (int32_t *)w.get((size_t)n * 4);
        rinv = (int32_t *)w.get((size_t)n * 4);
    }
    if (w.bufs.size() != (same ? 13u : 15u)) {
        set_error("device allocation of the solver workspace failed");
        return SPMV_E_NOMEM;
    }
    double *h = nullptr;   // pinned: [0] ||r||^2, [1] ||b||^2, [2] done, [3] iters
    if (cudaMallocHost((void **)&h, 4 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        set_error("pinned host allocation failed");
        return SPMV_E_NOMEM;
    }
    struct HostFree {
        double *h;
        ~HostFree() { cudaFreeHost(h); }
    } hf{h};

    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    struct Res {
        cudaStream_t &s;
        cudaEvent_t &ev;
        cudaGraph_t &g;
        cudaGraphExec_t &ge;
        ~Res()
        {
            if (ge) cudaGraphExecDestroy(ge);
            if (g) cudaGraphDestroy(g);
            if (ev) cudaEventDestroy(ev);
            if (s) cudaStreamDestroy(s);
        }
    } res{s, ev, graph, gexec};
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev, 0);
    if (e != cudaSuccess) return fail(e, "solver stream");

    // into column space; the composed permutation
    k_perm64<<<pgrid, kT, 0, s>>>(b, low->d_col_perm, n, bh, false);
    k_perm64<<<pgrid, kT, 0, s>>>(x, low->d_col_perm, n, xh, false);
    if (!same) {
        if (low->d_row_perm) k_inverse<<<pgrid, kT, 0, s>>>(low->d_row_perm, n, rinv);
        k_compose<<<pgrid, kT, 0, s>>>(low->d_row_perm ? rinv : nullptr, low->d_col_perm, n, qidx);
    }
    k_dot<double><<<grid, kT, 0, s>>>(bh, bh, n, part, nullptr);
    k_norm<<<1, kT, 0, s>>>(part, (int)grid, S, nrm);
    e = cudaMemcpyAsync(h + 1, nrm, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(e, "solver setup");
    const double bnorm2 = h[1];

    // one inner iteration (the batch the graph holds)
    auto iteration = [&]() -> cudaError_t {
        cudaError_t er = plan_run(low, p, same ? q : q_y, s);
        if (er != cudaSuccess) return er;
        if (!same) k_gather<T><<<grid, kT, 0, s>>>(q_y, qidx, n, q, S);
        k_dot<T><<<grid, kT, 0, s>>>(p, q, n, part, S);
        k_alpha<<<1, kT, 0, s>>>(part, (int)grid, S);
        k_step<T><<<grid, kT, 0, s>>>(d, r, p, q, n, part, S);
        k_beta<<<1, kT, 0, s>>>(part, (int)grid, S, o.inner_tol * o.inner_tol, o.max_inner);
        k_direction<T><<<grid, kT, 0, s>>>(p, r, n, S);
        return cudaGetLastError();
    };

    spmv_cg_info I{};
    I.rel_residual = bnorm2 > 0.0 ? 1.0 : 0.0;
    for (int32_t outer = 0; outer <= o.max_outer; ++outer) {
        // r64 = b - A x in FP64
        e = plan_run(f64, xh, same ? t_x : t_y, s);
        if (e != cudaSuccess) return fail(e, "residual product");
        if (!same) k_gather<double><<<grid, kT, 0, s>>>(t_y, qidx, n, t_x, nullptr);
        k_residual<<<grid, kT, 0, s>>>(bh, t_x, n, r64, part);
        k_norm<<<1, kT, 0, s>>>(part, (int)grid, S, nrm);
        e = cudaMemcpyAsync(h, nrm, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(e, "residual");
        I.rel_residual = bnorm2 > 0.0 ? std::sqrt(h[0] / bnorm2) : 0.0;
        I.outer = outer;
        if (I.rel_residual <= o.tol) {
            I.converged = 1;
            break;
        }
        if (outer == o.max_outer) break;

        // inner CG on A d = r / ||r|| in T
        k_inner_start<T><<<grid, kT, 0, s>>>(r64, r, p, d, n, part, S);
        k_rr0<<<1, kT, 0, s>>>(part, (int)grid, S);
        if (!gexec) {
            // one product outside the capture first, so that the launch
            // attributes the plan sets on first use are set before capturing
            e = plan_run(low, p, same ? q : q_y, s);
            if (e != cudaSuccess) return fail(e, "inner product");
            e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return fail(e, "graph capture");
            for (int it = 0; it < kInnerBatch && e == cudaSuccess; ++it) e = iteration();
            cudaGraph_t g = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(s, &g);
            graph = g;
            if (e != cudaSuccess) return fail(e, "captured iteration");
            if (e2 != cudaSuccess) return fail(e2, "graph capture");
            e = cudaGraphInstantiate(&gexec, graph, 0);
            if (e != cudaSuccess) return fail(e, "graph instantiate");
        }
        int32_t done = 0, iters = 0;
        for (int32_t launched = 0; launched < o.max_inner + kInnerBatch; launched += kInnerBatch) {
            e = cudaGraphLaunch(gexec, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h + 2, &S->done, 8, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return fail(e, "inner iterations");
            int32_t di[2];
            std::memcpy(di, h + 2, 8);
            done = di[0];
            iters = di[1];
            if (done) break;
        }
        I.inner_total += iters;
        if (done == 2 && iters == 0) {
            set_error("CG broke down: p.q <= 0 (is A symmetric positive definite?)");
            return SPMV_E_INVALID;
        }
        k_update_x<T><<<grid, kT, 0, s>>>(xh, d, n, S);
    }
    // back to the caller's order
    k_perm64<<<pgrid, kT, 0, s>>>(xh, low->d_col_perm, n, x, true);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(e, "solution");
    if (info) *info = I;
    return SPMV_OK;
}

}  // namespace

extern "C" spmv_status spmv_cg_ir(spmv_plan *low, spmv_plan *f64, const double *b, double *x,
                                  const spmv_cg_opts *opts, spmv_cg_info *info, void *stream)
{
    clear_error();
    if (!low || !f64 || (!b && low && low->info.n > 0) || (!x && low && low->info.n > 0)) {
        set_error("NULL plan or vector");
        return SPMV_E_INVALID;
    }
    const spmv_plan_info &L = low->info, &F = f64->info;
    if (L.m != L.n || F.m != L.m || F.n != L.n || L.nnz != F.nnz) {
        set_error("the plans must hold the same square matrix (m=%d n=%d vs m=%d n=%d)", L.m,
                  L.n, F.m, F.n);
        return SPMV_E_INVALID;
    }
    if (L.nrhs != 1 || F.nrhs != 1) {
        set_error("the solver takes plans with one right-hand side");
        return SPMV_E_UNSUPPORTED;
    }
    if (F.dtype != SPMV_F64) {
        set_error("the residual plan must be SPMV_F64");
        return SPMV_E_INVALID;
    }
    if (low->same_perm != f64->same_perm) {
        set_error("the plans must use the same permutations");
        return SPMV_E_INVALID;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != low->device || dev != f64->device) {
        cudaGetLastError();
        set_error("the plans must live on the current device");
        return SPMV_E_INVALID;
    }
    spmv_cg_opts o{};
    if (opts) o = *opts;
    if (!(o.tol > 0.0)) o.tol = 1e-10;
    if (!(o.inner_tol > 0.0)) o.inner_tol = L.dtype == SPMV_F64 ? 1e-12 : 1e-4;
    if (o.max_outer <= 0) o.max_outer = 50;
    if (o.max_inner <= 0) o.max_inner = 2000;
    if (info) *info = spmv_cg_info{};
    if (L.n == 0) {
        if (info) info->converged = 1;
        return SPMV_OK;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    try {
        if (L.dtype == SPMV_F64) return solve<double>(low, f64, b, x, o, info, s);
        return solve<float>(low, f64, b, x, o, info, s);
    } catch (...) {
        set_error("internal error");
        return SPMV_E_INTERNAL;
    }
}
