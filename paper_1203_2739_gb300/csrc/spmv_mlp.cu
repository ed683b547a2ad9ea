// Learned form selector (an extension; the paper picks its methods by
// experiment, Sec. 5): host features of a CSR matrix and the FP32 kernels of
// a small multilayer perceptron -- forward pass, gradients of the mean
// softmax cross-entropy, and an Adam step -- so that the network is trained
// on the GPU by this library's own kernels.
//
// Network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), z = W3 h2 + b3, with
// the parameters back to back in one device array (spmv_mlp_param_count).
// Every reduction runs in a fixed order, so results do not depend on the
// schedule.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "spmv_internal.h"

using namespace spmv;

namespace {

constexpr int kT = 256;

struct Layout {
    int64_t w1, b1, w2, b2, w3, b3, total;
};

Layout layout(int32_t nin, int32_t nh, int32_t nc)
{
    Layout L;
    L.w1 = 0;
    L.b1 = L.w1 + (int64_t)nh * nin;
    L.w2 = L.b1 + nh;
    L.b2 = L.w2 + (int64_t)nh * nh;
    L.w3 = L.b2 + nh;
    L.b3 = L.w3 + (int64_t)nc * nh;
    L.total = L.b3 + nc;
    return L;
}

// Y[b][o] = act(sum_i X[b][i] W[o][i] + bias[o]); one thread per (b, o)
__global__ void k_dense(const float *__restrict__ X, const float *__restrict__ W,
                        const float *__restrict__ bias, float *__restrict__ Y, int32_t batch,
                        int32_t nin, int32_t nout, bool relu)
{
    const int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (t >= (int64_t)batch * nout) return;
    const int32_t b = (int32_t)(t / nout), o = (int32_t)(t % nout);
    float a = bias[o];
    for (int32_t i = 0; i < nin; ++i) a = fmaf(X[(int64_t)b * nin + i], W[(int64_t)o * nin + i], a);
    Y[t] = relu ? fmaxf(a, 0.0f) : a;
}

// per sample: loss_b = logsumexp(z) - z[label]; dz = (softmax - onehot) / batch
__global__ void k_softmax_xent(const float *__restrict__ Z, const int32_t *__restrict__ labels,
                               int32_t batch, int32_t nc, float *__restrict__ dZ,
                               float *__restrict__ sample_loss)
{
    const int32_t b = blockIdx.x * kT + threadIdx.x;
    if (b >= batch) return;
    const float *z = Z + (int64_t)b * nc;
    float zmax = -INFINITY;
    for (int32_t o = 0; o < nc; ++o) zmax = fmaxf(zmax, z[o]);
    float se = 0.0f;
    for (int32_t o = 0; o < nc; ++o) se += expf(z[o] - zmax);
    const float lse = zmax + logf(se);
    const int32_t y = labels[b];
    if (y < 0 || y >= nc) {
        // a label outside [0, nc): no gradient, and the loss says so (NaN)
        sample_loss[b] = __int_as_float(0x7fc00000);
        for (int32_t o = 0; o < nc; ++o) dZ[(int64_t)b * nc + o] = 0.0f;
        return;
    }
    sample_loss[b] = lse - z[y];
    for (int32_t o = 0; o < nc; ++o)
        dZ[(int64_t)b * nc + o] = (expf(z[o] - lse) - (o == y ? 1.0f : 0.0f)) / (float)batch;
}

// loss = sum of the per-sample losses / batch, in a fixed order (one block)
__global__ void k_mean(const float *__restrict__ v, int32_t n, float *__restrict__ out)
{
    __shared__ float part[kT];
    float a = 0.0f;
    for (int32_t i = threadIdx.x; i < n; i += kT) a += v[i];
    part[threadIdx.x] = a;
    __syncthreads();
    for (int s = kT / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = part[0] / (float)n;
}

// dH[b][i] = (sum_o dY[b][o] W[o][i]) * (H[b][i] > 0); one thread per (b, i)
__global__ void k_back(const float *__restrict__ dY, const float *__restrict__ W,
                       const float *__restrict__ H, float *__restrict__ dH, int32_t batch,
                       int32_t nin, int32_t nout)
{
    const int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (t >= (int64_t)batch * nin) return;
    const int32_t b = (int32_t)(t / nin), i = (int32_t)(t % nin);
    float a = 0.0f;
    for (int32_t o = 0; o < nout; ++o) a = fmaf(dY[(int64_t)b * nout + o], W[(int64_t)o * nin + i], a);
    dH[t] = H[t] > 0.0f ? a : 0.0f;
}

// gW[o][i] = sum_b dY[b][o] H[b][i]; gb[o] = sum_b dY[b][o]; one thread per
// (o, i) with i = nin standing for the bias
__global__ void k_wgrad(const float *__restrict__ dY, const float *__restrict__ H,
                        float *__restrict__ gW, float *__restrict__ gb, int32_t batch,
                        int32_t nin, int32_t nout)
{
    const int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (t >= (int64_t)nout * (nin + 1)) return;
    const int32_t o = (int32_t)(t / (nin + 1)), i = (int32_t)(t % (nin + 1));
    float a = 0.0f;
    if (i < nin) {
        for (int32_t b = 0; b < batch; ++b)
            a = fmaf(dY[(int64_t)b * nout + o], H[(int64_t)b * nin + i], a);
        gW[(int64_t)o * nin + i] = a;
    } else {
        for (int32_t b = 0; b < batch; ++b) a += dY[(int64_t)b * nout + o];
        gb[o] = a;
    }
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int64_t n, float lr, float c1, float c2)
{
    const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (i >= n) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float mi = b1 * m[i] + (1.0f - b1) * g[i];
    const float vi = b2 * v[i] + (1.0f - b2) * g[i] * g[i];
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

unsigned blocks_for(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + kT - 1) / kT); }

spmv_status check_net(const spmv_mlp *net)
{
    if (!net || !net->params || net->nin < 1 || net->nh < 1 || net->nc < 2) {
        set_error("bad network (NULL parameters or sizes nin=%d nh=%d nc=%d)",
                  net ? net->nin : 0, net ? net->nh : 0, net ? net->nc : 0);
        return SPMV_E_INVALID;
    }
    return SPMV_OK;
}

spmv_status launch_status(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("%s: %s", what, cudaGetErrorString(e));
        return SPMV_E_CUDA;
    }
    return SPMV_OK;
}

// W1[o][i] <- W1[o][i] / sd[i]; b1[o] <- b1[o] - sum_i W1[o][i] mu[i] (new
// W1, i in order): the first layer then reads unscaled features
__global__ void k_fold_scaling(float *__restrict__ W1, float *__restrict__ b1,
                               const float *__restrict__ mu, const float *__restrict__ sd,
                               int32_t nin, int32_t nh)
{
    const int32_t o = blockIdx.x * kT + threadIdx.x;
    if (o >= nh) return;
    float acc = b1[o];
    for (int32_t i = 0; i < nin; ++i) {
        const float w = W1[(int64_t)o * nin + i] / sd[i];
        W1[(int64_t)o * nin + i] = w;
        acc = fmaf(-w, mu[i], acc);
    }
    b1[o] = acc;
}

// per sample: the class of the largest score (the lower class on ties) and
// its softmax probability, 1 / sum_k exp(z_k - z_max)
__global__ void k_predict(const float *__restrict__ Z, int32_t batch, int32_t nc,
                          int32_t *__restrict__ cls, float *__restrict__ conf)
{
    const int32_t b = blockIdx.x * kT + threadIdx.x;
    if (b >= batch) return;
    const float *z = Z + (int64_t)b * nc;
    int32_t best = 0;
    for (int32_t k = 1; k < nc; ++k)
        if (z[k] > z[best]) best = k;
    float sum = 0.0f;
    for (int32_t k = 0; k < nc; ++k) sum += expf(z[k] - z[best]);
    cls[b] = best;
    conf[b] = 1.0f / sum;
}

}  // namespace

extern "C" int64_t spmv_mlp_param_count(int32_t nin, int32_t nh, int32_t nc)
{
    return layout(nin, nh, nc).total;
}

extern "C" size_t spmv_mlp_work_bytes(int32_t nh, int32_t nc, int32_t batch)
{
    // h1, h2, d2, d1 (batch x nh), z, dz (batch x nc), per-sample losses
    return (size_t)batch * (4 * (size_t)nh + 2 * (size_t)nc + 1) * sizeof(float);
}

extern "C" spmv_status spmv_mlp_forward(const spmv_mlp *net, const float *X, int32_t batch,
                                        float *logits, void *work, void *stream)
{
    clear_error();
    spmv_status st = check_net(net);
    if (st != SPMV_OK) return st;
    if (batch < 0 || (batch > 0 && (!X || !logits || !work))) {
        set_error("NULL input, output or workspace");
        return SPMV_E_INVALID;
    }
    if (batch == 0) return SPMV_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const Layout L = layout(net->nin, net->nh, net->nc);
    const float *P = net->params;
    float *h1 = static_cast<float *>(work), *h2 = h1 + (size_t)batch * net->nh;
    k_dense<<<blocks_for((int64_t)batch * net->nh), kT, 0, s>>>(X, P + L.w1, P + L.b1, h1, batch,
                                                                net->nin, net->nh, true);
    k_dense<<<blocks_for((int64_t)batch * net->nh), kT, 0, s>>>(h1, P + L.w2, P + L.b2, h2, batch,
                                                                net->nh, net->nh, true);
    k_dense<<<blocks_for((int64_t)batch * net->nc), kT, 0, s>>>(h2, P + L.w3, P + L.b3, logits,
                                                                batch, net->nh, net->nc, false);
    return launch_status("MLP forward");
}

extern "C" spmv_status spmv_mlp_predict(const spmv_mlp *net, const float *X, int32_t batch,
                                        int32_t *cls, float *conf, void *work, void *stream)
{
    clear_error();
    spmv_status st = check_net(net);
    if (st != SPMV_OK) return st;
    if (batch < 0 || (batch > 0 && (!X || !cls || !conf || !work))) {
        set_error("NULL input, output or workspace");
        return SPMV_E_INVALID;
    }
    if (batch == 0) return SPMV_OK;
    // the logits go to the workspace after the two hidden layers
    float *z = static_cast<float *>(work) + 2 * (size_t)batch * net->nh;
    void *hw = work;
    st = spmv_mlp_forward(net, X, batch, z, hw, stream);
    if (st != SPMV_OK) return st;
    k_predict<<<blocks_for(batch), kT, 0, static_cast<cudaStream_t>(stream)>>>(z, batch, net->nc,
                                                                               cls, conf);
    return launch_status("MLP prediction");
}

extern "C" spmv_status spmv_mlp_fold_scaling(const spmv_mlp *net, const float *mu,
                                             const float *sd, void *stream)
{
    clear_error();
    spmv_status st = check_net(net);
    if (st != SPMV_OK) return st;
    if (!mu || !sd) {
        set_error("NULL feature means or deviations");
        return SPMV_E_INVALID;
    }
    const Layout L = layout(net->nin, net->nh, net->nc);
    k_fold_scaling<<<blocks_for(net->nh), kT, 0, static_cast<cudaStream_t>(stream)>>>(
        net->params + L.w1, net->params + L.b1, mu, sd, net->nin, net->nh);
    return launch_status("feature scaling fold");
}

extern "C" spmv_status spmv_mlp_grad(const spmv_mlp *net, const float *X, const int32_t *labels,
                                     int32_t batch, float *grads, float *loss, void *work,
                                     void *stream)
{
    clear_error();
    spmv_status st = check_net(net);
    if (st != SPMV_OK) return st;
    if (batch < 1 || !X || !labels || !grads || !loss || !work) {
        set_error("batch=%d: needs a non-empty batch, labels, gradient, loss and workspace",
                  batch);
        return SPMV_E_INVALID;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int32_t nin = net->nin, nh = net->nh, nc = net->nc;
    const Layout L = layout(nin, nh, nc);
    const float *P = net->params;
    float *h1 = static_cast<float *>(work);
    float *h2 = h1 + (size_t)batch * nh;
    float *d2 = h2 + (size_t)batch * nh;
    float *d1 = d2 + (size_t)batch * nh;
    float *z = d1 + (size_t)batch * nh;
    float *dz = z + (size_t)batch * nc;
    float *sl = dz + (size_t)batch * nc;
    k_dense<<<blocks_for((int64_t)batch * nh), kT, 0, s>>>(X, P + L.w1, P + L.b1, h1, batch, nin,
                                                           nh, true);
    k_dense<<<blocks_for((int64_t)batch * nh), kT, 0, s>>>(h1, P + L.w2, P + L.b2, h2, batch, nh,
                                                           nh, true);
    k_dense<<<blocks_for((int64_t)batch * nc), kT, 0, s>>>(h2, P + L.w3, P + L.b3, z, batch, nh,
                                                           nc, false);
    k_softmax_xent<<<blocks_for(batch), kT, 0, s>>>(z, labels, batch, nc, dz, sl);
    k_mean<<<1, kT, 0, s>>>(sl, batch, loss);
    k_wgrad<<<blocks_for((int64_t)nc * (nh + 1)), kT, 0, s>>>(dz, h2, grads + L.w3, grads + L.b3,
                                                              batch, nh, nc);
    k_back<<<blocks_for((int64_t)batch * nh), kT, 0, s>>>(dz, P + L.w3, h2, d2, batch, nh, nc);
    k_wgrad<<<blocks_for((int64_t)nh * (nh + 1)), kT, 0, s>>>(d2, h1, grads + L.w2, grads + L.b2,
                                                              batch, nh, nh);
    k_back<<<blocks_for((int64_t)batch * nh), kT, 0, s>>>(d2, P + L.w2, h1, d1, batch, nh, nh);
    k_wgrad<<<blocks_for((int64_t)nh * (nin + 1)), kT, 0, s>>>(d1, X, grads + L.w1, grads + L.b1,
                                                               batch, nin, nh);
    return launch_status("MLP gradient");
}

extern "C" spmv_status spmv_mlp_adam(const spmv_mlp *net, const float *grads, float *m, float *v,
                                     int32_t step, float lr, void *stream)
{
    clear_error();
    spmv_status st = check_net(net);
    if (st != SPMV_OK) return st;
    if (!grads || !m || !v || step < 1 || !(lr > 0.0f)) {
        set_error("Adam needs gradients, both moment buffers, step >= 1 and lr > 0");
        return SPMV_E_INVALID;
    }
    const int64_t n = layout(net->nin, net->nh, net->nc).total;
    const float c1 = 1.0f - std::pow(0.9f, (float)step), c2 = 1.0f - std::pow(0.999f, (float)step);
    k_adam<<<blocks_for(n), kT, 0, static_cast<cudaStream_t>(stream)>>>(net->params, grads, m, v,
                                                                         n, lr, c1, c2);
    return launch_status("Adam step");
}

// ------------------------------------------------------------- features --
extern "C" spmv_status spmv_features(const spmv_csr *A, float *out)
{
    clear_error();
    spmv_status st = validate_csr(A);
    if (st != SPMV_OK) return st;
    if (!out) {
        set_error("out is NULL");
        return SPMV_E_INVALID;
    }
    const int32_t m = A->m, n = A->n;
    const int64_t nnz = A->nnz;
    std::vector<int64_t> cdeg((size_t)std::max(n, 1), 0);
    double rs = 0, rs2 = 0, rmax = 0, band = 0, near = 0, long_nnz = 0;
    int64_t empty = 0;
    const int64_t win = std::max<int64_t>(1, n / 64);
    for (int32_t i = 0; i < m; ++i) {
        const int32_t a = A->rowptr[i], b = A->rowptr[i + 1], d = b - a;
        rs += d;
        rs2 += (double)d * d;
        rmax = std::max(rmax, (double)d);
        if (d == 0) ++empty;
        if (d > 64) long_nnz += d;
        // the row's diagonal position in a square view of the matrix
        const double di = n > 0 && m > 0 ? (double)i * n / m : 0.0;
        for (int32_t p = a; p < b; ++p) {
            const int32_t j = A->colidx[p];
            cdeg[j]++;
            const double dist = std::fabs((double)j - di);
            band += dist;
            near += dist < win;
        }
    }
    double cs2 = 0, cmax = 0;
    for (int32_t j = 0; j < n; ++j) {
        cs2 += (double)cdeg[j] * cdeg[j];
        cmax = std::max(cmax, (double)cdeg[j]);
    }
    // columns touched by more than one of 16 contiguous row blocks: a cheap
    // estimate of how much a 16-way row partition in the given order cuts
    std::vector<int8_t> owner((size_t)std::max(n, 1), -1);
    int64_t cut = 0, touched = 0;
    for (int32_t i = 0; i < m; ++i) {
        const int8_t blk = (int8_t)std::min<int64_t>(15, (int64_t)i * 16 / std::max(m, 1));
        for (int32_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p) {
            const int32_t j = A->colidx[p];
            if (owner[j] == -1) {
                owner[j] = blk;
                ++touched;
            } else if (owner[j] != blk && owner[j] != 16) {
                owner[j] = 16;      // counted once
                ++cut;
            }
        }
    }
    const double rmean = m > 0 ? rs / m : 0.0, cmean = n > 0 ? (double)nnz / n : 0.0;
    const double rvar = m > 0 ? std::max(0.0, rs2 / m - rmean * rmean) : 0.0;
    const double cvar = n > 0 ? std::max(0.0, cs2 / n - cmean * cmean) : 0.0;
    const double nz = std::max<int64_t>(nnz, 1);
    float f[SPMV_SEL_FEATURES] = {
        (float)std::log2(1.0 + m),
        (float)std::log2(1.0 + n),
        (float)std::log2(1.0 + nnz),
        (float)rmean,
        (float)(rmean > 0 ? std::sqrt(rvar) / rmean : 0.0),
        (float)std::log2(1.0 + rmax),
        (float)(rmean > 0 ? rmax / rmean : 0.0),
        (float)(cmean > 0 ? std::sqrt(cvar) / cmean : 0.0),
        (float)std::log2(1.0 + cmax),
        (float)(cmean > 0 ? cmax / cmean : 0.0),
        (float)(n > 0 ? band / nz / n : 0.0),
        (float)(near / nz),
        (float)(touched > 0 ? (double)cut / touched : 0.0),
        (float)(m > 0 ? (double)empty / m : 0.0),
        (float)(long_nnz / nz),
        (float)(std::log2(1.0 + (double)nnz * 12.0) - 27.0),   // CSR bytes against 128 MB (L2)
    };
    for (int k = 0; k < SPMV_SEL_FEATURES; ++k) out[k] = f[k];
    return SPMV_OK;
}
