// C ABI entry points (include/spmv.h): plan life cycle, execution, vector
// permutation.  Host arrays are built by spmv_plan.cpp; this file owns the
// device memory and the launches.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "spmv_plan_obj.h"

using namespace spmv;

namespace {

void *dev_alloc(spmv_plan *p, size_t bytes) { return plan_alloc(p, bytes); }
void dev_free(spmv_plan *p, void *ptr) { plan_free(p, ptr); }

spmv_status cuda_fail(cudaError_t e, const char *what)
{
    set_error("%s: %s", what, cudaGetErrorString(e));
    return SPMV_E_CUDA;
}

// Carves typed sub-arrays out of one allocation (256-byte aligned each).
struct Arena {
    struct Item {
        const void *host;
        size_t bytes;
        void **slot;
        bool zero;
    };
    std::vector<Item> items;
    size_t total = 0;
    void add(const void *host, size_t bytes, void **slot, bool zero = false)
    {
        items.push_back({host, bytes, slot, zero});
        total += (bytes + 255) & ~size_t(255);
    }
};

template <class T>
void add_vec(Arena &a, const std::vector<T> &v, const void **slot)
{
    a.add(v.data(), v.size() * sizeof(T), const_cast<void **>(slot));
}

spmv_status device_matches(const spmv_plan *p)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != p->device) {
        set_error("plan was built on device %d, current device is %d", p->device, dev);
        return SPMV_E_INVALID;
    }
    return SPMV_OK;
}

cudaError_t run(const spmv_plan *p, const void *x, void *y, cudaStream_t s)
{
    return plan_run(p, x, y, s);
}

}  // namespace

namespace spmv {

void *plan_alloc(spmv_plan *p, size_t bytes)
{
    if (bytes == 0) bytes = 256;
    if (p->alloc) return p->alloc(bytes, p->ctx);
    void *ptr = nullptr;
    if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return ptr;
}

void plan_free(spmv_plan *p, void *ptr)
{
    if (!ptr) return;
    if (p->release) p->release(ptr, p->ctx);
    else cudaFree(ptr);
}

cudaError_t plan_run(const spmv_plan *p, const void *x, void *y, cudaStream_t s)
{
    switch (p->hp.dtype) {
    case SPMV_F64: return exec_f64(p->dp, x, y, s);
    case SPMV_F32: return exec_f32(p->dp, x, y, s);
    default: return exec_bf16(p->dp, x, y, s);
    }
}

}  // namespace spmv

extern "C" spmv_status spmv_plan_create(const spmv_csr *A, const spmv_perm *perm,
                                        const spmv_splits *splits, const spmv_opts *opts,
                                        spmv_plan **out)
{
    clear_error();
    if (!out) {
        set_error("out is NULL");
        return SPMV_E_INVALID;
    }
    *out = nullptr;
    spmv_plan *p = nullptr;
    try {
        p = new spmv_plan();
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            nsm = 0;        // the plan falls back to GB300's 152 SMs
        }
        spmv_status st = build_host_plan(A, perm, splits, opts, nsm, &p->hp);
        if (st != SPMV_OK) {
            delete p;
            return st;
        }
        if (opts && (opts->alloc || opts->release)) {
            if (!opts->alloc || !opts->release) {
                set_error("alloc and release must be given together");
                delete p;
                return SPMV_E_INVALID;
            }
            p->alloc = opts->alloc;
            p->release = opts->release;
            p->ctx = opts->alloc_ctx;
        }
        cudaError_t e = cudaGetDevice(&p->device);
        if (e != cudaSuccess) {
            delete p;
            return cuda_fail(e, "cudaGetDevice");
        }
        HostPlan &hp = p->hp;
        DevPlan &dp = p->dp;
        const int vb = hp.dtype == SPMV_F64 ? 8 : (hp.dtype == SPMV_F32 ? 4 : 2);
        const int xb = hp.dtype == SPMV_F64 ? 8 : 4;
        const int r = hp.nrhs;

        // values in the plan's precision (round to nearest even from FP64)
        std::vector<double> v64;
        std::vector<float> v32;
        std::vector<uint16_t> v16;
        const void *vhost = nullptr;
        const size_t nelem = hp.val.size();        // stored elements (with padding)
        size_t vbytes = nelem * vb;
        if (hp.dtype == SPMV_F64) {
            vhost = hp.val.data();
        } else if (hp.dtype == SPMV_F32) {
            v32.resize(nelem);
            for (size_t q = 0; q < nelem; ++q) v32[q] = (float)hp.val[q];
            vhost = v32.data();
        } else {
            v16.resize(nelem);
            for (size_t q = 0; q < nelem; ++q) v16[q] = bf16_rne(hp.val[q]);
            vhost = v16.data();
        }

        const bool tiled = !hp.use_k1;
        const bool any_staged = tiled && hp.n_staged_tiles > 0;

        // SM-affine schedule: cut the tile sequence (tiles of a part are
        // consecutive) into one queue per SM with about equal nonzeros; the
        // long-row chunk tiles are dealt round-robin over the queues, first
        std::vector<int32_t> qbeg;
        int32_t nq = 0;
        if (tiled && (hp.flags & SPMV_FLAG_SM_AFFINE) && !hp.tiles.empty()) {
            int nsm = 0;
            e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device);
            if (e != cudaSuccess) {
                delete p;
                return cuda_fail(e, "cudaDeviceGetAttribute");
            }
            nq = std::max(1, nsm);
            auto weight = [&](const Tile &t) -> int64_t {
                if (t.kind == TILE_CHUNK) return t.e1 - t.e0;
                int64_t w = 0;
                for (int32_t v = t.vrow0; v < t.vrow0 + t.nvrows; ++v) w += hp.vrows[v].len;
                for (int32_t ch = t.chunk0; ch < t.chunk0 + t.nchunks; ++ch)
                    for (int32_t i = 0; i < 32; ++i) w += hp.slot_len[(size_t)ch * 32 + i];
                return w + 32;   // a little per-tile overhead
            };
            std::vector<std::vector<Tile>> q((size_t)nq);
            int64_t total = 0;
            std::vector<int64_t> w(hp.tiles.size());
            for (size_t i = 0; i < hp.tiles.size(); ++i) {
                w[i] = weight(hp.tiles[i]);
                if (hp.tiles[i].kind != TILE_CHUNK) total += w[i];
            }
            int32_t rr = 0;
            for (size_t i = 0; i < hp.tiles.size(); ++i)
                if (hp.tiles[i].kind == TILE_CHUNK) q[(size_t)(rr++ % nq)].push_back(hp.tiles[i]);
            int64_t acc = 0;
            for (size_t i = 0; i < hp.tiles.size(); ++i) {
                if (hp.tiles[i].kind == TILE_CHUNK) continue;
                // queue index by the tile's midpoint in the nonzero sequence
                const int64_t mid = acc + w[i] / 2;
                const int32_t k = (int32_t)std::min<int64_t>(nq - 1, total ? mid * nq / total : 0);
                q[(size_t)k].push_back(hp.tiles[i]);
                acc += w[i];
            }
            std::vector<Tile> ordered;
            ordered.reserve(hp.tiles.size());
            qbeg.assign((size_t)nq + 1, 0);
            for (int32_t k = 0; k < nq; ++k) {
                qbeg[k] = (int32_t)ordered.size();
                ordered.insert(ordered.end(), q[k].begin(), q[k].end());
            }
            qbeg[nq] = (int32_t)ordered.size();
            hp.tiles.swap(ordered);
        }

        Arena a;
        if (!tiled) add_vec(a, hp.rowptr, (const void **)&dp.rowptr);
        add_vec(a, hp.col32, (const void **)&dp.col32);
        a.add(vhost, vbytes, const_cast<void **>(&dp.val));
        if (tiled && hp.narrow_nnz + hp.delta_nnz > 0)
            add_vec(a, hp.col16, (const void **)&dp.col16);
        if (!tiled && !hp.long_rows.empty())
            add_vec(a, hp.long_rows, (const void **)&dp.long_rows);
        if (tiled) {
            add_vec(a, hp.tiles, (const void **)&dp.tiles);
            add_vec(a, hp.chunk_off, (const void **)&dp.chunk_off);
            add_vec(a, hp.chunk_mix, (const void **)&dp.chunk_mix);
            add_vec(a, hp.slot_dst, (const void **)&dp.slot_dst);
            add_vec(a, hp.slot_len, (const void **)&dp.slot_len);
            if (!hp.vrows.empty()) add_vec(a, hp.vrows, (const void **)&dp.vrows);
            if (!hp.xlist.empty()) add_vec(a, hp.xlist, (const void **)&dp.xlist);
            if (!hp.fixups.empty()) add_vec(a, hp.fixups, (const void **)&dp.fixups);
            if (hp.partial_slots > 0)
                a.add(nullptr, (size_t)hp.partial_slots * r * xb, &dp.partial);
            if (nq > 0) {
                add_vec(a, qbeg, (const void **)&dp.qbeg);
                a.add(nullptr, sizeof(int32_t) * ((size_t)nq + 1), (void **)&dp.qcount, true);
            } else if (hp.flags & SPMV_FLAG_PERSISTENT) {
                a.add(nullptr, 2 * sizeof(int32_t), (void **)&dp.ctr, true);
            }
        }
        a.add(nullptr, sizeof(int32_t), (void **)&dp.status, true);
        p->same_perm = hp.m == hp.n && hp.row_perm == hp.col_perm;
        if (!hp.row_perm.empty()) add_vec(a, hp.row_perm, (const void **)&p->d_row_perm);
        if (!hp.col_perm.empty()) add_vec(a, hp.col_perm, (const void **)&p->d_col_perm);

        p->arena_bytes = a.total;
        p->arena = dev_alloc(p, a.total);
        if (!p->arena) {
            set_error("device allocation of %zu bytes failed", a.total);
            delete p;
            return SPMV_E_NOMEM;
        }
        size_t off = 0;
        for (auto &it : a.items) {
            char *d = static_cast<char *>(p->arena) + off;
            *it.slot = d;
            if (it.host && it.bytes) {
                e = cudaMemcpy(d, it.host, it.bytes, cudaMemcpyHostToDevice);
                if (e != cudaSuccess) {
                    spmv_status s = cuda_fail(e, "upload");
                    spmv_plan_destroy(p);
                    return s;
                }
            } else if (it.zero && it.bytes) {
                e = cudaMemset(d, 0, it.bytes);
                if (e != cudaSuccess) {
                    spmv_status s = cuda_fail(e, "clear");
                    spmv_plan_destroy(p);
                    return s;
                }
            }
            off += (it.bytes + 255) & ~size_t(255);
        }

        dp.m = hp.m;
        dp.n = hp.n;
        dp.nrhs = r;
        dp.lanes = hp.lanes;
        dp.long_thresh = hp.long_thresh;
        dp.use_k1 = hp.use_k1;
        dp.n_long = (int32_t)hp.long_rows.size();
        dp.n_tiles = (int32_t)hp.tiles.size();
        dp.n_fixups = (int32_t)hp.fixups.size();
        dp.smem_bytes = any_staged ? (hp.max_staged * r * xb + 15) / 16 * 16 : 0;
        dp.nq = nq;
        dp.cta_threads = hp.cta_threads;
        dp.wait_limit = (hp.flags & SPMV_FLAG_TEST_WAIT_EXPIRES) ? 0u : (1u << 22);
        if (tiled) {
            e = cudaDeviceGetAttribute(&dp.n_sm, cudaDevAttrMultiProcessorCount, p->device);
            if (e != cudaSuccess) {
                spmv_status s = cuda_fail(e, "cudaDeviceGetAttribute");
                spmv_plan_destroy(p);
                return s;
            }
        }

        // info
        spmv_plan_info &I = p->info;
        I.m = hp.m;
        I.n = hp.n;
        I.nnz = hp.nnz;
        I.form = hp.form;
        I.K = hp.K;
        I.dtype = hp.dtype;
        I.nrhs = r;
        I.lanes = hp.lanes;
        I.tile_cols = hp.tile_cols;
        I.n_tiles = dp.n_tiles;
        I.n_staged_tiles = hp.n_staged_tiles;
        I.n_global_tiles = hp.n_global_tiles;
        I.n_chunk_tiles = hp.n_chunk_tiles;
        I.launches_per_exec = hp.m == 0 ? 0 : (tiled ? (dp.n_tiles > 0) + (dp.n_fixups > 0) : 1);
        I.smem_bytes = dp.smem_bytes;
        I.cta_threads = tiled ? hp.cta_threads : 0;
        I.delta_nnz = hp.delta_nnz;
        I.staged_entries = hp.staged_entries;
        I.list_entries = hp.list_entries;
        I.partial_slots = hp.partial_slots;
        I.fixup_rows = dp.n_fixups;
        I.device_bytes = (int64_t)a.total;
        I.compulsory_bytes = hp.nnz * (vb + 4) + ((int64_t)hp.m + 1) * 4 +
                             (int64_t)hp.n * r * xb + (int64_t)hp.m * r * xb;
        if (!tiled) {
            I.moved_bytes = I.compulsory_bytes + (int64_t)dp.n_long * 4;
        } else {
            // every element touched once: values and indices (16-bit in narrow
            // tiles and increment chunks) of the stored rows, chunk metadata,
            // tiles, staged x (+ list indices), x read directly (distinct
            // columns), y, partials, fix-ups
            std::vector<char> seen((size_t)hp.n, 0);
            int64_t gdistinct = 0;
            auto see = [&](int32_t c) {
                if (!seen[c]) {
                    seen[c] = 1;
                    ++gdistinct;
                }
            };
            for (const Tile &t : hp.tiles) {
                if (t.kind == TILE_CHUNK) {
                    for (int32_t e = t.e0; e < t.e1; ++e) see(hp.col32[e]);
                    continue;
                }
                if (t.kind == TILE_NARROW) continue;
                for (int32_t v = t.vrow0; v < t.vrow0 + t.nvrows; ++v)
                    for (int32_t k = 0; k < hp.vrows[v].len; ++k) {
                        const int32_t c = hp.col32[hp.vrows[v].e0 + k];
                        if (t.kind == TILE_MIXED) {
                            if (c < 0) see(~c);
                        } else {
                            see(c);
                        }
                    }
                for (int32_t ch = t.chunk0; ch < t.chunk0 + t.nchunks; ++ch)
                    for (int32_t i = 0; i < 32; ++i) {
                        const int32_t len = hp.slot_len[ch * 32 + i];
                        for (int32_t k = 0; k < len; ++k) {
                            const int32_t c = hp.col32[hp.chunk_off[ch] + k * 32 + i];
                            if (t.kind == TILE_MIXED) {
                                if (c < 0) see(~c);
                            } else {
                                see(c);
                            }
                        }
                    }
            }
            const int64_t short_idx = hp.narrow_nnz + hp.delta_nnz;
            I.moved_bytes = hp.nnz * vb + short_idx * 2 + (hp.nnz - short_idx) * 4 +
                            (int64_t)hp.slot_dst.size() * 8 + (int64_t)hp.chunk_off.size() * 8 +
                            (int64_t)hp.vrows.size() * 16 +
                            (int64_t)hp.tiles.size() * (int64_t)sizeof(Tile) +
                            hp.staged_entries * r * xb +
                            hp.list_entries * 4 + gdistinct * r * xb + (int64_t)hp.m * r * xb +
                            hp.partial_slots * r * xb * 2 + (int64_t)hp.fixups.size() * 16;
        }
        p->xbytes = (size_t)hp.n * r * xb;
        p->ybytes = (size_t)hp.m * r * xb;

        // the host image is no longer needed
        HostPlan meta;
        meta.m = hp.m;
        meta.n = hp.n;
        meta.nnz = hp.nnz;
        meta.form = hp.form;
        meta.K = hp.K;
        meta.dtype = hp.dtype;
        meta.nrhs = hp.nrhs;
        meta.lanes = hp.lanes;
        meta.tile_cols = hp.tile_cols;
        meta.long_thresh = hp.long_thresh;
        meta.use_k1 = hp.use_k1;
        p->hp = std::move(meta);
        *out = p;
        return SPMV_OK;
    } catch (const std::bad_alloc &) {
        set_error("out of host memory");
        if (p) spmv_plan_destroy(p);
        return SPMV_E_NOMEM;
    } catch (...) {
        set_error("internal error");
        if (p) spmv_plan_destroy(p);
        return SPMV_E_INTERNAL;
    }
}

extern "C" spmv_status spmv_exec(spmv_plan *plan, const void *x_hat, void *y_hat, void *stream)
{
    clear_error();
    if (!plan) {
        set_error("plan is NULL");
        return SPMV_E_INVALID;
    }
    if ((!x_hat && plan->info.n > 0) || (!y_hat && plan->info.m > 0)) {
        set_error("NULL vector");
        return SPMV_E_INVALID;
    }
    if (reinterpret_cast<uintptr_t>(x_hat) % 16 != 0) {
        set_error("x_hat is not 16-byte aligned");
        return SPMV_E_INVALID;
    }
    spmv_status st = device_matches(plan);
    if (st != SPMV_OK) return st;
    cudaError_t e = run(plan, x_hat, y_hat, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "spmv kernel launch");
    return SPMV_OK;
}

extern "C" spmv_status spmv_plan_check(spmv_plan *plan, void *stream)
{
    clear_error();
    if (!plan) {
        set_error("plan is NULL");
        return SPMV_E_INVALID;
    }
    spmv_status st = device_matches(plan);
    if (st != SPMV_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t flag = 0;
    cudaError_t e = cudaMemcpyAsync(&flag, plan->dp.status, sizeof(flag), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "reading the plan status");
    if (flag) {
        set_error("a bounded device wait gave up in an earlier spmv_exec: its y_hat is incomplete");
        return SPMV_E_TIMEOUT;
    }
    return SPMV_OK;
}

extern "C" spmv_status spmv_exec_host(spmv_plan *plan, const void *x_hat_host, void *y_hat_host,
                                      void *stream)
{
    clear_error();
    if (!plan) {
        set_error("plan is NULL");
        return SPMV_E_INVALID;
    }
    if ((!x_hat_host && plan->xbytes) || (!y_hat_host && plan->ybytes)) {
        set_error("NULL vector");
        return SPMV_E_INVALID;
    }
    spmv_status st = device_matches(plan);
    if (st != SPMV_OK) return st;
    if (!plan->io_x) {
        plan->io_x = dev_alloc(plan, plan->xbytes);
        plan->io_y = dev_alloc(plan, plan->ybytes);
        if (!plan->io_x || !plan->io_y) {
            set_error("device allocation of the host-I/O buffers failed");
            return SPMV_E_NOMEM;
        }
    }
    if (!plan->h_status) {
        cudaError_t e = cudaMallocHost(reinterpret_cast<void **>(&plan->h_status), sizeof(int32_t));
        if (e != cudaSuccess) {
            cudaGetLastError();
            plan->h_status = nullptr;
            set_error("pinned host allocation of the status word failed");
            return SPMV_E_NOMEM;
        }
        *plan->h_status = 0;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(plan->io_x, x_hat_host, plan->xbytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "copy of x to the device");
    e = run(plan, plan->io_x, plan->io_y, s);
    if (e != cudaSuccess) return cuda_fail(e, "spmv kernel launch");
    e = cudaMemcpyAsync(y_hat_host, plan->io_y, plan->ybytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "copy of y to the host");
    e = cudaMemcpyAsync(plan->h_status, plan->dp.status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "copy of the plan status");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    if (*plan->h_status) {
        set_error("a bounded device wait gave up: y_hat is incomplete");
        return SPMV_E_TIMEOUT;
    }
    return SPMV_OK;
}

static spmv_status permute_common(const spmv_plan *plan, const void *src, void *dst,
                                  bool is_x, void *stream)
{
    clear_error();
    if (!plan || !src || !dst) {
        set_error("NULL argument");
        return SPMV_E_INVALID;
    }
    spmv_status st = device_matches(plan);
    if (st != SPMV_OK) return st;
    const int xb = plan->info.dtype == SPMV_F64 ? 8 : 4;
    const int32_t count = is_x ? plan->info.n : plan->info.m;
    const int32_t *perm = is_x ? plan->d_col_perm : plan->d_row_perm;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (!perm) {
        e = cudaMemcpyAsync(dst, src, (size_t)count * plan->info.nrhs * xb,
                            cudaMemcpyDeviceToDevice, s);
    } else {
        e = permute_vector(xb, count, plan->info.nrhs, perm, src, dst, !is_x, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, is_x ? "permute x" : "unpermute y");
    return SPMV_OK;
}

extern "C" spmv_status spmv_permute_x(const spmv_plan *plan, const void *x, void *x_hat,
                                      void *stream)
{
    return permute_common(plan, x, x_hat, true, stream);
}

extern "C" spmv_status spmv_unpermute_y(const spmv_plan *plan, const void *y_hat, void *y,
                                        void *stream)
{
    return permute_common(plan, y_hat, y, false, stream);
}

extern "C" spmv_status spmv_plan_autotune(const spmv_csr *A, const spmv_perm *perm,
                                          const spmv_splits *splits,
                                          const spmv_opts *candidates, int32_t n_candidates,
                                          int32_t reps, void *stream, spmv_plan **out,
                                          int32_t *best, float *best_ms)
{
    clear_error();
    if (!out || !candidates || n_candidates < 1) {
        set_error("autotune needs an output and at least one candidate");
        return SPMV_E_INVALID;
    }
    *out = nullptr;
    if (reps < 1) reps = 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<spmv_plan *> plans;
    std::vector<cudaEvent_t> ev;
    void *xb = nullptr, *yb = nullptr;
    spmv_status st = SPMV_OK;
    int32_t keep_i = -1;
    float keep_ms = 0.0f;
    auto cleanup = [&](int32_t keep) {
        if (!plans.empty()) {
            cudaStreamSynchronize(s);
            dev_free(plans[0], xb);      // the scratch vectors come from the first
            dev_free(plans[0], yb);      // plan's allocator
        }
        for (size_t i = 0; i < plans.size(); ++i)
            if ((int32_t)i != keep) spmv_plan_destroy(plans[i]);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    };
    // every candidate plan is built first; then the timed calls go round
    // robin over the candidates (each call finds the caches as the previous
    // candidate left them, as in a sequence of different products) and each
    // candidate is judged by its median call
    // the candidates are built on host threads at once (each thread on the
    // caller's device); the first failure, in candidate order, is reported
    {
        int dev = 0;
        cudaError_t de = cudaGetDevice(&dev);
        if (de != cudaSuccess) return cuda_fail(de, "cudaGetDevice");
        std::vector<spmv_plan *> built((size_t)n_candidates, nullptr);
        std::vector<spmv_status> sts((size_t)n_candidates, SPMV_OK);
        std::vector<std::string> msgs((size_t)n_candidates);
        std::vector<std::thread> ts;
        for (int32_t i = 0; i < n_candidates; ++i)
            ts.emplace_back([&, i]() {
                cudaError_t e2 = cudaSetDevice(dev);
                if (e2 != cudaSuccess) {
                    sts[(size_t)i] = SPMV_E_CUDA;
                    msgs[(size_t)i] = cudaGetErrorString(e2);
                    return;
                }
                sts[(size_t)i] = spmv_plan_create(A, perm, splits, &candidates[i], &built[(size_t)i]);
                if (sts[(size_t)i] != SPMV_OK) msgs[(size_t)i] = spmv_last_error();
            });
        for (auto &t : ts) t.join();
        for (int32_t i = 0; i < n_candidates; ++i)
            if (built[(size_t)i]) plans.push_back(built[(size_t)i]);
        for (int32_t i = 0; i < n_candidates; ++i)
            if (sts[(size_t)i] != SPMV_OK) {
                cleanup(-1);
                set_error("candidate %d: %s", i, msgs[(size_t)i].c_str());
                return sts[(size_t)i];
            }
    }
    size_t xbytes = 0, ybytes = 0;
    for (int32_t j = 0; j < n_candidates; ++j) {
        const int rj = candidates[j].nrhs > 0 ? candidates[j].nrhs : 1;
        const size_t el = candidates[j].dtype == SPMV_F64 ? 8 : 4;
        xbytes = std::max(xbytes, (size_t)A->n * rj * el);
        ybytes = std::max(ybytes, (size_t)A->m * rj * el);
    }
    xb = dev_alloc(plans[0], xbytes);
    yb = dev_alloc(plans[0], ybytes);
    if (!xb || !yb) {
        set_error("device allocation for autotuning failed");
        cleanup(-1);
        return SPMV_E_NOMEM;
    }
    cudaError_t e = cudaMemsetAsync(xb, 0, xbytes, s);
    ev.assign((size_t)2 * n_candidates * reps, nullptr);
    for (size_t k = 0; k < ev.size() && e == cudaSuccess; ++k) e = cudaEventCreate(&ev[k]);
    for (int32_t i = 0; i < n_candidates && e == cudaSuccess; ++i) e = run(plans[i], xb, yb, s);
    for (int32_t k = 0; k < reps && e == cudaSuccess; ++k)
        for (int32_t i = 0; i < n_candidates && e == cudaSuccess; ++i) {
            const size_t q = 2 * ((size_t)k * n_candidates + i);
            e = cudaEventRecord(ev[q], s);
            if (e == cudaSuccess) e = run(plans[i], xb, yb, s);
            if (e == cudaSuccess) e = cudaEventRecord(ev[q + 1], s);
        }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        st = cuda_fail(e, "autotune timing");
        cleanup(-1);
        return st;
    }
    for (int32_t i = 0; i < n_candidates; ++i) {
        std::vector<float> t((size_t)reps);
        for (int32_t k = 0; k < reps && e == cudaSuccess; ++k) {
            const size_t q = 2 * ((size_t)k * n_candidates + i);
            e = cudaEventElapsedTime(&t[k], ev[q], ev[q + 1]);
        }
        if (e != cudaSuccess) {
            st = cuda_fail(e, "autotune timing");
            cleanup(-1);
            return st;
        }
        std::nth_element(t.begin(), t.begin() + reps / 2, t.end());
        const float med = t[reps / 2];
        if (keep_i < 0 || med < keep_ms) {
            keep_i = i;
            keep_ms = med;
        }
    }
    spmv_plan *keep = plans[keep_i];
    cleanup(keep_i);
    *out = keep;
    if (best) *best = keep_i;
    if (best_ms) *best_ms = keep_ms;
    return SPMV_OK;
}

extern "C" spmv_status spmv_plan_get_info(const spmv_plan *plan, spmv_plan_info *info)
{
    clear_error();
    if (!plan || !info) {
        set_error("NULL argument");
        return SPMV_E_INVALID;
    }
    *info = plan->info;
    return SPMV_OK;
}

extern "C" spmv_status spmv_plan_destroy(spmv_plan *plan)
{
    clear_error();
    if (!plan) return SPMV_OK;
    cudaError_t e = cudaSuccess;
    if (plan->arena || plan->io_x || plan->io_y) e = cudaDeviceSynchronize();
    dev_free(plan, plan->io_x);
    dev_free(plan, plan->io_y);
    dev_free(plan, plan->arena);
    if (plan->h_status) cudaFreeHost(plan->h_status);
    delete plan;
    if (e != cudaSuccess) return cuda_fail(e, "synchronize before destroy");
    return SPMV_OK;
}

// ------------------------------------------------------- permute kernels --
namespace spmv {

template <typename T>
__global__ void k_permute(int64_t total, int32_t r, const int32_t *__restrict__ perm,
                          const T *__restrict__ src, T *__restrict__ dst, bool scatter)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int64_t row = i / r, c = i - row * r;
    const int64_t other = (int64_t)perm[row] * r + c;
    if (scatter) dst[other] = src[i];
    else dst[i] = src[other];
}

cudaError_t permute_vector(int elem_bytes, int32_t count, int32_t r, const int32_t *perm,
                           const void *src, void *dst, bool scatter, cudaStream_t s)
{
    const int64_t total = (int64_t)count * r;
    if (total == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    if (elem_bytes == 8)
        k_permute<unsigned long long><<<blocks, 256, 0, s>>>(
            total, r, perm, static_cast<const unsigned long long *>(src),
            static_cast<unsigned long long *>(dst), scatter);
    else
        k_permute<unsigned int><<<blocks, 256, 0, s>>>(
            total, r, perm, static_cast<const unsigned int *>(src),
            static_cast<unsigned int *>(dst), scatter);
    return cudaGetLastError();
}

}  // namespace spmv
