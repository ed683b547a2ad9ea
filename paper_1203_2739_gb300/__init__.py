"""Python binding of the GB300 cache-size-aware SpMV library (include/spmv.h).

Argument marshalling only: every step of the product runs in the in-tree
shared library ``_build/libspmv.so`` (CUDA kernels for sm_103a and the host
plan builder / partitioner in C++).  PyTorch supplies device memory (the plan
allocates through torch's caching allocator) and streams.  There is no CPU
fallback: importing this package fails when the library has not been built.

Function names follow the C ABI:

    spmv_partition        recursive hypergraph bisection (Sec. 3.1, 3.2, 4.1)
    spmv_form_from_labels SB / DB form or split order from labels (eqs. 1-5)
    spmv_plan_create      validate, permute, split, tile, upload
    spmv_exec             y_hat <- A_hat x_hat (device tensors)
    spmv_exec_host        the same with host buffers (copies inside)
    spmv_plan_check       report a device wait that gave up (SPMV_E_TIMEOUT)
    spmv_cg_ir            mixed-precision CG with FP64 iterative refinement
    spmv_plan_create_batched  many matrices in one plan (one launch per exec)
    spmv_permute_x / spmv_unpermute_y
    spmv_plan_get_info / spmv_plan_destroy / spmv_last_error
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libspmv.so")

SPMV_OK, SPMV_E_INVALID, SPMV_E_STRUCTURE, SPMV_E_NOMEM, SPMV_E_CUDA, SPMV_E_TIMEOUT, \
    SPMV_E_UNSUPPORTED, SPMV_E_INTERNAL = range(8)
SPMV_F64, SPMV_F32, SPMV_BF16 = 0, 1, 2
SPMV_NATURAL, SPMV_SB, SPMV_DB, SPMV_SPLIT = 0, 1, 2, 3
SPMV_FLAG_NO_STAGING, SPMV_FLAG_TILED_NATURAL, SPMV_FLAG_SM_AFFINE = 1, 2, 4
SPMV_FLAG_PERSISTENT, SPMV_FLAG_STAGE = 8, 16
SPMV_FLAG_TEST_WAIT_EXPIRES = 32
SPMV_FLAG_COL_DELTA = 64
SPMV_PART_CN, SPMV_PART_ERCN, SPMV_PART_RCN, SPMV_PART_RANDOM, SPMV_PART_RN = 0, 1, 2, 3, 4
SPMV_ORDER_BFS, SPMV_ORDER_RCM, SPMV_ORDER_SBD, SPMV_ORDER_NESTED = 0, 1, 2, 3
SPMV_FIT_CSR, SPMV_FIT_X = 0, 1

STATUS_NAMES = {0: "SPMV_OK", 1: "SPMV_E_INVALID", 2: "SPMV_E_STRUCTURE", 3: "SPMV_E_NOMEM",
                4: "SPMV_E_CUDA", 5: "SPMV_E_TIMEOUT", 6: "SPMV_E_UNSUPPORTED",
                7: "SPMV_E_INTERNAL"}
DTYPE_NAMES = {SPMV_F64: "f64", SPMV_F32: "f32", SPMV_BF16: "bf16"}

# exported symbols of include/spmv.h (checked by the tests)
EXPORTS = ("spmv_plan_create", "spmv_exec", "spmv_exec_host", "spmv_permute_x",
           "spmv_unpermute_y", "spmv_plan_get_info", "spmv_plan_destroy",
           "spmv_form_from_labels", "spmv_partition", "spmv_partition_free",
           "spmv_last_error", "spmv_csr_exec_noalloc", "spmv_plan_autotune",
           "spmv_plan_check", "spmv_cg_ir", "spmv_plan_create_batched", "spmv_features",
           "spmv_mlp_param_count", "spmv_mlp_work_bytes", "spmv_mlp_forward", "spmv_mlp_grad",
           "spmv_mlp_adam", "spmv_plan_emulate", "spmv_reorder", "spmv_mlp_predict",
           "spmv_mlp_fold_scaling")
SPMV_EMULATE_STATS = 14
EMULATE_STATS = ("tiles", "chunk_tiles", "staged_tiles", "partial_slots", "fixups", "warp_rows",
                 "stored_chunk_elements", "plain_csr", "gathered_nnz", "fma_lanes",
                 "mixed_slots", "staged_entries", "two_run_tiles", "delta_nnz")
SPMV_NOALLOC_MAX_NNZ = 1073741824


class SpmvError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


# ------------------------------------------------------------- structures --
_i32p = ctypes.POINTER(ctypes.c_int32)
_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class spmv_csr(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("n", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("rowptr", _i32p), ("colidx", _i32p), ("vals", ctypes.POINTER(ctypes.c_double))]


class spmv_perm(ctypes.Structure):
    _fields_ = [("row_perm", _i32p), ("col_perm", _i32p)]


class spmv_splits(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int32), ("K", ctypes.c_int32), ("row_part_ptr", _i32p),
                ("col_part_ptr", _i32p), ("nz_part", _i32p)]


class spmv_opts(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("nrhs", ctypes.c_int32),
                ("tile_cols", ctypes.c_int32), ("tile_nnz", ctypes.c_int32),
                ("long_row", ctypes.c_int32), ("lanes", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("warp_rows", ctypes.c_int32),
                ("cta_threads", ctypes.c_int32),
                ("alloc", _ALLOC_T), ("release", _FREE_T),
                ("alloc_ctx", ctypes.c_void_p)]


class spmv_plan_info(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("n", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("form", ctypes.c_int32), ("K", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("nrhs", ctypes.c_int32), ("lanes", ctypes.c_int32),
                ("tile_cols", ctypes.c_int32), ("n_tiles", ctypes.c_int32),
                ("n_staged_tiles", ctypes.c_int32), ("n_global_tiles", ctypes.c_int32),
                ("n_chunk_tiles", ctypes.c_int32), ("launches_per_exec", ctypes.c_int32),
                ("smem_bytes", ctypes.c_int32), ("staged_entries", ctypes.c_int64),
                ("list_entries", ctypes.c_int64), ("partial_slots", ctypes.c_int64),
                ("fixup_rows", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("compulsory_bytes", ctypes.c_int64), ("moved_bytes", ctypes.c_int64),
                ("cta_threads", ctypes.c_int32), ("delta_nnz", ctypes.c_int64)]


class spmv_partition_opts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("K", ctypes.c_int32),
                ("part_bytes", ctypes.c_int64), ("fit_rule", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("imbalance", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


class spmv_partition_out(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int32), ("K", ctypes.c_int32), ("n_labels", ctypes.c_int32),
                ("labels", _i32p), ("row_perm", _i32p), ("col_perm", _i32p),
                ("row_part_ptr", _i32p), ("col_part_ptr", _i32p), ("cost", ctypes.c_int64),
                ("cost_cols", ctypes.c_int64), ("cost_rows", ctypes.c_int64),
                ("seconds", ctypes.c_double)]


class spmv_mlp(ctypes.Structure):
    _fields_ = [("nin", ctypes.c_int32), ("nh", ctypes.c_int32), ("nc", ctypes.c_int32),
                ("params", ctypes.c_void_p)]


SPMV_SEL_FEATURES = 16


class spmv_cg_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("inner_tol", ctypes.c_double),
                ("max_outer", ctypes.c_int32), ("max_inner", ctypes.c_int32)]


class spmv_cg_info(ctypes.Structure):
    _fields_ = [("outer", ctypes.c_int32), ("inner_total", ctypes.c_int32),
                ("rel_residual", ctypes.c_double), ("converged", ctypes.c_int32)]


# ---------------------------------------------------------------- library --
def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("the CUDA library %s is not built; run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    L.spmv_plan_create.argtypes = [ctypes.POINTER(spmv_csr), ctypes.POINTER(spmv_perm),
                                   ctypes.POINTER(spmv_splits), ctypes.POINTER(spmv_opts),
                                   ctypes.POINTER(vp)]
    L.spmv_exec.argtypes = [vp, vp, vp, vp]
    L.spmv_exec_host.argtypes = [vp, vp, vp, vp]
    L.spmv_plan_check.argtypes = [vp, vp]
    L.spmv_features.argtypes = [ctypes.POINTER(spmv_csr), ctypes.POINTER(ctypes.c_float)]
    L.spmv_mlp_param_count.argtypes = [ctypes.c_int32] * 3
    L.spmv_mlp_param_count.restype = ctypes.c_int64
    L.spmv_mlp_work_bytes.argtypes = [ctypes.c_int32] * 3
    L.spmv_mlp_work_bytes.restype = ctypes.c_size_t
    L.spmv_mlp_forward.argtypes = [ctypes.POINTER(spmv_mlp), vp, ctypes.c_int32, vp, vp, vp]
    L.spmv_mlp_grad.argtypes = [ctypes.POINTER(spmv_mlp), vp, vp, ctypes.c_int32, vp, vp, vp, vp]
    L.spmv_mlp_predict.argtypes = [ctypes.POINTER(spmv_mlp), vp, ctypes.c_int32, vp, vp, vp, vp]
    L.spmv_mlp_fold_scaling.argtypes = [ctypes.POINTER(spmv_mlp), vp, vp, vp]
    L.spmv_mlp_adam.argtypes = [ctypes.POINTER(spmv_mlp), vp, vp, vp, ctypes.c_int32,
                                ctypes.c_float, vp]
    L.spmv_plan_create_batched.argtypes = [ctypes.c_int32, ctypes.POINTER(spmv_csr),
                                           ctypes.POINTER(spmv_perm), ctypes.POINTER(spmv_splits),
                                           ctypes.POINTER(spmv_opts), ctypes.POINTER(vp)]
    L.spmv_cg_ir.argtypes = [vp, vp, vp, vp, ctypes.POINTER(spmv_cg_opts),
                             ctypes.POINTER(spmv_cg_info), vp]
    L.spmv_permute_x.argtypes = [vp, vp, vp, vp]
    L.spmv_unpermute_y.argtypes = [vp, vp, vp, vp]
    L.spmv_plan_get_info.argtypes = [vp, ctypes.POINTER(spmv_plan_info)]
    L.spmv_plan_destroy.argtypes = [vp]
    L.spmv_form_from_labels.argtypes = [ctypes.POINTER(spmv_csr), ctypes.c_int32,
                                        ctypes.c_int32, _i32p, _i32p, _i32p, _i32p, _i32p]
    L.spmv_reorder.argtypes = [ctypes.POINTER(spmv_csr), ctypes.c_int32, ctypes.c_int32,
                               _i32p, _i32p, _i32p]
    L.spmv_partition.argtypes = [ctypes.POINTER(spmv_csr), ctypes.POINTER(spmv_partition_opts),
                                 ctypes.POINTER(spmv_partition_out)]
    L.spmv_partition_free.argtypes = [ctypes.POINTER(spmv_partition_out)]
    L.spmv_partition_free.restype = None
    L.spmv_last_error.restype = ctypes.c_char_p
    L.spmv_csr_exec_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                        vp, vp, vp, vp, vp, vp]
    L.spmv_plan_autotune.argtypes = [ctypes.POINTER(spmv_csr), ctypes.POINTER(spmv_perm),
                                     ctypes.POINTER(spmv_splits), ctypes.POINTER(spmv_opts),
                                     ctypes.c_int32, ctypes.c_int32, vp, ctypes.POINTER(vp),
                                     ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_float)]
    L.spmv_plan_emulate.argtypes = [ctypes.POINTER(spmv_csr), ctypes.POINTER(spmv_perm),
                                    ctypes.POINTER(spmv_splits), ctypes.POINTER(spmv_opts),
                                    ctypes.c_int32, vp, vp, vp]
    for name in ("spmv_plan_create", "spmv_exec", "spmv_exec_host", "spmv_permute_x",
                 "spmv_unpermute_y", "spmv_plan_get_info", "spmv_plan_destroy",
                 "spmv_form_from_labels", "spmv_partition", "spmv_csr_exec_noalloc",
                 "spmv_plan_autotune", "spmv_plan_check", "spmv_cg_ir",
                 "spmv_plan_create_batched", "spmv_features", "spmv_mlp_forward",
                 "spmv_mlp_grad", "spmv_mlp_adam", "spmv_plan_emulate", "spmv_reorder",
                 "spmv_mlp_predict", "spmv_mlp_fold_scaling"):
        getattr(L, name).restype = ctypes.c_int
    return L


lib = _load()


def spmv_last_error():
    return lib.spmv_last_error().decode()


def _check(status):
    if status != SPMV_OK:
        raise SpmvError(status, spmv_last_error())


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_i32p)


def _csr_struct(m, n, rowptr, colidx, vals):
    rp, ci = _i32(rowptr), _i32(colidx)
    v = np.ascontiguousarray(vals if vals is not None else np.zeros(ci.size), dtype=np.float64)
    if rp.size != m + 1:
        raise ValueError("rowptr must have m+1 entries")
    s = spmv_csr(m, n, int(rp[-1]) if rp.size else 0, rp.ctypes.data_as(_i32p),
                 ci.ctypes.data_as(_i32p), v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return s, (rp, ci, v)


# --------------------------------------------------- torch device memory --
def _torch():
    import torch
    return torch


def _torch_alloc(size, ctx):
    try:
        return _torch().cuda.caching_allocator_alloc(int(size))
    except Exception:
        return None


def _torch_free(ptr, ctx):
    try:
        _torch().cuda.caching_allocator_delete(ptr)
    except Exception:
        pass


_ALLOC_CB = _ALLOC_T(_torch_alloc)
_FREE_CB = _FREE_T(_torch_free)


def _stream_handle(stream):
    if stream is None:
        return _torch().cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------------- plan --
class Plan:
    """Owner of a spmv_plan*; destroyed by spmv_plan_destroy (or on GC)."""

    def __init__(self, handle, info):
        self.handle = handle
        self.info = info

    def __del__(self):
        try:
            if self.handle:
                lib.spmv_plan_destroy(self.handle)
                self.handle = None
        except Exception:
            pass

    @property
    def xdtype(self):
        return "float64" if self.info["dtype"] == SPMV_F64 else "float32"


def spmv_plan_create(m, n, rowptr, colidx, vals, row_perm=None, col_perm=None,
                     form=SPMV_NATURAL, K=0, row_part_ptr=None, col_part_ptr=None,
                     nz_part=None, dtype=SPMV_F64, nrhs=1, tile_cols=0, tile_nnz=0,
                     long_row=0, lanes=0, flags=0, cta_threads=0, warp_rows=0,
                     allocator="torch"):
    A, keep = _csr_struct(m, n, rowptr, colidx, vals)
    rperm = None if row_perm is None else _i32(row_perm)
    cperm = None if col_perm is None else _i32(col_perm)
    perm = spmv_perm(_ptr(rperm), _ptr(cperm))
    rpp = None if row_part_ptr is None else _i32(row_part_ptr)
    cpp = None if col_part_ptr is None else _i32(col_part_ptr)
    nzp = None if nz_part is None else _i32(nz_part)
    splits = spmv_splits(form, K, _ptr(rpp), _ptr(cpp), _ptr(nzp))
    opts = spmv_opts(dtype, nrhs, tile_cols, tile_nnz, long_row, lanes, flags, warp_rows,
                     cta_threads)
    if allocator == "torch":
        opts.alloc, opts.release = _ALLOC_CB, _FREE_CB
    handle = ctypes.c_void_p()
    _check(lib.spmv_plan_create(ctypes.byref(A), ctypes.byref(perm), ctypes.byref(splits),
                                ctypes.byref(opts), ctypes.byref(handle)))
    plan = Plan(handle, None)
    plan.info = spmv_plan_get_info(plan)
    return plan


def spmv_plan_emulate(m, n, rowptr, colidx, vals, x, row_perm=None, col_perm=None,
                      form=SPMV_NATURAL, K=0, row_part_ptr=None, col_part_ptr=None,
                      nz_part=None, dtype=SPMV_F64, nrhs=1, tile_cols=0, tile_nnz=0,
                      long_row=0, lanes=0, flags=0, cta_threads=0, warp_rows=0, n_sm=0):
    """The host image spmv_plan_create would build (for n_sm SMs), evaluated
    on the host by walking it as the kernels do: (y, stats).  x: (n,) or
    (n, nrhs) float64 in the original order; y likewise (m rows).  No GPU."""
    A, keep = _csr_struct(m, n, rowptr, colidx, vals)
    rperm = None if row_perm is None else _i32(row_perm)
    cperm = None if col_perm is None else _i32(col_perm)
    perm = spmv_perm(_ptr(rperm), _ptr(cperm))
    rpp = None if row_part_ptr is None else _i32(row_part_ptr)
    cpp = None if col_part_ptr is None else _i32(col_part_ptr)
    nzp = None if nz_part is None else _i32(nz_part)
    splits = spmv_splits(form, K, _ptr(rpp), _ptr(cpp), _ptr(nzp))
    opts = spmv_opts(dtype, nrhs, tile_cols, tile_nnz, long_row, lanes, flags, warp_rows,
                     cta_threads)
    xs = np.ascontiguousarray(x, dtype=np.float64)
    if xs.size != n * max(nrhs, 1):
        raise ValueError("x has %d elements, expected %d" % (xs.size, n * max(nrhs, 1)))
    y = np.empty((m, nrhs) if xs.ndim == 2 else m, dtype=np.float64)
    stats = np.zeros(SPMV_EMULATE_STATS, dtype=np.int64)
    _check(lib.spmv_plan_emulate(ctypes.byref(A), ctypes.byref(perm), ctypes.byref(splits),
                                 ctypes.byref(opts), int(n_sm),
                                 ctypes.c_void_p(xs.ctypes.data), ctypes.c_void_p(y.ctypes.data),
                                 ctypes.c_void_p(stats.ctypes.data)))
    return y, dict(zip(EMULATE_STATS, stats.tolist()))


def spmv_plan_create_batched(mats, perms=None, nz_parts=None, K=0, dtype=SPMV_F64, nrhs=1,
                             tile_cols=0, tile_nnz=0, long_row=0, lanes=0, flags=0,
                             cta_threads=0, warp_rows=0, allocator="torch"):
    """One plan over the block-diagonal matrix of `mats` (a list of
    (m, n, rowptr, colidx, vals)); perms: None or a list of (row_perm,
    col_perm) pairs (None members = identity); nz_parts: None (natural form)
    or a list of per-matrix nonzero labels in [0, K) (split form).  x_hat and
    y_hat of the plan are the matrices' vectors back to back."""
    cnt = len(mats)
    csrs = (spmv_csr * cnt)()
    keep = []
    for b, (m, n, rp, ci, v) in enumerate(mats):
        A, k = _csr_struct(m, n, rp, ci, v)
        csrs[b] = A
        keep.append(k)
    pp = None
    if perms is not None:
        pp = (spmv_perm * cnt)()
        for b, pr in enumerate(perms):
            rperm = None if pr is None or pr[0] is None else _i32(pr[0])
            cperm = None if pr is None or pr[1] is None else _i32(pr[1])
            keep.append((rperm, cperm))
            pp[b] = spmv_perm(_ptr(rperm), _ptr(cperm))
    sp = None
    if nz_parts is not None:
        sp = (spmv_splits * cnt)()
        for b, lab in enumerate(nz_parts):
            nzp = _i32(lab)
            keep.append(nzp)
            sp[b] = spmv_splits(SPMV_SPLIT, K, None, None, _ptr(nzp))
    opts = spmv_opts(dtype, nrhs, tile_cols, tile_nnz, long_row, lanes, flags, warp_rows,
                     cta_threads)
    if allocator == "torch":
        opts.alloc, opts.release = _ALLOC_CB, _FREE_CB
    handle = ctypes.c_void_p()
    _check(lib.spmv_plan_create_batched(cnt, csrs, pp, sp, ctypes.byref(opts),
                                        ctypes.byref(handle)))
    plan = Plan(handle, None)
    plan.info = spmv_plan_get_info(plan)
    return plan


def spmv_plan_autotune(m, n, rowptr, colidx, vals, candidates, reps=5, stream=None,
                       row_perm=None, col_perm=None, form=SPMV_NATURAL, K=0,
                       row_part_ptr=None, col_part_ptr=None, nz_part=None,
                       allocator="torch"):
    """Build one plan per candidate (dicts of spmv_opts fields), time each on
    the GPU and keep the fastest.  Returns (plan, index, ms per call)."""
    A, keep = _csr_struct(m, n, rowptr, colidx, vals)
    rperm = None if row_perm is None else _i32(row_perm)
    cperm = None if col_perm is None else _i32(col_perm)
    perm = spmv_perm(_ptr(rperm), _ptr(cperm))
    rpp = None if row_part_ptr is None else _i32(row_part_ptr)
    cpp = None if col_part_ptr is None else _i32(col_part_ptr)
    nzp = None if nz_part is None else _i32(nz_part)
    splits = spmv_splits(form, K, _ptr(rpp), _ptr(cpp), _ptr(nzp))
    arr = (spmv_opts * len(candidates))()
    for i, c in enumerate(candidates):
        o = arr[i]
        for k in ("dtype", "nrhs", "tile_cols", "tile_nnz", "long_row", "lanes", "flags",
                  "warp_rows", "cta_threads"):
            setattr(o, k, int(c.get(k, 0)))
        if allocator == "torch":
            o.alloc, o.release = _ALLOC_CB, _FREE_CB
    handle = ctypes.c_void_p()
    best = ctypes.c_int32(-1)
    ms = ctypes.c_float(0.0)
    _check(lib.spmv_plan_autotune(ctypes.byref(A), ctypes.byref(perm), ctypes.byref(splits), arr,
                                  len(candidates), reps, ctypes.c_void_p(_stream_handle(stream)),
                                  ctypes.byref(handle), ctypes.byref(best), ctypes.byref(ms)))
    plan = Plan(handle, None)
    plan.info = spmv_plan_get_info(plan)
    return plan, best.value, ms.value


def spmv_plan_get_info(plan):
    info = spmv_plan_info()
    _check(lib.spmv_plan_get_info(plan.handle, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in spmv_plan_info._fields_}


def spmv_plan_destroy(plan):
    if plan.handle:
        h, plan.handle = plan.handle, None
        _check(lib.spmv_plan_destroy(h))


def _check_vec(plan, t, rows, what):
    torch = _torch()
    want = torch.float64 if plan.info["dtype"] == SPMV_F64 else torch.float32
    if not t.is_cuda or t.dtype != want or not t.is_contiguous():
        raise ValueError("%s must be a contiguous CUDA %s tensor" % (what, want))
    if t.numel() != rows * plan.info["nrhs"]:
        raise ValueError("%s has %d elements, expected %d" % (what, t.numel(),
                                                              rows * plan.info["nrhs"]))


def spmv_exec(plan, x_hat, y_hat, stream=None):
    """y_hat <- A_hat x_hat on device tensors (float64 for F64 plans, float32
    otherwise), on `stream` (default: torch's current stream)."""
    _check_vec(plan, x_hat, plan.info["n"], "x_hat")
    _check_vec(plan, y_hat, plan.info["m"], "y_hat")
    _check(lib.spmv_exec(plan.handle, ctypes.c_void_p(x_hat.data_ptr()),
                         ctypes.c_void_p(y_hat.data_ptr()), ctypes.c_void_p(_stream_handle(stream))))


def spmv_plan_check(plan, stream=None):
    """Synchronise `stream` and raise SpmvError (SPMV_E_TIMEOUT) if a bounded
    device wait of an earlier spmv_exec of the plan gave up."""
    _check(lib.spmv_plan_check(plan.handle, ctypes.c_void_p(_stream_handle(stream))))


def spmv_cg_ir(low, f64, b, x, tol=0.0, inner_tol=0.0, max_outer=0, max_inner=0,
               stream=None):
    """Solve A x = b (A symmetric positive definite) by CG with iterative
    refinement: inner products with plan `low`, FP64 residuals with plan
    `f64` (same matrix and permutations).  b, x: float64 CUDA tensors of n
    entries in the original order; x is the initial guess and receives the
    solution.  Returns the solver's info as a dict."""
    torch = _torch()
    n = low.info["n"]
    for t, what in ((b, "b"), (x, "x")):
        if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != n:
            raise ValueError("%s must be a contiguous CUDA float64 tensor of %d entries"
                             % (what, n))
    o = spmv_cg_opts(tol, inner_tol, max_outer, max_inner)
    info = spmv_cg_info()
    _check(lib.spmv_cg_ir(low.handle, f64.handle, ctypes.c_void_p(b.data_ptr()),
                          ctypes.c_void_p(x.data_ptr()), ctypes.byref(o), ctypes.byref(info),
                          ctypes.c_void_p(_stream_handle(stream))))
    return {"outer": info.outer, "inner_total": info.inner_total,
            "rel_residual": info.rel_residual, "converged": bool(info.converged)}


def spmv_features(m, n, rowptr, colidx):
    """The selector's SPMV_SEL_FEATURES features of a CSR matrix (host)."""
    A, keep = _csr_struct(m, n, rowptr, colidx, None)
    out = (ctypes.c_float * SPMV_SEL_FEATURES)()
    _check(lib.spmv_features(ctypes.byref(A), out))
    return np.array(out[:], dtype=np.float32)


def spmv_mlp_param_count(nin, nh, nc):
    return int(lib.spmv_mlp_param_count(nin, nh, nc))


def spmv_mlp_work_bytes(nh, nc, batch):
    return int(lib.spmv_mlp_work_bytes(nh, nc, batch))


def _net(params, nin, nh, nc):
    torch = _torch()
    if (not params.is_cuda or params.dtype != torch.float32 or not params.is_contiguous()
            or params.numel() != spmv_mlp_param_count(nin, nh, nc)):
        raise ValueError("params must be a contiguous CUDA float32 tensor of "
                         "spmv_mlp_param_count(nin, nh, nc) entries")
    return spmv_mlp(nin, nh, nc, params.data_ptr())


def spmv_mlp_predict(params, nin, nh, nc, X, cls, conf, work, stream=None):
    """cls (int32) and conf (float32) per row of X: the network's class and
    its softmax probability, computed by the library's kernels."""
    net = _net(params, nin, nh, nc)
    vp = ctypes.c_void_p
    _check(lib.spmv_mlp_predict(ctypes.byref(net), vp(X.data_ptr()), X.shape[0],
                                vp(cls.data_ptr()), vp(conf.data_ptr()), vp(work.data_ptr()),
                                vp(_stream_handle(stream))))


def spmv_mlp_fold_scaling(params, nin, nh, nc, mu, sd, stream=None):
    """Fold (x - mu) / sd into the first layer (device float32 tensors)."""
    net = _net(params, nin, nh, nc)
    vp = ctypes.c_void_p
    _check(lib.spmv_mlp_fold_scaling(ctypes.byref(net), vp(mu.data_ptr()), vp(sd.data_ptr()),
                                     vp(_stream_handle(stream))))


def spmv_mlp_forward(params, nin, nh, nc, X, logits, work, stream=None):
    """logits (batch x nc) = net(X); float32 CUDA tensors; work: a CUDA byte
    tensor of at least spmv_mlp_work_bytes(nh, nc, batch)."""
    net = _net(params, nin, nh, nc)
    _check(lib.spmv_mlp_forward(ctypes.byref(net), ctypes.c_void_p(X.data_ptr()), X.shape[0],
                                ctypes.c_void_p(logits.data_ptr()),
                                ctypes.c_void_p(work.data_ptr()),
                                ctypes.c_void_p(_stream_handle(stream))))


def spmv_mlp_grad(params, nin, nh, nc, X, labels, grads, loss, work, stream=None):
    """Gradient of the mean softmax cross-entropy into grads (like params) and
    the loss into loss (one float); labels: int32 CUDA tensor."""
    net = _net(params, nin, nh, nc)
    _check(lib.spmv_mlp_grad(ctypes.byref(net), ctypes.c_void_p(X.data_ptr()),
                             ctypes.c_void_p(labels.data_ptr()), X.shape[0],
                             ctypes.c_void_p(grads.data_ptr()), ctypes.c_void_p(loss.data_ptr()),
                             ctypes.c_void_p(work.data_ptr()),
                             ctypes.c_void_p(_stream_handle(stream))))


def spmv_mlp_adam(params, nin, nh, nc, grads, m, v, step, lr, stream=None):
    net = _net(params, nin, nh, nc)
    _check(lib.spmv_mlp_adam(ctypes.byref(net), ctypes.c_void_p(grads.data_ptr()),
                             ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                             int(step), float(lr), ctypes.c_void_p(_stream_handle(stream))))


def _host_ptr(a, rows, plan, what):
    want = np.float64 if plan.info["dtype"] == SPMV_F64 else np.float32
    if hasattr(a, "data_ptr"):          # torch CPU tensor (pinned for DMA)
        if a.is_cuda or a.numel() != rows * plan.info["nrhs"] or not a.is_contiguous():
            raise ValueError("%s must be a contiguous host tensor of %d elements" % (what, rows))
        if (a.element_size() != np.dtype(want).itemsize):
            raise ValueError("%s has the wrong dtype" % what)
        return ctypes.c_void_p(a.data_ptr())
    if not (isinstance(a, np.ndarray) and a.dtype == want and a.flags.c_contiguous
            and a.size == rows * plan.info["nrhs"]):
        raise ValueError("%s must be a contiguous %s array of %d elements" % (what, want, rows))
    return ctypes.c_void_p(a.ctypes.data)


def spmv_exec_host(plan, x_hat_host, y_hat_host, stream=None):
    """spmv_exec with host buffers (copies in and out, synchronises)."""
    xp = _host_ptr(x_hat_host, plan.info["n"], plan, "x_hat_host")
    yp = _host_ptr(y_hat_host, plan.info["m"], plan, "y_hat_host")
    _check(lib.spmv_exec_host(plan.handle, xp, yp, ctypes.c_void_p(_stream_handle(stream))))


def spmv_permute_x(plan, x, x_hat, stream=None):
    _check_vec(plan, x, plan.info["n"], "x")
    _check_vec(plan, x_hat, plan.info["n"], "x_hat")
    _check(lib.spmv_permute_x(plan.handle, ctypes.c_void_p(x.data_ptr()),
                              ctypes.c_void_p(x_hat.data_ptr()),
                              ctypes.c_void_p(_stream_handle(stream))))


def spmv_unpermute_y(plan, y_hat, y, stream=None):
    _check_vec(plan, y_hat, plan.info["m"], "y_hat")
    _check_vec(plan, y, plan.info["m"], "y")
    _check(lib.spmv_unpermute_y(plan.handle, ctypes.c_void_p(y_hat.data_ptr()),
                                ctypes.c_void_p(y.data_ptr()),
                                ctypes.c_void_p(_stream_handle(stream))))


def spmv_csr_exec_noalloc(m, n, rowptr, colidx, vals, x, y, stream=None):
    """y = A x for a CSR matrix held in device tensors (int32 rowptr/colidx,
    float64 vals, x, y), through the entry point that allocates nothing: for
    callers that cannot allocate device memory at this point.  Partial sums
    use the library's fixed scratch array; overlapping calls race."""
    torch = _torch()
    for t, dt, cnt, what in ((rowptr, torch.int32, m + 1, "rowptr"),
                             (colidx, torch.int32, None, "colidx"),
                             (vals, torch.float64, None, "vals"),
                             (x, torch.float64, n, "x"), (y, torch.float64, m, "y")):
        if not t.is_cuda or t.dtype != dt or not t.is_contiguous():
            raise ValueError("%s must be a contiguous CUDA %s tensor" % (what, dt))
        if cnt is not None and t.numel() != cnt:
            raise ValueError("%s has %d elements, expected %d" % (what, t.numel(), cnt))
    nnz = colidx.numel()
    if vals.numel() != nnz:
        raise ValueError("vals and colidx differ in length")
    vp = ctypes.c_void_p
    _check(lib.spmv_csr_exec_noalloc(m, n, nnz, vp(rowptr.data_ptr()), vp(colidx.data_ptr()),
                                     vp(vals.data_ptr()), vp(x.data_ptr()), vp(y.data_ptr()),
                                     vp(_stream_handle(stream))))


# ---------------------------------------------------- host preprocessing --
def spmv_form_from_labels(m, n, rowptr, colidx, form, K, labels):
    A, keep = _csr_struct(m, n, rowptr, colidx, None)
    lab = _i32(labels)
    rperm = np.empty(m, dtype=np.int32)
    cperm = np.empty(n, dtype=np.int32)
    rpp = np.empty(K + 2, dtype=np.int32)
    cpp = np.empty(K + 2, dtype=np.int32)
    _check(lib.spmv_form_from_labels(ctypes.byref(A), form, K, _ptr(lab), _ptr(rperm),
                                     _ptr(cperm), _ptr(rpp), _ptr(cpp)))
    return rperm, cperm, rpp, cpp


def spmv_reorder(m, n, rowptr, colidx, method, K=0, labels=None):
    """Row and column orders of the comparison methods (sBFS, sRCM, and the
    nested separated block-diagonal order of sHP_RN from column labels) and
    the nested border order of SB / DB forms (from row labels):
    (row_perm, col_perm), new -> old."""
    A, keep = _csr_struct(m, n, rowptr, colidx, None)
    lab = None if labels is None else _i32(labels)
    rperm = np.empty(m, dtype=np.int32)
    cperm = np.empty(n, dtype=np.int32)
    _check(lib.spmv_reorder(ctypes.byref(A), method, K, _ptr(lab), _ptr(rperm), _ptr(cperm)))
    return rperm, cperm


def spmv_partition(m, n, rowptr, colidx, method, K=0, part_bytes=0, fit_rule=SPMV_FIT_CSR,
                   seed=0, threads=0, imbalance=0.0):
    """Recursive hypergraph bisection; returns a dict with labels, perms,
    part pointers, the form, K and the reported cost."""
    A, keep = _csr_struct(m, n, rowptr, colidx, None)
    opts = spmv_partition_opts(method, K, part_bytes, fit_rule, threads, imbalance, seed)
    out = spmv_partition_out()
    _check(lib.spmv_partition(ctypes.byref(A), ctypes.byref(opts), ctypes.byref(out)))
    try:
        Kp = out.K

        def arr(p, size):
            return np.ctypeslib.as_array(p, shape=(size,)).copy() if size else \
                np.zeros(0, dtype=np.int32)
        res = dict(form=out.form, K=Kp, labels=arr(out.labels, out.n_labels),
                   row_perm=arr(out.row_perm, m), col_perm=arr(out.col_perm, n),
                   row_part_ptr=arr(out.row_part_ptr, Kp + 2),
                   col_part_ptr=arr(out.col_part_ptr, Kp + 2), cost=out.cost,
                   cost_cols=out.cost_cols, cost_rows=out.cost_rows, seconds=out.seconds)
    finally:
        lib.spmv_partition_free(ctypes.byref(out))
    return res
