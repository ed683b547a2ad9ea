"""CPU oracle for the cache-size-aware SpMxV method (test infrastructure).

Plain, slow, obviously correct FP64 code written from the paper (Akbudak,
Kayaaslan, Aykanat, "Analyzing and enhancing OSKI for sparse matrix-vector
multiplication").  It exists to check the CUDA path and shares no code with it:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The product library never loads it.

What each function restates (the C file ``ref.c`` holds the loops):

* ``spmv``            y = A x from the CSR definition (Sec. 2.1), Neumaier
                      compensated FP64 sums; also returns (|A||x|)_i.
* ``spmv_plain``      the plain CSR loop of Sec. 2.1 (the timed CPU baseline,
                      OpenMP over the host's cores when built with it).
* ``permute``         A_hat = P_r A P_c (Sec. 3).
* ``form_rows``       SB form, eqs. (1)-(3); DB form, eq. (5), from row labels.
* ``form_split``      row/column order of a split by first-touching part (Sec. 4).
* ``split_parts``     GCSR of each A^k (Sec. 4 and Sec. 5.2).
* ``lambda_rows``     lambda(c_j) (eq. 3), lambda'(c_j) (eq. 5).
* ``lambda_split``    lambda(r_i), lambda(c_j) of a split (Sec. 4.1).
* ``bound_sb/db/split``  the right-hand sides of eqs. (4), (6), Theorem 3, (7).
* ``check_structure`` no nonzero outside the diagonal blocks and borders.
* ``part_bytes``/``fits``  the "fits into the cache" predicate (Sec. 3, Sec. 5.1).
* ``cachesim_*``      fully associative LRU cache misses of the CSR access order.
* ``cg``              FP64 conjugate gradients.

Two plain-Python modules sit beside it: ``order.py`` (the comparison orders
sBFS, sRCM and sHP_RN of Sec. 5.1, and the nested order of the SB / DB
border) and ``icsr.py`` (ICSR's colDiff and rowJump, Sec. 2.1, with the
product loop over them), pinned in ``tests/test_orders.py`` and
``tests/test_icsr_oracle.py``.

Pins (``tests/test_oracle_pins.py``, run with ``-m "not gpu"``): brute-force
dense products with exact integer data, the Laplacian's closed-form
eigenvectors and row sums, exact permutation and split identities,
hand-worked fixtures in ``tests/golden`` for the forms, the bounds, the LRU
simulator and the Table 1 byte accounting, and the theorems' bounds as
invariants of the simulator.  The bounds' proofs are not in the paper, so
beyond that invariant check the theorems themselves are parity unpinned.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.ref_spmv.argtypes = [_i32, _i64p, _i32p, _f64p, _f64p, _i32, _f64p, ctypes.c_void_p]
        L.ref_spmv.restype = None
        L.ref_spmv_plain.argtypes = [_i32, _i64p, _i32p, _f64p, _f64p, _f64p, _i32]
        L.ref_spmv_plain.restype = None
        L.ref_plain_max_threads.argtypes = []
        L.ref_plain_max_threads.restype = _i32
        L.ref_is_perm.argtypes = [_i32, _i32p]
        L.ref_is_perm.restype = _i32
        L.ref_permute_csr.argtypes = [_i32, _i32, _i64p, _i32p, _f64p, _i32p, _i32p,
                                      _i64p, _i32p, _f64p]
        L.ref_permute_csr.restype = None
        L.ref_lambda_rows.argtypes = [_i32, _i32, _i64p, _i32p, _i32, _i32p, _i32p, _i32p]
        L.ref_lambda_rows.restype = None
        L.ref_lambda_split.argtypes = [_i32, _i32, _i64p, _i32p, _i32, _i32p, _i32p, _i32p]
        L.ref_lambda_split.restype = None
        L.ref_form_rows.argtypes = [_i32, _i32, _i64p, _i32p, _i32, _i32p, _i32,
                                    _i32p, _i32p, _i32p, _i32p]
        L.ref_form_rows.restype = _i32
        L.ref_form_split.argtypes = [_i32, _i32, _i64p, _i32p, _i32, _i32p,
                                     _i32p, _i32p, _i32p, _i32p]
        L.ref_form_split.restype = _i32
        L.ref_split_parts.argtypes = [_i32, _i64p, _i32, _i32p, _i64p, _i32p, _i64p, _i64p]
        L.ref_split_parts.restype = _i64
        L.ref_check_structure.argtypes = [_i32, _i32, _i64p, _i32p, _i32p, _i32p, _i32,
                                          _i32p, _i32p, _i32p]
        L.ref_check_structure.restype = _i64
        L.ref_cachesim_csr.argtypes = [_i32, _i64p, _i32p, _i64, _i64, _i64p]
        L.ref_cachesim_csr.restype = None
        L.ref_cachesim_gcsr.argtypes = [_i64, _i32p, _i64p, _i32p, _i64, _i64, _i64p]
        L.ref_cachesim_gcsr.restype = None
        L.ref_cachesim_trace.argtypes = [_i64, _i32p, _i64p, _i64, _i64, _i64p]
        L.ref_cachesim_trace.restype = None
        L.ref_cg.argtypes = [_i32, _i64p, _i32p, _f64p, _f64p, _f64p, ctypes.c_double,
                             _i32, ctypes.POINTER(ctypes.c_double)]
        L.ref_cg.restype = _i32
        L.ref_mlp_loss_grad.argtypes = [_i32, _i32, _i32, _i32, _f64p, _i32p] + [_f64p] * 13
        L.ref_mlp_loss_grad.restype = ctypes.c_double
        _lib = L
    return _lib


def _csr(rowptr, colidx, vals=None):
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(colidx, dtype=np.int32)
    if vals is None:
        return rp, ci
    return rp, ci, np.ascontiguousarray(vals, dtype=np.float64)


# ------------------------------------------------------------------ SpMV ---

def spmv(m, n, rowptr, colidx, vals, x):
    """y = A x and (|A||x|) in FP64 (Sec. 2.1).  x is (n,) or (n, r)."""
    rp, ci, v = _csr(rowptr, colidx, vals)
    x = np.ascontiguousarray(x, dtype=np.float64)
    r = 1 if x.ndim == 1 else x.shape[1]
    if x.shape[0] != n:
        raise ValueError("x has wrong length")
    y = np.empty((m, r) if x.ndim == 2 else m, dtype=np.float64)
    a = np.empty_like(y)
    lib().ref_spmv(m, rp, ci, v, x.reshape(-1), r, y.reshape(-1),
                   a.ctypes.data_as(ctypes.c_void_p))
    return y, a


def spmv_plain(m, rowptr, colidx, vals, x, threads=1, out=None):
    """The plain CSR loop of Sec. 2.1 (one FP64 running sum per row, no
    compensation): the timed CPU baseline.  threads > 1 uses OpenMP when the
    oracle was built with it.  rowptr must already be int64, colidx int32 and
    vals / x float64 (no conversion inside the timed call)."""
    y = np.empty(m, dtype=np.float64) if out is None else out
    lib().ref_spmv_plain(m, rowptr, colidx, vals, x, y, int(threads))
    return y


def plain_max_threads():
    """Threads spmv_plain can use (1 when the oracle was built without OpenMP)."""
    return int(lib().ref_plain_max_threads())


def spmv_rows(rowptr, colidx, vals, x, rows):
    """y_i for a sample of rows only (for full-size parity checks)."""
    rows = np.asarray(rows, dtype=np.int64)
    rp = np.asarray(rowptr, dtype=np.int64)
    starts, ends = rp[rows], rp[rows + 1]
    sub_rp = np.zeros(rows.size + 1, dtype=np.int64)
    np.cumsum(ends - starts, out=sub_rp[1:])
    idx = np.concatenate([np.arange(s, e) for s, e in zip(starts, ends)]) \
        if rows.size else np.zeros(0, dtype=np.int64)
    return spmv(rows.size, np.asarray(x).shape[0], sub_rp,
                np.asarray(colidx)[idx], np.asarray(vals)[idx], x)


# --------------------------------------------------------- permutations ---

def is_perm(perm):
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    return bool(lib().ref_is_perm(perm.size, perm))


def permute(m, n, rowptr, colidx, vals, row_perm, col_perm):
    """A_hat = P_r A P_c with perms new -> old (Sec. 3)."""
    rp, ci, v = _csr(rowptr, colidx, vals)
    orp = np.empty(m + 1, dtype=np.int64)
    oci = np.empty(ci.size, dtype=np.int32)
    ov = np.empty(ci.size, dtype=np.float64)
    lib().ref_permute_csr(m, n, rp, ci, v, np.ascontiguousarray(row_perm, dtype=np.int32),
                          np.ascontiguousarray(col_perm, dtype=np.int32), orp, oci, ov)
    return orp, oci, ov


# -------------------------------------------------------- connectivity ---

def lambda_rows(m, n, rowptr, colidx, K, labels):
    rp, ci = _csr(rowptr, colidx)
    lam = np.empty(n, dtype=np.int32)
    one = np.empty(n, dtype=np.int32)
    lib().ref_lambda_rows(m, n, rp, ci, K, np.ascontiguousarray(labels, dtype=np.int32), lam, one)
    return lam, one


def lambda_split(m, n, rowptr, colidx, K, nz_part):
    rp, ci = _csr(rowptr, colidx)
    lr = np.empty(m, dtype=np.int32)
    lc = np.empty(n, dtype=np.int32)
    lib().ref_lambda_split(m, n, rp, ci, K, np.ascontiguousarray(nz_part, dtype=np.int32), lr, lc)
    return lr, lc


# ----------------------------------------------------------------- forms ---

def form_rows(m, n, rowptr, colidx, K, labels, border=False):
    """SB (eq. 1) or DB (eq. 5) form from row labels; label K = row border."""
    rp, ci = _csr(rowptr, colidx)
    rperm = np.empty(m, dtype=np.int32)
    cperm = np.empty(n, dtype=np.int32)
    rptr = np.empty(K + 2, dtype=np.int32)
    cptr = np.empty(K + 2, dtype=np.int32)
    rc = lib().ref_form_rows(m, n, rp, ci, K, np.ascontiguousarray(labels, dtype=np.int32),
                             1 if border else 0, rperm, cperm, rptr, cptr)
    if rc != 0:
        raise ValueError("label out of range")
    return rperm, cperm, rptr, cptr


def form_split(m, n, rowptr, colidx, K, nz_part):
    """Row/column order of a split by first-touching part (Sec. 4)."""
    rp, ci = _csr(rowptr, colidx)
    rperm = np.empty(m, dtype=np.int32)
    cperm = np.empty(n, dtype=np.int32)
    rptr = np.empty(K + 2, dtype=np.int32)
    cptr = np.empty(K + 2, dtype=np.int32)
    rc = lib().ref_form_split(m, n, rp, ci, K, np.ascontiguousarray(nz_part, dtype=np.int32),
                              rperm, cperm, rptr, cptr)
    if rc != 0:
        raise ValueError("label out of range")
    return rperm, cperm, rptr, cptr


def split_parts(m, rowptr, K, nz_part):
    """GCSR of each A^k: (part_row_ptr, part_rows, gcsr_ptr, nz_pos)."""
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    nnz = int(rp[-1])
    prp = np.empty(K + 1, dtype=np.int64)
    prows = np.empty(max(nnz, 1), dtype=np.int32)
    gptr = np.empty(max(nnz, 1) + 1, dtype=np.int64)
    pos = np.empty(max(nnz, 1), dtype=np.int64)
    total = lib().ref_split_parts(m, rp, K, np.ascontiguousarray(nz_part, dtype=np.int32),
                                  prp, prows, gptr, pos)
    return prp, prows[:total].copy(), gptr[:total + 1].copy(), pos[:nnz].copy()


def check_structure(m, n, rowptr, colidx, row_perm, col_perm, K, row_part_ptr, col_part_ptr):
    """Number of nonzeros of R_k outside C_k and C_B, and the first one."""
    rp, ci = _csr(rowptr, colidx)
    first = np.empty(2, dtype=np.int32)
    bad = lib().ref_check_structure(
        m, n, rp, ci, np.ascontiguousarray(row_perm, dtype=np.int32),
        np.ascontiguousarray(col_perm, dtype=np.int32), K,
        np.ascontiguousarray(row_part_ptr, dtype=np.int32),
        np.ascontiguousarray(col_part_ptr, dtype=np.int32), first)
    return int(bad), (int(first[0]), int(first[1]))


# ---------------------------------------------------------------- bounds ---

def bound_sb(m, n, rowptr, colidx, K, labels):
    """Right-hand side of eq. (4): sum_j lambda(c_j)."""
    lam, _ = lambda_rows(m, n, rowptr, colidx, K, labels)
    return int(lam.astype(np.int64).sum())


def bound_db(m, n, rowptr, colidx, K, labels):
    """Right-hand side of eq. (6): sum over A'_SB columns of lambda'(c_j) plus
    the nonzeros of the row border R_B (rows labelled K)."""
    lam, _ = lambda_rows(m, n, rowptr, colidx, K, labels)
    rp = np.asarray(rowptr, dtype=np.int64)
    border = np.asarray(labels) == K
    return int(lam.astype(np.int64).sum()) + int((rp[1:] - rp[:-1])[border].sum())


def bound_split(m, n, rowptr, colidx, K, nz_part):
    """Theorem 3 / eq. (7): (sum_j lambda(c_j), sum_i lambda(r_i))."""
    lr, lc = lambda_split(m, n, rowptr, colidx, K, nz_part)
    return int(lc.astype(np.int64).sum()), int(lr.astype(np.int64).sum())


# -------------------------------------------------------------- fitting ---

def part_bytes(rows, nnz, cols, gcsr=False, vb=8, ib=4, xb=8, yb=8):
    """CSR storage of a submatrix together with its x and y subvectors
    (Sec. 3; Sec. 5.1): values + column indices + row starts + x + y, plus
    one row index per non-empty row for GCSR."""
    size = nnz * (vb + ib) + (rows + 1) * 4 + cols * xb + rows * yb
    if gcsr:
        size += rows * 4
    return size


def fits(size, cache_bytes):
    """"Smaller than the size of the cache": strict."""
    return size < cache_bytes


# ------------------------------------------------------- cache simulator ---

ARRAYS = ("rowptr", "col", "val", "x", "y", "rowlist")


def cachesim_csr(m, rowptr, colidx, cache_bytes, line_bytes=8):
    rp, ci = _csr(rowptr, colidx)
    out = np.zeros(6, dtype=np.int64)
    lib().ref_cachesim_csr(m, rp, ci, cache_bytes, line_bytes, out)
    return dict(zip(ARRAYS, out.tolist()))


def cachesim_gcsr(part_rows, gcsr_ptr, gcsr_col, cache_bytes, line_bytes=8):
    pr = np.ascontiguousarray(part_rows, dtype=np.int32)
    gp = np.ascontiguousarray(gcsr_ptr, dtype=np.int64)
    gc = np.ascontiguousarray(gcsr_col, dtype=np.int32)
    out = np.zeros(6, dtype=np.int64)
    lib().ref_cachesim_gcsr(pr.size, pr, gp, gc, cache_bytes, line_bytes, out)
    return dict(zip(ARRAYS, out.tolist()))


def cachesim_trace(arrays, indices, cache_bytes, line_bytes=8):
    a = np.ascontiguousarray(arrays, dtype=np.int32)
    i = np.ascontiguousarray(indices, dtype=np.int64)
    out = np.zeros(6, dtype=np.int64)
    lib().ref_cachesim_trace(a.size, a, i, cache_bytes, line_bytes, out)
    return out


# -------------------------------------------------------------------- CG ---

def cg(n, rowptr, colidx, vals, b, x0=None, tol=1e-10, maxit=10000):
    rp, ci, v = _csr(rowptr, colidx, vals)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    rel = ctypes.c_double(0.0)
    it = lib().ref_cg(n, rp, ci, v, np.ascontiguousarray(b, dtype=np.float64), x, tol, maxit,
                      ctypes.byref(rel))
    return x, int(it), rel.value


def mlp_loss_grad(X, labels, params, grads=True):
    """Selector network (extension): params = (W1, b1, W2, b2, W3, b3) with
    W row major [out][in]; returns (loss, logits, grads or None), FP64."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    W1, b1, W2, b2, W3, b3 = [np.ascontiguousarray(p, dtype=np.float64) for p in params]
    batch, nin = X.shape
    nh, nc = W1.shape[0], W3.shape[0]
    logits = np.zeros((batch, nc))
    g = [np.zeros_like(p) for p in (W1, b1, W2, b2, W3, b3)]
    loss = lib().ref_mlp_loss_grad(batch, nin, nh, nc, X, labels, W1, b1, W2, b2, W3, b3,
                                   *g, logits)
    return loss, logits, (g if grads else None)

