"""Seeded synthetic input generators.

This module builds the sparse matrices, vectors, permutations and random labels
that both the CPU oracle and the CUDA path are fed.  It holds none of the
method's arithmetic: no SpMV, no form derivation, no connectivity counting, no
partitioning.  Every generator returns plain numpy arrays:

    rowptr  int32[m+1]   CSR row starts
    colidx  int32[nnz]   column indices, sorted and unique within each row
    vals    float64[nnz] values

Workload recipes (the paper's 17 University of Florida matrices are not
available; these families span the same regimes of row/column irregularity as
Table 1 of the paper):

* ``zipf_matrix``: 16,384^2, row degree d ~ P(d) proportional to d^-1.7498 on
  [1, 512] (mean 8.000, max 512), columns drawn from a Zipf(s=1.2) law over a
  seeded random permutation of the columns, without replacement inside a row.
* ``mesh5``: 5-point stencil on an nx x nx grid, values U(-1,1), symmetric
  random permutation.
* ``rmat``: R-MAT (a,b,c,d) = (.57,.19,.19,.05) on 2^scale vertices, exactly
  deg * 2^scale distinct (i,j) pairs, values U(-1,1).
* ``blocks``: nb diagonal bs x bs blocks at a given fill plus a fraction of
  random off-block nonzeros, symmetric random permutation.
* ``laplacian3d``: 7-point Dirichlet Laplacian on an n^3 grid (6 / -1),
  optionally symmetrically permuted (stays SPD).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "coo_to_csr", "zipf_matrix", "mesh5", "rmat", "blocks", "laplacian3d",
    "random_perm", "uniform_x", "integer_x", "integer_values", "random_labels",
    "random_sparse", "symmetric_permute", "csr_to_dense",
]


def _rng(seed):
    return np.random.default_rng(np.random.SeedSequence(int(seed)))


def coo_to_csr(m, n, rows, cols, vals):
    """Assemble CSR from COO triplets with unique (row, col) pairs."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    key = rows * np.int64(n) + cols
    order = np.argsort(key, kind="stable")
    key_sorted = key[order]
    if key_sorted.size > 1 and np.any(key_sorted[1:] == key_sorted[:-1]):
        raise ValueError("duplicate (row, col) pair in COO input")
    r = rows[order]
    counts = np.bincount(r, minlength=m)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32 row pointers")
    return (rowptr.astype(np.int32), cols[order].astype(np.int32),
            vals[order].copy())


def csr_to_dense(m, n, rowptr, colidx, vals):
    a = np.zeros((m, n), dtype=np.float64)
    for i in range(m):
        for p in range(rowptr[i], rowptr[i + 1]):
            a[i, colidx[p]] += vals[p]
    return a


def random_perm(n, seed):
    return _rng(seed).permutation(n).astype(np.int32)


def symmetric_permute(m, rowptr, colidx, vals, perm):
    """Return P A P^T in CSR, where perm maps new index -> old index."""
    perm = np.asarray(perm, dtype=np.int64)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size, dtype=np.int64)
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(rowptr))
    return coo_to_csr(m, m, inv[rows], inv[colidx.astype(np.int64)], vals)


def uniform_x(n, seed, nrhs=1):
    x = _rng(seed).uniform(-1.0, 1.0, size=(n, nrhs) if nrhs > 1 else n)
    return np.ascontiguousarray(x, dtype=np.float64)


def integer_x(n, seed, nrhs=1, lo=-8, hi=8):
    x = _rng(seed).integers(lo, hi + 1, size=(n, nrhs) if nrhs > 1 else n)
    return np.ascontiguousarray(x, dtype=np.float64)


def integer_values(nnz, seed, lo=-8, hi=8):
    """Small nonzero integers, so that every FP64 sum of products is exact."""
    v = _rng(seed).integers(lo, hi, size=nnz).astype(np.float64)
    v[v >= 0] += 1.0          # map [lo, hi) onto [lo, hi] without 0
    return v


def random_labels(count, K, seed, border_frac=0.0):
    """Uniform labels in [0, K); with border_frac > 0 a fraction get label K."""
    rng = _rng(seed)
    lab = rng.integers(0, K, size=count).astype(np.int32)
    if border_frac > 0:
        lab[rng.random(count) < border_frac] = K
    return lab


def random_sparse(m, n, density, seed, integer=True, empty_rows=0.0):
    """Small random CSR matrix (tests).  Optionally leaves some rows empty."""
    rng = _rng(seed)
    mask = rng.random((m, n)) < density
    if empty_rows > 0:
        mask[rng.random(m) < empty_rows, :] = False
    r, c = np.nonzero(mask)
    if integer:
        v = integer_values(r.size, seed + 7919)
    else:
        v = rng.uniform(-1.0, 1.0, size=r.size)
    return coo_to_csr(m, n, r, c, v)


def zipf_matrix(m=16384, n=16384, seed=0, s_rows=1.7498, dmax=512, s_cols=1.2):
    """Power-law rows (mean 8, max 512) with Zipf-distributed columns."""
    rng = _rng(seed)
    d = np.arange(1, dmax + 1, dtype=np.float64)
    pd = d ** -s_rows
    pd /= pd.sum()
    deg = rng.choice(np.arange(1, dmax + 1), size=m, p=pd)
    ranks = np.arange(1, n + 1, dtype=np.float64)
    pc = ranks ** -s_cols
    cdf = np.cumsum(pc / pc.sum())
    cdf[-1] = 1.0
    colperm = rng.permutation(n)
    rows_out, cols_out = [], []
    for i in range(m):
        want = int(min(deg[i], n))
        chosen = np.empty(0, dtype=np.int64)
        while chosen.size < want:
            draw = np.searchsorted(cdf, rng.random(2 * (want - chosen.size) + 8),
                                   side="right")
            allc = np.concatenate([chosen, draw])
            _, first = np.unique(allc, return_index=True)
            chosen = allc[np.sort(first)][:want]
        rows_out.append(np.full(want, i, dtype=np.int64))
        cols_out.append(colperm[chosen])
    rows = np.concatenate(rows_out)
    cols = np.concatenate(cols_out)
    vals = rng.uniform(-1.0, 1.0, size=rows.size)
    return coo_to_csr(m, n, rows, cols, vals)


def mesh5(nx=1024, seed=0, permute=True, return_points=False):
    """5-point stencil on an nx x nx grid, values U(-1,1).  With
    return_points, also the grid point (gy * nx + gx) of every row."""
    rng = _rng(seed)
    N = nx * nx
    idx = np.arange(N, dtype=np.int64)
    gx, gy = idx % nx, idx // nx
    rows, cols = [idx], [idx]
    for dx, dy in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        ok = (gx + dx >= 0) & (gx + dx < nx) & (gy + dy >= 0) & (gy + dy < nx)
        rows.append(idx[ok])
        cols.append(idx[ok] + dx + dy * nx)
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = rng.uniform(-1.0, 1.0, size=rows.size)
    points = idx
    if permute:
        perm = rng.permutation(N)
        inv = np.empty_like(perm)
        inv[perm] = np.arange(N)
        rows, cols = inv[rows], inv[cols]
        points = perm
    out = coo_to_csr(N, N, rows, cols, vals)
    return out + (points,) if return_points else out


def rmat(scale=20, deg=16, a=0.57, b=0.19, c=0.19, seed=0, chunk=1 << 22):
    """R-MAT graph with exactly deg * 2^scale distinct directed pairs: edges
    are drawn in batches, and the first deg * 2^scale distinct pairs in draw
    order are kept."""
    rng = _rng(seed)
    n = 1 << scale
    target = deg * n
    ab, abc = np.float32(a + b), np.float32(a + b + c)
    fa = np.float32(a)
    batches = []
    drawn = 0
    want = int(target * 1.3) + chunk
    while True:
        while drawn < want:
            k = min(chunk, want - drawn)
            i = np.zeros(k, dtype=np.int64)
            j = np.zeros(k, dtype=np.int64)
            for _ in range(scale):
                u = rng.random(k, dtype=np.float32)
                i = (i << 1) | (u >= ab)
                j = (j << 1) | (((u >= fa) & (u < ab)) | (u >= abc))
            batches.append((i << scale) | j)
            drawn += k
        keys = np.concatenate(batches)
        uniq, first = np.unique(keys, return_index=True)
        if uniq.size >= target:
            keys = keys[np.sort(first)[:target]]
            break
        want = drawn + int((target - uniq.size) * 1.5) + chunk
    rows, cols = keys >> scale, keys & (n - 1)
    vals = rng.uniform(-1.0, 1.0, size=rows.size)
    return coo_to_csr(n, n, rows, cols, vals)


def blocks(nb=64, bs=16384, fill=0.002, border_frac=0.05, seed=0, permute=True):
    """nb diagonal bs x bs blocks at `fill`, plus border_frac * (block nnz)
    random off-block nonzeros, symmetrically permuted."""
    rng = _rng(seed)
    N = nb * bs
    per_block = int(round(fill * bs * bs))
    keys = []
    for blk in range(nb):
        got = np.empty(0, dtype=np.int64)
        while got.size < per_block:
            draw = rng.integers(0, bs * bs, size=int(1.02 * (per_block - got.size)) + 64)
            got = np.unique(np.concatenate([got, draw]))
        got = got[np.sort(rng.permutation(got.size)[:per_block])]
        r, cc = got // bs + blk * bs, got % bs + blk * bs
        keys.append(r * N + cc)
    n_border = int(round(border_frac * per_block * nb))
    bkeys = np.empty(0, dtype=np.int64)
    while bkeys.size < n_border:
        r = rng.integers(0, N, size=int(1.1 * (n_border - bkeys.size)) + 64)
        cc = rng.integers(0, N, size=r.size)
        off = (r // bs) != (cc // bs)
        bkeys = np.unique(np.concatenate([bkeys, r[off] * N + cc[off]]))
    bkeys = bkeys[np.sort(rng.permutation(bkeys.size)[:n_border])]
    allk = np.concatenate(keys + [bkeys])
    rows, cols = allk // N, allk % N
    vals = rng.uniform(-1.0, 1.0, size=rows.size)
    if permute:
        perm = rng.permutation(N)
        inv = np.empty_like(perm)
        inv[perm] = np.arange(N)
        rows, cols = inv[rows], inv[cols]
    return coo_to_csr(N, N, rows, cols, vals)


def laplacian3d(n=128, seed=0, permute=True):
    """7-point Dirichlet Laplacian on an n^3 grid: 6 on the diagonal, -1 to
    each in-grid neighbour."""
    N = n * n * n
    idx = np.arange(N, dtype=np.int64)
    gx, gy, gz = idx % n, (idx // n) % n, idx // (n * n)
    rows, cols, vals = [idx], [idx], [np.full(N, 6.0)]
    for d, g in ((1, gx), (n, gy), (n * n, gz)):
        for s in (-1, 1):
            ok = (g + s >= 0) & (g + s < n)
            rows.append(idx[ok])
            cols.append(idx[ok] + s * d)
            vals.append(np.full(int(ok.sum()), -1.0))
    rows, cols, vals = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
    if permute:
        perm = _rng(seed).permutation(N)
        inv = np.empty_like(perm)
        inv[perm] = np.arange(N)
        rows, cols = inv[rows], inv[cols]
    return coo_to_csr(N, N, rows, cols, vals)


def weighted_laplacian3d(n=16, seed=0, shift=0.5, permute=True):
    """Graph Laplacian of the n^3 7-point grid with edge weights U(0.5, 1.5),
    plus shift on the diagonal: symmetric positive definite, with values that
    BF16 does not hold exactly.  Symmetrically permuted."""
    rng = _rng(seed)
    N = n * n * n
    idx = np.arange(N, dtype=np.int64)
    x, y, z = idx % n, (idx // n) % n, idx // (n * n)
    er, ec, ew = [], [], []
    for dx, dy, dz in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
        ok = (x + dx < n) & (y + dy < n) & (z + dz < n)
        a = idx[ok]
        er.append(a)
        ec.append(a + dx + dy * n + dz * n * n)
        ew.append(rng.uniform(0.5, 1.5, size=a.size))
    er, ec, ew = np.concatenate(er), np.concatenate(ec), np.concatenate(ew)
    diag = np.full(N, float(shift))
    np.add.at(diag, er, ew)
    np.add.at(diag, ec, ew)
    rows = np.concatenate([idx, er, ec])
    cols = np.concatenate([idx, ec, er])
    vals = np.concatenate([diag, -ew, -ew])
    if permute:
        perm = rng.permutation(N)
        inv = np.empty_like(perm)
        inv[perm] = np.arange(N)
        rows, cols = inv[rows], inv[cols]
    return coo_to_csr(N, N, rows, cols, vals)


def rmat_batch_specs(count=64, lo=1024, hi=65536, deg_lo=8, deg_hi=32, seed=0):
    """The members of rmat_batch as (scale, degree, seed) triples: row counts
    drawn log-uniformly in [lo, hi] and rounded to a power of two (R-MAT's
    own sizes), average degree uniform in [deg_lo, deg_hi], seeds
    seed..seed+count-1."""
    rng = _rng(seed)
    out = []
    for b in range(count):
        scale = int(round(rng.uniform(np.log2(lo), np.log2(hi))))
        deg = int(rng.integers(deg_lo, deg_hi + 1))
        out.append((scale, deg, seed + b))
    return out


def rmat_batch_member(scale, deg, seed):
    """One member of rmat_batch: (m, n, rowptr, colidx, vals)."""
    rp, ci, v = rmat(scale, deg, seed=seed, chunk=1 << 18)
    return (1 << scale, 1 << scale, rp, ci, v)


def rmat_batch(count=64, lo=1024, hi=65536, deg_lo=8, deg_hi=32, seed=0):
    """`count` R-MAT matrices (a, b, c = .57, .19, .19) with the sizes and
    degrees of rmat_batch_specs.  Returns a list of (m, n, rowptr, colidx,
    vals)."""
    return [rmat_batch_member(*s) for s in rmat_batch_specs(count, lo, hi, deg_lo, deg_hi, seed)]


def block_diagonal(mats):
    """CSR of diag(A_1, ..., A_B) from a list of (m, n, rowptr, colidx, vals)."""
    M = sum(m for m, *_ in mats)
    rps, cis, vs = [np.zeros(1, dtype=np.int64)], [], []
    r_off = c_off = e_off = 0
    for m, n, rp, ci, v in mats:
        rps.append(rp[1:].astype(np.int64) + e_off)
        cis.append(ci.astype(np.int64) + c_off)
        vs.append(v)
        c_off += n
        e_off += int(rp[-1])
        r_off += m
    rowptr = np.concatenate(rps)
    assert rowptr.size == M + 1
    return rowptr.astype(np.int32), np.concatenate(cis).astype(np.int32), np.concatenate(vs)

