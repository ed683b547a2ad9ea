"""ICSR, the incremental compressed storage by rows of Sec. 2.1, restated
plainly for the tests (test infrastructure; pure Python loops, small cases).

ICSR replaces CSR's colIndex by colDiff, the increments between the column
indices of successive stored nonzeros, and rowStart by rowJump, the
increments between the indices of successive nonzero rows.  Empty rows cost
nothing.  The paper does not say how the product loop finds where a row
ends without rowStart.  Reading: the increment stored at the first nonzero
of each row after the first carries an extra n.  The running column index
then reaches n or more exactly there; the loop writes the finished row,
subtracts n, and advances the row index by the next rowJump.  The running
column starts at 0 and the row index at rowJump[0], the first nonzero row.
Rows no nonzero reaches get 0.
"""
import numpy as np


def icsr_encode(m, n, rowptr, colidx):
    """(colDiff, rowJump) of a CSR matrix, nonzeros in row-major order."""
    rp = [int(t) for t in rowptr]
    ci = [int(t) for t in colidx]
    col_diff, row_jump = [], []
    prev_col, prev_row = 0, None
    for i in range(m):
        if rp[i] == rp[i + 1]:
            continue
        row_jump.append(i if prev_row is None else i - prev_row)
        for p in range(rp[i], rp[i + 1]):
            d = ci[p] - prev_col
            if p == rp[i] and prev_row is not None:
                d += n                         # the row-change signal
            col_diff.append(d)
            prev_col = ci[p]
        prev_row = i
    return np.array(col_diff, dtype=np.int64), np.array(row_jump, dtype=np.int64)


def icsr_spmv(m, n, col_diff, row_jump, vals, x):
    """y = A x from the ICSR arrays, with the loop described above."""
    y = np.zeros(m)
    if len(col_diff) == 0:
        return y
    i = int(row_jump[0])
    j = 1
    c = 0
    s = 0.0
    for k in range(len(col_diff)):
        c += int(col_diff[k])
        if c >= n:
            y[i] = s
            s = 0.0
            c -= n
            i += int(row_jump[j])
            j += 1
        s += float(vals[k]) * float(x[c])
    y[i] = s
    return y


def icsr_decode(m, n, col_diff, row_jump):
    """CSR (rowptr, colidx) back from the ICSR arrays."""
    rows, cols = [], []
    if len(col_diff):
        i = int(row_jump[0])
        j = 1
        c = 0
        for k in range(len(col_diff)):
            c += int(col_diff[k])
            if c >= n:
                c -= n
                i += int(row_jump[j])
                j += 1
            rows.append(i)
            cols.append(c)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    for i in rows:
        rowptr[i + 1] += 1
    return np.cumsum(rowptr), np.array(cols, dtype=np.int64)
