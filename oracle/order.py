"""Comparison reorderings of the paper's experiments (Sec. 5.1), restated
plainly for the tests (test infrastructure; pure Python loops, small cases).

The bipartite graph of A has a vertex per row (ids 0 .. m-1) and per column
(ids m .. m+n-1) and an edge per nonzero.  Ties go to the lower id.

* ``bfs_order``  sBFS: breadth-first search from vertex 0 with neighbours
  taken in increasing id; when the queue is empty the search restarts at the
  lowest unvisited vertex.  Rows and columns in visiting order.
* ``rcm_order``  sRCM: reverse Cuthill-McKee.  For each connected component,
  in order of its lowest vertex: start at the component's vertex of least
  degree, replace it by the least-degree vertex of its last breadth-first
  level while that lengthens the level structure (George and Liu's
  pseudo-peripheral vertex), then visit breadth first, each vertex enqueueing
  its unvisited neighbours by increasing degree.  The whole visiting sequence
  is reversed.
* ``sbd_order``  the order sHP_RN gives a row-net partition: columns by (part,
  index); a row whose columns lie in one leaf k of the bisection tree (K
  leaves, K a power of two, left subtree first) in block k; a row whose parts
  span leaves a < b in the separator of the bisection that parted a from b,
  placed between that bisection's halves; empty rows last; ties by index.
* ``nested_order``  the nested reading of the SB / DB border (the parts of a
  row-side bisection tree, K leaves, K a power of two, left subtree first;
  label K marks the DB row border): rows by (part, index), the row border
  last; a column whose rows outside the row border all lie in part k in
  column block k; a column whose rows span parts a < b in the border of the
  bisection that parted a from b, placed between that bisection's halves;
  columns no part touches last; ties by index.
"""
from collections import deque

import numpy as np


def _graph(m, n, rowptr, colidx):
    rp = [int(t) for t in rowptr]
    ci = [int(t) for t in colidx]
    adj = [[] for _ in range(m + n)]
    for i in range(m):
        for p in range(rp[i], rp[i + 1]):
            adj[i].append(m + ci[p])
            adj[m + ci[p]].append(i)
    for a in adj:
        a.sort()
    return adj


def _split(m, seq):
    rows = [v for v in seq if v < m]
    cols = [v - m for v in seq if v >= m]
    return np.array(rows, dtype=np.int32), np.array(cols, dtype=np.int32)


def bfs_order(m, n, rowptr, colidx):
    adj = _graph(m, n, rowptr, colidx)
    seen = [False] * (m + n)
    seq = []
    for s in range(m + n):
        if seen[s]:
            continue
        seen[s] = True
        q = deque([s])
        while q:
            v = q.popleft()
            seq.append(v)
            for u in adj[v]:
                if not seen[u]:
                    seen[u] = True
                    q.append(u)
    return _split(m, seq)


def _levels(adj, s, done):
    """Breadth-first distances from s over vertices not done."""
    dist = {s: 0}
    q = deque([s])
    while q:
        v = q.popleft()
        for u in adj[v]:
            if not done[u] and u not in dist:
                dist[u] = dist[v] + 1
                q.append(u)
    return dist


def rcm_order(m, n, rowptr, colidx):
    adj = _graph(m, n, rowptr, colidx)
    deg = [len(a) for a in adj]
    key = lambda v: (deg[v], v)            # noqa: E731
    done = [False] * (m + n)
    seq = []
    for s0 in range(m + n):
        if done[s0]:
            continue
        comp = _levels(adj, s0, done)
        v = min(comp, key=key)
        dist = _levels(adj, v, done)
        ecc = max(dist.values())
        while True:
            u = min((w for w, d in dist.items() if d == ecc), key=key)
            du = _levels(adj, u, done)
            eu = max(du.values())
            if eu <= ecc:
                break
            v, dist, ecc = u, du, eu
        done[v] = True
        q = deque([v])
        while q:
            w = q.popleft()
            seq.append(w)
            nxt = sorted((u for u in adj[w] if not done[u]), key=key)
            for u in nxt:
                done[u] = True
                q.append(u)
    seq.reverse()
    return _split(m, seq)


def sbd_order(m, n, rowptr, colidx, K, col_labels):
    lab = [int(t) for t in col_labels]
    cols = sorted(range(n), key=lambda j: (lab[j], j))

    def block(i):
        parts = [lab[int(colidx[p])] for p in range(int(rowptr[i]), int(rowptr[i + 1]))]
        if not parts:
            return (2 * K, i)
        a, b = min(parts), max(parts)
        if a == b:
            return (2 * a, i)
        # walk down the bisection tree from the root until a and b part
        lo, hi = 0, K
        while True:
            mid = (lo + hi) // 2
            if b < mid:
                hi = mid
            elif a >= mid:
                lo = mid
            else:
                return (2 * mid - 1, i)

    rows = sorted(range(m), key=block)
    return np.array(rows, dtype=np.int32), np.array(cols, dtype=np.int32)


def _between(a, b, K):
    """Key of a block spanning leaves a < b: walk down the bisection tree from
    the root until a and b fall on different sides; the border of that
    bisection sits just before its right half's first leaf."""
    lo, hi = 0, K
    while True:
        mid = (lo + hi) // 2
        if b < mid:
            hi = mid
        elif a >= mid:
            lo = mid
        else:
            return 2 * mid - 1


def nested_order(m, n, rowptr, colidx, K, row_labels):
    lab = [int(t) for t in row_labels]
    rows = sorted(range(m), key=lambda i: (lab[i], i))
    parts = [[] for _ in range(n)]
    for i in range(m):
        if lab[i] == K:
            continue                      # the DB row border
        for p in range(int(rowptr[i]), int(rowptr[i + 1])):
            parts[int(colidx[p])].append(lab[i])

    def block(j):
        if not parts[j]:
            return (2 * K, j)
        a, b = min(parts[j]), max(parts[j])
        return (2 * a, j) if a == b else (_between(a, b, K), j)

    cols = sorted(range(n), key=block)
    return np.array(rows, dtype=np.int32), np.array(cols, dtype=np.int32)
