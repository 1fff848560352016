"""Oracle: reverse Cuthill-McKee ordering of the unknowns.  Test infrastructure only.

The paper does not reorder (it hands a CSC matrix to SciPy/CuPy, Sect. 2.2.2);
the ordering is a property of this library's device layout, so the oracle fixes
one exact rule for it and checks the library against that rule bit for bit:

  * the graph is the off-diagonal structural pattern of the n = 1 operator
    (mesh edges for vertex placements, shared edges for cells);
  * degree = number of neighbours;
  * each connected component starts at the unvisited vertex of least
    (degree, id); breadth-first search appends the unvisited neighbours of the
    vertex being expanded in increasing (degree, id);
  * the concatenated sequence is reversed.

`rcm_order` runs that rule with plain Python loops (small graphs);
`check_rcm_order` verifies any permutation against the rule at any size by the
properties that characterise the breadth-first sequence uniquely.
Parity: pinned on hand-worked graphs (tests).
"""

import numpy as np


def _neighbours(indptr, indices):
    n = len(indptr) - 1
    out = []
    for i in range(n):
        row = indices[indptr[i]:indptr[i + 1]]
        out.append([int(j) for j in row if j != i])
    return out


def rcm_order(indptr, indices):
    """Returns order with order[new] = old index."""
    nb = _neighbours(indptr, indices)
    n = len(nb)
    deg = [len(x) for x in nb]
    by_key = sorted(range(n), key=lambda v: (deg[v], v))
    visited = [False] * n
    seq = []
    scan = 0
    while len(seq) < n:
        while visited[by_key[scan]]:
            scan += 1
        s = by_key[scan]
        visited[s] = True
        queue = [s]
        head = 0
        while head < len(queue):
            u = queue[head]
            head += 1
            seq.append(u)
            fresh = [w for w in nb[u] if not visited[w]]
            fresh.sort(key=lambda w: (deg[w], w))
            for w in fresh:
                visited[w] = True
                queue.append(w)
    return np.asarray(seq[::-1], dtype=np.int64)


def check_rcm_order(indptr, indices, order):
    """True iff `order` (order[new] = old) is exactly the ordering defined above.
    Raises AssertionError with the first violated property otherwise."""
    indptr = np.asarray(indptr, dtype=np.int64)
    indices = np.asarray(indices, dtype=np.int64)
    order = np.asarray(order, dtype=np.int64)
    n = indptr.size - 1
    assert order.size == n, "length"
    assert np.array_equal(np.sort(order), np.arange(n)), "not a permutation"
    q = order[::-1]                      # breadth-first sequence
    pos = np.empty(n, dtype=np.int64)
    pos[q] = np.arange(n)
    rows = np.repeat(np.arange(n), np.diff(indptr))
    off = indices != rows
    r, c = rows[off], indices[off]
    deg = np.bincount(r, minlength=n)
    big = np.int64(n + 1)
    # s(v): earliest position among v's neighbours (the vertex that discovered it)
    s = np.full(n, big, dtype=np.int64)
    np.minimum.at(s, r, pos[c])
    sq = s[q]
    t = np.arange(n)
    start = sq > t
    key = deg.astype(np.int64) * (n + 1) + np.arange(n)
    kq = key[q]
    # starts: least (degree, id) among the vertices not yet placed
    suff = np.minimum.accumulate(kq[::-1])[::-1]
    assert np.all(suff[start] == kq[start]), "component start is not least (degree, id)"
    # non-starts: discovered after the last start and before themselves
    last_start = np.maximum.accumulate(np.where(start, t, -1))
    ns = ~start
    assert np.all(sq[ns] < t[ns]), "vertex placed before its discoverer"
    assert np.all(sq[ns] >= last_start[ns]), "vertex placed after a later component start"
    # consecutive non-starts of one component: increasing (s, degree, id)
    both = ns[1:] & ns[:-1]
    k3_prev = (sq[:-1], deg[q][:-1], q[:-1])
    k3_next = (sq[1:], deg[q][1:], q[1:])
    lt = (k3_prev[0] < k3_next[0]) | ((k3_prev[0] == k3_next[0]) & (
        (k3_prev[1] < k3_next[1]) | ((k3_prev[1] == k3_next[1]) & (k3_prev[2] < k3_next[2]))))
    assert np.all(lt[both]), "breadth-first children not in (degree, id) order"
    return True
