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


# ---------------------------------------------------------------- space-filling curve
# A second device order the library offers: unknowns sorted by a Hilbert-curve
# key of their position, ties by id.  The oracle restates the rule on its own:
#   * position: the vertex, or the corner average ((a + b) + c) / 3 of a triangle;
#   * sphere: cube face of the direction (largest |component|, ties to x then y,
#     face 2k for +axis k and 2k+1 for -axis k), the two other components divided
#     by the largest, mapped to [0, 1] by (t + 1) / 2; plane: coordinates scaled
#     to the bounding box of all vertices;
#   * each coordinate quantised to 16 bits as floor(t * 2^16) clamped to the grid;
#   * key = face * 2^32 + Hilbert index on the 2^16 x 2^16 grid, the curve
#     starting at (0, 0) and ending at (2^16 - 1, 0).

CURVE_BITS = 16


def hilbert_index(x, y, bits):
    """Position of grid cell (x, y) along the Hilbert curve of order `bits`.

    Recursive definition: the square splits into four quadrants visited in the
    order lower-left, upper-left, upper-right, lower-right; each quadrant holds
    a copy of the curve, transposed in the two lower quadrants and additionally
    reflected through the centre in the lower-right one, so that consecutive
    quadrants join."""
    if bits == 0:
        return 0
    half = 1 << (bits - 1)
    right, upper = x >= half, y >= half
    lx, ly = x - half * right, y - half * upper
    if not upper:
        if right:
            lx, ly = half - 1 - lx, half - 1 - ly
        lx, ly = ly, lx
    quadrant = {(False, False): 0, (False, True): 1, (True, True): 2, (True, False): 3}[(right, upper)]
    return quadrant * half * half + hilbert_index(lx, ly, bits - 1)


def _quantise(t):
    q = np.floor(np.asarray(t, dtype=np.float64) * float(1 << CURVE_BITS))
    return np.clip(np.nan_to_num(q, nan=0.0), 0, (1 << CURVE_BITS) - 1).astype(np.int64)


def curve_keys(pos, sphere, all_coords=None):
    """Keys of points `pos` [n][2 or 3]; `all_coords` gives the bounding box (plane)."""
    pos = np.asarray(pos, dtype=np.float64)
    n = pos.shape[0]
    if sphere:
        a = np.abs(pos)
        axis = np.where((a[:, 0] >= a[:, 1]) & (a[:, 0] >= a[:, 2]), 0, np.where(a[:, 1] >= a[:, 2], 1, 2))
        face = 2 * axis + (pos[np.arange(n), axis] < 0)
        others = {0: (1, 2), 1: (0, 2), 2: (0, 1)}
        u = np.empty(n)
        v = np.empty(n)
        for k in range(3):
            sel = axis == k
            m = a[sel, k]
            u[sel] = pos[sel, others[k][0]] / m
            v[sel] = pos[sel, others[k][1]] / m
        iu, iv = _quantise((u + 1.0) * 0.5), _quantise((v + 1.0) * 0.5)
    else:
        c = np.asarray(all_coords, dtype=np.float64)
        lo, hi = c[:, :2].min(axis=0), c[:, :2].max(axis=0)
        span = np.where(hi > lo, hi - lo, 1.0)
        iu, iv = _quantise((pos[:, 0] - lo[0]) / span[0]), _quantise((pos[:, 1] - lo[1]) / span[1])
        face = np.zeros(n, dtype=np.int64)
    d = np.array([hilbert_index(int(x), int(y), CURVE_BITS) for x, y in zip(iu, iv)], dtype=np.int64)
    return face.astype(np.int64) * (1 << (2 * CURVE_BITS)) + d


def curve_order(mesh, placement):
    """Device order of the unknowns under the curve rule: original ids, order[new]."""
    from .mesh import ocean_subset
    coords = np.asarray(mesh["coords"], dtype=np.float64)
    tri = np.asarray(mesh["tri"])
    sphere = coords.shape[1] == 3
    kept, verts, _ = ocean_subset(coords.shape[0], tri, mesh.get("ocean"))
    if placement == "cell":
        t = tri[kept]
        pos = ((coords[t[:, 0]] + coords[t[:, 1]]) + coords[t[:, 2]]) / 3.0
        ids = np.asarray(kept)
    else:
        pos = coords[verts]
        ids = np.asarray(verts)
    keys = curve_keys(pos, sphere, coords)
    idx = np.lexsort((np.arange(ids.size), keys))
    return ids[idx]
