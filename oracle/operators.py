"""Oracle: the discrete operators of the paper's Sect. 2.1.  Test infrastructure only.

All matrices are scipy.sparse CSR in FP64 on the unknowns of `mesh.ocean_subset`
/ `mesh.cell_subset`; their structural pattern keeps explicit zeros (an edge of
a split-square grid whose cotangent weight is exactly 0 is still an entry).

  scalar_vertex_operators : K (the l-free P1 stiffness, D~ = l^2 K) and the lumped
                            mass A_v of median-dual control volumes (Sect. 2.1.1).
  vector_vertex_operators : K~ = stiffness + (R^-2 + m^2) x consistent P1 mass, the
                            metric operator T (T_vv' = l^2 Tm_vv'), A_v and the
                            cell-to-vertex projection R_vc = int N_v M_c (Sect. 2.1.2).
  cell_operators          : A * (graph Laplacian of edge-adjacent ocean triangles) and
                            the triangle areas A_c (Eq. 6).
  voronoi_vertex_operators: quasi-hexagonal finite volumes around the vertices (Eq. 3-5).
  circumcenter_cell_operators: finite volumes for scalars at triangle circumcentres.
  order_operator          : G_n = K (M^-1 K)^(n-1), so that S = M + (1/2) l^(2n) G_n
                            (Sect. 2.1.1 for n = 2; the paper notes the generalisation).

Parity: the scalar and cell operators are pinned by closed forms on regular
periodic grids and by a brute-force gradient re-derivation (tests).  The vector
operator is pinned by its reduction to two scalar problems on the plane, by
symmetry of [[K~, T], [-T, K~]], by a quadrature re-derivation of T and of the
metric mass term, and on the sphere by the exact filter response of vector
spherical harmonics (rigid rotation, poloidal and toroidal Y_2^1 are
eigenfunctions of the vector Laplacian whose components carry the metric
terms): second-order convergence, and a flipped sign of T or of the metric
term fails it.  The finite-volume operators are pinned by the cotangent
identity, area tiling, lattice closed forms and brute-force circumcentres.
"""

import numpy as np
import scipy.sparse as sp

from .mesh import ocean_subset, cell_subset, edge_vectors


def _coo(rows, cols, vals, n, m=None):
    return sp.coo_matrix((vals, (rows, cols)), shape=(n, n if m is None else m)).tocsr()


def scalar_vertex_operators(mesh):
    """Returns dict(K, A, vert_ids, kept_tri, tri_local)."""
    V = mesh["coords"].shape[0]
    tri = np.asarray(mesh["tri"], dtype=np.int64)
    kept_tri, vert_ids, tl = ocean_subset(V, tri, mesh.get("ocean"))
    t = tri[kept_tri]
    n = vert_ids.size
    rows, cols, vals = [], [], []
    # For each corner k, the opposite edge (a, b) receives -1/2 cot(angle at k),
    # the P1 value of int grad N_a . grad N_b over the triangle (a != b).
    for k, a, b in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
        u = edge_vectors(mesh, t[:, k], t[:, a])
        v = edge_vectors(mesh, t[:, k], t[:, b])
        cot = np.einsum("ij,ij->i", u, v) / np.linalg.norm(np.cross(u, v), axis=1)
        w = -0.5 * cot
        rows += [tl[:, a], tl[:, b]]
        cols += [tl[:, b], tl[:, a]]
        vals += [w, w]
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    # Diagonal: int |grad N_a|^2 = minus the sum of the row's off-diagonal entries
    # (the basis functions sum to one, so their gradients sum to zero).
    diag = -np.bincount(rows, weights=vals, minlength=n)
    idx = np.arange(n)
    K = _coo(np.concatenate([rows, idx]), np.concatenate([cols, idx]),
             np.concatenate([vals, diag]), n)
    e1 = edge_vectors(mesh, t[:, 0], t[:, 1])
    e2 = edge_vectors(mesh, t[:, 0], t[:, 2])
    area = 0.5 * np.linalg.norm(np.cross(e1, e2), axis=1)
    # Median-dual control volume: a third of each adjacent triangle.
    A = np.bincount(tl.ravel(), weights=np.repeat(area / 3.0, 3), minlength=n)
    return dict(K=K, A=A, vert_ids=vert_ids, kept_tri=kept_tri, tri_local=tl, tri_area=area)


def p1_gradients(mesh, t):
    """Gradients of the three P1 basis functions on each flat triangle (3-D
    vectors in the triangle's plane): grad N_k = n x (x_b - x_a) / (2 A), with
    (k, a, b) cyclic and n the unit normal of the counter-clockwise triangle."""
    e1 = edge_vectors(mesh, t[:, 0], t[:, 1])
    e2 = edge_vectors(mesh, t[:, 0], t[:, 2])
    nrm = np.cross(e1, e2)
    twoA = np.linalg.norm(nrm, axis=1)
    nh = nrm / twoA[:, None]
    g = []
    for k, a, b in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
        eab = edge_vectors(mesh, t[:, a], t[:, b])
        g.append(np.cross(nh, eab) / twoA[:, None])
    return g, 0.5 * twoA


def metric_factors(mesh, t):
    """Per triangle: m = tan(theta)/R_e with theta the latitude of the centroid
    direction, and the unit zonal (east) vector there.  Zero / x-axis on planes."""
    if mesh["geom"] != "sphere":
        ex = np.zeros((t.shape[0], 3))
        ex[:, 0] = 1.0
        return np.zeros(t.shape[0]), ex, 0.0
    x = np.asarray(mesh["coords"], dtype=np.float64)
    c = x[t[:, 0]] + x[t[:, 1]] + x[t[:, 2]]
    c = c / np.linalg.norm(c, axis=1, keepdims=True)
    lat = np.arcsin(np.clip(c[:, 2], -1.0, 1.0))
    R = float(mesh["radius"])
    m = np.tan(lat) / R
    east = np.stack([-c[:, 1], c[:, 0], np.zeros_like(c[:, 0])], 1)
    east /= np.linalg.norm(east, axis=1, keepdims=True)
    return m, east, 1.0 / (R * R)


def vector_vertex_operators(mesh):
    """Returns dict(Kt, Tm, A, R, vert_ids, kept_tri).

    Kt_vv' = int grad N_v . grad N_v' + (R_e^-2 + m^2) N_v N_v'
    Tm_vv' = int m (-N_v' d_x N_v + N_v d_x N_v')      (T = l^2 Tm)
    R_vc   = int N_v M_c = A_c / 3 for the corners v of c.
    """
    base = scalar_vertex_operators(mesh)
    tri = np.asarray(mesh["tri"], dtype=np.int64)
    t = tri[base["kept_tri"]]
    tl = base["tri_local"]
    n = base["vert_ids"].size
    grads, area = p1_gradients(mesh, t)
    m, east, inv_r2 = metric_factors(mesh, t)
    coef = inv_r2 + m * m
    rows, cols, vals = [], [], []
    trows, tcols, tvals = [], [], []
    dx = [np.einsum("ij,ij->i", g, east) for g in grads]
    for a in range(3):
        for b in range(3):
            # consistent P1 mass: A/6 on the diagonal, A/12 off it
            mab = area / 6.0 if a == b else area / 12.0
            rows.append(tl[:, a])
            cols.append(tl[:, b])
            vals.append(coef * mab)
            if a != b:
                # int N = A/3 and m, d_x N constant on the triangle
                trows.append(tl[:, a])
                tcols.append(tl[:, b])
                tvals.append(m * (area / 3.0) * (dx[b] - dx[a]))
    metric_mass = _coo(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), n)
    Kt = (base["K"] + metric_mass).tocsr()
    if trows:
        Tm = _coo(np.concatenate(trows), np.concatenate(tcols), np.concatenate(tvals), n)
    else:
        Tm = sp.csr_matrix((n, n))
    nc = t.shape[0]
    R = _coo(tl.ravel(), np.repeat(np.arange(nc), 3), np.repeat(area / 3.0, 3), n, nc)
    return dict(Kt=Kt, Tm=Tm, A=base["A"], R=R, vert_ids=base["vert_ids"],
                kept_tri=base["kept_tri"], K=base["K"])


def cell_operators(mesh, cell_A=None):
    """Returns dict(K, A, cell_ids) with K = A_const * L, L the graph Laplacian
    of edge-adjacent kept triangles (Eq. 6: A_c (D u)_c = A l^2 sum (u_c - u_c')),
    and A the triangle areas."""
    V = mesh["coords"].shape[0]
    tri = np.asarray(mesh["tri"], dtype=np.int64)
    kept, pairs = cell_subset(V, tri, mesh.get("ocean"))
    n = kept.size
    Aconst = np.sqrt(3.0) if cell_A is None else float(cell_A)
    i, j = pairs[:, 0], pairs[:, 1]
    deg = np.bincount(np.concatenate([i, j]), minlength=n).astype(np.float64)
    idx = np.arange(n)
    L = _coo(np.concatenate([i, j, idx]), np.concatenate([j, i, idx]),
             np.concatenate([-np.ones(i.size), -np.ones(j.size), deg]), n)
    t = tri[kept]
    e1 = edge_vectors(mesh, t[:, 0], t[:, 1])
    e2 = edge_vectors(mesh, t[:, 0], t[:, 2])
    area = 0.5 * np.linalg.norm(np.cross(e1, e2), axis=1)
    return dict(K=(Aconst * L).tocsr(), A=area, cell_ids=kept, pairs=pairs)


def _circumcentres(e1, e2):
    """Circumcentre of each flat triangle as a vector from its corner 0 (e1, e2 the
    edges from corner 0): the point O = a e1 + b e2 equidistant from the three
    corners, from the 2 x 2 Gram system O . e1 = |e1|^2 / 2, O . e2 = |e2|^2 / 2."""
    g11 = np.einsum("ij,ij->i", e1, e1)
    g22 = np.einsum("ij,ij->i", e2, e2)
    g12 = np.einsum("ij,ij->i", e1, e2)
    det = g11 * g22 - g12 * g12
    a = (0.5 * g11 * g22 - 0.5 * g22 * g12) / det
    b = (0.5 * g22 * g11 - 0.5 * g11 * g12) / det
    return a[:, None] * e1 + b[:, None] * e2


def voronoi_vertex_operators(mesh):
    """Quasi-hexagonal control volumes around the vertices (Eq. 3-5):
    A_v (D phi)_v = l^2 sum_v' (phi_v - phi_v') l_vv' / d_vv' with d_vv' the edge
    length and l_vv' the distance between the circumcentres of the triangles on
    both sides (signed: a circumcentre beyond the edge counts negative; on a
    coast the edge midpoint stands in for the missing side), and A_v the area
    of the circumcentric dual cell (sum of the kites d h / 4 of the half-dual
    segments h around v).  Returns dict(K, A, vert_ids, kept_tri) with K the
    l-free operator."""
    V = mesh["coords"].shape[0]
    tri = np.asarray(mesh["tri"], dtype=np.int64)
    kept_tri, vert_ids, tl = ocean_subset(V, tri, mesh.get("ocean"))
    t = tri[kept_tri]
    n = vert_ids.size
    e1 = edge_vectors(mesh, t[:, 0], t[:, 1])
    e2 = edge_vectors(mesh, t[:, 0], t[:, 2])
    nrm = np.cross(e1, e2)
    nhat = nrm / np.linalg.norm(nrm, axis=1)[:, None]
    O = _circumcentres(e1, e2)
    corner = [np.zeros_like(e1), e1, e2]  # corners relative to corner 0
    rows, cols, vals = [], [], []
    area = np.zeros(n)
    for k, a, b in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
        pab = corner[b] - corner[a]
        d = np.linalg.norm(pab, axis=1)
        # signed distance of O from the line (a, b), positive on the side of corner k
        h = np.einsum("ij,ij->i", np.cross(pab, O - corner[a]), nhat) / d
        w = -h / d
        rows += [tl[:, a], tl[:, b]]
        cols += [tl[:, b], tl[:, a]]
        vals += [w, w]
        area += np.bincount(tl[:, a], weights=0.25 * d * h, minlength=n)
        area += np.bincount(tl[:, b], weights=0.25 * d * h, minlength=n)
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    diag = -np.bincount(rows, weights=vals, minlength=n)
    idx = np.arange(n)
    K = _coo(np.concatenate([rows, idx]), np.concatenate([cols, idx]), np.concatenate([vals, diag]), n)
    return dict(K=K, A=area, vert_ids=vert_ids, kept_tri=kept_tri)


def circumcenter_cell_operators(mesh):
    """Scalars at triangle circumcentres (the paper's equation for them):
    A_c (D phi)_c = l^2 sum_c' (phi_c - phi_c') l_e / d_cc' with l_e the length
    of the shared edge and d_cc' the distance between the two circumcentres;
    A_c the triangle area.  Returns dict(K, A, cell_ids)."""
    V = mesh["coords"].shape[0]
    tri = np.asarray(mesh["tri"], dtype=np.int64)
    kept, pairs = cell_subset(V, tri, mesh.get("ocean"))
    n = kept.size
    t = tri[kept]
    e1 = edge_vectors(mesh, t[:, 0], t[:, 1])
    e2 = edge_vectors(mesh, t[:, 0], t[:, 2])
    area = 0.5 * np.linalg.norm(np.cross(e1, e2), axis=1)
    O = _circumcentres(e1, e2)  # from each triangle's corner 0
    i, j = pairs[:, 0], pairs[:, 1]
    w = np.empty(i.size)
    for q in range(i.size):
        ti, tj = t[i[q]], t[j[q]]
        shared = [v for v in ti if v in set(tj.tolist())]
        a, b = shared[0], shared[1]
        le = np.linalg.norm(edge_vectors(mesh, np.array([a]), np.array([b]))[0])
        # both circumcentres as vectors from the shared vertex a
        oi = O[i[q]] - edge_vectors(mesh, np.array([ti[0]]), np.array([a]))[0]
        oj = O[j[q]] - edge_vectors(mesh, np.array([tj[0]]), np.array([a]))[0]
        w[q] = le / np.linalg.norm(oi - oj)
    deg = np.bincount(np.concatenate([i, j]), weights=np.concatenate([w, w]), minlength=n)
    idx = np.arange(n)
    K = _coo(np.concatenate([i, j, idx]), np.concatenate([j, i, idx]), np.concatenate([-w, -w, deg]), n)
    return dict(K=K.tocsr(), A=area, cell_ids=kept, pairs=pairs)


def order_operator(K, A, n):
    """G_n = K (M^-1 K)^(n-1) with M = diag(A), as an explicit sparse matrix."""
    G = K.copy()
    Minv_K = sp.diags(1.0 / A) @ K
    for _ in range(n - 1):
        G = G @ Minv_K
    return G.tocsr()
