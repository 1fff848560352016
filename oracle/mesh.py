"""Oracle: ocean subset and flat-triangle geometry.  Test infrastructure only.

Readings of the paper used here:
  * Land boundary (Sect. 2.1, no-normal-flux condition of Eq. 1-2): a triangle is
    in the ocean domain iff its three vertices are ocean; the vertex unknowns
    are the vertices of kept triangles, the cell unknowns are the kept
    triangles, both numbered by increasing original id.  Fluxes through coast
    edges are omitted, which is the natural boundary condition of the weak form.
  * Sphere geometry: every triangle is the flat (chordal) triangle spanned by
    its three vertices in 3-D; on a doubly periodic plane, edge vectors take the
    minimum image.
Parity: pinned (closed-form areas and weights on regular grids, tests).
"""

import numpy as np


def ocean_subset(n_vert, tri, ocean):
    """Kept triangles and vertices.

    Returns (kept_tri_ids, vert_ids, tri_local): original ids of kept triangles,
    original ids of the vertex unknowns (ascending), and the kept triangles'
    corners renumbered to unknown ids."""
    tri = np.asarray(tri, dtype=np.int64)
    if ocean is None:
        keep = np.ones(tri.shape[0], dtype=bool)
    else:
        oc = np.asarray(ocean).astype(bool)
        keep = oc[tri[:, 0]] & oc[tri[:, 1]] & oc[tri[:, 2]]
    kept_tri_ids = np.nonzero(keep)[0]
    used = np.zeros(n_vert, dtype=bool)
    used[tri[keep].ravel()] = True
    vert_ids = np.nonzero(used)[0]
    new_id = np.full(n_vert, -1, dtype=np.int64)
    new_id[vert_ids] = np.arange(vert_ids.size)
    return kept_tri_ids, vert_ids, new_id[tri[keep]]


def cell_subset(n_vert, tri, ocean):
    """Cell unknowns: kept triangles (ascending original id) and their
    edge-neighbour pairs among kept triangles.

    Returns (kept_tri_ids, pairs) with pairs an int64 [E, 2] array of
    unknown-index pairs (i < j) whose triangles share an edge."""
    kept_tri_ids, _, _ = ocean_subset(n_vert, tri, ocean)
    t = np.asarray(tri, dtype=np.int64)[kept_tri_ids]
    # one record per (triangle, edge) with the edge's sorted vertex pair
    recs = []
    for a, b in ((0, 1), (1, 2), (2, 0)):
        lo = np.minimum(t[:, a], t[:, b])
        hi = np.maximum(t[:, a], t[:, b])
        recs.append(np.stack([lo, hi, np.arange(t.shape[0])], 1))
    r = np.concatenate(recs, 0)
    order = np.lexsort((r[:, 2], r[:, 1], r[:, 0]))
    r = r[order]
    same = (r[1:, 0] == r[:-1, 0]) & (r[1:, 1] == r[:-1, 1])
    i = r[:-1][same, 2]
    j = r[1:][same, 2]
    pairs = np.stack([np.minimum(i, j), np.maximum(i, j)], 1)
    return kept_tri_ids, pairs


def edge_vectors(mesh, a, b):
    """x_b - x_a as 3-D vectors (planar meshes get z = 0), minimum image on a
    doubly periodic plane."""
    x = np.asarray(mesh["coords"], dtype=np.float64)
    d = x[b] - x[a]
    if mesh["geom"] == "planar_periodic":
        px, py = mesh["period_x"], mesh["period_y"]
        d = d.copy()
        d[:, 0] -= px * np.round(d[:, 0] / px)
        d[:, 1] -= py * np.round(d[:, 1] / py)
    if d.shape[1] == 2:
        d = np.concatenate([d, np.zeros((d.shape[0], 1))], 1)
    return d


def triangle_frames(mesh, tri_local_orig):
    """Per triangle (original vertex ids, [T, 3]): the three corner-to-corner
    vectors e1 = x1 - x0, e2 = x2 - x0 (3-D) and the area 1/2 |e1 x e2|."""
    t = tri_local_orig
    e1 = edge_vectors(mesh, t[:, 0], t[:, 1])
    e2 = edge_vectors(mesh, t[:, 0], t[:, 2])
    area = 0.5 * np.linalg.norm(np.cross(e1, e2), axis=1)
    return e1, e2, area
