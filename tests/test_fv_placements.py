"""The two finite-volume placements (no GPU): quasi-hexagonal control volumes
around the vertices (Eq. 3-5) and scalars at triangle circumcentres.

Oracle pins, each against something other than the oracle's own formula:
  * the Voronoi weights l/d equal the P1 cotangent weights computed from
    gradients (the identity l_e = (d/2)(cot a + cot b) of circumcentric duals);
  * the Voronoi areas tile the ocean domain exactly;
  * closed forms on the split square (5-point stencil, unit squares, and the
    hypotenuse gets weight 0) and on the equilateral lattice (hexagons of area
    (sqrt 3 / 2) a^2, weight 1/sqrt 3; circumcentre weight sqrt 3, which is
    Eq. 6 with A = sqrt 3);
  * circumcentres recomputed by brute force as the in-plane point equidistant
    from the three corners;
  * filter invariants (constants pass, the area-weighted mean is kept) and
    the CG solve against a dense solve.
Then the library's host preparation against the oracle (permutation and
pattern bit for bit, values to rounding) and its rejection of meshes the
placements cannot discretise.
"""

import os

import numpy as np
import pytest

import oracle
import synth
from oracle.mesh import edge_vectors

FV = ["vertex_voronoi", "cell_circumcenter"]


def _sphere(level, seed, land=0.3):
    m = synth.icosphere(level, radius=6371.0, jitter=0.2, seed=seed)
    m["ocean"] = synth.land_mask(m["coords"], land, seed=seed + 1, polar_cap_deg=8.0) if land else None
    return m


def _tri_areas(m, t):
    e1 = edge_vectors(m, t[:, 0], t[:, 1])
    e2 = edge_vectors(m, t[:, 0], t[:, 2])
    return 0.5 * np.linalg.norm(np.cross(e1, e2), axis=1)


def test_voronoi_weights_are_cotangent_weights():
    m = _sphere(3, 71)
    so = oracle.scalar_vertex_operators(m)
    vo = oracle.voronoi_vertex_operators(m)
    assert np.array_equal(so["vert_ids"], vo["vert_ids"])
    assert abs(so["K"] - vo["K"]).max() <= 1e-13 * abs(so["K"]).max()


def test_voronoi_areas_tile_the_domain():
    m = _sphere(3, 73)
    vo = oracle.voronoi_vertex_operators(m)
    t = np.asarray(m["tri"], dtype=np.int64)[vo["kept_tri"]]
    total = _tri_areas(m, t).sum()
    assert abs(vo["A"].sum() - total) <= 1e-12 * total
    assert (vo["A"] > 0).all()


def test_voronoi_split_square_closed_form():
    h = 0.5
    m = synth.periodic_split_square(8, 8, h=h)
    vo = oracle.voronoi_vertex_operators(m)
    np.testing.assert_allclose(vo["A"], h * h, rtol=1e-14)
    K = vo["K"].toarray()
    x = np.asarray(m["coords"])
    n = x.shape[0]
    for v in range(n):
        d = x - x[v]
        d -= 8 * h * np.round(d / (8 * h))
        r = np.hypot(d[:, 0], d[:, 1])
        axis = np.isclose(r, h)
        assert np.allclose(K[v, axis], -1.0, atol=1e-14)           # l / d = h / h
        other = ~axis & (np.arange(n) != v)
        assert np.abs(K[v, other]).max() <= 1e-14                    # hypotenuse: l = 0
        assert abs(K[v, v] - 4.0) <= 1e-14


def test_equilateral_lattice_closed_forms():
    a = 2.0
    m = synth.periodic_equilateral(6, 6, a=a)
    vo = oracle.voronoi_vertex_operators(m)
    np.testing.assert_allclose(vo["A"], np.sqrt(3) / 2 * a * a, rtol=1e-13)
    K = vo["K"].tocoo()
    off = K.data[K.row != K.col]
    assert off.size == 6 * 36
    np.testing.assert_allclose(off, -1 / np.sqrt(3), rtol=1e-13)
    co = oracle.circumcenter_cell_operators(m)
    np.testing.assert_allclose(co["A"], np.sqrt(3) / 4 * a * a, rtol=1e-13)
    ce = oracle.cell_operators(m, np.sqrt(3))
    assert abs(co["K"] - ce["K"]).max() <= 1e-13 * np.sqrt(3)


def _bruteforce_circumcentre(p0, p1, p2):
    """Solve |x - p0|^2 = |x - p1|^2 = |x - p2|^2 with x in the triangle's plane
    (3 x 3 linear system), independent of the Gram-system route."""
    n = np.cross(p1 - p0, p2 - p0)
    A = np.stack([2 * (p1 - p0), 2 * (p2 - p0), n])
    b = np.array([p1 @ p1 - p0 @ p0, p2 @ p2 - p0 @ p0, n @ p0])
    return np.linalg.solve(A, b)


def test_circumcentre_weights_by_bruteforce():
    m = _sphere(2, 75)
    co = oracle.circumcenter_cell_operators(m)
    x = np.asarray(m["coords"], dtype=np.float64)
    t = np.asarray(m["tri"], dtype=np.int64)[co["cell_ids"]]
    O = np.array([_bruteforce_circumcentre(*x[tt]) for tt in t])
    K = co["K"].tocsr()
    for i, j in co["pairs"]:
        shared = sorted(set(t[i].tolist()) & set(t[j].tolist()))
        le = np.linalg.norm(x[shared[0]] - x[shared[1]])
        w = le / np.linalg.norm(O[i] - O[j])
        assert abs(K[i, j] + w) <= 1e-12 * w
    np.testing.assert_allclose(co["A"], _tri_areas(m, t), rtol=1e-13)
    assert abs(K - K.T).max() == 0
    assert np.abs(K @ np.ones(K.shape[0])).max() <= 1e-12 * abs(K).max()


@pytest.mark.parametrize("placement", FV)
def test_constant_passes_and_mean_is_kept(placement):
    m = _sphere(3, 77)
    P = oracle.build_problem(m, placement)
    f = np.full((1, P.n_in), 1.75)
    out, _ = oracle.filter_field(P, f, [2 * np.pi / 3000.0, 2 * np.pi / 300.0], 2)
    assert np.max(np.abs(out - 1.75)) < 1e-12
    rng = np.random.default_rng(3)
    g = rng.normal(size=(1, P.n_in))
    ids = P.out_ids
    for order in (1, 2):
        out, _ = oracle.filter_field(P, g, [2 * np.pi / 2000.0], order, rtol=1e-13)
        assert np.isclose(P.A @ out[0, 0][ids], P.A @ g[0][ids], rtol=1e-9, atol=1e-9 * np.abs(P.A).sum())


@pytest.mark.parametrize("placement", FV)
@pytest.mark.parametrize("order", [1, 2])
def test_cg_matches_dense_solve(placement, order):
    m = _sphere(2, 79)
    P = oracle.build_problem(m, placement)
    rng = np.random.default_rng(1)
    f = rng.normal(size=(P.n_comp, P.n_in))
    ks = 2 * np.pi / np.array([5000.0, 2000.0, 800.0])
    a, _ = oracle.filter_field(P, f, ks, order)
    b = oracle.filter_dense(P, f, ks, order)
    assert np.max(np.abs(a - b)) < 1e-11 * np.max(np.abs(b))
    for o in (1, 2):
        S = oracle.solve.dense_S(P, 3000.0, o)
        assert np.max(np.abs(S - S.T)) <= 1e-12 * np.max(np.abs(S))
        assert np.linalg.eigvalsh(0.5 * (S + S.T)).min() > 0


# ---- the library's host preparation ------------------------------------------------


@pytest.fixture(scope="module")
def api():
    from paper_2404_07398_gb300 import api as a
    if not os.path.exists(a.LIB_PATH):
        from paper_2404_07398_gb300 import build
        build.build()
    a.load()
    return a


@pytest.mark.parametrize("placement", FV)
@pytest.mark.parametrize("reorder", [0, 1])
def test_host_prepare_matches_oracle(api, placement, reorder):
    import scipy.sparse as sp
    m = _sphere(3, 81)
    h = api.prepare_mesh_host(m, placement, max_order=2, reorder=reorder)
    P = oracle.build_problem(m, placement)
    ids = P.parts["vert_ids"] if placement == "vertex_voronoi" else P.parts["cell_ids"]
    order = oracle.rcm_order(P.K.indptr, P.K.indices) if reorder else np.arange(ids.size)
    assert h.info["n_comp"] == 1 and h.info["n_rows"] == ids.size
    assert np.array_equal(h.export("perm"), ids[order])
    inv = np.empty_like(order)
    inv[order] = np.arange(order.size)
    C = P.K.tocoo()
    B = sp.coo_matrix((C.data, (inv[C.row], inv[C.col])), shape=P.K.shape).tocsr()
    B.sort_indices()
    assert np.array_equal(h.export("k_rowptr"), B.indptr.astype(np.int64))
    assert np.array_equal(h.export("k_col"), B.indices.astype(np.int32))
    assert np.max(np.abs(h.export("k_val") - B.data)) <= 1e-13 * np.abs(B.data).max()
    np.testing.assert_allclose(h.export("mass"), P.A[order], rtol=1e-13)
    h.release()


def test_coincident_circumcentres_are_rejected(api):
    """Split squares are right triangles: both triangles of a square share the
    hypotenuse midpoint as circumcentre, so d_cc' = 0 and the circumcentre
    placement has no flux weight there.  The library refuses the mesh; the
    Voronoi placement of the same mesh is fine (that edge gets weight 0)."""
    m = synth.periodic_split_square(6, 6, h=1.0)
    with pytest.raises(api.IfiltError):
        api.prepare_mesh_host(m, "cell_circumcenter", max_order=1)
    h = api.prepare_mesh_host(m, "vertex_voronoi", max_order=1)
    np.testing.assert_allclose(h.export("mass"), 1.0, rtol=1e-14)
    h.release()


def test_negative_dual_area_is_rejected(api):
    """A coast vertex whose only triangle is very obtuse elsewhere has a
    negative circumcentric dual area (the circumcentre lies outside); the
    Voronoi placement cannot lump a mass there and the library refuses."""
    coords = np.array([[0.0, 0.0], [1.0, 0.0], [0.5, 0.1], [0.5, -0.8]])
    tri = np.array([[0, 1, 2], [0, 3, 1]], dtype=np.int32)
    m = dict(coords=coords, tri=tri, geom="planar", period_x=0.0, period_y=0.0, radius=0.0)
    vo = oracle.voronoi_vertex_operators(m)
    assert (vo["A"] <= 0).any()
    with pytest.raises(api.IfiltError):
        api.prepare_mesh_host(m, "vertex_voronoi", max_order=1)
    # the same mesh is fine for the P1 placement (lumped mass A/3 > 0)
    api.prepare_mesh_host(m, "vertex_scalar", max_order=1).release()
