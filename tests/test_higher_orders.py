"""Filter orders n >= 3 on the host (no GPU): the prepared operators
G_n = K (M^-1 K)^(n-1) are the products scipy forms from the exported K and
lumped mass (the vertex-vector placement through its real 2x2-block form), and
for the scalar placements they are the oracle's G_n in device order.  The
structural pattern is bit-exact, values agree to rounding, and the cache
keeps them."""

import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth

PLACEMENTS = ["vertex_scalar", "vertex_vector", "cell", "vertex_voronoi", "cell_circumcenter"]


@pytest.fixture(scope="module")
def api():
    from paper_2404_07398_gb300 import api as a
    if not os.path.exists(a.LIB_PATH):
        from paper_2404_07398_gb300 import build
        build.build()
    a.load()
    return a


def _mesh(level=3, seed=101):
    m = synth.icosphere(level, radius=6371.0, jitter=0.05, seed=seed)
    m["ocean"] = synth.land_mask(m["coords"], 0.3, seed=seed + 1, polar_cap_deg=8.0)
    return m


def _real(rowptr, col, val, n, blk):
    """Real matrix of the CSR (2x2 blocks [[a, b], [-b, a]] as (u block, v block))."""
    if not blk:
        return sp.csr_matrix((val, col, rowptr), shape=(n, n))
    A = sp.csr_matrix((val[0::2], col, rowptr), shape=(n, n))
    B = sp.csr_matrix((val[1::2], col, rowptr), shape=(n, n))
    return sp.bmat([[A, B], [-B, A]]).tocsr()


@pytest.mark.parametrize("placement", PLACEMENTS)
def test_gn_is_the_product_of_k_and_mass(api, placement):
    h = api.prepare_mesh_host(_mesh(), placement, max_order=4)
    n = h.info["n_rows"]
    blk = placement == "vertex_vector"
    K = _real(h.export("k_rowptr"), h.export("k_col"), h.export("k_val"), n, blk)
    mass = h.export("mass")
    Minv = sp.diags(1.0 / (np.concatenate([mass, mass]) if blk else mass))
    G = K.copy()
    # the structural pattern of K^n (explicit zeros kept by the library)
    P = sp.csr_matrix((np.ones(h.export("k_col").size), h.export("k_col"), h.export("k_rowptr")), shape=(n, n))
    pat = P.copy()
    for order in (2, 3, 4):
        G = (G @ Minv @ K).tocsr()
        pat = (pat @ P).tocsr()
        pat.sort_indices()
        rp, cl, vl = (h.export_gn(order, w) for w in ("rowptr", "col", "val"))
        assert np.array_equal(rp, pat.indptr.astype(np.int64)), order
        assert np.array_equal(cl, pat.indices.astype(np.int32)), order
        L = _real(rp, cl, vl, n, blk)
        scale = abs(G).max()
        assert abs(L - G).max() <= 1e-12 * scale, order
        assert abs(L - L.T).max() <= 1e-12 * scale, order       # G_n is symmetric (S stays SPD)
    # order 2 through the general export is the G2 of ifilt_mesh_export
    assert np.array_equal(h.export_gn(2, "val"), h.export("g2_val"))
    h.release()


@pytest.mark.parametrize("placement", ["vertex_scalar", "cell", "vertex_voronoi"])
def test_gn_matches_the_oracle(api, placement):
    m = _mesh(3, 103)
    h = api.prepare_mesh_host(m, placement, max_order=3)
    P = oracle.build_problem(m, placement)
    ids = P.parts["vert_ids"] if placement != "cell" else P.parts["cell_ids"]
    order = np.searchsorted(ids, h.export("perm"))
    assert np.array_equal(ids[order], h.export("perm"))
    G = oracle.order_operator(P.K, P.A, 3).tocsr()
    G = G[order][:, order].tocsr()
    n = h.info["n_rows"]
    L = sp.csr_matrix((h.export_gn(3, "val"), h.export_gn(3, "col"), h.export_gn(3, "rowptr")), shape=(n, n))
    assert abs(L - G).max() <= 1e-12 * abs(G).max()
    h.release()


def test_orders_checked_and_cached(api, tmp_path):
    m = _mesh(2, 105)
    with pytest.raises(api.IfiltError) as e:
        api.prepare_mesh_host(m, "cell", max_order=5)
    assert e.value.status == -1
    h = api.prepare_mesh_host(m, "cell", max_order=3)
    for bad in (1, 4):
        with pytest.raises(api.IfiltError):
            h.export_gn(bad, "val")
    h.save(tmp_path / "g.ifmesh")
    g = api.load_mesh_host(tmp_path / "g.ifmesh", h.key)
    for order in (2, 3):
        for w in ("rowptr", "col", "val"):
            assert np.array_equal(h.export_gn(order, w), g.export_gn(order, w))
    h.release()
    g.release()
