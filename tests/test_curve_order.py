"""Space-filling-curve device order: the oracle's rule pinned by the defining
properties of the Hilbert curve, then the library's order checked against it
bit for bit (host preparation, no GPU)."""

import numpy as np
import pytest

import oracle
import synth


def test_hilbert_order_one_is_the_u_shape():
    assert [oracle.hilbert_index(x, y, 1) for x, y in ((0, 0), (0, 1), (1, 1), (1, 0))] == [0, 1, 2, 3]


@pytest.mark.parametrize("bits", [1, 2, 3, 4, 5])
def test_hilbert_curve_is_a_continuous_bijection(bits):
    n = 1 << bits
    pos = {}
    for x in range(n):
        for y in range(n):
            d = oracle.hilbert_index(x, y, bits)
            assert d not in pos
            pos[d] = (x, y)
    assert sorted(pos) == list(range(n * n))
    assert pos[0] == (0, 0) and pos[n * n - 1] == (n - 1, 0)
    for d in range(n * n - 1):
        (x0, y0), (x1, y1) = pos[d], pos[d + 1]
        assert abs(x0 - x1) + abs(y0 - y1) == 1


def test_cube_faces_and_ties():
    pts = np.array([[1.0, 0.2, -0.1], [-1.0, 0.0, 0.0], [0.1, 2.0, 0.3], [0.0, -3.0, 1.0],
                    [0.2, 0.1, 5.0], [0.0, 0.0, -1.0], [1.0, 1.0, 0.5], [0.0, -1.0, -1.0]])
    faces = oracle.curve_keys(pts, True) >> (2 * 16)
    assert list(faces) == [0, 1, 2, 3, 4, 5, 0, 3]
    # the face centre maps to the middle of the grid
    k = oracle.curve_keys(np.array([[0.0, 0.0, 1.0]]), True)[0] & ((1 << 32) - 1)
    assert k == oracle.hilbert_index(1 << 15, 1 << 15, 16)


def _mesh(kind):
    if kind == "sphere":
        m = synth.icosphere(4, radius=6371.0, jitter=0.2, seed=41)
        m["ocean"] = synth.land_mask(m["coords"], 0.3, seed=42, polar_cap_deg=8.0)
        return m
    m = synth.periodic_split_square(24, 20, 1.0)
    m["ocean"] = None
    return m


@pytest.mark.parametrize("kind,placement", [("sphere", "vertex_scalar"), ("sphere", "vertex_vector"),
                                            ("sphere", "cell"), ("plane", "vertex_scalar"), ("plane", "cell")])
def test_library_curve_order_matches_oracle(kind, placement):
    from paper_2404_07398_gb300 import api
    api.load()
    m = _mesh(kind)
    h = api.prepare_mesh_host(m, placement, max_order=1, reorder=api.REORDER_HILBERT)
    assert np.array_equal(h.export("perm"), oracle.curve_order(m, placement))


def test_curve_order_is_local():
    """Consecutive unknowns sit close together: on the sphere the mean distance
    between device neighbours is a small multiple of the edge length, far below
    that of the original numbering's random jitter."""
    from paper_2404_07398_gb300 import api
    api.load()
    m = _mesh("sphere")
    h = api.prepare_mesh_host(m, "vertex_scalar", max_order=1, reorder=api.REORDER_HILBERT)
    p = m["coords"][h.export("perm")]
    step = np.linalg.norm(np.diff(p, axis=0), axis=1)
    edge = 6371.0 * 1.1 / (2 ** 4)
    assert np.median(step) < 2 * edge
