"""Pins of the oracle's ocean subset and reverse Cuthill-McKee rule (no GPU)."""

import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth
from oracle.mesh import ocean_subset, cell_subset

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rcm_hand_cases.txt")


def _cases():
    out = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, n, edges, order = [s.strip() for s in line.split("|")]
        e = [tuple(int(v) for v in s.split("-")) for s in edges.split()]
        out.append((name, int(n), e, [int(v) for v in order.split()]))
    return out


def _csr(n, edges):
    r = [a for a, b in edges] + [b for a, b in edges] + list(range(n))
    c = [b for a, b in edges] + [a for a, b in edges] + list(range(n))
    A = sp.coo_matrix((np.ones(len(r)), (r, c)), shape=(n, n)).tocsr()
    return A.indptr, A.indices


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_rcm_hand_cases(case):
    name, n, edges, expected = case
    ip, ix = _csr(n, edges)
    assert list(oracle.rcm_order(ip, ix)) == expected
    assert oracle.check_rcm_order(ip, ix, expected)


def test_rcm_checker_rejects_other_orders():
    name, n, edges, expected = _cases()[2]
    ip, ix = _csr(n, edges)
    bad = list(expected)
    bad[1], bad[2] = bad[2], bad[1]
    with pytest.raises(AssertionError):
        oracle.check_rcm_order(ip, ix, bad)


def test_rcm_checker_agrees_with_loop_version_on_masked_sphere():
    m = synth.icosphere(4, radius=1.0, jitter=0.2, seed=3)
    m["ocean"] = synth.land_mask(m["coords"], 0.3, seed=4)
    P = oracle.build_problem(m, "vertex_scalar")
    K = P.K
    order = oracle.rcm_order(K.indptr, K.indices)
    assert oracle.check_rcm_order(K.indptr, K.indices, order)
    rng = np.random.default_rng(0)
    for _ in range(3):
        o2 = order.copy()
        i, j = rng.choice(order.size, 2, replace=False)
        o2[i], o2[j] = o2[j], o2[i]
        with pytest.raises(AssertionError):
            oracle.check_rcm_order(K.indptr, K.indices, o2)


def test_ocean_subset_hand_example():
    # square 0-1-2-3 split into (0,1,2), (0,2,3) plus a third triangle (1,4,2)
    tri = np.array([[0, 1, 2], [0, 2, 3], [1, 4, 2]])
    ocean = np.array([1, 1, 1, 0, 1], dtype=np.uint8)      # vertex 3 is land
    kept, vids, tl = ocean_subset(5, tri, ocean)
    assert list(kept) == [0, 2]
    assert list(vids) == [0, 1, 2, 4]
    assert tl.tolist() == [[0, 1, 2], [1, 3, 2]]
    kc, pairs = cell_subset(5, tri, ocean)
    assert list(kc) == [0, 2] and pairs.tolist() == [[0, 1]]
