"""Host logic of the locally refined mesh in the CUDA library (no device work):
the constraint matrix P that efe_octree_constraints builds against the oracle's
(oracle.octree.OctreeMesh), node for node, on meshes of degrees 2, 3 and 5."""
import numpy as np
import pytest

MESHES = [
    ([0, 0, 0], [3, 3, 3], 3, 3, 5, [(1, 1, 1), (2, 1, 1), (0, 0, 0)]),
    ([0, 0, 0], [3, 2, 2], 3, 3, 5, [(1, 0, 0), (2, 1, 1)]),
    ([-1, 0, 0.5], [2, 2, 2.5], 4, 2, 4, [(i, j, k) for i in (1, 2) for j in (1, 2) for k in (1, 2)]),
    ([0, 0, 0], [2, 2, 2], 2, 5, 7, [(0, 0, 0)]),
]


def _lib_or_skip():
    import os
    import __graft_entry__ as g
    from paper_2210_14421_gb300 import _binding
    if not os.path.exists(_binding.LIB_PATH):
        g.build()
    return _binding


def _key(x):
    return [tuple(r) for r in np.round(np.asarray(x) * 1e6).astype(np.int64)]


@pytest.mark.parametrize("mesh", MESHES)
def test_octree_constraints_match_oracle(mesh):
    from oracle.octree import OctreeMesh
    B = _lib_or_skip()
    lo, hi, nc, p, nq, ref = mesh
    rs, col, val, axyz, fxyz = B.octree_constraints(lo, hi, nc, p, nq, ref)
    m = OctreeMesh(lo, hi, nc, p, ref)
    assert len(axyz) == m.n_all and len(fxyz) == len(m.free)
    arow = {k: i for i, k in enumerate(_key(m.nodes))}
    fcol = {k: j for j, k in enumerate(_key(m.nodes[m.free]))}
    to_o = np.array([fcol[k] for k in _key(fxyz)])
    P = np.zeros((m.n_all, len(m.free)))
    for n, k in enumerate(_key(axyz)):
        for e in range(rs[n], rs[n + 1]):
            P[arow[k], to_o[col[e]]] += val[e]
    assert np.max(np.abs(P - m.P.toarray())) < 1e-13


def test_octree_constraints_reject_bad_input():
    B = _lib_or_skip()
    with pytest.raises(B.EfeError):
        B.octree_constraints([0, 0, 0], [1, 1, 1], 2, 3, 3)           # n_quad < p + 1
    with pytest.raises(B.EfeError):
        B.octree_constraints([0, 0, 0], [1, 1, 1], 2, 3, 5, [(0, 0, 2)])
