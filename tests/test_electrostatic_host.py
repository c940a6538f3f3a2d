"""Host logic of the electrostatic enrichment in the CUDA library (no device
work), through its host-only diagnostics: the atomic Hartree tables against the
oracle's RadialAtom (reading H1) and the adaptive cell rule's boxes against the
oracle's adaptive_box (reading Q1), box for box."""
import os

import numpy as np
import pytest

import efe_workloads as W


def _binding():
    import __graft_entry__ as g
    from paper_2210_14421_gb300 import _binding
    if not os.path.exists(_binding.LIB_PATH):
        g.build()
    return _binding


def _shells(wl, J):
    out = []
    for f in wl.enrich:
        t = (f.radial, f.n, f.l, f.zeta)
        if f.atom == J and t not in out:
            out.append(t)
    return out


@pytest.mark.parametrize("make", [lambda: W.na_cluster(n_atoms=2, cells_per_axis=5),
                                  lambda: W.small_cluster(n_atoms=2), lambda: W.h2()])
def test_atom_tables_match_radial_atom(make):
    from oracle import electrostatic as es
    B = _binding()
    wl = make()
    r, v, q, nel = B.atom_hartree_table(wl.enrich, wl.Z)
    for J in range(len(wl.Z)):
        A = es.RadialAtom(_shells(wl, J), float(wl.Z[J]))
        assert np.max(np.abs(r - A.r)) <= 1e-14 * A.r[-1]
        assert np.max(np.abs(v[J] - A.v)) <= 1e-12 * np.max(np.abs(A.v))
        assert np.max(np.abs(q[J] - A.q)) <= 1e-12 * np.max(np.abs(A.q))
        assert abs(nel[J] - A.n_el) <= 1e-12 * A.n_el


def test_adaptive_boxes_match_oracle():
    """Every cell of a small two-atom mesh: the library's refinement keeps the same
    boxes as the oracle's (same trial integrands: the smeared charge and the
    truncated smeared-nucleus potentials)."""
    from oracle import electrostatic as es
    from oracle import quadrature as qd
    from oracle.enrich import cutoff
    from oracle.mesh import Mesh
    B = _binding()
    wl = W.small_cluster(n_atoms=2, cells_per_axis=5, degree=3, n_quad=5, n_orb=3)
    sigma, r0, s, n, tol, depth = 0.3, 3.0, 1.5, 5, 1e-6, 3
    Z, R = list(wl.Z), [np.asarray(x) for x in wl.R]
    rad = [es.nuclear_radial(z, sigma) for z in Z]

    def trial(p):
        cols = [es.smeared_charge(Z, R, sigma, p)]
        for J in range(len(Z)):
            rr = np.linalg.norm(p - R[J][None, :], axis=1)
            cols.append(rad[J](rr)[0] * cutoff(rr, r0, s)[0])
        return np.stack(cols, axis=1)

    m = Mesh(wl.xb, wl.yb, wl.zb, wl.degree, wl.n_quad)
    refined = 0
    for c in range(m.n_cells):
        lo, h = m.x0[c], m.h[c]
        _, w = qd.adaptive_box(lo, lo + h, trial, n, tol, depth)
        boxes = B.adaptive_cell_boxes(lo, h, Z, np.array(R), sigma, r0, s, n, tol, depth)
        assert len(boxes) * n ** 3 == len(w), c
        refined += len(boxes) > 8
        # the boxes tile the reference cell
        vol = np.prod(boxes[:, 3:] - boxes[:, :3], axis=1).sum()
        assert abs(vol - 8.0) < 1e-12
    assert refined > 0
