"""Pins of the adaptive cell quadrature (oracle.quadrature, reading Q1)."""
import math

import numpy as np
from scipy.special import erf

from oracle import quadrature as q


def test_polynomials_need_no_refinement():
    """A product of per-axis polynomials of degree <= 2n - 1 is integrated
    exactly by the first comparison, which then stops (8 n^3 points)."""
    n = 4
    lo, hi = np.array([-1.0, 0.5, 2.0]), np.array([0.5, 2.0, 2.5])

    def f(p):
        return ((p[:, 0] ** 7 - 2 * p[:, 0]) * (p[:, 1] ** 5 + 1.0) * p[:, 2] ** 6)[:, None]

    pts, w = q.adaptive_box(lo, hi, f, n, 1e-12, 5)
    assert len(w) == 8 * n ** 3
    ix = (hi[0] ** 8 / 8 - hi[0] ** 2) - (lo[0] ** 8 / 8 - lo[0] ** 2)
    iy = (hi[1] ** 6 / 6 + hi[1]) - (lo[1] ** 6 / 6 + lo[1])
    iz = (hi[2] ** 7 - lo[2] ** 7) / 7
    assert abs(w @ f(pts)[:, 0] - ix * iy * iz) < 1e-12 * abs(ix * iy * iz)


def test_narrow_gaussian_converges_with_the_tolerance():
    """A Gaussian of width 0.1 off-centre in a box of side 2: the error follows
    the requested tolerance (closed form by error functions)."""
    c0, sg = np.array([0.31, -0.17, 0.44]), 0.1
    lo, hi = -np.ones(3), np.ones(3)

    def f(p):
        return np.exp(-np.sum((p - c0) ** 2, axis=1) / (2 * sg * sg))[:, None]

    exact = np.prod([math.sqrt(math.pi / 2) * sg * (erf((hi[a] - c0[a]) / (math.sqrt(2) * sg))
                                                    - erf((lo[a] - c0[a]) / (math.sqrt(2) * sg))) for a in range(3)])
    errs, npts = [], []
    for tol in (1e-6, 1e-9):
        pts, w = q.adaptive_box(lo, hi, f, 6, tol, 6)
        errs.append(abs(w @ f(pts)[:, 0] - exact))
        npts.append(len(w))
    assert errs[0] < 1e-7 and errs[1] < 1e-10, errs
    assert npts[1] > npts[0]


def test_adaptive_rule_serves_the_enriched_poisson_solve():
    """The nuclear enriched solve with the adaptive rule (trial integrands: the
    smeared charge and the atomic potential) matches the uniform 4^3-sub-cell
    rule's accuracy with at most half its points: refinement goes to the cells
    around the nucleus only."""
    from oracle import electrostatic as es
    from oracle.mesh import Mesh
    b = np.linspace(-6.0, 6.0, 5)
    m = Mesh(b, b, b, 4, 6)
    Z, R, sg = [5.0], [np.zeros(3)], 0.25
    pot = es.nuclear_radial(5.0, sg)

    def trial(p):
        return np.stack([es.smeared_charge(Z, R, sg, p), pot(np.linalg.norm(p, axis=1))[0]], axis=1)

    def error(P):
        phi, phiE = P.solve()
        err = ref = 0.0
        for c in range(m.n_cells):
            pts, val = P.evaluate(phi, phiE, c)
            ex = es.smeared_potential(Z, R, sg, pts)
            err, ref = max(err, np.abs(val - ex).max()), max(ref, np.abs(ex).max())
        return err / ref

    e_uniform = error(es.NuclearEFE(m, Z, R, sg, r0=5.5, s=4.0, sub=4, n=6))
    rule = q.AdaptiveRule(m, trial, 6, 1e-7, 4)
    e_adapt = error(es.NuclearEFE(m, Z, R, sg, r0=5.5, s=4.0, rule=rule))
    assert abs(e_adapt - e_uniform) < 0.05 * e_uniform
    assert rule.n_points(m) <= 0.5 * m.n_cells * 24 ** 3
