"""Adaptive cell quadrature for the enrichment integrals (Sec. "Enriched finite
element basis": cells are refined recursively until trial integrals of the
enrichment functions converge).

Test infrastructure only (see `oracle/__init__.py`).

Reading Q1 (the paper gives the idea, not the rule): a box is integrated with
the n^3 Gauss-Legendre rule and, again, as the sum of the same rule on its
eight half-size children; where the two estimates of every trial integral agree
to `tol` (absolute), the children's points are kept, otherwise each child is
treated the same way, down to `max_depth` levels.
"""
from __future__ import annotations

import numpy as np

from .basis import gauss_legendre, lagrange


def _box_rule(lo: np.ndarray, hi: np.ndarray, xg: np.ndarray, wg: np.ndarray):
    """Gauss-Legendre tensor rule on the box [lo, hi]: points (n^3, 3), weights."""
    n = len(xg)
    k3, k2, k1 = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    Q = np.stack([k1.ravel(), k2.ravel(), k3.ravel()], axis=1)
    mid, half = 0.5 * (lo + hi), 0.5 * (hi - lo)
    pts = mid[None, :] + xg[Q] * half[None, :]
    w = wg[Q[:, 0]] * wg[Q[:, 1]] * wg[Q[:, 2]] * np.prod(half)
    return pts, w


def _children(lo: np.ndarray, hi: np.ndarray):
    mid = 0.5 * (lo + hi)
    for i in range(8):
        b = [(i >> a) & 1 for a in range(3)]
        clo = np.where(b, mid, lo)
        chi = np.where(b, hi, mid)
        yield clo, chi


def adaptive_box(lo, hi, trial, n: int, tol: float, max_depth: int):
    """Points and weights on the box [lo, hi] by reading Q1.  trial(pts) returns
    (npts, m) values of the trial integrands."""
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    xg, wg = gauss_legendre(n)
    out_p, out_w = [], []

    def rec(l, h, depth):
        p, w = _box_rule(l, h, xg, wg)
        coarse = w @ trial(p)
        kids = [_box_rule(cl, ch, xg, wg) for cl, ch in _children(l, h)]
        fine = sum(kw @ trial(kp) for kp, kw in kids)
        if depth >= max_depth or np.all(np.abs(fine - coarse) <= tol):
            for kp, kw in kids:
                out_p.append(kp)
                out_w.append(kw)
            return
        for cl, ch in _children(l, h):
            rec(cl, ch, depth + 1)

    rec(lo, hi, 0)
    return np.concatenate(out_p), np.concatenate(out_w)


class AdaptiveRule:
    """Per-cell adaptive rules for a mesh, cached, with the cell basis's values
    and physical gradients at the points (the interface of
    electrostatic.CompositeRule: rule.cell(mesh, c) -> pts, w, B, G)."""

    def __init__(self, mesh, trial, n: int, tol: float, max_depth: int = 4):
        self.trial, self.n, self.tol, self.max_depth = trial, n, tol, max_depth
        self._cache = {}
        p1 = mesh.p + 1
        i3, i2, i1 = np.meshgrid(np.arange(p1), np.arange(p1), np.arange(p1), indexing="ij")
        self.loc = np.stack([i1.ravel(), i2.ravel(), i3.ravel()], axis=1)

    def n_points(self, mesh) -> int:
        return sum(len(self.cell(mesh, c)[1]) for c in range(mesh.n_cells))

    def cell(self, mesh, c: int):
        if c in self._cache:
            return self._cache[c]
        lo = mesh.x0[c]
        hi = lo + mesh.h[c]
        pts, w = adaptive_box(lo, hi, self.trial, self.n, self.tol, self.max_depth)
        ref = 2.0 * (pts - lo[None, :]) / mesh.h[c][None, :] - 1.0
        L = [lagrange(mesh.xi, ref[:, a]) for a in range(3)]
        loc = self.loc
        val = [L[a][0][:, loc[:, a]] for a in range(3)]
        der = [L[a][1][:, loc[:, a]] for a in range(3)]
        B = val[0] * val[1] * val[2]
        G = [der[0] * val[1] * val[2] * (2.0 / mesh.h[c, 0]), val[0] * der[1] * val[2] * (2.0 / mesh.h[c, 1]),
             val[0] * val[1] * der[2] * (2.0 / mesh.h[c, 2])]
        self._cache[c] = (pts, w, B, G)
        return self._cache[c]
