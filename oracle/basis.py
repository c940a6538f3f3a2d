"""Quadrature rules and 1D Lagrange tables (Sec. "Spectral finite elements").

Test infrastructure only (see `oracle/__init__.py`).

The classical FE basis is the tensor product of degree-p Lagrange polynomials
whose nodes are the p+1 Gauss-Lobatto-Legendre (GLL) points of [-1, 1]; using
the GLL rule for the overlap makes the classical-classical block M^cc diagonal.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg


def gauss_legendre(n: int):
    """n-point Gauss-Legendre rule on [-1, 1] (exact for degree <= 2n - 1)."""
    x, w = npleg.leggauss(n)
    return np.asarray(x, dtype=np.float64), np.asarray(w, dtype=np.float64)


def gauss_lobatto(p: int):
    """(p+1)-point Gauss-Lobatto-Legendre rule on [-1, 1]: the end points and
    the roots of P_p'; weights 2 / (p (p+1) P_p(x_i)^2).  Exact for degree
    <= 2p - 1."""
    if p < 1:
        raise ValueError("degree must be >= 1")
    c = np.zeros(p + 1)
    c[p] = 1.0
    inner = np.sort(np.real(npleg.legroots(npleg.legder(c)))) if p > 1 else np.zeros(0)
    x = np.concatenate([[-1.0], inner, [1.0]])
    Pp = npleg.legval(x, c)
    w = 2.0 / (p * (p + 1) * Pp ** 2)
    return x, w


def lagrange(nodes: np.ndarray, x: np.ndarray):
    """Values L[k, i] = l_i(x_k) and derivatives dL[k, i] = l_i'(x_k) of the
    Lagrange polynomials on `nodes`, from the product formula."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    n = len(nodes)
    L = np.ones((len(x), n))
    dL = np.zeros((len(x), n))
    for i in range(n):
        for j in range(n):
            if j != i:
                L[:, i] *= (x - nodes[j]) / (nodes[i] - nodes[j])
        for m in range(n):
            if m == i:
                continue
            term = np.full(len(x), 1.0 / (nodes[i] - nodes[m]))
            for j in range(n):
                if j != i and j != m:
                    term *= (x - nodes[j]) / (nodes[i] - nodes[j])
            dL[:, i] += term
    return L, dL
