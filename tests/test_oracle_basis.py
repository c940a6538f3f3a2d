"""Pins of the oracle's quadrature rules, Lagrange tables and mesh against
closed forms (Sec. "Spectral finite elements")."""
import math

import numpy as np
import pytest

import efe_workloads as W
from oracle import basis, mesh, operators


@pytest.mark.parametrize("n", [2, 3, 5, 6, 7])
def test_gauss_legendre_exact_to_degree_2n_minus_1(n):
    x, w = basis.gauss_legendre(n)
    for k in range(2 * n):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * x ** k) - exact) < 1e-14
    # and not beyond: x^(2n) is integrated with an error
    assert abs(np.sum(w * x ** (2 * n)) - 2.0 / (2 * n + 1)) > 1e-6


def test_gll_closed_forms():
    x, w = basis.gauss_lobatto(2)
    assert np.allclose(x, [-1, 0, 1], atol=1e-15)
    assert np.allclose(w, [1 / 3, 4 / 3, 1 / 3], atol=1e-15)
    x, w = basis.gauss_lobatto(4)
    s = math.sqrt(3.0 / 7.0)
    assert np.allclose(x, [-1, -s, 0, s, 1], atol=1e-15)
    assert np.allclose(w, [0.1, 49 / 90, 32 / 45, 49 / 90, 0.1], atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_gll_exact_to_degree_2p_minus_1(p):
    x, w = basis.gauss_lobatto(p)
    for k in range(2 * p):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * x ** k) - exact) < 1e-14


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_lagrange_tables(p):
    nodes, _ = basis.gauss_lobatto(p)
    L, dL = basis.lagrange(nodes, nodes)
    assert np.allclose(L, np.eye(p + 1), atol=1e-14)
    xs = np.linspace(-1, 1, 17)
    L, dL = basis.lagrange(nodes, xs)
    assert np.allclose(L.sum(axis=1), 1.0, atol=1e-13)      # partition of unity
    assert np.allclose(dL.sum(axis=1), 0.0, atol=1e-12)
    # reproduces x^k exactly for k <= p, derivatives too
    for k in range(p + 1):
        assert np.allclose(L @ nodes ** k, xs ** k, atol=1e-13)
        assert np.allclose(dL @ nodes ** k, k * xs ** max(k - 1, 0) if k else 0.0, atol=1e-11)


def _mesh(n=(3, 4, 2), p=3, nq=5, L=(6.0, 8.0, 5.0)):
    b = [np.sort(np.concatenate([[-l / 2, l / 2], np.random.default_rng(1).uniform(-l / 2, l / 2, k - 1)]))
         for l, k in zip(L, n)]
    return mesh.Mesh(b[0], b[1], b[2], p, nq), b


def test_lumped_mass_sums_to_volume():
    m, b = _mesh()
    vol = np.prod([bb[-1] - bb[0] for bb in b])
    M = m.lumped_mass()
    assert np.all(M > 0)
    assert abs(M.sum() - vol) < 1e-12 * vol
    assert abs(m.wJ.sum() - vol) < 1e-12 * vol


def _system_no_enrichment(n=3, p=3, nq=5, L=8.0, graded=True):
    if graded:
        b = W.graded_bounds(L, [0.3], 0.8, 3.0, n)
    else:
        b = W.uniform_bounds(L, n)
    wl = W.h2().with_(xb=b, yb=b, zb=b, degree=p, n_quad=nq, enrich=[], Z=np.zeros(0), R=np.zeros((0, 3)))
    return operators.System(wl)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_stiffness_on_polynomials(p):
    """1/2 int grad N_i . grad u = -1/2 int N_i lap u for interior i: zero for
    linear u, -int N_i for u = x^2 (pins the kinetic 1/2 and the assembly)."""
    S = _system_no_enrichment(n=3, p=p, nq=p + 2)
    X = S.mesh.nodes
    I = S.mesh.interior
    Vone = S.potential_blocks(np.ones(S.mesh.wJ.shape))[0]
    intN = Vone @ np.ones(S.n_h)                     # int N_i (partition of unity)
    for u in (X[:, 0], X[:, 1] - 2 * X[:, 2] + 0.5):
        assert np.max(np.abs((S.Kcc @ u)[I])) < 1e-12
    r = S.Kcc @ (X[:, 0] ** 2)
    assert np.allclose(r[I], -intN[I], rtol=1e-11, atol=1e-13)
    r = S.Kcc @ np.sum(X ** 2, axis=1)
    assert np.allclose(r[I], -3 * intN[I], rtol=1e-11, atol=1e-13)


def test_potential_matrix_integrals():
    S = _system_no_enrichment(n=3, p=3, nq=5)
    vol = S.mesh.wJ.sum()
    one = np.ones(S.n_h)
    V = S.potential_blocks(np.ones(S.mesh.wJ.shape))[0]
    assert abs(one @ V @ one - vol) < 1e-11 * vol
    # int x^2 over the box with v = x and u = x nodal
    X = S.mesh.nodes
    Vx = S.potential_blocks(S.mesh.xq[:, :, 0])[0]
    bx = S.mesh.b[0]
    by, bz = S.mesh.b[1], S.mesh.b[2]
    exact = (bx[-1] ** 3 - bx[0] ** 3) / 3 * (by[-1] - by[0]) * (bz[-1] - bz[0])   # int x * x
    assert abs(one @ Vx @ X[:, 0] - exact) < 1e-10 * abs(exact)
