"""Pins of the enrichment functions (Eq. EFEAtomic) against closed forms and
finite differences."""
import math

import numpy as np
import pytest

from oracle import enrich


def test_cutoff_values_and_derivative():
    r0, s = 6.0, 3.0
    r = np.linspace(0.0, 8.0, 801)
    u, du = enrich.cutoff(r, r0, s)
    assert np.all(u[r <= r0 - s] == 1.0)
    assert np.all(u[r >= r0] == 0.0)
    assert np.all(np.diff(u) <= 1e-15)                # monotone non-increasing
    rm = np.linspace(3.05, 5.95, 59)
    h = 1e-6
    fd = (enrich.cutoff(rm + h, r0, s)[0] - enrich.cutoff(rm - h, r0, s)[0]) / (2 * h)
    assert np.allclose(enrich.cutoff(rm, r0, s)[1], fd, atol=1e-8)
    # symmetric step: u(r0 - s/2) = 1/2
    assert abs(enrich.cutoff(np.array([r0 - s / 2]), r0, s)[0][0] - 0.5) < 1e-15


def test_hydrogenic_shapes_closed_forms():
    r = np.linspace(0.01, 5.0, 50)
    Z = 3.0
    rho = Z * r
    f, _ = enrich.radial(enrich.RADIAL_HYDROGENIC, 1, 0, Z, r)
    assert np.allclose(f, np.exp(-rho))
    f, _ = enrich.radial(enrich.RADIAL_HYDROGENIC, 2, 0, Z, r)
    assert np.allclose(f, (2 - rho) * np.exp(-rho / 2))
    f, _ = enrich.radial(enrich.RADIAL_HYDROGENIC, 2, 1, Z, r)          # R_21 / r
    assert np.allclose(f * r, rho * np.exp(-rho / 2))
    f, _ = enrich.radial(enrich.RADIAL_HYDROGENIC, 3, 0, Z, r)
    assert np.allclose(f * 9.0, (27 - 18 * rho + 2 * rho ** 2) * np.exp(-rho / 3))
    f, _ = enrich.radial(enrich.RADIAL_SLATER, 1, 0, 1.0, r)
    assert np.allclose(f, np.exp(-r))


@pytest.mark.parametrize("kind,n,l,zeta", [(0, 1, 0, 1.3), (0, 2, 1, 0.9), (1, 2, 0, 2.5), (1, 3, 0, 1.5),
                                           (1, 3, 1, 2.0), (1, 3, 2, 2.0), (2, 1, 0, 0.7)])
def test_radial_derivatives(kind, n, l, zeta):
    r = np.linspace(0.1, 6.0, 40)
    h = 1e-6
    f, df = enrich.radial(kind, n, l, zeta, r)
    fd = (enrich.radial(kind, n, l, zeta, r + h)[0] - enrich.radial(kind, n, l, zeta, r - h)[0]) / (2 * h)
    assert np.allclose(df, fd, rtol=1e-6, atol=1e-9)


def test_solid_harmonics_orthogonal_on_sphere():
    # product Gauss-Legendre (cos theta) x uniform (phi) rule, exact for these degrees
    ct, wt = np.polynomial.legendre.leggauss(12)
    ph = np.linspace(0, 2 * np.pi, 24, endpoint=False)
    CT, PH = np.meshgrid(ct, ph, indexing="ij")
    st = np.sqrt(1 - CT ** 2)
    d = np.stack([(st * np.cos(PH)).ravel(), (st * np.sin(PH)).ravel(), CT.ravel()], axis=1)
    w = (wt[:, None] * np.full(len(ph), 2 * np.pi / len(ph))[None, :]).ravel()
    lm = [(0, 0)] + [(1, m) for m in (-1, 0, 1)] + [(2, m) for m in (-2, -1, 0, 1, 2)]
    vals = [enrich.solid_harmonic(l, m, d)[0] for (l, m) in lm]
    G = np.array([[np.sum(w * a * b) for b in vals] for a in vals])
    off = G - np.diag(np.diag(G))
    assert np.max(np.abs(off)) < 1e-13
    assert abs(G[0, 0] - 4 * math.pi) < 1e-12
    assert abs(G[1, 1] - 4 * math.pi / 3) < 1e-12


@pytest.mark.parametrize("l,m", [(0, 0), (1, -1), (1, 0), (1, 1), (2, 0), (2, 2)])
def test_enrichment_gradient_fd(l, m):
    class F:
        pass
    fn = F()
    fn.radial, fn.n, fn.l, fn.m, fn.zeta = enrich.RADIAL_HYDROGENIC, 3, l, m, 1.7
    c = np.array([0.2, -0.1, 0.3])
    pts = np.random.default_rng(4).uniform(-4, 4, size=(200, 3))
    v, g = enrich.evaluate(fn, c, pts, 5.0, 2.0)
    h = 1e-6
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        fd = (enrich.evaluate(fn, c, pts + e, 5.0, 2.0)[0] - enrich.evaluate(fn, c, pts - e, 5.0, 2.0)[0]) / (2 * h)
        assert np.allclose(g[:, a], fd, rtol=1e-6, atol=1e-8)
