"""Pins of the LDA (Slater + PW92) and of the Hartree solve."""
import math

import numpy as np
import pytest
from scipy.special import erf

import efe_workloads as W
from oracle import operators, poisson, xc


def test_slater_closed_form():
    rho = np.array([1.0, 0.1, 1e-3])
    ex, vx = xc.slater_exchange(rho)
    cx = 0.75 * (3.0 / math.pi) ** (1.0 / 3.0)            # 0.738559...
    assert abs(cx - 0.7385587663820224) < 1e-15
    assert np.allclose(ex, -cx * rho ** (1 / 3), rtol=1e-14)
    assert np.allclose(vx, 4.0 / 3.0 * ex, rtol=1e-14)


def test_potentials_are_derivatives_of_energy_density():
    rho = np.logspace(-6, 2, 40)
    h = 1e-5 * rho
    ex_p, _ = xc.lda(rho + h)
    ex_m, _ = xc.lda(rho - h)
    fd = ((rho + h) * ex_p - (rho - h) * ex_m) / (2 * h)
    _, v = xc.lda(rho)
    assert np.allclose(v, fd, rtol=1e-8)
    ec_p, _ = xc.pw92_correlation(rho + h)
    ec_m, _ = xc.pw92_correlation(rho - h)
    fdc = ((rho + h) * ec_p - (rho - h) * ec_m) / (2 * h)
    assert np.allclose(xc.pw92_correlation(rho)[1], fdc, rtol=1e-7)


def test_pw92_high_density_limit_constants():
    """PW92 is built so that eps_c -> c0 ln r_s - c1 as r_s -> 0 with
    c0 = (1 - ln 2) / pi^2 and c1 = 0.046644: A = c0,
    beta1 = exp(-c1 / (2 c0)) / (2 c0), beta2 = 2 A beta1^2."""
    c0 = (1.0 - math.log(2.0)) / math.pi ** 2
    c1 = 0.046644
    assert abs(xc.PW92_A - c0) < 1e-6
    b1 = math.exp(-c1 / (2 * c0)) / (2 * c0)
    assert abs(xc.PW92_BETA[0] - b1) < 2e-3
    assert abs(xc.PW92_BETA[1] - 2 * c0 * b1 ** 2) < 2e-3
    rs = np.array([1e-4, 1e-5])
    ec, _ = xc.pw92_eps_c(rs)
    assert np.allclose(ec, c0 * np.log(rs) - c1, atol=2e-3 * np.abs(np.log(rs)).max() * 1e-1 + 1e-3)


def test_correlation_negative_and_floor():
    ec, vc = xc.pw92_correlation(np.logspace(-10, 3, 30))
    assert np.all(ec < 0) and np.all(vc < 0)
    e, v = xc.lda(np.array([0.0, 1e-15]))
    assert np.all(e == 0) and np.all(v == 0)


@pytest.mark.parametrize("n", [4, 6])
def test_hartree_gaussian_charge(n):
    """rho = Q (a/pi)^3/2 exp(-a r^2) has v_H = Q erf(sqrt(a) r) / r; with the
    boundary value Q / r (a point charge Q at the centre) the FE solution
    converges to it."""
    Q, a = 2.0, 1.0
    b = W.uniform_bounds(16.0, n)
    wl = W.h2().with_(xb=b, yb=b, zb=b, degree=4, n_quad=6, enrich=[], Z=np.array([Q]),
                      R=np.array([[0.0, 0.0, 0.0]]))
    S = operators.System(wl)
    r = np.sqrt(np.sum(S.mesh.xq ** 2, axis=2))
    rho = Q * (a / math.pi) ** 1.5 * np.exp(-a * r * r)
    phi, vq = poisson.solve(S, rho)
    exact = Q * erf(math.sqrt(a) * r) / r
    err = np.max(np.abs(vq - exact))
    assert err < (0.05 if n == 4 else 0.01)
    # boundary values are the prescribed point-charge potential
    assert np.allclose(phi[S.mesh.boundary], Q / np.linalg.norm(S.mesh.nodes[S.mesh.boundary], axis=1))
