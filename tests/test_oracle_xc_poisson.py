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


def _vwn5_ec(rs):
    """Vosko-Wilk-Nusair (Can. J. Phys. 58, 1200 (1980)) paramagnetic correlation energy per
    electron, their Pade interpolation of the Ceperley-Alder data ("VWN5"), in Hartree:
    x = sqrt(r_s), X(x) = x^2 + b x + c, Q = sqrt(4c - b^2),
    eps_c = A [ln(x^2/X) + (2b/Q) atan(Q/(2x+b))
               - (b x0 / X(x0)) (ln((x-x0)^2/X) + (2(b + 2 x0)/Q) atan(Q/(2x+b)))]
    with A = 0.0310907, x0 = -0.10498, b = 3.72744, c = 12.9352."""
    A, x0, b, c = 0.0310907, -0.10498, 3.72744, 12.9352
    x = np.sqrt(rs)
    X = x * x + b * x + c
    X0 = x0 * x0 + b * x0 + c
    Q = math.sqrt(4.0 * c - b * b)
    t = np.arctan(Q / (2.0 * x + b))
    return A * (np.log(x * x / X) + 2.0 * b / Q * t - b * x0 / X0 * (np.log((x - x0) ** 2 / X) + 2.0 * (b + 2.0 * x0) / Q * t))


def _pw92_vs_vwn5(beta=None, alpha1=None):
    rs = np.linspace(2.0, 20.0, 181)
    old_b, old_a = xc.PW92_BETA, xc.PW92_ALPHA1
    try:
        if beta is not None:
            xc.PW92_BETA = beta
        if alpha1 is not None:
            xc.PW92_ALPHA1 = alpha1
        ec = xc.pw92_eps_c(rs)[0]
    finally:
        xc.PW92_BETA, xc.PW92_ALPHA1 = old_b, old_a
    return float(np.max(np.abs(ec - _vwn5_ec(rs))))


def test_pw92_matches_an_independent_fit_of_the_same_data():
    """PW92 and VWN5 are two closed forms with their own constants fitted to the same
    Ceperley-Alder correlation energies; on the metallic range r_s in [2, 20] they agree to
    1e-4 Ha.  That holds the constants the high-density limit leaves free (alpha1, beta3,
    beta4) at that level: a transposed digit of alpha1 or beta3 moves eps_c by 2e-4 .. 1e-3
    Ha there and fails (checked below); changes of beta4 below ~0.2% are not resolved."""
    assert _pw92_vs_vwn5() < 1e-4


def test_pw92_pin_catches_transposed_constants():
    b = list(xc.PW92_BETA)
    b3 = b.copy()
    b3[2] = 1.6832                     # 1.6382 with two digits swapped
    assert _pw92_vs_vwn5(beta=tuple(b3)) > 1e-4
    b4 = b.copy()
    b4[3] = 0.94294                    # 0.49294 with two digits swapped
    assert _pw92_vs_vwn5(beta=tuple(b4)) > 1e-4
    assert _pw92_vs_vwn5(alpha1=0.21730) > 1e-4
    assert _pw92_vs_vwn5(alpha1=0.23170) > 1e-4
