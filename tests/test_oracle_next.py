"""Pins of the oracle's optional pieces: the Perdew-Zunger parametrisation
of Ceperley-Alder correlation (the paper's functional) and the
potential-extrapolation variant of the Magnus step."""
import numpy as np
import pytest

import efe_workloads as W
from oracle import operators, tdks, xc


def test_pz81_potential_is_derivative_of_energy():
    """v_c = d(rho eps_c)/d rho, checked by central differences on both branches."""
    rho = np.concatenate([np.logspace(-5, -1.2, 20), np.logspace(-0.9, 2, 20)])   # r_s > 1 and r_s < 1
    h = 1e-6 * rho
    ep, _ = xc.pz81_correlation(rho + h)
    em, _ = xc.pz81_correlation(rho - h)
    fd = ((rho + h) * ep - (rho - h) * em) / (2 * h)
    assert np.allclose(xc.pz81_correlation(rho)[1], fd, rtol=1e-7, atol=0)


def test_pz81_branches_meet_at_rs_one():
    lo = xc.pz81_eps_c(np.array([1.0]))
    g, b1, b2 = xc.PZ81_LOW
    A, B, C, D = xc.PZ81_HIGH
    e_hi, e_lo = B + D, g / (1.0 + b1 + b2)
    v_lo = e_lo * (1.0 + 7.0 / 6.0 * b1 + 4.0 / 3.0 * b2) / (1.0 + b1 + b2)
    v_hi = (B - A / 3.0) + (2.0 * D - C) / 3.0
    assert abs(e_hi - e_lo) < 1e-4 and abs(v_hi - v_lo) < 1e-4
    assert abs(lo[0][0] - e_lo) < 1e-15


def test_pz81_high_density_coefficient_and_agreement_with_pw92():
    """The ln r_s coefficient is the exact high-density one, (1 - ln 2) / pi^2,
    and the two independent fits of the Ceperley-Alder data agree within
    1.5 mHa for 0.01 <= r_s <= 100."""
    A = xc.PZ81_HIGH[0]
    assert abs(A - (1.0 - np.log(2.0)) / np.pi ** 2) < 1e-3 * A
    rs = np.logspace(-2, 2, 200)
    assert np.max(np.abs(xc.pz81_eps_c(rs)[0] - xc.pw92_eps_c(rs)[0])) < 1.5e-3
    rho = 3.0 / (4.0 * np.pi * rs ** 3)
    e1, v1 = xc.lda(rho, "pz81")
    e2, v2 = xc.lda(rho, "pw92")
    assert np.max(np.abs(e1 - e2)) < 1.5e-3 and np.max(np.abs(v1 - v2)) < 3e-3


@pytest.fixture(scope="module")
def tiny():
    wl = W.small_cluster(n_atoms=1, cells_per_axis=3, degree=2, n_quad=4, L=10.0, n_orb=1, Zval=2.0)
    S = operators.System(wl)
    psi0 = S.initial_orbitals()
    psi0 /= np.linalg.norm(psi0, axis=0)
    f = W.Field(kind=W.FIELD_GAUSS, amp=0.2, t0=0.2, sigma=0.1, direction=(1.0, 0.0, 0.0))
    return S, psi0, f


def _run(S, psi0, f, dt, T, scheme, xc_kind="pw92"):
    occ = np.array([2.0])
    st = tdks.make_state(S, psi0, occ, 1, xc_kind)
    psi = psi0.copy()
    vN = tdks.nuclear_potential(S)
    n = int(round(T / dt))
    for k in range(n):
        psi, st, mu, _ = tdks.magnus_step(S, psi, st, k * dt, dt, [f], occ, 1e-13, 40, vN=vN, scheme=scheme,
                                          xc_kind=xc_kind)
    return mu[0]


@pytest.mark.parametrize("scheme", ["pc", "extrapolated"])
def test_schemes_are_second_order(tiny, scheme):
    """Dipole error at T = 0.4 against a dt = 0.00625 run: halving dt divides
    it by ~4 for both schemes (a wrong extrapolation weight makes it first
    order, ratio ~2)."""
    S, psi0, f = tiny
    ref = _run(S, psi0, f, 0.00625, 0.4, "pc")
    e1 = np.linalg.norm(_run(S, psi0, f, 0.05, 0.4, scheme) - ref)
    e2 = np.linalg.norm(_run(S, psi0, f, 0.025, 0.4, scheme) - ref)
    assert e2 > 1e-10
    assert 3.0 < e1 / e2 < 5.5, (e1, e2)


def test_pz81_step_differs_from_pw92_by_the_functional_only(tiny):
    """The functional option reaches the step: PZ81 and PW92 trajectories
    differ, by an amount of the order of the functionals' difference."""
    S, psi0, f = tiny
    a = _run(S, psi0, f, 0.05, 0.2, "pc", "pw92")
    b = _run(S, psi0, f, 0.05, 0.2, "pc", "pz81")
    d = np.linalg.norm(a - b)
    assert 1e-9 < d < 1e-2
