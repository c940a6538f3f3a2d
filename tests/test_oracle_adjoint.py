"""Pins of the oracle's adjoint: its pieces against definitions and finite
differences, and the whole gradient against central finite differences of the
forward run."""
import dataclasses

import numpy as np
import pytest

import efe_workloads as W
from oracle import adjoint, operators, tdks, xc


def test_fxc_is_derivative_of_vxc():
    rho = np.logspace(-6, 2, 40)
    h = 1e-6 * rho
    fd = (xc.lda(rho + h)[1] - xc.lda(rho - h)[1]) / (2 * h)
    assert np.allclose(adjoint.fxc(rho), fd, rtol=1e-7)
    assert np.all(adjoint.fxc(np.array([0.0, 1e-15])) == 0.0)


def test_field_derivatives():
    f = W.Field(kind=W.FIELD_SINE_GAUSS, amp=0.05, omega=0.8, t0=0.2, sigma=0.3, direction=(0.0, 1.0, 0.0))
    t = 0.37
    _, dE = adjoint.field_and_derivs(f, t)
    for k, name in enumerate(["amp", "omega", "sigma"]):
        h = 1e-6 * getattr(f, name)
        ep, _ = adjoint.field_and_derivs(dataclasses.replace(f, **{name: getattr(f, name) + h}), t)
        em, _ = adjoint.field_and_derivs(dataclasses.replace(f, **{name: getattr(f, name) - h}), t)
        assert np.allclose(dE[k], (ep - em) / (2 * h), rtol=1e-7, atol=1e-14)


@pytest.fixture(scope="module")
def tiny_adjoint():
    wl = W.small_cluster(n_atoms=1, cells_per_axis=3, degree=2, n_quad=4, L=10.0, n_orb=1, Zval=2.0)
    S = operators.System(wl)
    return S, adjoint.Adjoint(S)


def test_phi_reproduces_hbar(tiny_adjoint):
    S, A = tiny_adjoint
    vq = tdks.nuclear_potential(S) + 0.1 * S.mesh.xq[:, :, 2]
    assert np.max(np.abs(A.hbar(vq.reshape(-1)) - S.hbar(vq).toarray())) < 1e-12


def test_adjoint_gradient_matches_finite_differences(tiny_adjoint):
    """dJ/d(amp, omega, sigma) of the window-averaged dipole through the
    predictor-corrector steps, against central differences (h = 1e-4 |theta|)."""
    S, A = tiny_adjoint
    f = W.Field(kind=W.FIELD_SINE_GAUSS, amp=0.05, omega=0.8, t0=0.2, sigma=0.3, direction=(1.0, 0.0, 0.0))
    psi0 = S.initial_orbitals()
    psi0 /= np.linalg.norm(psi0, axis=0)
    occ = np.array([2.0])
    dt, N, window = 0.05, 6, [4, 5, 6]
    J, g = A.gradient(psi0, f, dt, N, occ, window, (1, 0, 0))
    for k, name in enumerate(["amp", "omega", "sigma"]):
        val = getattr(f, name)
        h = 1e-4 * abs(val)
        Jp, _ = A.run(psi0, dataclasses.replace(f, **{name: val + h}), dt, N, occ, window, (1, 0, 0))
        Jm, _ = A.run(psi0, dataclasses.replace(f, **{name: val - h}), dt, N, occ, window, (1, 0, 0))
        fd = (Jp - Jm) / (2 * h)
        assert abs(g[k] - fd) <= 1e-6 * abs(fd), (name, g[k], fd)
