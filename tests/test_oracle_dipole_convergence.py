"""Pins of the oracle's dipole (Sec. Results: dipole moment, Eq. DipoleSemi) and of
the kick and propagation that produce it, against a closed form, with its mesh
convergence rate.

Closed form: in a harmonic trap v = (1/2) w^2 r^2 the centre of mass of the
electrons obeys Ehrenfest's equation d^2<x>/dt^2 = -w^2 <x> whatever the initial
state, as long as the other potentials exert no net force on it.  The Hartree
solve is replaced by zero; the LDA exchange-correlation potential exerts none in
the continuum (rho grad v_xc is the gradient of a function of rho).  A delta kick
exp(i kappa x) gives every orbital momentum kappa, so with N electrons
mu_x(t) = mu_x(0) - N (kappa / w) sin(w t)
(mu = sum Z R - int x rho; no nuclei here).  The finite element error of that
dipole must vanish with the mesh size at least at the rate p the paper reports
for the dipole (Sec. Results, convergence study), here for degrees 2 and 3."""
import numpy as np

import efe_workloads as W
from oracle import operators, tdks

OMEGA, KAPPA, L = 1.0, 1e-3, 12.0


def _trap_dipole_error(n_cells, p, n_steps=6, dt=0.05, sign=1.0):
    wl = W.h2(n_cells=n_cells, degree=p, n_quad=p + 2, L=L, kick=KAPPA)
    # one doubly occupied orbital, the trap's ground-state Gaussian; no enrichment
    wl = wl.with_(enrich=[], enr_coefs=np.zeros((1, 0), complex), orb_centers=np.zeros((1, 1, 3)),
                  orb_exps=np.array([[OMEGA / 2.0]]), orb_coefs=np.ones((1, 1), complex))
    S = operators.System(wl)
    vN = 0.5 * OMEGA ** 2 * np.sum(S.mesh.xq ** 2, axis=2)

    def no_hartree(system, rho):
        return np.zeros(system.n_h), np.zeros_like(rho)

    psi = S.initial_orbitals()
    psi = psi / np.linalg.norm(psi, axis=0)
    mu0 = tdks.dipole(S, tdks.make_state(S, psi, wl.occ, 1, hartree=no_hartree).rho[0])
    psi = tdks.kick(S, psi, wl.fields, wl.n_orb, tol=1e-14, k_max=40)
    st = tdks.make_state(S, psi, wl.occ, 1, hartree=no_hartree)
    n_el = float(np.sum(wl.occ))
    err = 0.0
    for n in range(n_steps):
        psi, st, mu, _ = tdks.magnus_step(S, psi, st, n * dt, dt, wl.fields, wl.occ, 1e-13, 40, vN=vN,
                                          hartree=no_hartree)
        t = (n + 1) * dt
        exact = mu0[0] - sign * n_el * KAPPA / OMEGA * np.sin(OMEGA * t)
        err = max(err, abs(mu[0, 0] - exact))
    return err


def _rate(p, cells):
    errs = np.array([_trap_dipole_error(n, p) for n in cells])
    h = L / np.asarray(cells, float)
    return np.polyfit(np.log(h), np.log(errs), 1)[0], errs


def test_dipole_mesh_convergence_against_closed_form_p2():
    slope, errs = _rate(2, [4, 6, 8])
    assert slope >= 2.0 - 0.3, (slope, errs)
    assert errs[-1] < 3e-5, errs          # 1.3e-5 of an oscillation amplitude of 2e-3


def test_dipole_mesh_convergence_against_closed_form_p3():
    slope, errs = _rate(3, [4, 6, 8])
    assert slope >= 3.0 - 0.3, (slope, errs)
    assert errs[-1] < 3e-6, errs          # 1.0e-6


def test_closed_form_detects_a_sign_error():
    """The same comparison with the opposite sign of the response (a sign slip in the kick or the
    dipole) stays at the size of the signal on the finest mesh."""
    assert _trap_dipole_error(8, 3, sign=-1.0) > 1e-4
