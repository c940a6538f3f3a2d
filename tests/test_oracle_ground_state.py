"""The oracle's self-consistent ground state (`tdks.ground_state`) against a published value.

The helium atom in the local-density approximation: Z = 2 at a vertex of a graded 6^3-cell mesh
of degree 3 on a 12-bohr cube, one doubly occupied orbital, one 1s Slater enrichment function
(zeta = 27/16).  The 1s eigenvalue of the converged Kohn-Sham state is held to the tabulated
all-electron value (`tests/golden/he_lda_1s.txt`) within 2e-3 hartree: the mesh's
discretisation error (1.25e-3 measured here, 2.8e-4 on 8^3 cells) plus the difference between
the PW92 correlation the oracle uses and the VWN correlation of the table (1.7e-4 on this mesh).
The eigenvalue depends on every part of the self-consistent potential (Eq. VN, the Hartree
solve of Eq. Hartree_possion, the LDA of the exchange-correlation term, the density with its
occupation): dropping the correlation moves it by +5.2e-2, a wrong factor in the Hartree or the
exchange term by more."""
import os

import numpy as np
import pytest

import efe_workloads as W
from oracle import operators, tdks

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "he_lda_1s.txt")


def _golden():
    vals = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                vals[line[0]] = float(line[1])
    return vals


def _helium():
    b = W.graded_bounds(12.0, [0.0], 0.3, 3.0, 6)
    assert np.any(np.abs(b) < 1e-12)          # the nucleus sits on cell faces, not inside a cell
    return W.h2().with_(xb=b, yb=b.copy(), zb=b.copy(), degree=3, n_quad=8,
                        enrich=[W.EnrichFn(0, 1, 0, 0, W.RADIAL_SLATER, 27.0 / 16.0)],
                        Z=np.array([2.0]), R=np.array([[0.0, 0.0, 0.0]]), r0=4.0, s=2.0,
                        orb_centers=np.zeros((1, 1, 3)), orb_exps=np.array([[1.5]]),
                        orb_coefs=np.ones((1, 1), dtype=np.complex128),
                        enr_coefs=np.ones((1, 1), dtype=np.complex128))


@pytest.mark.slow
def test_helium_lda_eigenvalue_matches_tabulated_value():
    S = operators.System(_helium())
    psi, eps = tdks.ground_state(S, 1, np.array([2.0]), mix=0.6, tol=1e-7)
    assert abs(eps[0] - _golden()["eps_1s"]) <= 2e-3
    # the state is normalised in the Loewdin-scaled basis and carries the two electrons
    assert abs(np.linalg.norm(psi[:, 0]) - 1.0) <= 1e-10
    rho = tdks.density(S, psi, np.array([2.0]), 1)[0]
    assert abs(np.sum(rho * S.mesh.wJ) - 2.0) <= 1e-3

    # a planted mistake in the oracle (the correlation dropped from the LDA) fails the pin
    from oracle import xc
    saved = xc.XC_KINDS["pw92"]
    try:
        xc.XC_KINDS["pw92"] = lambda r: (np.zeros_like(r), np.zeros_like(r))
        _, eps_x = tdks.ground_state(S, 1, np.array([2.0]), mix=0.6, tol=1e-7, psi_guess=psi)
    finally:
        xc.XC_KINDS["pw92"] = saved
    assert abs(eps_x[0] - _golden()["eps_1s"]) > 2e-2
