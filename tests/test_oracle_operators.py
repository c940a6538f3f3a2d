"""Pins of the oracle's EFE operators: block-diagonal overlap (Eq. M), the
Loewdin-transformed Hamiltonian (Eqs. Hmn, TDKSDiscrete2) against textbook
spectra, and the enrichment coupling (Eqs. EFESplit, EFEOrtho)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import efe_workloads as W
from oracle import operators, tdks


def _lowest(S, vq, k=4):
    H = S.hbar(vq)
    keep = np.concatenate([S.mesh.interior, np.ones(S.n_E, bool)])
    idx = np.where(keep)[0]
    return np.sort(spla.eigsh(H[idx][:, idx], k=k, which="SA")[0])


def _ho(n, p, nq, enrich=True):
    b = W.uniform_bounds(16.0, n)
    enr = [W.EnrichFn(0, 1, 0, 0, W.RADIAL_GAUSSIAN, 0.5)] if enrich else []
    wl = W.h2().with_(xb=b, yb=b, zb=b, degree=p, n_quad=nq, enrich=enr, Z=np.array([1.0]),
                      R=np.array([[0.0, 0.0, 0.0]]), r0=7.0, s=2.5)
    return operators.System(wl)


def test_overlap_block_diagonal(h2_system):
    S = h2_system
    Mo = S.overlap_efe().toarray()
    assert np.max(np.abs(Mo[:S.n_h, S.n_h:])) < 1e-14 * np.max(np.abs(Mo))
    lam = np.linalg.eigvalsh(S.Mee)
    assert lam.min() > 0


def test_mee_is_schur_complement():
    """The orthogonalised block equals the Schur complement of the extended
    Gram matrix [[M^cc, b^T], [b, <A,A>]] (computed here with dense solves)."""
    S = operators.System(W.small_cluster(n_atoms=2, cells_per_axis=3, degree=3, n_quad=5))
    I = S.mesh.interior
    m = S.mesh
    MAA = np.einsum("cq,cqm,cqn->mn", m.wJ, S.Aq, S.Aq)
    Mcc = np.diag(S.M[I])
    bI = S.b[:, I]
    schur = MAA - bI @ np.linalg.solve(Mcc, bI.T)
    assert np.allclose(S.Mee, schur, rtol=1e-12, atol=1e-15)
    assert np.allclose(S.Mee_mhalf @ S.Mee @ S.Mee_mhalf, np.eye(S.n_E), atol=1e-10)


def test_hbar_symmetric(h2_system):
    S = h2_system
    H = S.hbar(tdks.nuclear_potential(S) + 0.1 * S.mesh.xq[:, :, 1])
    assert abs(H - H.T).max() < 1e-13 * abs(H).max()
    bnd = np.concatenate([S.mesh.boundary, np.zeros(S.n_E, bool)])
    assert abs(H[np.where(bnd)[0]]).max() == 0.0


def test_harmonic_oscillator_spectrum_converges():
    """v = r^2 / 2: the lowest eigenvalues of Hbar approach 3/2, 5/2 (x3)
    as h -> 0 with degree 4 (classical basis only)."""
    e4 = _lowest(_ho(4, 4, 6, enrich=False), None or 0.5 * np.sum(_ho(4, 4, 6, False).mesh.xq ** 2, axis=2))
    S8 = _ho(8, 4, 6, enrich=False)
    e8 = _lowest(S8, 0.5 * np.sum(S8.mesh.xq ** 2, axis=2))
    exact = np.array([1.5, 2.5, 2.5, 2.5])
    err4, err8 = np.abs(e4 - exact), np.abs(e8 - exact)
    assert np.all(err8 < 1e-3)
    assert np.all(err8 < err4 / 16)        # at least h^4 for p = 4


def test_enrichment_captures_exact_state_on_coarse_mesh():
    """With the exact ground state exp(-r^2/2) as enrichment function, a
    coarse degree-3 mesh gives 3/2 to 1e-4 although the classical basis alone
    is off by 0.15: pins orthogonalisation, M^ee, the coupling blocks and the
    Loewdin scaling together."""
    S = _ho(4, 3, 8, enrich=True)
    e = _lowest(S, 0.5 * np.sum(S.mesh.xq ** 2, axis=2), k=1)
    assert abs(e[0] - 1.5) < 1e-4
    S0 = _ho(4, 3, 8, enrich=False)
    e0 = _lowest(S0, 0.5 * np.sum(S0.mesh.xq ** 2, axis=2), k=1)
    assert abs(e0[0] - 1.5) > 0.1


def test_hydrogen_atom_ground_state():
    """Z = 1, one electron, no Hartree or XC: the lowest eigenvalue tends to
    -1/2 hartree as mesh and quadrature refine."""
    res = []
    for n, nq in [(4, 6), (8, 10)]:
        b = W.uniform_bounds(16.0, n)
        wl = W.h2().with_(xb=b, yb=b, zb=b, degree=3, n_quad=nq, enrich=[W.EnrichFn(0, 1, 0, 0, W.RADIAL_SLATER, 1.0)],
                          Z=np.array([1.0]), R=np.array([[0.0, 0.0, 0.0]]), r0=6.0, s=2.0)
        S = operators.System(wl)
        res.append(_lowest(S, tdks.nuclear_potential(S), 1)[0])
    assert abs(res[1] + 0.5) < 2e-3
    assert abs(res[1] + 0.5) < abs(res[0] + 0.5) / 5


def test_dense_reference_of_hbar_matches_sparse():
    """Hbar from dense algebra on the extended basis (independent of the
    sparse P^T H P route) on a tiny mesh."""
    S = operators.System(W.small_cluster(n_atoms=1, cells_per_axis=2, degree=2, n_quad=4, L=8.0))
    vq = tdks.nuclear_potential(S) + 0.3
    H = S.hbar(vq).toarray()
    Vcc, VcA, VAA = S.potential_blocks(vq)
    Hext = np.block([[S.Kcc.toarray() + Vcc.toarray(), S.KcA + VcA], [(S.KcA + VcA).T, S.KAA + VAA]])
    nh, nE = S.n_h, S.n_E
    P = np.eye(nh + nE)
    P[:nh, nh:] = -S.C.T
    D = np.zeros((nh + nE, nh + nE))
    D[:nh, :nh] = np.diag(S.Dc)
    D[nh:, nh:] = sla.fractional_matrix_power(S.Mee, -0.5).real
    Href = D @ P.T @ Hext @ P @ D
    assert np.allclose(H, Href, rtol=1e-10, atol=1e-10 * np.abs(Href).max())
