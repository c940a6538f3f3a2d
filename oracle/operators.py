"""Discrete EFE operators: overlap, orthogonalisation, Hamiltonian, Loewdin
transform (Secs. "Enriched finite element discretization", "Spectral finite
elements").

Test infrastructure only (see `oracle/__init__.py`).

What this module computes, in the paper's notation:

* Eq. PsiEFE / EFESplit / EFEOrtho: psi = sum_i N^C_i psi^C_i + sum_nu N^E_nu
  psi^E_nu with N^E_nu = N^A_nu - sum_l c_{nu l} N^C_l.  With the
  coefficients a^C = psi^C - C^T psi^E of the "extended" basis [N^C, N^A],
  the EFE coefficient vector maps to the extended one through
  P = [[I, -C^T], [0, I]].
* Orthogonality int N^E_nu N^C_i = 0 fixes c_{nu i} = b_{nu i} / M^cc_ii with
  b_{nu i} = int N^A_nu N^C_i.  Reading: the classical-classical overlap
  uses the GLL rule (diagonal M^cc, Sec. "Spectral finite elements") and
  every integral with an atomic factor uses the Gauss-Legendre rule, so M is
  exactly block diagonal (Eq. M) and
  M^ee = <N^A, N^A> - b diag(M^cc)^-1 b^T.
* Eq. Hmn: H_mn = 1/2 int grad N_m . grad N_n + int v N_m N_n, assembled in
  the extended basis (H_ext) and carried to the EFE basis by P^T H_ext P.
* Eq. TDKSDiscrete2 / MSquareRoot: Hbar = M^-1/2 H M^-1/2, with
  (M^ee)^{+-1/2} from a symmetric eigendecomposition.

All classical nodes are kept; boundary nodes are removed from the operator by
a zero in the diagonal scaling (the orbitals vanish on the boundary).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import enrich as _enr
from .mesh import Mesh


class EnrichmentError(RuntimeError):
    pass


class System:
    """Everything in the method that does not depend on the potential."""

    def __init__(self, wl):
        self.wl = wl
        self.mesh = m = Mesh(wl.xb, wl.yb, wl.zb, wl.degree, wl.n_quad)
        self.n_h = m.n_nodes
        self.n_E = len(wl.enrich)
        self.n_dof = self.n_h + self.n_E
        self.M = m.lumped_mass()
        self.mask = m.interior.astype(np.float64)
        # enrichment values / gradients at every quadrature point of every cell
        nc, nq, nE = m.n_cells, m.nq, self.n_E
        pts = m.xq.reshape(-1, 3)
        self.Aq = np.zeros((nc, nq, nE))
        self.dAq = np.zeros((nc, nq, nE, 3))
        for nu, fn in enumerate(wl.enrich):
            v, g = _enr.evaluate(fn, np.asarray(wl.R[fn.atom], np.float64), pts, wl.r0, wl.s)
            self.Aq[:, :, nu] = v.reshape(nc, nq)
            self.dAq[:, :, nu, :] = g.reshape(nc, nq, 3)
        # b_{nu i} = int N^A_nu N^C_i  (Gauss-Legendre)
        b = np.zeros((nE, self.n_h))
        for c in range(nc):
            contrib = (m.B.T @ (m.wJ[c][:, None] * self.Aq[c]))      # (nn, nE)
            np.add.at(b.T, m.conn[c], contrib)
        b[:, m.boundary] = 0.0      # only interior classical functions exist
        self.b = b
        Minv = np.where(m.interior, 1.0 / self.M, 0.0)
        self.C = b * Minv[None, :]                                     # c_{nu i}
        MAA = np.einsum("cq,cqm,cqn->mn", m.wJ, self.Aq, self.Aq)
        self.Mee = MAA - (b * Minv[None, :]) @ b.T
        self.Mee = 0.5 * (self.Mee + self.Mee.T)
        if nE:
            lam, U = np.linalg.eigh(self.Mee)
            if lam.min() <= 0.0:
                raise EnrichmentError("M^ee is not positive definite (min eigenvalue %g)" % lam.min())
            self.Mee_half = (U * np.sqrt(lam)) @ U.T
            self.Mee_mhalf = (U / np.sqrt(lam)) @ U.T
        else:
            self.Mee_half = np.zeros((0, 0))
            self.Mee_mhalf = np.zeros((0, 0))
        # kinetic pieces (v-independent)
        self.Kcc = self._assemble_cc(lambda c, G: 0.5 * sum(G[a].T @ (m.wJ[c][:, None] * G[a]) for a in range(3)))
        KcA = np.zeros((self.n_h, nE))
        for c in range(nc):
            G = m.grad_tables(c)
            loc = 0.5 * sum(G[a].T @ (m.wJ[c][:, None] * self.dAq[c, :, :, a]) for a in range(3))
            np.add.at(KcA, m.conn[c], loc)
        self.KcA = KcA
        self.KAA = 0.5 * np.einsum("cq,cqma,cqna->mn", m.wJ, self.dAq, self.dAq)
        # P = [[I, -C^T], [0, I]]
        self.P = sp.bmat([[sp.identity(self.n_h, format="csr"), sp.csr_matrix(-self.C.T)],
                          [None, sp.identity(nE, format="csr")]], format="csr")
        # Loewdin scaling D = blockdiag(mask / sqrt(M^cc), (M^ee)^-1/2)
        self.Dc = np.where(m.interior, 1.0 / np.sqrt(self.M), 0.0)
        self.D = sp.block_diag([sp.diags(self.Dc), sp.csr_matrix(self.Mee_mhalf)], format="csr")
        self.Dhalf = sp.block_diag([sp.diags(np.where(m.interior, np.sqrt(self.M), 0.0)),
                                    sp.csr_matrix(self.Mee_half)], format="csr")

    # ------------------------------------------------------------------
    def _assemble_cc(self, element):
        m = self.mesh
        rows, cols, vals = [], [], []
        for c in range(m.n_cells):
            G = m.grad_tables(c)
            Ke = element(c, G)
            rows.append(np.repeat(m.conn[c], m.nn))
            cols.append(np.tile(m.conn[c], m.nn))
            vals.append(Ke.ravel())
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.n_h, self.n_h))

    def potential_blocks(self, vq: np.ndarray):
        """V^cc (sparse), V^cA, V^AA for v given at the quadrature points
        (n_cells, nq): int v N_m N_n by Gauss-Legendre quadrature."""
        m = self.mesh
        Vcc = self._assemble_cc(lambda c, G: m.B.T @ ((m.wJ[c] * vq[c])[:, None] * m.B))
        VcA = np.zeros((self.n_h, self.n_E))
        for c in range(m.n_cells):
            np.add.at(VcA, m.conn[c], m.B.T @ ((m.wJ[c] * vq[c])[:, None] * self.Aq[c]))
        VAA = np.einsum("cq,cqm,cqn->mn", m.wJ * vq, self.Aq, self.Aq)
        return Vcc, VcA, VAA

    def hamiltonian_efe(self, vq: np.ndarray, kin: float = 1.0) -> sp.csr_matrix:
        """H in the EFE basis (Eq. Hmn), P^T H_ext P, before the Loewdin scaling."""
        Vcc, VcA, VAA = self.potential_blocks(vq)
        Hcc = kin * self.Kcc + Vcc
        HcA = kin * self.KcA + VcA
        HAA = kin * self.KAA + VAA
        Hext = sp.bmat([[Hcc, sp.csr_matrix(HcA)], [sp.csr_matrix(HcA.T), sp.csr_matrix(HAA)]], format="csr")
        return (self.P.T @ Hext @ self.P).tocsr()

    def hbar(self, vq: np.ndarray, kin: float = 1.0) -> sp.csr_matrix:
        """Hbar = M^-1/2 H M^-1/2 (Eq. TDKSDiscrete2) on the full DOF layout
        [all classical nodes; enrichment]; boundary rows and columns are zero."""
        return (self.D @ self.hamiltonian_efe(vq, kin) @ self.D).tocsr()

    def overlap_efe(self) -> sp.csr_matrix:
        """The full EFE overlap P^T M_ext P in the mixed inner product: GLL for
        classical-classical, Gauss-Legendre for anything with an atomic factor.
        Its classical-enriched block is zero by construction (Eq. M)."""
        m = self.mesh
        MAA = np.einsum("cq,cqm,cqn->mn", m.wJ, self.Aq, self.Aq)
        Mext = sp.bmat([[sp.diags(self.M * self.mask), sp.csr_matrix(self.b.T)],
                        [sp.csr_matrix(self.b), sp.csr_matrix(MAA)]], format="csr")
        return (self.P.T @ Mext @ self.P).tocsr()

    # ------------------------------------------------------------------
    def to_efe(self, psi_bar: np.ndarray) -> np.ndarray:
        """psi = M^-1/2 psi_bar (EFE coefficients), boundary rows zero."""
        return self.D @ psi_bar

    def from_efe(self, psi: np.ndarray) -> np.ndarray:
        """psi_bar = M^1/2 psi."""
        return self.Dhalf @ psi

    def values_at_quad(self, psi_bar: np.ndarray) -> np.ndarray:
        """psi(x_q) for every cell and quadrature point: (n_cells, nq, ncols).
        psi(x) = sum_i N^C_i a^C_i + sum_nu N^A_nu psi^E_nu with a^C = psi^C - C^T psi^E."""
        m = self.mesh
        psi = self.to_efe(psi_bar)
        pc, pe = psi[:self.n_h], psi[self.n_h:]
        aC = pc - self.C.T @ pe
        out = np.einsum("qn,cnk->cqk", m.B, aC[m.conn]) + np.einsum("cqe,ek->cqk", self.Aq, pe)
        return out

    def node_coords(self) -> np.ndarray:
        return self.mesh.nodes

    def initial_orbitals(self) -> np.ndarray:
        """psi_bar at t = 0 from the workload's Gaussian descriptors: the
        classical coefficients are the Gaussians' nodal values (zero on the
        boundary), the enrichment coefficients are given; psi_bar = M^1/2 psi."""
        wl = self.wl
        X = self.mesh.nodes
        nb = wl.n_orb
        psi = np.zeros((self.n_dof, nb), dtype=np.complex128)
        for a in range(nb):
            d2 = np.sum((X[:, None, :] - wl.orb_centers[a][None, :, :]) ** 2, axis=2)
            psi[:self.n_h, a] = np.exp(-d2 * wl.orb_exps[a][None, :]) @ wl.orb_coefs[a]
            psi[self.n_h:, a] = wl.enr_coefs[a]
        psi[:self.n_h][self.mesh.boundary] = 0.0
        return self.from_efe(psi)
