"""Hartree potential from the finite-element Poisson problem (Eqs.
Hartree_possion, DiscretePoisson).

Test infrastructure only (see `oracle/__init__.py`).

-(1/4 pi) lap v_H = rho in the box, v_H = f on the boundary with
f(r) = sum_I Z_I / |r - R_I|.  Discretised on the classical basis:
A phi = d with A_mn = (1/4 pi) int grad N_m . grad N_n (reading: the gradient
on N_n is missing from the printed Eq. DiscretePoisson and is restored) and
d_m = int rho N_m, the density integral taken with the Gauss-Legendre rule at
the quadrature points where rho is known.  Boundary nodes hold f; the interior
system A_II phi_I = d_I - A_IB phi_B is solved exactly (sparse LU).  v_H at the
quadrature points is the FE interpolant of phi.  The electrostatic enrichment
of Eq. PhiEFE is not used.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla


def boundary_values(system) -> np.ndarray:
    wl = system.wl
    m = system.mesh
    X = m.nodes[m.boundary]
    f = np.zeros(len(X))
    for Z, R in zip(wl.Z, wl.R):
        f += Z / np.linalg.norm(X - R[None, :], axis=1)
    return f


def rhs(system, rho_q: np.ndarray) -> np.ndarray:
    """d_i = int rho N_i for every classical node."""
    m = system.mesh
    d = np.zeros(system.n_h)
    for c in range(m.n_cells):
        np.add.at(d, m.conn[c], m.B.T @ (m.wJ[c] * rho_q[c]))
    return d


def solve(system, rho_q: np.ndarray):
    """Nodal phi (n_h,) and v_H at the quadrature points (n_cells, nq)."""
    m = system.mesh
    A = (2.0 * system.Kcc / (4.0 * np.pi)).tocsr()   # Kcc carries the kinetic 1/2
    d = rhs(system, rho_q)
    I = np.where(m.interior)[0]
    Bn = np.where(m.boundary)[0]
    phi = np.zeros(system.n_h)
    phi[Bn] = boundary_values(system)
    AII = A[I][:, I].tocsc()
    AIB = A[I][:, Bn]
    phi[I] = spla.spsolve(AII, d[I] - AIB @ phi[Bn])
    vq = np.einsum("qn,cn->cq", m.B, phi[m.conn])
    return phi, vq
