"""Rectilinear hexahedral mesh with spectral (GLL) nodes and Gauss-Legendre
quadrature points (Secs. "Enriched finite element discretization",
"Spectral finite elements").

Test infrastructure only (see `oracle/__init__.py`).

Numbering: cells c = cx + ncx (cy + ncy cz); local nodes l = i1 + (p+1)(i2 +
(p+1) i3); global nodes g = ix + Nx (iy + Ny iz) with ix = cx p + i1; local
quadrature points q = q1 + nq (q2 + nq q3).  Boundary nodes carry the
homogeneous Dirichlet condition of the orbitals (Sec. "Rate of convergence").
"""
from __future__ import annotations

import numpy as np

from .basis import gauss_legendre, gauss_lobatto, lagrange


class Mesh:
    def __init__(self, xb, yb, zb, p: int, n_quad: int):
        self.b = [np.asarray(xb, np.float64), np.asarray(yb, np.float64), np.asarray(zb, np.float64)]
        self.p = int(p)
        self.nq1 = int(n_quad)
        self.nc = [len(b) - 1 for b in self.b]
        self.N = [n * self.p + 1 for n in self.nc]
        self.n_cells = int(np.prod(self.nc))
        self.n_nodes = int(np.prod(self.N))
        self.nn = (self.p + 1) ** 3
        self.nq = self.nq1 ** 3
        self.xi, self.wl = gauss_lobatto(self.p)          # GLL nodes / weights
        self.xg, self.wg = gauss_legendre(self.nq1)       # GL points / weights
        # 1D node coordinates
        self.coord1d = []
        for a in range(3):
            b = self.b[a]
            c = np.empty(self.N[a])
            for k in range(self.nc[a]):
                h = b[k + 1] - b[k]
                c[k * self.p:(k + 1) * self.p + 1] = b[k] + 0.5 * (self.xi + 1.0) * h
            self.coord1d.append(c)
        # cell index arrays
        cz, cy, cx = np.meshgrid(np.arange(self.nc[2]), np.arange(self.nc[1]), np.arange(self.nc[0]), indexing="ij")
        self.cell_ijk = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1)  # (n_cells, 3), cx fastest
        i3, i2, i1 = np.meshgrid(np.arange(self.p + 1), np.arange(self.p + 1), np.arange(self.p + 1), indexing="ij")
        loc = np.stack([i1.ravel(), i2.ravel(), i3.ravel()], axis=1)          # (nn, 3), i1 fastest
        gi = self.cell_ijk[:, None, :] * self.p + loc[None, :, :]
        self.conn = gi[:, :, 0] + self.N[0] * (gi[:, :, 1] + self.N[1] * gi[:, :, 2])  # (n_cells, nn)
        self.h = np.stack([self.b[a][self.cell_ijk[:, a] + 1] - self.b[a][self.cell_ijk[:, a]] for a in range(3)], axis=1)
        self.x0 = np.stack([self.b[a][self.cell_ijk[:, a]] for a in range(3)], axis=1)
        self.detJ = np.prod(self.h, axis=1) / 8.0
        # node coordinates (n_nodes, 3)
        Z3, Y3, X3 = np.meshgrid(self.coord1d[2], self.coord1d[1], self.coord1d[0], indexing="ij")
        self.nodes = np.stack([X3.ravel(), Y3.ravel(), Z3.ravel()], axis=1)
        # boundary mask
        gz, gy, gx = np.meshgrid(np.arange(self.N[2]), np.arange(self.N[1]), np.arange(self.N[0]), indexing="ij")
        bnd = ((gx == 0) | (gx == self.N[0] - 1) | (gy == 0) | (gy == self.N[1] - 1) |
               (gz == 0) | (gz == self.N[2] - 1))
        self.boundary = bnd.ravel()
        self.interior = ~self.boundary
        # reference tables at GL points
        L1, dL1 = lagrange(self.xi, self.xg)
        self.L1, self.dL1 = L1, dL1                 # (nq1, p+1)
        q3, q2, q1 = np.meshgrid(np.arange(self.nq1), np.arange(self.nq1), np.arange(self.nq1), indexing="ij")
        self.qidx = np.stack([q1.ravel(), q2.ravel(), q3.ravel()], axis=1)  # (nq, 3)
        # B[q, l] = l_i1(xg_q1) l_i2(xg_q2) l_i3(xg_q3); D_a = derivative along axis a (reference coords)
        Q, Lc = self.qidx, loc
        self.B = L1[Q[:, 0][:, None], Lc[:, 0][None, :]] * L1[Q[:, 1][:, None], Lc[:, 1][None, :]] * \
            L1[Q[:, 2][:, None], Lc[:, 2][None, :]]
        self.Dref = []
        for a in range(3):
            f = [L1, L1, L1]
            f[a] = dL1
            self.Dref.append(f[0][Q[:, 0][:, None], Lc[:, 0][None, :]] * f[1][Q[:, 1][:, None], Lc[:, 1][None, :]] *
                             f[2][Q[:, 2][:, None], Lc[:, 2][None, :]])
        self.wq_ref = self.wg[Q[:, 0]] * self.wg[Q[:, 1]] * self.wg[Q[:, 2]]
        self.wl_ref = (self.wl[loc[:, 0]] * self.wl[loc[:, 1]] * self.wl[loc[:, 2]])
        # quadrature points and weights per cell
        self.xq = self.x0[:, None, :] + 0.5 * (self.xg[self.qidx][None, :, :] + 1.0) * self.h[:, None, :]
        self.wJ = self.wq_ref[None, :] * self.detJ[:, None]          # (n_cells, nq)

    def lumped_mass(self) -> np.ndarray:
        """Diagonal M^cc from GLL collocation: M_ii = sum over cells holding
        node i of the GLL weight product times |J| (Sec. "Spectral finite
        elements")."""
        M = np.zeros(self.n_nodes)
        np.add.at(M, self.conn.ravel(), (self.wl_ref[None, :] * self.detJ[:, None]).ravel())
        return M

    def grad_tables(self, c: int):
        """Physical gradients of the cell's basis at its quadrature points:
        list of three (nq, nn) arrays."""
        return [self.Dref[a] * (2.0 / self.h[c, a]) for a in range(3)]
