"""A locally refined hexahedral mesh with hanging-node constraints (the paper's
adaptive mesh: an octree whose non-conforming faces are made conforming by
constraints on the finer side; Sec. "Enriched finite element basis", mesh
adaption).

Test infrastructure only (see `oracle/__init__.py`).

Reading O1 (the paper uses the octree of its references): one refinement
level over a uniform coarse grid — a chosen set of coarse cells is split into
2 x 2 x 2 children, so neighbouring leaves differ by at most one level — with
degree-p Lagrange functions on GLL nodes in every leaf.  Coincident nodes of
leaves are one node.  A node of a fine leaf that lies on the boundary of a
coarse leaf without being one of its nodes is hanging: its value is the coarse
leaf's interpolant there, u(x_h) = sum_j N^C_j(x_h) u_j over the coarse leaf's
nodes, which are never hanging (one level).  The constrained space is
u_all = P u_free; operators are P^T K P.

Reading O2 (the paper's Loewdin transform needs a diagonal mass; with hanging
nodes P^T M P is not diagonal): the mass of the constrained space is the
row-sum lumping of P^T M_GLL P, i.e. P^T m_all with m_all the GLL-lumped
weights of all nodes; it integrates constants exactly and reduces to the
rectilinear lumped mass without refinement.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .basis import gauss_legendre, gauss_lobatto, lagrange


class OctreeMesh:
    def __init__(self, lo, hi, nc: int, p: int, refine, n_quad: int = None):
        lo, hi = np.asarray(lo, float), np.asarray(hi, float)
        self.lo, self.hi, self.p = lo, hi, p
        self.xi, _ = gauss_lobatto(p)
        hc = (hi - lo) / nc
        refine = set(tuple(r) for r in refine)
        leaves = []     # (x0, h, coarse flag)
        for k in range(nc):
            for j in range(nc):
                for i in range(nc):
                    x0 = lo + np.array([i, j, k]) * hc
                    if (i, j, k) in refine:
                        for c in range(8):
                            b = np.array([(c >> a) & 1 for a in range(3)])
                            leaves.append((x0 + 0.5 * b * hc, 0.5 * hc, False))
                    else:
                        leaves.append((x0, hc.copy(), True))
        self.leaves = leaves
        p1 = p + 1
        i3, i2, i1 = np.meshgrid(np.arange(p1), np.arange(p1), np.arange(p1), indexing="ij")
        self.loc = np.stack([i1.ravel(), i2.ravel(), i3.ravel()], axis=1)
        # nodes of every leaf, merged by position
        scale = 1.0 / (np.min(hc) * 1e-9)
        key_of, coords, conn = {}, [], []
        for x0, h, _ in leaves:
            X = x0[None, :] + 0.5 * (self.xi[self.loc] + 1.0) * h[None, :]
            ids = []
            for x in X:
                key = tuple(np.rint(x * scale).astype(np.int64))
                if key not in key_of:
                    key_of[key] = len(coords)
                    coords.append(x)
                ids.append(key_of[key])
            conn.append(ids)
        self.nodes = np.array(coords)
        self.conn = np.array(conn)
        self.n_all = len(coords)
        # hanging nodes: on the closed box of a coarse leaf, not one of its nodes
        hang = {}
        tol = 1e-9 * np.min(hc)
        for li, (x0, h, coarse) in enumerate(leaves):
            if not coarse:
                continue
            own = set(self.conn[li])
            inside = np.all((self.nodes >= x0[None, :] - tol) & (self.nodes <= x0[None, :] + h[None, :] + tol), axis=1)
            for n in np.where(inside)[0]:
                if n in own or n in hang:
                    continue
                ref = 2.0 * (self.nodes[n] - x0) / h - 1.0
                L = [lagrange(self.xi, np.array([ref[a]]))[0][0] for a in range(3)]
                w = L[0][self.loc[:, 0]] * L[1][self.loc[:, 1]] * L[2][self.loc[:, 2]]
                keep = np.abs(w) > 1e-14
                hang[n] = (self.conn[li][keep], w[keep])
        self.hanging = hang
        free = [n for n in range(self.n_all) if n not in hang]
        self.free = np.array(free)
        col = {n: i for i, n in enumerate(free)}
        rows, cols, vals = [], [], []
        for n in range(self.n_all):
            if n in hang:
                masters, w = hang[n]
                for mm, ww in zip(masters, w):
                    rows.append(n)
                    cols.append(col[mm])
                    vals.append(ww)
            else:
                rows.append(n)
                cols.append(col[n])
                vals.append(1.0)
        self.P = sp.csr_matrix((vals, (rows, cols)), shape=(self.n_all, len(free)))
        # quadrature tables
        nq1 = n_quad or p + 2
        xg, wg = gauss_legendre(nq1)
        L1, dL1 = lagrange(self.xi, xg)
        k3, k2, k1 = np.meshgrid(np.arange(nq1), np.arange(nq1), np.arange(nq1), indexing="ij")
        Q = np.stack([k1.ravel(), k2.ravel(), k3.ravel()], axis=1)
        lc = self.loc
        tab = lambda f0, f1, f2: f0[Q[:, 0][:, None], lc[:, 0][None, :]] * f1[Q[:, 1][:, None], lc[:, 1][None, :]] \
            * f2[Q[:, 2][:, None], lc[:, 2][None, :]]
        self.B = tab(L1, L1, L1)
        self.Dref = [tab(dL1, L1, L1), tab(L1, dL1, L1), tab(L1, L1, dL1)]
        self.xq_ref = xg[Q]
        self.wq = wg[Q[:, 0]] * wg[Q[:, 1]] * wg[Q[:, 2]]
        on_bnd = np.any((np.abs(self.nodes - lo[None, :]) < tol) | (np.abs(self.nodes - hi[None, :]) < tol), axis=1)
        self.boundary_free = on_bnd[self.free]

    def stiffness_and_load(self, f):
        """K = P^T K_all P with K_all = int grad N . grad N over the leaves, and
        F = P^T int f N (Gauss-Legendre (p+2)^3 per leaf)."""
        rows, cols, vals = [], [], []
        F = np.zeros(self.n_all)
        for li, (x0, h, _) in enumerate(self.leaves):
            idx = self.conn[li]
            G = [self.Dref[a] * (2.0 / h[a]) for a in range(3)]
            w = self.wq * np.prod(h) / 8.0
            Kc = sum(G[a].T @ (w[:, None] * G[a]) for a in range(3))
            rows.append(np.repeat(idx, len(idx)))
            cols.append(np.tile(idx, len(idx)))
            vals.append(Kc.ravel())
            pts = x0[None, :] + 0.5 * (self.xq_ref + 1.0) * h[None, :]
            np.add.at(F, idx, self.B.T @ (w * f(pts)))
        K_all = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                              shape=(self.n_all, self.n_all))
        return (self.P.T @ K_all @ self.P).tocsr(), self.P.T @ F

    def lumped_mass(self):
        """Diagonal mass of the constrained space (reading O2): the row sums of
        P^T M_GLL P, M_GLL the GLL-lumped mass of all nodes (Sec. "Spectral finite
        elements": diagonal mass from GLL collocation); since every row of P sums
        to one these are P^T m_all."""
        _, w = gauss_lobatto(self.p)
        w3 = w[self.loc[:, 0]] * w[self.loc[:, 1]] * w[self.loc[:, 2]]
        m_all = np.zeros(self.n_all)
        for li, (x0, h, _) in enumerate(self.leaves):
            np.add.at(m_all, self.conn[li], w3 * np.prod(h) / 8.0)
        return self.P.T @ m_all

    def hbar(self, vq, kin: float = 1.0):
        """The Loewdin-scaled Hamiltonian on the interior free nodes,
        D H_II D with D = M^-1/2 of lumped_mass (Eq. TDKSDiscrete2 on the
        locally refined mesh)."""
        I = np.where(~self.boundary_free)[0]
        d = 1.0 / np.sqrt(self.lumped_mass()[I])
        H = self.hamiltonian(vq, kin)[I][:, I]
        return sp.diags(d) @ H @ sp.diags(d)

    def density(self, psi_bar, occ):
        """rho at every leaf's Gauss-Legendre points, (n_leaves, nq), for orbitals
        psi_bar (n_free, n_orb) complex in the Loewdin basis: psi = D psi_bar with
        D = mask / sqrt(lumped_mass), rho = sum_a occ_a |sum_i N_i psi_a,i|^2
        (Eq. rho on the locally refined mesh)."""
        d = np.where(self.boundary_free, 0.0, 1.0 / np.sqrt(self.lumped_mass()))
        psi_all = self.P @ (d[:, None] * psi_bar)
        rho = np.zeros((len(self.leaves), len(self.wq)))
        for li in range(len(self.leaves)):
            vals = self.B @ psi_all[self.conn[li]]
            rho[li] = np.abs(vals) ** 2 @ np.asarray(occ, float)
        return rho

    def hartree(self, rho, Z, R):
        """v_H at every leaf's Gauss-Legendre points: -lap v_H = 4 pi rho (rho at
        those points, load by the same rule) with the Dirichlet data sum Z / |x - R|
        (Eqs. Hartree_possion, DiscretePoisson on the locally refined mesh).  Those
        data are the electrons' far field only for a neutral system (total charge of
        rho equal to sum Z), which callers must supply."""
        K, _ = self.stiffness_and_load(lambda x: np.zeros(len(x)))
        F_all = np.zeros(self.n_all)
        for li, (x0, h, _) in enumerate(self.leaves):
            w = self.wq * np.prod(h) / 8.0
            np.add.at(F_all, self.conn[li], self.B.T @ (w * 4.0 * np.pi * rho[li]))
        F = self.P.T @ F_all
        xf = self.nodes[self.free]
        g = sum(z / np.linalg.norm(xf - np.asarray(r)[None, :], axis=1) for z, r in zip(Z, R))
        B = np.where(self.boundary_free)[0]
        I = np.where(~self.boundary_free)[0]
        u = np.zeros(len(self.free))
        u[B] = g[B]
        u[I] = spla.spsolve(K[I][:, I].tocsc(), F[I] - K[I][:, B] @ u[B])
        ua = self.P @ u
        return np.stack([self.B @ ua[self.conn[li]] for li in range(len(self.leaves))])

    def potential(self, rho, Z, R, E, xc_kind: str = "pw92"):
        """v = v_N + v_H + v_xc - E . x at every leaf's Gauss-Legendre points."""
        from .xc import lda
        xq = self.quad_points()
        vN = np.zeros(xq.shape[:2])
        for z, r in zip(Z, R):
            vN -= z / np.linalg.norm(xq - np.asarray(r)[None, None, :], axis=2)
        return vN + self.hartree(rho, Z, R) + lda(rho, xc_kind)[1] - xq @ np.asarray(E, float)

    def magnus_step(self, psi_bar, occ, Z, R, dt, k, E):
        """One predictor-corrector step (Eq. ApproxMagnus) on the locally refined mesh
        with the field E at the mid-point and a fixed Krylov dimension k:
        psi_p = exp(-i dt Hbar[v(rho_n)]) psi_n, rho_mid = (rho_n + rho(psi_p)) / 2,
        psi_n+1 = exp(-i dt Hbar[v(rho_mid)]) psi_n.  psi_bar: (n_free, n_orb) complex,
        zero on the boundary free nodes."""
        from .krylov import expm_block
        I = np.where(~self.boundary_free)[0]

        def kexp(v, psi):
            out = np.zeros_like(psi)
            out[I] = expm_block(self.hbar(v), psi[I], dt, 1e-14, k, fixed_k=k)[0]
            return out
        rho_n = self.density(psi_bar, occ)
        psi_p = kexp(self.potential(rho_n, Z, R, E), psi_bar)
        rho_mid = 0.5 * (rho_n + self.density(psi_p, occ))
        return kexp(self.potential(rho_mid, Z, R, E), psi_bar)

    def quad_points(self):
        """Physical Gauss-Legendre points of every leaf, (n_leaves, nq, 3), in the
        order of self.wq (first axis fastest)."""
        return np.stack([x0[None, :] + 0.5 * (self.xq_ref + 1.0) * h[None, :] for x0, h, _ in self.leaves])

    def hamiltonian(self, vq, kin: float = 1.0):
        """P^T (kin (1/2) K_all + V_all) P with V_all = sum over leaves of
        int v N_m N_n, v given at every leaf's Gauss-Legendre points
        (n_leaves, nq) (the operator of Eq. Hmn on the locally refined mesh,
        constrained space)."""
        rows, cols, vals = [], [], []
        for li, (x0, h, _) in enumerate(self.leaves):
            idx = self.conn[li]
            G = [self.Dref[a] * (2.0 / h[a]) for a in range(3)]
            w = self.wq * np.prod(h) / 8.0
            Hc = kin * 0.5 * sum(G[a].T @ (w[:, None] * G[a]) for a in range(3)) + self.B.T @ ((w * vq[li])[:, None] * self.B)
            rows.append(np.repeat(idx, len(idx)))
            cols.append(np.tile(idx, len(idx)))
            vals.append(Hc.ravel())
        H_all = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                              shape=(self.n_all, self.n_all))
        return (self.P.T @ H_all @ self.P).tocsr()

    def solve_poisson(self, f, g):
        """-lap u = f with u = g on the boundary, in the constrained space: free
        values (n_free,) and all node values (n_all,)."""
        K, F = self.stiffness_and_load(f)
        B = np.where(self.boundary_free)[0]
        I = np.where(~self.boundary_free)[0]
        u = np.zeros(len(self.free))
        u[B] = g(self.nodes[self.free[B]])
        u[I] = spla.spsolve(K[I][:, I].tocsc(), F[I] - K[I][:, B] @ u[B])
        return u, self.P @ u

    def evaluate(self, u_all, li: int, pts):
        """Values at physical points inside leaf li."""
        x0, h, _ = self.leaves[li]
        ref = 2.0 * (np.asarray(pts) - x0[None, :]) / h[None, :] - 1.0
        L = [lagrange(self.xi, ref[:, a])[0] for a in range(3)]
        B = L[0][:, self.loc[:, 0]] * L[1][:, self.loc[:, 1]] * L[2][:, self.loc[:, 2]]
        return B @ u_all[self.conn[li]]
