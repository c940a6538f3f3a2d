"""Electrostatic potentials (nuclear and Hartree) in the enriched finite element
basis (Eqs. PhiEFE, DiscretePoisson).

Test infrastructure only (see `oracle/__init__.py`).

phi^h = sum_j N^C_j phi^C_j + sum_I N^{E,phi}_I phi^E_I (Eq. PhiEFE) with one
enrichment function per atom, N^{E,phi}_I = N^{A,phi}_I - sum_i c_Ii N^C_i: the
atomic part is the smoothly truncated, spherically symmetric electrostatic
potential of the isolated atom, and the orthogonalising part is the combination
of the interior classical functions with c_Ii = int N^{A,phi}_I N^C_i / M_i, M the
GLL-lumped classical mass (the inner product the spectral classical basis is
orthogonal in, as for the wavefunction enrichment in module operators).  The
discrete Poisson problem is A phi = d (Eq. DiscretePoisson) with
A_mn = (1/4 pi) int grad N_m . grad N_n over the classical and enriched
functions, d_m = int b N_m, and the classical boundary nodes holding the
Dirichlet data (the enrichment functions vanish on the boundary: their support
r < r0 lies inside the box).

Readings (the paper leaves b and the atomic potential to its references):
  E1  b(r) = -sum_I Z_I g(|r - R_I|), g the normalised Gaussian of width sigma:
      a point charge has no finite-energy weak form.  Its potential, and the
      Dirichlet data, is v(r) = -sum_I Z_I erf(|r - R_I| / (sqrt2 sigma)) / |r - R_I|.
  E2  N^{A,phi}_I = -Z_I erf(r / (sqrt2 sigma)) / r * u(r; r0, s), u the smooth
      cutoff of the wavefunction enrichment (module enrich).
  E3  Cell integrals use Gauss-Legendre n^3 rules on sub^3 sub-cells of every
      cell: the Gaussian core is narrower than the cells around a nucleus (the
      paper's adaptive quadrature is a later item).
  H1  for the Hartree potential, the atomic part is the Hartree potential of
      the isolated neutral atom whose density fills the shells of its
      wavefunction enrichment functions (class RadialAtom).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.special import erf

from .basis import gauss_legendre, lagrange
from .enrich import cutoff


class CompositeRule:
    """Reference rule on [-1, 1]^3: sub^3 sub-cells with n^3 Gauss-Legendre
    points each; values (nq, nn) and reference derivatives of the cell's
    Lagrange basis there, in the mesh's local node order (i1 fastest)."""

    def __init__(self, mesh, sub: int, n: int):
        xg, wg = gauss_legendre(n)
        x1, w1 = [], []
        for k in range(sub):
            a, b = -1.0 + 2.0 * k / sub, -1.0 + 2.0 * (k + 1) / sub
            x1.append(0.5 * (b - a) * xg + 0.5 * (a + b))
            w1.append(0.5 * (b - a) * wg)
        x1, w1 = np.concatenate(x1), np.concatenate(w1)
        L, dL = lagrange(mesh.xi, x1)
        m1 = len(x1)
        k3, k2, k1 = np.meshgrid(np.arange(m1), np.arange(m1), np.arange(m1), indexing="ij")
        Q = np.stack([k1.ravel(), k2.ravel(), k3.ravel()], axis=1)
        p1 = mesh.p + 1
        i3, i2, i1 = np.meshgrid(np.arange(p1), np.arange(p1), np.arange(p1), indexing="ij")
        loc = np.stack([i1.ravel(), i2.ravel(), i3.ravel()], axis=1)
        self.x = x1[Q]
        self.w = w1[Q[:, 0]] * w1[Q[:, 1]] * w1[Q[:, 2]]
        tab = lambda f, a: f[a][Q[:, 0][:, None], loc[:, 0][None, :]] * f[a + 1][Q[:, 1][:, None], loc[:, 1][None, :]] \
            * f[a + 2][Q[:, 2][:, None], loc[:, 2][None, :]]
        self.B = tab([L, L, L], 0)
        self.D = [tab([dL, L, L], 0), tab([L, dL, L], 0), tab([L, L, dL], 0)]

    def cell(self, mesh, c: int):
        """Physical points (nq, 3), weights (nq,), values (nq, nn) and physical
        gradients [3 x (nq, nn)] of the basis on cell c."""
        h = mesh.h[c]
        pts = mesh.x0[c][None, :] + 0.5 * (self.x + 1.0) * h[None, :]
        w = self.w * mesh.detJ[c]
        G = [self.D[a] * (2.0 / h[a]) for a in range(3)]
        return pts, w, self.B, G


def smeared_potential(Z, R, sigma: float, pts: np.ndarray) -> np.ndarray:
    """v(r) = -sum_I Z_I erf(|r - R_I| / (sqrt2 sigma)) / |r - R_I| (reading E1)."""
    v = np.zeros(len(pts))
    for z, r0 in zip(Z, R):
        r = np.linalg.norm(pts - np.asarray(r0)[None, :], axis=1)
        with np.errstate(invalid="ignore", divide="ignore"):
            f = np.where(r > 0, erf(r / (math.sqrt(2.0) * sigma)) / r, math.sqrt(2.0 / math.pi) / sigma)
        v -= z * f
    return v


def smeared_charge(Z, R, sigma: float, pts: np.ndarray) -> np.ndarray:
    """b(r) = -sum_I Z_I (2 pi sigma^2)^(-3/2) exp(-|r - R_I|^2 / (2 sigma^2)) (reading E1)."""
    b = np.zeros(len(pts))
    norm = (2.0 * math.pi * sigma * sigma) ** -1.5
    for z, r0 in zip(Z, R):
        r2 = np.sum((pts - np.asarray(r0)[None, :]) ** 2, axis=1)
        b -= z * norm * np.exp(-r2 / (2.0 * sigma * sigma))
    return b


def nuclear_radial(z: float, sigma: float):
    """r -> (f, df/dr) for f = -z erf(r / (sqrt2 sigma)) / r, the potential of one
    smeared nucleus (readings E1, E2; df/dr -> 0 as r -> 0)."""
    a = 1.0 / (math.sqrt(2.0) * sigma)

    def f(r):
        r = np.asarray(r, float)
        with np.errstate(invalid="ignore", divide="ignore"):
            v = np.where(r > 0, -z * erf(a * r) / r, -z * 2.0 * a / math.sqrt(math.pi))
            dv = np.where(r > 1e-8, -z * (2.0 * a * np.exp(-(a * r) ** 2) / (math.sqrt(math.pi) * r)
                                          - erf(a * r) / r ** 2), 0.0)
        return v, dv
    return f


class EnrichedPoisson:
    """A phi = d in the classical basis plus one orthogonalised enrichment
    function per atom (Eqs. PhiEFE, DiscretePoisson): atomic parts
    potentials[I](r) -> (f, df/dr) times the cutoff u, the load d = int charge N,
    Dirichlet data on the classical boundary nodes.  enrich=False gives the
    classical-only solve on the same mesh and rule."""

    def __init__(self, mesh, centers, potentials, charge, dirichlet, r0: float, s: float, sub: int = 2,
                 n: int = None, enrich: bool = True, rule=None):
        self.mesh, self.R = mesh, [np.asarray(x, float) for x in centers]
        self.potentials, self.charge, self.dirichlet = list(potentials), charge, dirichlet
        self.r0, self.s = r0, s
        # cell rule: uniform sub-cells (reading E3) unless given (e.g. quadrature.AdaptiveRule)
        self.rule = rule if rule is not None else CompositeRule(mesh, sub, n or mesh.nq1)
        self.nE = len(self.R) if enrich else 0
        n_h = mesh.n_nodes
        M = mesh.lumped_mass()
        Minv = np.where(mesh.interior, 1.0 / M, 0.0)
        # orthogonalisation coefficients c_Ii = int N^A_I N^C_i / M_i (interior i)
        bA = np.zeros((self.nE, n_h))
        for c in range(mesh.n_cells):
            pts, w, Bc, _ = self.rule.cell(mesh, c)
            for I in range(self.nE):
                va, _ = self._atomic(I, pts)
                np.add.at(bA[I], mesh.conn[c], Bc.T @ (w * va))
        self.C = bA * Minv[None, :]
        # assembly of A (classical, classical-enriched, enriched) and of d = int charge N
        rows, cols, vals = [], [], []
        ACE = np.zeros((n_h, self.nE))
        AEE = np.zeros((self.nE, self.nE))
        dC = np.zeros(n_h)
        dE = np.zeros(self.nE)
        k = 1.0 / (4.0 * math.pi)
        for c in range(mesh.n_cells):
            pts, w, Bc, G = self.rule.cell(mesh, c)
            idx = mesh.conn[c]
            Kc = k * sum(G[a].T @ (w[:, None] * G[a]) for a in range(3))
            rows.append(np.repeat(idx, len(idx)))
            cols.append(np.tile(idx, len(idx)))
            vals.append(Kc.ravel())
            b = charge(pts)
            dC[idx] += Bc.T @ (w * b)
            if self.nE:
                vE, gE = self._enriched_at(c, pts, Bc, G)
                for a in range(3):
                    ACE[idx] += k * (G[a].T @ (w[:, None] * gE[a]))
                    AEE += k * (gE[a].T @ (w[:, None] * gE[a]))
                dE += vE.T @ (w * b)
        self.Acc = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n_h, n_h))
        self.ACE, self.AEE, self.dC, self.dE = ACE, AEE, dC, dE

    def _atomic(self, I: int, pts):
        """Values and gradients of the atomic part N^{A,phi}_I = f(r) u(r)."""
        d = pts - self.R[I][None, :]
        r = np.sqrt(np.sum(d * d, axis=1))
        f, df = self.potentials[I](r)
        with np.errstate(invalid="ignore", divide="ignore"):
            rhat = np.where(r[:, None] > 0, d / r[:, None], 0.0)
        u, du = cutoff(r, self.r0, self.s)
        return f * u, (df * u + f * du)[:, None] * rhat

    def _enriched_at(self, c: int, pts, Bc, G):
        """Values (nq, nE) and gradients [3 x (nq, nE)] of the orthogonalised
        enrichment functions on cell c."""
        idx = self.mesh.conn[c]
        v = np.zeros((len(pts), self.nE))
        g = [np.zeros((len(pts), self.nE)) for _ in range(3)]
        for I in range(self.nE):
            va, ga = self._atomic(I, pts)
            cI = self.C[I, idx]
            v[:, I] = va - Bc @ cI
            for a in range(3):
                g[a][:, I] = ga[:, a] - G[a] @ cI
        return v, g

    def system(self):
        """The Galerkin matrix on the interior classical and enrichment unknowns."""
        I = np.where(self.mesh.interior)[0]
        AII = self.Acc[I][:, I]
        if not self.nE:
            return AII.tocsc()
        top = sp.hstack([AII, sp.csr_matrix(self.ACE[I])])
        bot = sp.hstack([sp.csr_matrix(self.ACE[I].T), sp.csr_matrix(self.AEE)])
        return sp.vstack([top, bot]).tocsc()

    def solve(self, phiB=None, dC=None, dE=None):
        """Classical nodal values (n_h,) and enrichment coefficients (nE,): the
        boundary nodes hold phiB (default: the analytic potential of b), the
        interior and the enrichment coefficients solve the Galerkin system with
        the loads dC, dE (default: int b N)."""
        m = self.mesh
        I = np.where(m.interior)[0]
        Bn = np.where(m.boundary)[0]
        if phiB is None:
            phiB = self.dirichlet(m.nodes[Bn])
        dC = self.dC if dC is None else dC
        dE = self.dE if dE is None else dE
        AIB = self.Acc[I][:, Bn]
        K = self.system()
        rhs = dC[I] - AIB @ phiB
        if self.nE:
            rhs = np.concatenate([rhs, dE - self.ACE[Bn].T @ phiB])
        x = spla.spsolve(K, rhs)
        phi = np.zeros(m.n_nodes)
        phi[Bn] = phiB
        phi[I] = x[:len(I)]
        return phi, x[len(I):]

    def evaluate(self, phi: np.ndarray, phiE: np.ndarray, c: int):
        """phi^h at the rule's points of cell c (points, values)."""
        pts, w, Bc, G = self.rule.cell(self.mesh, c)
        val = Bc @ phi[self.mesh.conn[c]]
        if self.nE:
            vE, _ = self._enriched_at(c, pts, Bc, G)
            val = val + vE @ phiE
        return pts, val


class NuclearEFE(EnrichedPoisson):
    """The nuclear potential of smeared point charges (readings E1-E3)."""

    def __init__(self, mesh, Z, R, sigma: float, r0: float, s: float, sub: int = 2, n: int = None,
                 enrich: bool = True, rule=None):
        self.Z, self.sigma = list(Z), sigma
        super().__init__(mesh, R, [nuclear_radial(z, sigma) for z in self.Z],
                         lambda p: smeared_charge(self.Z, R, sigma, p),
                         lambda p: smeared_potential(self.Z, R, sigma, p), r0, s, sub, n, enrich, rule)


# ---------------------------------------------------------------------------
# Hartree potential with atomic Hartree potentials as enrichment (Eq. PhiEFE,
# "the electrostatic potential ... of an isolated atom": Hartree part).
# Reading H1: the isolated neutral atom's density fills the shells of its
# wavefunction enrichment functions (same n, l, radial shape and zeta) in the
# order of n, then l, two electrons per orbital: rho_I(r) = sum_nl occ_nl
# R_nl(r)^2 / (4 pi int R_nl^2 r^2 dr).  Its Hartree potential is the spherical
# solution v(r) = (4 pi / r) int_0^r rho s^2 ds + 4 pi int_r^inf rho s ds, with
# dv/dr = -Q(r) / r^2, Q the enclosed charge, on a radial grid.
# ---------------------------------------------------------------------------
class RadialAtom:
    """Density and Hartree potential of one isolated atom (reading H1), tabulated
    on r = rmax t^2 with n points uniform in t (cumulative trapezoid integrals in t)."""

    def __init__(self, shells, n_el: float, rmax: float = 60.0, n: int = 24001):
        from .enrich import radial
        tt = np.linspace(0.0, 1.0, n)
        r = rmax * tt * tt            # dense near the nucleus, where the core shells vary fastest
        rho = np.zeros_like(r)
        left = float(n_el)
        for (kind, nn, l, zeta) in sorted(shells, key=lambda x: (x[1], x[2])):
            occ = min(left, 2.0 * (2 * l + 1))
            if occ <= 0:
                break
            f, _ = radial(kind, nn, l, zeta, r)
            R = f * r ** l
            norm = _trapezoid_total(R * R * r * r, r)
            rho += occ * R * R / (4.0 * math.pi * norm)
            left -= occ
        self.r, self.rho = r, rho
        q = 4.0 * math.pi * _cum_trapezoid(rho * r * r, r)          # enclosed charge Q(r)
        outer = 4.0 * math.pi * (_trapezoid_total(rho * r, r) - _cum_trapezoid(rho * r, r))
        with np.errstate(invalid="ignore", divide="ignore"):
            self.v = np.where(r > 0, q / r, 0.0) + outer
        self.v[0] = 4.0 * math.pi * _trapezoid_total(rho * r, r)
        self.q = q
        self.n_el = q[-1]

    def density(self, r):
        return np.interp(r, self.r, self.rho, right=0.0)

    def potential(self, r):
        """v(r) and dv/dr = -Q(r) / r^2 (v -> Q/r beyond the table)."""
        r = np.asarray(r, float)
        v = np.where(r <= self.r[-1], np.interp(r, self.r, self.v), self.n_el / np.maximum(r, 1e-300))
        Q = np.interp(r, self.r, self.q, right=self.n_el)
        with np.errstate(invalid="ignore", divide="ignore"):
            dv = np.where(r > 0, -Q / (r * r), 0.0)
        return v, dv


def _cum_trapezoid(y, x):
    """Cumulative integral of y dr on the grid r = rmax t^2: the trapezoid rule
    in t with dr = 2 rmax t dt (uniform in t)."""
    t = np.sqrt(x / x[-1])
    g = y * 2.0 * x[-1] * t
    out = np.zeros_like(y)
    out[1:] = np.cumsum(0.5 * (g[1:] + g[:-1]) * np.diff(t))
    return out


def _trapezoid_total(y, x):
    return float(_cum_trapezoid(y, x)[-1])


class HartreeEFE(EnrichedPoisson):
    """The Hartree potential of a density given as a function of position, with
    the atoms' Hartree potentials (reading H1) as enrichment; Dirichlet data
    from `dirichlet` (default: the superposition of the atomic potentials, the
    exact solution when the density is the superposition of atomic densities)."""

    def __init__(self, mesh, atoms, centers, density, r0: float, s: float, dirichlet=None, sub: int = 2,
                 n: int = None, enrich: bool = True):
        self.atoms = list(atoms)
        centers = [np.asarray(x, float) for x in centers]
        if dirichlet is None:
            def dirichlet(p):
                v = np.zeros(len(p))
                for A, R in zip(self.atoms, centers):
                    v += A.potential(np.linalg.norm(p - R[None, :], axis=1))[0]
                return v
        super().__init__(mesh, centers, [A.potential for A in self.atoms], density, dirichlet, r0, s, sub, n,
                         enrich)
