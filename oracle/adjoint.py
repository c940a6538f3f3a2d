"""Adjoint (reverse-mode) gradient of a windowed dipole signal with respect to
the external-field parameters, through the second-order Magnus
predictor-corrector step (Eq. ApproxMagnus) with exact exponentials.

Test infrastructure only (see `oracle/__init__.py`).  The paper has no
adjoint; this is the exact discrete adjoint of the step written in
`oracle/tdks.py` (readings there), with every exponential exp(-i dt Hbar)
evaluated exactly by a dense eigendecomposition, so it is usable on small
systems only.

Objective: J = (1 / |W|) sum_{n in W} mu_d(rho_n), mu_d = d . (sum Z R - int x rho).
Parameters theta = (amp, omega, sigma) of a FIELD_SINE_GAUSS (or the
amplitude-like parameters of the other kinds).

Reverse sweep per step n (forward: v1 = V(rho_n) + f_n, psi^p = U(v1) psi_n,
rho_m = (rho_n + rho(psi^p)) / 2, v2 = V(rho_m) + f_n, psi_n+1 = U(v2) psi_n):
  psi_bar_n += U(v2)^H lam_n+1 + U(v1)^H lam_p
  v_bar(v, psi, lam)_q = Re <lam, dU_v[dH/dv_q] psi>  (Frechet derivative of the
      exponential, Daleckii-Krein: in the eigenbasis of Hbar,
      dU[E]_jk = E_jk (e^{-i dt l_j} - e^{-i dt l_k}) / (l_j - l_k))
  rho_bar += V'(rho)^T v_bar with V'(rho)^T g = w * Interp(A_II^-1 Interp^T g) + f_xc(rho) g
  psi_bar_a += 2 occ_a Phi^T (rho_bar * Phi psi_a)
  theta_bar += -(dE/dtheta)(t_mid) . sum_q x_q (v_bar1 + v_bar2)_q
Inner products are real parts of the Hermitian ones (psi is complex, theta real).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse.linalg as spla

from . import poisson, tdks, xc
from .operators import System


def field_and_derivs(f, t: float):
    """E(t) (3-vector) and dE/d(amp, omega, sigma) (3 x 3-vectors) for the
    field kinds with those parameters."""
    d = np.asarray(f.direction, dtype=np.float64)
    if f.kind == tdks.FIELD_SINE_GAUSS:
        g = math.exp(-(t - f.t0) ** 2 / (2.0 * f.sigma ** 2))
        sn, cs = math.sin(f.omega * t), math.cos(f.omega * t)
        e = f.amp * sn * g
        de = [sn * g, f.amp * t * cs * g, f.amp * sn * g * (t - f.t0) ** 2 / f.sigma ** 3]
    elif f.kind == tdks.FIELD_GAUSS:
        g = math.exp(-(t - f.t0) ** 2 / (2.0 * f.sigma ** 2))
        e = f.amp * g
        de = [g, 0.0, f.amp * g * (t - f.t0) ** 2 / f.sigma ** 3]
    else:
        raise ValueError("field kind without (amp, omega, sigma) derivatives")
    return e * d, [x * d for x in de]


def fxc(rho: np.ndarray) -> np.ndarray:
    """d v_xc / d rho for Slater exchange + PW92 correlation (0 below the floor)."""
    rho = np.asarray(rho, dtype=np.float64)
    ok = rho > xc.RHO_FLOOR
    r = np.where(ok, rho, 1.0)
    dvx = -(1.0 / 3.0) * np.cbrt(3.0 / np.pi) * r ** (-2.0 / 3.0)
    A, a1 = xc.PW92_A, xc.PW92_ALPHA1
    b1, b2, b3, b4 = xc.PW92_BETA
    rs = np.cbrt(3.0 / (4.0 * np.pi * r))
    srs = np.sqrt(rs)
    Q = 2 * A * (b1 * srs + b2 * rs + b3 * rs * srs + b4 * rs * rs)
    dQ = 2 * A * (0.5 * b1 / srs + b2 + 1.5 * b3 * srs + 2 * b4 * rs)
    d2Q = 2 * A * (-0.25 * b1 / (rs * srs) + 0.75 * b3 / srs + 2 * b4)
    L = np.log1p(1.0 / Q)
    dL = -dQ / (Q * (Q + 1.0))
    d2L = -d2Q / (Q * (Q + 1.0)) + dQ * dQ * (2 * Q + 1.0) / (Q * (Q + 1.0)) ** 2
    dG = -2 * A * a1 * L - 2 * A * (1 + a1 * rs) * dL
    d2G = -4 * A * a1 * dL - 2 * A * (1 + a1 * rs) * d2L
    dvc_drs = (2.0 / 3.0) * dG - rs / 3.0 * d2G
    dvc = dvc_drs * (-rs / (3.0 * r))
    return np.where(ok, dvx + dvc, 0.0)


class Adjoint:
    """Exact-exponential forward run and its reverse sweep on a small system."""

    def __init__(self, system: System):
        self.S = S = system
        m = S.mesh
        keep = np.concatenate([m.interior, np.ones(S.n_E, bool)])
        self.idx = np.where(keep)[0]
        # Phi: psi_bar (full DOF layout) -> values at all quadrature points
        n = S.n_dof
        eye = np.eye(n)
        vals = S.values_at_quad(eye)                      # (nc, nq, n)
        self.Phi = vals.reshape(-1, n)
        self.w = m.wJ.reshape(-1)
        self.xq = m.xq.reshape(-1, 3)
        self.vN = tdks.nuclear_potential(S)
        self.K0 = S.hbar(np.zeros_like(m.wJ)).toarray()   # kinetic part of Hbar
        # Hartree pieces: interior stiffness and interpolation
        A = (2.0 * S.Kcc / (4.0 * np.pi)).tocsr()
        self.I = np.where(m.interior)[0]
        self.AII = A[self.I][:, self.I].tocsc()
        self.Bq = np.zeros((m.n_cells * m.nq, S.n_h))     # nodal -> quadrature interpolation
        for c in range(m.n_cells):
            self.Bq[c * m.nq:(c + 1) * m.nq, m.conn[c]] += m.B

    # ---------------------------------------------------------------- pieces
    def hbar(self, v_flat):
        return self.K0 + self.Phi.T @ ((self.w * v_flat)[:, None] * self.Phi)

    def expm(self, H, dt):
        Hs = H[np.ix_(self.idx, self.idx)]
        lam, V = np.linalg.eigh(0.5 * (Hs + Hs.T))
        return lam, V

    def U(self, lamV, dt, X):
        lam, V = lamV
        out = np.zeros_like(X)
        out[self.idx] = V @ (np.exp(-1j * dt * lam)[:, None] * (V.T @ X[self.idx]))
        return out

    def density(self, psi, occ):
        u = self.Phi @ psi
        return np.sum(occ[None, :] * np.abs(u) ** 2, axis=1)

    def potential(self, rho):
        rq = rho.reshape(self.S.mesh.wJ.shape)
        _, vH = poisson.solve(self.S, rq)
        return (self.vN + vH + xc.lda(rq)[1]).reshape(-1)

    def field_pot(self, E):
        return -(self.xq @ E)

    def VT(self, rho, g):
        """V'(rho)^T g = w * Interp(A_II^-1 Interp^T g) + f_xc(rho) g."""
        b = self.Bq.T @ g
        phi = np.zeros(self.S.n_h)
        phi[self.I] = spla.spsolve(self.AII, b[self.I])
        return self.w * (self.Bq @ phi) + fxc(rho) * g

    def frechet_vjp(self, lamV, dt, psi, lam_bar):
        """v_bar_q = Re <lam_bar, dU[dH/dv_q] psi> summed over columns, by the
        Daleckii-Krein form of the Frechet derivative."""
        lam, V = lamV
        e = np.exp(-1j * dt * lam)
        dl = lam[:, None] - lam[None, :]
        with np.errstate(divide="ignore", invalid="ignore"):
            G = np.where(np.abs(dl) > 1e-12 * (1 + np.abs(lam[:, None])), (e[:, None] - e[None, :]) / dl,
                         -1j * dt * e[:, None])
        PV = self.Phi[:, self.idx] @ V                      # (nqpts, m)
        a = V.T @ lam_bar[self.idx]                         # (m, cols)
        b = V.T @ psi[self.idx]
        # Re sum_cols sum_jk conj(a_j) G_jk PV_qj PV_qk b_k
        out = np.zeros(self.Phi.shape[0])
        for col in range(psi.shape[1]):
            M = np.conj(a[:, col])[:, None] * G * b[:, col][None, :]     # (m, m)
            out += np.real(np.einsum("qj,jk,qk->q", PV, M, PV))
        return self.w * out

    # ---------------------------------------------------------------- drivers
    def step(self, psi, rho, E, dt, occ):
        f = self.field_pot(E)
        v1 = self.potential(rho) + f
        lv1 = self.expm(self.hbar(v1), dt)
        psip = self.U(lv1, dt, psi)
        rhop = self.density(psip, occ)
        rhom = 0.5 * (rho + rhop)
        v2 = self.potential(rhom) + f
        lv2 = self.expm(self.hbar(v2), dt)
        new = self.U(lv2, dt, psi)
        return new, dict(lv1=lv1, psip=psip, rhom=rhom, lv2=lv2)

    def dipole_d(self, rho, direction):
        wl = self.S.wl
        nuc = np.sum(wl.Z[:, None] * wl.R, axis=0)
        return float(np.dot(direction, nuc - (self.w * rho) @ self.xq))

    def run(self, psi0, field, dt, n_steps, occ, window, direction):
        """Forward run; returns J and the stored states."""
        d = np.asarray(direction, dtype=np.float64)
        psi = psi0.copy()
        rho = self.density(psi, occ)
        states = [(psi, rho)]
        J = 0.0
        for n in range(n_steps):
            E, _ = field_and_derivs(field, n * dt + 0.5 * dt)
            psi, _ = self.step(psi, rho, E, dt, occ)
            rho = self.density(psi, occ)
            states.append((psi, rho))
            if n + 1 in window:
                J += self.dipole_d(rho, d) / len(window)
        return J, states

    def gradient(self, psi0, field, dt, n_steps, occ, window, direction):
        """(J, dJ/d(amp, omega, sigma)) by the reverse sweep."""
        d = np.asarray(direction, dtype=np.float64)
        J, states = self.run(psi0, field, dt, n_steps, occ, window, direction)
        theta_bar = np.zeros(3)
        psi_bar = np.zeros_like(psi0)
        rho_bar = np.zeros_like(states[0][1])
        for n in range(n_steps, 0, -1):
            psi_n1, rho_n1 = states[n]
            if n in window:
                rho_bar = rho_bar - (self.w * (self.xq @ d)) / len(window)
            # rho_{n+1} = rho(psi_{n+1})
            psi_bar = psi_bar + 2.0 * (self.Phi.T @ (rho_bar[:, None] * (self.Phi @ psi_n1))) * occ[None, :]
            rho_bar = np.zeros_like(rho_bar)
            # recompute step n-1 -> n
            psi, rho = states[n - 1]
            tm = (n - 1) * dt + 0.5 * dt
            E, dE = field_and_derivs(field, tm)
            _, st = self.step(psi, rho, E, dt, occ)
            lam_next = psi_bar
            psi_bar = self._Uh(st["lv2"], dt, lam_next)
            vb2 = self.frechet_vjp(st["lv2"], dt, psi, lam_next)
            rb_m = self.VT(st["rhom"], vb2)
            rho_bar = rho_bar + 0.5 * rb_m
            rb_p = 0.5 * rb_m
            lam_p = 2.0 * (self.Phi.T @ (rb_p[:, None] * (self.Phi @ st["psip"]))) * occ[None, :]
            psi_bar = psi_bar + self._Uh(st["lv1"], dt, lam_p)
            vb1 = self.frechet_vjp(st["lv1"], dt, psi, lam_p)
            rho_bar = rho_bar + self.VT(rho, vb1)
            fb = vb1 + vb2
            s = self.xq.T @ fb                                    # sum_q x_q f_bar_q
            theta_bar += np.array([-float(np.dot(de, s)) for de in dE])
        return J, theta_bar

    def _Uh(self, lamV, dt, X):
        """U^H X = exp(+i dt Hbar) X."""
        return self.U(lamV, -dt, X)
