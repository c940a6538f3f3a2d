"""Density, potentials, dipole and the second-order Magnus predictor-corrector
step (Secs. "Time dependent Kohn-Sham equations", "Magnus Propagator").

Test infrastructure only (see `oracle/__init__.py`).

Columns of psi_bar are ordered member-major: column b * n_orb + alpha is
orbital alpha of batch member b; every batch member has its own density,
potentials and field.

Readings (the paper defers the predictor-corrector to its references):
  S1  psi^p   = Kexp(Hbar[v(rho_n), E(t_n + dt/2)]) psi_n
  S2  rho^p   = rho(psi^p)
  S3  rho_mid = (rho_n + rho^p) / 2
  S4  v_mid   = v_N + v_H[rho_mid] + v_xc[rho_mid] - E(t_n + dt/2) . x
  S5  psi_n+1 = Kexp(Hbar[v_mid]) psi_n
  S6  rho_n+1, v_H[rho_n+1], v_xc[rho_n+1] (reused by the next S1), mu(t_n+1)
Potential-extrapolation variant (scheme "extrapolated", one exponential per
step): the Hartree + xc potential at the mid-point is the linear
extrapolation from the two latest steps, v_Hxc(t_n + dt/2) ~
(3 v_Hxc(t_n) - v_Hxc(t_n-1)) / 2, and psi_n+1 = Kexp(Hbar[v_N + v_Hxc +
v_f(t_n + dt/2)]) psi_n; a step without history (the first of a run) is a
predictor-corrector step.  Both schemes are second order in dt (pinned).
v_N = -sum Z_I / |x - R_I| is evaluated in closed form at the quadrature
points (the nuclear Poisson problem with point sources needs the
electrostatic enrichment, which is not used).  Eq. VField: v_f = -E(t) . x.
Dipole: mu = sum_I Z_I R_I - int x rho.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import krylov, poisson, xc
from .operators import System

FIELD_NONE, FIELD_GAUSS, FIELD_SINE_GAUSS, FIELD_SINE_TRAP, FIELD_SINE_SINE = 0, 1, 2, 3, 4


def field_value(f, t: float) -> np.ndarray:
    """E(t) as a 3-vector for one field description."""
    d = np.asarray(f.direction, dtype=np.float64)
    if f.kind == FIELD_NONE:
        a = 0.0
    elif f.kind == FIELD_GAUSS:
        a = f.amp * math.exp(-(t - f.t0) ** 2 / (2.0 * f.sigma ** 2))
    elif f.kind == FIELD_SINE_GAUSS:
        a = f.amp * math.sin(f.omega * t) * math.exp(-(t - f.t0) ** 2 / (2.0 * f.sigma ** 2))
    elif f.kind == FIELD_SINE_TRAP:
        env = min(t / f.ramp, (f.period - t) / f.ramp, 1.0) if f.ramp > 0 else 1.0
        env = max(env, 0.0) if 0.0 <= t <= f.period else 0.0
        a = f.amp * math.sin(f.omega * t) * env
    elif f.kind == FIELD_SINE_SINE:
        a = f.amp * math.sin(math.pi * t / f.period) * math.sin(f.omega * t) if 0.0 <= t <= f.period else 0.0
    else:
        raise ValueError("unknown field kind")
    return a * d


def nuclear_potential(system: System) -> np.ndarray:
    """v_N = -sum_I Z_I / |x_q - R_I| (Eq. VN) at the quadrature points."""
    wl = system.wl
    xq = system.mesh.xq
    v = np.zeros(xq.shape[:2])
    for Z, R in zip(wl.Z, wl.R):
        v -= Z / np.sqrt(np.sum((xq - R[None, None, :]) ** 2, axis=2))
    return v


def density(system: System, psi_bar: np.ndarray, occ: np.ndarray, batch: int) -> np.ndarray:
    """rho_q = sum_alpha f_alpha |psi_alpha(x_q)|^2 per batch member:
    (batch, n_cells, nq)."""
    vals = system.values_at_quad(psi_bar)
    n_orb = len(occ)
    rho = np.zeros((batch,) + vals.shape[:2])
    for b in range(batch):
        blk = vals[:, :, b * n_orb:(b + 1) * n_orb]
        rho[b] = np.sum(occ[None, None, :] * np.abs(blk) ** 2, axis=2)
    return rho


def dipole(system: System, rho_q: np.ndarray) -> np.ndarray:
    """mu = sum_I Z_I R_I - int x rho for one density (n_cells, nq)."""
    wl = system.wl
    m = system.mesh
    nuc = np.sum(wl.Z[:, None] * wl.R, axis=0)
    el = np.einsum("cq,cqa->a", m.wJ * rho_q, m.xq)
    return nuc - el


@dataclass
class State:
    rho: np.ndarray    # (batch, n_cells, nq)
    vH: np.ndarray     # (batch, n_cells, nq)
    vxc: np.ndarray    # (batch, n_cells, nq)
    phi: np.ndarray    # (batch, n_h) nodal Hartree potential
    vhxc_prev: np.ndarray = None   # v_H + v_xc of the previous step (None: no history)


def potentials(system: System, rho: np.ndarray, xc_kind: str = "pw92", hartree=None):
    """v_H and v_xc for a batch of densities.  hartree(system, rho_b) -> (classical
    nodal values, v_H at the quadrature points) replaces the classical Poisson
    solve (e.g. an enriched solve of module electrostatic)."""
    solve = hartree or poisson.solve
    vH = np.zeros_like(rho)
    vxc = np.zeros_like(rho)
    phi = np.zeros((rho.shape[0], system.n_h))
    for b in range(rho.shape[0]):
        phi[b], vH[b] = solve(system, rho[b])
        vxc[b] = xc.lda(rho[b], xc_kind)[1]
    return vH, vxc, phi


def make_state(system: System, psi_bar: np.ndarray, occ: np.ndarray, batch: int, xc_kind: str = "pw92",
               hartree=None, reduce=None) -> State:
    """reduce(rho) -> rho summed over processes, when the orbitals are split among them
    (rho is a sum over orbitals; None: all orbitals are here)."""
    rho = density(system, psi_bar, occ, batch)
    if reduce is not None:
        rho = reduce(rho)
    vH, vxc, phi = potentials(system, rho, xc_kind, hartree)
    return State(rho=rho, vH=vH, vxc=vxc, phi=phi)


def field_potential(system: System, E: np.ndarray) -> np.ndarray:
    return -np.einsum("cqa,a->cq", system.mesh.xq, E)


def kexp_members(system: System, psi_bar, v_members, n_orb, dt, tol, k_max, fixed_k=0, kin=1.0, reorth=False):
    out = np.empty_like(psi_bar)
    ks = []
    for b, vq in enumerate(v_members):
        H = system.hbar(vq, kin)
        sl = slice(b * n_orb, (b + 1) * n_orb)
        out[:, sl], k, _ = krylov.expm_block(H, psi_bar[:, sl], dt, tol, k_max, fixed_k, reorth)
        ks.append(k)
    return out, np.concatenate(ks)


def magnus_step(system: System, psi_bar: np.ndarray, state: State, t: float, dt: float, fields, occ,
                tol: float, k_max: int, fixed_k: int = 0, vN=None, scheme: str = "pc", xc_kind: str = "pw92",
                hartree=None, reduce=None, reorth=False):
    """One step: predictor-corrector S1..S6 (scheme "pc"), or the
    potential-extrapolation step (scheme "extrapolated"; predictor-corrector
    while the state has no history).  Returns (psi_new, state_new, mu
    (batch, 3), info dict).  With the orbitals split among processes, psi_bar
    and occ are this process's and reduce(rho) sums a density over the
    processes (each orbital's exponential is independent of the others).  reorth: the
    Lanczos recurrence of every exponential with CGS2 reorthogonalisation."""
    red = (lambda r: r) if reduce is None else reduce
    batch = len(fields)
    n_orb = len(occ)
    if vN is None:
        vN = nuclear_potential(system)
    Emid = [field_value(f, t + 0.5 * dt) for f in fields]
    vhxc = state.vH + state.vxc
    if scheme == "extrapolated" and state.vhxc_prev is not None:
        vx = 1.5 * vhxc - 0.5 * state.vhxc_prev
        v2 = [vN + vx[b] + field_potential(system, Emid[b]) for b in range(batch)]
        k1 = np.zeros(0, dtype=int)
    elif scheme in ("pc", "extrapolated"):
        v1 = [vN + vhxc[b] + field_potential(system, Emid[b]) for b in range(batch)]
        psi_p, k1 = kexp_members(system, psi_bar, v1, n_orb, dt, tol, k_max, fixed_k, reorth=reorth)
        rho_p = red(density(system, psi_p, occ, batch))
        rho_mid = 0.5 * (state.rho + rho_p)
        vH_mid, vxc_mid, _ = potentials(system, rho_mid, xc_kind, hartree)
        v2 = [vN + vH_mid[b] + vxc_mid[b] + field_potential(system, Emid[b]) for b in range(batch)]
    else:
        raise ValueError("unknown scheme")
    psi_new, k2 = kexp_members(system, psi_bar, v2, n_orb, dt, tol, k_max, fixed_k, reorth=reorth)
    new_state = make_state(system, psi_new, occ, batch, xc_kind, hartree, reduce)
    new_state.vhxc_prev = vhxc
    mu = np.stack([dipole(system, new_state.rho[b]) for b in range(batch)])
    return psi_new, new_state, mu, {"k_pred": k1, "k_corr": k2}


def kick(system: System, psi_bar: np.ndarray, fields, n_orb: int, tol: float = 1e-14, k_max: int = 30):
    """Delta kick psi_bar <- exp(i kappa d.Xbar) psi_bar per batch member, with
    Xbar = M^-1/2 P^T X_ext P M^-1/2 and X_ext the matrix of int (d.x) N_m N_n.
    Computed as the Lanczos exponential of the potential-only operator with
    v = -(d.x) and time step kappa."""
    out = psi_bar.copy()
    for b, f in enumerate(fields):
        if f.kick == 0.0:
            continue
        vq = field_potential(system, np.asarray(f.direction, dtype=np.float64))
        H = system.hbar(vq, kin=0.0)
        sl = slice(b * n_orb, (b + 1) * n_orb)
        out[:, sl], _, _ = krylov.expm_block(H, psi_bar[:, sl], f.kick, tol, k_max)
    return out


def ground_state(system: System, n_orb: int, occ: np.ndarray, mix: float = 0.3, tol: float = 1e-10,
                 max_iter: int = 200, psi_guess=None):
    """Self-consistent ground state by diagonalisation of Hbar on the
    interior + enrichment DOFs with linear density mixing.  Pinned by its
    results: the helium atom's LDA 1s eigenvalue against the tabulated
    all-electron value (tests/test_oracle_ground_state.py), and the H2 state's
    stationarity under the Magnus propagation.  The phase of each orbital is
    fixed so that its overlap with the guess is real and positive."""
    import scipy.sparse.linalg as spla
    keep = np.concatenate([system.mesh.interior, np.ones(system.n_E, dtype=bool)])
    idx = np.where(keep)[0]
    vN = nuclear_potential(system)
    if psi_guess is None:
        psi_guess = system.initial_orbitals()
    rho = density(system, psi_guess, occ, 1)
    eps = None
    for it in range(max_iter):
        vH, vxc, _ = potentials(system, rho)
        H = system.hbar(vN + vH[0] + vxc[0])
        Hs = H[idx][:, idx]
        lam, U = spla.eigsh(Hs, k=n_orb, which="SA", tol=1e-14, maxiter=100000)
        order = np.argsort(lam)
        lam, U = lam[order], U[:, order]
        psi = np.zeros((system.n_dof, n_orb), dtype=np.complex128)
        psi[idx] = U
        rho_new = density(system, psi, occ, 1)
        change = float(np.max(np.abs(rho_new - rho)))
        eps = lam
        if change < tol:
            rho = rho_new
            break
        rho = (1.0 - mix) * rho + mix * rho_new
    # fix phases against the guess
    for a in range(n_orb):
        ov = np.vdot(psi[:, a], psi_guess[:, a])
        if abs(ov) > 0:
            psi[:, a] *= ov / abs(ov)
    return psi, eps
