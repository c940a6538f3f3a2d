"""Adaptive Lanczos (Krylov) approximation of exp(-i dt Hbar) psi_bar (Eqs.
AdaptiveKrylov, AdaptiveKrylovErr).

Test infrastructure only (see `oracle/__init__.py`).

Per column, in the paper's order:
  q_1 = psi / ||psi||;  for j = 1, 2, ...:
     w = Hbar q_j;  alpha_j = Re <q_j, w>;  w <- w - alpha_j q_j - beta_{j-1} q_{j-1};
     beta_j = ||w||;  T_j = tridiag(alpha, beta);  y = exp(-i dt T_j) e_1
     (from the eigendecomposition of the real symmetric T_j);
     eps_j = |dt| * beta_j * ||psi|| * |y_j|;
     stop when eps_j <= tol (or beta_j == 0, or j == k_max);  q_{j+1} = w / beta_j
  result = ||psi|| Q_k y.
Readings: T_k of Eq. AdaptiveKrylov is that of A~ = -i dt Hbar, so its
(k+1, k) entry has magnitude |dt| * beta_k, which is where the |dt| in eps_k
comes from; the paper is silent on reorthogonalisation: by default the plain
three-term recurrence is used, and with reorth=True every new w is made
orthogonal to q_1 .. q_j by classical Gram-Schmidt applied twice (CGS2:
w <- w - Q (Q^H w), two times) before beta_j = ||w|| is taken, alpha_j and the
recurrence itself unchanged; with fixed_k > 0 exactly fixed_k steps are taken
(used by tests that must not depend on where a threshold falls).
"""
from __future__ import annotations

import numpy as np


def tridiag_expm_e1(alpha, beta, dt):
    """y = exp(-i dt T) e_1 for the real symmetric tridiagonal T."""
    k = len(alpha)
    T = np.diag(np.asarray(alpha, dtype=np.float64))
    if k > 1:
        T += np.diag(np.asarray(beta[:k - 1], dtype=np.float64), 1) + np.diag(np.asarray(beta[:k - 1]), -1)
    lam, U = np.linalg.eigh(T)
    return U @ (np.exp(-1j * dt * lam) * U[0, :])


def expm_column(matvec, psi: np.ndarray, dt: float, tol: float, k_max: int, fixed_k: int = 0, reorth: bool = False,
                return_basis: bool = False):
    """Returns (exp(-i dt Hbar) psi approximation, k used, eps_k, hit_cap), and the normalised
    Lanczos vectors q_1 .. q_k (columns) as a fifth item with return_basis."""
    nrm = np.linalg.norm(psi)
    if nrm == 0.0:
        return psi.copy(), 0, 0.0, False
    q = psi / nrm
    Q = [q]
    alphas, betas = [], []
    q_prev = np.zeros_like(q)
    beta_prev = 0.0
    y = np.array([1.0 + 0j])
    eps = 0.0
    hit_cap = False
    for j in range(1, k_max + 1):
        w = matvec(q)
        a = float(np.real(np.vdot(q, w)))
        w = w - a * q - beta_prev * q_prev
        if reorth:
            Qm = np.stack(Q, axis=1)
            for _ in range(2):
                w = w - Qm @ (Qm.conj().T @ w)
        b = float(np.linalg.norm(w))
        alphas.append(a)
        betas.append(b)
        y = tridiag_expm_e1(alphas, betas, dt)
        eps = abs(dt) * b * nrm * abs(y[-1])
        if fixed_k > 0:
            if j == fixed_k:
                break
        elif eps <= tol or b == 0.0:
            break
        if j == k_max:
            hit_cap = fixed_k <= 0
            break
        q_prev, beta_prev = q, b
        q = w / b
        Q.append(q)
    k = len(alphas)
    Qk = np.stack(Q[:k], axis=1)
    out = nrm * (Qk @ y)
    if return_basis:
        return out, k, eps, hit_cap, Qk
    return out, k, eps, hit_cap


def expm_block(Hbar, psi: np.ndarray, dt: float, tol: float, k_max: int, fixed_k: int = 0, reorth: bool = False):
    """Columns propagated independently; returns (result, ks, eps)."""
    out = np.empty_like(psi)
    ks, eps = [], []
    mv = (lambda v: Hbar @ v) if not callable(Hbar) else Hbar
    for col in range(psi.shape[1]):
        r, k, e, _ = expm_column(mv, psi[:, col], dt, tol, k_max, fixed_k, reorth)
        out[:, col] = r
        ks.append(k)
        eps.append(e)
    return out, np.asarray(ks), np.asarray(eps)
