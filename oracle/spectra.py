"""Spectra from dipole traces (Sec. Results: absorption spectrum of the
weak-perturbation study, power spectrum of the high-harmonic study).

Test infrastructure only (see `oracle/__init__.py`).

Samples f_n = f(t_n), t_n = n dt, n = 0..N.  Time integrals are the
trapezoid rule, F[f](w) = dt sum_n c_n f_n e^{i w t_n} with c_0 = c_N = 1/2,
c_n = 1 otherwise.

Absorption (readings: the printed formula divides by the field's transform
outside the trace; it is read as the division that defines alpha):
  alpha_jj(w) = F[g (mu_j^(j) - mu_j^(j)(0))](w) / F[E_0](w),   g(t) = e^{-t/tau}
  S(w)        = (4 w / (3 pi)) sum_j Im alpha_jj(w)
where mu^(j) is the dipole trace of the run perturbed along axis j; for a
delta kick of strength kappa, F[E_0] = kappa.

Power spectrum (reading: "d/dt^2" is the second derivative):
  P(w) = | dt sum_{n=1}^{N-1} e^{-i w t_n} a_n e^{-t_n^2 / tau} |^2,
  a_n  = (mu_{n+1} - 2 mu_n + mu_{n-1}) / dt^2
(central second differences at the interior samples, rectangle weights).
"""
from __future__ import annotations

import numpy as np


def trapezoid_weights(n_samples: int) -> np.ndarray:
    c = np.ones(n_samples)
    c[0] = c[-1] = 0.5
    return c


def fourier(f: np.ndarray, dt: float, omegas: np.ndarray, sign: float = +1.0) -> np.ndarray:
    """dt sum_n c_n f_n e^{sign i w t_n} for every w (f real, 1D)."""
    t = dt * np.arange(len(f))
    ph = np.exp(sign * 1j * np.outer(omegas, t))
    return dt * ph @ (trapezoid_weights(len(f)) * f)


def absorption_spectrum(mu: np.ndarray, dt: float, omegas: np.ndarray, tau: float, field=None, kick=None):
    """mu: (3, N + 1, 3) dipole traces, mu[j, n, :] for the run perturbed along j;
    field: (N + 1,) samples of E_0 (or kick = kappa for a delta kick)."""
    t = dt * np.arange(mu.shape[1])
    g = np.exp(-t / tau)
    FE = kick if field is None else fourier(np.asarray(field, dtype=np.float64), dt, omegas)
    S = np.zeros(len(omegas))
    for j in range(3):
        d = (mu[j, :, j] - mu[j, 0, j]) * g
        S += np.imag(fourier(d, dt, omegas) / FE)
    return 4.0 * omegas / (3.0 * np.pi) * S


def power_spectrum(mu_x: np.ndarray, dt: float, omegas: np.ndarray, tau: float) -> np.ndarray:
    mu_x = np.asarray(mu_x, dtype=np.float64)
    n = len(mu_x)
    t = dt * np.arange(n)
    a = np.zeros(n)
    a[1:-1] = (mu_x[2:] - 2.0 * mu_x[1:-1] + mu_x[:-2]) / dt ** 2
    w = a * np.exp(-t ** 2 / tau)
    F = dt * np.exp(-1j * np.outer(omegas, t)) @ w
    return np.abs(F) ** 2
