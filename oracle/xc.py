"""Adiabatic local-density exchange-correlation (Sec. "Time dependent Kohn-Sham
equations").

Test infrastructure only (see `oracle/__init__.py`).

Reading: the paper names the Ceperley-Alder form; the workloads fix Slater
exchange plus the Perdew-Wang 1992 (PW92) parametrisation of the
unpolarised correlation energy, which is what is written here:

  eps_x = -(3/4) (3 rho / pi)^(1/3),       v_x = (4/3) eps_x
  r_s   = (3 / (4 pi rho))^(1/3)
  eps_c = -2A (1 + a1 r_s) ln(1 + 1 / (2A (b1 r_s^1/2 + b2 r_s + b3 r_s^3/2 + b4 r_s^2)))
  v_c   = eps_c - (r_s / 3) d eps_c / d r_s

with A = 0.031091, a1 = 0.21370, b1..b4 = 7.5957, 3.5876, 1.6382, 0.49294
(Perdew & Wang, Phys. Rev. B 45, 13244 (1992), Table I, unpolarised column).
Below rho = 1e-14 both the energy and the potential are set to zero.

The paper's own functional, Ceperley-Alder correlation, is available as the
Perdew-Zunger 1981 parametrisation (Phys. Rev. B 23, 5048 (1981), unpolarised
fit to the Ceperley-Alder data), kind "pz81":
  r_s >= 1: eps_c = g / (1 + b1 r_s^1/2 + b2 r_s),  g = -0.1423, b1 = 1.0529, b2 = 0.3334
  r_s <  1: eps_c = A ln r_s + B + C r_s ln r_s + D r_s,
            A = 0.0311, B = -0.048, C = 0.0020, D = -0.0116
with v_c = eps_c - (r_s / 3) d eps_c / d r_s from the same expressions.
"""
from __future__ import annotations

import numpy as np

PW92_A = 0.031091
PW92_ALPHA1 = 0.21370
PW92_BETA = (7.5957, 3.5876, 1.6382, 0.49294)
RHO_FLOOR = 1e-14
PZ81_LOW = (-0.1423, 1.0529, 0.3334)              # gamma, beta1, beta2 (r_s >= 1)
PZ81_HIGH = (0.0311, -0.048, 0.0020, -0.0116)     # A, B, C, D (r_s < 1)


def slater_exchange(rho: np.ndarray):
    rho = np.asarray(rho, dtype=np.float64)
    ok = rho > RHO_FLOOR
    r = np.where(ok, rho, 1.0)
    ex = -0.75 * np.cbrt(3.0 * r / np.pi)
    vx = -np.cbrt(3.0 * r / np.pi)
    return np.where(ok, ex, 0.0), np.where(ok, vx, 0.0)


def pw92_eps_c(rs: np.ndarray):
    """PW92 eps_c(r_s) and d eps_c / d r_s."""
    A, a1 = PW92_A, PW92_ALPHA1
    b1, b2, b3, b4 = PW92_BETA
    srs = np.sqrt(rs)
    Q = 2.0 * A * (b1 * srs + b2 * rs + b3 * rs * srs + b4 * rs * rs)
    dQ = 2.0 * A * (0.5 * b1 / srs + b2 + 1.5 * b3 * srs + 2.0 * b4 * rs)
    lg = np.log1p(1.0 / Q)
    ec = -2.0 * A * (1.0 + a1 * rs) * lg
    dec = -2.0 * A * a1 * lg + 2.0 * A * (1.0 + a1 * rs) * dQ / (Q * (Q + 1.0))
    return ec, dec


def pw92_correlation(rho: np.ndarray):
    rho = np.asarray(rho, dtype=np.float64)
    ok = rho > RHO_FLOOR
    r = np.where(ok, rho, 1.0)
    rs = np.cbrt(3.0 / (4.0 * np.pi * r))
    ec, dec = pw92_eps_c(rs)
    vc = ec - rs / 3.0 * dec
    return np.where(ok, ec, 0.0), np.where(ok, vc, 0.0)


def pz81_eps_c(rs: np.ndarray):
    """Perdew-Zunger eps_c(r_s) and d eps_c / d r_s, branch by branch."""
    g, b1, b2 = PZ81_LOW
    A, B, C, D = PZ81_HIGH
    rs = np.asarray(rs, dtype=np.float64)
    srs = np.sqrt(rs)
    den = 1.0 + b1 * srs + b2 * rs
    e_lo = g / den
    de_lo = -g * (0.5 * b1 / srs + b2) / den ** 2
    lr = np.log(rs)
    e_hi = A * lr + B + C * rs * lr + D * rs
    de_hi = A / rs + C * (lr + 1.0) + D
    lo = rs >= 1.0
    return np.where(lo, e_lo, e_hi), np.where(lo, de_lo, de_hi)


def pz81_correlation(rho: np.ndarray):
    rho = np.asarray(rho, dtype=np.float64)
    ok = rho > RHO_FLOOR
    r = np.where(ok, rho, 1.0)
    rs = np.cbrt(3.0 / (4.0 * np.pi * r))
    ec, dec = pz81_eps_c(rs)
    vc = ec - rs / 3.0 * dec
    return np.where(ok, ec, 0.0), np.where(ok, vc, 0.0)


XC_KINDS = {"pw92": pw92_correlation, "pz81": pz81_correlation}


def lda(rho: np.ndarray, kind: str = "pw92"):
    """(eps_xc, v_xc) at every point: Slater exchange plus the correlation `kind`."""
    ex, vx = slater_exchange(rho)
    ec, vc = XC_KINDS[kind](rho)
    return ex + ec, vx + vc
