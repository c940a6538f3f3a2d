"""Atom-centred enrichment functions, Eq. EFEAtomic.

Test infrastructure only (see `oracle/__init__.py`).

N^A_nu(x) = f(r) * S_lm(x - R_I) * u(r; r0, s), r = |x - R_I|, where
S_lm is a real solid harmonic (r^l times a real spherical harmonic, without
normalisation: the overlap block M^ee absorbs any constant factor) and
f = R_nl / r^l is the radial shape divided by r^l.

Readings (the paper defers the cutoff and the atomic orbitals to its
references):
* cutoff u: 1 for r <= r0 - s, 0 for r >= r0, and 1 - S(t) in between with
  t = (r - r0 + s) / s and the C-infinity step S(t) = g(t) / (g(t) + g(1-t)),
  g(t) = exp(-1/t);
* radial shapes: Slater r^(n-1) e^(-zeta r), hydrogen-like R_nl(zeta r) built
  from the generalised Laguerre polynomial, or a Gaussian r^l e^(-zeta r^2).
"""
from __future__ import annotations

import math

import numpy as np

RADIAL_SLATER = 0
RADIAL_HYDROGENIC = 1
RADIAL_GAUSSIAN = 2


def _laguerre(k: int, a: int, x: np.ndarray) -> np.ndarray:
    """Generalised Laguerre polynomial L_k^(a)(x) = sum_i (-1)^i C(k+a, k-i) x^i / i!."""
    out = np.zeros_like(x)
    for i in range(k + 1):
        out += (-1) ** i * math.comb(k + a, k - i) * x ** i / math.factorial(i)
    return out


def radial(kind: int, n: int, l: int, zeta: float, r: np.ndarray):
    """f(r) = R_nl(r) / r^l and its derivative df/dr."""
    r = np.asarray(r, dtype=np.float64)
    if kind == RADIAL_SLATER:
        e = n - 1 - l
        if e < 0:
            raise ValueError("Slater function needs n - 1 >= l")
        f = r ** e * np.exp(-zeta * r)
        df = (e * r ** (e - 1) if e > 0 else 0.0) * np.exp(-zeta * r) - zeta * f
        return f, df
    if kind == RADIAL_HYDROGENIC:
        k = n - l - 1
        if k < 0:
            raise ValueError("hydrogen-like function needs n > l")
        x = 2.0 * zeta * r / n
        Lk = _laguerre(k, 2 * l + 1, x)
        dLk = -_laguerre(k - 1, 2 * l + 2, x) if k >= 1 else np.zeros_like(x)
        ex = np.exp(-zeta * r / n)
        f = zeta ** l * Lk * ex
        df = zeta ** l * (dLk * (2.0 * zeta / n) - (zeta / n) * Lk) * ex
        return f, df
    if kind == RADIAL_GAUSSIAN:
        f = np.exp(-zeta * r * r)
        return f, -2.0 * zeta * r * f
    raise ValueError("unknown radial kind")


def solid_harmonic(l: int, m: int, d: np.ndarray):
    """Real solid harmonics S_lm(d) (unnormalised) and gradients, l <= 2.
    l = 1: m = -1, 0, 1 -> y, z, x.  l = 2: m = -2..2 -> xy, yz, 2z^2-x^2-y^2, xz, x^2-y^2."""
    x, y, z = d[:, 0], d[:, 1], d[:, 2]
    one, zero = np.ones_like(x), np.zeros_like(x)
    if l == 0:
        return one, np.stack([zero, zero, zero], axis=1)
    if l == 1:
        if m == -1:
            return y.copy(), np.stack([zero, one, zero], axis=1)
        if m == 0:
            return z.copy(), np.stack([zero, zero, one], axis=1)
        if m == 1:
            return x.copy(), np.stack([one, zero, zero], axis=1)
    if l == 2:
        if m == -2:
            return x * y, np.stack([y, x, zero], axis=1)
        if m == -1:
            return y * z, np.stack([zero, z, y], axis=1)
        if m == 0:
            return 2 * z * z - x * x - y * y, np.stack([-2 * x, -2 * y, 4 * z], axis=1)
        if m == 1:
            return x * z, np.stack([z, zero, x], axis=1)
        if m == 2:
            return x * x - y * y, np.stack([2 * x, -2 * y, zero], axis=1)
    raise ValueError("unsupported (l, m)")


def cutoff(r: np.ndarray, r0: float, s: float):
    """Smooth cutoff u(r; r0, s) and du/dr (reading stated in the module doc)."""
    r = np.asarray(r, dtype=np.float64)
    t = (r - (r0 - s)) / s
    u = np.where(t <= 0.0, 1.0, 0.0)
    du = np.zeros_like(r)
    mid = (t > 0.0) & (t < 1.0)
    tm = t[mid]
    g1 = np.exp(-1.0 / tm)
    g2 = np.exp(-1.0 / (1.0 - tm))
    S = g1 / (g1 + g2)
    dg1 = g1 / tm ** 2
    dg2 = g2 / (1.0 - tm) ** 2          # d/dt g(1 - t) = -g'(1-t); sign handled below
    dS = (dg1 * g2 + g1 * dg2) / (g1 + g2) ** 2
    u[mid] = 1.0 - S
    du[mid] = -dS / s
    return u, du


def evaluate(fn, center: np.ndarray, pts: np.ndarray, r0: float, s: float):
    """Values (npts,) and gradients (npts, 3) of one enrichment function."""
    d = pts - center[None, :]
    r = np.sqrt(np.sum(d * d, axis=1))
    f, df = radial(fn.radial, fn.n, fn.l, fn.zeta, r)
    S, dS = solid_harmonic(fn.l, fn.m, d)
    u, du = cutoff(r, r0, s)
    val = f * S * u
    with np.errstate(invalid="ignore", divide="ignore"):
        rhat = np.where(r[:, None] > 0.0, d / r[:, None], 0.0)
    grad = ((df * u + f * du) * S)[:, None] * rhat + (f * u)[:, None] * dS
    return val, grad
