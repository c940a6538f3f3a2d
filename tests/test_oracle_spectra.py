"""Pins of the oracle's spectra: closed-form transforms, the oscillator
f-sum, and the power-spectrum peak of a pure harmonic."""
import numpy as np

from oracle import spectra


def test_fourier_of_damped_cosine_closed_form():
    """int_0^T e^{-t/tau} cos(w0 t) e^{i w t} dt in closed form, against the
    trapezoid sum (error O(dt^2))."""
    dt, T, tau, w0 = 0.005, 40.0, 8.0, 1.3
    t = np.arange(0.0, T + dt / 2, dt)
    f = np.exp(-t / tau) * np.cos(w0 * t)
    om = np.linspace(0.2, 3.0, 15)
    got = spectra.fourier(f, dt, om)

    def prim(a):   # int_0^T e^{a t} dt
        return (np.exp(a * T) - 1.0) / a
    ref = 0.5 * (prim(-1.0 / tau + 1j * (om + w0)) + prim(-1.0 / tau + 1j * (om - w0)))
    assert np.max(np.abs(got - ref)) < 1e-5 * np.max(np.abs(ref))


def test_absorption_of_an_oscillator_obeys_the_f_sum():
    """A kicked damped oscillator of strength f at w0 along each axis,
    mu_j(t) - mu_j(0) = kappa (f / w0) sin(w0 t) e^{-gamma t / 2}: S peaks at w0
    and int S dw = 2 f (the factor 4 / (3 pi), the trace over three axes and
    the sign of Im alpha all enter)."""
    dt, T, w0, f, gam, kappa = 0.02, 400.0, 0.8, 0.7, 0.02, 1e-3
    t = np.arange(0.0, T + dt / 2, dt)
    mu = np.zeros((3, len(t), 3))
    for j in range(3):
        mu[j, :, j] = 5.0 + kappa * (f / w0) * np.sin(w0 * t) * np.exp(-0.5 * gam * t)
    om = np.linspace(0.01, 3.0, 3000)
    S = spectra.absorption_spectrum(mu, dt, om, tau=1e9, kick=kappa)
    assert abs(om[np.argmax(S)] - w0) < 2e-3
    assert abs(np.trapezoid(S, om) / (2.0 * f) - 1.0) < 0.03
    # the same run described by its field samples: a delta of weight kappa at t = 0
    E = np.zeros(len(t))
    E[0] = 2.0 * kappa / dt
    S2 = spectra.absorption_spectrum(mu, dt, om, tau=1e9, field=E)
    assert np.max(np.abs(S2 - S)) < 1e-12 * np.max(np.abs(S))


def test_power_spectrum_of_a_harmonic():
    """mu = sin(W t): the acceleration is -W^2 sin(W t), so P peaks at W with
    height (W^2 T / 2)^2 up to the O(dt^2) second difference and O(1/T) edges."""
    dt, T, W = 0.01, 200.0, 2.0
    t = np.arange(0.0, T + dt / 2, dt)
    om = np.linspace(1.5, 2.5, 2001)
    P = spectra.power_spectrum(np.sin(W * t), dt, om, tau=1e12)
    assert abs(om[np.argmax(P)] - W) < 1e-3
    assert abs(P.max() / (W ** 2 * T / 2.0) ** 2 - 1.0) < 0.01
