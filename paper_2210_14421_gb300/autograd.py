"""torch.autograd wrapper of efe_adjoint_dipole: the window-averaged dipole
J(amp, omega, sigma) of a field-driven propagation as a differentiable
function of the three field parameters.

The forward call runs the library's forward sweep and its reverse sweep
together (the reverse sweep needs the forward's checkpoints), so backward only
scales the stored gradient.  Both run in the CUDA library; nothing here
computes."""
from __future__ import annotations

import types

import torch


def _field_with(field, theta):
    amp, omega, sigma = (float(x) for x in theta)
    keys = ("kind", "amp", "omega", "t0", "sigma", "period", "ramp", "direction", "kick")
    d = {k: getattr(field, k, 0.0) for k in keys}
    d.update(amp=amp, omega=omega, sigma=sigma)
    return types.SimpleNamespace(**d)


class WindowedDipole(torch.autograd.Function):
    """J = (1/|W|) sum_{n in W} d . mu(rho_n) after propagating psi0 under the
    field with parameters theta = (amp, omega, sigma); dJ/dtheta by the adjoint."""

    @staticmethod
    def forward(ctx, theta, context, psi0, field, n_steps, dt, direction, window, checkpoint_every=4, n_quad_s=8):
        th = theta.detach().to("cpu", torch.float64)
        J, g = context.adjoint_dipole(psi0, n_steps, dt, _field_with(field, th.tolist()), direction, window,
                                      checkpoint_every, n_quad_s)
        ctx.save_for_backward(torch.as_tensor(g, dtype=theta.dtype, device=theta.device))
        return theta.new_tensor(J)

    @staticmethod
    def backward(ctx, gJ):
        (g,) = ctx.saved_tensors
        return (gJ * g,) + (None,) * 9


def windowed_dipole(theta, context, psi0, field, n_steps, dt, direction, window, checkpoint_every=4, n_quad_s=8):
    return WindowedDipole.apply(theta, context, psi0, field, n_steps, dt, direction, window, checkpoint_every,
                                n_quad_s)
