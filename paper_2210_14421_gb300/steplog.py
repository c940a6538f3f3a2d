"""Per-step metrics of a propagation as JSON lines.

One line per Magnus step (Eq. ApproxMagnus): the step index and time, the largest Lanczos
dimension of the predictor and of the corrector exponential (Eq. AdaptiveKrylov), the columns
that reached k_max, the largest error estimate (Eq. AdaptiveKrylovErr), the Krylov sub-steps,
the Hartree CG iterations, the library's status, the dipole of each batch member and the
step's host wall time.  The numbers come from `Context.magnus_step` (its `efe_step_info`) and
from the dipole the step wrote; nothing here computes on the orbitals.
"""
from __future__ import annotations

import json
import time

import numpy as np


class StepLog:
    """Appends one JSON object per step to `path` (or to an open text stream)."""

    KEYS = ("k_pred", "k_corr", "cap", "cg_iters", "eps_max", "substeps", "status")

    def __init__(self, path_or_stream, flush_every: int = 1):
        if hasattr(path_or_stream, "write"):
            self._f, self._own = path_or_stream, False
        else:
            self._f, self._own = open(path_or_stream, "a", encoding="utf-8"), True
        self.flush_every = max(1, int(flush_every))
        self.n = 0

    def record(self, step: int, t: float, info: dict, mu=None, ms: float | None = None, **extra):
        """Writes the line of one step.  info: the dict `Context.magnus_step` returns; mu: the
        dipole [batch][3] (a host array, a device tensor or None); ms: the step's wall time."""
        line = {"step": int(step), "t": float(t)}
        for k in self.KEYS:
            if k in info:
                v = info[k]
                line[k] = float(v) if k == "eps_max" else int(v)
        if mu is not None:
            if hasattr(mu, "detach"):
                mu = mu.detach().cpu().numpy()
            line["mu"] = np.asarray(mu, dtype=np.float64).reshape(-1, 3).tolist()
        if ms is not None:
            line["ms"] = float(ms)
        line.update(extra)
        self._f.write(json.dumps(line) + "\n")
        self.n += 1
        if self.n % self.flush_every == 0:
            self._f.flush()
        return line

    def close(self):
        if self._own and not self._f.closed:
            self._f.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def propagate(ctx, psi, n_steps: int, dt: float, fields, mu, log: StepLog | None = None, t0: float = 0.0,
              first_step: int = 0):
    """n_steps Magnus steps of `psi` in place from t0; mu ([batch][3] on the device) receives
    each step's dipole.  With `log`, one line per step.  Returns the infos of the steps."""
    infos = []
    for n in range(n_steps):
        t = t0 + n * dt
        w0 = time.perf_counter()
        info = ctx.magnus_step(psi, t, dt, fields, mu)   # synchronises: info is host-visible
        ms = 1000.0 * (time.perf_counter() - w0)
        infos.append(info)
        if log is not None:
            log.record(first_step + n + 1, t + dt, info, mu, ms)
    return infos
