"""The per-step JSON-lines log (host logic, no device): one parseable line per step with the
step's statistics, the dipole per batch member and the wall time; `propagate` drives a context
and logs every step."""
import io
import json

import numpy as np

from paper_2210_14421_gb300.steplog import StepLog, propagate


class _FakeContext:
    """Stands in for Context.magnus_step: writes a dipole and returns step statistics."""

    def __init__(self):
        self.calls = []

    def magnus_step(self, psi, t, dt, fields, mu=None):
        self.calls.append((t, dt))
        psi *= 1.0
        mu[:] = np.array([[t, 2.0 * t, 3.0 * t]])
        return {"k_pred": 12, "k_corr": 13, "cap": 0, "cg_iters": 1, "eps_max": 3.5e-8, "substeps": 1, "status": 0}


def test_record_writes_one_json_line(tmp_path):
    p = tmp_path / "steps.jsonl"
    with StepLog(p) as log:
        log.record(1, 0.05, {"k_pred": 9, "k_corr": 10, "cap": 1, "eps_max": 2e-7, "status": 5},
                   mu=np.array([[1.0, 0.0, -2.0], [0.5, 0.5, 0.5]]), ms=12.5, note="x")
        log.record(2, 0.10, {"k_pred": 8})
    lines = [json.loads(l) for l in p.read_text().splitlines()]
    assert len(lines) == 2
    assert lines[0] == {"step": 1, "t": 0.05, "k_pred": 9, "k_corr": 10, "cap": 1, "eps_max": 2e-7, "status": 5,
                        "mu": [[1.0, 0.0, -2.0], [0.5, 0.5, 0.5]], "ms": 12.5, "note": "x"}
    assert lines[1] == {"step": 2, "t": 0.1, "k_pred": 8}


def test_propagate_logs_every_step():
    ctx, buf = _FakeContext(), io.StringIO()
    psi, mu = np.ones((4, 2)), np.zeros((1, 3))
    infos = propagate(ctx, psi, 3, 0.05, fields=None, mu=mu, log=StepLog(buf), t0=1.0, first_step=10)
    assert len(infos) == 3 and [c[0] for c in ctx.calls] == [1.0, 1.05, 1.1]
    lines = [json.loads(l) for l in buf.getvalue().splitlines()]
    assert [l["step"] for l in lines] == [11, 12, 13]
    assert np.allclose([l["t"] for l in lines], [1.05, 1.1, 1.15])
    # the dipole a step wrote is the one its line carries
    assert np.allclose(lines[2]["mu"], [[1.1, 2.2, 3.3]])
    assert all(l["k_corr"] == 13 and l["ms"] >= 0.0 for l in lines)


def test_dipole_given_as_nested_lists_or_one_member():
    buf = io.StringIO()
    log = StepLog(buf)
    assert log.record(1, 0.0, {}, mu=[[1, 2, 3]])["mu"] == [[1.0, 2.0, 3.0]]
    assert log.record(2, 0.0, {}, mu=np.array([4.0, 5.0, 6.0]))["mu"] == [[4.0, 5.0, 6.0]]
