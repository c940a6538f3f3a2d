"""The orbital partition through the C ABI (efe_set_density_reduce) on one GPU.

- one process: a reduction that leaves the density as it is gets called once per density the
  step forms and changes nothing (to the run-to-run rounding of the scatter's atomic adds);
- two ranks emulated by two host threads, each with its own context (half of the orbitals) and
  its own CUDA stream: the reduction copies the partial density to the host, meets the other
  thread at a barrier (with a time limit), adds the two partials in rank order and copies the
  sum back.  No kernel waits on another: only host threads wait.  The ranks' orbitals and
  dipoles equal one context's with all orbitals;
- an exception raised by the reduction ends the step and reaches the caller;
- the adjoint refuses a context with a reduction installed."""
import threading

import numpy as np
import pytest

import efe_workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N_STEPS = 3


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _wl():
    return W.small_cluster(n_atoms=2, cells_per_axis=4, degree=3, n_quad=5, n_orb=4, tol=1e-12, k_max=24)


def _sub(wl, cols):
    return wl.with_(n_orb=len(cols), occ=wl.occ[cols], orb_centers=wl.orb_centers[cols],
                    orb_exps=wl.orb_exps[cols], orb_coefs=wl.orb_coefs[cols], enr_coefs=wl.enr_coefs[cols])


def _psi0(wl):
    from oracle import operators
    return torch.from_numpy(np.ascontiguousarray(operators.System(wl).initial_orbitals())).cuda()


def _run(ctx, psi, wl, scheme_steps=N_STEPS):
    mu = torch.zeros((wl.batch, 3), dtype=torch.float64, device="cuda")
    ctx.kick(psi, wl.fields)
    mus = []
    for n in range(scheme_steps):
        ctx.magnus_step(psi, n * wl.dt, wl.dt, wl.fields, mu)
        mus.append(mu.cpu().numpy().copy())
    return np.array(mus)


@pytest.mark.parametrize("scheme", [0, 1])
def test_identity_reduction_is_called_per_density_and_changes_nothing(scheme):
    from paper_2210_14421_gb300 import Context
    wl = _wl()
    a = Context(wl, scheme=scheme, krylov_tol=1e-12)
    psi_a = _psi0(wl)
    mus_a = _run(a, psi_a, wl)
    a.close()

    calls = []
    b = Context(wl, scheme=scheme, krylov_tol=1e-12)
    b.set_density_reduce(lambda rho: calls.append(rho.numel()))
    psi_b = _psi0(wl)
    mus_b = _run(b, psi_b, wl)
    n = b.n_cells * b.n_q * wl.batch
    # the start's state density, then per step the predictor density (S2) and the new state's
    # (the extrapolated scheme forms no predictor density once it has a previous potential)
    expect = 1 + 2 * N_STEPS if scheme == 0 else 1 + 2 + (N_STEPS - 1)
    assert calls == [n] * expect
    # two runs differ only in the order of the scatter's atomic adds
    assert torch.max(torch.abs(psi_a - psi_b)).item() <= 1e-12 * torch.max(torch.abs(psi_a)).item()
    assert np.max(np.abs(mus_a - mus_b)) <= 1e-12 * max(np.max(np.abs(mus_a)), 1e-3)
    b.set_density_reduce(None)
    b.close()


class _HostAllReduce:
    """Sum over emulated ranks through host memory, in rank order."""

    def __init__(self, world):
        self.parts = [None] * world
        self.bar = threading.Barrier(world, timeout=120.0)

    def fn(self, rank):
        def reduce(rho):
            self.parts[rank] = rho.cpu()      # on the step's stream; waits for the density
            self.bar.wait()
            total = self.parts[0].clone()
            for p in self.parts[1:]:
                total += p
            self.bar.wait()                   # every rank has read every part
            rho.copy_(total.to(rho.device))
        return reduce


@pytest.mark.parametrize("scheme", [0, 1])
def test_two_emulated_ranks_match_one_context(scheme):
    from paper_2210_14421_gb300 import Context
    wl = _wl()
    full = Context(wl, scheme=scheme, krylov_tol=1e-12)
    psi_full = _psi0(wl)
    mus_full = _run(full, psi_full, wl)
    full.close()

    world = 2
    red = _HostAllReduce(world)
    splits = [np.arange(r, wl.n_orb, world) for r in range(world)]
    ctxs, psis, out, errs = [], [], [None] * world, []
    for r in range(world):
        sub = _sub(wl, splits[r])
        c = Context(sub, scheme=scheme, krylov_tol=1e-12)
        c.set_density_reduce(red.fn(r))
        ctxs.append(c)
        psis.append(_psi0(wl)[:, splits[r]].contiguous())
    torch.cuda.synchronize()

    def rank_main(r):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                out[r] = _run(ctxs[r], psis[r], _sub(wl, splits[r]))
                s.synchronize()
        except BaseException as e:   # noqa: BLE001
            errs.append(e)
            red.bar.abort()

    th = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=600)
    assert not errs, errs
    scale = torch.max(torch.abs(psi_full)).item()
    for r in range(world):
        assert torch.max(torch.abs(psis[r] - psi_full[:, splits[r]])).item() <= 1e-11 * scale
        assert np.max(np.abs(out[r] - mus_full)) <= 1e-11 * max(np.max(np.abs(mus_full)), 1e-3)
        ctxs[r].close()


def test_reduction_error_reaches_the_caller_and_adjoint_refuses():
    from paper_2210_14421_gb300 import Context, EfeError
    wl = _wl()
    ctx = Context(wl, krylov_tol=1e-12)
    psi = _psi0(wl)

    def broken(rho):
        raise RuntimeError("peer lost")

    ctx.set_density_reduce(broken)
    mu = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError, match="peer lost"):
        ctx.magnus_step(psi, 0.0, wl.dt, wl.fields, mu)
    ctx.set_density_reduce(lambda rho: None)
    with pytest.raises(EfeError, match="all orbitals"):
        ctx.adjoint_dipole(psi, 2, wl.dt, W.Field(kind=W.FIELD_GAUSS, amp=1e-3, t0=0.1, sigma=0.05,
                                                  direction=(1.0, 0.0, 0.0)), (1.0, 0.0, 0.0), (1, 2))
    ctx.set_density_reduce(None)
    ctx.reset_state()
    ctx.magnus_step(psi, 0.0, wl.dt, wl.fields, mu)    # usable again
    ctx.close()
