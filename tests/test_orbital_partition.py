"""The orbital (column) partition of the step across processes, on CPU with the gloo backend
and two ranks: each rank owns half of the orbitals, propagates them through the step, and sums
every density it forms over the ranks (one all-reduce of rho_q per density: the state density
and the predictor density of S2) before LDA, the Hartree solve (replicated) and the dipole.
The ranks' orbitals and dipoles must equal the single-process step's, which holds because the
density is a sum over orbitals and each orbital's Krylov exponential is independent of the
others (Section 4.2).  A reduction left out (each rank using its own partial density) must
show, so the comparison can see a missing all-reduce."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

N_STEPS = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    import efe_workloads as W
    return W.small_cluster(n_atoms=2, cells_per_axis=3, degree=2, n_quad=4, n_orb=4, tol=1e-12, k_max=20)


def _run(wl, cols, scheme, reduce):
    """Kick + N_STEPS steps of the orbitals `cols` of the case; returns (psi, mus, n_reduce)."""
    from oracle import operators, tdks
    S = operators.System(wl)
    psi = S.initial_orbitals()[:, cols]
    occ = wl.occ[cols]
    calls = [0]

    def red(rho):
        calls[0] += 1
        return rho if reduce is None else reduce(rho)

    psi = tdks.kick(S, psi, wl.fields, len(occ))
    st = tdks.make_state(S, psi, occ, 1, reduce=red)
    mus = []
    for n in range(N_STEPS):
        psi, st, mu, _ = tdks.magnus_step(S, psi, st, n * wl.dt, wl.dt, wl.fields, occ, wl.krylov_tol, wl.k_max,
                                          scheme=scheme, reduce=red)
        mus.append(mu)
    return psi, np.array(mus), calls[0]


def _allreduce(rho):
    t = torch.from_numpy(np.ascontiguousarray(rho, dtype=np.float64))
    dist.all_reduce(t)
    return t.numpy()


def _rank_main(rank, world, port, scheme, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        wl = _case()
        cols = np.arange(rank, wl.n_orb, world)          # a strided split: ranks hold unequal orbitals
        psi, mus, calls = _run(wl, cols, scheme, _allreduce)
        out.put((rank, cols, psi, mus, calls))
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("scheme", ["pc", "extrapolated"])
def test_two_rank_orbital_partition_matches_one_process(scheme):
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, scheme, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=600) for _ in range(world)), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0

    wl = _case()
    psi_ref, mus_ref, calls_ref = _run(wl, np.arange(wl.n_orb), scheme, None)
    # one reduction per density: the state density of the start and of every step, and the
    # predictor density of S2 (the extrapolated scheme has none after its first step)
    expect = 1 + N_STEPS * 2 if scheme == "pc" else 1 + 2 + (N_STEPS - 1)
    scale = np.max(np.abs(psi_ref))
    for rank, cols, psi, mus, calls in res:
        assert calls == calls_ref == expect
        assert np.max(np.abs(psi - psi_ref[:, cols])) <= 1e-12 * scale
        assert np.max(np.abs(mus - mus_ref)) <= 1e-12 * max(np.max(np.abs(mus_ref)), 1e-3)


def test_a_missing_density_reduction_is_seen():
    """Each half propagated with its own partial density (no all-reduce) is a different
    step: the comparison above would fail."""
    wl = _case()
    psi_ref, mus_ref, _ = _run(wl, np.arange(wl.n_orb), "pc", None)
    cols = np.arange(0, wl.n_orb, 2)
    psi, mus, _ = _run(wl, cols, "pc", None)
    assert np.max(np.abs(psi - psi_ref[:, cols])) > 1e-9 * np.max(np.abs(psi_ref))
    assert np.max(np.abs(mus - mus_ref)) > 1e-6
