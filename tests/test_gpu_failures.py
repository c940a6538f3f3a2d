"""Failure statuses of the C ABI, made to happen on purpose without faulting the GPU, and the
forward checkpoint/resume file.

- EFE_ERR_CG_NOCONV: the Jacobi-PCG Hartree solve limited to one iteration;
- EFE_ERR_NOT_SPD: an enrichment function given twice makes M^ee singular at set-up;
- EFE_WARN_KRYLOV_CAP: a Krylov cap of 2 far below what the tolerance needs; the step is
  still taken (norms conserved);
- EFE_ERR_TIMEOUT: the tensor-core apply's progress waits limited to one poll give up; the
  kernel stops, drains its copies and MMAs and returns, the next step reports the status, and
  the context then reproduces a fresh context's step;
- checkpoint: a run saved after two steps and resumed in a new context takes the same next
  steps as the uninterrupted run; a damaged file or one of another context is refused."""
import numpy as np
import pytest

import efe_workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _wl(**kw):
    return W.small_cluster(n_atoms=2, cells_per_axis=4, degree=3, n_quad=5, n_orb=2, **kw)


def _psi0(wl):
    from oracle import operators
    return torch.from_numpy(np.ascontiguousarray(operators.System(wl).initial_orbitals())).cuda()


def _steps(ctx, psi, wl, n, t0=0.0):
    mu = torch.zeros((wl.batch, 3), dtype=torch.float64, device="cuda")
    mus = []
    for k in range(n):
        ctx.magnus_step(psi, t0 + k * wl.dt, wl.dt, wl.fields, mu)
        mus.append(mu.cpu().numpy().copy())
    return np.array(mus)


def test_cg_nonconvergence_is_reported():
    from paper_2210_14421_gb300 import EFE_HARTREE_PCG, Context, EfeError
    wl = _wl()
    ctx = Context(wl, hartree_method=EFE_HARTREE_PCG, cg_tol=1e-14, cg_max_it=1)
    psi = _psi0(wl)
    with pytest.raises(EfeError, match="EFE_ERR_CG_NOCONV"):
        _steps(ctx, psi, wl, 1)
    rho = torch.empty((1, ctx.n_cells, ctx.n_q), dtype=torch.float64, device="cuda")
    vH = torch.empty_like(rho)
    ctx.density_vxc(psi, rho)
    with pytest.raises(EfeError, match="EFE_ERR_CG_NOCONV"):
        ctx.hartree(rho, vH, tol=1e-14, max_it=1)
    assert ctx.hartree(rho, vH, tol=1e-10, max_it=20000) > 1   # converges with room to iterate
    ctx.close()


def test_duplicate_enrichment_is_not_spd():
    from paper_2210_14421_gb300 import Context, EfeError
    wl = _wl()
    dup = wl.with_(enrich=wl.enrich + [wl.enrich[0]],
                   enr_coefs=np.concatenate([wl.enr_coefs, wl.enr_coefs[:, :1]], axis=1))
    with pytest.raises(EfeError, match="EFE_ERR_NOT_SPD"):
        Context(dup)
    Context(wl).close()   # the same set-up without the copy is fine


def test_krylov_cap_is_a_warning_and_the_step_is_taken():
    from paper_2210_14421_gb300 import Context
    from paper_2210_14421_gb300._binding import EFE_WARN_KRYLOV_CAP
    wl = _wl()
    ctx = Context(wl, k_max=2, krylov_tol=1e-14)
    psi = _psi0(wl)
    n0 = torch.linalg.norm(psi, dim=0)
    before = psi.clone()
    mu = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    info = ctx.magnus_step(psi, 0.0, wl.dt, wl.fields, mu)
    assert info["status"] == EFE_WARN_KRYLOV_CAP and info["cap"] > 0 and info["k_corr"] == 2
    assert torch.max(torch.abs(psi - before)).item() > 0.0                     # the step was taken
    assert torch.max(torch.abs(torch.linalg.norm(psi, dim=0) - n0)).item() < 1e-12 * n0.max().item()
    ctx.close()


def test_tensor_core_wait_timeout_is_reported_and_the_context_recovers():
    from paper_2210_14421_gb300 import EFE_TC, Context, EfeError
    wl = _wl(tol=1e-10)
    ref_ctx = Context(wl, precision=EFE_TC, krylov_tol=1e-10, k_max=16)
    ref = _psi0(wl)
    ref_ctx.kick(ref, wl.fields)
    mu_ref = _steps(ref_ctx, ref, wl, 1)
    ref_ctx.close()

    ctx = Context(wl, precision=EFE_TC, krylov_tol=1e-10, k_max=16)
    psi = _psi0(wl)
    ctx.kick(psi, wl.fields)
    ctx.set_wait_limit(1)
    with pytest.raises(EfeError, match="EFE_ERR_TIMEOUT"):
        _steps(ctx, psi, wl, 1)
    ctx.set_wait_limit(0)
    ctx.reset_state()
    psi = _psi0(wl)
    ctx.kick(psi, wl.fields)
    mu = _steps(ctx, psi, wl, 1)
    assert torch.max(torch.abs(psi - ref)).item() <= 1e-9 * torch.max(torch.abs(ref)).item()
    assert np.max(np.abs(mu - mu_ref)) <= 1e-9 * max(np.max(np.abs(mu_ref)), 1e-3)
    ctx.close()


@pytest.mark.parametrize("scheme", [0, 1])
def test_checkpoint_resume_reproduces_the_run(tmp_path, scheme):
    """Kick + 2 steps, save, 2 more steps; a new context loads the file and takes the same 2
    steps (the predictor-corrector and the extrapolated scheme, whose next step needs the
    previous v_Hxc from the file)."""
    from paper_2210_14421_gb300 import Context, EfeError
    wl = _wl(tol=1e-12)
    path = tmp_path / "run.ckpt"
    a = Context(wl, scheme=scheme, krylov_tol=1e-12)
    psi = _psi0(wl)
    a.kick(psi, wl.fields)
    _steps(a, psi, wl, 2)
    a.checkpoint_save(path, psi, 2 * wl.dt, 2)
    mu_a = _steps(a, psi, wl, 2, t0=2 * wl.dt)
    psi_a = psi.clone()
    a.close()

    b = Context(wl, scheme=scheme, krylov_tol=1e-12)
    psi_b = torch.zeros_like(psi_a)
    t, step = b.checkpoint_load(path, psi_b)
    assert (t, step) == (2 * wl.dt, 2)
    mu_b = _steps(b, psi_b, wl, 2, t0=t)
    assert torch.max(torch.abs(psi_b - psi_a)).item() <= 1e-12 * torch.max(torch.abs(psi_a)).item()
    assert np.max(np.abs(mu_b - mu_a)) <= 1e-12 * max(np.max(np.abs(mu_a)), 1e-3)
    b.close()

    raw = path.read_bytes()
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(raw[:200] + bytes([raw[200] ^ 1]) + raw[201:])
    c = Context(wl, scheme=scheme)
    with pytest.raises(EfeError, match="checksum"):
        c.checkpoint_load(bad, psi_b)
    c.close()
    other = _wl(tol=1e-12).with_(n_orb=1, occ=np.array([2.0]), orb_centers=wl.orb_centers[:1],
                                 orb_exps=wl.orb_exps[:1], orb_coefs=wl.orb_coefs[:1], enr_coefs=wl.enr_coefs[:1])
    d = Context(other)
    with pytest.raises(EfeError, match="other sizes"):
        d.checkpoint_load(path, torch.zeros((d.n_dof, 1), dtype=torch.complex128, device="cuda"))
    d.close()
