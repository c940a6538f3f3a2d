"""Parity of the optional pieces of the CUDA path with the oracle: the
Perdew-Zunger functional and the potential-extrapolation Magnus step."""
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


WORKLOADS = {
    "h2": lambda: W.h2(),
    "small2_p3": lambda: W.small_cluster(n_atoms=2, cells_per_axis=5, degree=3, n_quad=5, n_orb=3),
    "small1_p2_batch2": lambda: W.small_cluster(n_atoms=1, cells_per_axis=3, degree=2, n_quad=4, L=10.0, n_orb=2,
                                                batch=2),
}


def _oracle_run(S, wl, psi0, n_steps, fixed_k, scheme, xc_kind):
    from oracle import tdks
    psi = tdks.kick(S, psi0, wl.fields, wl.n_orb, tol=1e-14, k_max=fixed_k)
    st = tdks.make_state(S, psi, wl.occ, wl.batch, xc_kind)
    vN = tdks.nuclear_potential(S)
    mus = []
    for n in range(n_steps):
        psi, st, mu, _ = tdks.magnus_step(S, psi, st, n * wl.dt, wl.dt, wl.fields, wl.occ, 1e-14, fixed_k,
                                          fixed_k=fixed_k, vN=vN, scheme=scheme, xc_kind=xc_kind)
        mus.append(mu)
    return psi, np.array(mus)


def _gpu_run(wl, psi0, n_steps, fixed_k, scheme, xc):
    from paper_2210_14421_gb300 import Context
    ctx = Context(wl, fixed_k=fixed_k, krylov_tol=1e-14, k_max=fixed_k, cg_tol=1e-14, cg_max_it=20000, xc=xc,
                  scheme=scheme)
    psi = _dev(psi0)
    ctx.kick(psi, wl.fields)
    mu = torch.zeros((wl.batch, 3), dtype=torch.float64, device="cuda")
    mus, infos = [], []
    for n in range(n_steps):
        infos.append(ctx.magnus_step(psi, n * wl.dt, wl.dt, wl.fields, mu))
        mus.append(mu.cpu().numpy().copy())
    return psi.cpu().numpy(), np.array(mus), infos


def test_lda_pz81_matches_oracle():
    """v_xc and eps_xc of the PZ81 option against the oracle's formula on the
    same density, point by point."""
    from oracle import operators, xc
    from paper_2210_14421_gb300 import EFE_XC_PZ81, Context
    wl = WORKLOADS["small2_p3"]()
    S = operators.System(wl)
    ctx = Context(wl, xc=EFE_XC_PZ81)
    psi = _dev(S.initial_orbitals())
    shape = (1, S.mesh.n_cells, S.mesh.nq)
    rho, vxc, exc = (torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(3))
    ctx.density_vxc(psi, rho, vxc, exc)
    r = rho.cpu().numpy()
    e_ref, v_ref = xc.lda(r, "pz81")
    assert np.max(np.abs(vxc.cpu().numpy() - v_ref)) <= 1e-13 * np.max(np.abs(v_ref))
    assert np.max(np.abs(exc.cpu().numpy() - e_ref)) <= 1e-13 * np.max(np.abs(e_ref))
    # both branches of the fit are exercised
    rs = np.cbrt(3.0 / (4.0 * np.pi * r[r > 1e-14]))
    assert rs.min() < 1.0 < rs.max()


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_extrapolated_scheme_matches_oracle(name):
    """Kick + 4 steps of the potential-extrapolation scheme (the first one
    predictor-corrector) with a fixed Krylov dimension: orbitals and dipoles to
    relative 1e-10; the later steps take a single exponential."""
    from oracle import operators
    from paper_2210_14421_gb300 import EFE_STEP_EXTRAPOLATED, EFE_XC_PW92
    wl = WORKLOADS[name]()
    S = operators.System(wl)
    psi0 = np.tile(S.initial_orbitals(), (1, wl.batch))
    ref_psi, ref_mu = _oracle_run(S, wl, psi0, 4, 8, "extrapolated", "pw92")
    got_psi, got_mu, infos = _gpu_run(wl, psi0, 4, 8, EFE_STEP_EXTRAPOLATED, EFE_XC_PW92)
    assert np.linalg.norm(got_psi - ref_psi) <= 1e-10 * np.linalg.norm(ref_psi)
    assert np.max(np.abs(got_psi - ref_psi)) <= 1e-10 * np.max(np.abs(ref_psi))   # element-wise
    assert np.max(np.abs(got_mu - ref_mu)) <= 1e-10 * max(np.max(np.abs(ref_mu)), 1e-3)
    assert infos[0]["k_pred"] == 8 and all(i["k_pred"] == 0 for i in infos[1:])


def test_pz81_steps_match_oracle():
    from oracle import operators
    from paper_2210_14421_gb300 import EFE_STEP_PC, EFE_XC_PZ81
    wl = WORKLOADS["small2_p3"]()
    S = operators.System(wl)
    psi0 = S.initial_orbitals()
    ref_psi, ref_mu = _oracle_run(S, wl, psi0, 3, 8, "pc", "pz81")
    got_psi, got_mu, _ = _gpu_run(wl, psi0, 3, 8, EFE_STEP_PC, EFE_XC_PZ81)
    assert np.linalg.norm(got_psi - ref_psi) <= 1e-10 * np.linalg.norm(ref_psi)
    assert np.max(np.abs(got_psi - ref_psi)) <= 1e-10 * np.max(np.abs(ref_psi))   # element-wise
    assert np.max(np.abs(got_mu - ref_mu)) <= 1e-10 * max(np.max(np.abs(ref_mu)), 1e-3)


def test_reset_state_restarts_the_history():
    """After efe_reset_state the extrapolation scheme takes a predictor-corrector
    step again (it has no v_Hxc of a previous step)."""
    from paper_2210_14421_gb300 import EFE_STEP_EXTRAPOLATED, Context
    wl = WORKLOADS["h2"]()
    from oracle import operators
    S = operators.System(wl)
    ctx = Context(wl, krylov_tol=1e-12, k_max=16, scheme=EFE_STEP_EXTRAPOLATED)
    psi = _dev(S.initial_orbitals())
    mu = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    ks = [ctx.magnus_step(psi, n * wl.dt, wl.dt, wl.fields, mu)["k_pred"] for n in range(3)]
    ctx.reset_state()
    ks.append(ctx.magnus_step(psi, 3 * wl.dt, wl.dt, wl.fields, mu)["k_pred"])
    assert ks[0] > 0 and ks[1] == 0 and ks[2] == 0 and ks[3] > 0


def test_adjoint_rejects_other_functional_and_scheme():
    from paper_2210_14421_gb300 import EFE_STEP_EXTRAPOLATED, EFE_XC_PZ81, Context, EfeError
    wl = W.small_cluster(n_atoms=1, cells_per_axis=3, degree=2, n_quad=4, L=10.0, n_orb=1, Zval=2.0)
    f = W.Field(kind=W.FIELD_GAUSS, amp=0.02, t0=0.1, sigma=0.1, direction=(1.0, 0.0, 0.0))
    for kw in ({"xc": EFE_XC_PZ81}, {"scheme": EFE_STEP_EXTRAPOLATED}):
        ctx = Context(wl, **kw)
        psi = torch.zeros((ctx.n_dof, 1), dtype=torch.complex128, device="cuda")
        ctx.init_orbitals(psi)
        with pytest.raises(EfeError):
            ctx.adjoint_dipole(psi, 3, 0.05, f, (1.0, 0.0, 0.0), (2, 3))
