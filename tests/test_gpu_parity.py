"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same
seeded inputs.  FP64 results must agree to relative 1e-10 (orbitals, dipole)
or to a rounding bound (single applies); the mixed path is held to the error
stated in the test."""
import numpy as np
import pytest

import efe_workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module", autouse=True)
def _built():
    _require_gpu()
    import __graft_entry__ as g
    g.build()


def _ctx(wl, **kw):
    from paper_2210_14421_gb300 import Context
    return Context(wl, **kw)


def _sys(wl):
    from oracle import operators
    return operators.System(wl)


def _to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


WORKLOADS = {
    "h2": lambda: W.h2(),
    "small2_p3": lambda: W.small_cluster(n_atoms=2, cells_per_axis=5, degree=3, n_quad=5, n_orb=3),
    "small1_p2_11orb": lambda: W.small_cluster(n_atoms=1, cells_per_axis=3, degree=2, n_quad=4, L=10.0, n_orb=11),
    "small2_p5": lambda: W.small_cluster(n_atoms=2, cells_per_axis=3, degree=5, n_quad=7, n_orb=2, L=12.0),
}


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_geometry_and_initial_state(name):
    wl = WORKLOADS[name]()
    S = _sys(wl)
    ctx = _ctx(wl)
    assert ctx.n_nodes == S.n_h and ctx.n_enrich == S.n_E and ctx.n_cells == S.mesh.n_cells
    nodes, quad = ctx.coords()
    assert np.allclose(nodes.cpu().numpy(), S.mesh.nodes, rtol=0, atol=1e-13)
    assert np.allclose(quad.cpu().numpy(), S.mesh.xq, rtol=0, atol=1e-13)
    psi = torch.zeros((ctx.n_dof, ctx.n_cols), dtype=torch.complex128, device="cuda")
    ctx.init_orbitals(psi)
    ref = S.initial_orbitals()
    got = psi.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_integer_pipe_conversions_match_hardware():
    from paper_2210_14421_gb300 import _binding
    assert _binding.selftest(1 << 24) == 0


def _rounding_bound(H, X):
    return abs(H) @ np.abs(X)


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_apply_H_fp64_matches_oracle(name):
    """Y = Hbar X against the oracle's assembled P^T H P, element by element,
    within 1e-12 of the rounding scale sum_j |Hbar_ij| |X_j|."""
    wl = WORKLOADS[name]()
    S = _sys(wl)
    from oracle import tdks
    rng = np.random.default_rng(7)
    vq = tdks.nuclear_potential(S) + 0.05 * np.sum(S.mesh.xq ** 2, axis=2)
    H = S.hbar(vq)
    ncols = wl.n_orb
    X = rng.normal(size=(S.n_dof, ncols)) + 1j * rng.normal(size=(S.n_dof, ncols))
    X[:S.n_h][S.mesh.boundary] = 0.0
    ref = H @ X
    ctx = _ctx(wl)
    ctx.set_potential(_to_dev(vq[None]))
    Xd = _to_dev(X)
    Yd = torch.empty_like(Xd)
    ctx.apply_H(Xd, Yd)
    got = Yd.cpu().numpy()
    bound = _rounding_bound(H, X)
    assert np.all(np.abs(got - ref) <= 1e-12 * bound + 1e-300)
    # mixed: float32 contraction; error within 2e-5 of the same scale
    from paper_2210_14421_gb300 import EFE_MIXED, EFE_PAIR
    ctx.apply_H(Xd, Yd, precision=EFE_MIXED)
    got32 = Yd.cpu().numpy()
    assert np.all(np.abs(got32 - ref) <= 2e-5 * bound + 1e-300)
    # float32 pairs: error-free products and sums, ~2^-44 per operation
    ctx.apply_H(Xd, Yd, precision=EFE_PAIR)
    gotp = Yd.cpu().numpy()
    assert np.all(np.abs(gotp - ref) <= 1e-11 * bound + 1e-300)


def test_apply_H_batched_potentials():
    """Two batch members with different potentials in one apply."""
    wl = W.small_cluster(n_atoms=2, cells_per_axis=4, degree=3, n_quad=5, n_orb=3, batch=2)
    S = _sys(wl)
    from oracle import tdks
    v0 = tdks.nuclear_potential(S)
    v1 = v0 + 0.2 * S.mesh.xq[:, :, 0]
    rng = np.random.default_rng(3)
    X = rng.normal(size=(S.n_dof, 6)) + 1j * rng.normal(size=(S.n_dof, 6))
    X[:S.n_h][S.mesh.boundary] = 0.0
    ref = np.concatenate([S.hbar(v0) @ X[:, :3], S.hbar(v1) @ X[:, 3:]], axis=1)
    ctx = _ctx(wl)
    ctx.set_potential(_to_dev(np.stack([v0, v1])))
    Xd = _to_dev(X)
    Yd = torch.empty_like(Xd)
    ctx.apply_H(Xd, Yd)
    bound = np.concatenate([_rounding_bound(S.hbar(v0), X[:, :3]), _rounding_bound(S.hbar(v1), X[:, 3:])], axis=1)
    assert np.all(np.abs(Yd.cpu().numpy() - ref) <= 1e-12 * bound + 1e-300)


@pytest.mark.parametrize("name,method", [("h2", 0), ("small2_p3", 0), ("small1_p2_11orb", 0), ("h2", 1),
                                         ("small2_p3", 1)])
def test_density_lda_hartree_dipole(name, method):
    """Density, LDA, Hartree (method 0: fast diagonalisation, 1: Jacobi PCG)
    and dipole against the oracle's definitions (Hartree: sparse LU)."""
    wl = WORKLOADS[name]()
    S = _sys(wl)
    from oracle import poisson, tdks, xc
    ctx = _ctx(wl, cg_tol=1e-14, hartree_method=method)
    psi0 = S.initial_orbitals()
    psi = _to_dev(psi0)
    rho = torch.empty((1, S.mesh.n_cells, S.mesh.nq), dtype=torch.float64, device="cuda")
    vxc = torch.empty_like(rho)
    exc = torch.empty_like(rho)
    ctx.density_vxc(psi, rho, vxc, exc)
    rho_ref = tdks.density(S, psi0, wl.occ, 1)
    assert np.max(np.abs(rho.cpu().numpy() - rho_ref)) <= 1e-12 * np.max(rho_ref)
    e_ref, v_ref = xc.lda(rho_ref)
    assert np.allclose(vxc.cpu().numpy(), v_ref, rtol=1e-11, atol=1e-14)
    assert np.allclose(exc.cpu().numpy(), e_ref, rtol=1e-11, atol=1e-14)
    vH = torch.empty_like(rho)
    its = ctx.hartree(rho, vH, tol=1e-14, max_it=20000)
    assert its > 0
    _, vH_ref = poisson.solve(S, rho_ref[0])
    assert np.max(np.abs(vH.cpu().numpy()[0] - vH_ref)) <= 1e-10 * np.max(np.abs(vH_ref))
    mu = torch.empty((1, 3), dtype=torch.float64, device="cuda")
    ctx.dipole(rho, mu)
    mu_ref = tdks.dipole(S, rho_ref[0])
    assert np.allclose(mu.cpu().numpy()[0], mu_ref, rtol=1e-12, atol=1e-12)


def _oracle_run(S, wl, psi0, n_steps, fixed_k, tol, kmax, kick=True, reorth=False):
    from oracle import tdks
    psi = psi0
    if kick:
        psi = tdks.kick(S, psi, wl.fields, wl.n_orb, tol=tol, k_max=kmax)
    st = tdks.make_state(S, psi, wl.occ, wl.batch)
    mus = []
    vN = tdks.nuclear_potential(S)
    for n in range(n_steps):
        psi, st, mu, info = tdks.magnus_step(S, psi, st, n * wl.dt, wl.dt, wl.fields, wl.occ, tol, kmax,
                                             fixed_k=fixed_k, vN=vN, reorth=reorth)
        mus.append(mu)
    return psi, np.array(mus)


def _gpu_run(wl, psi0, n_steps, fixed_k, tol, kmax, precision=0, kick=True, use_graphs=False, krylov_block=0,
             krylov_substeps=1):
    ctx = _ctx(wl, precision=precision, fixed_k=fixed_k, krylov_tol=tol, k_max=kmax, cg_tol=1e-14, cg_max_it=20000,
               use_graphs=use_graphs, krylov_block=krylov_block, krylov_substeps=krylov_substeps)
    psi = _to_dev(psi0)
    if kick:
        ctx.kick(psi, wl.fields)
    mu = torch.zeros((wl.batch, 3), dtype=torch.float64, device="cuda")
    mus, infos = [], []
    for n in range(n_steps):
        infos.append(ctx.magnus_step(psi, n * wl.dt, wl.dt, wl.fields, mu))
        mus.append(mu.cpu().numpy().copy())
    return psi.cpu().numpy(), np.array(mus), infos


@pytest.mark.parametrize("name", ["h2", "small2_p3", "small1_p2_11orb"])
def test_magnus_steps_fixed_k_match_oracle(name):
    """Kick + 3 predictor-corrector steps with a fixed Krylov dimension:
    orbitals and dipoles to relative 1e-10."""
    wl = WORKLOADS[name]()
    S = _sys(wl)
    psi0 = S.initial_orbitals()
    if wl.batch > 1:
        psi0 = np.tile(psi0, (1, wl.batch))
    ref_psi, ref_mu = _oracle_run(S, wl, psi0, 3, fixed_k=8, tol=1e-14, kmax=8)
    got_psi, got_mu, _ = _gpu_run(wl, psi0, 3, fixed_k=8, tol=1e-14, kmax=8)
    assert np.linalg.norm(got_psi - ref_psi) <= 1e-10 * np.linalg.norm(ref_psi)
    assert np.max(np.abs(got_psi - ref_psi)) <= 1e-10 * np.max(np.abs(ref_psi))   # element-wise
    assert np.max(np.abs(got_mu - ref_mu)) <= 1e-10 * max(np.max(np.abs(ref_mu)), 1e-3)


@pytest.mark.parametrize("substeps", [2, 0])
def test_krylov_substeps_match_the_converged_step(substeps):
    """exp(-i dt Hbar) taken as sub-steps of the same operator (Eq. ApproxMagnus; they compose
    exactly): two fixed sub-steps, and the adaptive count under a cap of 6 Lanczos vectors that
    one exponential of dt cannot meet at tolerance 1e-12, against the oracle's converged single
    exponentials: orbitals and dipoles to relative 1e-9."""
    wl = WORKLOADS["small2_p3"]()
    S = _sys(wl)
    psi0 = S.initial_orbitals()
    ref_psi, ref_mu = _oracle_run(S, wl, psi0, 3, fixed_k=0, tol=1e-13, kmax=40, kick=False)
    kmax = 24 if substeps == 2 else 6
    got_psi, got_mu, infos = _gpu_run(wl, psi0, 3, fixed_k=0, tol=1e-12, kmax=kmax, kick=False,
                                      krylov_substeps=substeps)
    assert all(i["cap"] == 0 for i in infos)
    if substeps == 2:
        assert all(i["substeps"] == 2 for i in infos)
    else:
        assert min(i["substeps"] for i in infos) > 1
        _, _, single = _gpu_run(wl, psi0, 1, fixed_k=0, tol=1e-12, kmax=kmax, kick=False)
        assert single[0]["cap"] > 0          # one exponential of dt does not converge under this cap
    assert np.linalg.norm(got_psi - ref_psi) <= 1e-9 * np.linalg.norm(ref_psi)
    assert np.max(np.abs(got_psi - ref_psi)) <= 1e-9 * np.max(np.abs(ref_psi))   # element-wise
    assert np.max(np.abs(got_mu - ref_mu)) <= 1e-9 * max(np.max(np.abs(ref_mu)), 1e-3)


def test_reorthogonalised_steps_match_oracle():
    """krylov_reorth (classical Gram-Schmidt twice in every Lanczos iteration): 2 steps at fixed
    k = 14 against the oracle's reorthogonalised steps (orbitals and dipoles to relative 1e-10),
    and the basis of the last Lanczos run orthogonal to 1e-11."""
    from paper_2210_14421_gb300 import Context
    wl = WORKLOADS["small2_p3"]()
    S = _sys(wl)
    psi0 = S.initial_orbitals()
    ref_psi, ref_mu = _oracle_run(S, wl, psi0, 2, fixed_k=14, tol=1e-14, kmax=14, kick=False, reorth=True)
    ctx = Context(wl, fixed_k=14, krylov_tol=1e-14, k_max=14, cg_tol=1e-14, cg_max_it=20000, krylov_reorth=True)
    psi = _to_dev(psi0)
    mu = torch.zeros((wl.batch, 3), dtype=torch.float64, device="cuda")
    mus = []
    for n in range(2):
        ctx.magnus_step(psi, n * wl.dt, wl.dt, wl.fields, mu)
        mus.append(mu.cpu().numpy().copy())
    got = psi.cpu().numpy()
    assert np.linalg.norm(got - ref_psi) <= 1e-10 * np.linalg.norm(ref_psi)
    assert np.max(np.abs(got - ref_psi)) <= 1e-10 * np.max(np.abs(ref_psi))   # element-wise
    assert np.max(np.abs(np.array(mus) - ref_mu)) <= 1e-10 * max(np.max(np.abs(ref_mu)), 1e-3)
    loss, ks = ctx.krylov_orthogonality(3)
    assert ks and loss <= 1e-11
    ctx.close()


def test_hartree_batched_members():
    """Two densities solved in one call (both Hartree methods) against the
    oracle member by member."""
    wl = W.small_cluster(n_atoms=2, cells_per_axis=4, degree=3, n_quad=5, n_orb=2, batch=2)
    S = _sys(wl)
    from oracle import poisson, tdks
    psi0 = S.initial_orbitals()
    rho0 = tdks.density(S, psi0, wl.occ, 1)[0]
    rho = np.stack([rho0, 0.5 * rho0 + 0.01 * np.exp(-np.sum(S.mesh.xq ** 2, axis=2))])
    for method in (0, 1):
        ctx = _ctx(wl, hartree_method=method)
        vH = torch.empty((2, S.mesh.n_cells, S.mesh.nq), dtype=torch.float64, device="cuda")
        ctx.hartree(_to_dev(rho), vH, tol=1e-14, max_it=20000)
        for m in range(2):
            ref = poisson.solve(S, rho[m])[1]
            assert np.max(np.abs(vH.cpu().numpy()[m] - ref)) <= 1e-10 * np.max(np.abs(ref))


@pytest.mark.parametrize("variant", [0, 1])
def test_apply_both_tile_variants(variant):
    """Both tile widths the autotuner chooses between give the oracle's result."""
    wl = WORKLOADS["small2_p3"]()
    S = _sys(wl)
    from oracle import tdks
    from paper_2210_14421_gb300 import EFE_FP64, EFE_MIXED, EFE_PAIR
    vq = tdks.nuclear_potential(S)
    H = S.hbar(vq)
    rng = np.random.default_rng(17)
    X = rng.normal(size=(S.n_dof, wl.n_orb)) + 1j * rng.normal(size=(S.n_dof, wl.n_orb))
    X[:S.n_h][S.mesh.boundary] = 0.0
    ref = H @ X
    bound = _rounding_bound(H, X)
    ctx = _ctx(wl)
    ctx.set_potential(_to_dev(vq[None]))
    Xd = _to_dev(X)
    Yd = torch.empty_like(Xd)
    for prec, tol in ((EFE_FP64, 1e-12), (EFE_MIXED, 2e-5), (EFE_PAIR, 1e-11)):
        assert ctx.tuning(prec, force_variant=variant)["variant"] == variant
        ctx.apply_H(Xd, Yd, precision=prec)
        assert np.all(np.abs(Yd.cpu().numpy() - ref) <= tol * bound + 1e-300)


def test_graph_mode_matches_eager_and_oracle():
    """Lanczos exponentials replayed as captured CUDA graphs (k_max iterations,
    finished columns skipped on the device) give the eager / oracle result."""
    wl = W.small_cluster(n_atoms=2, cells_per_axis=4, degree=3, n_quad=5, n_orb=2, batch=2, tol=1e-10)
    S = _sys(wl)
    psi0 = np.tile(S.initial_orbitals(), (1, 2))
    ref_psi, ref_mu = _oracle_run(S, wl, psi0, 4, fixed_k=0, tol=1e-10, kmax=16)
    ctx = _ctx(wl, fixed_k=0, krylov_tol=1e-10, k_max=16, use_graphs=True)
    psi = _to_dev(psi0)
    ctx.kick(psi, wl.fields)
    mu = torch.zeros((2, 3), dtype=torch.float64, device="cuda")
    for n in range(4):      # the first step runs eagerly, later ones replay the captured graphs
        if n % 2 == 0:
            ctx.magnus_step(psi, n * wl.dt, wl.dt, wl.fields, mu)
        else:
            from paper_2210_14421_gb300 import fields_array
            ctx.magnus_step_async(psi, n * wl.dt, wl.dt, fields_array(wl.fields), mu)
    torch.cuda.synchronize()
    got = psi.cpu().numpy()
    assert np.linalg.norm(got - ref_psi) <= 1e-8 * np.linalg.norm(ref_psi)
    assert np.max(np.abs(got - ref_psi)) <= 1e-8 * np.max(np.abs(ref_psi))   # element-wise
    assert np.max(np.abs(mu.cpu().numpy() - ref_mu[-1])) <= 1e-8


def test_magnus_adaptive_k_and_batch():
    """Adaptive Lanczos (tol 1e-10) with two batch members kicked along x and y."""
    wl = W.small_cluster(n_atoms=2, cells_per_axis=4, degree=3, n_quad=5, n_orb=2, batch=2, tol=1e-10)
    S = _sys(wl)
    psi0 = np.tile(S.initial_orbitals(), (1, 2))
    ref_psi, ref_mu = _oracle_run(S, wl, psi0, 2, fixed_k=0, tol=1e-10, kmax=16)
    got_psi, got_mu, infos = _gpu_run(wl, psi0, 2, fixed_k=0, tol=1e-10, kmax=16)
    # columns may stop one Lanczos step apart where eps_k sits on the threshold:
    # both results are then within the Krylov tolerance of the exponential
    assert np.linalg.norm(got_psi - ref_psi) <= 1e-8 * np.linalg.norm(ref_psi)
    assert np.max(np.abs(got_psi - ref_psi)) <= 1e-8 * np.max(np.abs(ref_psi))   # element-wise
    assert np.max(np.abs(got_mu - ref_mu)) <= 1e-8
    assert all(i["k_corr"] <= 16 for i in infos)
    assert np.abs(ref_mu[-1, 0, 0] - ref_mu[-1, 1, 0]) > 0   # members differ


def test_mixed_precision_dipole_error():
    """Mixed path (float32 contraction) against the FP64 path on the same
    inputs: the dipole error stays below 1e-5 a.u. over 5 steps."""
    wl = WORKLOADS["small2_p3"]()
    S = _sys(wl)
    psi0 = S.initial_orbitals()
    _, mu64, _ = _gpu_run(wl, psi0, 5, fixed_k=0, tol=1e-10, kmax=16, precision=0)
    _, mu32, _ = _gpu_run(wl, psi0, 5, fixed_k=0, tol=1e-10, kmax=16, precision=1)
    assert np.max(np.abs(mu32 - mu64)) <= 1e-5


def test_pair_precision_steps_match_fp64():
    """Float32-pair path against the FP64 path: orbitals and dipoles after
    5 adaptive steps agree to 1e-9 (the pair arithmetic carries ~2^-44)."""
    wl = WORKLOADS["small2_p3"]()
    S = _sys(wl)
    psi0 = S.initial_orbitals()
    p64, mu64, _ = _gpu_run(wl, psi0, 5, fixed_k=0, tol=1e-10, kmax=16, precision=0)
    pp, mup, _ = _gpu_run(wl, psi0, 5, fixed_k=0, tol=1e-10, kmax=16, precision=2)
    assert np.max(np.abs(mup - mu64)) <= 1e-9
    assert np.max(np.abs(pp - p64)) <= 1e-9 * np.max(np.abs(p64))


def test_unitary_and_hermitian_at_scale():
    """Properties that hold at any size, on a mid-size graded cluster:
    <X, Hbar Y> = <Hbar X, Y> and the step conserves every column's norm."""
    wl = W.na_cluster(n_atoms=2, L=24.0, cells_per_axis=9, n_orb=5, n_steps=2, tol=1e-9)
    ctx = _ctx(wl)
    rng = np.random.default_rng(11)
    n = ctx.n_dof
    nodes, quad = ctx.coords()
    v = torch.from_numpy(-1.0 / (1.0 + np.sum(quad.cpu().numpy() ** 2, axis=2))[None]).cuda()
    ctx.set_potential(v.contiguous())
    X = torch.from_numpy(rng.normal(size=(n, 5)) + 1j * rng.normal(size=(n, 5))).cuda()
    Y = torch.from_numpy(rng.normal(size=(n, 5)) + 1j * rng.normal(size=(n, 5))).cuda()
    # zero boundary rows
    HX, HY = torch.empty_like(X), torch.empty_like(Y)
    ctx.apply_H(X, HX)
    ctx.apply_H(HX.clone(), HY)   # exercise a second call
    ctx.apply_H(Y, HY)
    lhs = torch.sum(X.conj() * HY, dim=0)
    rhs = torch.sum(HX.conj() * Y, dim=0)
    scale = torch.linalg.norm(HX, dim=0) * torch.linalg.norm(Y, dim=0)
    assert torch.max(torch.abs(lhs - rhs) / scale).item() < 1e-13
    psi = torch.zeros((n, wl.n_orb), dtype=torch.complex128, device="cuda")
    ctx.init_orbitals(psi)
    n0 = torch.linalg.norm(psi, dim=0)
    ctx.kick(psi, wl.fields)
    mu = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    ctx.magnus_step(psi, 0.0, wl.dt, wl.fields, mu)
    n1 = torch.linalg.norm(psi, dim=0)
    assert torch.max(torch.abs(n1 - n0) / n0).item() < 1e-11


@pytest.mark.parametrize("precision", [0, 3])
def test_krylov_blocks_match_one_run(precision):
    """Lanczos exponentials over column blocks (krylov_block = 2 of 11 orbitals: five full blocks
    and a ragged one, the way a workload too large for one Krylov basis runs) give the steps of a
    single run over all columns, since the columns are independent in the exponential: FP64 to
    rounding (1e-12), the tensor-core apply to its splitting accuracy (1e-9).  The FP64 blocked run
    also matches the oracle (1e-10)."""
    wl = WORKLOADS["small1_p2_11orb"]()
    S = _sys(wl)
    psi0 = S.initial_orbitals()
    one, mu_one, info_one = _gpu_run(wl, psi0, 2, fixed_k=0, tol=1e-12, kmax=12, precision=precision)
    blk, mu_blk, info_blk = _gpu_run(wl, psi0, 2, fixed_k=0, tol=1e-12, kmax=12, precision=precision, krylov_block=2)
    tol = 1e-12 if precision == 0 else 1e-9
    assert np.linalg.norm(blk - one) <= tol * np.linalg.norm(one)
    assert np.max(np.abs(mu_blk - mu_one)) <= tol * max(np.max(np.abs(mu_one)), 1e-3)
    assert [i["k_corr"] for i in info_blk] == [i["k_corr"] for i in info_one] or precision != 0
    if precision == 0:
        ref_psi, ref_mu = _oracle_run(S, wl, psi0, 2, fixed_k=8, tol=1e-14, kmax=8)
        got_psi, got_mu, _ = _gpu_run(wl, psi0, 2, fixed_k=8, tol=1e-14, kmax=8, krylov_block=3)
        assert np.linalg.norm(got_psi - ref_psi) <= 1e-10 * np.linalg.norm(ref_psi)
        assert np.max(np.abs(got_psi - ref_psi)) <= 1e-10 * np.max(np.abs(ref_psi))   # element-wise
        assert np.max(np.abs(got_mu - ref_mu)) <= 1e-10 * max(np.max(np.abs(ref_mu)), 1e-3)


def test_krylov_member_blocks_match_one_run():
    """Two batch members with their own fields propagated with a Krylov basis of one member
    (krylov_block = n_orb: the operator is viewed at each member's offset) give the steps of one
    run over both members (FP64, 1e-12)."""
    wl = W.small_cluster(n_atoms=2, cells_per_axis=4, degree=3, n_quad=5, n_orb=2, batch=2, tol=1e-12)
    S = _sys(wl)
    psi0 = np.tile(S.initial_orbitals(), (1, 2))
    one, mu_one, _ = _gpu_run(wl, psi0, 2, fixed_k=0, tol=1e-12, kmax=12)
    blk, mu_blk, _ = _gpu_run(wl, psi0, 2, fixed_k=0, tol=1e-12, kmax=12, krylov_block=wl.n_orb)
    assert np.linalg.norm(blk - one) <= 1e-12 * np.linalg.norm(one)
    assert np.max(np.abs(mu_blk - mu_one)) <= 1e-12 * max(np.max(np.abs(mu_one)), 1e-3)


def test_adjoint_rejects_a_blocked_krylov_basis():
    """The adjoint recombines one Krylov basis of every orbital: a context whose basis holds fewer
    columns (krylov_block) is refused with EFE_ERR_ARG, not run wrongly."""
    from paper_2210_14421_gb300 import EfeError
    wl = W.small_cluster(n_atoms=2, cells_per_axis=3, degree=3, n_quad=5, L=10.0, n_orb=2)
    S = _sys(wl)
    f = W.Field(kind=W.FIELD_GAUSS, amp=0.02, omega=0.0, t0=0.15, sigma=0.25, direction=(0.0, 0.6, 0.8))
    psi = _to_dev(S.initial_orbitals())
    ok = _ctx(wl, krylov_tol=1e-13, k_max=40)
    ok.adjoint_dipole(psi, 2, 0.04, f, (0.0, 0.6, 0.8), (1, 2), checkpoint_every=1)   # the same call runs whole
    ctx = _ctx(wl, krylov_tol=1e-13, k_max=40, krylov_block=1)
    with pytest.raises(EfeError, match="Krylov basis of all orbitals"):
        ctx.adjoint_dipole(psi, 2, 0.04, f, (0.0, 0.6, 0.8), (1, 2), checkpoint_every=1)
