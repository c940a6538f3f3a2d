"""The tensor-core precision (EFE_TC: dense cell matrices and enrichment coupling
split into four bf16 slices, exact slice products, float32 tensor-memory
accumulation) against the FP64 oracle and the FP64 GPU path.

Error model: every operand is rounded to 31 bits of its row's (or column's)
power-of-two scale, slice pairs past the fourth group are dropped and the third
accumulator rounds in binary32, so per element of y = Hbar x the error is a few
2^-31 K max|H_ik| max|x_k| (K <= 176 terms).  The tests hold it to 1e-7 of
sum_k |Hbar_ik| max_k |x_k| per column: well inside what 31 bits allow and well
below what a binary32 contraction reaches on the same inputs."""
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


def _to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _sys(wl):
    from oracle import operators
    return operators.System(wl)


def _tc_bound(H, X):
    """sum_k |Hbar_ik| max_k |X_kn| for every (i, n)."""
    return np.abs(H) @ np.ones(H.shape[1])[:, None] * np.max(np.abs(X), axis=0)[None, :]


WORKLOADS = {
    "h2": lambda: W.h2(),
    "small2_p3": lambda: W.small_cluster(n_atoms=2, cells_per_axis=5, degree=3, n_quad=5, n_orb=3),
    "small1_p2_11orb": lambda: W.small_cluster(n_atoms=1, cells_per_axis=3, degree=2, n_quad=4, L=10.0, n_orb=11),
}


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_tc_apply_matches_oracle(name):
    from oracle import tdks
    from paper_2210_14421_gb300 import EFE_MIXED, EFE_TC, Context
    wl = WORKLOADS[name]()
    S = _sys(wl)
    rng = np.random.default_rng(17)
    vq = tdks.nuclear_potential(S) + 0.05 * np.sum(S.mesh.xq ** 2, axis=2)
    H = S.hbar(vq)
    X = rng.normal(size=(S.n_dof, wl.n_orb)) + 1j * rng.normal(size=(S.n_dof, wl.n_orb))
    X[:S.n_h][S.mesh.boundary] = 0.0
    ref = H @ X
    ctx = Context(wl)
    ctx.set_potential(_to_dev(vq[None]))
    Xd = _to_dev(X)
    Yd = torch.empty_like(Xd)
    ctx.apply_H(Xd, Yd, precision=EFE_TC)
    got = Yd.cpu().numpy()
    bound = _tc_bound(H, X.real) + _tc_bound(H, X.imag)
    err = np.abs(got - ref)
    assert np.all(err <= 1e-7 * bound + 1e-300), float(np.max(err / bound))
    # an order of magnitude better than the binary32 contraction on the same inputs
    ctx.apply_H(Xd, Yd, precision=EFE_MIXED)
    err32 = np.abs(Yd.cpu().numpy() - ref)
    assert np.max(err) * 10 < np.max(err32), (float(np.max(err)), float(np.max(err32)))
    # repeated applies give the same result (slices are rebuilt only with the operator)
    ctx.apply_H(Xd, Yd, precision=EFE_TC)
    assert np.max(np.abs(Yd.cpu().numpy() - got)) <= 1e-12 * np.max(np.abs(got))


def test_tc_batched_potentials_and_rebuild():
    """Two batch members with their own potentials; a new potential rebuilds the slices."""
    from oracle import tdks
    from paper_2210_14421_gb300 import EFE_TC, Context
    wl = W.small_cluster(n_atoms=2, cells_per_axis=4, degree=3, n_quad=5, n_orb=3, batch=2)
    S = _sys(wl)
    v0 = tdks.nuclear_potential(S)
    v1 = v0 + 0.2 * S.mesh.xq[:, :, 0]
    rng = np.random.default_rng(5)
    X = rng.normal(size=(S.n_dof, 6)) + 1j * rng.normal(size=(S.n_dof, 6))
    X[:S.n_h][S.mesh.boundary] = 0.0
    ctx = Context(wl)
    Xd = _to_dev(X)
    Yd = torch.empty_like(Xd)
    for va, vb in ((v0, v1), (v1, v0)):
        ctx.set_potential(_to_dev(np.stack([va, vb])))
        ctx.apply_H(Xd, Yd, precision=EFE_TC)
        Ha, Hb = S.hbar(va), S.hbar(vb)
        ref = np.concatenate([Ha @ X[:, :3], Hb @ X[:, 3:]], axis=1)
        bound = np.concatenate([_tc_bound(Ha, np.abs(X[:, :3])), _tc_bound(Hb, np.abs(X[:, 3:]))], axis=1)
        assert np.all(np.abs(Yd.cpu().numpy() - ref) <= 2e-7 * bound + 1e-300)


def test_tc_apply_at_scale_matches_fp64():
    """729 graded cells with enrichment (more cells than SMs: the persistent loop
    takes several cells per CTA), against the FP64 GPU apply."""
    from paper_2210_14421_gb300 import EFE_FP64, EFE_TC, Context
    wl = W.na_cluster(n_atoms=2, L=24.0, cells_per_axis=9, n_orb=5, n_steps=2, tol=1e-9)
    ctx = Context(wl)
    _, quad = ctx.coords()
    v = (-1.0 / (1.0 + (quad ** 2).sum(-1)))[None].contiguous()
    ctx.set_potential(v)
    rng = np.random.default_rng(23)
    X = _to_dev(rng.normal(size=(ctx.n_dof, 5)) + 1j * rng.normal(size=(ctx.n_dof, 5)))
    Y64, Ytc = torch.empty_like(X), torch.empty_like(X)
    ctx.apply_H(X, Y64, precision=EFE_FP64)
    ctx.apply_H(X, Ytc, precision=EFE_TC)
    rel = (torch.abs(Ytc - Y64).max() / torch.abs(Y64).max()).item()
    assert rel < 1e-7, rel
    # Hermitian to the splitting's accuracy
    Y = _to_dev(rng.normal(size=(ctx.n_dof, 5)) + 1j * rng.normal(size=(ctx.n_dof, 5)))
    HY = torch.empty_like(Y)
    ctx.apply_H(Y, HY, precision=EFE_TC)
    lhs = torch.sum(X.conj() * HY, dim=0)
    rhs = torch.sum(Ytc.conj() * Y, dim=0)
    scale = torch.linalg.norm(Ytc, dim=0) * torch.linalg.norm(Y, dim=0)
    assert torch.max(torch.abs(lhs - rhs) / scale).item() < 1e-7


def test_tc_steps_match_fp64():
    """Context precision EFE_TC (slices built with every operator): five adaptive
    predictor-corrector steps against the FP64 path.  The apply carries ~3e-9 of its
    row scales; the dipoles here are ~30 a.u., so 1e-6 a.u. (10x inside the 1e-5
    bound of the reduced-precision forms) leaves room for five steps of it."""
    from paper_2210_14421_gb300 import EFE_FP64, EFE_TC, Context
    wl = WORKLOADS["small2_p3"]()
    S = _sys(wl)
    psi0 = S.initial_orbitals()
    out = {}
    for prec in (EFE_FP64, EFE_TC):
        ctx = Context(wl, precision=prec, krylov_tol=1e-10, k_max=16, cg_tol=1e-14, cg_max_it=20000)
        psi = _to_dev(psi0)
        ctx.kick(psi, wl.fields)
        mu = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
        mus = []
        for n in range(5):
            ctx.magnus_step(psi, n * wl.dt, wl.dt, wl.fields, mu)
            mus.append(mu.cpu().numpy().copy())
        out[prec] = (psi.cpu().numpy(), np.array(mus))
    p64, mu64 = out[EFE_FP64]
    ptc, mutc = out[EFE_TC]
    assert np.max(np.abs(mutc - mu64)) <= 1e-6
    assert np.max(np.abs(ptc - p64)) <= 1e-6 * np.max(np.abs(p64))


def test_tc_graph_mode_matches_eager():
    """Captured Lanczos graphs with the tensor-core apply (finished columns gate the
    persistent kernel) reproduce the eager EFE_TC run."""
    from paper_2210_14421_gb300 import EFE_TC, Context, fields_array
    wl = W.small_cluster(n_atoms=2, cells_per_axis=4, degree=3, n_quad=5, n_orb=2, batch=2, tol=1e-10)
    S = _sys(wl)
    psi0 = np.tile(S.initial_orbitals(), (1, 2))
    res = []
    for graphs in (False, True):
        ctx = Context(wl, precision=EFE_TC, krylov_tol=1e-10, k_max=16, use_graphs=graphs)
        psi = _to_dev(psi0)
        ctx.kick(psi, wl.fields)
        mu = torch.zeros((2, 3), dtype=torch.float64, device="cuda")
        for n in range(4):
            if n % 2 == 0:
                ctx.magnus_step(psi, n * wl.dt, wl.dt, wl.fields, mu)
            else:
                ctx.magnus_step_async(psi, n * wl.dt, wl.dt, fields_array(wl.fields), mu)
        torch.cuda.synchronize()
        res.append((psi.cpu().numpy(), mu.cpu().numpy()))
    assert np.linalg.norm(res[1][0] - res[0][0]) <= 1e-9 * np.linalg.norm(res[0][0])
    assert np.max(np.abs(res[1][1] - res[0][1])) <= 1e-9


def test_tc_unsupported_cases_are_rejected():
    """Degree 5 (216 nodes per cell) is outside the 128-row tile: EFE_ARG, not a fallback."""
    from paper_2210_14421_gb300 import EFE_TC, Context, EfeError
    wl = W.small_cluster(n_atoms=2, cells_per_axis=3, degree=5, n_quad=7, n_orb=2, L=12.0)
    with pytest.raises(EfeError):
        Context(wl, precision=EFE_TC)
    ctx = Context(wl)
    _, quad = ctx.coords()
    ctx.set_potential((-1.0 / (1.0 + (quad ** 2).sum(-1)))[None].contiguous())
    X = torch.zeros((ctx.n_dof, 2), dtype=torch.complex128, device="cuda")
    Y = torch.empty_like(X)
    with pytest.raises(EfeError):
        ctx.apply_H(X, Y, precision=EFE_TC)


def test_tc_apply_split_cells_and_column_blocks_match_fp64():
    """An organic-27-like mesh coarsened to 7^3 cells: 87 enrichment functions, cells coupled to up
    to 87 of them (the apply splits such a cell into work items of at most 48 functions, the first
    one carrying H_c) and 59 orbitals (118 real columns: blocks of 96 and 22).  Against the FP64
    apply, element-wise to 1e-7 of the row scale, and to the FP64 result as a whole to 1e-8."""
    from paper_2210_14421_gb300 import EFE_FP64, EFE_TC, Context
    wl = W.organic27(cells_per_axis=7)
    ctx = Context(wl)
    _, quad = ctx.coords()
    v = torch.zeros(quad.shape[:2], dtype=torch.float64, device="cuda")
    for Z, R in zip(wl.Z, wl.R):
        v -= float(Z) / torch.sqrt(((quad - torch.tensor(R, dtype=torch.float64, device="cuda")) ** 2).sum(-1))
    ctx.set_potential(v[None].contiguous())
    assert ctx.n_pairs > 48 * ctx.n_cells // 4   # many cells beyond one work item
    rng = np.random.default_rng(31)
    X = _to_dev(rng.normal(size=(ctx.n_dof, wl.n_orb)) + 1j * rng.normal(size=(ctx.n_dof, wl.n_orb)))
    Y64, Ytc = torch.empty_like(X), torch.empty_like(X)
    ctx.apply_H(X, Y64, precision=EFE_FP64)
    ctx.apply_H(X, Ytc, precision=EFE_TC)
    rel = (torch.abs(Ytc - Y64).max() / torch.abs(Y64).max()).item()
    assert rel < 1e-8, rel
    err = torch.abs(Ytc - Y64)
    scale = torch.abs(Y64).amax(dim=1, keepdim=True) + torch.abs(Y64).max() * 1e-6
    assert torch.max(err / scale).item() < 1e-7
    ctx.close()
