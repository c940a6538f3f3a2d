"""The constrained Hamiltonian apply on the locally refined mesh
(efe_octree_apply: gather through the hanging-node constraints P, per-leaf
kinetic and potential operator, scatter through P^T) against the oracle's
P^T H P (oracle.octree.OctreeMesh.hamiltonian), and its properties on a larger
mesh."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


# (lo, hi, nc, degree, n_quad, refined cells): degrees 2, 3, 5; one refined cell,
# neighbouring refined cells, a refined 2^3 block; non-cubic boxes
MESHES = {
    "p3_three": ([0, 0, 0], [3, 3, 3], 3, 3, 5, [(1, 1, 1), (2, 1, 1), (0, 0, 0)]),
    "p3_box": ([0, 0, 0], [3, 2, 2], 3, 3, 5, [(1, 0, 0), (2, 1, 1)]),
    "p2_block": ([-1, 0, 0.5], [2, 2, 2.5], 4, 2, 4, [(i, j, k) for i in (1, 2) for j in (1, 2) for k in (1, 2)]),
    "p5_corner": ([0, 0, 0], [2, 2, 2], 2, 5, 7, [(0, 0, 0)]),
}


def _key(x):
    return [tuple(r) for r in np.round(np.asarray(x) * 1e6).astype(np.int64)]


@pytest.mark.parametrize("mask", [False, True])
@pytest.mark.parametrize("name", list(MESHES))
def test_octree_apply_matches_oracle(name, mask):
    from oracle.octree import OctreeMesh
    from paper_2210_14421_gb300 import Octree
    lo, hi, nc, p, nq, ref = MESHES[name]
    m = OctreeMesh(lo, hi, nc, p, ref, n_quad=nq)
    o = Octree(lo, hi, nc, p, nq, ref)
    assert o.n_all == m.n_all and o.n_free == len(m.free) and o.n_hanging == len(m.hanging)
    fx, qx, bnd = o.coords()
    assert np.allclose(qx, m.quad_points(), rtol=0, atol=1e-13)
    pos = {k: j for j, k in enumerate(_key(m.nodes[m.free]))}
    perm = np.array([pos[k] for k in _key(fx)])          # GPU free node -> oracle free index
    assert np.array_equal(bnd, m.boundary_free[perm])
    rng = np.random.default_rng(7)
    vq = np.sin(qx[:, :, 0]) + qx[:, :, 1] ** 2 - 0.3 * qx[:, :, 2]
    X = rng.standard_normal((o.n_free, 3))
    H = m.hamiltonian(vq, kin=0.8)
    Xo = np.zeros((len(m.free), 3))
    Xo[perm] = X
    if mask:
        I = ~m.boundary_free
        ref_y = np.zeros_like(Xo)
        ref_y[I] = H[I][:, I] @ Xo[I]
        scale = np.zeros_like(Xo)                   # full free-node length: indexed by perm below
        scale[I] = abs(H[I][:, I]) @ np.abs(Xo[I])
    else:
        ref_y = H @ Xo
        scale = abs(H) @ np.abs(Xo)
    Y = torch.zeros((o.n_free, 3), dtype=torch.float64, device="cuda")
    o.apply(torch.from_numpy(np.ascontiguousarray(vq)).cuda(), torch.from_numpy(X).cuda(), Y, kin=0.8,
            mask_boundary=mask)
    got = Y.cpu().numpy()
    ref_g = ref_y[perm]
    assert np.max(np.abs(got - ref_g) - 1e-12 * scale[perm] - 1e-300) <= 0.0, name
    o.close()


def test_octree_rejects_bad_meshes():
    from paper_2210_14421_gb300 import EfeError, Octree
    with pytest.raises(EfeError):
        Octree([0, 0, 0], [1, 1, 1], 2, 3, 3, [])          # n_quad < p + 1
    with pytest.raises(EfeError):
        Octree([0, 0, 0], [1, 1, 1], 2, 3, 5, [(2, 0, 0)])  # refined cell outside the grid
    with pytest.raises(EfeError):
        Octree([0, 0, 0], [0, 1, 1], 2, 3, 5, [])          # empty box


def test_octree_larger_mesh_properties():
    """16^3 coarse cells of degree 4 with a refined 4^3 block (the local refinement
    around a nucleus): the operator is symmetric, the kinetic part annihilates
    constants, and <1, V 1> = c |box| for a constant potential (the constrained
    space holds the constants and the leaf rules integrate them exactly)."""
    from paper_2210_14421_gb300 import Octree
    ref = [(i, j, k) for i in range(6, 10) for j in range(6, 10) for k in range(6, 10)]
    o = Octree([-8, -8, -8], [8, 8, 8], 16, 4, 6, ref)
    assert o.n_hanging > 0
    _, qx, _ = o.coords()
    rng = np.random.default_rng(3)
    vq = torch.from_numpy(-1.0 / np.sqrt(1.0 + np.sum(qx ** 2, axis=2))).cuda()
    X = torch.from_numpy(rng.standard_normal((o.n_free, 2))).cuda()
    Y = torch.zeros_like(X)
    o.apply(vq, X, Y, kin=1.0)
    lhs = (X[:, 0] * Y[:, 1]).sum().item()
    rhs = (Y[:, 0] * X[:, 1]).sum().item()
    assert abs(lhs - rhs) <= 1e-11 * (torch.linalg.norm(X) * torch.linalg.norm(Y)).item()
    one = torch.ones((o.n_free, 1), dtype=torch.float64, device="cuda")
    K1 = torch.zeros_like(one)
    o.apply(torch.zeros_like(vq), one, K1, kin=1.0)
    assert torch.max(torch.abs(K1)).item() < 1e-10
    V1 = torch.zeros_like(one)
    o.apply(torch.full_like(vq, 0.7), one, V1, kin=0.0)
    assert abs(V1.sum().item() - 0.7 * 16.0 ** 3) < 1e-9 * 16.0 ** 3
    o.close()


def test_octree_poisson_matches_oracle():
    """-lap u = f for a Gaussian bump on a vertex of 1-bohr cells, the eight cells
    around it refined (the oracle's local-refinement case): the CUDA conjugate
    gradients against the oracle's sparse direct solve of the same constrained
    system, node by node (1e-9)."""
    from oracle.octree import OctreeMesh
    from paper_2210_14421_gb300 import Octree
    c0, s0 = np.array([1.0, 1.0, 1.0]), 0.25

    def ex(x):
        return np.exp(-np.sum((x - c0) ** 2, axis=-1) / (2 * s0 * s0))

    def f(x):
        r2 = np.sum((x - c0) ** 2, axis=-1)
        return (3 / s0 ** 2 - r2 / s0 ** 4) * ex(x)

    ref_cells = [(i, j, k) for i in (0, 1) for j in (0, 1) for k in (0, 1)]
    m = OctreeMesh([0, 0, 0], [3, 3, 3], 3, 3, ref_cells)
    u_ref, _ = m.solve_poisson(f, ex)
    o = Octree([0, 0, 0], [3, 3, 3], 3, 3, 5, ref_cells)
    fx, qx, _ = o.coords()
    u, its = o.poisson(torch.from_numpy(f(qx)).cuda(), torch.from_numpy(ex(fx)).cuda(), tol=1e-13, max_it=20000)
    pos = {k: j for j, k in enumerate(_key(m.nodes[m.free]))}
    perm = np.array([pos[k] for k in _key(fx)])
    assert its > 0
    assert np.max(np.abs(u.cpu().numpy() - u_ref[perm])) <= 1e-9 * np.max(np.abs(u_ref))
    o.close()


@pytest.mark.parametrize("name", ["p3_box", "p5_corner"])
def test_octree_loewdin_apply_matches_oracle(name):
    """The Loewdin-scaled operator D P^T H P D on the interior free nodes (D from
    the lumped constrained mass) against the oracle's OctreeMesh.hbar."""
    from oracle.octree import OctreeMesh
    from paper_2210_14421_gb300 import Octree
    lo, hi, nc, p, nq, ref = MESHES[name]
    m = OctreeMesh(lo, hi, nc, p, ref, n_quad=nq)
    o = Octree(lo, hi, nc, p, nq, ref)
    fx, qx, _ = o.coords()
    pos = {k: j for j, k in enumerate(_key(m.nodes[m.free]))}
    perm = np.array([pos[k] for k in _key(fx)])
    vq = 0.5 * np.sum(qx ** 2, axis=2)
    X = np.random.default_rng(11).standard_normal((o.n_free, 2))
    Xo = np.zeros_like(X)
    Xo[perm] = X
    I = np.where(~m.boundary_free)[0]
    Hb = m.hbar(vq, kin=1.0)
    ref_y = np.zeros_like(Xo)
    ref_y[I] = Hb @ Xo[I]
    scale = np.zeros_like(Xo)
    scale[I] = abs(Hb) @ np.abs(Xo[I])
    Y = torch.zeros((o.n_free, 2), dtype=torch.float64, device="cuda")
    o.apply(torch.from_numpy(np.ascontiguousarray(vq)).cuda(), torch.from_numpy(X).cuda(), Y, kin=1.0, lowdin=True)
    got = Y.cpu().numpy()
    assert np.max(np.abs(got - ref_y[perm]) - 1e-12 * scale[perm] - 1e-300) <= 0.0
    o.close()


@pytest.mark.parametrize("name", ["p3_box", "p5_corner", "p2_block"])
def test_octree_density_matches_oracle(name):
    """rho at the leaves' Gauss-Legendre points from Loewdin-basis orbitals against
    OctreeMesh.density (1e-12 relative)."""
    from oracle.octree import OctreeMesh
    from paper_2210_14421_gb300 import Octree
    lo, hi, nc, p, nq, ref = MESHES[name]
    m = OctreeMesh(lo, hi, nc, p, ref, n_quad=nq)
    o = Octree(lo, hi, nc, p, nq, ref)
    fx, _, _ = o.coords()
    pos = {k: j for j, k in enumerate(_key(m.nodes[m.free]))}
    perm = np.array([pos[k] for k in _key(fx)])
    rng = np.random.default_rng(3)
    psi = rng.standard_normal((o.n_free, 3)) + 1j * rng.standard_normal((o.n_free, 3))
    occ = np.array([2.0, 2.0, 1.0])
    rho = o.density(torch.from_numpy(psi).cuda(), occ).cpu().numpy()
    po = np.zeros_like(psi)
    po[perm] = psi
    ref_rho = m.density(po, occ)
    assert np.max(np.abs(rho - ref_rho)) <= 1e-12 * np.max(np.abs(ref_rho))
    o.close()


def test_octree_krylov_exponential_matches_oracle():
    """psi <- exp(-i dt Hbar) psi on the locally refined mesh (harmonic potential,
    fixed Krylov dimension 8) against the oracle's Lanczos exponential of
    OctreeMesh.hbar (1e-10 relative); norms conserved."""
    from oracle import krylov
    from oracle.octree import OctreeMesh
    from paper_2210_14421_gb300 import Octree
    lo, hi, nc, p, nq, ref = [-5, -5, -5], [5, 5, 5], 3, 3, 5, [(1, 1, 1)]
    m = OctreeMesh(lo, hi, nc, p, ref, n_quad=nq)
    o = Octree(lo, hi, nc, p, nq, ref)
    fx, qx, bnd = o.coords()
    pos = {k: j for j, k in enumerate(_key(m.nodes[m.free]))}
    perm = np.array([pos[k] for k in _key(fx)])
    vq = 0.5 * np.sum(qx ** 2, axis=2)
    rng = np.random.default_rng(9)
    psi = rng.standard_normal((o.n_free, 2)) + 1j * rng.standard_normal((o.n_free, 2))
    psi[bnd] = 0.0
    po = np.zeros_like(psi)
    po[perm] = psi
    I = np.where(~m.boundary_free)[0]
    ref_out, _, _ = krylov.expm_block(m.hbar(vq, 1.0), po[I], 0.05, 1e-14, 8, fixed_k=8)
    g = torch.from_numpy(np.ascontiguousarray(psi)).cuda()
    o.kexp(torch.from_numpy(np.ascontiguousarray(vq)).cuda(), g, 0.05, 8)
    got = np.zeros_like(po)
    got[perm] = g.cpu().numpy()
    assert np.max(np.abs(got[I] - ref_out)) <= 1e-10 * np.max(np.abs(ref_out))
    assert abs(np.linalg.norm(got) - np.linalg.norm(psi)) <= 1e-12 * np.linalg.norm(psi)
    o.close()


def test_octree_adaptive_krylov_dimension():
    """The adaptive form (Eqs. AdaptiveKrylov, AdaptiveKrylovErr): each column stops at the first
    dimension whose estimate meets the tolerance.  Against the oracle's Lanczos exponential of
    OctreeMesh.hbar converged to 1e-13: within 10x the tolerance (1e-9) of the orbital's norm,
    with fewer vectors than the cap; a cap far below what the tolerance needs is reported, not
    raised."""
    from oracle import krylov
    from oracle.octree import OctreeMesh
    from paper_2210_14421_gb300 import Octree
    lo, hi, nc, p, nq, ref = [-5, -5, -5], [5, 5, 5], 3, 3, 5, [(1, 1, 1)]
    m = OctreeMesh(lo, hi, nc, p, ref, n_quad=nq)
    o = Octree(lo, hi, nc, p, nq, ref)
    fx, qx, bnd = o.coords()
    pos = {k: j for j, k in enumerate(_key(m.nodes[m.free]))}
    perm = np.array([pos[k] for k in _key(fx)])
    vq = 0.5 * np.sum(qx ** 2, axis=2)
    rng = np.random.default_rng(12)
    psi = rng.standard_normal((o.n_free, 2)) + 1j * rng.standard_normal((o.n_free, 2))
    psi[bnd] = 0.0
    po = np.zeros_like(psi)
    po[perm] = psi
    I = np.where(~m.boundary_free)[0]
    ref_out, ks, _ = krylov.expm_block(m.hbar(vq, 1.0), po[I], 0.05, 1e-13, 64)
    vd = torch.from_numpy(np.ascontiguousarray(vq)).cuda()
    g = torch.from_numpy(np.ascontiguousarray(psi)).cuda()
    ku = o.kexp(vd, g, 0.05, 64, tol=1e-9)
    assert 1 < ku < 64
    got = np.zeros_like(po)
    got[perm] = g.cpu().numpy()
    assert np.max(np.linalg.norm(got[I] - ref_out, axis=0) / np.linalg.norm(psi, axis=0)) <= 1e-8
    g2 = torch.from_numpy(np.ascontiguousarray(psi)).cuda()
    assert o.kexp(vd, g2, 0.05, 3, tol=1e-14) == 3        # the cap, reported by the status
    o.close()


@pytest.mark.parametrize("name", ["p3_box", "p5_corner"])
def test_octree_interpolation_matches_oracle(name):
    """Nodal columns of the constrained space at the leaves' Gauss-Legendre points
    against OctreeMesh.evaluate of P u (1e-12 relative)."""
    from oracle.octree import OctreeMesh
    from paper_2210_14421_gb300 import Octree
    lo, hi, nc, p, nq, ref = MESHES[name]
    m = OctreeMesh(lo, hi, nc, p, ref, n_quad=nq)
    o = Octree(lo, hi, nc, p, nq, ref)
    fx, qx, _ = o.coords()
    pos = {k: j for j, k in enumerate(_key(m.nodes[m.free]))}
    perm = np.array([pos[k] for k in _key(fx)])
    u = np.random.default_rng(2).standard_normal((o.n_free, 2))
    out = o.interp(torch.from_numpy(u).cuda()).cpu().numpy()
    uo = np.zeros_like(u)
    uo[perm] = u
    for c in range(2):
        ua = m.P @ uo[:, c]
        ref_v = np.stack([m.evaluate(ua, li, qx[li]) for li in range(o.n_leaves)])
        assert np.max(np.abs(out[c] - ref_v)) <= 1e-12 * np.max(np.abs(ref_v))
    o.close()


@pytest.mark.parametrize("xc", ["pw92", "pz81"])
def test_context_free_lda_matches_oracle(xc):
    """efe_lda_points (the LDA for meshes without a context) against the oracle's
    LDA on densities spanning the floor and both PZ81 branches (1e-12)."""
    from oracle import xc as oxc
    from paper_2210_14421_gb300 import EFE_XC_PW92, EFE_XC_PZ81, lda_points
    rho = np.concatenate([np.logspace(-16, 3, 400), [0.0, 1e-14, 2e-14]])
    vxc, exc = lda_points(torch.from_numpy(rho).cuda(), EFE_XC_PW92 if xc == "pw92" else EFE_XC_PZ81)
    e_ref, v_ref = oxc.lda(rho, xc)[:2]
    assert np.max(np.abs(vxc.cpu().numpy() - v_ref) - 1e-12 * np.abs(v_ref)) <= 1e-300
    assert np.max(np.abs(exc.cpu().numpy() - e_ref) - 1e-12 * np.abs(e_ref)) <= 1e-300


def test_octree_magnus_step_matches_oracle():
    """One predictor-corrector step on the locally refined mesh (two nuclei, a field,
    Hartree and LDA potentials, Krylov dimension 8) against the oracle's step
    OctreeMesh.magnus_step (1e-10)."""
    from oracle.octree import OctreeMesh
    from paper_2210_14421_gb300 import Octree
    lo, hi, nc, p, nq, ref = [-5, -5, -5], [5, 5, 5], 3, 3, 5, [(1, 1, 1)]
    Z, R = [1.0, 1.0], [np.array([-0.7, 0.1, 0.0]), np.array([0.7, -0.1, 0.2])]
    m = OctreeMesh(lo, hi, nc, p, ref, n_quad=nq)
    o = Octree(lo, hi, nc, p, nq, ref)
    fx, _, bnd = o.coords()
    pos = {k: j for j, k in enumerate(_key(m.nodes[m.free]))}
    perm = np.array([pos[k] for k in _key(fx)])
    rng = np.random.default_rng(8)
    psi = rng.standard_normal((o.n_free, 2)) + 1j * rng.standard_normal((o.n_free, 2))
    psi[bnd] = 0.0
    psi /= np.linalg.norm(psi, axis=0)       # neutral: occ . ||psi||^2 = sum Z (the Dirichlet data's premise)
    po = np.zeros_like(psi)
    po[perm] = psi
    occ, E = np.array([1.0, 1.0]), np.array([0.0, 0.0, 0.01])
    ref_out = m.magnus_step(po, occ, Z, R, 0.05, 8, E)
    g = torch.from_numpy(np.ascontiguousarray(psi)).cuda()
    o.magnus_step(g, occ, Z, np.array(R), 0.05, 8, field=E, cg_tol=1e-13)
    got = np.zeros_like(po)
    got[perm] = g.cpu().numpy()
    assert np.max(np.abs(got - ref_out)) <= 1e-10 * np.max(np.abs(ref_out))
    o.close()
