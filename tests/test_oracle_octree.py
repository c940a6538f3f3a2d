"""Pins of the locally refined mesh with hanging-node constraints
(oracle.octree, reading O1)."""
import numpy as np

from oracle.octree import OctreeMesh

REFINE = [(1, 1, 1), (2, 1, 1), (0, 0, 0)]


def test_constrained_space_reproduces_tensor_polynomials():
    """Every function of Q_p (degree <= p per axis) is in the constrained space:
    its values at the free nodes, spread by the constraints, are its values at
    every node, hanging ones included (a wrong master set or weight breaks it)."""
    m = OctreeMesh([0, 0, 0], [3, 3, 3], 3, 3, REFINE)
    assert len(m.hanging) > 0
    rng = np.random.default_rng(4)
    for _ in range(3):   # random full-degree factors: no systematic zeros on the mesh planes
        cf = rng.uniform(0.5, 1.5, (3, 4))
        poly = lambda x, cf=cf: np.prod([np.polyval(cf[a], x[:, a]) for a in range(3)], axis=0)
        u_all = m.P @ poly(m.nodes[m.free])
        assert np.max(np.abs(u_all - poly(m.nodes))) < 1e-12 * np.max(np.abs(poly(m.nodes)))


def test_constrained_functions_are_continuous_across_refinement_faces():
    """A random constrained function evaluated on the faces of every coarse leaf,
    from the coarse leaf and from each refined leaf touching the same points,
    takes the same values."""
    m = OctreeMesh([0, 0, 0], [3, 3, 3], 3, 3, REFINE)
    rng = np.random.default_rng(0)
    u_all = m.P @ rng.standard_normal(len(m.free))
    worst, checked = 0.0, 0
    for li, (x0, h, coarse) in enumerate(m.leaves):
        if not coarse:
            continue
        for a in range(3):
            for side in (0, 1):
                pts = x0[None, :] + rng.uniform(0, 1, (40, 3)) * h[None, :]
                pts[:, a] = x0[a] + side * h[a]
                for lj, (y0, k, c2) in enumerate(m.leaves):
                    if c2:
                        continue
                    inside = np.all((pts >= y0 - 1e-12) & (pts <= y0 + k + 1e-12), axis=1)
                    if inside.any():
                        d = np.abs(m.evaluate(u_all, li, pts[inside]) - m.evaluate(u_all, lj, pts[inside])).max()
                        worst, checked = max(worst, d), checked + int(inside.sum())
    assert checked > 100
    assert worst < 1e-12


def test_constrained_stiffness_is_symmetric_positive_definite():
    m = OctreeMesh([0, 0, 0], [2, 2, 2], 2, 2, [(0, 0, 0)])
    K, _ = m.stiffness_and_load(lambda x: np.zeros(len(x)))
    I = np.where(~m.boundary_free)[0]
    KI = K[I][:, I].toarray()
    assert np.allclose(KI, KI.T, atol=1e-13 * np.abs(KI).max())
    assert np.linalg.eigvalsh(KI).min() > 0.0


def test_local_refinement_resolves_a_local_feature():
    """-lap u = f for a Gaussian bump (width 0.25) on a vertex of 1-bohr cells:
    refining the eight cells around it reaches the uniformly refined mesh's
    error with well under half its unknowns, an order of magnitude below the
    coarse mesh's error."""
    c, s = np.array([1.0, 1.0, 1.0]), 0.25

    def ex(x):
        return np.exp(-np.sum((x - c) ** 2, axis=1) / (2 * s * s))

    def f(x):
        r2 = np.sum((x - c) ** 2, axis=1)
        return (3 / s ** 2 - r2 / s ** 4) * ex(x)

    rng = np.random.default_rng(2)
    P = np.clip(np.concatenate([rng.uniform(0, 3, (3000, 3)), c + rng.normal(0, 0.3, (2000, 3))]), 0, 2.999)

    def error(m, ua):
        out = np.zeros(len(P))
        for li, (x0, h, _) in enumerate(m.leaves):
            ins = np.all((P >= x0) & (P < x0 + h), axis=1)
            if ins.any():
                out[ins] = m.evaluate(ua, li, P[ins])
        return np.abs(out - ex(P)).max()

    res = {}
    for name, nc, ref in (("coarse", 3, []), ("local", 3, [(i, j, k) for i in (0, 1) for j in (0, 1) for k in (0, 1)]),
                          ("fine", 6, [])):
        m = OctreeMesh([0, 0, 0], [3, 3, 3], nc, 3, ref)
        _, ua = m.solve_poisson(f, ex)
        res[name] = (error(m, ua), len(m.free))
    assert res["local"][0] <= 1.05 * res["fine"][0], res
    assert res["local"][1] < 0.4 * res["fine"][1]
    assert res["local"][0] * 10 < res["coarse"][0]


def test_hamiltonian_potential_part_integrates_and_is_symmetric():
    """The octree Hamiltonian's potential part against closed forms: with
    kin = 0 and v = c, <1, H 1> = c |box| (the constant is in the constrained
    space and the consistent mass integrates it exactly); with v = x,
    <1, H 1> = int x = |box| x_centre; H is symmetric; the kinetic part
    annihilates constants."""
    m = OctreeMesh([0, 0, 0], [3, 2, 2], 3, 3, [(1, 0, 0), (2, 1, 1)])
    xq = m.quad_points()
    one = np.ones(len(m.free))
    vol = 3.0 * 2.0 * 2.0
    H = m.hamiltonian(np.full(xq.shape[:2], 0.7), kin=0.0)
    assert abs(one @ (H @ one) - 0.7 * vol) < 1e-12 * vol
    H = m.hamiltonian(xq[:, :, 0], kin=0.0)
    assert abs(one @ (H @ one) - 1.5 * vol) < 1e-12 * vol
    H = m.hamiltonian(xq[:, :, 1] ** 2 - xq[:, :, 2], kin=1.0)
    assert abs(H - H.T).max() < 1e-13 * abs(H).max()
    K = m.hamiltonian(np.zeros(xq.shape[:2]), kin=1.0)
    assert np.abs(K @ one).max() < 1e-12 * abs(K).max()


def test_constrained_lumped_mass_and_loewdin_hamiltonian():
    """Reading O2 against closed forms and the rectilinear oracle: the lumped
    constrained mass sums to the box volume and, without refinement, equals the
    rectilinear mesh's GLL-lumped mass node by node; the Loewdin-scaled
    harmonic-oscillator Hamiltonian (v = r^2 / 2) has its lowest eigenvalue at
    the exact 1.5 Ha within 5e-5 once the cells around the minimum are refined,
    closer than on the unrefined mesh (6e-4)."""
    import scipy.sparse.linalg as spla
    from oracle.mesh import Mesh
    m0 = OctreeMesh([-5, -5, -5], [5, 5, 5], 4, 4, [])
    b = np.linspace(-5, 5, 5)
    r = Mesh(b, b, b, 4, 6)
    pos = {tuple(k): i for i, k in enumerate(np.round(r.nodes * 1e6).astype(np.int64))}
    idx = [pos[tuple(k)] for k in np.round(m0.nodes[m0.free] * 1e6).astype(np.int64)]
    assert np.max(np.abs(m0.lumped_mass() - r.lumped_mass()[idx])) < 1e-14
    ref = [(i, j, k) for i in (1, 2) for j in (1, 2) for k in (1, 2)]
    m1 = OctreeMesh([-5, -5, -5], [5, 5, 5], 4, 4, ref)
    assert abs(m1.lumped_mass().sum() - 1000.0) < 1e-10
    lam = []
    for m in (m0, m1):
        xq = m.quad_points()
        Hb = m.hbar(0.5 * np.sum(xq ** 2, axis=2)).tocsc()
        assert abs(Hb - Hb.T).max() < 1e-13 * abs(Hb).max()
        lam.append(spla.eigsh(Hb, k=1, sigma=0, which="LM")[0][0])
    assert abs(lam[1] - 1.5) < 5e-5 and abs(lam[1] - 1.5) < abs(lam[0] - 1.5) / 5, lam


def test_density_integrates_to_the_mass_quadratic_form():
    """int rho = sum_a occ_a psi_a^H (P^T M P) psi_a with psi = D psi_bar, the
    consistent mass taken from the Hamiltonian's potential part with v = 1 and
    kin = 0 (an independent assembly); rho >= 0."""
    m = OctreeMesh([0, 0, 0], [3, 2, 2], 3, 3, [(1, 0, 0), (2, 1, 1)])
    rng = np.random.default_rng(5)
    psi_bar = rng.standard_normal((len(m.free), 2)) + 1j * rng.standard_normal((len(m.free), 2))
    occ = np.array([2.0, 1.0])
    rho = m.density(psi_bar, occ)
    assert rho.min() >= 0.0
    w = np.stack([m.wq * np.prod(h) / 8.0 for _, h, _ in m.leaves])
    d = np.where(m.boundary_free, 0.0, 1.0 / np.sqrt(m.lumped_mass()))
    psi = d[:, None] * psi_bar
    Mc = m.hamiltonian(np.ones(w.shape), kin=0.0)
    ref = sum(occ[a] * np.real(np.conj(psi[:, a]) @ (Mc @ psi[:, a])) for a in range(2))
    assert abs(np.sum(w * rho) - ref) < 1e-12 * ref


def test_magnus_step_reduces_to_the_rectilinear_step():
    """Without refinement the locally refined mesh is the rectilinear mesh: the
    predictor-corrector step there (classical basis, fixed Krylov dimension 8)
    equals the rectilinear oracle's step (oracle.tdks) node for node."""
    import efe_workloads as W
    from oracle import operators, tdks
    wl = W.small_cluster(n_atoms=2, cells_per_axis=3, degree=3, n_quad=5, L=10.0, n_orb=2)
    b = np.linspace(-5, 5, 4)
    wl = wl.with_(xb=b, yb=b.copy(), zb=b.copy(), enrich=[], enr_coefs=np.zeros((wl.n_orb, 0), dtype=complex))
    S = operators.System(wl)
    m = OctreeMesh([-5, -5, -5], [5, 5, 5], 3, 3, [])
    pos = {tuple(k): i for i, k in enumerate(np.round(S.mesh.nodes * 1e6).astype(np.int64))}
    idx = np.array([pos[tuple(k)] for k in np.round(m.nodes[m.free] * 1e6).astype(np.int64)])
    rng = np.random.default_rng(4)
    psi_r = (rng.standard_normal((S.n_h, 2)) + 1j * rng.standard_normal((S.n_h, 2))) * S.mesh.interior[:, None]
    field = W.Field(kind=W.FIELD_GAUSS, amp=0.0, omega=0.0, t0=0.0, sigma=1.0, direction=(0.0, 0.0, 1.0))
    st = tdks.make_state(S, psi_r, wl.occ, 1)
    out_r = tdks.magnus_step(S, psi_r, st, 0.0, 0.05, [field], wl.occ, 1e-14, 8, fixed_k=8)[0]
    out_o = m.magnus_step(psi_r[idx], wl.occ, wl.Z, wl.R, 0.05, 8, np.zeros(3))
    assert np.max(np.abs(out_o - out_r[idx])) < 1e-12 * np.max(np.abs(out_r))
