"""Parity of the electrostatically enriched nuclear potential (efe_nuclear_enriched:
smeared nuclei, one enrichment function per atom, block elimination around the
direct Poisson solver) with the oracle's enriched Galerkin solve
(oracle.electrostatic.NuclearEFE) on the same mesh and composite rule, of
propagation steps that use it, and its properties on the Na8 workload at full
size."""
import math

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


def _oracle_vN(wl, sigma, r0, s, sub, n_quad=None):
    """The oracle's enriched nuclear potential at the quadrature points of every
    cell ([n_cells][n_q]) and its enrichment coefficients."""
    from oracle import electrostatic as es
    from oracle.mesh import Mesh
    m = Mesh(wl.xb, wl.yb, wl.zb, wl.degree, wl.n_quad)
    P = es.NuclearEFE(m, list(wl.Z), list(wl.R), sigma, r0=r0, s=s, sub=sub, n=n_quad)
    phi, phiE = P.solve()
    gl = es.CompositeRule(m, 1, m.nq1)
    out = np.empty((m.n_cells, m.nq))
    for c in range(m.n_cells):
        pts, _, Bc, G = gl.cell(m, c)
        vE, _ = P._enriched_at(c, pts, Bc, G)
        out[c] = Bc @ phi[m.conn[c]] + vE @ phiE
    return out, phiE


# (workload, sigma, r0, s, sub, n_quad): degrees 2 to 5, one and two atoms with
# overlapping supports, the plain cell rule (sub = 1) and finer composite rules
CASES = {
    "small2_p3_sub2": (lambda: W.small_cluster(n_atoms=2, cells_per_axis=5, degree=3, n_quad=5, n_orb=3),
                       0.3, 3.0, 1.5, 2, 0),
    "h2_p4_sub3": (lambda: W.h2(), 0.25, 3.0, 1.5, 3, 0),
    "small1_p2_sub1": (lambda: W.small_cluster(n_atoms=1, cells_per_axis=3, degree=2, n_quad=4, L=10.0, n_orb=11),
                       0.5, 3.0, 1.0, 1, 0),
    "small2_p5_sub2_n6": (lambda: W.small_cluster(n_atoms=2, cells_per_axis=3, degree=5, n_quad=7, n_orb=2, L=12.0),
                          0.3, 3.0, 1.5, 2, 6),
}


@pytest.mark.parametrize("name", list(CASES))
def test_nuclear_enriched_matches_oracle(name):
    from paper_2210_14421_gb300 import Context
    make, sigma, r0, s, sub, nq = CASES[name]
    wl = make()
    ref, ref_E = _oracle_vN(wl, sigma, r0, s, sub, nq or None)
    ctx = Context(wl)
    vN, phiE = ctx.nuclear_enriched(sigma, r0, s, sub=sub, n_quad=nq)
    got = vN.cpu().numpy()
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref)), name
    assert np.max(np.abs(phiE - ref_E)) <= 1e-10 * np.max(np.abs(ref_E)), (phiE, ref_E)
    ctx.close()


def test_steps_with_enriched_nucleus_match_oracle():
    """Kick + 2 predictor-corrector steps (fixed Krylov dimension) with the
    enriched nuclear potential installed: orbitals and dipoles to 1e-10."""
    from oracle import operators, tdks
    from paper_2210_14421_gb300 import Context
    make, sigma, r0, s, sub, nq = CASES["small2_p3_sub2"]
    wl = make()
    S = operators.System(wl)
    vN_ref, _ = _oracle_vN(wl, sigma, r0, s, sub)
    psi0 = S.initial_orbitals()
    psi = tdks.kick(S, psi0, wl.fields, wl.n_orb, tol=1e-14, k_max=8)
    st = tdks.make_state(S, psi, wl.occ, wl.batch)
    mus = []
    for n in range(2):
        psi, st, mu, _ = tdks.magnus_step(S, psi, st, n * wl.dt, wl.dt, wl.fields, wl.occ, 1e-14, 8, fixed_k=8,
                                          vN=vN_ref)
        mus.append(mu)
    ctx = Context(wl, fixed_k=8, krylov_tol=1e-14, k_max=8)
    ctx.nuclear_enriched(sigma, r0, s, sub=sub)
    g = torch.from_numpy(np.ascontiguousarray(psi0)).cuda()
    ctx.kick(g, wl.fields)
    m = torch.zeros((wl.batch, 3), dtype=torch.float64, device="cuda")
    got_mu = []
    for n in range(2):
        ctx.magnus_step(g, n * wl.dt, wl.dt, wl.fields, m)
        got_mu.append(m.cpu().numpy().copy())
    got = g.cpu().numpy()
    assert np.linalg.norm(got - psi) <= 1e-10 * np.linalg.norm(psi)
    ref_mu = np.array(mus)
    assert np.max(np.abs(np.array(got_mu) - ref_mu)) <= 1e-10 * max(np.max(np.abs(ref_mu)), 1e-3)
    ctx.close()


def test_nuclear_enriched_rejects_bad_arguments():
    from paper_2210_14421_gb300 import Context, EfeError
    wl = W.h2()
    ctx = Context(wl)
    for args in ((0.0, 3.0, 1.5, 2, 0),      # sigma
                 (0.25, 1.0, 1.5, 2, 0),     # r0 <= s
                 (0.25, 3.0, 1.5, 0, 0),     # sub
                 (0.25, 3.0, 1.5, 2, 4),     # n_quad < p + 1
                 (0.25, 9.0, 1.5, 2, 0)):    # support reaching the boundary (atoms 7.3 bohr inside)
        with pytest.raises(EfeError):
            ctx.nuclear_enriched(*args[:3], sub=args[3], n_quad=args[4])
    ctx.close()


def test_full_size_enriched_nucleus_properties():
    """Na8 at full size (31^3 graded cells, 1.95M nodes): the enriched
    smeared-nucleus potential stays close to its closed form, the exact
    potential of the smeared charges in free space (the Dirichlet data are
    exact; the smooth remainder is resolved by the graded mesh), and every
    enrichment coefficient is near 1 (the enrichment function is the core of
    the exact potential)."""
    from scipy.special import erf
    from paper_2210_14421_gb300 import Context
    wl = W.na8()
    sigma = 0.25
    ctx = Context(wl)
    vN, phiE = ctx.nuclear_enriched(sigma, 4.0, 2.0, sub=2)
    _, quad = ctx.coords()
    x = quad.cpu().numpy().reshape(-1, 3)
    exact = np.zeros(len(x))
    for z, R in zip(wl.Z, wl.R):
        r = np.linalg.norm(x - R[None, :], axis=1)
        exact -= z * erf(r / (math.sqrt(2.0) * sigma)) / r
    got = vN.cpu().numpy().ravel()
    assert np.all(np.isfinite(got))
    err = np.max(np.abs(got - exact)) / np.max(np.abs(exact))
    assert err < 1e-2, err
    assert np.all(np.abs(phiE - 1.0) < 0.1), phiE
    ctx.close()
    torch.cuda.empty_cache()
