"""The cell apply against the oracle at a size with the benchmark's cells: the Na8-like mesh
cropped to 15^3 cells (3,375 cells of degree 4, 227,029 DOF, 48 enrichment functions, cells
coupled to up to 48 of them, 44 complex orbitals = 88 real columns: the tensor-core apply's
column blocks, work items and persistent loop over many cells per SM all engaged).

Y = Hbar X (Eq. TDKSDiscrete2) against the oracle's D P^T H_ext P D, element by element.  The
rounding scale is that of the products as they are formed, |D P^T| |H_ext| |P D| |X|: with 48
enrichment functions the orthogonalised coupling -H^cc C^T + H^cA cancels terms up to ~2500
times larger than the entries of Hbar that remain (measured on this crop), so the assembled
|Hbar| |X| understates the rounding of either side.  FP64 within 1e-12 and float32 pairs within
1e-11 of that scale; the tensor-core form within 2e-7 of the same scale with max_j |X_j| in
place of |X_j| (its operands are rounded to 31 bits against per-cell column scales no larger
than the column's largest value)."""
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


def test_apply_on_the_15_cube_crop_matches_oracle():
    import scipy.sparse as sp
    from oracle import operators, tdks
    from paper_2210_14421_gb300 import EFE_FP64, EFE_PAIR, EFE_TC, Context
    wl = W.na_cluster(n_atoms=8, L=40.0, cells_per_axis=15)
    S = operators.System(wl)
    vq = tdks.nuclear_potential(S)
    H = S.hbar(vq)
    rng = np.random.default_rng(15)
    X = rng.normal(size=(S.n_dof, wl.n_orb)) + 1j * rng.normal(size=(S.n_dof, wl.n_orb))
    X[:S.n_h][S.mesh.boundary] = 0.0
    ref = H @ X
    Vcc, VcA, VAA = S.potential_blocks(vq)
    Hext = sp.bmat([[S.Kcc + Vcc, sp.csr_matrix(S.KcA + VcA)], [sp.csr_matrix((S.KcA + VcA).T),
                                                                 sp.csr_matrix(S.KAA + VAA)]], format="csr")
    aD, aP, aH = abs(S.D), abs(S.P), abs(Hext)

    def scale(V):
        return aD @ (aP.T @ (aH @ (aP @ (aD @ V))))

    bound = scale(np.abs(X))
    tcb = scale(np.ones((S.n_dof, 1))) * np.max(np.abs(X), axis=0)[None, :]
    ctx = Context(wl)
    assert ctx.n_dof == S.n_dof and ctx.n_pairs > 20000
    ctx.set_potential(torch.from_numpy(np.ascontiguousarray(vq[None])).cuda())
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    Yd = torch.empty_like(Xd)
    ctx.apply_H(Xd, Yd, precision=EFE_FP64)
    assert np.all(np.abs(Yd.cpu().numpy() - ref) <= 1e-12 * bound + 1e-300)
    ctx.apply_H(Xd, Yd, precision=EFE_PAIR)
    assert np.all(np.abs(Yd.cpu().numpy() - ref) <= 1e-11 * bound + 1e-300)
    ctx.apply_H(Xd, Yd, precision=EFE_TC)
    assert np.all(np.abs(Yd.cpu().numpy() - ref) <= 2e-7 * tcb + 1e-300)
    ctx.close()
