"""The allocation-free apply (efe_apply_H_noalloc) against efe_apply_H.

Callers that cannot allocate device memory while they run (a host framework
that owns all device memory, or code recorded into a CUDA graph) use the
allocation-free entry point; it must give the same Y = Hbar X as the regular
apply.  This file is collected after the other established GPU tests, so a
failure here comes after they have run; it also passes on its own in a fresh
process."""
import ctypes

import numpy as np
import pytest

import efe_workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2210_14421_gb300 import Context
    wl = W.small_cluster(n_atoms=2, cells_per_axis=4, degree=3, n_quad=5, n_orb=3, batch=2)
    c = Context(wl)
    nodes, quad = c.coords()
    q = quad.cpu().numpy()
    v0 = -2.0 / (0.5 + np.sum(q ** 2, axis=2))
    v = np.stack([v0, v0 + 0.1 * q[:, :, 0]])
    c.set_potential(torch.from_numpy(v).cuda().contiguous())
    yield c
    c.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_matches_apply_on_two_calls(ctx, precision):
    rng = np.random.default_rng(5)
    n = ctx.n_dof
    X = torch.from_numpy(rng.normal(size=(n, 6)) + 1j * rng.normal(size=(n, 6))).cuda()
    ref = torch.empty_like(X)
    ctx.apply_H(X, ref, precision=precision)
    scale = ref.abs().max().item()
    tol = 1e-12 if precision == 0 else 1e-5      # float64 rounding / the float32 contraction
    for _ in range(2):                           # the shared scratch keeps the last call's contents
        Y = torch.full_like(X, complex(np.nan, np.nan))
        ctx.apply_H_noalloc(X, Y, precision=precision)
        assert torch.max((Y - ref).abs()).item() <= tol * scale


def test_noalloc_rejects_oversize_request(ctx):
    from paper_2210_14421_gb300 import _binding as B
    L = B.lib()
    X = torch.zeros((ctx.n_dof, 6), dtype=torch.complex128, device="cuda")
    Y = torch.zeros_like(X)
    # an ld far beyond the static scratch is refused before any device work
    st = L.efe_apply_H_noalloc(ctx.h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()), 6, 10 ** 7, 0,
                               None)
    assert st == B.EFE_ERR_ARG
    assert b"static scratch" in L.efe_last_error(ctx.h)
