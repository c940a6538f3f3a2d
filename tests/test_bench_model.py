"""bench.py's algorithmic work model of the dominant kernel (the cell apply), checked on the
CPU against the definition written out by hand for the Na8-like workload: 29,791 cells of
degree 4 (N_n = 125 nodes), 232,002 cell-function pairs, 1,953,173 DOF, 44 orbitals (88 real
columns).  Work per apply: the dense cell contraction N_c 2 N_n^2 R plus the enrichment coupling
E_c x^E and E_c^T x^C, 4 N_n n_pairs R.  The roofline fraction is that work over the kernel's
CUDA-event time over the measured peak, so the figure in a bench line can be recomputed from
its own keys."""
from types import SimpleNamespace

import efe_workloads as W


def test_apply_model_matches_the_definition():
    import bench
    wl = W.na8()
    ctx = SimpleNamespace(n_cells=29791, n_pairs=232002, n_dof=1953173, n_nodes=1953125)
    assert wl.n_cells == ctx.n_cells and wl.n_dof == ctx.n_dof and wl.n_orb == 44
    R = 88
    flops_def = 29791 * 2 * 125 ** 2 * R + 4 * 125 * 232002 * R
    for prec in ("tc", "pair", "mixed", "fp64"):
        _, flops, _ = bench.apply_model(ctx, wl, prec)
        assert flops == flops_def == 92_133_338_000
    # tensor-core bytes: X and Y once in complex128, the four bf16 slices of every 128 x 128
    # cell matrix, and the slices of each pair's E_c and E_c^T blocks
    bytes_tc, _, issued = bench.apply_model(ctx, wl, "tc")
    assert bytes_tc == 2 * 1953173 * R * 8 + 29791 * 4 * 128 * 128 * 2 + 232002 * 2 * 4 * 125 * 2
    assert issued == 13 * 2 * R * (29791 * 128 * 128 + 2 * 128 * 232002)


def test_roofline_fraction_recomputes_from_the_line():
    """The measured Na8 line (k_tc_apply<5> at 7.7036 ms per launch against the sustained bf16
    peak of 1726.6 TFLOP/s) gives 11.96 TFLOP/s and a fraction of 0.00693."""
    achieved = 92_133_338_000 / 7.7036e-3 / 1e12
    assert abs(achieved - 11.96) < 0.01
    assert abs(achieved / 1726.6 - 0.00693) < 1e-5
