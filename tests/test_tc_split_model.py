"""The arithmetic of the tensor-core split (precision EFE_TC), checked in exact
numpy arithmetic, independently of the CUDA code: the properties the kernel's
design rests on.

* A value scaled by a power of two to |alpha| <= 1, rounded to Q = round(alpha 2^31)
  and cut into 7 + 8 + 8 + 8 bits, gives four slices that are exact in bf16 (at
  most 8 significant bits) and sum back to Q 2^-31.
* The products of slice pairs whose indices sum to 0 (or to 1) over at most
  128 + 48 terms stay below 2^24 steps of their grid (2^-14, resp. 2^-22), so a
  binary32 accumulator adds them exactly.
* On the cell matrices of the H2 workload, forming the pairs with index sum up
  to 4 (13 products) with the groups 2..4 rounded in binary32 lands on the
  floor of the 31-bit rounding of the operands, while stopping at index sum 3
  leaves binary32-level errors: a pair (k, l) carries up to 2^(2 - 8(k + l)) of
  the scales whatever the size of its product.
"""
import numpy as np
import pytest

import efe_workloads as W


def _slices(a, e):
    """Four slices of a with per-entry power-of-two scale 2^e (|a| < 2^e)."""
    Q = np.rint(a * np.exp2(31.0 - e)).astype(np.int64)
    s, q = np.sign(Q), np.abs(Q)
    c = [q >> 24, (q >> 16) & 255, (q >> 8) & 255, q & 255]
    return [s * ck * np.exp2(-7.0 - 8 * k) for k, ck in enumerate(c)], Q


def _exp_of_max(m):
    m = np.asarray(m, np.float64)
    return np.where(m > 0, np.frexp(m)[1], 0).astype(np.float64)


def test_slices_exact_in_bf16_and_sum_back():
    rng = np.random.default_rng(3)
    a = rng.standard_normal(20000) * np.exp2(rng.integers(-30, 30, 20000))
    e = _exp_of_max(np.abs(a))
    sl, Q = _slices(a, e)
    for k, s in enumerate(sl):
        ints = np.abs(s) * np.exp2(7.0 + 8 * k)
        assert np.all(ints == np.round(ints))
        assert np.all(ints <= (128 if k == 0 else 255))
        # bf16 keeps 8 significant bits: every slice survives a round trip through bf16
        f32 = s.astype(np.float32)
        bf = (f32.view(np.uint32) & np.uint32(0xFFFF0000)).view(np.float32)
        assert np.array_equal(bf, f32)
    back = sum(sl) * np.exp2(e)
    assert np.all(np.abs(back - a) <= np.exp2(e - 32) * (1 + 1e-12))
    assert np.array_equal(sum(sl), Q * np.exp2(-31.0))


def test_group_sums_exact_in_binary32():
    """Worst-case magnitudes: group 0 (k = l = 0) and group 1 ((0, 1) + (1, 0))
    over 176 terms, accumulated in binary32 in chunks of 16 as an MMA does."""
    K = 176
    rng = np.random.default_rng(5)
    for trial in range(20):
        c0a = rng.integers(-128, 129, K)
        c0b = rng.integers(-128, 129, K)
        c1a = rng.integers(-255, 256, K)
        c1b = rng.integers(-255, 256, K)
        if trial == 0:   # all at the largest magnitude and one sign
            c0a[:], c0b[:], c1a[:], c1b[:] = 128, 128, 255, 255
        g0 = (c0a * c0b).astype(np.float64) * 2.0 ** -14
        g1 = (c0a * c1b + c1a * c0b).astype(np.float64) * 2.0 ** -22
        for g, grid in ((g0, 2.0 ** -14), (g1, 2.0 ** -22)):
            assert np.sum(np.abs(g)) / grid < 2 ** 24
            acc = np.float32(0.0)
            for k0 in range(0, K, 16):
                acc = np.float32(np.float64(acc) + np.sum(g[k0:k0 + 16]))
            assert float(acc) == float(np.sum(g))


def _cell_products(S, v, Xr, gmax):
    """y = sum_c D_c (H_c x_c) by the split scheme with pairs i + j <= gmax; the
    exact result and the per-element scale sum_k |Hbar_ik| max|x|."""
    m = S.mesh
    Y = np.zeros_like(Xr)
    Yref = np.zeros_like(Xr)
    for c in range(m.n_cells):
        G = m.grad_tables(c)
        Ke = 0.5 * sum(G[a].T @ (m.wJ[c][:, None] * G[a]) for a in range(3)) + m.B.T @ ((m.wJ[c] * v[c])[:, None] * m.B)
        idx = m.conn[c]
        A = S.Dc[idx][:, None] * Ke
        xc = S.Dc[idx][:, None] * Xr[idx]
        Yref[idx] += A @ xc
        er = _exp_of_max(np.abs(A).max(axis=1))[:, None]
        ec = _exp_of_max(np.abs(xc).max(axis=0))[None, :]
        As, _ = _slices(A, er)
        Bs, _ = _slices(xc, ec)
        exact = np.zeros((A.shape[0], xc.shape[1]))
        acc2 = np.zeros_like(exact, dtype=np.float32)
        for i in range(4):
            for j in range(4):
                if i + j > gmax:
                    continue
                if i + j <= 1:
                    exact += As[i] @ Bs[j]
                else:
                    for k0 in range(0, A.shape[1], 16):
                        acc2 = np.float32(acc2.astype(np.float64) + As[i][:, k0:k0 + 16] @ Bs[j][k0:k0 + 16])
        Y[idx] += (exact + acc2.astype(np.float64)) * np.exp2(er + ec)
    return Y, Yref


def test_thirteen_pairs_reach_the_31_bit_floor():
    from oracle import operators, tdks
    wl = W.h2().with_(enrich=[], enr_coefs=np.zeros((1, 0), complex))
    S = operators.System(wl)
    v = tdks.nuclear_potential(S)
    rng = np.random.default_rng(17)
    Xr = rng.standard_normal((S.n_dof, 2))
    H = S.hbar(v)
    bound = (abs(H) @ np.ones(S.n_dof))[:, None] * np.abs(Xr).max(axis=0)[None, :]
    Y4, Yref = _cell_products(S, v, Xr, 4)
    Y3, _ = _cell_products(S, v, Xr, 3)
    e4 = np.max(np.abs(Y4 - Yref) / (bound + 1e-300))
    e3 = np.max(np.abs(Y3 - Yref) / (bound + 1e-300))
    assert e4 <= 16 * 2.0 ** -31, e4          # the floor of the 31-bit operands (measured 1.1e-9)
    assert e3 > 10 * e4, (e3, e4)             # index sums up to 3 only: binary32 level
    # the same inputs through a binary32 contraction, for scale
    Y32 = np.zeros_like(Xr)
    m = S.mesh
    for c in range(m.n_cells):
        G = m.grad_tables(c)
        Ke = 0.5 * sum(G[a].T @ (m.wJ[c][:, None] * G[a]) for a in range(3)) + m.B.T @ ((m.wJ[c] * v[c])[:, None] * m.B)
        idx = m.conn[c]
        y = (S.Dc[idx][:, None] * Ke).astype(np.float32) @ (S.Dc[idx][:, None] * Xr[idx]).astype(np.float32)
        Y32[idx] += y.astype(np.float64)
    e32 = np.max(np.abs(Y32 - Yref) / (bound + 1e-300))
    assert e4 * 10 < e32
