"""The checkpoint file of libefe on the host (no device): written from host arrays, read back
by the validator, and refused when damaged (corrupt byte, truncation, trailing bytes, foreign
magic) or incomplete (a state without all its parts)."""
import os

import numpy as np
import pytest


@pytest.fixture(scope="module")
def B():
    import __graft_entry__ as g
    g.build()
    from paper_2210_14421_gb300 import _binding
    return _binding


SIZES = (7, 3, 2, 4, 5, 6)   # n_dof, complex columns, batch, cells, points per cell, classical nodes


def _arrays(seed=0):
    rng = np.random.default_rng(seed)
    n_dof, C, batch, nc, nq, nh = SIZES
    return dict(psi=rng.normal(size=(n_dof, 2 * C)), rho=rng.random((batch, nc, nq)),
                vH=rng.normal(size=(batch, nc, nq)), vxc=rng.normal(size=(batch, nc, nq)),
                phi=rng.normal(size=(nh, batch)), vprev=rng.normal(size=(batch, nc, nq)))


def test_write_and_inspect(B, tmp_path):
    p = tmp_path / "run.ckpt"
    B.checkpoint_write_host(p, SIZES, 1.25, 25, **_arrays())
    sizes, t, step, has_state, has_prev = B.checkpoint_inspect(p)
    assert sizes == SIZES and t == 1.25 and step == 25 and has_state and has_prev
    assert not os.path.exists(str(p) + ".tmp")
    q = tmp_path / "orbitals_only.ckpt"
    B.checkpoint_write_host(q, SIZES, 0.0, 0, _arrays()["psi"])
    assert B.checkpoint_inspect(q)[3:] == (False, False)
    # header + payload, nothing more
    n_dof, C, batch, nc, nq, nh = SIZES
    payload = 8 * (2 * n_dof * C + 4 * batch * nc * nq + nh * batch)
    assert os.path.getsize(p) - payload == os.path.getsize(q) - 8 * 2 * n_dof * C


def test_damaged_files_are_refused(B, tmp_path):
    from paper_2210_14421_gb300 import EfeError
    p = tmp_path / "good.ckpt"
    B.checkpoint_write_host(p, SIZES, 1.0, 10, **_arrays())
    raw = p.read_bytes()
    cases = {
        "checksum": raw[:-9] + bytes([raw[-9] ^ 0x10]) + raw[-8:],   # one bit of the last payload double
        "truncated": raw[:-8],
        "trailing": raw + b"\0",
        "magic": b"EFECKPT2" + raw[8:],
        "header_only": raw[:40],
    }
    for name, data in cases.items():
        bad = tmp_path / (name + ".ckpt")
        bad.write_bytes(data)
        with pytest.raises(EfeError):
            B.checkpoint_inspect(bad)
    with pytest.raises(EfeError, match="cannot open"):
        B.checkpoint_inspect(tmp_path / "missing.ckpt")


def test_incomplete_state_is_refused(B, tmp_path):
    from paper_2210_14421_gb300 import EfeError
    a = _arrays()
    with pytest.raises(EfeError, match="together"):
        B.checkpoint_write_host(tmp_path / "x.ckpt", SIZES, 0.0, 0, a["psi"], rho=a["rho"])
    with pytest.raises(EfeError, match="previous potential"):
        B.checkpoint_write_host(tmp_path / "y.ckpt", SIZES, 0.0, 0, a["psi"], vprev=a["vprev"])


def test_null_path_is_refused_with_a_message(B):
    import ctypes as C
    L = B.lib()
    i64, i32 = C.c_int64, C.c_int32
    sz, t, step, hs, hp = (i64 * 6)(), C.c_double(), i64(), i32(), i32()
    st = L.efe_checkpoint_inspect(None, sz, C.byref(t), C.byref(step), C.byref(hs), C.byref(hp))
    assert st == B.EFE_ERR_ARG
    assert b"path is NULL" in L.efe_checkpoint_last_error()
