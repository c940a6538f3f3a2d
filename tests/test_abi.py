"""The C-ABI library loads and exports every entry point include/efe.h
declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "efe.h")).read()
    return sorted(set(re.findall(r"^(?:efe_status|const char\*)\s+(efe_\w+)\(", txt, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["efe_setup", "efe_apply_H", "efe_magnus_step", "efe_density_vxc", "efe_hartree",
                     "efe_dipole", "efe_destroy", "efe_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    import shutil
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available to build the library")
    from paper_2210_14421_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
    from paper_2210_14421_gb300 import EXPORTED
    assert sorted(EXPORTED) == _declared()


def test_setup_rejects_bad_arguments_without_gpu_work():
    """Argument validation happens before any device call."""
    import numpy as np
    from paper_2210_14421_gb300 import _binding as B
    lib = B.lib()
    xb = np.linspace(-1, 1, 3)
    mesh = B.MeshDesc(2, 2, 2, B._dptr(xb), B._dptr(xb), B._dptr(xb), 7, 9)   # degree 7 unsupported
    occ = np.ones(1)
    opts = B.Options(1, 1, B._dptr(occ), 1e-8, 8, 0, 1e-10, 100, 0)
    h = ctypes.c_void_p()
    st = lib.efe_setup(ctypes.byref(mesh), None, 0, None, ctypes.byref(opts), ctypes.byref(h))
    assert st == B.EFE_ERR_ARG
    assert b"degree" in lib.efe_last_error(None)
    mesh = B.MeshDesc(2, 2, 2, B._dptr(xb), B._dptr(xb), B._dptr(xb), 4, 6)
    opts = B.Options(1, 1, B._dptr(occ), 1e-8, 99, 0, 1e-10, 100, 0, 0)                # k_max too large
    st = lib.efe_setup(ctypes.byref(mesh), None, 0, None, ctypes.byref(opts), ctypes.byref(h))
    assert st == B.EFE_ERR_ARG


def test_missing_library_fails_loudly(tmp_path):
    """Without the built library the binding raises: there is no CPU fallback to fall into."""
    from paper_2210_14421_gb300 import _binding as B
    saved = B._lib
    try:
        B._lib = None
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            B.lib(str(tmp_path / "libefe.so"))
    finally:
        B._lib = saved


def test_plain_c_program_links_and_calls_the_library(tmp_path):
    """The boundary is a C ABI: a C99 program that includes include/efe.h alone links against
    libefe.so, takes the address of every declared entry point and makes a host-only call (no
    device work) whose status and message come back through C."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    import __graft_entry__ as g
    g.build()
    from paper_2210_14421_gb300 import _binding as B
    libdir = os.path.dirname(B.LIB_PATH)
    names = _declared()
    src = tmp_path / "use_efe.c"
    src.write_text(
        '#include <stdio.h>\n#include <string.h>\n#include "efe.h"\n'
        "typedef void (*fn_t)(void);\n"
        "int main(void) {\n"
        "  fn_t fns[] = {" + ", ".join("(fn_t)%s" % n for n in names) + "};\n"
        "  int n = 0;\n"
        "  for (size_t i = 0; i < sizeof fns / sizeof fns[0]; ++i) n += fns[i] != 0;\n"
        "  int64_t sizes[6]; double t; int64_t step; int32_t hs, hp;\n"
        "  efe_status st = efe_checkpoint_inspect(NULL, sizes, &t, &step, &hs, &hp);\n"
        '  printf("%d %d %s\\n", n, (int)st, efe_checkpoint_last_error());\n'
        "  return 0;\n}\n")
    exe = tmp_path / "use_efe"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(exe), str(B.LIB_PATH), "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split(maxsplit=2)
    assert int(out[0]) == len(names)
    assert int(out[1]) == B.EFE_ERR_ARG and "path is NULL" in out[2]
