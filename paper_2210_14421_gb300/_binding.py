"""ctypes binding of libefe (include/efe.h): the same entry points, with torch
tensors marshalled to device pointers.  No numerical step runs here: every
call goes to the CUDA library, and loading fails loudly if it is missing."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libefe.so")

EFE_OK, EFE_ERR_ARG, EFE_ERR_NOMEM, EFE_ERR_CUDA, EFE_ERR_NOT_SPD = 0, 1, 2, 3, 4
EFE_WARN_KRYLOV_CAP, EFE_ERR_CG_NOCONV, EFE_ERR_TIMEOUT, EFE_ERR_STATE = 5, 6, 7, 8
EFE_FP64, EFE_MIXED, EFE_PAIR, EFE_TC = 0, 1, 2, 3
EFE_HARTREE_FDM, EFE_HARTREE_PCG = 0, 1
EFE_XC_PW92, EFE_XC_PZ81 = 0, 1
EFE_STEP_PC, EFE_STEP_EXTRAPOLATED = 0, 1
STATUS_NAMES = {0: "EFE_OK", 1: "EFE_ERR_ARG", 2: "EFE_ERR_NOMEM", 3: "EFE_ERR_CUDA", 4: "EFE_ERR_NOT_SPD",
                5: "EFE_WARN_KRYLOV_CAP", 6: "EFE_ERR_CG_NOCONV", 7: "EFE_ERR_TIMEOUT", 8: "EFE_ERR_STATE"}

EXPORTED = ["efe_setup", "efe_destroy", "efe_last_error", "efe_sizes", "efe_coords", "efe_set_potential",
            "efe_apply_H", "efe_magnus_step", "efe_reset_state", "efe_density_vxc", "efe_hartree", "efe_dipole",
            "efe_kick", "efe_init_orbitals", "efe_profile", "efe_profile_read", "efe_selftest",
            "efe_apply_H_noalloc", "efe_tuning", "efe_adjoint_dipole",
            "efe_absorption_spectrum", "efe_power_spectrum", "efe_nuclear_enriched",
            "efe_hartree_enriched", "efe_octree_setup", "efe_octree_destroy", "efe_octree_last_error",
            "efe_octree_sizes", "efe_octree_coords", "efe_octree_apply", "efe_octree_constraints",
            "efe_atom_hartree_table", "efe_adaptive_cell_boxes", "efe_octree_poisson",
            "efe_octree_density", "efe_octree_kexp", "efe_octree_interp", "efe_lda_points",
            "efe_octree_magnus_step", "efe_pipe_peaks", "efe_checkpoint_save", "efe_checkpoint_load",
            "efe_checkpoint_write_host", "efe_checkpoint_inspect", "efe_checkpoint_last_error",
            "efe_set_wait_limit", "efe_set_density_reduce", "efe_krylov_basis"]


class MeshDesc(C.Structure):
    _fields_ = [("ncx", C.c_int32), ("ncy", C.c_int32), ("ncz", C.c_int32), ("xb_host", C.POINTER(C.c_double)),
                ("yb_host", C.POINTER(C.c_double)), ("zb_host", C.POINTER(C.c_double)), ("degree", C.c_int32),
                ("n_quad", C.c_int32)]


class Atom(C.Structure):
    _fields_ = [("Z", C.c_double), ("R", C.c_double * 3)]


class EnrichFn(C.Structure):
    _fields_ = [("atom", C.c_int32), ("n", C.c_int32), ("l", C.c_int32), ("m", C.c_int32), ("radial", C.c_int32),
                ("zeta", C.c_double)]


class EnrichDesc(C.Structure):
    _fields_ = [("n_fn", C.c_int32), ("fns_host", C.POINTER(EnrichFn)), ("r0", C.c_double), ("s", C.c_double)]


class Field(C.Structure):
    _fields_ = [("kind", C.c_int32), ("amp", C.c_double), ("omega", C.c_double), ("t0", C.c_double),
                ("sigma", C.c_double), ("period", C.c_double), ("ramp", C.c_double), ("dir", C.c_double * 3),
                ("kick", C.c_double)]


class Options(C.Structure):
    _fields_ = [("n_orb", C.c_int32), ("batch", C.c_int32), ("occ_host", C.POINTER(C.c_double)),
                ("krylov_tol", C.c_double), ("k_max", C.c_int32), ("fixed_k", C.c_int32), ("cg_tol", C.c_double),
                ("cg_max_it", C.c_int32), ("precision", C.c_int32), ("hartree_method", C.c_int32),
                ("use_graphs", C.c_int32), ("xc", C.c_int32), ("scheme", C.c_int32), ("krylov_block", C.c_int32),
                ("krylov_substeps", C.c_int32), ("krylov_reorth", C.c_int32)]


class StepInfo(C.Structure):
    _fields_ = [("k_pred_max", C.c_int32), ("k_corr_max", C.c_int32), ("krylov_cap_hit", C.c_int32),
                ("cg_iters", C.c_int32), ("eps_max", C.c_double), ("substeps", C.c_int32)]


_lib = None


def lib(path: str = LIB_PATH):
    """Loads libefe.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libefe.so not found at %s: build it with `python -c \"import __graft_entry__ as g; "
                           "g.build()\"`; there is no CPU fallback" % path)
    L = C.CDLL(path)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    pdbl = C.POINTER(C.c_double)
    L.efe_setup.argtypes = [C.POINTER(MeshDesc), C.POINTER(Atom), i32, C.POINTER(EnrichDesc), C.POINTER(Options),
                            C.POINTER(vp)]
    L.efe_destroy.argtypes = [vp]
    L.efe_last_error.argtypes = [vp]
    L.efe_last_error.restype = C.c_char_p
    L.efe_sizes.argtypes = [vp] + [C.POINTER(i64)] * 5
    L.efe_coords.argtypes = [vp, vp, vp, vp]
    L.efe_set_potential.argtypes = [vp, vp, i32, dbl, vp]
    L.efe_apply_H.argtypes = [vp, vp, vp, i64, i64, i32, vp]
    L.efe_apply_H_noalloc.argtypes = [vp, vp, vp, i64, i64, i32, vp]
    L.efe_magnus_step.argtypes = [vp, vp, dbl, dbl, C.POINTER(Field), vp, C.POINTER(StepInfo), vp]
    L.efe_reset_state.argtypes = [vp]
    L.efe_density_vxc.argtypes = [vp, vp, vp, vp, vp, vp]
    L.efe_hartree.argtypes = [vp, vp, vp, dbl, i32, C.POINTER(i32), vp]
    L.efe_dipole.argtypes = [vp, vp, vp, vp]
    L.efe_kick.argtypes = [vp, vp, C.POINTER(Field), vp]
    L.efe_init_orbitals.argtypes = [vp, vp, i32, pdbl, pdbl, pdbl, pdbl, vp]
    L.efe_profile.argtypes = [vp, i32]
    L.efe_selftest.argtypes = [i64, C.POINTER(i64)]
    L.efe_pipe_peaks.argtypes = [pdbl, pdbl]
    L.efe_checkpoint_save.argtypes = [vp, C.c_char_p, vp, dbl, i64, vp]
    L.efe_checkpoint_load.argtypes = [vp, C.c_char_p, vp, pdbl, C.POINTER(i64), vp]
    L.efe_checkpoint_write_host.argtypes = [C.c_char_p, C.POINTER(i64), dbl, i64, vp, vp, vp, vp, vp, vp]
    L.efe_checkpoint_inspect.argtypes = [C.c_char_p, C.POINTER(i64), pdbl, C.POINTER(i64), C.POINTER(i32),
                                         C.POINTER(i32)]
    L.efe_set_wait_limit.argtypes = [vp, i64]
    L.efe_set_density_reduce.argtypes = [vp, ReduceFn, vp]
    L.efe_krylov_basis.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(i64)]
    L.efe_checkpoint_last_error.argtypes = []
    L.efe_checkpoint_last_error.restype = C.c_char_p
    L.efe_tuning.argtypes = [vp, i32, i32, C.POINTER(i32), C.POINTER(C.c_float), C.POINTER(C.c_float)]
    L.efe_profile_read.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(dbl)]
    L.efe_absorption_spectrum.argtypes = [vp, i64, i64, i64, dbl, vp, dbl, vp, i64, dbl, vp, vp]
    L.efe_power_spectrum.argtypes = [vp, i64, i64, dbl, vp, i64, dbl, vp, vp]
    L.efe_adjoint_dipole.argtypes = [vp, vp, i32, dbl, C.POINTER(Field), pdbl, i32, i32, i32, i32, C.POINTER(dbl),
                                     pdbl, vp]
    L.efe_nuclear_enriched.argtypes = [vp, dbl, dbl, dbl, i32, i32, dbl, i32, vp, pdbl, vp]
    L.efe_hartree_enriched.argtypes = [vp, dbl, dbl, i32, i32, vp]
    L.efe_octree_setup.argtypes = [pdbl, pdbl, i32, i32, i32, C.POINTER(i32), i32, C.POINTER(vp)]
    L.efe_octree_destroy.argtypes = [vp]
    L.efe_octree_last_error.argtypes = [vp]
    L.efe_octree_last_error.restype = C.c_char_p
    L.efe_octree_sizes.argtypes = [vp] + [C.POINTER(i64)] * 5
    L.efe_octree_coords.argtypes = [vp, pdbl, pdbl, C.POINTER(C.c_uint8)]
    L.efe_octree_apply.argtypes = [vp, vp, dbl, vp, vp, i64, i32, vp]
    L.efe_octree_constraints.argtypes = [pdbl, pdbl, i32, i32, i32, C.POINTER(i32), i32, C.POINTER(i64),
                                         C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(i32), pdbl, pdbl,
                                         pdbl]
    L.efe_octree_poisson.argtypes = [vp, vp, vp, vp, dbl, i32, C.POINTER(i32), vp]
    L.efe_octree_density.argtypes = [vp, vp, i32, pdbl, vp, vp]
    L.efe_octree_kexp.argtypes = [vp, vp, dbl, vp, i32, dbl, i32, dbl, C.POINTER(i32), vp]
    L.efe_octree_interp.argtypes = [vp, vp, i32, vp, vp]
    L.efe_lda_points.argtypes = [vp, vp, vp, i64, i32, vp]
    L.efe_octree_magnus_step.argtypes = [vp, vp, i32, pdbl, pdbl, i32, pdbl, dbl, i32, dbl, dbl, i32, vp]
    L.efe_atom_hartree_table.argtypes = [C.POINTER(EnrichFn), i32, pdbl, i32, i32, dbl, pdbl, pdbl, pdbl, pdbl]
    L.efe_adaptive_cell_boxes.argtypes = [pdbl, pdbl, pdbl, i32, dbl, dbl, dbl, i32, dbl, i32, C.POINTER(i64), pdbl,
                                          i64]
    for name in EXPORTED:
        if name not in ("efe_last_error", "efe_octree_last_error", "efe_checkpoint_last_error"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def selftest(n: int = 1 << 24) -> int:
    """Mismatches of the integer-pipe float conversions against the hardware ones."""
    m = C.c_int64()
    st = lib().efe_selftest(int(n), C.byref(m))
    if st != EFE_OK:
        raise EfeError(st, lib().efe_last_error(None).decode())
    return m.value


def checkpoint_write_host(path, sizes, t, step, psi, rho=None, vH=None, vxc=None, phi=None, vprev=None):
    """Writes a checkpoint file from host float64 arrays (see efe_checkpoint_write_host)."""
    arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in (psi, rho, vH, vxc, phi, vprev)]
    sz = (C.c_int64 * 6)(*[int(x) for x in sizes])
    ptrs = [None if a is None else a.ctypes.data_as(C.c_void_p) for a in arrs]
    st = lib().efe_checkpoint_write_host(str(path).encode(), sz, float(t), int(step), *ptrs)
    if st != EFE_OK:
        raise EfeError(st, lib().efe_checkpoint_last_error().decode())


def checkpoint_inspect(path):
    """(sizes, t, step, has_state, has_prev) of a valid checkpoint file; raises EfeError otherwise."""
    sz = (C.c_int64 * 6)()
    t, step, hs, hp = C.c_double(), C.c_int64(), C.c_int32(), C.c_int32()
    st = lib().efe_checkpoint_inspect(str(path).encode(), sz, C.byref(t), C.byref(step), C.byref(hs), C.byref(hp))
    if st != EFE_OK:
        raise EfeError(st, lib().efe_checkpoint_last_error().decode())
    return tuple(sz), t.value, step.value, bool(hs.value), bool(hp.value)


def pipe_peaks():
    """Measured float32 and float64 FMA-pipe throughput of the current device (TFLOP/s)."""
    a, b = C.c_double(), C.c_double()
    st = lib().efe_pipe_peaks(C.byref(a), C.byref(b))
    if st != EFE_OK:
        raise EfeError(st, "efe_pipe_peaks failed")
    return a.value, b.value


class EfeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


# int fn(double* rho_dev, int64_t n, void* stream, void* user): the density reduction callback
ReduceFn = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p)


class _DeviceArray:
    """A vector in device memory the library owns (float64, or another type string), seen by torch
    without a copy."""

    def __init__(self, ptr: int, n: int, typestr: str = "<f8"):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 2, "strides": None}


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def fields_array(fields):
    arr = (Field * len(fields))()
    for i, f in enumerate(fields):
        arr[i].kind = int(f.kind)
        arr[i].amp, arr[i].omega, arr[i].t0 = float(f.amp), float(f.omega), float(f.t0)
        arr[i].sigma, arr[i].period, arr[i].ramp = float(f.sigma), float(f.period), float(f.ramp)
        for k in range(3):
            arr[i].dir[k] = float(f.direction[k])
        arr[i].kick = float(f.kick)
    return arr


def absorption_spectrum(mu, dt, omegas, tau, field=None, kick=None):
    """S(w) from three dipole traces on the device: mu[j, n, k] = component k of the
    dipole at t = n dt of the run perturbed along axis j (float64, any strides with
    the component innermost); field: E_0 samples [n_t] or None with kick."""
    import torch
    assert mu.dtype == torch.float64 and mu.is_cuda and mu.dim() == 3 and mu.shape[0] == 3 and mu.stride(2) == 1
    out = torch.empty(omegas.shape[0], dtype=torch.float64, device=mu.device)
    st = lib().efe_absorption_spectrum(_ptr(mu), int(mu.shape[1]), int(mu.stride(0)), int(mu.stride(1)), float(dt),
                                       _ptr(field), float(kick or 0.0), _ptr(omegas), int(omegas.shape[0]),
                                       float(tau), _ptr(out), _stream())
    if st != EFE_OK:
        raise EfeError(st, lib().efe_last_error(None).decode())
    return out


def power_spectrum(mu_x, dt, omegas, tau):
    """P(w) of the dipole acceleration from one trace mu_x[n] on the device."""
    import torch
    assert mu_x.dtype == torch.float64 and mu_x.is_cuda and mu_x.dim() == 1
    out = torch.empty(omegas.shape[0], dtype=torch.float64, device=mu_x.device)
    st = lib().efe_power_spectrum(_ptr(mu_x), int(mu_x.shape[0]), int(mu_x.stride(0)), float(dt), _ptr(omegas),
                                  int(omegas.shape[0]), float(tau), _ptr(out), _stream())
    if st != EFE_OK:
        raise EfeError(st, lib().efe_last_error(None).decode())
    return out


class Context:
    """Owns one efe_ctx built from an `efe_workloads.Workload`."""

    def __init__(self, wl, precision: int = EFE_FP64, krylov_tol=None, k_max=None, fixed_k: int = 0,
                 cg_tol: float = 1e-12, cg_max_it: int = 5000, hartree_method: int = EFE_HARTREE_FDM,
                 use_graphs: bool = False, xc: int = EFE_XC_PW92, scheme: int = EFE_STEP_PC,
                 krylov_block: int = 0, krylov_substeps: int = 1, krylov_reorth: bool = False):
        L = lib()
        self.wl = wl
        self._keep = []
        xb, yb, zb = (np.ascontiguousarray(b, dtype=np.float64) for b in (wl.xb, wl.yb, wl.zb))
        self._keep += [xb, yb, zb]
        mesh = MeshDesc(len(xb) - 1, len(yb) - 1, len(zb) - 1, _dptr(xb), _dptr(yb), _dptr(zb), int(wl.degree),
                        int(wl.n_quad))
        na = len(wl.Z)
        atoms = (Atom * max(na, 1))()
        for i in range(na):
            atoms[i].Z = float(wl.Z[i])
            for k in range(3):
                atoms[i].R[k] = float(wl.R[i][k])
        fns = (EnrichFn * max(len(wl.enrich), 1))()
        for i, f in enumerate(wl.enrich):
            fns[i] = EnrichFn(int(f.atom), int(f.n), int(f.l), int(f.m), int(f.radial), float(f.zeta))
        enr = EnrichDesc(len(wl.enrich), fns, float(wl.r0), float(wl.s))
        occ = np.ascontiguousarray(wl.occ, dtype=np.float64)
        self._keep.append(occ)
        opts = Options(int(wl.n_orb), int(wl.batch), _dptr(occ),
                       float(wl.krylov_tol if krylov_tol is None else krylov_tol),
                       int(wl.k_max if k_max is None else k_max), int(fixed_k), float(cg_tol), int(cg_max_it),
                       int(precision), int(hartree_method), int(bool(use_graphs)), int(xc), int(scheme),
                       int(krylov_block), int(krylov_substeps), int(bool(krylov_reorth)))
        h = C.c_void_p()
        st = L.efe_setup(C.byref(mesh), atoms, na, C.byref(enr), C.byref(opts), C.byref(h))
        if st != EFE_OK:
            raise EfeError(st, L.efe_last_error(None).decode())
        self.h = h
        v = [C.c_int64() for _ in range(5)]
        L.efe_sizes(self.h, *[C.byref(x) for x in v])
        self.n_nodes, self.n_enrich, self.n_cells, self.n_q, self.n_pairs = (x.value for x in v)
        self.n_dof = self.n_nodes + self.n_enrich
        self.n_cols = wl.n_orb * wl.batch

    def _check(self, st, allow=(EFE_OK,)):
        if st not in allow:
            exc, self._reduce_exc = getattr(self, "_reduce_exc", None), None
            if exc is not None:
                raise exc
            raise EfeError(st, lib().efe_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            lib().efe_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- entry points (same names as the C ABI, without the prefix)
    def coords(self):
        import torch
        nodes = torch.empty((self.n_nodes, 3), dtype=torch.float64, device="cuda")
        quad = torch.empty((self.n_cells, self.n_q, 3), dtype=torch.float64, device="cuda")
        self._check(lib().efe_coords(self.h, _ptr(nodes), _ptr(quad), _stream()))
        return nodes, quad

    def set_potential(self, v, kin_scale: float = 1.0):
        assert v.is_cuda and v.dtype.is_floating_point and v.is_contiguous()
        batch = v.shape[0] if v.dim() == 3 else 1
        self._check(lib().efe_set_potential(self.h, _ptr(v), int(batch), float(kin_scale), _stream()))

    def apply_H(self, X, Y, precision: int = EFE_FP64):
        """X, Y: complex128 [n_dof, n_cols] (or any ld >= n_cols) on the device."""
        n_cols = X.shape[1]
        ld = X.stride(0)
        assert Y.stride(0) == ld and X.dtype == Y.dtype
        self._check(lib().efe_apply_H(self.h, _ptr(X), _ptr(Y), int(n_cols), int(ld), int(precision), _stream()))
        return Y

    def apply_H_noalloc(self, X, Y, precision: int = EFE_FP64):
        """Same as apply_H, with the library's static scratch (no device allocation)."""
        n_cols = X.shape[1]
        ld = X.stride(0)
        assert Y.stride(0) == ld and X.dtype == Y.dtype
        self._check(lib().efe_apply_H_noalloc(self.h, _ptr(X), _ptr(Y), int(n_cols), int(ld), int(precision),
                                              _stream()))
        return Y

    def magnus_step(self, psi, t, dt, fields, mu=None):
        info = StepInfo()
        arr = fields_array(fields)
        st = lib().efe_magnus_step(self.h, _ptr(psi), float(t), float(dt), arr, _ptr(mu), C.byref(info), _stream())
        self._check(st, allow=(EFE_OK, EFE_WARN_KRYLOV_CAP))
        return {"k_pred": info.k_pred_max, "k_corr": info.k_corr_max, "cap": info.krylov_cap_hit,
                "cg_iters": info.cg_iters, "eps_max": info.eps_max, "substeps": info.substeps, "status": st}

    def magnus_step_async(self, psi, t, dt, fields_arr, mu=None):
        """Same as magnus_step with a prepared field array and no host-visible info."""
        st = lib().efe_magnus_step(self.h, _ptr(psi), float(t), float(dt), fields_arr, _ptr(mu), None, _stream())
        return self._check(st, allow=(EFE_OK, EFE_WARN_KRYLOV_CAP))

    def reset_state(self):
        self._check(lib().efe_reset_state(self.h))

    def set_wait_limit(self, polls: int):
        """Polls before a tensor-core progress wait gives up (0: the default); for timeout tests."""
        self._check(lib().efe_set_wait_limit(self.h, int(polls)))

    def set_density_reduce(self, fn):
        """Orbital partition across processes: fn(rho) must replace the device float64 tensor
        rho (this context's partial density, [batch * n_cells * n_q]) by its sum over all
        processes, e.g. ``torch.distributed.all_reduce``; it runs with the step's stream as
        torch's current stream.  None removes it.  An exception raised by fn ends the step and
        is raised again by the call that ran it."""
        if fn is None:
            self._reduce_cb = None
            self._check(lib().efe_set_density_reduce(self.h, ReduceFn(), None))
            return
        import torch

        def cb(ptr, n, stream, _user):
            try:
                rho = torch.as_tensor(_DeviceArray(ptr, n), device="cuda")
                ext = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
                with torch.cuda.stream(ext):
                    fn(rho)
                return 0
            except BaseException as e:   # noqa: BLE001 -- handed back to the caller of the step
                self._reduce_exc = e
                return 1

        self._reduce_cb = ReduceFn(cb)   # kept alive as long as the library may call it
        self._check(lib().efe_set_density_reduce(self.h, self._reduce_cb, None))

    def krylov_orthogonality(self, n_cols: int = 4):
        """Diagnostics: max |Q^H Q - I| over the normalised Lanczos vectors q_j = V_j / s_j of the
        first n_cols columns of the last Lanczos run, and the vectors each used."""
        import torch
        q, nr, ku, c = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_int64()
        self._check(lib().efe_krylov_basis(self.h, C.byref(q), C.byref(nr), C.byref(ku), C.byref(c)))
        cols = c.value
        kused = torch.as_tensor(_DeviceArray(ku.value, cols, "<i4"), device="cuda").cpu().tolist()
        kmax = max(kused)
        norms = torch.as_tensor(_DeviceArray(nr.value, kmax * cols), device="cuda").view(kmax, cols)
        V = torch.as_tensor(_DeviceArray(q.value, kmax * self.n_dof * cols * 2), device="cuda")
        V = torch.view_as_complex(V.view(kmax, self.n_dof, cols, 2))
        worst, ks = 0.0, []
        for col in range(min(n_cols, cols)):
            k = kused[col]
            if k < 2:
                continue
            s = torch.ones(k, dtype=torch.float64, device="cuda")
            s[1:] = norms[:k - 1, col]   # |V_j| = beta_{j-1}
            Qn = V[:k, :, col] / s[:, None]
            G = Qn.conj() @ Qn.T
            worst = max(worst, (G - torch.eye(k, dtype=G.dtype, device="cuda")).abs().max().item())
            ks.append(k)
        return worst, ks

    def checkpoint_save(self, path, psi, t, step):
        self._check(lib().efe_checkpoint_save(self.h, str(path).encode(), _ptr(psi), float(t), int(step), _stream()))

    def checkpoint_load(self, path, psi):
        """Restores psi (device, in place) and the state; returns (t, step)."""
        t, step = C.c_double(), C.c_int64()
        self._check(lib().efe_checkpoint_load(self.h, str(path).encode(), _ptr(psi), C.byref(t), C.byref(step),
                                              _stream()))
        return t.value, step.value

    def density_vxc(self, psi, rho, vxc=None, exc=None):
        self._check(lib().efe_density_vxc(self.h, _ptr(psi), _ptr(rho), _ptr(vxc), _ptr(exc), _stream()))

    def hartree(self, rho, vH, tol=1e-12, max_it=5000):
        its = C.c_int32()
        st = lib().efe_hartree(self.h, _ptr(rho), _ptr(vH), float(tol), int(max_it), C.byref(its), _stream())
        self._check(st)
        return its.value

    def dipole(self, rho, mu):
        self._check(lib().efe_dipole(self.h, _ptr(rho), _ptr(mu), _stream()))

    def nuclear_enriched(self, sigma: float, r0: float, s: float, sub: int = 2, n_quad: int = 0,
                         adapt_tol: float = 0.0, adapt_depth: int = 4):
        """Installs the nuclear potential of Gaussian-smeared nuclei solved in the
        electrostatically enriched basis (cell integrals on sub^3 boxes, or on the
        adaptive rule when adapt_tol > 0); returns it at the quadrature points
        (device float64 [n_cells, n_q]) and the enrichment coefficients (numpy [n_atoms])."""
        import torch
        vN = torch.empty((self.n_cells, self.n_q), dtype=torch.float64, device="cuda")
        phiE = np.zeros(len(self.wl.Z))
        self._check(lib().efe_nuclear_enriched(self.h, float(sigma), float(r0), float(s), int(sub), int(n_quad),
                                               float(adapt_tol), int(adapt_depth), _ptr(vN), _dptr(phiE), _stream()))
        return vN, phiE

    def hartree_enriched(self, r0: float, s: float, sub: int = 2, n_quad: int = 0):
        """Installs the enriched Hartree solve (atomic Hartree potentials as enrichment)
        for every later Hartree solve of the context."""
        self._check(lib().efe_hartree_enriched(self.h, float(r0), float(s), int(sub), int(n_quad), _stream()))

    def kick(self, psi, fields):
        st = lib().efe_kick(self.h, _ptr(psi), fields_array(fields), _stream())
        return self._check(st, allow=(EFE_OK, EFE_WARN_KRYLOV_CAP))

    def adjoint_dipole(self, psi0, n_steps, dt, field, direction, window, checkpoint_every: int = 4,
                       n_quad_s: int = 8):
        """(J, dJ/d(amp, omega, sigma)) of the window-averaged dipole d . mu over steps
        window = (first, last) from psi0 (device complex128 [n_dof, n_orb])."""
        d = np.ascontiguousarray(direction, dtype=np.float64)
        g = np.zeros(3)
        J = C.c_double()
        st = lib().efe_adjoint_dipole(self.h, _ptr(psi0), int(n_steps), float(dt), fields_array([field]), _dptr(d),
                                      int(window[0]), int(window[1]), int(checkpoint_every), int(n_quad_s),
                                      C.byref(J), _dptr(g), _stream())
        self._check(st, allow=(EFE_OK, EFE_WARN_KRYLOV_CAP))
        return J.value, g

    def tuning(self, precision: int = EFE_MIXED, force_variant: int = -1):
        v, a, b = C.c_int32(), C.c_float(), C.c_float()
        self._check(lib().efe_tuning(self.h, int(precision), int(force_variant), C.byref(v), C.byref(a), C.byref(b)))
        return {"variant": v.value, "ms": [a.value, b.value]}

    def profile(self, enable: bool = True):
        self._check(lib().efe_profile(self.h, int(bool(enable))))

    def profile_read(self):
        a, b, ms = C.c_int64(), C.c_int64(), C.c_double()
        self._check(lib().efe_profile_read(self.h, C.byref(a), C.byref(b), C.byref(ms)))
        return {"launches": a.value, "apply_launches": b.value, "apply_ms": ms.value}

    def init_orbitals(self, psi):
        wl = self.wl
        G = wl.orb_centers.shape[1]
        cen = np.ascontiguousarray(wl.orb_centers, dtype=np.float64)
        ex = np.ascontiguousarray(wl.orb_exps, dtype=np.float64)
        co = np.ascontiguousarray(np.stack([wl.orb_coefs.real, wl.orb_coefs.imag], axis=-1), dtype=np.float64)
        en = np.ascontiguousarray(np.stack([wl.enr_coefs.real, wl.enr_coefs.imag], axis=-1), dtype=np.float64)
        if en.size == 0:
            en = np.zeros(2)
        self._check(lib().efe_init_orbitals(self.h, _ptr(psi), int(G), _dptr(cen), _dptr(ex), _dptr(co), _dptr(en),
                                            _stream()))
        return psi


class Octree:
    """Owns one efe_octree (locally refined mesh with hanging-node constraints)."""

    def __init__(self, lo, hi, nc: int, degree: int, n_quad: int, refine=()):
        L = lib()
        lo = np.ascontiguousarray(lo, dtype=np.float64)
        hi = np.ascontiguousarray(hi, dtype=np.float64)
        ref = np.ascontiguousarray(np.asarray(list(refine), dtype=np.int32).reshape(-1, 3))
        h = C.c_void_p()
        st = L.efe_octree_setup(_dptr(lo), _dptr(hi), int(nc), int(degree), int(n_quad),
                                ref.ctypes.data_as(C.POINTER(C.c_int32)), int(len(ref)), C.byref(h))
        if st != EFE_OK:
            raise EfeError(st, L.efe_octree_last_error(None).decode())
        self.h = h
        v = [C.c_int64() for _ in range(5)]
        L.efe_octree_sizes(self.h, *[C.byref(x) for x in v])
        self.n_free, self.n_all, self.n_leaves, self.n_q, self.n_hanging = (x.value for x in v)

    def coords(self):
        """(free-node coordinates [n_free, 3], quadrature points [n_leaves, n_q, 3],
        boundary flags [n_free]) as numpy arrays."""
        fx = np.zeros((self.n_free, 3))
        qx = np.zeros((self.n_leaves, self.n_q, 3))
        bd = np.zeros(self.n_free, dtype=np.uint8)
        st = lib().efe_octree_coords(self.h, _dptr(fx), _dptr(qx), bd.ctypes.data_as(C.POINTER(C.c_uint8)))
        if st != EFE_OK:
            raise EfeError(st, lib().efe_octree_last_error(self.h).decode())
        return fx, qx, bd.astype(bool)

    def apply(self, vq, X, Y, kin: float = 1.0, mask_boundary: bool = False, lowdin: bool = False):
        """Y = P^T (kin K/2 + V) P X (lowdin: D P^T (kin K/2 + V) P D X on the interior, D the
        inverse square root of the lumped constrained mass); vq device [n_leaves, n_q],
        X, Y device [n_free, n_cols] float64."""
        import torch
        for t in (vq, X, Y):
            assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
        assert vq.numel() == self.n_leaves * self.n_q
        assert X.dim() == 2 and X.shape[0] == self.n_free and tuple(Y.shape) == tuple(X.shape)
        mode = 2 if lowdin else int(bool(mask_boundary))
        st = lib().efe_octree_apply(self.h, _ptr(vq), float(kin), _ptr(X), _ptr(Y), int(X.shape[1]), mode,
                                    _stream())
        if st != EFE_OK:
            raise EfeError(st, lib().efe_octree_last_error(self.h).decode())
        return Y

    def poisson(self, fq, g, tol: float = 1e-12, max_it: int = 10000):
        """-lap u = f (f at the leaves' GL points, device [n_leaves, n_q]) with u = g on the
        boundary (g device [n_free]); returns (u device [n_free], CG iterations)."""
        import torch
        for t in (fq, g):
            assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
        assert fq.numel() == self.n_leaves * self.n_q and g.numel() == self.n_free
        u = torch.zeros(self.n_free, dtype=torch.float64, device="cuda")
        its = C.c_int32()
        st = lib().efe_octree_poisson(self.h, _ptr(fq), _ptr(g), _ptr(u), float(tol), int(max_it), C.byref(its),
                                      _stream())
        if st != EFE_OK:
            raise EfeError(st, lib().efe_octree_last_error(self.h).decode())
        return u, its.value

    def density(self, psi_bar, occ):
        """rho at the leaves' GL points (device [n_leaves, n_q]) of Loewdin-basis orbitals
        psi_bar (device complex128 [n_free, n_orb])."""
        import torch
        assert psi_bar.is_cuda and psi_bar.dtype == torch.complex128 and psi_bar.is_contiguous()
        assert psi_bar.dim() == 2 and psi_bar.shape[0] == self.n_free
        occ = np.ascontiguousarray(occ, dtype=np.float64)
        assert len(occ) == psi_bar.shape[1]
        rho = torch.zeros((self.n_leaves, self.n_q), dtype=torch.float64, device="cuda")
        st = lib().efe_octree_density(self.h, _ptr(psi_bar), int(psi_bar.shape[1]), _dptr(occ), _ptr(rho), _stream())
        if st != EFE_OK:
            raise EfeError(st, lib().efe_octree_last_error(self.h).decode())
        return rho

    def magnus_step(self, psi_bar, occ, Z, R, dt: float, k: int, field=(0.0, 0.0, 0.0), cg_tol: float = 1e-12,
                    xc: int = EFE_XC_PW92, krylov_tol: float = 0.0):
        """One predictor-corrector step of psi_bar (device complex128 [n_free, n_orb], in place);
        krylov_tol > 0: adaptive Krylov dimension up to k."""
        import torch
        assert psi_bar.is_cuda and psi_bar.dtype == torch.complex128 and psi_bar.is_contiguous()
        assert psi_bar.dim() == 2 and psi_bar.shape[0] == self.n_free
        occ = np.ascontiguousarray(occ, dtype=np.float64)
        at = np.ascontiguousarray(np.column_stack([np.asarray(Z, float), np.asarray(R, float).reshape(-1, 3)]))
        E = np.ascontiguousarray(field, dtype=np.float64)
        st = lib().efe_octree_magnus_step(self.h, _ptr(psi_bar), int(psi_bar.shape[1]), _dptr(occ), _dptr(at), len(Z),
                                          _dptr(E), float(dt), int(k), float(krylov_tol), float(cg_tol), int(xc),
                                          _stream())
        if st != EFE_OK:
            raise EfeError(st, lib().efe_octree_last_error(self.h).decode())
        return psi_bar

    def interp(self, u):
        """Values at the leaves' GL points (device [n_cols, n_leaves, n_q]) of real nodal columns
        u (device float64 [n_free] or [n_free, n_cols])."""
        import torch
        assert u.is_cuda and u.dtype == torch.float64 and u.is_contiguous() and u.shape[0] == self.n_free
        nc = 1 if u.dim() == 1 else int(u.shape[1])
        out = torch.empty((nc, self.n_leaves, self.n_q), dtype=torch.float64, device="cuda")
        st = lib().efe_octree_interp(self.h, _ptr(u), nc, _ptr(out), _stream())
        if st != EFE_OK:
            raise EfeError(st, lib().efe_octree_last_error(self.h).decode())
        return out

    def kexp(self, vq, psi_bar, dt: float, k: int, kin: float = 1.0, tol: float = 0.0):
        """psi_bar <- exp(-i dt Hbar) psi_bar in place (device complex128 [n_free, n_cols]): k Lanczos
        steps per column, or (tol > 0) each column up to k until its estimate meets tol.  Returns the
        largest Krylov dimension used."""
        import torch
        assert psi_bar.is_cuda and psi_bar.dtype == torch.complex128 and psi_bar.is_contiguous()
        assert psi_bar.dim() == 2 and psi_bar.shape[0] == self.n_free
        assert vq.is_cuda and vq.dtype == torch.float64 and vq.is_contiguous() and vq.numel() == self.n_leaves * self.n_q
        ku = C.c_int32()
        st = lib().efe_octree_kexp(self.h, _ptr(vq), float(kin), _ptr(psi_bar), int(psi_bar.shape[1]), float(dt),
                                   int(k), float(tol), C.byref(ku), _stream())
        if st not in (EFE_OK, EFE_WARN_KRYLOV_CAP):
            raise EfeError(st, lib().efe_octree_last_error(self.h).decode())
        return ku.value

    def close(self):
        if getattr(self, "h", None):
            lib().efe_octree_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def octree_constraints(lo, hi, nc: int, degree: int, n_quad: int, refine=()):
    """Host-only description of a locally refined mesh: (row_start, col, val) of the
    constraint matrix P over all nodes, all-node and free-node coordinates."""
    L = lib()
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    ref = np.ascontiguousarray(np.asarray(list(refine), dtype=np.int32).reshape(-1, 3))
    rp = ref.ctypes.data_as(C.POINTER(C.c_int32))
    na, nf, nz = C.c_int64(), C.c_int64(), C.c_int64()
    args = (_dptr(lo), _dptr(hi), int(nc), int(degree), int(n_quad), rp, int(len(ref)))
    st = L.efe_octree_constraints(*args, C.byref(na), C.byref(nf), C.byref(nz), None, None, None, None, None)
    if st != EFE_OK:
        raise EfeError(st, L.efe_octree_last_error(None).decode())
    rs = np.zeros(na.value + 1, dtype=np.int64)
    col = np.zeros(nz.value, dtype=np.int32)
    val = np.zeros(nz.value)
    axyz = np.zeros((na.value, 3))
    fxyz = np.zeros((nf.value, 3))
    st = L.efe_octree_constraints(*args, C.byref(na), C.byref(nf), C.byref(nz),
                                  rs.ctypes.data_as(C.POINTER(C.c_int64)), col.ctypes.data_as(C.POINTER(C.c_int32)),
                                  _dptr(val), _dptr(axyz), _dptr(fxyz))
    if st != EFE_OK:
        raise EfeError(st, L.efe_octree_last_error(None).decode())
    return rs, col, val, axyz, fxyz


def atom_hartree_table(enrich, Z, n_tab: int = 24001, rmax: float = 60.0):
    """Host-only: the atomic Hartree potentials of the enriched Hartree solve for
    atoms with charges Z and wavefunction enrichment functions `enrich`
    (efe_workloads.EnrichFn list): (r [n_tab], v [n_atoms, n_tab], Q [n_atoms, n_tab], n_el [n_atoms])."""
    L = lib()
    Z = np.ascontiguousarray(Z, dtype=np.float64)
    fns = (EnrichFn * max(len(enrich), 1))()
    for i, f in enumerate(enrich):
        fns[i] = EnrichFn(int(f.atom), int(f.n), int(f.l), int(f.m), int(f.radial), float(f.zeta))
    r = np.zeros(n_tab)
    v = np.zeros((len(Z), n_tab))
    q = np.zeros((len(Z), n_tab))
    nel = np.zeros(len(Z))
    st = L.efe_atom_hartree_table(fns, len(enrich), _dptr(Z), len(Z), int(n_tab), float(rmax), _dptr(r), _dptr(v),
                                  _dptr(q), _dptr(nel))
    if st != EFE_OK:
        raise EfeError(st, "efe_atom_hartree_table: invalid argument")
    return r, v, q, nel


def adaptive_cell_boxes(origin, size, Z, R, sigma, r0, s, n_quad, tol, max_depth):
    """Host-only: the boxes (reference coordinates, [n, 6] = lo, hi) of the adaptive
    cell rule of efe_nuclear_enriched for one cell."""
    L = lib()
    o = np.ascontiguousarray(origin, dtype=np.float64)
    h = np.ascontiguousarray(size, dtype=np.float64)
    at = np.ascontiguousarray(np.column_stack([np.asarray(Z, float), np.asarray(R, float).reshape(-1, 3)]))
    n = C.c_int64()
    args = (_dptr(o), _dptr(h), _dptr(at), len(Z), float(sigma), float(r0), float(s), int(n_quad), float(tol),
            int(max_depth), C.byref(n))
    st = L.efe_adaptive_cell_boxes(*args, None, 0)
    if st != EFE_OK:
        raise EfeError(st, "efe_adaptive_cell_boxes: invalid argument")
    boxes = np.zeros((n.value, 6))
    st = L.efe_adaptive_cell_boxes(*args, _dptr(boxes), int(n.value))
    if st != EFE_OK:
        raise EfeError(st, "efe_adaptive_cell_boxes: invalid argument")
    return boxes


def lda_points(rho, xc: int = EFE_XC_PW92):
    """(v_xc, e_xc) at the points of a device float64 density array (any shape)."""
    import torch
    assert rho.is_cuda and rho.dtype == torch.float64 and rho.is_contiguous()
    vxc = torch.empty_like(rho)
    exc = torch.empty_like(rho)
    st = lib().efe_lda_points(_ptr(rho), _ptr(vxc), _ptr(exc), int(rho.numel()), int(xc), _stream())
    if st != EFE_OK:
        raise EfeError(st, "efe_lda_points: invalid argument")
    return vxc, exc
