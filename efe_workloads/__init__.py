"""Seeded synthetic workloads for the EFE real-time TDDFT hot path.

This module only lays out inputs: atom positions and charges, the 1D cell
boundaries of a rectilinear hexahedral mesh, the list of enrichment functions
(which atom, which n/l/m, which radial shape), the cutoff parameters, Gaussian
descriptors of the initial orbitals, the external-field parameters and the
time-step settings.  It draws every random number from a seeded generator and
holds none of the method's arithmetic: no basis functions, no quadrature, no
operators, no propagator.  Both the FP64 oracle and the CUDA library take
their inputs from here, and neither shares any other code with the other.

The paper's molecules, atomic ground-state orbitals and adaptive meshes are
not available, so the workloads below are synthetic stand-ins with the shapes
of the paper's benchmark systems (Sec. "Results and Discussion"): a hydrogen
molecule for the small exact-parity case, a sodium-cluster-like system, a
50-atom sodium-like cluster, a 27-atom organic-like molecule and a batched
magnesium-dimer-like sweep.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import List, Sequence

import numpy as np

# Field kinds (shared vocabulary; each side evaluates E(t) itself).
FIELD_NONE = 0
FIELD_GAUSS = 1        # E(t) = A exp(-(t - t0)^2 / (2 s^2)) d
FIELD_SINE_GAUSS = 2   # E(t) = A sin(w t) exp(-(t - t0)^2 / (2 s^2)) d
FIELD_SINE_TRAP = 3    # E(t) = A sin(w t) env(t) d, trapezoid envelope
FIELD_SINE_SINE = 4    # E(t) = A sin(pi t / T) sin(w t) d, 0 <= t <= T

RADIAL_SLATER = 0      # r^(n-1) exp(-zeta r)
RADIAL_HYDROGENIC = 1  # hydrogen-like R_nl(zeta r), zeta = effective charge
RADIAL_GAUSSIAN = 2    # r^l exp(-zeta r^2)


@dataclass
class EnrichFn:
    """One atom-centred enrichment function N^A = R_nl(r) * S_lm * u(r)."""
    atom: int
    n: int
    l: int
    m: int
    radial: int
    zeta: float


@dataclass
class Field:
    kind: int = FIELD_NONE
    amp: float = 0.0
    omega: float = 0.0
    t0: float = 0.0
    sigma: float = 1.0
    period: float = 0.0      # T for FIELD_SINE_SINE; total length for FIELD_SINE_TRAP
    ramp: float = 0.0        # ramp length for FIELD_SINE_TRAP
    direction: tuple = (1.0, 0.0, 0.0)
    kick: float = 0.0        # delta-kick strength applied at t = 0 (0: none)


@dataclass
class Workload:
    name: str
    xb: np.ndarray           # cell boundaries along x (ncx + 1)
    yb: np.ndarray
    zb: np.ndarray
    degree: int              # p: GLL nodes per cell edge = p + 1
    n_quad: int              # Gauss-Legendre points per direction
    Z: np.ndarray            # (Na,) nuclear charges
    R: np.ndarray            # (Na, 3) positions (bohr)
    enrich: List[EnrichFn]
    r0: float                # enrichment cutoff radius
    s: float                 # enrichment cutoff smoothing width
    n_orb: int
    occ: np.ndarray          # (n_orb,) occupations
    batch: int
    fields: List[Field]      # one per batch member
    dt: float
    n_steps: int
    krylov_tol: float
    k_max: int
    # Initial orbitals: psi_alpha(x) = sum_g c[alpha, g] exp(-a[alpha, g] |x - X[alpha, g]|^2)
    # at the classical nodes, plus enrichment coefficients e[alpha, nu].
    orb_centers: np.ndarray  # (n_orb, G, 3)
    orb_exps: np.ndarray     # (n_orb, G)
    orb_coefs: np.ndarray    # (n_orb, G) complex
    enr_coefs: np.ndarray    # (n_orb, n_E) complex
    seed: int = 0

    @property
    def n_cells(self) -> int:
        return (len(self.xb) - 1) * (len(self.yb) - 1) * (len(self.zb) - 1)

    @property
    def n_nodes(self) -> int:
        p = self.degree
        return ((len(self.xb) - 1) * p + 1) * ((len(self.yb) - 1) * p + 1) * ((len(self.zb) - 1) * p + 1)

    @property
    def n_enrich(self) -> int:
        return len(self.enrich)

    @property
    def n_dof(self) -> int:
        return self.n_nodes + self.n_enrich

    @property
    def n_cols(self) -> int:
        return self.n_orb * self.batch

    def with_(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


# ----------------------------------------------------------------------------
# geometry helpers (pure layout)
# ----------------------------------------------------------------------------

def uniform_bounds(L: float, n: int) -> np.ndarray:
    return np.linspace(-L / 2.0, L / 2.0, n + 1)


def graded_bounds(L: float, centers: Sequence[float], h_near: float, h_far: float, n_cells: int) -> np.ndarray:
    """Cell boundaries on [-L/2, L/2] whose local size follows
    h(x) = clamp(h_near + g * d(x), h_near, h_far), d = distance to the nearest
    atom coordinate on this axis, with g chosen so that exactly n_cells cells fit.
    Symmetric centre sets give symmetric meshes."""
    xs = np.linspace(-L / 2.0, L / 2.0, 200001)
    c = np.asarray(centers, dtype=np.float64).reshape(-1)
    d = np.min(np.abs(xs[:, None] - c[None, :]), axis=1)

    def count(g):
        h = np.clip(h_near + g * d, h_near, h_far)
        f = 1.0 / h
        return np.concatenate([[0.0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(xs))])

    lo, hi = 1e-6, 1e6
    if count(lo)[-1] < n_cells:
        # even the coarsest grading gives too few cells: use uniform spacing
        return uniform_bounds(L, n_cells)
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        if count(mid)[-1] > n_cells:
            lo = mid
        else:
            hi = mid
    cum = count(hi)
    cum *= n_cells / cum[-1]
    b = np.interp(np.arange(n_cells + 1, dtype=np.float64), cum, xs)
    b[0], b[-1] = -L / 2.0, L / 2.0
    # symmetrise when the centre set is symmetric about 0
    if np.allclose(np.sort(c), np.sort(-c)):
        b = 0.5 * (b - b[::-1])
    return b


def _random_cluster(rng, n_atoms, dmin, dmax, max_tries=100000):
    pos = [np.zeros(3)]
    tries = 0
    while len(pos) < n_atoms:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("cluster placement failed")
        base = pos[rng.integers(len(pos))]
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        cand = base + v * rng.uniform(dmin, dmax)
        dist = np.linalg.norm(np.asarray(pos) - cand, axis=1)
        if np.all(dist >= dmin):
            pos.append(cand)
    P = np.asarray(pos)
    return P - P.mean(axis=0)


def _orbital_descriptors(rng, n_orb, R, a_lo, a_hi, n_e, enr_scale):
    Na = len(R)
    centers = np.broadcast_to(R[None, :, :], (n_orb, Na, 3)).copy()
    exps = rng.uniform(a_lo, a_hi, size=(n_orb, Na))
    coefs = (rng.normal(size=(n_orb, Na)) + 1j * rng.normal(size=(n_orb, Na))) / math.sqrt(2.0)
    enr = enr_scale * (rng.normal(size=(n_orb, n_e)) + 1j * rng.normal(size=(n_orb, n_e))) / math.sqrt(2.0)
    return centers, exps, coefs, enr


def _shell_functions(atom, Z, shells, radial):
    """shells: list of (n, l, zeta); l = 1 expands to m = -1, 0, 1."""
    out = []
    for (n, l, zeta) in shells:
        for m in range(-l, l + 1):
            out.append(EnrichFn(atom=atom, n=n, l=l, m=m, radial=radial, zeta=zeta))
    return out


def _hydrogenic_shells(Z, occupied):
    """Hydrogen-like radial shapes with a crude screening: Z_eff = Z for n = 1,
    Z - 2 for n = 2, Z - 10 for n = 3 (never below 1)."""
    table = {"1s": (1, 0, Z), "2s": (2, 0, max(Z - 2, 1)), "2p": (2, 1, max(Z - 2, 1)),
             "3s": (3, 0, max(Z - 10, 1))}
    return [table[s] for s in occupied]


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

def h2(n_cells: int = 4, degree: int = 4, n_quad: int = 6, L: float = 16.0, kick: float = 1e-3,
       dt: float = 0.05, n_steps: int = 20, tol: float = 1e-12, k_max: int = 10, seed: int = 2211) -> Workload:
    """Two Z=1 atoms at (+-0.7, 0, 0) in a 16-bohr cube, 4x4x4 uniform cells,
    degree-4 Lagrange (4913 nodes), 6^3 Gauss-Legendre, one exp(-r) enrichment
    function per atom with a 3-bohr cutoff, one doubly occupied orbital, delta
    kick along x, dt = 0.05, 20 steps."""
    rng = np.random.default_rng(seed)
    R = np.array([[-0.7, 0.0, 0.0], [0.7, 0.0, 0.0]])
    Z = np.array([1.0, 1.0])
    enrich = [EnrichFn(0, 1, 0, 0, RADIAL_SLATER, 1.0), EnrichFn(1, 1, 0, 0, RADIAL_SLATER, 1.0)]
    b = uniform_bounds(L, n_cells)
    # initial guess: bonding-like combination of two Gaussians, seeded jitter
    centers = R[None, :, :].copy()
    exps = np.full((1, 2), 0.6) + 0.05 * rng.uniform(size=(1, 2))
    coefs = np.ones((1, 2), dtype=np.complex128) + 0.05 * rng.normal(size=(1, 2))
    enr = 0.2 * np.ones((1, 2), dtype=np.complex128)
    return Workload(name="h2", xb=b, yb=b.copy(), zb=b.copy(), degree=degree, n_quad=n_quad, Z=Z, R=R,
                    enrich=enrich, r0=3.0, s=1.5, n_orb=1, occ=np.array([2.0]), batch=1,
                    fields=[Field(kind=FIELD_NONE, kick=kick, direction=(1.0, 0.0, 0.0))],
                    dt=dt, n_steps=n_steps, krylov_tol=tol, k_max=k_max,
                    orb_centers=centers, orb_exps=exps, orb_coefs=coefs, enr_coefs=enr, seed=seed)


def na_cluster(n_atoms: int = 8, L: float = 40.0, cells_per_axis: int = 31, degree: int = 4, n_quad: int = 6,
               h_near: float = 0.3, h_far: float = 3.0, r0: float = 6.0, n_orb: int | None = None,
               batch: int = 1, kick: float = 1e-3, dt: float = 0.05, n_steps: int = 2000,
               tol: float = 1e-7, k_max: int = 16, seed: int = 2212) -> Workload:
    """Sodium-like cluster: Z = 11 atoms placed by random sequential growth with
    nearest-neighbour distance in [5.5, 6.5] bohr, centred in an L-bohr cube,
    graded mesh from h_near near the nuclei to h_far; 4 hydrogen-like radial
    shells per atom (1s, 2s, 2p, 3s -> 6 functions), cutoff r0; 11 electrons
    per atom, doubly occupied.  batch > 1 cycles the kick over x, y, z."""
    rng = np.random.default_rng(seed)
    R = _random_cluster(rng, n_atoms, 5.5, 6.5)
    Z = np.full(n_atoms, 11.0)
    enrich = []
    for I in range(n_atoms):
        enrich += _shell_functions(I, 11.0, _hydrogenic_shells(11.0, ["1s", "2s", "2p", "3s"]), RADIAL_HYDROGENIC)
    if n_orb is None:
        n_orb = int(round(Z.sum())) // 2
    xb = graded_bounds(L, R[:, 0], h_near, h_far, cells_per_axis)
    yb = graded_bounds(L, R[:, 1], h_near, h_far, cells_per_axis)
    zb = graded_bounds(L, R[:, 2], h_near, h_far, cells_per_axis)
    centers, exps, coefs, enr = _orbital_descriptors(rng, n_orb, R, 0.15, 0.6, len(enrich), 0.1)
    dirs = [(1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)]
    fields = [Field(kind=FIELD_NONE, kick=kick, direction=dirs[b % 3]) for b in range(batch)]
    return Workload(name=f"na{n_atoms}", xb=xb, yb=yb, zb=zb, degree=degree, n_quad=n_quad, Z=Z, R=R,
                    enrich=enrich, r0=r0, s=r0 / 2.0, n_orb=n_orb, occ=np.full(n_orb, 2.0), batch=batch,
                    fields=fields, dt=dt, n_steps=n_steps, krylov_tol=tol, k_max=k_max,
                    orb_centers=centers, orb_exps=exps, orb_coefs=coefs, enr_coefs=enr, seed=seed)


def na8(**kw) -> Workload:
    """Na8-like cluster, 40-bohr cube, ~30k cells (31^3), degree 4, 44 orbitals."""
    return na_cluster(n_atoms=8, L=40.0, cells_per_axis=31, seed=kw.pop("seed", 2212), **kw)


def na50(**kw) -> Workload:
    """50-atom sodium-like cluster, 60-bohr cube, ~80k cells (43^3), 275 orbitals."""
    kw.setdefault("n_steps", 500)
    return na_cluster(n_atoms=50, L=60.0, cells_per_axis=43, seed=kw.pop("seed", 2213), **kw)


def organic27(cells_per_axis: int = 27, L: float = 30.0, degree: int = 4, n_quad: int = 6, r0: float = 6.0,
              amp: float = 1e-3, omega: float = 0.1, t0: float = 25.0, sigma: float = 5.0, dt: float = 0.05,
              n_steps: int = 1000, tol: float = 1e-7, k_max: int = 16, seed: int = 2214) -> Workload:
    """27-atom organic-like molecule: 15 atoms with Z in {6, 7, 8} grown as a
    random tree with bond lengths 1.9-2.9 bohr, 12 hydrogens attached; an
    even electron count; Gaussian-envelope sine pulse along x."""
    rng = np.random.default_rng(seed)
    heavy = [np.zeros(3)]
    while len(heavy) < 15:
        base = heavy[rng.integers(len(heavy))]
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        cand = base + v * rng.uniform(2.5, 2.9)
        if np.all(np.linalg.norm(np.asarray(heavy) - cand, axis=1) >= 2.4):
            heavy.append(cand)
    hyd = []
    while len(hyd) < 12:
        base = heavy[rng.integers(15)]
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        cand = base + v * rng.uniform(1.9, 2.1)
        allp = np.asarray(heavy + hyd)
        if np.all(np.linalg.norm(allp - cand, axis=1) >= 1.85):
            hyd.append(cand)
    R = np.asarray(heavy + hyd)
    R -= R.mean(axis=0)
    Zh = rng.choice([6.0, 7.0, 8.0], size=15)
    if int(Zh.sum() + 12) % 2 == 1:
        Zh[0] = 7.0 if Zh[0] != 7.0 else 6.0
    Z = np.concatenate([Zh, np.ones(12)])
    enrich = []
    for I in range(15):
        enrich += _shell_functions(I, Zh[I], _hydrogenic_shells(Zh[I], ["1s", "2s", "2p"]), RADIAL_HYDROGENIC)
    for I in range(15, 27):
        enrich += _shell_functions(I, 1.0, [(1, 0, 1.0)], RADIAL_HYDROGENIC)
    n_orb = int(round(Z.sum())) // 2
    xb = graded_bounds(L, R[:, 0], 0.3, 3.0, cells_per_axis)
    yb = graded_bounds(L, R[:, 1], 0.3, 3.0, cells_per_axis)
    zb = graded_bounds(L, R[:, 2], 0.3, 3.0, cells_per_axis)
    centers, exps, coefs, enr = _orbital_descriptors(rng, n_orb, R, 0.2, 0.8, len(enrich), 0.1)
    f = Field(kind=FIELD_SINE_GAUSS, amp=amp, omega=omega, t0=t0, sigma=sigma, direction=(1.0, 0.0, 0.0))
    return Workload(name="organic27", xb=xb, yb=yb, zb=zb, degree=degree, n_quad=n_quad, Z=Z, R=R,
                    enrich=enrich, r0=r0, s=r0 / 2.0, n_orb=n_orb, occ=np.full(n_orb, 2.0), batch=1,
                    fields=[f], dt=dt, n_steps=n_steps, krylov_tol=tol, k_max=k_max,
                    orb_centers=centers, orb_exps=exps, orb_coefs=coefs, enr_coefs=enr, seed=seed)


def mg2_batch(cells_per_axis: int = 25, L: float = 40.0, degree: int = 5, n_quad: int = 7, r0: float = 6.0,
              n_amp: int = 16, omega: float = 0.057, dt: float = 0.02, n_steps: int = 5000, tol: float = 1e-7,
              k_max: int = 16, seed: int = 2215) -> Workload:
    """Mg2-like dimer (Z = 12, 7.4 bohr apart), 12 doubly occupied orbitals;
    n_amp field amplitudes in [1e-3, 2e-2] x 3 polarisations, each a sine pulse
    with a 10-cycle trapezoid envelope (2-cycle ramps)."""
    rng = np.random.default_rng(seed)
    R = np.array([[-3.7, 0.0, 0.0], [3.7, 0.0, 0.0]])
    Z = np.array([12.0, 12.0])
    enrich = []
    for I in range(2):
        enrich += _shell_functions(I, 12.0, _hydrogenic_shells(12.0, ["1s", "2s", "2p", "3s"]), RADIAL_HYDROGENIC)
    n_orb = 12
    xb = graded_bounds(L, R[:, 0], 0.3, 3.0, cells_per_axis)
    yb = graded_bounds(L, R[:, 1], 0.3, 3.0, cells_per_axis)
    zb = graded_bounds(L, R[:, 2], 0.3, 3.0, cells_per_axis)
    centers, exps, coefs, enr = _orbital_descriptors(rng, n_orb, R, 0.2, 0.8, len(enrich), 0.1)
    period = 2.0 * math.pi / omega
    amps = np.linspace(1e-3, 2e-2, n_amp)
    dirs = [(1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)]
    fields = [Field(kind=FIELD_SINE_TRAP, amp=float(a), omega=omega, period=10 * period, ramp=2 * period,
                    direction=d) for a in amps for d in dirs]
    return Workload(name="mg2x%d" % len(fields), xb=xb, yb=yb, zb=zb, degree=degree, n_quad=n_quad, Z=Z, R=R,
                    enrich=enrich, r0=r0, s=r0 / 2.0, n_orb=n_orb, occ=np.full(n_orb, 2.0), batch=len(fields),
                    fields=fields, dt=dt, n_steps=n_steps, krylov_tol=tol, k_max=k_max,
                    orb_centers=centers, orb_exps=exps, orb_coefs=coefs, enr_coefs=enr, seed=seed)


def small_cluster(n_atoms: int = 2, cells_per_axis: int = 5, L: float = 16.0, degree: int = 3, n_quad: int = 5,
                  n_orb: int = 3, batch: int = 1, r0: float = 3.0, seed: int = 2219, Zval: float = 3.0,
                  kick: float = 1e-3, dt: float = 0.05, tol: float = 1e-10, k_max: int = 12) -> Workload:
    """A few-cell cluster used for parity tests: ragged sizes (odd cell counts,
    several orbitals, a graded mesh, l = 1 enrichment) that the oracle finishes
    in seconds."""
    rng = np.random.default_rng(seed)
    if n_atoms == 1:
        R = np.array([[0.31, -0.27, 0.22]])
    else:
        R = _random_cluster(rng, n_atoms, 2.0, 2.6) + np.array([0.13, -0.07, 0.05])
    Z = np.full(n_atoms, Zval)
    enrich = []
    for I in range(n_atoms):
        enrich += _shell_functions(I, Zval, [(1, 0, Zval), (2, 1, max(Zval - 2.0, 1.0))], RADIAL_HYDROGENIC)
    xb = graded_bounds(L, R[:, 0], 1.0, 5.0, cells_per_axis)
    yb = graded_bounds(L, R[:, 1], 1.0, 5.0, cells_per_axis)
    zb = graded_bounds(L, R[:, 2], 1.0, 5.0, cells_per_axis)
    centers, exps, coefs, enr = _orbital_descriptors(rng, n_orb, R, 0.3, 0.8, len(enrich), 0.1)
    dirs = [(1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)]
    fields = [Field(kind=FIELD_NONE, kick=kick, direction=dirs[b % 3]) for b in range(batch)]
    return Workload(name="small%d" % n_atoms, xb=xb, yb=yb, zb=zb, degree=degree, n_quad=n_quad, Z=Z, R=R,
                    enrich=enrich, r0=r0, s=r0 / 2.0, n_orb=n_orb, occ=np.full(n_orb, 2.0), batch=batch,
                    fields=fields, dt=dt, n_steps=4, krylov_tol=tol, k_max=k_max,
                    orb_centers=centers, orb_exps=exps, orb_coefs=coefs, enr_coefs=enr, seed=seed)


CONFIGS = {
    "h2": h2,
    "na8": na8,
    "na50": na50,
    "organic27": organic27,
    "mg2x48": mg2_batch,
    "small": small_cluster,
}
