"""FP64 CPU oracle for the EFE real-time TDDFT hot path.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of Kanungo, Rufus & Gavini, "Efficient all-electron
time-dependent density functional theory calculations using an enriched
finite element basis" (arXiv 2210.14421), written in NumPy/SciPy float64 and
complex128.  Only the test suite (`tests/`), `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` may import it.  The
CUDA library never imports, links or calls it, and the two share no code: the
only common input is `efe_workloads`, which draws seeded inputs and holds none
of the method's arithmetic.

Modules
-------
basis     Gauss-Legendre / Gauss-Lobatto-Legendre rules and Lagrange tables
          (Sec. "Spectral finite elements").
mesh      rectilinear hexahedral mesh, nodes, GLL-lumped mass (Sec. "Spectral
          finite elements").
enrich    atom-centred enrichment functions, Eq. EFEAtomic.
operators H, M, orthogonalisation and the Loewdin transform, Eqs. PsiEFE,
          EFESplit, EFEOrtho, Hmn, M, TDKSDiscrete2, MSquareRoot.
xc        Slater exchange + Perdew-Wang 1992 correlation (local density).
poisson   Hartree potential, Eqs. Hartree_possion and DiscretePoisson.
electrostatic  nuclear and Hartree potentials in the enriched basis, Eqs.
          PhiEFE and DiscretePoisson.
quadrature  adaptive cell quadrature for the enrichment integrals.
octree    locally refined mesh with hanging-node constraints.
krylov    adaptive Lanczos exponential, Eqs. AdaptiveKrylov, AdaptiveKrylovErr.
tdks      density, dipole, fields, second-order Magnus predictor-corrector
          step (Eq. ApproxMagnus), delta kick, ground state.

Parity status of each function is stated in its docstring; every function is
pinned by a `-m "not gpu"` test in `tests/test_oracle_*.py` (no function is
"parity unpinned"; values taken from the literature sit in `tests/golden/`
with their citations).
"""
