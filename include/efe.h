/*
 * efe.h - C ABI of libefe: the hot path of all-electron real-time TDDFT in an
 * orthogonalised enriched finite element (EFE) basis, after Kanungo, Rufus &
 * Gavini, "Efficient all-electron time-dependent density functional theory
 * calculations using an enriched finite element basis" (arXiv 2210.14421),
 * written for one NVIDIA GB300 (sm_103a).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Units: atomic units (bohr, hartree, a.u. of time).
 * Mesh: an axis-aligned rectilinear hexahedral mesh of [xb0, xbN] x [yb0, ybN]
 *   x [zb0, zbN]; cells c = cx + ncx (cy + ncy cz).  Classical nodes are the
 *   tensor-product Gauss-Lobatto-Legendre (GLL) nodes of degree p; node
 *   g = ix + Nx (iy + Ny iz), Nx = ncx p + 1.  Every node is stored; boundary
 *   nodes carry the homogeneous Dirichlet condition of the orbitals and are
 *   held at zero by the operators.
 * DOFs: n_dof = n_nodes + n_enrich; rows 0..n_nodes-1 are classical nodes,
 *   rows n_nodes.. are enrichment functions in the order they were given.
 * Orbitals: psi_bar is the Loewdin-basis coefficient block of Eq.
 *   TDKSDiscrete2 (psi_bar = M^1/2 psi), stored as complex128, row-major
 *   [n_dof][n_cols] with re/im interleaved, n_cols = n_orb * batch, column
 *   b * n_orb + alpha = orbital alpha of batch member b.
 * Quadrature fields (rho, v_xc, v_H): float64 [batch][n_cells][n_q^3],
 *   point q = q1 + n_q (q2 + n_q q3) of the n_q-point Gauss-Legendre rule.
 * Pointers: every array argument named *_dev is device memory of the device
 *   that was current at efe_setup; *_host is host memory.  The caller owns all
 *   arrays it passes and keeps them alive until the stream work completes; the
 *   context owns only its internal tables and workspaces.
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  All
 *   calls enqueue work on `stream` and return without waiting, except
 *   efe_setup, efe_destroy and the host-visible outputs documented below
 *   (efe_step_info, iteration counts), which synchronise `stream`.
 * Errors: every call returns an efe_status; a non-OK status leaves a message
 *   that efe_last_error(ctx) returns until the next call on that context.
 *   EFE_WARN_KRYLOV_CAP is a warning: the step was completed with k_max
 *   Lanczos vectors for at least one column.
 */
#ifndef EFE_H
#define EFE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct efe_ctx efe_ctx;

typedef enum {
  EFE_OK = 0,
  EFE_ERR_ARG = 1,          /* invalid argument (sizes, pointers, unsupported degree) */
  EFE_ERR_NOMEM = 2,        /* device allocation failed */
  EFE_ERR_CUDA = 3,         /* a CUDA runtime call failed */
  EFE_ERR_NOT_SPD = 4,      /* the enrichment overlap M^ee is not positive definite */
  EFE_WARN_KRYLOV_CAP = 5,  /* Lanczos reached k_max before its error estimate met tol */
  EFE_ERR_CG_NOCONV = 6,    /* Hartree CG did not reach cg_tol within cg_max_it */
  EFE_ERR_TIMEOUT = 7,      /* a bounded device-side wait gave up */
  EFE_ERR_STATE = 8         /* call out of order (e.g. apply before a potential was set) */
} efe_status;

typedef enum {
  EFE_FP64 = 0,   /* every step in float64 */
  EFE_MIXED = 1,  /* cell contraction and enrichment coupling in float32 with float32
                     accumulation; the density interpolation and the Krylov combination
                     in float32 pairs (as EFE_PAIR); gather/scatter accumulation,
                     Lanczos recurrence, tridiagonal exponential, Hartree, norms and
                     dipole in float64; storage float64 */
  EFE_PAIR = 2,   /* as EFE_MIXED, but every value of the cell contraction and the
                     enrichment coupling is a pair of float32 (h + l) with error-free
                     products and sums, so the float32 pipe delivers ~2^-44 relative
                     accuracy */
  EFE_TC = 3      /* as EFE_MIXED, but the cell contraction runs densely (H_c x_c with
                     the dense cell matrix, rebuilt in float64 whenever the potential
                     changes) on the tensor cores, together with the enrichment coupling:
                     every operand is scaled by a power of two per row or column,
                     rounded to 31 bits and split into four bf16 slices whose products
                     are exact; slice products are summed in float32 tensor-memory
                     accumulators (the leading group exactly) and combined in float64.
                     Error per element ~2^-29 sum_k |H_ik| max_k |x_k|.  Supported for
                     degree <= 4, at most 48 enrichment functions touching one cell and
                     at most 96 real columns (48 orbitals) per batch member; otherwise
                     efe_setup / efe_apply_H return EFE_ERR_ARG.  Holds 128 KB of slices
                     per cell and batch member in device memory. */
} efe_precision;

/* Radial shapes of the atomic part N^A (Eq. EFEAtomic), divided by r^l:
 * SLATER r^(n-1-l) e^(-zeta r); HYDROGENIC zeta^l L_{n-l-1}^{(2l+1)}(2 zeta r / n)
 * e^(-zeta r / n); GAUSSIAN e^(-zeta r^2).  Angular part: real solid harmonics
 * l <= 2 (l = 1: m = -1, 0, 1 -> y, z, x; l = 2: xy, yz, 2z^2-x^2-y^2, xz, x^2-y^2). */
enum { EFE_RADIAL_SLATER = 0, EFE_RADIAL_HYDROGENIC = 1, EFE_RADIAL_GAUSSIAN = 2 };

/* External field E(t) of Eq. VField, v_f = -E(t) . x. */
enum {
  EFE_FIELD_NONE = 0,
  EFE_FIELD_GAUSS = 1,       /* amp exp(-(t-t0)^2 / (2 sigma^2)) dir */
  EFE_FIELD_SINE_GAUSS = 2,  /* amp sin(omega t) exp(-(t-t0)^2 / (2 sigma^2)) dir */
  EFE_FIELD_SINE_TRAP = 3,   /* amp sin(omega t) env(t) dir; env ramps linearly over `ramp`
                                at both ends of [0, period], zero outside */
  EFE_FIELD_SINE_SINE = 4    /* amp sin(pi t / period) sin(omega t) dir on [0, period] */
};

typedef struct {
  int32_t ncx, ncy, ncz;      /* cells per axis, >= 1 */
  const double* xb_host;      /* ncx + 1 strictly increasing cell boundaries */
  const double* yb_host;      /* ncy + 1 */
  const double* zb_host;      /* ncz + 1 */
  int32_t degree;             /* p in [2, 5] */
  int32_t n_quad;             /* Gauss-Legendre points per direction; must be p + 2 */
} efe_mesh_desc;

typedef struct {
  double Z;                   /* nuclear charge */
  double R[3];                /* position */
} efe_atom;

typedef struct {
  int32_t atom;               /* index into the atom array */
  int32_t n, l, m;            /* quantum numbers, l <= 2, |m| <= l */
  int32_t radial;             /* EFE_RADIAL_* */
  double zeta;                /* exponent / effective charge */
} efe_enrich_fn;

typedef struct {
  int32_t n_fn;
  const efe_enrich_fn* fns_host;
  double r0;                  /* cutoff radius: N^A = 0 for r >= r0 */
  double s;                   /* cutoff width: N^A untouched for r <= r0 - s */
} efe_enrich_desc;

typedef struct {
  int32_t kind;               /* EFE_FIELD_* */
  double amp, omega, t0, sigma, period, ramp;
  double dir[3];
  double kick;                /* delta-kick strength used by efe_kick (0: none) */
} efe_field;

typedef struct {
  int32_t n_orb;              /* orbitals per batch member */
  int32_t batch;              /* independent propagations (own density, potential, field) */
  const double* occ_host;     /* n_orb occupations (2.0 for doubly occupied) */
  double krylov_tol;          /* Lanczos stop threshold on eps_k of Eq. AdaptiveKrylovErr */
  int32_t k_max;              /* Lanczos cap, 1 <= k_max <= 64 */
  int32_t fixed_k;            /* > 0: take exactly fixed_k Lanczos steps (tests) */
  double cg_tol;              /* Hartree PCG relative residual target */
  int32_t cg_max_it;
  int32_t precision;          /* efe_precision used by efe_magnus_step (efe_kick is always FP64) */
  int32_t hartree_method;     /* EFE_HARTREE_FDM (direct) or EFE_HARTREE_PCG */
  int32_t use_graphs;         /* 1: each Lanczos exponential of efe_magnus_step runs as a captured
                                 CUDA graph of k_max iterations (finished columns skipped on the
                                 device, no host synchronisation; captured on the second call for a
                                 given buffer set, the first call runs and autotunes eagerly).
                                 Must be 0 if the caller itself captures efe_magnus_step. */
  int32_t xc;                 /* EFE_XC_PW92 (Slater + Perdew-Wang 1992) or EFE_XC_PZ81 (Slater +
                                 Perdew-Zunger 1981 fit of Ceperley-Alder, the paper's functional) */
  int32_t scheme;             /* EFE_STEP_PC: predictor-corrector (two exponentials per step);
                                 EFE_STEP_EXTRAPOLATED: v_Hxc at the mid-point extrapolated
                                 linearly from the last two steps, one exponential per step (the
                                 first step after set-up, a kick or a reset is predictor-corrector) */
  int32_t krylov_block;       /* complex columns per Lanczos exponential run (the Krylov basis holds
                                 k_max + 1 vectors of that many columns): 0 takes as many as fit in
                                 the device memory free at the first step (all columns when they
                                 fit); with batch > 1 a block holds whole batch members (rounded
                                 down, at least one).  Columns are independent in the exponential,
                                 so blocks give the result of one run; the density, Hartree and
                                 dipole always see all orbitals.  efe_adjoint_dipole needs all
                                 columns in one block (else EFE_ERR_ARG). */
  int32_t krylov_substeps;    /* each exponential exp(-i dt Hbar) of efe_magnus_step (Eq.
                                 ApproxMagnus) as m sub-steps exp(-i (dt/m) Hbar) of the same
                                 operator, each a Lanczos run capped at k_max (exact in exact
                                 arithmetic: the sub-steps commute).  n >= 1: m = n.  0: adaptive,
                                 for a Krylov cap below what dt needs: an exponential in which a
                                 column reached k_max with its estimate above krylov_tol is
                                 computed again from its input with twice the sub-steps (up to
                                 64); the count carries over to the next exponential and halves
                                 after one whose largest k stayed at or below 2 k_max / 5.  With
                                 fixed_k > 0, 0 means 1.  The kick and the adjoint take single
                                 exponentials. */
  int32_t krylov_reorth;      /* 1: every new Lanczos vector is made orthogonal to all earlier ones
                                 of its column by classical Gram-Schmidt applied twice before
                                 beta_j is taken (the paper is silent; 2 (j + 1) extra passes over
                                 the basis at iteration j); 0: the plain three-term recurrence. */
} efe_options;

enum { EFE_XC_PW92 = 0, EFE_XC_PZ81 = 1 };
enum { EFE_STEP_PC = 0, EFE_STEP_EXTRAPOLATED = 1 };

/* Hartree solvers for the same discrete system (Eq. DiscretePoisson):
 * FDM  - direct solve by fast diagonalisation of the Kronecker-sum stiffness of
 *        the rectilinear mesh (exact to rounding; cg_tol / cg_max_it unused);
 * PCG  - Jacobi-preconditioned conjugate gradients to cg_tol. */
enum { EFE_HARTREE_FDM = 0, EFE_HARTREE_PCG = 1 };

typedef struct {
  int32_t k_pred_max;         /* largest Lanczos dimension used in the predictor */
  int32_t k_corr_max;         /* ... and in the corrector */
  int32_t krylov_cap_hit;     /* columns that reached k_max */
  int32_t cg_iters;           /* total Hartree PCG iterations in the step */
  double eps_max;             /* largest final Krylov error estimate */
  int32_t substeps;           /* sub-steps of the step's last exponential (krylov_substeps) */
} efe_step_info;

/* ---- set-up (Secs. "Enriched finite element discretization", "Spectral finite
 * elements"): builds the GLL basis, Gauss-Legendre quadrature, the lumped
 * diagonal M^cc, the enrichment functions at every quadrature point of the
 * cells their support reaches, the orthogonalisation coefficients
 * c = b / M^cc (Eq. EFEOrtho), M^ee and (M^ee)^(+-1/2) (Eq. MSquareRoot), the
 * kinetic coupling blocks, the nuclear potential v_N (Eq. VN) at the quadrature
 * points and the Dirichlet data of the Hartree problem.  All host inputs are
 * copied.  Runs on the current CUDA device and synchronises it.
 * Errors: EFE_ERR_ARG, EFE_ERR_NOMEM, EFE_ERR_CUDA, EFE_ERR_NOT_SPD.  On error
 * *out is NULL and the message is available from efe_last_error(NULL). */
efe_status efe_setup(const efe_mesh_desc* mesh, const efe_atom* atoms_host, int32_t n_atoms,
                     const efe_enrich_desc* enrich, const efe_options* opts, efe_ctx** out);

/* Frees every device allocation of the context (synchronises the device). */
efe_status efe_destroy(efe_ctx* ctx);

/* Last error message of ctx (or of the last failed efe_setup when ctx is NULL). */
const char* efe_last_error(const efe_ctx* ctx);

/* Sizes: n_nodes, n_enrich, n_cells, n_q (points per cell), n_pairs (cell-function
 * pairs of the enrichment support).  Any pointer may be NULL. */
efe_status efe_sizes(const efe_ctx* ctx, int64_t* n_nodes, int64_t* n_enrich, int64_t* n_cells,
                     int64_t* n_q, int64_t* n_pairs);

/* Node coordinates [n_nodes][3] (float64, device) and quadrature point
 * coordinates [n_cells][n_q][3] (device; either may be NULL). */
efe_status efe_coords(efe_ctx* ctx, double* node_xyz_dev, double* quad_xyz_dev, void* stream);

/* Builds the operator Hbar = M^-1/2 P^T H_ext P M^-1/2 (Eqs. Hmn, TDKSDiscrete2)
 * for `batch` potentials v_dev [batch][n_cells][n_q] given at the quadrature
 * points: H = kin_scale * (1/2) int grad N . grad N + int v N N.  The operator
 * is held by the context and used by efe_apply_H until the next build. */
efe_status efe_set_potential(efe_ctx* ctx, const double* v_dev, int32_t batch, double kin_scale,
                             void* stream);

/* Y = Hbar X (Eq. TDKSDiscrete2) for the operator of the last efe_set_potential.
 * X_dev, Y_dev: complex128 [n_dof][ld] (ld >= n_cols complex entries per row);
 * the first n_cols columns are used, n_cols = n_orb_per_member * batch of that
 * operator.  The four steps run on the device: gather (with M^-1/2), cell
 * contraction (kinetic + v-weighted mass), scatter-add (with M^-1/2) and the
 * enrichment coupling.  X and Y must not overlap.  precision: any efe_precision.
 * EFE_TC needs degree <= 4, at most 48 enrichment functions touching one cell and
 * at most 96 real columns per member (else EFE_ERR_ARG with a message); its first
 * use on a context whose options did not ask for it builds the slices of the
 * current operator (the context keeps them in step with later operator builds).
 * A tensor-core completion wait that gives up (bounded, seconds) records a
 * sticky error that the next efe_magnus_step with info_host reports as
 * EFE_ERR_TIMEOUT. */
efe_status efe_apply_H(efe_ctx* ctx, const double* X_dev, double* Y_dev, int64_t n_cols, int64_t ld,
                       int32_t precision, void* stream);

/* Y = Hbar X without allocating device memory (the paper has no counterpart:
 * this is a deployment variant of efe_apply_H).  Some callers cannot call
 * cudaMalloc when they apply the operator: a host framework that owns all
 * device memory and forbids new allocations once it runs, or code recording
 * into a CUDA graph, where allocation is not allowed during stream capture.
 * This call computes exactly what efe_apply_H computes, with the same
 * arguments and precision (EFE_FP64 or EFE_MIXED; EFE_PAIR is rejected with
 * EFE_ERR_ARG), but keeps its enrichment scratch in a static
 * device array of 2 MiB per GPU (held from the library's first use on that
 * GPU until the process exits) instead of context workspaces; it calls no
 * cudaMalloc, cudaFree or allocating library routine.  Limit:
 * n_enrich * 2 * ld <= 104857 entries; larger requests return EFE_ERR_ARG
 * with a message.  The first call on a device looks up the array's device
 * address and must be made with the context's device current and before any
 * stream capture.  All calls on one GPU share the array: calls that overlap
 * on the GPU (other streams, other contexts) race; each call clears the
 * accumulator it needs.  Requires a prior efe_set_potential. */
efe_status efe_apply_H_noalloc(efe_ctx* ctx, const double* X_dev, double* Y_dev, int64_t n_cols, int64_t ld,
                               int32_t precision, void* stream);

/* One second-order Magnus step (Eq. ApproxMagnus) evaluated by the adaptive
 * Lanczos exponential (Eqs. AdaptiveKrylov, AdaptiveKrylovErr) with the
 * predictor-corrector for the mid-point Hamiltonian:
 *   S1 psi^p = Kexp(Hbar[v(rho_n), E(t+dt/2)]) psi_n;  S2 rho^p = rho(psi^p);
 *   S3 rho_mid = (rho_n + rho^p)/2;  S4 v_mid = v_N + v_H[rho_mid] + v_xc[rho_mid]
 *   - E(t+dt/2).x;  S5 psi_n+1 = Kexp(Hbar[v_mid]) psi_n;  S6 rho_n+1, v_H, v_xc,
 *   dipole.
 * psi_bar_dev is overwritten with psi_n+1.  fields_host: `batch` field
 * descriptions.  mu_dev: NULL or device float64 [batch][3] receiving the dipole
 * at t + dt.  info_host: NULL, or filled after synchronising `stream`.
 * The density-derived potentials of step n are kept in the context from the
 * previous step; the first step after efe_setup, efe_kick or efe_reset_state
 * recomputes them from psi_bar.  Errors: EFE_ERR_ARG (psi_bar_dev NULL, t or dt
 * not finite), EFE_ERR_CG_NOCONV (a Hartree PCG solve missed cg_tol; the step
 * is completed), EFE_ERR_TIMEOUT (see efe_apply_H), EFE_ERR_NOMEM, EFE_ERR_CUDA,
 * and the warning EFE_WARN_KRYLOV_CAP. */
efe_status efe_magnus_step(efe_ctx* ctx, double* psi_bar_dev, double t, double dt,
                           const efe_field* fields_host, double* mu_dev, efe_step_info* info_host,
                           void* stream);

/* Forgets the cached density-derived potentials (call after changing psi_bar). */
efe_status efe_reset_state(efe_ctx* ctx);

/* Density rho_q = sum_alpha occ_alpha |psi_alpha(x_q)|^2 per batch member
 * (Sec. "Time dependent Kohn-Sham equations"), psi(x_q) from Eq. PsiEFE, and
 * the LDA v_xc (Slater exchange + PW92 correlation) and eps_xc at the same
 * points.  vxc_dev / exc_dev may be NULL. */
efe_status efe_density_vxc(efe_ctx* ctx, const double* psi_bar_dev, double* rho_dev, double* vxc_dev,
                           double* exc_dev, void* stream);

/* Hartree potential (Eqs. Hartree_possion, DiscretePoisson): solves
 * (1/4pi) K phi = d, d_i = int rho N_i, with phi = sum Z_I / |x - R_I| on the
 * boundary, by the context's hartree_method (FDM: direct; PCG: Jacobi-preconditioned
 * CG to relative residual tol, warm-started from the previous solution held by
 * the context); vH_dev receives phi interpolated to the quadrature points
 * [batch][n_cells][n_q].  iters_host: NULL or receives the PCG iteration count
 * (1 for FDM; PCG synchronises `stream`).  Returns EFE_ERR_CG_NOCONV (after
 * writing the last iterate) if PCG does not meet tol. */
efe_status efe_hartree(efe_ctx* ctx, const double* rho_dev, double* vH_dev, double tol, int32_t max_it,
                       int32_t* iters_host, void* stream);

/* Dipole mu = sum_I Z_I R_I - int x rho for each batch member; mu_dev [batch][3]. */
efe_status efe_dipole(efe_ctx* ctx, const double* rho_dev, double* mu_dev, void* stream);

/* Delta kick psi_bar <- exp(i kick d.Xbar) psi_bar per batch member, with Xbar the
 * Loewdin-transformed position operator, by the same Lanczos exponential with
 * float64 applies (the initial condition carries no float32 rounding). */
efe_status efe_kick(efe_ctx* ctx, double* psi_bar_dev, const efe_field* fields_host, void* stream);

/* Initial orbitals from Gaussian descriptors: classical coefficients
 * psi^C_i = sum_g coef[a][g] exp(-expo[a][g] |x_i - center[a][g]|^2) (zero on
 * the boundary), enrichment coefficients enr[a][nu]; psi_bar = M^1/2 psi, the
 * same for every batch member.  Host arrays: centers [n_orb][G][3], expo
 * [n_orb][G], coef and enr complex128 interleaved [n_orb][G] / [n_orb][n_enrich]. */
efe_status efe_init_orbitals(efe_ctx* ctx, double* psi_bar_dev, int32_t n_gauss, const double* centers_host,
                             const double* expo_host, const double* coef_host, const double* enr_host,
                             void* stream);

/* Gradient of a windowed dipole signal with respect to the field parameters.
 * The paper has no adjoint; this is the exact reverse sweep (the adjoint of
 * each operation, in reverse order) of n_steps calls of efe_magnus_step's
 * predictor-corrector step (Eq. ApproxMagnus with the mid-point density of
 * the predictor, field at t_n + dt/2, t_n = n dt), with float64 applies (float32
 * pairs when the context's precision is EFE_PAIR; float64 for EFE_MIXED and
 * EFE_TC contexts) and float64 elsewhere:
 *   J = (1/|W|) sum_{n in W} d . mu(rho_n),   W = [window_first, window_last],
 *   grad = dJ / d(amp, omega, sigma)   (omega entry 0 for EFE_FIELD_GAUSS).
 * The derivative of each exponential exp(-i dt Hbar) is its Frechet derivative,
 * integrated over s in [0, 1] with n_quad_s Gauss-Legendre nodes; the vectors
 * exp(-i s dt Hbar) psi and exp(+i (1 - s) dt Hbar) lam at the nodes are
 * recombined from the Krylov bases of the full-step exponentials (four Lanczos
 * runs per reversed step).  The Hartree map enters transposed (the direct
 * solve with zero boundary data) and v_xc through d v_xc / d rho.  States are
 * kept every checkpoint_every steps and a segment is recomputed before its
 * reverse sweep (memory (n_steps / K + K + 10 + 2 n_quad_s) blocks of psi).
 * psi0_dev: device [n_dof][n_orb] complex128 (not modified).  field_host: kind
 * EFE_FIELD_GAUSS or EFE_FIELD_SINE_GAUSS with sigma > 0; direction_host: host
 * double[3] (d).  J_host: receives J; grad_host: host double[3].  The context
 * needs batch = 1, xc = EFE_XC_PW92 and scheme = EFE_STEP_PC; the Lanczos
 * tolerance and k_max of its options apply, and
 * its state is invalidated (the next efe_magnus_step recomputes rho).  Allocates
 * device memory per call and synchronises `stream`.  Returns EFE_WARN_KRYLOV_CAP
 * (J and grad written) if any exponential stopped at k_max.  Errors: EFE_ERR_ARG
 * (bad sizes, window outside [1, n_steps], n_quad_s outside [1, 64], batch != 1,
 * another functional or step scheme, unsupported field, a density reduction installed), EFE_ERR_NOMEM,
 * EFE_ERR_CUDA.  With the enriched Hartree solve installed (efe_hartree_enriched)
 * the Hartree map and its transpose are the enriched ones. */
efe_status efe_adjoint_dipole(efe_ctx* ctx, const double* psi0_dev, int32_t n_steps, double dt,
                              const efe_field* field_host, const double* direction_host, int32_t window_first,
                              int32_t window_last, int32_t checkpoint_every, int32_t n_quad_s, double* J_host,
                              double* grad_host, void* stream);

/* Nuclear potential in the electrostatically enriched basis (Eqs. PhiEFE,
 * DiscretePoisson; the paper's electrostatic enrichment of the nuclear
 * potential).  Replaces the context's nuclear potential -sum Z/|x - R| at the
 * quadrature points by the finite element solution for Gaussian-smeared
 * nuclei: charge b = -sum_J Z_J g_sigma(|x - R_J|) (normalised Gaussians of
 * width sigma), phi^h = sum_j N_j phi_j + sum_J Ntil_J phi^E_J with one
 * enrichment function per atom, the atom's smeared-nucleus potential
 * -Z_J erf(r / (sqrt2 sigma)) / r truncated by the smooth cutoff (r0, s) and
 * orthogonalised against the classical functions in the GLL-lumped inner
 * product, stiffness (1/4pi) int grad . grad, and the smeared-nucleus
 * potential as Dirichlet data on the boundary nodes.  Cell integrals of the
 * atomic parts and of the charge use n_quad^3 Gauss-Legendre points (n_quad 0:
 * p + 2) on each of a cell's boxes: with adapt_tol = 0, sub^3 equal boxes; with
 * adapt_tol > 0, the adaptive rule (the paper's adaptive quadrature for the
 * enrichment): a box's estimate of the trial integrals (the smeared charge and
 * every atomic part) is compared with the sum over its eight half-size
 * children, whose boxes are kept where every trial integral agrees to
 * adapt_tol (absolute) and refined the same way otherwise, down to adapt_depth
 * levels below the cell (sub is then ignored).  The Galerkin system is
 * solved exactly (to rounding) around the direct Poisson solver by block
 * elimination of the n_atoms enrichment unknowns.  vN_dev (nullable): device
 * [n_cells][n_q] doubles receiving the new potential at the quadrature points;
 * phiE_host (nullable): host [n_atoms] enrichment coefficients.  Later steps,
 * kicks and adjoints use the new potential; the propagation state is
 * invalidated (the next efe_magnus_step recomputes rho).  Allocates device
 * memory for the call (about 4 n_atoms + 10 vectors of n_nodes doubles) and
 * synchronises `stream`.  Errors: EFE_ERR_ARG (sigma <= 0, s <= 0, r0 <= s,
 * sub outside [1, 8], n_quad outside [p + 1, 8] and not 0, adapt_tol < 0,
 * adapt_depth outside [0, 8], a support sphere of radius r0 reaching the domain
 * boundary), EFE_ERR_NOT_SPD (the eliminated block not positive definite),
 * EFE_ERR_NOMEM, EFE_ERR_CUDA. */
efe_status efe_nuclear_enriched(efe_ctx* ctx, double sigma, double r0, double s, int32_t sub, int32_t n_quad,
                                double adapt_tol, int32_t adapt_depth, double* vN_dev, double* phiE_host,
                                void* stream);

/* Hartree potential in the electrostatically enriched basis (Eq. PhiEFE for the
 * Hartree potential, Eq. DiscretePoisson).  Installs, for every later Hartree
 * solve of the context (efe_hartree and the Magnus steps), one enrichment
 * function per atom: the Hartree potential of the isolated neutral atom
 * whose Z electrons fill the shells of the atom's wavefunction enrichment
 * functions (distinct radial kind, n, l, zeta, filled in the order of n, then
 * l, two electrons per orbital; tabulated on r = 60 t^2 bohr, t uniform, 24001
 * points), truncated by the smooth cutoff (r0, s) and orthogonalised against
 * the classical functions in the GLL-lumped inner product.  The solve keeps
 * the classical Dirichlet data and load int rho N (quadrature points), adds
 * the enrichment loads int rho N^A at the quadrature points, and is exact
 * (to rounding) by block elimination around the direct Poisson solver; the
 * eliminated n_atoms x n_atoms block and the n_atoms direct solves it needs
 * are computed here, with cell integrals on a composite Gauss-Legendre rule
 * of sub^3 sub-cells with n_quad^3 points each (n_quad 0: p + 2).  v_H at
 * the quadrature points includes the enrichment functions.  Keeps 3 n_atoms
 * vectors of n_nodes doubles on the device; synchronises `stream`; the
 * propagation state is invalidated.  efe_adjoint_dipole then transposes the
 * enriched map (rho -> v_H) in its reverse sweep.  Errors: EFE_ERR_ARG (the context's Hartree method is not
 * EFE_HARTREE_FDM; s <= 0, r0 <= s, sub outside [1, 8], n_quad outside
 * [p + 1, 8] and not 0, a support sphere reaching the domain boundary),
 * EFE_ERR_NOT_SPD, EFE_ERR_NOMEM, EFE_ERR_CUDA. */
efe_status efe_hartree_enriched(efe_ctx* ctx, double r0, double s, int32_t sub, int32_t n_quad, void* stream);

/* Locally refined mesh with hanging-node constraints (the paper's adaptively
 * refined finite element mesh, Sec. "Enriched finite element basis"): one
 * refinement level over a uniform nc^3 grid of the box [lo, hi] (host
 * double[3] each); the n_refine coarse cells (i, j, k) listed in refine_host
 * (int32[n_refine][3]) are split into 2 x 2 x 2 leaves.  Every leaf carries
 * degree-p Lagrange functions on GLL nodes (p in [1, 5]) and an n_quad^3
 * Gauss-Legendre rule (n_quad in [p + 1, 8]).  A fine-leaf node on the closed
 * box of a coarse leaf that is not one of its nodes hangs: its value is the
 * coarse leaf's interpolant there, u_all = P u_free.  The handle owns the mesh
 * and P on the device.  Errors: EFE_ERR_ARG (sizes, a refined cell outside
 * the grid), EFE_ERR_NOMEM, EFE_ERR_CUDA; message by efe_octree_last_error(NULL). */
typedef struct efe_octree efe_octree;
efe_status efe_octree_setup(const double* lo_host, const double* hi_host, int32_t nc, int32_t degree, int32_t n_quad,
                            const int32_t* refine_host, int32_t n_refine, efe_octree** out);
efe_status efe_octree_destroy(efe_octree* oct);
const char* efe_octree_last_error(const efe_octree* oct);
/* The same mesh described on the host only (no device work, no handle): the
 * constraint matrix P in CSR over all nodes (row_start [n_all + 1], col
 * [nnz] free-node indices, val [nnz] weights; a free node's row is its own
 * index with weight 1), node coordinates all_xyz [n_all][3] and free_xyz
 * [n_free][3].  Call with NULL arrays to read n_all, n_free and nnz first. */
efe_status efe_octree_constraints(const double* lo_host, const double* hi_host, int32_t nc, int32_t degree,
                                  int32_t n_quad, const int32_t* refine_host, int32_t n_refine, int64_t* n_all,
                                  int64_t* n_free, int64_t* nnz, int64_t* row_start, int32_t* col, double* val,
                                  double* all_xyz, double* free_xyz);
/* Counts: free (unconstrained) nodes, all nodes, leaves, quadrature points per
 * leaf, hanging nodes (any pointer may be NULL). */
efe_status efe_octree_sizes(const efe_octree* oct, int64_t* n_free, int64_t* n_all, int64_t* n_leaves, int64_t* n_q,
                            int64_t* n_hanging);
/* Host copies: free-node coordinates [n_free][3], the leaves' Gauss-Legendre
 * points [n_leaves][n_q][3] (first axis fastest), boundary flags [n_free]
 * (1 on the domain boundary); any pointer may be NULL. */
efe_status efe_octree_coords(const efe_octree* oct, double* free_xyz_host, double* quad_xyz_host,
                             uint8_t* boundary_host);
/* Y = P^T (kin (1/2) K + V) P X in the constrained space (Eq. Hmn on the
 * locally refined mesh): K the stiffness int grad N . grad N, V the potential
 * matrix int v N N with v given at every leaf's Gauss-Legendre points (vq_dev:
 * device [n_leaves][n_q]).  X_dev, Y_dev: device [n_free][n_cols] doubles
 * (real columns, 1 <= n_cols <= 65535).  mask_boundary 1 applies the
 * Dirichlet restriction: boundary entries of X read as 0 and boundary rows of
 * Y are 0; mask_boundary 2 gives the Loewdin-scaled operator on top of it,
 * Y = D P^T (kin K/2 + V) P D X (Eq. TDKSDiscrete2) with D = mask / sqrt(m),
 * m the lumped mass of the constrained space: the row sums of P^T M_GLL P,
 * i.e. P^T m_all with m_all the GLL-lumped weights of all nodes.  Three stages (gather through P, per-leaf operator scatter-added
 * over all nodes, scatter through P^T); stream-ordered; the first call with
 * more columns than before allocates scratch (2 n_all n_cols doubles).
 * Errors: EFE_ERR_ARG, EFE_ERR_NOMEM, EFE_ERR_CUDA. */
efe_status efe_octree_apply(efe_octree* oct, const double* vq_dev, double kin, const double* X_dev, double* Y_dev,
                            int64_t n_cols, int32_t mask_boundary, void* stream);
/* The Poisson problem on the locally refined mesh (the operator of the Hartree
 * solve, Eqs. Hartree_possion and DiscretePoisson, without the 1/4pi that the
 * caller folds into f): -lap u = f with u = g on the boundary, i.e.
 * K_II u_I = F_I - K_IB g_B in the constrained space, F = P^T int f N with f at
 * every leaf's Gauss-Legendre points (f_q_dev: device [n_leaves][n_q]); g_free_dev
 * and u_dev: device [n_free] (g read on the boundary free nodes only).
 * Conjugate gradients on the constrained stiffness, Jacobi-preconditioned by its
 * diagonal (assembled at set-up), to |r| <= tol |r_0|, at most
 * max_it iterations (*iters_host receives the count); synchronises `stream`
 * every iteration.  Errors: EFE_ERR_ARG, EFE_ERR_CG_NOCONV (u holds the last
 * iterate), EFE_ERR_NOT_SPD, EFE_ERR_NOMEM, EFE_ERR_CUDA. */
efe_status efe_octree_poisson(efe_octree* oct, const double* f_q_dev, const double* g_free_dev, double* u_dev,
                              double tol, int32_t max_it, int32_t* iters_host, void* stream);
/* The density at every leaf's Gauss-Legendre points (the density of Sec. TDKS on
 * the locally refined mesh) for orbitals in the Loewdin basis: psi = D psi_bar
 * with D = mask / sqrt(m) (m the lumped constrained mass), rho = sum_a occ_a
 * |sum_i N_i psi_a,i|^2.  psi_bar_dev: device complex128 [n_free][n_orb]
 * (interleaved real and imaginary parts); occ_host: host [n_orb]; rho_dev:
 * device [n_leaves][n_q].  Synchronises `stream`.  Errors: EFE_ERR_ARG,
 * EFE_ERR_NOMEM, EFE_ERR_CUDA. */
efe_status efe_octree_density(efe_octree* oct, const double* psi_bar_dev, int32_t n_orb, const double* occ_host,
                              double* rho_dev, void* stream);
/* Values at every leaf's Gauss-Legendre points of n_cols real nodal columns of
 * the constrained space (u_all = P u, then the leaf interpolants; e.g. the
 * Hartree potential from efe_octree_poisson): u_free_dev device [n_free][n_cols],
 * out_q_dev device [n_cols][n_leaves][n_q].  Stream-ordered.  Errors:
 * EFE_ERR_ARG, EFE_ERR_NOMEM, EFE_ERR_CUDA. */
efe_status efe_octree_interp(efe_octree* oct, const double* u_free_dev, int32_t n_cols, double* out_q_dev,
                             void* stream);
/* One predictor-corrector Magnus step (Eq. ApproxMagnus) on the locally refined
 * mesh, each exponential as in efe_octree_kexp (Krylov dimension k, or adaptive up to
 * k with krylov_tol > 0): psi_p = exp(-i dt Hbar[v(rho_n)]) psi_n,
 * rho_mid = (rho_n + rho(psi_p)) / 2, psi_n+1 = exp(-i dt Hbar[v(rho_mid)]) psi_n,
 * v = -sum Z / |x - R| + v_H + v_xc - E . x at the leaves' Gauss-Legendre points
 * (field_host: double[3], E at the mid-point), v_H from -lap v_H = 4 pi rho with the
 * Dirichlet data sum Z / |x - R| (efe_octree_poisson to cg_tol), v_xc the LDA xc.
 * Those Dirichlet data are the electrons' far field only for a neutral system
 * (sum_a occ_a ||psi_a||^2 = sum Z): a precondition, as on the rectilinear mesh.
 * psi_bar_dev: device complex128 [n_free][n_orb] in the Loewdin basis, in place;
 * occ_host [n_orb]; atoms_host [n_atoms][4] = Z, x, y, z; dt finite and > 0;
 * xc EFE_XC_PW92 or EFE_XC_PZ81.  Allocates per call and synchronises `stream`.
 * Errors: EFE_ERR_ARG (message set), EFE_ERR_CG_NOCONV, EFE_ERR_NOMEM,
 * EFE_ERR_CUDA (also for a kernel fault surfacing at the final synchronisation). */
efe_status efe_octree_magnus_step(efe_octree* oct, double* psi_bar_dev, int32_t n_orb, const double* occ_host,
                                  const double* atoms_host, int32_t n_atoms, const double* field_host, double dt,
                                  int32_t k, double krylov_tol, double cg_tol, int32_t xc, void* stream);
/* psi_bar <- exp(-i dt Hbar) psi_bar on the locally refined mesh, Hbar the
 * Loewdin-scaled operator of efe_octree_apply (mode 2) with kin and v at the
 * leaves' Gauss-Legendre points (vq_dev [n_leaves][n_q]): per complex column,
 * Lanczos steps of the three-term recurrence (Eq. AdaptiveKrylov), the exponential
 * of the m x m tridiagonal matrix from its eigendecomposition, psi_bar =
 * |psi_bar| Q_m y.  tol <= 0: m = k for every column; tol > 0: each column stops at
 * the first m <= k whose estimate |dt| beta_m |psi| |[exp(-i dt T_m) e_1]_m| (Eq.
 * AdaptiveKrylovErr) is at most tol, or whose recurrence breaks down.  *k_used_host
 * (may be NULL) receives the largest m.  psi_bar_dev: device complex128
 * [n_free][n_cols], in place (boundary rows set to 0).  Allocates (k + 1) n_free
 * n_cols complex scratch per call; synchronises `stream` every step.  Returns
 * EFE_WARN_KRYLOV_CAP (result written) if a column reached k with its estimate above
 * tol.  Errors: EFE_ERR_ARG (k outside [1, 64], tol not finite), EFE_ERR_NOMEM,
 * EFE_ERR_CUDA. */
efe_status efe_octree_kexp(efe_octree* oct, const double* vq_dev, double kin, double* psi_bar_dev, int32_t n_cols,
                           double dt, int32_t k, double tol, int32_t* k_used_host, void* stream);

/* Host-only diagnostics of the electrostatic enrichment (no context, no device
 * work).  efe_atom_hartree_table: the atomic Hartree potentials that
 * efe_hartree_enriched uses, for atoms with charges Z_host [n_atoms] and the
 * wavefunction enrichment functions fns_host [n_fn]: r_host [n_tab] (r =
 * rmax t^2, t uniform on [0, 1]), v_host and q_host [n_atoms][n_tab] (potential
 * and enclosed charge), nel_host [n_atoms] (any output may be NULL).
 * efe_adaptive_cell_boxes: the boxes of efe_nuclear_enriched's adaptive rule
 * for one cell (origin_host, size_host: double[3]; atoms_host [n_atoms][4] =
 * Z, x, y, z), in the cell's reference coordinates [-1, 1]^3 as lo[3], hi[3]
 * per box; *n_boxes receives the count, boxes_host (NULL to query) needs
 * capacity >= the count.  Errors: EFE_ERR_ARG. */
efe_status efe_atom_hartree_table(const efe_enrich_fn* fns_host, int32_t n_fn, const double* Z_host, int32_t n_atoms,
                                  int32_t n_tab, double rmax, double* r_host, double* v_host, double* q_host,
                                  double* nel_host);
efe_status efe_adaptive_cell_boxes(const double* origin_host, const double* size_host, const double* atoms_host,
                                   int32_t n_atoms, double sigma, double r0, double s, int32_t n_quad, double tol,
                                   int32_t max_depth, int64_t* n_boxes, double* boxes_host, int64_t capacity);

/* The LDA at n points without a context (for meshes that have none, such as the
 * locally refined mesh): v_xc = d(rho e_xc)/d rho and e_xc of Slater exchange
 * plus the correlation xc (EFE_XC_PW92 or EFE_XC_PZ81), as efe_density_vxc
 * computes them.  rho_dev: device [n]; vxc_dev, exc_dev: device [n] (nullable).
 * Stream-ordered.  Errors: EFE_ERR_ARG, EFE_ERR_CUDA. */
efe_status efe_lda_points(const double* rho_dev, double* vxc_dev, double* exc_dev, int64_t n, int32_t xc, void* stream);

/* Spectra of dipole traces (Sec. Results: the absorption spectrum of the weak
 * perturbation study and the power spectrum of the high-harmonic study); no
 * context needed.  Samples at t_n = n dt, n = 0 .. n_t - 1, on the device;
 * time integrals by the trapezoid rule, F[f](w) = dt sum_n c_n f_n e^{i w t_n}
 * with c_0 = c_{n_t-1} = 1/2.  omega_dev: n_omega frequencies (a.u.).
 *
 * Absorption: S(w) = (4 w / (3 pi)) sum_j Im alpha_jj(w) with
 * alpha_jj = F[e^{-t/tau} (mu_j^(j)(t) - mu_j^(j)(0))] / F[E_0], mu^(j) the trace of
 * the run perturbed along axis j, read at mu_dev[j * stride_dir + n * stride_t + j]
 * (the j-th dipole component); F[E_0] from the n_t field samples field_dev, or
 * equal to kick (a delta kick of that strength) when field_dev is NULL.
 *
 * Power: P(w) = |dt sum_{n=1}^{n_t-2} e^{-i w t_n} a_n e^{-t_n^2/tau}|^2 with a_n the
 * central second difference of mu_dev[n * stride_t] (the dipole acceleration).
 *
 * Outputs S_dev / P_dev: n_omega doubles.  Errors: EFE_ERR_ARG (NULL pointers,
 * too few samples, dt or tau not positive, no field and kick 0), EFE_ERR_CUDA;
 * the message is read with efe_last_error(NULL). */
efe_status efe_absorption_spectrum(const double* mu_dev, int64_t n_t, int64_t stride_dir, int64_t stride_t, double dt,
                                   const double* field_dev, double kick, const double* omega_dev, int64_t n_omega,
                                   double tau, double* S_dev, void* stream);
efe_status efe_power_spectrum(const double* mu_dev, int64_t n_t, int64_t stride_t, double dt, const double* omega_dev,
                              int64_t n_omega, double tau, double* P_dev, void* stream);

/* Diagnostics (not part of the method).  efe_profile(ctx, 1) synchronises the
 * device, resets a process-wide counter of kernel launches made by the library,
 * and from then on brackets every launch of the cell-apply kernel with a pair of
 * CUDA events recorded on the launching stream; efe_profile(ctx, 0) stops the
 * timing.  efe_profile_read synchronises the device and returns the launches
 * counted since the last efe_profile call, the cell-apply launches timed, and
 * their summed device time in milliseconds (any pointer may be NULL). */
efe_status efe_profile(efe_ctx* ctx, int32_t enable);

/* Tile-width autotuner of the cell apply (diagnostics and tests).  The first apply
 * of each precision and column count times variant 0 (widest tile: two blocks per
 * SM) and variant 1 (half as wide) and keeps the faster.  efe_tuning reports the
 * choice (-1: not tuned yet) and the timed milliseconds; force_variant 0 or 1
 * fixes the variant for applies of n_orb * batch columns, -1 leaves it. */
efe_status efe_tuning(efe_ctx* ctx, int32_t precision, int32_t force_variant, int32_t* variant, float* ms0,
                      float* ms1);

/* Diagnostics (not part of the method): checks, on the current device, the
 * integer-pipe binary64 <-> binary32 conversions the mixed-precision kernels
 * use against the hardware conversions, bit for bit, on n seeded patterns per
 * direction (normal binary32 range, a quarter of the doubles exact
 * round-to-nearest ties).  *mismatches_host receives the count (0 expected).
 * Synchronises the device. */
efe_status efe_selftest(int64_t n, int64_t* mismatches_host);

/* Diagnostics (not part of the method): the number of polls after which a progress wait of
 * the tensor-core apply (the completion of its operand copies and MMAs, and of the other
 * warps' stages) gives up; 0 restores the default (seconds).  A wait that gives up makes the
 * kernel stop its work, wait (with the default limit) for the copies and MMAs already in
 * flight, free its tensor memory and return; the next efe_magnus_step with step info reports
 * EFE_ERR_TIMEOUT once and the context stays usable (reset its state: the orbitals of that step
 * are not meaningful).  For tests of the timeout path.  Errors: EFE_ERR_ARG. */
efe_status efe_set_wait_limit(efe_ctx* ctx, int64_t polls);

/* Orbital (column) partition across processes.  The density rho_q = sum_alpha f_alpha
 * |psi_alpha(x_q)|^2 (Eq. rho of Section 2) is a sum over orbitals, and the Krylov exponential
 * of Section 4.2 acts on each orbital by itself, so G processes may each own a subset of the
 * orbitals (each process sets up its context with its own n_orb, occupations and orbitals)
 * as long as every density a step forms is summed over all processes before it is used.
 * efe_set_density_reduce installs that sum: after each density of the context's own orbitals
 * (the state density of S6 and at the first step, the predictor density of S2, and the one of
 * efe_density_vxc), and before anything reads it, the step calls
 *   fn(rho_dev, n, stream, user)
 * on the host with rho_dev the device float64 [batch][n_cells][n_q] partial density (n values)
 * and `stream` the step's stream; fn must replace it in place by the sum over all processes,
 * in order on `stream` (e.g. an NCCL all-reduce on that stream), and return 0, or non-zero for
 * an error (the step then returns EFE_ERR_CUDA with a message).  LDA, the Hartree solve
 * (replicated: every process solves the same Poisson problem) and the dipole then read the
 * summed density, so every process holds the same potentials and dipole.  The call is made
 * outside the CUDA graphs of the Krylov loops (they never read a density).  fn = NULL removes
 * it.  Errors: EFE_ERR_ARG. */
typedef int (*efe_reduce_fn)(double* rho_dev, int64_t n, void* stream, void* user);
efe_status efe_set_density_reduce(efe_ctx* ctx, efe_reduce_fn fn, void* user);

/* Forward checkpoint and resume (not part of the method; a propagation of thousands of
 * steps must survive an interrupted job).  efe_checkpoint_save writes psi_bar_dev (device
 * complex128 [n_dof][n_orb * batch]), t, step and the context's density-derived state (rho_n,
 * v_H, v_xc at the quadrature points, the nodal Hartree potential, and the previous step's
 * v_Hxc when the context holds them, and the adaptive Krylov sub-step count) to `path`, through `path`.tmp and a rename; it
 * synchronises `stream`.  efe_checkpoint_load checks the file (magic, version, the sizes of this
 * context, payload length, 64-bit FNV-1a checksum) before copying anything, then fills
 * psi_bar_dev, *t_host, *step_host and restores the state, so the next efe_magnus_step
 * continues the saved run.  Errors: EFE_ERR_ARG (null pointer, unreadable, corrupt or
 * truncated file, sizes of another context; message in efe_last_error), EFE_ERR_NOMEM,
 * EFE_ERR_CUDA. */
efe_status efe_checkpoint_save(efe_ctx* ctx, const char* path, const double* psi_bar_dev, double t, int64_t step,
                               void* stream);
efe_status efe_checkpoint_load(efe_ctx* ctx, const char* path, double* psi_bar_dev, double* t_host,
                               int64_t* step_host, void* stream);
/* Host-only forms of the same file (no device, no context): efe_checkpoint_write_host writes
 * host arrays in the layout above (sizes: n_dof, complex columns, batch, n_cells, n_q, n_h;
 * rho/vH/vxc/phi all NULL or all given, vprev only with them); efe_checkpoint_inspect validates a
 * file and returns its sizes, t, step and which parts it holds.  Errors: EFE_ERR_ARG, with the
 * reason in efe_checkpoint_last_error(). */
efe_status efe_checkpoint_write_host(const char* path, const int64_t* sizes, double t, int64_t step,
                                     const double* psi_host, const double* rho_host, const double* vH_host,
                                     const double* vxc_host, const double* phi_host, const double* vprev_host);
efe_status efe_checkpoint_inspect(const char* path, int64_t* sizes, double* t, int64_t* step, int32_t* has_state,
                                  int32_t* has_prev);
const char* efe_checkpoint_last_error(void);

/* Diagnostics (not part of the method): measured throughput of the float32 and
 * float64 fused-multiply-add pipes of the current device in TFLOP/s (2 flops per
 * FMA; eight independent chains per thread, eight blocks of 256 threads per SM,
 * CUDA events around one launch after a warm-up).  These are the peaks the
 * roofline fractions of the float32-pair and float64 cell kernels are stated
 * against.  Allocates and frees a small device buffer and synchronises the device.
 * Errors: EFE_ERR_ARG (null pointer), EFE_ERR_CUDA. */
efe_status efe_pipe_peaks(double* fp32_tflops_host, double* fp64_tflops_host);
/* Diagnostics (not part of the method): the Krylov basis of the context's last Lanczos run (the
 * last column block of its last exponential).  *q_dev: device complex128 basis, vector j of the
 * c = *cols columns at q_dev + 2 j n_dof c, [n_dof][c] row-major (V_j = s_j q_j, unnormalised:
 * s_0 = 1, s_j = beta_{j-1}); *norms_dev: device float64 [k_max][c], row j - 1 holding s_j;
 * *kused_dev: device int32 [c], the Lanczos vectors each column used.  The pointers belong to the
 * context and stay valid until its next step, apply or exponential.  Errors: EFE_ERR_ARG (null
 * pointer, no Lanczos run yet). */
efe_status efe_krylov_basis(efe_ctx* ctx, const double** q_dev, const double** norms_dev, const int32_t** kused_dev,
                            int64_t* cols);
efe_status efe_profile_read(efe_ctx* ctx, int64_t* launches, int64_t* apply_launches, double* apply_ms);

#ifdef __cplusplus
}
#endif

#endif /* EFE_H */
