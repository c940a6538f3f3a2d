// Internal declarations of libefe (not part of the public C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/efe.h"

namespace efe {

constexpr int kMaxP1 = 6;    // degree <= 5
constexpr int kMaxNQ1 = 7;   // n_quad = p + 2
constexpr int kMaxK = 64;    // Lanczos cap
constexpr int kThreads = 256;

// A value held as an unevaluated sum h + l of two binary32 numbers (the
// FP32-pair precision of the cell apply; arithmetic in sumfact.cuh).
struct __align__(8) df32 {
  float h, l;
  df32() = default;
  __host__ __device__ constexpr df32(float h_, float l_ = 0.0f) : h(h_), l(l_) {}
  // nearest pair to a double (host side: tables and set-up)
  static df32 split(double x) {
    const float h = (float)x;
    return df32(h, (float)(x - (double)h));
  }
};

// 1D reference tables on [-1, 1], passed to kernels by value (parameter space is
// the constant bank, so warp-uniform reads broadcast).
struct RefTables {
  double B1[kMaxNQ1 * kMaxP1];   // l_i(xg_q), [q][i]
  double D1[kMaxNQ1 * kMaxP1];   // l_i'(xg_q)
  double K1[kMaxP1 * kMaxP1];    // int l_i' l_j'
  double M1[kMaxP1 * kMaxP1];    // int l_i l_j
  double wg[kMaxNQ1];            // GL weights
  double xg[kMaxNQ1];            // GL points
  float B1f[kMaxNQ1 * kMaxP1];
  float D1f[kMaxNQ1 * kMaxP1];
  float K1f[kMaxP1 * kMaxP1];
  float M1f[kMaxP1 * kMaxP1];
  df32 B1p[kMaxNQ1 * kMaxP1];
  df32 D1p[kMaxNQ1 * kMaxP1];
  df32 K1p[kMaxP1 * kMaxP1];
  df32 M1p[kMaxP1 * kMaxP1];
};

// Rectilinear mesh, device view (pointers to per-axis arrays).
struct MeshView {
  int ncx, ncy, ncz;
  int Nx, Ny, Nz;
  int p;
  int nc;
  long long n_h;
  const double* x0;   // cell origins, x then y then z, size ncx + ncy + ncz
  const double* h;    // cell sizes, same layout
};

__host__ __device__ inline void cell_ijk(const MeshView& m, int c, int& cx, int& cy, int& cz) {
  cx = c % m.ncx;
  int t = c / m.ncx;
  cy = t % m.ncy;
  cz = t / m.ncy;
}

__host__ __device__ inline long long node_index(const MeshView& m, int cx, int cy, int cz, int i1, int i2, int i3) {
  return (long long)(cx * m.p + i1) + (long long)m.Nx * ((long long)(cy * m.p + i2) + (long long)m.Ny * (cz * m.p + i3));
}

// Operator held by the context (one per batch member for the v-dependent parts).
struct Operator {
  int batch = 0;
  double kin = 1.0;
  double* W64 = nullptr;    // [batch][nc][nq]  w_q |J| v(x_q)
  float* W32 = nullptr;
  double* E64 = nullptr;    // [batch][n_pairs][nn] classical-enriched coupling E_c
  float* E32 = nullptr;
  df32* W2 = nullptr;       // FP32-pair copies for EFE_PAIR
  df32* E2 = nullptr;
  double* HEE = nullptr;    // [batch][nE][nE] enriched-enriched block (before M^ee^-1/2 scaling)
  bool valid = false;
};

// Tensor-core form of the operator (EFE_TC): bf16 slices of the dense cell matrices and
// of the enrichment coupling in the shared-memory image the MMA reads (k_tc.cu).
struct TcState {
  int batch = 0;                  // members the slices are allocated for
  unsigned char* H = nullptr;     // [batch][nc][4 slices][128 x 128 bf16]
  int* rexp = nullptr;            // [batch][nc][128] row exponents of H_c
  int* rexpE = nullptr;           // [batch][n_items][128] row exponents of E_c (per item)
  unsigned char* E = nullptr;     // [batch][e_total][2048 B]: per cell, [E_c slice i | E_c^T slice i], i = 0..3
  int* hexp = nullptr;            // [batch][n_pairs] row exponents of E_c^T
  long long* eoff = nullptr;      // [n_items + 1] prefix sums of the padded function counts
  long long e_total = 0;
  // work items: a cell coupled to more enrichment functions than one pass takes is split into
  // several items (the first carries H_c); [4][n_items]: cell, first pair, pairs, flags
  int n_items = 0;
  int* items = nullptr;
  int* first_item = nullptr;      // [nc + 1] first item of each cell
  int* err = nullptr;             // set by a tensor-core wait that gave up
  int n_sm = 0;                   // SMs of the context's device (persistent grid)
};

// Hartree potential in the electrostatically enriched basis (k_electro.cu), installed by
// efe_hartree_enriched: one enrichment function per atom, the atom's Hartree potential
// (shell-filled neutral atom, tabulated) times the smooth cutoff; the eliminated block is
// precomputed so that every solve is the direct Poisson solve plus rank-nA corrections.
struct HartreeEnr {
  bool on = false;
  int nA = 0, n_tab = 0;
  double r0 = 0, s = 0, rmax = 0;
  double* C = nullptr;       // [nA][n_h] orthogonalisation coefficients int N^A_J N_i / M_i
  double* G = nullptr;       // [nA][n_h] int grad N^A_J . grad N_n
  double* X = nullptr;       // [nA][n_h] A_II^-1 A_IJ
  double* Sinv = nullptr;    // [nA][nA] (A_EE - A_EI X)^-1
  double* atoms = nullptr;   // [nA][4] Z, x, y, z
  double* r = nullptr;       // [n_tab] radial grid
  double* v = nullptr;       // [nA][n_tab] atomic Hartree potentials
  double* q = nullptr;       // [nA][n_tab] enclosed charges
  double* nel = nullptr;     // [nA] electrons per atom
  int* pair_cell = nullptr;  // (cell, atom) pairs of the supports, for the per-solve loads
  int* pair_fn = nullptr;
  long long n_pairs = 0;
  double* small = nullptr;   // [6][nA][batch] loads int rho N^A, right sides, coefficients, 3 partial dots
};
void hen_free(HartreeEnr& h);

// Per-launch timing of the cell-apply kernel (enabled by efe_profile).
struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> pool;   // pairs (start, stop)
  size_t used = 0;                 // events used since the last read
  long long apply_launches = 0;
};

struct Ctx {
  int device = 0;
  Prof prof;
  std::string err;
  // sizes
  int p = 0, P1 = 0, NQ1 = 0, nn = 0, nq = 0;
  int ncx = 0, ncy = 0, ncz = 0, nc = 0;
  int Nx = 0, Ny = 0, Nz = 0;
  long long n_h = 0;
  int nE = 0;
  long long n_dof = 0;
  int n_atoms = 0;
  std::vector<double> Z, R;               // host copies
  std::vector<efe_enrich_fn> fns;
  double r0 = 0, s = 0;
  std::vector<double> xb, yb, zb;
  RefTables tab{};
  MeshView mesh{};
  // options
  int n_orb = 0, batch = 0;
  std::vector<double> occ;
  double krylov_tol = 1e-12;
  int k_max = 16, fixed_k = 0;
  double cg_tol = 1e-12;
  int cg_max_it = 2000;
  int precision = EFE_FP64;
  int hartree_method = EFE_HARTREE_FDM;
  int xc = EFE_XC_PW92;
  int scheme = EFE_STEP_PC;
  // device tables
  double* d_geo = nullptr;     // x0 (ncx+ncy+ncz) then h (ncx+ncy+ncz)
  double* d_Dsc = nullptr;     // [n_h] mask / sqrt(M)
  double* d_M = nullptr;       // [n_h] lumped mass
  double* d_occ = nullptr;     // [n_orb]
  double* d_vN = nullptr;      // [nc][nq]
  double* d_wJ = nullptr;      // [nc][nq]
  double* d_xq = nullptr;      // [nc][nq][3]
  // enrichment support: pairs (cell, function), CSR by cell
  long long n_pairs = 0;
  int* d_pair_start = nullptr; // [nc + 1]
  int* d_pair_fn = nullptr;    // [n_pairs]
  int* d_pair_cell = nullptr;  // [n_pairs]
  double* d_Atil = nullptr;    // [n_pairs][nq] values of N^E at quadrature points
  double* d_KE = nullptr;      // [n_pairs][nn] 1/2 int grad N_i . grad N^E
  double* d_KEE = nullptr;     // [nE][nE] 1/2 int grad N^E . grad N^E
  double* d_S = nullptr;       // [nE][nE] (M^ee)^-1/2
  double* d_Shalf = nullptr;   // [nE][nE] (M^ee)^1/2
  std::vector<double> Mee, S, Shalf;
  int max_pairs_per_cell = 0;
  // Poisson
  double* d_diagA = nullptr;   // [n_h] diagonal of (1/4pi) K at interior nodes (1 elsewhere)
  double* d_phiB = nullptr;    // [n_h] Dirichlet data (zero inside)
  double* d_phi = nullptr;     // [n_h][batch] warm start / last solution
  double* d_phiB_nb = nullptr; // [n_h][batch] Dirichlet data per member
  int fdm_n[3] = {0, 0, 0};    // interior 1D sizes
  double* d_fdmV[3] = {nullptr, nullptr, nullptr};   // 1D generalised eigenvectors
  double* d_fdmL[3] = {nullptr, nullptr, nullptr};   // 1D eigenvalues
  double* d_fdmT = nullptr;    // [2][batch][nx ny nz] transform scratch
  // operators
  Operator op;                 // current operator (efe_set_potential / magnus)
  TcState tc;                  // its tensor-core slices, rebuilt with it while tc_on
  HartreeEnr hen;              // enriched Hartree solve (off unless installed)
  bool tc_on = false;
  // autotuned cell-apply tile width per precision [FP64, MIXED, PAIR]: variant 0 (widest tile
  // fitting two blocks per SM) or 1 (half as wide); -1 until timed
  const int* apply_gate = nullptr;   // device count of active Lanczos columns (graph mode), else NULL
  // CUDA graphs of the Lanczos exponential, keyed by (in, out, precision, columns, kin, generation)
  struct KexpGraph {
    const double* in;
    double* out;
    int precision;
    long long C;
    double kin;
    long long gen;
    cudaGraphExec_t exec;
  };
  std::vector<KexpGraph> graphs;
  std::vector<KexpGraph> graph_seen;   // keys run eagerly once (tuning) before capture
  long long ws_gen = 0;                // bumped whenever workspaces or operator buffers move
  bool use_graphs = false;
  int kblock_opt = 0;          // krylov_block option (0: automatic)
  int substeps_opt = 1;        // krylov_substeps option (0: adaptive)
  bool reorth = false;         // krylov_reorth: CGS2 reorthogonalisation in the Lanczos loop
  int substeps_cur = 1;        // adaptive: sub-steps of the next exponential
  uint32_t tc_wait_limit = 0;  // polls of the tensor-core apply's progress waits (0: the default)
  efe_reduce_fn rho_reduce = nullptr;  // sum of the partial densities over processes (orbital partition)
  void* rho_reduce_user = nullptr;
  long long kblock = 0;        // complex columns per Lanczos run (the Krylov basis width)
  long long lz_last_C = 0;     // columns of the last Lanczos run (0: none yet)
  cudaStream_t cap_stream = nullptr;
  int tile_choice[3] = {-1, -1, -1};
  long long tile_cols[3] = {-1, -1, -1};
  float tile_ms[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  // state (density-derived potentials of the current step)
  bool state_valid = false;
  bool has_prev = false;       // d_vprev holds v_H + v_xc of the previous step
  double* d_vprev = nullptr;   // [batch][nc][nq]
  double* d_rho = nullptr;     // [batch][nc][nq]
  double* d_vH = nullptr;
  double* d_vxc = nullptr;
  // workspaces
  long long ws_cols = 0;       // complex columns the workspaces are sized for
  double* d_Q = nullptr;       // [(k_max + 1)][n_dof][cols] complex
  double* d_psi_p = nullptr;   // [n_dof][cols] complex
  double* d_xE = nullptr;      // [nE][2 cols] S x^E
  float* d_xE32 = nullptr;     // float copy
  df32* d_xE2 = nullptr;       // pair copy
  double* d_yE = nullptr;      // [nE][2 cols] enriched accumulator
  double* d_lz = nullptr;      // Lanczos scalars per column (see k_vector.cu)
  int* d_lzi = nullptr;        // Lanczos integer state per column
  double* h_lz = nullptr;      // pinned mirror for step info
  int* h_flag = nullptr;       // pinned flag
  double* d_rho2 = nullptr;    // [batch][nc][nq] scratch densities
  double* d_v = nullptr;       // [batch][nc][nq] potential scratch
  double* d_cg = nullptr;      // CG vectors [5][n_h][batch] + scalars
  double* d_red = nullptr;     // reduction scratch
  ~Ctx();
};

// process-wide count of kernel launches (diagnostics)
void note_launch();
long long launch_count();
void reset_launch_count();
// returns (start, stop) events to bracket one cell-apply launch, or nulls when timing is off
void prof_pair(Ctx& c, cudaEvent_t& a, cudaEvent_t& b);

cudaError_t run_selftest_cvt(long long n, long long* mismatches);

// ---- host math (host_math.cu)
void gauss_legendre(int n, double* x, double* w);
void gauss_lobatto(int p, double* x, double* w);
void lagrange_tables(int n_nodes, const double* nodes, int n_pts, const double* pts, double* L, double* dL);
bool jacobi_eigen(int n, std::vector<double>& A, std::vector<double>& V, std::vector<double>& lam);

// ---- launch wrappers (k_*.cu); all return cudaGetLastError() of the launch
cudaError_t launch_geometry(const Ctx& c, cudaStream_t s);                       // wJ, xq, vN
cudaError_t launch_enrich_setup(Ctx& c, cudaStream_t s);                         // Atil, KE, KEE, Mee parts
cudaError_t launch_poisson_setup(Ctx& c, cudaStream_t s);                        // diagA, phiB
cudaError_t launch_coords(const Ctx& c, double* nodes, double* quad, cudaStream_t s);
cudaError_t launch_init_orbitals(const Ctx& c, double* psi, int n_gauss, const double* d_centers,
                                 const double* d_expo, const double* d_coef, const double* d_enr, cudaStream_t s);

// operator build: W = wJ * v (per member), E = kin*KE + B^T (W Atil), HEE = kin*KEE + Atil^T W Atil
cudaError_t launch_build_operator(Ctx& c, const double* v, int batch, double kin, cudaStream_t s);
// Y = Hbar X on n_cols complex columns (per member operator), ld in complex entries
cudaError_t launch_apply(Ctx& c, const double* X, double* Y, long long n_cols, long long ld, int precision,
                         cudaStream_t s);

// enrichment pre/post steps of an apply: xE = S X^E (and float copies); Y^E = S (yE + HEE xE)
cudaError_t launch_enr_pre(Ctx& c, const double* X, long long ld2, int ncols2, cudaStream_t s);
cudaError_t launch_enr_post(Ctx& c, double* Y, long long ld2, int ncols2, int cols_member, cudaStream_t s);
// tensor-core operator (k_tc.cu): reason EFE_TC cannot serve this context, or NULL
const char* tc_unsupported(const Ctx& c, int cols_member);
cudaError_t launch_tc_build(Ctx& c, int batch, cudaStream_t s);
cudaError_t launch_tc_apply(Ctx& c, const double* X, double* Y, long long n_cols, long long ld, cudaStream_t s);
void tc_free(TcState& t);

// Lanczos exponential: out = Kexp(-i dt_col Hbar) in for every complex column, with the
// operator held in Ctx::op; dts_host [n_cols]; host-visible statistics after a stream sync.
cudaError_t run_kexp_cols(Ctx& c, const double* in, double* out, const double* dts_host, int precision,
                          int* kmax_used, int* cap_hits, double* eps_max, cudaStream_t s, bool need_stats = true);

// out = Kexp(-i dt_col Hbar) in again, for the start vectors of the last run_kexp_cols, from its
// Krylov basis and tridiagonal matrices (|dt_col| no larger than that run's; no applies)
// device pointers to the norms of the basis vectors (beta_{j-1} for V_j: [kMaxK][C]) and used
// dimensions (int [C]) of the last Lanczos run
void lz_last_views(const Ctx& c, const double** norms, const int** kused);
cudaError_t run_kexp_recombine(Ctx& c, double* out, const double* dts_host, cudaStream_t s);

// density / xc / dipole
cudaError_t launch_density(Ctx& c, const double* psi, double* rho, cudaStream_t s);
cudaError_t launch_lda(const Ctx& c, const double* rho, double* vxc, double* exc, long long n, cudaStream_t s);
cudaError_t launch_dipole(const Ctx& c, const double* rho, double* mu, cudaStream_t s);
double field_amp(const efe_field& f, double t);
cudaError_t launch_potential_sum(const Ctx& c, const double* vH, const double* vxc, const double* E_host,
                                 bool nuclear, double* v, cudaStream_t s);
cudaError_t launch_laplace(const Ctx& c, const double* x, double* y, int nb, int mask_in, double scale,
                           cudaStream_t s);
cudaError_t launch_load_vector(const Ctx& c, const double* f, double* d, int nb, cudaStream_t s);
cudaError_t launch_interp(const Ctx& c, const double* x, double* out, int nb, cudaStream_t s);
cudaError_t launch_axpby(double* y, const double* a, const double* b, double ca, double cb, long long n,
                         cudaStream_t s);
// fast-diagonalisation Hartree solve (k_poisson.cu)
cudaError_t setup_fdm(Ctx& c);
cudaError_t fdm_solve(Ctx& c, const double* d, double* Ap, double* phi, int nb, cudaStream_t s,
                      bool homogeneous = false, const double* phiB = nullptr);
// nuclear potential of smeared nuclei in the electrostatically enriched basis (k_electro.cu):
// replaces d_vN; phiE_host [n_atoms] receives the enrichment coefficients (nullable)
efe_status nuclear_enriched(Ctx& c, double sigma, double r0, double s, int sub, int n_quad, double adapt_tol,
                            int adapt_depth, double* phiE_host, cudaStream_t st);
// installs the enriched Hartree solve (k_electro.cu)
efe_status hartree_enrich_install(Ctx& c, double r0, double s, int sub, int n_quad, cudaStream_t st);
// the enriched Hartree solve for the load d = int rho N ([n_h][batch], assembled): the classical part
// into c.d_phi, v_H at the quadrature points into vH; Ap, Lz, u: [n_h][batch] scratch
cudaError_t hartree_enriched_solve(Ctx& c, const double* rho, double* vH, const double* d, double* Ap, double* Lz,
                                   double* u, cudaStream_t s);
// its transpose for the adjoint (batch 1): out = I (Z h - W^T t) + sum_J t_J N^A_J for gw = g / w
// (out may alias gw; the caller multiplies by w); s1..s6 [n_h] scratch
cudaError_t hartree_enriched_vt(Ctx& c, const double* gw, double* out, double* s1, double* s2, double* s3, double* s4,
                                double* s5, double* s6, cudaStream_t s);
// context workspaces for C complex columns of leading dimension ld; the operator of v (api.cu)
efe_status ensure_ws(Ctx& c, long long C, long long ld);
efe_status ensure_krylov(Ctx& c);   // the Krylov basis (first exponential)
efe_status build_op(Ctx& c, const double* v, int batch, double kin, cudaStream_t s);
// reverse sweep of the dipole objective through n_steps Magnus steps (adjoint.cu)
efe_status adjoint_dipole(Ctx& c, const double* psi0, int n_steps, double dt, const efe_field& f, const double dir[3],
                          int w_first, int w_last, int K, int n_s, double* J_out, double grad[3], cudaStream_t s);
// spectra of dipole traces (spectra.cu)
cudaError_t launch_absorption(const double* mu, long long n_t, long long sdir, long long st, double dt,
                              const double* E, double kick, const double* om, long long n_om, double tau, double* S,
                              cudaStream_t s);
cudaError_t launch_power(const double* mu, long long n_t, long long st, double dt, const double* om, long long n_om,
                         double tau, double* P, cudaStream_t s);
// Hartree solve (direct or PCG); iters returned (synchronises for PCG)
efe_status run_hartree(Ctx& c, const double* rho, double* vH, double tol, int max_it, int* iters, cudaStream_t s);

}  // namespace efe

// The opaque handle of the C ABI wraps the context.
struct efe_ctx {
  efe::Ctx c;
};

#define EFE_CUDA_TRY(expr)                                                   \
  do {                                                                       \
    cudaError_t _e = (expr);                                                 \
    if (_e != cudaSuccess) return _e;                                        \
  } while (0)
