// C ABI of libefe (declared in include/efe.h): context lifecycle, set-up
// orchestration and the per-step drivers.  Every numerical step runs in the
// kernels of k_setup.cu, k_apply.cu and k_vector.cu; this file only sizes,
// allocates, validates and sequences them.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "efe_internal.h"


#include <atomic>

namespace efe {

static thread_local std::string g_setup_err;
static std::atomic<long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
void reset_launch_count() { g_launches.store(0); }

void prof_pair(Ctx& c, cudaEvent_t& a, cudaEvent_t& b) {
  a = b = nullptr;
  if (!c.prof.on) return;
  if (c.prof.used + 2 > c.prof.pool.size()) {
    for (int i = 0; i < 64; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      c.prof.pool.push_back(e);
    }
  }
  a = c.prof.pool[c.prof.used];
  b = c.prof.pool[c.prof.used + 1];
  c.prof.used += 2;
  c.prof.apply_launches += 1;
}

template <typename T>
static void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

Ctx::~Ctx() {
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  dfree(d_geo); dfree(d_Dsc); dfree(d_M); dfree(d_xE32); dfree(d_xE2);
  dfree(d_occ); dfree(d_vN); dfree(d_wJ); dfree(d_xq);
  dfree(d_pair_start); dfree(d_pair_fn); dfree(d_pair_cell); dfree(d_Atil); dfree(d_KE); dfree(d_KEE);
  if (d_phiB_nb != d_phiB) dfree(d_phiB_nb);
  d_phiB_nb = nullptr;
  dfree(d_S); dfree(d_Shalf); dfree(d_diagA); dfree(d_phiB); dfree(d_phi);
  for (int a = 0; a < 3; ++a) { dfree(d_fdmV[a]); dfree(d_fdmL[a]); }
  dfree(d_fdmT);
  dfree(op.W64); dfree(op.W32); dfree(op.E64); dfree(op.E32); dfree(op.W2); dfree(op.E2); dfree(op.HEE);
  tc_free(tc);
  hen_free(hen);
  dfree(d_rho); dfree(d_vH); dfree(d_vxc); dfree(d_vprev); dfree(d_Q); dfree(d_psi_p); dfree(d_xE); dfree(d_yE);
  dfree(d_lz); dfree(d_lzi); dfree(d_rho2); dfree(d_v); dfree(d_cg); dfree(d_red);
  for (cudaEvent_t e : prof.pool) cudaEventDestroy(e);
  for (auto& g : graphs) cudaGraphExecDestroy(g.exec);
  graphs.clear();
  if (cap_stream) cudaStreamDestroy(cap_stream);
  cap_stream = nullptr;
  if (h_flag) cudaFreeHost(h_flag);
  h_flag = nullptr;
  if (prev >= 0) cudaSetDevice(prev);
}

struct Fail {
  efe_status st;
};

static efe_status cuda_fail(Ctx& c, cudaError_t e, const char* what) {
  c.err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? EFE_ERR_NOMEM : EFE_ERR_CUDA;
}

#define TRY_CUDA(ctx, expr, what)                        \
  do {                                                   \
    cudaError_t _e = (expr);                             \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, what); \
  } while (0)

template <typename T>
static cudaError_t dalloc(T*& p, size_t n) {
  dfree(p);
  if (n == 0) n = 1;
  return cudaMalloc((void**)&p, sizeof(T) * n);
}

// Workspaces for C complex columns (predictor block, enrichment scratch, Lanczos scalars).  The
// Krylov basis is allocated by ensure_krylov at the first exponential.
efe_status ensure_ws(Ctx& c, long long C, long long ld) {
  const long long need_ld = std::max(C, ld);
  if (c.ws_cols >= need_ld) return EFE_OK;
  const long long n = c.n_dof;
  c.ws_gen += 1;   // captured graphs refer to the old buffers
  dfree(c.d_Q);
  c.kblock = 0;
  TRY_CUDA(c, dalloc(c.d_psi_p, (size_t)n * 2 * need_ld), "allocating the predictor block");
  TRY_CUDA(c, dalloc(c.d_xE, (size_t)std::max(c.nE, 1) * 2 * need_ld), "allocating enrichment scratch");
  TRY_CUDA(c, dalloc(c.d_xE32, (size_t)std::max(c.nE, 1) * 2 * need_ld), "allocating enrichment scratch");
  TRY_CUDA(c, dalloc(c.d_xE2, (size_t)std::max(c.nE, 1) * 2 * need_ld), "allocating enrichment scratch");
  TRY_CUDA(c, dalloc(c.d_yE, (size_t)std::max(c.nE, 1) * 2 * need_ld), "allocating enrichment scratch");
  TRY_CUDA(c, dalloc(c.d_lz, (size_t)(8 * kMaxK + 8) * need_ld), "allocating Lanczos scalars");
  TRY_CUDA(c, dalloc(c.d_lzi, (size_t)3 * need_ld + 8), "allocating Lanczos state");
  c.ws_cols = need_ld;
  return EFE_OK;
}

// The Krylov basis: k_max + 1 vectors of c.kblock complex columns, all n_orb * batch when they fit
// in the free device memory (or the krylov_block option), else the largest block that does (whole
// batch members when batch > 1); run_kexp_cols then runs the columns block by block.  The free
// memory left aside covers the densities and operator rebuilds and, for EFE_TC before its first
// build, the tensor-core operator; the basis takes at most three quarters of the rest.
efe_status ensure_krylov(Ctx& c) {
  if (c.d_Q && c.kblock > 0) return EFE_OK;
  const long long C = (long long)c.n_orb * c.batch;
  const size_t per_col = sizeof(double) * (size_t)(c.k_max + 1) * c.n_dof * 2;
  long long blk = C;
  if (c.kblock_opt > 0) {
    blk = std::min<long long>(C, c.kblock_opt);
  } else {
    size_t free_b = 0, total_b = 0;
    TRY_CUDA(c, cudaMemGetInfo(&free_b, &total_b), "querying device memory");
    size_t reserve = (size_t)8 << 30;
    if (c.precision == EFE_TC && !c.tc_on)
      reserve += (size_t)c.batch * ((size_t)c.nc * (4 * 128 * 128 * 2 + 2 * 128 * 4) +
                                    ((size_t)c.n_pairs + 16 * (size_t)c.nc) * (2048 + 4));
    // at most three quarters of what is left: the caller's own tensors come after the first step
    const long long fit = free_b > reserve ? (long long)((free_b - reserve) / 4 * 3 / per_col) : 1;
    blk = std::max<long long>(1, std::min(C, fit));
  }
  if (c.batch > 1 && blk < C) blk = std::max<long long>(1, blk / c.n_orb) * c.n_orb;   // whole members
  c.ws_gen += 1;
  TRY_CUDA(c, dalloc(c.d_Q, per_col / sizeof(double) * (size_t)blk), "allocating the Krylov basis");
  c.kblock = blk;
  return EFE_OK;
}

static efe_status ensure_batch_buffers(Ctx& c) {
  if (c.d_rho) return EFE_OK;
  const size_t nqb = (size_t)c.batch * c.nc * c.nq;
  TRY_CUDA(c, dalloc(c.d_rho, nqb), "allocating densities");
  TRY_CUDA(c, dalloc(c.d_vprev, nqb), "allocating the potential history");
  TRY_CUDA(c, dalloc(c.d_vH, nqb), "allocating potentials");
  TRY_CUDA(c, dalloc(c.d_vxc, nqb), "allocating potentials");
  TRY_CUDA(c, dalloc(c.d_rho2, nqb), "allocating densities");
  TRY_CUDA(c, dalloc(c.d_v, nqb), "allocating potentials");
  TRY_CUDA(c, dalloc(c.d_cg, (size_t)6 * c.n_h * c.batch + 5 * c.batch), "allocating CG vectors");
  TRY_CUDA(c, dalloc(c.d_phi, (size_t)c.n_h * c.batch), "allocating the Hartree potential");
  TRY_CUDA(c, cudaMemset(c.d_phi, 0, sizeof(double) * c.n_h * c.batch), "zeroing phi");
  return EFE_OK;
}

static efe_status ensure_operator(Ctx& c, int batch) {
  if (c.op.W64 && c.op.batch == batch) return EFE_OK;
  const size_t nqb = (size_t)batch * c.nc * c.nq;
  c.ws_gen += 1;
  TRY_CUDA(c, dalloc(c.op.W64, nqb), "allocating the operator");
  TRY_CUDA(c, dalloc(c.op.W32, nqb), "allocating the operator");
  TRY_CUDA(c, dalloc(c.op.E64, (size_t)batch * c.n_pairs * c.nn), "allocating the coupling blocks");
  TRY_CUDA(c, dalloc(c.op.E32, (size_t)batch * c.n_pairs * c.nn), "allocating the coupling blocks");
  TRY_CUDA(c, dalloc(c.op.W2, nqb), "allocating the operator");
  TRY_CUDA(c, dalloc(c.op.E2, (size_t)batch * c.n_pairs * c.nn), "allocating the coupling blocks");
  TRY_CUDA(c, dalloc(c.op.HEE, (size_t)batch * std::max(c.nE, 1) * std::max(c.nE, 1)), "allocating H_EE");
  c.op.batch = batch;
  c.op.valid = false;
  return EFE_OK;
}

efe_status build_op(Ctx& c, const double* v, int batch, double kin, cudaStream_t s) {
  efe_status st = ensure_operator(c, batch);
  if (st != EFE_OK) return st;
  c.op.kin = kin;
  TRY_CUDA(c, launch_build_operator(c, v, batch, kin, s), "building the operator");
  if (c.tc_on) TRY_CUDA(c, launch_tc_build(c, batch, s), "building the tensor-core operator");
  c.op.valid = true;
  return EFE_OK;
}

// ------------------------------------------------------------------ set-up
static bool validate(const efe_mesh_desc* mesh, const efe_atom* atoms, int n_atoms, const efe_enrich_desc* enr,
                     const efe_options* o, std::string& why) {
  if (!mesh || !o) { why = "mesh and options are required"; return false; }
  if (mesh->degree < 2 || mesh->degree > 5) { why = "degree must be in [2, 5]"; return false; }
  if (mesh->n_quad != mesh->degree + 2) { why = "n_quad must be degree + 2"; return false; }
  if (mesh->ncx < 1 || mesh->ncy < 1 || mesh->ncz < 1) { why = "cell counts must be >= 1"; return false; }
  if (!mesh->xb_host || !mesh->yb_host || !mesh->zb_host) { why = "cell boundaries are required"; return false; }
  const double* b[3] = {mesh->xb_host, mesh->yb_host, mesh->zb_host};
  const int n[3] = {mesh->ncx, mesh->ncy, mesh->ncz};
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < n[a]; ++k)
      if (!(b[a][k + 1] > b[a][k])) { why = "cell boundaries must increase strictly"; return false; }
  long long cells = (long long)mesh->ncx * mesh->ncy * mesh->ncz;
  if (cells > (1LL << 30)) { why = "too many cells"; return false; }
  if (n_atoms < 0 || (n_atoms > 0 && !atoms)) { why = "bad atom array"; return false; }
  if (enr && enr->n_fn > 0) {
    if (!enr->fns_host) { why = "enrichment functions missing"; return false; }
    if (!(enr->r0 > 0.0) || !(enr->s > 0.0) || enr->s > enr->r0) { why = "need 0 < s <= r0"; return false; }
    for (int i = 0; i < enr->n_fn; ++i) {
      const efe_enrich_fn& f = enr->fns_host[i];
      if (f.atom < 0 || f.atom >= n_atoms) { why = "enrichment atom index out of range"; return false; }
      if (f.l < 0 || f.l > 2 || f.m < -f.l || f.m > f.l) { why = "unsupported (l, m)"; return false; }
      if (f.radial == EFE_RADIAL_SLATER && f.n - 1 < f.l) { why = "Slater function needs n - 1 >= l"; return false; }
      if (f.radial == EFE_RADIAL_HYDROGENIC && f.n <= f.l) { why = "hydrogen-like function needs n > l"; return false; }
      if (f.radial < 0 || f.radial > 2) { why = "unknown radial kind"; return false; }
    }
  }
  if (o->n_orb < 1 || o->batch < 1 || !o->occ_host) { why = "n_orb, batch >= 1 and occupations required"; return false; }
  if (o->k_max < 1 || o->k_max > kMaxK) { why = "k_max must be in [1, 64]"; return false; }
  if (o->fixed_k < 0 || o->fixed_k > o->k_max) { why = "fixed_k must be in [0, k_max]"; return false; }
  if (o->precision != EFE_FP64 && o->precision != EFE_MIXED && o->precision != EFE_PAIR && o->precision != EFE_TC) {
    why = "unknown precision";
    return false;
  }
  if (o->xc != EFE_XC_PW92 && o->xc != EFE_XC_PZ81) { why = "unknown xc"; return false; }
  if (o->scheme != EFE_STEP_PC && o->scheme != EFE_STEP_EXTRAPOLATED) { why = "unknown step scheme"; return false; }
  if (o->krylov_block < 0) { why = "krylov_block must be >= 0"; return false; }
  if (o->krylov_substeps < 0 || o->krylov_substeps > 64) { why = "krylov_substeps must be in [0, 64]"; return false; }
  if (o->krylov_reorth != 0 && o->krylov_reorth != 1) { why = "krylov_reorth must be 0 or 1"; return false; }
  if (o->hartree_method != EFE_HARTREE_FDM && o->hartree_method != EFE_HARTREE_PCG) {
    why = "unknown Hartree method";
    return false;
  }
  return true;
}

static efe_status setup_impl(Ctx& c, const efe_mesh_desc* mesh, const efe_atom* atoms, int n_atoms,
                             const efe_enrich_desc* enr, const efe_options* o) {
  cudaGetDevice(&c.device);
  cudaStream_t s = 0;
  c.p = mesh->degree;
  c.P1 = c.p + 1;
  c.NQ1 = mesh->n_quad;
  c.nn = c.P1 * c.P1 * c.P1;
  c.nq = c.NQ1 * c.NQ1 * c.NQ1;
  c.ncx = mesh->ncx; c.ncy = mesh->ncy; c.ncz = mesh->ncz;
  c.nc = c.ncx * c.ncy * c.ncz;
  c.Nx = c.ncx * c.p + 1; c.Ny = c.ncy * c.p + 1; c.Nz = c.ncz * c.p + 1;
  c.n_h = (long long)c.Nx * c.Ny * c.Nz;
  c.xb.assign(mesh->xb_host, mesh->xb_host + c.ncx + 1);
  c.yb.assign(mesh->yb_host, mesh->yb_host + c.ncy + 1);
  c.zb.assign(mesh->zb_host, mesh->zb_host + c.ncz + 1);
  c.n_atoms = n_atoms;
  for (int a = 0; a < n_atoms; ++a) {
    c.Z.push_back(atoms[a].Z);
    for (int k = 0; k < 3; ++k) c.R.push_back(atoms[a].R[k]);
  }
  if (enr && enr->n_fn > 0) {
    c.fns.assign(enr->fns_host, enr->fns_host + enr->n_fn);
    c.r0 = enr->r0;
    c.s = enr->s;
  }
  c.nE = (int)c.fns.size();
  c.n_dof = c.n_h + c.nE;
  c.n_orb = o->n_orb;
  c.batch = o->batch;
  c.occ.assign(o->occ_host, o->occ_host + o->n_orb);
  c.krylov_tol = o->krylov_tol;
  c.k_max = o->k_max;
  c.fixed_k = o->fixed_k;
  c.cg_tol = o->cg_tol > 0 ? o->cg_tol : 1e-12;
  c.cg_max_it = o->cg_max_it > 0 ? o->cg_max_it : 2000;
  c.precision = o->precision;
  c.hartree_method = o->hartree_method;
  c.xc = o->xc;
  c.scheme = o->scheme;
  c.use_graphs = o->use_graphs != 0;
  c.kblock_opt = o->krylov_block;
  c.substeps_opt = o->krylov_substeps;
  c.reorth = o->krylov_reorth != 0;
  c.substeps_cur = 1;

  // reference tables
  double xi[kMaxP1], wl[kMaxP1], xg[kMaxNQ1], wg[kMaxNQ1];
  gauss_lobatto(c.p, xi, wl);
  gauss_legendre(c.NQ1, xg, wg);
  double L[kMaxNQ1 * kMaxP1], dL[kMaxNQ1 * kMaxP1];
  lagrange_tables(c.P1, xi, c.NQ1, xg, L, dL);
  RefTables& t = c.tab;
  for (int q = 0; q < c.NQ1; ++q) {
    t.wg[q] = wg[q];
    t.xg[q] = xg[q];
    for (int i = 0; i < c.P1; ++i) {
      t.B1[q * c.P1 + i] = L[q * c.P1 + i];
      t.D1[q * c.P1 + i] = dL[q * c.P1 + i];
    }
  }
  for (int i = 0; i < c.P1; ++i)
    for (int j = 0; j < c.P1; ++j) {
      double k = 0.0, m = 0.0;
      for (int q = 0; q < c.NQ1; ++q) {
        k += wg[q] * dL[q * c.P1 + i] * dL[q * c.P1 + j];
        m += wg[q] * L[q * c.P1 + i] * L[q * c.P1 + j];
      }
      t.K1[i * c.P1 + j] = k;
      t.M1[i * c.P1 + j] = m;
    }
  for (int i = 0; i < kMaxNQ1 * kMaxP1; ++i) {
    t.B1f[i] = (float)t.B1[i];
    t.D1f[i] = (float)t.D1[i];
    t.B1p[i] = df32::split(t.B1[i]);
    t.D1p[i] = df32::split(t.D1[i]);
  }
  for (int i = 0; i < kMaxP1 * kMaxP1; ++i) {
    t.K1f[i] = (float)t.K1[i];
    t.M1f[i] = (float)t.M1[i];
    t.K1p[i] = df32::split(t.K1[i]);
    t.M1p[i] = df32::split(t.M1[i]);
  }

  // mesh geometry and the lumped GLL mass (a tensor product of 1D lumped masses)
  std::vector<double> geo;
  const std::vector<double>* bb[3] = {&c.xb, &c.yb, &c.zb};
  const int nca[3] = {c.ncx, c.ncy, c.ncz};
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < nca[a]; ++k) geo.push_back((*bb[a])[k]);
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < nca[a]; ++k) geo.push_back((*bb[a])[k + 1] - (*bb[a])[k]);
  TRY_CUDA(c, dalloc(c.d_geo, geo.size()), "allocating geometry");
  TRY_CUDA(c, cudaMemcpy(c.d_geo, geo.data(), sizeof(double) * geo.size(), cudaMemcpyHostToDevice), "copy");
  const int ntot = c.ncx + c.ncy + c.ncz;
  c.mesh = MeshView{c.ncx, c.ncy, c.ncz, c.Nx, c.Ny, c.Nz, c.p, c.nc, c.n_h, c.d_geo, c.d_geo + ntot};
  std::vector<double> m1[3];
  const int Na[3] = {c.Nx, c.Ny, c.Nz};
  for (int a = 0; a < 3; ++a) {
    m1[a].assign(Na[a], 0.0);
    for (int k = 0; k < nca[a]; ++k) {
      const double h = (*bb[a])[k + 1] - (*bb[a])[k];
      for (int i = 0; i < c.P1; ++i) m1[a][k * c.p + i] += wl[i] * 0.5 * h;
    }
  }
  {
    std::vector<double> Dsc((size_t)c.n_h);
    for (int iz = 0; iz < c.Nz; ++iz)
      for (int iy = 0; iy < c.Ny; ++iy)
        for (int ix = 0; ix < c.Nx; ++ix) {
          const bool bnd = ix == 0 || iy == 0 || iz == 0 || ix == c.Nx - 1 || iy == c.Ny - 1 || iz == c.Nz - 1;
          const double M = m1[0][ix] * m1[1][iy] * m1[2][iz];
          Dsc[(size_t)ix + (size_t)c.Nx * ((size_t)iy + (size_t)c.Ny * iz)] = bnd ? 0.0 : 1.0 / std::sqrt(M);
        }
    TRY_CUDA(c, dalloc(c.d_Dsc, Dsc.size()), "allocating D");
    TRY_CUDA(c, cudaMemcpy(c.d_Dsc, Dsc.data(), sizeof(double) * Dsc.size(), cudaMemcpyHostToDevice), "copy");
  }
  TRY_CUDA(c, dalloc(c.d_occ, c.occ.size()), "allocating occupations");
  TRY_CUDA(c, cudaMemcpy(c.d_occ, c.occ.data(), sizeof(double) * c.occ.size(), cudaMemcpyHostToDevice), "copy");
  TRY_CUDA(c, dalloc(c.d_wJ, (size_t)c.nc * c.nq), "allocating quadrature");
  TRY_CUDA(c, dalloc(c.d_xq, (size_t)c.nc * c.nq * 3), "allocating quadrature");
  TRY_CUDA(c, dalloc(c.d_vN, (size_t)c.nc * c.nq), "allocating v_N");
  TRY_CUDA(c, launch_geometry(c, s), "geometry");

  // enrichment support: a cell pairs with function nu when it shares a node with
  // a cell that meets the ball |x - R_I| < r0 (the support of N^E_nu = N^A_nu - sum c N^C).
  std::vector<std::vector<int>> cell_fns(c.nc);
  for (int nu = 0; nu < c.nE; ++nu) {
    const double* R = &c.R[3 * c.fns[nu].atom];
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = nca[a];
      hi[a] = -1;
      for (int k = 0; k < nca[a]; ++k) {
        const double x0 = (*bb[a])[k], x1 = (*bb[a])[k + 1];
        const double d = R[a] < x0 ? x0 - R[a] : (R[a] > x1 ? R[a] - x1 : 0.0);
        if (d < c.r0) { lo[a] = std::min(lo[a], k); hi[a] = std::max(hi[a], k); }
      }
    }
    if (hi[0] < 0 || hi[1] < 0 || hi[2] < 0) continue;
    const int ex = hi[0] - lo[0] + 1, ey = hi[1] - lo[1] + 1, ez = hi[2] - lo[2] + 1;
    std::vector<char> core((size_t)ex * ey * ez, 0);
    for (int kz = lo[2]; kz <= hi[2]; ++kz)
      for (int ky = lo[1]; ky <= hi[1]; ++ky)
        for (int kx = lo[0]; kx <= hi[0]; ++kx) {
          const int kk[3] = {kx, ky, kz};
          double d2 = 0.0;
          for (int a = 0; a < 3; ++a) {
            const double x0 = (*bb[a])[kk[a]], x1 = (*bb[a])[kk[a] + 1];
            const double d = R[a] < x0 ? x0 - R[a] : (R[a] > x1 ? R[a] - x1 : 0.0);
            d2 += d * d;
          }
          if (d2 < c.r0 * c.r0) core[(size_t)(kx - lo[0]) + (size_t)ex * ((ky - lo[1]) + (size_t)ey * (kz - lo[2]))] = 1;
        }
    for (int kz = std::max(lo[2] - 1, 0); kz <= std::min(hi[2] + 1, c.ncz - 1); ++kz)
      for (int ky = std::max(lo[1] - 1, 0); ky <= std::min(hi[1] + 1, c.ncy - 1); ++ky)
        for (int kx = std::max(lo[0] - 1, 0); kx <= std::min(hi[0] + 1, c.ncx - 1); ++kx) {
          bool hit = false;
          for (int dz = -1; dz <= 1 && !hit; ++dz)
            for (int dy = -1; dy <= 1 && !hit; ++dy)
              for (int dx = -1; dx <= 1 && !hit; ++dx) {
                const int X = kx + dx - lo[0], Y = ky + dy - lo[1], Z = kz + dz - lo[2];
                if (X < 0 || Y < 0 || Z < 0 || X >= ex || Y >= ey || Z >= ez) continue;
                if (core[(size_t)X + (size_t)ex * (Y + (size_t)ey * Z)]) hit = true;
              }
          if (hit) cell_fns[(size_t)kx + (size_t)c.ncx * (ky + (size_t)c.ncy * kz)].push_back(nu);
        }
  }
  std::vector<int> pstart(c.nc + 1, 0), pfn, pcell;
  for (int cc = 0; cc < c.nc; ++cc) {
    pstart[cc + 1] = pstart[cc] + (int)cell_fns[cc].size();
    c.max_pairs_per_cell = std::max(c.max_pairs_per_cell, (int)cell_fns[cc].size());
    for (int nu : cell_fns[cc]) {
      pfn.push_back(nu);
      pcell.push_back(cc);
    }
  }
  c.n_pairs = (long long)pfn.size();
  TRY_CUDA(c, dalloc(c.d_pair_start, pstart.size()), "allocating pairs");
  TRY_CUDA(c, dalloc(c.d_pair_fn, pfn.size()), "allocating pairs");
  TRY_CUDA(c, dalloc(c.d_pair_cell, pcell.size()), "allocating pairs");
  TRY_CUDA(c, cudaMemcpy(c.d_pair_start, pstart.data(), sizeof(int) * pstart.size(), cudaMemcpyHostToDevice), "copy");
  if (c.n_pairs) {
    TRY_CUDA(c, cudaMemcpy(c.d_pair_fn, pfn.data(), sizeof(int) * pfn.size(), cudaMemcpyHostToDevice), "copy");
    TRY_CUDA(c, cudaMemcpy(c.d_pair_cell, pcell.data(), sizeof(int) * pcell.size(), cudaMemcpyHostToDevice), "copy");
  }
  TRY_CUDA(c, dalloc(c.d_Atil, (size_t)c.n_pairs * c.nq), "allocating enrichment tables");
  TRY_CUDA(c, dalloc(c.d_KE, (size_t)c.n_pairs * c.nn), "allocating enrichment tables");
  TRY_CUDA(c, dalloc(c.d_KEE, (size_t)std::max(c.nE, 1) * std::max(c.nE, 1)), "allocating K_EE");
  if (c.nE > 0) {
    TRY_CUDA(c, launch_enrich_setup(c, s), "enrichment set-up");
    // (M^ee)^(+-1/2) by symmetric eigendecomposition (Eq. MSquareRoot)
    std::vector<double> A = c.Mee, V, lam;
    const int nE = c.nE;
    jacobi_eigen(nE, A, V, lam);
    double lmax = 0.0, lmin = 1e300;
    for (double l : lam) { lmax = std::max(lmax, l); lmin = std::min(lmin, l); }
    if (!(lmin > 0.0) || lmin < 1e-14 * lmax) {
      char buf[160];
      snprintf(buf, sizeof buf, "M^ee is not positive definite (eigenvalues %.3e .. %.3e)", lmin, lmax);
      c.err = buf;
      return EFE_ERR_NOT_SPD;
    }
    c.S.assign((size_t)nE * nE, 0.0);
    c.Shalf.assign((size_t)nE * nE, 0.0);
    for (int i = 0; i < nE; ++i)
      for (int j = 0; j < nE; ++j) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < nE; ++k) {
          a += V[(size_t)i * nE + k] * V[(size_t)j * nE + k] / std::sqrt(lam[k]);
          b += V[(size_t)i * nE + k] * V[(size_t)j * nE + k] * std::sqrt(lam[k]);
        }
        c.S[(size_t)i * nE + j] = a;
        c.Shalf[(size_t)i * nE + j] = b;
      }
    TRY_CUDA(c, dalloc(c.d_S, c.S.size()), "allocating S");
    TRY_CUDA(c, dalloc(c.d_Shalf, c.Shalf.size()), "allocating S");
    TRY_CUDA(c, cudaMemcpy(c.d_S, c.S.data(), sizeof(double) * c.S.size(), cudaMemcpyHostToDevice), "copy");
    TRY_CUDA(c, cudaMemcpy(c.d_Shalf, c.Shalf.data(), sizeof(double) * c.Shalf.size(), cudaMemcpyHostToDevice), "copy");
  }
  TRY_CUDA(c, dalloc(c.d_diagA, (size_t)c.n_h), "allocating Poisson data");
  TRY_CUDA(c, dalloc(c.d_phiB, (size_t)c.n_h), "allocating Poisson data");
  TRY_CUDA(c, launch_poisson_setup(c, s), "Poisson set-up");
  if (c.batch == 1) {
    c.d_phiB_nb = c.d_phiB;
  } else {
    TRY_CUDA(c, dalloc(c.d_phiB_nb, (size_t)c.n_h * c.batch), "allocating Dirichlet data");
    std::vector<double> hb((size_t)c.n_h), hbn((size_t)c.n_h * c.batch);
    TRY_CUDA(c, cudaMemcpy(hb.data(), c.d_phiB, sizeof(double) * c.n_h, cudaMemcpyDeviceToHost), "copy");
    for (long long g = 0; g < c.n_h; ++g)
      for (int m = 0; m < c.batch; ++m) hbn[(size_t)g * c.batch + m] = hb[(size_t)g];
    TRY_CUDA(c, cudaMemcpy(c.d_phiB_nb, hbn.data(), sizeof(double) * hbn.size(), cudaMemcpyHostToDevice), "copy");
  }
  {
    cudaError_t e = setup_fdm(c);
    if (e == cudaErrorInvalidValue) {
      c.err = "fast-diagonalisation set-up failed (1D mass matrix not positive definite)";
      return EFE_ERR_NOT_SPD;
    }
    TRY_CUDA(c, e, "fast-diagonalisation set-up");
  }
  TRY_CUDA(c, dalloc(c.d_red, (size_t)std::max(64, 3 * c.batch + 64)), "allocating scratch");
  TRY_CUDA(c, cudaMallocHost((void**)&c.h_flag, sizeof(int) * 4), "allocating pinned flag");
  TRY_CUDA(c, cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking), "creating the capture stream");
  efe_status st = ensure_batch_buffers(c);
  if (st != EFE_OK) return st;
  if (c.precision == EFE_TC) {
    const char* why = tc_unsupported(c, 2 * c.n_orb);
    if (why) {
      c.err = why;
      return EFE_ERR_ARG;
    }
    c.tc_on = true;
  }
  TRY_CUDA(c, cudaDeviceSynchronize(), "set-up");
  return EFE_OK;
}

// ------------------------------------------------------------------ drivers
static void field_vectors(const Ctx& c, const efe_field* fields, double t, std::vector<double>& E) {
  E.assign(3 * (size_t)c.batch, 0.0);
  if (!fields) return;
  for (int m = 0; m < c.batch; ++m) {
    const double a = field_amp(fields[m], t);
    for (int k = 0; k < 3; ++k) E[3 * m + k] = a * fields[m].dir[k];
  }
}

// the partial density of this process's orbitals -> the sum over all processes (orbital partition)
static efe_status reduce_rho(Ctx& c, double* rho, cudaStream_t s) {
  if (!c.rho_reduce) return EFE_OK;
  const long long n = (long long)c.batch * c.nc * c.nq;
  const int rc = c.rho_reduce(rho, (int64_t)n, (void*)s, c.rho_reduce_user);
  if (rc != 0) {
    c.err = "the density reduction across processes failed (code " + std::to_string(rc) + ")";
    return EFE_ERR_CUDA;
  }
  return EFE_OK;
}

// rho, v_xc, v_H of psi into the context state
static efe_status compute_state(Ctx& c, const double* psi, int* cg_its, cudaStream_t s) {
  TRY_CUDA(c, launch_density(c, psi, c.d_rho, s), "density");
  {
    const efe_status r = reduce_rho(c, c.d_rho, s);
    if (r != EFE_OK) return r;
  }
  TRY_CUDA(c, launch_lda(c, c.d_rho, c.d_vxc, nullptr, (long long)c.batch * c.nc * c.nq, s), "LDA");
  int its = 0;
  efe_status st = run_hartree(c, c.d_rho, c.d_vH, c.cg_tol, c.cg_max_it, &its, s);
  if (cg_its) *cg_its += its;
  if (st == EFE_OK) c.state_valid = true;
  return st;
}

// out = exp(-i dt Hbar) in as m sub-steps exp(-i (dt/m) Hbar), each a Lanczos run capped at
// k_max (the operator is the same for all of them, so they compose exactly).  Adaptive
// (krylov_substeps = 0, no fixed k): a pass in which a column reached k_max with its estimate
// above the tolerance is repeated from `in` with twice the sub-steps (in and out must differ),
// up to 64; the count is kept for the next exponential, halved after one whose largest k
// stayed at or below 2 k_max / 5.  Statistics: the largest k, the cap hits and the largest
// estimate of the pass that was kept.
static efe_status kexp_substeps(Ctx& c, const double* in, double* out, double dt, int* kmax, int* caps, double* eps,
                                int* m_used, cudaStream_t s, bool stats) {
  constexpr int kMaxSub = 64;
  const long long C = (long long)c.n_orb * c.batch;
  const bool adaptive = c.substeps_opt == 0 && c.fixed_k <= 0 && in != out;
  int m = adaptive ? c.substeps_cur : (c.substeps_opt > 0 ? c.substeps_opt : 1);
  for (;;) {
    std::vector<double> dts((size_t)C, dt / m);
    int km = 0, cp = 0;
    double em = 0.0;
    for (int q = 0; q < m; ++q) {
      int k = 0, p = 0;
      double e = 0.0;
      TRY_CUDA(c, run_kexp_cols(c, q == 0 ? in : out, out, dts.data(), c.precision, &k, &p, &e, s, stats || adaptive),
               "Krylov exponential");
      km = std::max(km, k);
      cp += p;
      em = std::max(em, e);
    }
    if (!adaptive || cp == 0 || m >= kMaxSub) {
      if (adaptive) c.substeps_cur = (m > 1 && 5 * km <= 2 * c.k_max) ? m / 2 : m;
      *kmax = km;
      *caps = cp;
      *eps = em;
      *m_used = m;
      return EFE_OK;
    }
    m *= 2;
  }
}

static efe_status magnus_impl(Ctx& c, double* psi, double t, double dt, const efe_field* fields, double* mu,
                              efe_step_info* info, cudaStream_t s) {
  const long long C = (long long)c.n_orb * c.batch;
  efe_status st = ensure_ws(c, C, C);
  if (st != EFE_OK) return st;
  efe_status warn = EFE_OK;
  int cg_its = 0;
  if (!c.state_valid) {
    st = compute_state(c, psi, &cg_its, s);
    if (st == EFE_ERR_CG_NOCONV) warn = st; else if (st != EFE_OK) return st;
  }
  std::vector<double> E;
  field_vectors(c, fields, t + 0.5 * dt, E);
  int k1 = 0, cap1 = 0, k2 = 0, cap2 = 0, m1 = 1, m2 = 1;
  double e1 = 0.0, e2 = 0.0;
  const bool stats = info != nullptr;
  const long long nqb = (long long)c.batch * c.nc * c.nq;
  if (c.scheme == EFE_STEP_EXTRAPOLATED && c.has_prev) {
    // v_mid = v_N + (3 v_Hxc(t_n) - v_Hxc(t_n-1)) / 2 - E(t_n + dt/2) . x, then keep v_Hxc(t_n)
    TRY_CUDA(c, launch_axpby(c.d_rho2, c.d_vH, c.d_vxc, 1.5, 1.5, nqb, s), "extrapolation");
    TRY_CUDA(c, launch_axpby(c.d_rho2, c.d_rho2, c.d_vprev, 1.0, -0.5, nqb, s), "extrapolation");
    TRY_CUDA(c, launch_potential_sum(c, c.d_rho2, nullptr, E.data(), true, c.d_v, s), "potential");
    TRY_CUDA(c, launch_axpby(c.d_vprev, c.d_vH, c.d_vxc, 1.0, 1.0, nqb, s), "potential history");
  } else {
    TRY_CUDA(c, launch_axpby(c.d_vprev, c.d_vH, c.d_vxc, 1.0, 1.0, nqb, s), "potential history");
    // S1: predictor with v(rho_n) and the mid-point field
    TRY_CUDA(c, launch_potential_sum(c, c.d_vH, c.d_vxc, E.data(), true, c.d_v, s), "potential");
    st = build_op(c, c.d_v, c.batch, 1.0, s);
    if (st != EFE_OK) return st;
    st = kexp_substeps(c, psi, c.d_psi_p, dt, &k1, &cap1, &e1, &m1, s, stats);
    if (st != EFE_OK) return st;
    // S2, S3: rho_mid = (rho_n + rho^p) / 2
    TRY_CUDA(c, launch_density(c, c.d_psi_p, c.d_rho2, s), "density");
    st = reduce_rho(c, c.d_rho2, s);
    if (st != EFE_OK) return st;
    TRY_CUDA(c, launch_axpby(c.d_rho2, c.d_rho, c.d_rho2, 0.5, 0.5, nqb, s), "mid-point density");
    // S4: v_mid
    TRY_CUDA(c, launch_lda(c, c.d_rho2, c.d_vxc, nullptr, nqb, s), "LDA");
    int its = 0;
    st = run_hartree(c, c.d_rho2, c.d_vH, c.cg_tol, c.cg_max_it, &its, s);
    cg_its += its;
    if (st == EFE_ERR_CG_NOCONV) warn = st; else if (st != EFE_OK) return st;
    TRY_CUDA(c, launch_potential_sum(c, c.d_vH, c.d_vxc, E.data(), true, c.d_v, s), "potential");
  }
  st = build_op(c, c.d_v, c.batch, 1.0, s);
  if (st != EFE_OK) return st;
  // S5: corrector from psi_n, written in place (adaptive sub-steps: into the predictor's buffer,
  // free by now, so that a pass can be repeated from psi_n, then copied back)
  if (c.substeps_opt == 0 && c.fixed_k <= 0) {
    st = kexp_substeps(c, psi, c.d_psi_p, dt, &k2, &cap2, &e2, &m2, s, stats);
    if (st != EFE_OK) return st;
    TRY_CUDA(c, cudaMemcpyAsync(psi, c.d_psi_p, sizeof(double) * 2 * (size_t)c.n_dof * C, cudaMemcpyDeviceToDevice, s),
             "corrector");
  } else {
    st = kexp_substeps(c, psi, psi, dt, &k2, &cap2, &e2, &m2, s, stats);
    if (st != EFE_OK) return st;
  }
  // S6: state of step n+1 and the dipole
  c.state_valid = false;
  st = compute_state(c, psi, &cg_its, s);
  if (st == EFE_ERR_CG_NOCONV) warn = st; else if (st != EFE_OK) return st;
  c.has_prev = true;
  if (mu) TRY_CUDA(c, launch_dipole(c, c.d_rho, mu, s), "dipole");
  if (info) {
    TRY_CUDA(c, cudaStreamSynchronize(s), "step");
    if (c.tc.err) {
      int h = 0;
      TRY_CUDA(c, cudaMemcpy(&h, c.tc.err, sizeof(int), cudaMemcpyDeviceToHost), "tensor-core status");
      if (h) {   // reported once; the context stays usable for the next step
        TRY_CUDA(c, cudaMemset(c.tc.err, 0, sizeof(int)), "tensor-core status");
        c.err = "a tensor-core completion wait gave up";
        return EFE_ERR_TIMEOUT;
      }
    }
    info->k_pred_max = k1;
    info->k_corr_max = k2;
    info->krylov_cap_hit = cap1 + cap2;
    info->cg_iters = cg_its;
    info->eps_max = std::max(e1, e2);
    info->substeps = m2;
  }
  if (warn == EFE_OK && cap1 + cap2 > 0) warn = EFE_WARN_KRYLOV_CAP;
  return warn;
}

}  // namespace efe

using namespace efe;

static cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

#define CHECK_CTX(ctx)                       \
  do {                                       \
    if (!(ctx)) return EFE_ERR_ARG;          \
    (ctx)->c.err.clear();                    \
  } while (0)

extern "C" {

efe_status efe_setup(const efe_mesh_desc* mesh, const efe_atom* atoms_host, int32_t n_atoms,
                     const efe_enrich_desc* enrich, const efe_options* opts, efe_ctx** out) {
  if (!out) return EFE_ERR_ARG;
  *out = nullptr;
  std::string why;
  if (!validate(mesh, atoms_host, n_atoms, enrich, opts, why)) {
    g_setup_err = why;
    return EFE_ERR_ARG;
  }
  efe_ctx* ctx = new efe_ctx();
  efe_status st = setup_impl(ctx->c, mesh, atoms_host, n_atoms, enrich, opts);
  if (st != EFE_OK) {
    g_setup_err = ctx->c.err;
    delete ctx;
    return st;
  }
  g_setup_err.clear();
  *out = ctx;
  return EFE_OK;
}

efe_status efe_destroy(efe_ctx* ctx) {
  if (!ctx) return EFE_ERR_ARG;
  cudaSetDevice(ctx->c.device);
  cudaDeviceSynchronize();
  delete ctx;
  return EFE_OK;
}

const char* efe_last_error(const efe_ctx* ctx) { return ctx ? ctx->c.err.c_str() : g_setup_err.c_str(); }

efe_status efe_sizes(const efe_ctx* ctx, int64_t* n_nodes, int64_t* n_enrich, int64_t* n_cells, int64_t* n_q,
                     int64_t* n_pairs) {
  if (!ctx) return EFE_ERR_ARG;
  if (n_nodes) *n_nodes = ctx->c.n_h;
  if (n_enrich) *n_enrich = ctx->c.nE;
  if (n_cells) *n_cells = ctx->c.nc;
  if (n_q) *n_q = ctx->c.nq;
  if (n_pairs) *n_pairs = ctx->c.n_pairs;
  return EFE_OK;
}

efe_status efe_coords(efe_ctx* ctx, double* node_xyz_dev, double* quad_xyz_dev, void* stream) {
  CHECK_CTX(ctx);
  TRY_CUDA(ctx->c, launch_coords(ctx->c, node_xyz_dev, quad_xyz_dev, as_stream(stream)), "coordinates");
  return EFE_OK;
}

efe_status efe_set_potential(efe_ctx* ctx, const double* v_dev, int32_t batch, double kin_scale, void* stream) {
  CHECK_CTX(ctx);
  if (!v_dev || batch < 1) {
    ctx->c.err = "efe_set_potential: v_dev is NULL or batch < 1";
    return EFE_ERR_ARG;
  }
  return build_op(ctx->c, v_dev, batch, kin_scale, as_stream(stream));
}

efe_status efe_apply_H(efe_ctx* ctx, const double* X_dev, double* Y_dev, int64_t n_cols, int64_t ld, int32_t precision,
                       void* stream) {
  CHECK_CTX(ctx);
  Ctx& c = ctx->c;
  if (!c.op.valid) {
    c.err = "no operator: call efe_set_potential first";
    return EFE_ERR_STATE;
  }
  if (!X_dev || !Y_dev || X_dev == Y_dev || n_cols < 1 || ld < n_cols || n_cols % c.op.batch != 0 ||
      (precision != EFE_FP64 && precision != EFE_MIXED && precision != EFE_PAIR && precision != EFE_TC)) {
    c.err = "bad arguments to efe_apply_H (n_cols must be a multiple of the operator's batch, ld >= n_cols)";
    return EFE_ERR_ARG;
  }
  efe_status st = ensure_ws(c, n_cols, ld);
  if (st != EFE_OK) return st;
  if (precision == EFE_TC) {
    const char* why = tc_unsupported(c, (int)(2 * n_cols / c.op.batch));
    if (why) {
      c.err = why;
      return EFE_ERR_ARG;
    }
    if (!c.tc_on) {   // first tensor-core apply of this context: slices of the current operator
      c.tc_on = true;
      TRY_CUDA(c, launch_tc_build(c, c.op.batch, as_stream(stream)), "building the tensor-core operator");
    }
  }
  TRY_CUDA(c, launch_apply(c, X_dev, Y_dev, n_cols, ld, precision, as_stream(stream)), "apply");
  return EFE_OK;
}

efe_status efe_magnus_step(efe_ctx* ctx, double* psi_bar_dev, double t, double dt, const efe_field* fields_host,
                           double* mu_dev, efe_step_info* info_host, void* stream) {
  CHECK_CTX(ctx);
  if (!psi_bar_dev || !std::isfinite(t) || !std::isfinite(dt)) {
    ctx->c.err = "efe_magnus_step: psi_bar_dev is NULL or t, dt not finite";
    return EFE_ERR_ARG;
  }
  return magnus_impl(ctx->c, psi_bar_dev, t, dt, fields_host, mu_dev, info_host, as_stream(stream));
}

efe_status efe_reset_state(efe_ctx* ctx) {
  CHECK_CTX(ctx);
  ctx->c.state_valid = false;
  ctx->c.has_prev = false;
  ctx->c.substeps_cur = 1;
  return EFE_OK;
}

efe_status efe_density_vxc(efe_ctx* ctx, const double* psi_bar_dev, double* rho_dev, double* vxc_dev, double* exc_dev,
                           void* stream) {
  CHECK_CTX(ctx);
  Ctx& c = ctx->c;
  if (!psi_bar_dev || !rho_dev) {
    c.err = "efe_density_vxc: psi_bar_dev and rho_dev are required";
    return EFE_ERR_ARG;
  }
  efe_status st = ensure_ws(c, (long long)c.n_orb * c.batch, (long long)c.n_orb * c.batch);
  if (st != EFE_OK) return st;
  cudaStream_t s = as_stream(stream);
  TRY_CUDA(c, launch_density(c, psi_bar_dev, rho_dev, s), "density");
  st = reduce_rho(c, rho_dev, s);
  if (st != EFE_OK) return st;
  if (vxc_dev || exc_dev)
    TRY_CUDA(c, launch_lda(c, rho_dev, vxc_dev, exc_dev, (long long)c.batch * c.nc * c.nq, s), "LDA");
  return EFE_OK;
}

efe_status efe_hartree(efe_ctx* ctx, const double* rho_dev, double* vH_dev, double tol, int32_t max_it,
                       int32_t* iters_host, void* stream) {
  CHECK_CTX(ctx);
  if (!rho_dev || !vH_dev || !(tol > 0.0) || max_it < 1) {
    ctx->c.err = "efe_hartree: rho_dev and vH_dev are required, tol > 0, max_it >= 1";
    return EFE_ERR_ARG;
  }
  int its = 0;
  efe_status st = run_hartree(ctx->c, rho_dev, vH_dev, tol, max_it, &its, as_stream(stream));
  if (iters_host) *iters_host = its;
  if (st == EFE_ERR_CG_NOCONV) ctx->c.err = "Hartree CG did not reach the tolerance";
  return st;
}

efe_status efe_dipole(efe_ctx* ctx, const double* rho_dev, double* mu_dev, void* stream) {
  CHECK_CTX(ctx);
  if (!rho_dev || !mu_dev) {
    ctx->c.err = "efe_dipole: rho_dev and mu_dev are required";
    return EFE_ERR_ARG;
  }
  TRY_CUDA(ctx->c, launch_dipole(ctx->c, rho_dev, mu_dev, as_stream(stream)), "dipole");
  return EFE_OK;
}

efe_status efe_nuclear_enriched(efe_ctx* ctx, double sigma, double r0, double s, int32_t sub, int32_t n_quad,
                                double adapt_tol, int32_t adapt_depth, double* vN_dev, double* phiE_host,
                                void* stream) {
  CHECK_CTX(ctx);
  Ctx& c = ctx->c;
  cudaStream_t st = as_stream(stream);
  efe_status r = nuclear_enriched(c, sigma, r0, s, sub, n_quad, adapt_tol, adapt_depth, phiE_host, st);
  if (r != EFE_OK) return r;
  if (vN_dev)
    TRY_CUDA(c, cudaMemcpyAsync(vN_dev, c.d_vN, sizeof(double) * c.nc * c.nq, cudaMemcpyDeviceToDevice, st), "copy");
  return EFE_OK;
}

efe_status efe_hartree_enriched(efe_ctx* ctx, double r0, double s, int32_t sub, int32_t n_quad, void* stream) {
  CHECK_CTX(ctx);
  return hartree_enrich_install(ctx->c, r0, s, sub, n_quad, as_stream(stream));
}

efe_status efe_kick(efe_ctx* ctx, double* psi_bar_dev, const efe_field* fields_host, void* stream) {
  CHECK_CTX(ctx);
  Ctx& c = ctx->c;
  if (!psi_bar_dev || !fields_host) {
    c.err = "efe_kick: psi_bar_dev and fields_host are required";
    return EFE_ERR_ARG;
  }
  const long long C = (long long)c.n_orb * c.batch;
  efe_status st = ensure_ws(c, C, C);
  if (st != EFE_OK) return st;
  cudaStream_t s = as_stream(stream);
  std::vector<double> E(3 * (size_t)c.batch), dts((size_t)C);
  for (int m = 0; m < c.batch; ++m) {
    for (int k = 0; k < 3; ++k) E[3 * m + k] = fields_host[m].dir[k];
    for (int a = 0; a < c.n_orb; ++a) dts[(size_t)m * c.n_orb + a] = fields_host[m].kick;
  }
  // potential-only operator with v = -(d . x): exp(-i kick (-d.Xbar)) = exp(i kick d.Xbar)
  TRY_CUDA(c, launch_potential_sum(c, nullptr, nullptr, E.data(), false, c.d_v, s), "kick potential");
  st = build_op(c, c.d_v, c.batch, 0.0, s);
  if (st != EFE_OK) return st;
  int k = 0, cap = 0;
  double e = 0.0;
  TRY_CUDA(c, run_kexp_cols(c, psi_bar_dev, psi_bar_dev, dts.data(), EFE_FP64, &k, &cap, &e, s), "kick");
  c.state_valid = false;
  c.has_prev = false;
  c.op.valid = false;
  return cap > 0 ? EFE_WARN_KRYLOV_CAP : EFE_OK;
}

efe_status efe_init_orbitals(efe_ctx* ctx, double* psi_bar_dev, int32_t n_gauss, const double* centers_host,
                             const double* expo_host, const double* coef_host, const double* enr_host, void* stream) {
  CHECK_CTX(ctx);
  Ctx& c = ctx->c;
  if (!psi_bar_dev || n_gauss < 0 || (n_gauss > 0 && (!centers_host || !expo_host || !coef_host)) ||
      (c.nE > 0 && !enr_host))
    return EFE_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  const size_t G = (size_t)std::max(n_gauss, 1);
  double *dc = nullptr, *de = nullptr, *dk = nullptr, *dn = nullptr;
  TRY_CUDA(c, dalloc(dc, (size_t)c.n_orb * G * 3), "alloc");
  TRY_CUDA(c, dalloc(de, (size_t)c.n_orb * G), "alloc");
  TRY_CUDA(c, dalloc(dk, (size_t)c.n_orb * G * 2), "alloc");
  TRY_CUDA(c, dalloc(dn, (size_t)c.n_orb * std::max(c.nE, 1) * 2), "alloc");
  if (n_gauss > 0) {
    TRY_CUDA(c, cudaMemcpy(dc, centers_host, sizeof(double) * c.n_orb * n_gauss * 3, cudaMemcpyHostToDevice), "copy");
    TRY_CUDA(c, cudaMemcpy(de, expo_host, sizeof(double) * c.n_orb * n_gauss, cudaMemcpyHostToDevice), "copy");
    TRY_CUDA(c, cudaMemcpy(dk, coef_host, sizeof(double) * c.n_orb * n_gauss * 2, cudaMemcpyHostToDevice), "copy");
  }
  if (c.nE > 0)
    TRY_CUDA(c, cudaMemcpy(dn, enr_host, sizeof(double) * c.n_orb * c.nE * 2, cudaMemcpyHostToDevice), "copy");
  cudaError_t e = launch_init_orbitals(c, psi_bar_dev, n_gauss, dc, de, dk, dn, s);
  dfree(dc); dfree(de); dfree(dk); dfree(dn);
  if (e != cudaSuccess) return cuda_fail(c, e, "initial orbitals");
  c.state_valid = false;
  c.has_prev = false;
  return EFE_OK;
}

efe_status efe_adjoint_dipole(efe_ctx* ctx, const double* psi0_dev, int32_t n_steps, double dt,
                              const efe_field* field_host, const double* direction_host, int32_t window_first,
                              int32_t window_last, int32_t checkpoint_every, int32_t n_quad_s, double* J_host,
                              double* grad_host, void* stream) {
  CHECK_CTX(ctx);
  Ctx& c = ctx->c;
  if (!psi0_dev || !field_host || !direction_host || !J_host || !grad_host || n_steps < 1 || !(dt != 0.0) ||
      !std::isfinite(dt) || window_first < 1 || window_last < window_first || window_last > n_steps ||
      checkpoint_every < 1 || n_quad_s < 1 || n_quad_s > 64) {
    c.err = "efe_adjoint_dipole: invalid argument";
    return EFE_ERR_ARG;
  }
  if (c.batch != 1) {
    c.err = "efe_adjoint_dipole needs a context with batch = 1";
    return EFE_ERR_ARG;
  }
  if (c.rho_reduce) {
    c.err = "efe_adjoint_dipole needs all orbitals in one context (no density reduction installed)";
    return EFE_ERR_ARG;
  }
  if (c.xc != EFE_XC_PW92 || c.scheme != EFE_STEP_PC) {
    c.err = "efe_adjoint_dipole differentiates the predictor-corrector step with the PW92 functional";
    return EFE_ERR_ARG;
  }
  if ((field_host->kind != EFE_FIELD_GAUSS && field_host->kind != EFE_FIELD_SINE_GAUSS) || !(field_host->sigma > 0.0)) {
    c.err = "efe_adjoint_dipole: the field must be EFE_FIELD_GAUSS or EFE_FIELD_SINE_GAUSS with sigma > 0";
    return EFE_ERR_ARG;
  }
  return adjoint_dipole(c, psi0_dev, n_steps, dt, *field_host, direction_host, window_first, window_last,
                        checkpoint_every, n_quad_s, J_host, grad_host, as_stream(stream));
}

efe_status efe_absorption_spectrum(const double* mu_dev, int64_t n_t, int64_t stride_dir, int64_t stride_t, double dt,
                                   const double* field_dev, double kick, const double* omega_dev, int64_t n_omega,
                                   double tau, double* S_dev, void* stream) {
  g_setup_err.clear();
  if (!mu_dev || !omega_dev || !S_dev || n_t < 2 || n_omega < 1 || n_omega > 2147483647LL || !(dt > 0.0) ||
      !(tau > 0.0) || (!field_dev && kick == 0.0)) {
    g_setup_err = "efe_absorption_spectrum: invalid argument";
    return EFE_ERR_ARG;
  }
  const cudaError_t e = launch_absorption(mu_dev, n_t, stride_dir, stride_t, dt, field_dev, kick, omega_dev, n_omega,
                                          tau, S_dev, as_stream(stream));
  if (e != cudaSuccess) {
    g_setup_err = std::string("absorption spectrum: ") + cudaGetErrorString(e);
    return EFE_ERR_CUDA;
  }
  return EFE_OK;
}

efe_status efe_power_spectrum(const double* mu_dev, int64_t n_t, int64_t stride_t, double dt, const double* omega_dev,
                              int64_t n_omega, double tau, double* P_dev, void* stream) {
  g_setup_err.clear();
  if (!mu_dev || !omega_dev || !P_dev || n_t < 3 || n_omega < 1 || n_omega > 2147483647LL || !(dt > 0.0) ||
      !(tau > 0.0)) {
    g_setup_err = "efe_power_spectrum: invalid argument";
    return EFE_ERR_ARG;
  }
  const cudaError_t e = launch_power(mu_dev, n_t, stride_t, dt, omega_dev, n_omega, tau, P_dev, as_stream(stream));
  if (e != cudaSuccess) {
    g_setup_err = std::string("power spectrum: ") + cudaGetErrorString(e);
    return EFE_ERR_CUDA;
  }
  return EFE_OK;
}

efe_status efe_selftest(int64_t n, int64_t* mismatches_host) {
  if (n < 0 || !mismatches_host) return EFE_ERR_ARG;
  long long m = 0;
  cudaError_t e = run_selftest_cvt(n, &m);
  if (e != cudaSuccess) {
    g_setup_err = std::string("self-test: ") + cudaGetErrorString(e);
    return EFE_ERR_CUDA;
  }
  *mismatches_host = m;
  return EFE_OK;
}

efe_status efe_set_density_reduce(efe_ctx* ctx, efe_reduce_fn fn, void* user) {
  CHECK_CTX(ctx);
  ctx->c.rho_reduce = fn;
  ctx->c.rho_reduce_user = fn ? user : nullptr;
  return EFE_OK;
}

efe_status efe_set_wait_limit(efe_ctx* ctx, int64_t polls) {
  CHECK_CTX(ctx);
  if (polls < 0 || polls > 0xFFFFFFFFLL) {
    ctx->c.err = "efe_set_wait_limit: polls must be in [0, 2^32)";
    return EFE_ERR_ARG;
  }
  ctx->c.tc_wait_limit = (uint32_t)polls;
  return EFE_OK;
}

efe_status efe_tuning(efe_ctx* ctx, int32_t precision, int32_t force_variant, int32_t* variant, float* ms0,
                      float* ms1) {
  CHECK_CTX(ctx);
  Ctx& c = ctx->c;
  if (precision != EFE_FP64 && precision != EFE_MIXED && precision != EFE_PAIR) {
    c.err = "efe_tuning: precision must be EFE_FP64, EFE_MIXED or EFE_PAIR";
    return EFE_ERR_ARG;
  }
  const int p = precision;
  if (force_variant == 0 || force_variant == 1) {
    c.tile_choice[p] = force_variant;
    c.tile_cols[p] = (long long)c.n_orb * c.batch;
  } else if (force_variant != -1) {
    return EFE_ERR_ARG;
  }
  if (variant) *variant = c.tile_choice[p];
  if (ms0) *ms0 = c.tile_ms[p][0];
  if (ms1) *ms1 = c.tile_ms[p][1];
  return EFE_OK;
}

efe_status efe_profile(efe_ctx* ctx, int32_t enable) {
  CHECK_CTX(ctx);
  Ctx& c = ctx->c;
  TRY_CUDA(c, cudaDeviceSynchronize(), "profile");
  c.prof.on = enable != 0;
  c.prof.used = 0;
  c.prof.apply_launches = 0;
  reset_launch_count();
  return EFE_OK;
}

efe_status efe_krylov_basis(efe_ctx* ctx, const double** q_dev, const double** norms_dev, const int32_t** kused_dev,
                            int64_t* cols) {
  CHECK_CTX(ctx);
  Ctx& c = ctx->c;
  if (!q_dev || !norms_dev || !kused_dev || !cols) {
    c.err = "efe_krylov_basis: every output pointer is required";
    return EFE_ERR_ARG;
  }
  if (c.lz_last_C <= 0 || !c.d_Q) {
    c.err = "efe_krylov_basis: no Lanczos run yet";
    return EFE_ERR_ARG;
  }
  *q_dev = c.d_Q;
  lz_last_views(c, norms_dev, kused_dev);
  *cols = c.lz_last_C;
  return EFE_OK;
}

efe_status efe_profile_read(efe_ctx* ctx, int64_t* launches, int64_t* apply_launches, double* apply_ms) {
  CHECK_CTX(ctx);
  Ctx& c = ctx->c;
  TRY_CUDA(c, cudaDeviceSynchronize(), "profile");
  double total = 0.0;
  for (size_t i = 0; i + 1 < c.prof.used; i += 2) {
    float ms = 0.0f;
    TRY_CUDA(c, cudaEventElapsedTime(&ms, c.prof.pool[i], c.prof.pool[i + 1]), "profile events");
    total += ms;
  }
  if (launches) *launches = launch_count();
  if (apply_launches) *apply_launches = c.prof.apply_launches;
  if (apply_ms) *apply_ms = total;
  return EFE_OK;
}

}  // extern "C"
