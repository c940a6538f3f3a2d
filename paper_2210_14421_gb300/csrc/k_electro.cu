// Nuclear potential in the electrostatically enriched basis (Eqs. PhiEFE,
// DiscretePoisson): the potential of Gaussian-smeared nuclei, written as a
// classical part on the mesh plus one enrichment function per atom,
//   phi^h = sum_j N_j phi_j + sum_J Ntil_J phi^E_J,
//   Ntil_J = N^A_J - sum_i C_Ji N_i,   N^A_J = f_J(r) u(r),
//   f_J = -Z_J erf(r / (sqrt2 sigma)) / r,   C_Ji = int N^A_J N_i / M_i (interior i),
// with A = (1/4pi) int grad . grad over the classical and enriched functions,
// the load d = int b (.) of the smeared charge b = -sum Z_J g_sigma(|x - R_J|),
// and the smeared-nucleus potential as Dirichlet data on the boundary nodes.
//
// The Galerkin system is solved around the direct (fast-diagonalisation)
// Poisson solver by block elimination:
//   z = A_II^-1 (d_I - A_IB phi_B),  X_J = A_II^-1 A_IJ,
//   S = A_EE - A_EI X,  phi^E = S^-1 (d_E - A_EB phi_B - A_EI z),  phi_I = z - X phi^E.
// Only products of the atomic parts with the classical functions are
// integrated cell by cell (with a composite Gauss-Legendre rule of sub^3
// sub-cells, fine enough for the Gaussian cores); every term that involves
// the orthogonalising combination is assembled from those by linear algebra:
//   A_nJ  = k G_J[n] - k (K C_J)[n],                 G_J[n] = int grad N^A_J . grad N_n,
//   A_JK  = k (AA_JK - C_K . G_J - C_J . G_K) + C_J . (k K C_K),
//   d_J   = int b N^A_J - C_J . d,
// with k = 1/4pi and K the classical stiffness (applied by the existing
// Laplacian kernel, exact for the polynomial integrands).  The result at the
// quadrature points is interp(phi - sum_J phi^E_J C_J) + sum_J phi^E_J N^A_J.
//
// Set-up work, run once: plain loops, no tuning.
#include <algorithm>
#include <cmath>
#include <vector>

#include "efe_internal.h"
#include "radial.cuh"

namespace efe {

namespace {

constexpr int kNucThreads = 128;
constexpr double kPi = 3.14159265358979323846;

unsigned nblk(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// f(r) = -z erf(a r) / r and df/dr for one smeared nucleus, a = 1 / (sqrt2 sigma),
// with the limits f(0) = -2 z a / sqrt(pi) and df/dr -> 0 at the centre
__device__ __forceinline__ void nuc_radial(double z, double a, double r, double& f, double& df) {
  const double rsqpi = 0.56418958354775628695;   // 1 / sqrt(pi)
  f = r > 0.0 ? -z * erf(a * r) / r : -z * 2.0 * a * rsqpi;
  df = r > 1e-8 ? -z * (2.0 * a * exp(-(a * r) * (a * r)) * rsqpi / r - erf(a * r) / (r * r)) : 0.0;
}

// Atomic part N^A = f u of the atom at (ax, ay, az) with charge z, and its gradient.
__device__ __forceinline__ void nuc_atomic(double z, double ax, double ay, double az, double a, double r0, double s,
                                           double x, double y, double w, double& v, double g[3]) {
  const double dx = x - ax, dy = y - ay, dz = w - az;
  const double r = sqrt(dx * dx + dy * dy + dz * dz);
  double f, df, u, du;
  nuc_radial(z, a, r, f, df);
  cutoff(r, r0, s, u, du);
  v = f * u;
  const double rad = df * u + f * du;
  const double inv = r > 0.0 ? 1.0 / r : 0.0;
  g[0] = rad * dx * inv;
  g[1] = rad * dy * inv;
  g[2] = rad * dz * inv;
}

struct CellGeo {
  int cx, cy, cz;
  double ox, oy, oz, hx, hy, hz;
};

__device__ __forceinline__ CellGeo cell_geo(const MeshView& mesh, int c) {
  CellGeo g;
  cell_ijk(mesh, c, g.cx, g.cy, g.cz);
  g.hx = mesh.h[g.cx];
  g.hy = mesh.h[mesh.ncx + g.cy];
  g.hz = mesh.h[mesh.ncx + mesh.ncy + g.cz];
  g.ox = mesh.x0[g.cx];
  g.oy = mesh.x0[mesh.ncx + g.cy];
  g.oz = mesh.x0[mesh.ncx + mesh.ncy + g.cz];
  return g;
}

// Sum over the block (blockDim.x == kNucThreads); the result is valid in thread 0.
__device__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = kNucThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  return red[0];
}

// Cell integrals with the composite rule (m1 points per axis, tables `rule` =
// L [m1][P1], dL [m1][P1], xs [m1], ws [m1] on [-1, 1]).  One block per item:
// for fn[k] = J >= 0, over cell cells[k]
//   bA[J][g] += int N^A_J N_g,  G[J][g] += int grad N^A_J . grad N_g,  ba[J] += int b N^A_J;
// for fn[k] < 0 the charge load dC[g] += int b N_g.
__global__ void __launch_bounds__(kNucThreads)
k_nuc_cells(const MeshView mesh, const double* __restrict__ rule, int m1, const int* __restrict__ cells,
            const int* __restrict__ fn, const double* __restrict__ atoms, int n_atoms, double a, double norm,
            double inv2s2, double r0, double s, double* __restrict__ bA, double* __restrict__ G,
            double* __restrict__ ba, double* __restrict__ dC) {
  extern __shared__ double sh[];
  const int P1 = mesh.p + 1, nn = P1 * P1 * P1;
  double* L = sh;
  double* dL = L + m1 * P1;
  double* xs = dL + m1 * P1;
  double* ws = xs + m1;
  double* fv = ws + m1;
  double* gx = fv + kNucThreads;
  double* gy = gx + kNucThreads;
  double* gz = gy + kNucThreads;
  double* red = gz + kNucThreads;
  for (int i = threadIdx.x; i < 2 * m1 * P1 + 2 * m1; i += blockDim.x) sh[i] = rule[i];
  const int c = cells[blockIdx.x], J = fn[blockIdx.x];
  const CellGeo cg = cell_geo(mesh, c);
  const double sc0 = 2.0 / cg.hx, sc1 = 2.0 / cg.hy, sc2 = 2.0 / cg.hz;
  const double detJ = cg.hx * cg.hy * cg.hz / 8.0;
  const int npts = m1 * m1 * m1;
  double accB[2] = {0.0, 0.0}, accG[2] = {0.0, 0.0};
  double bacc = 0.0;
  __syncthreads();
  for (int q0 = 0; q0 < npts; q0 += kNucThreads) {
    const int q = q0 + threadIdx.x;
    double v = 0.0, g[3] = {0.0, 0.0, 0.0};
    if (q < npts) {
      const int q1 = q % m1, q2 = (q / m1) % m1, q3 = q / (m1 * m1);
      const double x = cg.ox + 0.5 * (xs[q1] + 1.0) * cg.hx;
      const double y = cg.oy + 0.5 * (xs[q2] + 1.0) * cg.hy;
      const double zc = cg.oz + 0.5 * (xs[q3] + 1.0) * cg.hz;
      const double w = ws[q1] * ws[q2] * ws[q3] * detJ;
      double b = 0.0;
      for (int t = 0; t < n_atoms; ++t) {
        const double dx = x - atoms[4 * t + 1], dy = y - atoms[4 * t + 2], dz = zc - atoms[4 * t + 3];
        b -= atoms[4 * t] * norm * exp(-(dx * dx + dy * dy + dz * dz) * inv2s2);
      }
      if (J < 0) {
        v = w * b;
      } else {
        double na, gn[3];
        nuc_atomic(atoms[4 * J], atoms[4 * J + 1], atoms[4 * J + 2], atoms[4 * J + 3], a, r0, s, x, y, zc, na, gn);
        v = w * na;
        g[0] = w * gn[0];
        g[1] = w * gn[1];
        g[2] = w * gn[2];
        bacc += w * b * na;
      }
    }
    fv[threadIdx.x] = v;
    gx[threadIdx.x] = g[0];
    gy[threadIdx.x] = g[1];
    gz[threadIdx.x] = g[2];
    __syncthreads();
    const int cnt = min(kNucThreads, npts - q0);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int l = threadIdx.x + j * kNucThreads;
      if (l >= nn) continue;
      const int i1 = l % P1, i2 = (l / P1) % P1, i3 = l / (P1 * P1);
      double ab = 0.0, ag = 0.0;
      for (int qq = 0; qq < cnt; ++qq) {
        const int qa = q0 + qq;
        const int q1 = qa % m1, q2 = (qa / m1) % m1, q3 = qa / (m1 * m1);
        const double l1 = L[q1 * P1 + i1], l2 = L[q2 * P1 + i2], l3 = L[q3 * P1 + i3];
        ab += fv[qq] * l1 * l2 * l3;
        if (J >= 0)
          ag += sc0 * gx[qq] * dL[q1 * P1 + i1] * l2 * l3 + sc1 * gy[qq] * l1 * dL[q2 * P1 + i2] * l3 +
                sc2 * gz[qq] * l1 * l2 * dL[q3 * P1 + i3];
      }
      accB[j] += ab;
      accG[j] += ag;
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int l = threadIdx.x + j * kNucThreads;
    if (l >= nn) continue;
    const long long g = node_index(mesh, cg.cx, cg.cy, cg.cz, l % P1, (l / P1) % P1, l / (P1 * P1));
    if (J < 0) {
      atomicAdd(&dC[g], accB[j]);
    } else {
      atomicAdd(&bA[(long long)J * mesh.n_h + g], accB[j]);
      atomicAdd(&G[(long long)J * mesh.n_h + g], accG[j]);
    }
  }
  if (J >= 0) {   // block-uniform branch
    const double tot = block_sum(bacc, red);
    if (threadIdx.x == 0) atomicAdd(&ba[J], tot);
  }
}

// AA[J][K] (and AA[K][J]) += int grad N^A_J . grad N^A_K over cell cells[k], J = fa[k] <= K = fb[k].
__global__ void __launch_bounds__(kNucThreads)
k_nuc_aa(const MeshView mesh, const double* __restrict__ rule, int m1, const int* __restrict__ cells,
         const int* __restrict__ fa, const int* __restrict__ fb, const double* __restrict__ atoms, double a, double r0,
         double s, int nA, double* __restrict__ AA) {
  __shared__ double red[kNucThreads];
  const int P1 = mesh.p + 1;
  const double* xs = rule + 2 * m1 * P1;
  const double* ws = xs + m1;
  const int c = cells[blockIdx.x], J = fa[blockIdx.x], K = fb[blockIdx.x];
  const CellGeo cg = cell_geo(mesh, c);
  const double detJ = cg.hx * cg.hy * cg.hz / 8.0;
  const int npts = m1 * m1 * m1;
  double acc = 0.0;
  for (int q = threadIdx.x; q < npts; q += blockDim.x) {
    const int q1 = q % m1, q2 = (q / m1) % m1, q3 = q / (m1 * m1);
    const double x = cg.ox + 0.5 * (xs[q1] + 1.0) * cg.hx;
    const double y = cg.oy + 0.5 * (xs[q2] + 1.0) * cg.hy;
    const double zc = cg.oz + 0.5 * (xs[q3] + 1.0) * cg.hz;
    const double w = ws[q1] * ws[q2] * ws[q3] * detJ;
    double va, ga[3], vb, gb[3];
    nuc_atomic(atoms[4 * J], atoms[4 * J + 1], atoms[4 * J + 2], atoms[4 * J + 3], a, r0, s, x, y, zc, va, ga);
    nuc_atomic(atoms[4 * K], atoms[4 * K + 1], atoms[4 * K + 2], atoms[4 * K + 3], a, r0, s, x, y, zc, vb, gb);
    acc += w * (ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2]);
  }
  const double tot = block_sum(acc, red);
  if (threadIdx.x == 0) {
    atomicAdd(&AA[J * nA + K], tot);
    if (J != K) atomicAdd(&AA[K * nA + J], tot);
  }
}

// C[J][g] = bA[J][g] / M_g at interior nodes (Dsc^2 = mask / M), 0 on the boundary; in place
__global__ void k_nuc_orth(double* __restrict__ bA, const double* __restrict__ Dsc, long long n_h, int nA) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n_h * nA) return;
  const double d = Dsc[idx % n_h];
  bA[idx] *= d * d;
}

// ACE[J][g] = k G[J][g] - LC[J][g] at interior nodes, 0 on the boundary; in place on LC
__global__ void k_nuc_ace(const double* __restrict__ G, const double* __restrict__ Dsc, long long n_h, int nA,
                          double k, double* __restrict__ LC) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n_h * nA) return;
  LC[idx] = Dsc[idx % n_h] != 0.0 ? k * G[idx] - LC[idx] : 0.0;
}

// out[i][j] = sum_g A[i lda + g] B[j ldb + g], one block per (i, j)
__global__ void __launch_bounds__(kNucThreads)
k_nuc_dots(const double* __restrict__ A, long long lda, const double* __restrict__ B, long long ldb, long long n,
           int nb, double* __restrict__ out) {
  __shared__ double red[kNucThreads];
  const int i = blockIdx.x / nb, j = blockIdx.x % nb;
  const double* a = A + (long long)i * lda;
  const double* b = B + (long long)j * ldb;
  double acc = 0.0;
  for (long long g = threadIdx.x; g < n; g += blockDim.x) acc += a[g] * b[g];
  const double tot = block_sum(acc, red);
  if (threadIdx.x == 0) out[blockIdx.x] = tot;
}

// phi_B[g] = -sum Z erf(a r) / r at boundary nodes (Dsc == 0), 0 inside
__global__ void k_nuc_bc(const double* __restrict__ nodes, const double* __restrict__ Dsc, long long n_h,
                         const double* __restrict__ atoms, int n_atoms, double a, double* __restrict__ phiB) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= n_h) return;
  double v = 0.0;
  if (Dsc[g] == 0.0) {
    for (int t = 0; t < n_atoms; ++t) {
      const double dx = nodes[3 * g] - atoms[4 * t + 1], dy = nodes[3 * g + 1] - atoms[4 * t + 2],
                   dz = nodes[3 * g + 2] - atoms[4 * t + 3];
      double f, df;
      nuc_radial(atoms[4 * t], a, sqrt(dx * dx + dy * dy + dz * dz), f, df);
      v += f;
    }
  }
  phiB[g] = v;
}

// u[g] = z[g] - sum_J xE[J] (X[J][g] + C[J][g])
__global__ void k_nuc_combine(const double* __restrict__ z, const double* __restrict__ X,
                              const double* __restrict__ C, const double* __restrict__ xE, long long n_h, int nA,
                              double* __restrict__ u) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= n_h) return;
  double v = z[g];
  for (int J = 0; J < nA; ++J) v -= xE[J] * (X[(long long)J * n_h + g] + C[(long long)J * n_h + g]);
  u[g] = v;
}

// vN[m] += sum_J xE[J] N^A_J(x_m) at the quadrature points
__global__ void k_nuc_add_atomic(const double* __restrict__ xq, long long npts, const double* __restrict__ atoms,
                                 int nA, double a, double r0, double s, const double* __restrict__ xE,
                                 double* __restrict__ vN) {
  const long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (m >= npts) return;
  double v = 0.0;
  for (int J = 0; J < nA; ++J) {
    double na, g[3];
    nuc_atomic(atoms[4 * J], atoms[4 * J + 1], atoms[4 * J + 2], atoms[4 * J + 3], a, r0, s, xq[3 * m],
               xq[3 * m + 1], xq[3 * m + 2], na, g);
    v += xE[J] * na;
  }
  vN[m] += v;
}

// distance from a point to an axis-aligned box
double box_distance(const double lo[3], const double hi[3], const double* R) {
  double d2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double e = std::max({lo[a] - R[a], R[a] - hi[a], 0.0});
    d2 += e * e;
  }
  return std::sqrt(d2);
}

// device buffers freed on every path
struct Bufs {
  std::vector<void*> p;
  template <class T>
  cudaError_t alloc(T*& out, size_t n) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, sizeof(T) * std::max<size_t>(n, 1));
    if (e != cudaSuccess) return e;
    p.push_back(q);
    out = static_cast<T*>(q);
    return cudaSuccess;
  }
  ~Bufs() {
    for (void* q : p) cudaFree(q);
  }
};

}  // namespace

efe_status nuclear_enriched(Ctx& c, double sigma, double r0, double s, int sub, int n_quad, double* phiE_host,
                            cudaStream_t st) {
  if (n_quad == 0) n_quad = c.p + 2;
  if (!(sigma > 0.0) || !(s > 0.0) || !(r0 > s) || sub < 1 || sub > 8 || n_quad < c.p + 1 || n_quad > 8 ||
      c.P1 > kMaxP1) {
    c.err = "nuclear enrichment: need sigma > 0, 0 < s < r0, sub in [1, 8], n_quad in [p + 1, 8]";
    return EFE_ERR_ARG;
  }
  const int nA = c.n_atoms;
  if (nA < 1) {
    c.err = "nuclear enrichment: the context has no atoms";
    return EFE_ERR_ARG;
  }
  const double lo[3] = {c.xb.front(), c.yb.front(), c.zb.front()};
  const double hi[3] = {c.xb.back(), c.yb.back(), c.zb.back()};
  for (int J = 0; J < nA; ++J)
    for (int a = 0; a < 3; ++a)
      if (c.R[3 * J + a] - lo[a] < r0 || hi[a] - c.R[3 * J + a] < r0) {
        c.err = "nuclear enrichment: every support (radius r0) must lie inside the box";
        return EFE_ERR_ARG;
      }
#define NUC_CK(x, what)                                                 \
  do {                                                                  \
    cudaError_t _e = (x);                                               \
    if (_e != cudaSuccess) {                                            \
      c.err = std::string(what) + ": " + cudaGetErrorString(_e);        \
      return _e == cudaErrorMemoryAllocation ? EFE_ERR_NOMEM : EFE_ERR_CUDA; \
    }                                                                   \
  } while (0)
  // composite 1D rule on [-1, 1] and the cell basis's Lagrange tables at its points
  const int m1 = sub * n_quad, P1 = c.P1;
  std::vector<double> xg(n_quad), wg(n_quad), gll(P1), gllw(P1);
  gauss_legendre(n_quad, xg.data(), wg.data());
  gauss_lobatto(c.p, gll.data(), gllw.data());
  std::vector<double> rule((size_t)2 * m1 * P1 + 2 * m1);
  double* xs = rule.data() + 2 * m1 * P1;
  double* ws = xs + m1;
  for (int k = 0; k < sub; ++k) {
    const double a0 = -1.0 + 2.0 * k / sub, b0 = -1.0 + 2.0 * (k + 1) / sub;
    for (int j = 0; j < n_quad; ++j) {
      xs[k * n_quad + j] = 0.5 * (b0 - a0) * xg[j] + 0.5 * (a0 + b0);
      ws[k * n_quad + j] = 0.5 * (b0 - a0) * wg[j];
    }
  }
  lagrange_tables(P1, gll.data(), m1, xs, rule.data(), rule.data() + m1 * P1);
  // work lists: (cell, atom) pairs of the supports, cells carrying charge, (cell, atom, atom) of overlaps
  const double reach = 40.0 * sigma;   // exp(-(40)^2 / 2) underflows: no charge beyond
  std::vector<int> it_cell, it_fn, aa_cell, aa_a, aa_b;
  std::vector<int> local;
  for (int cz = 0; cz < c.ncz; ++cz)
    for (int cy = 0; cy < c.ncy; ++cy)
      for (int cx = 0; cx < c.ncx; ++cx) {
        const int cell = cx + c.ncx * (cy + c.ncy * cz);
        const double blo[3] = {c.xb[cx], c.yb[cy], c.zb[cz]};
        const double bhi[3] = {c.xb[cx + 1], c.yb[cy + 1], c.zb[cz + 1]};
        local.clear();
        bool charged = false;
        for (int J = 0; J < nA; ++J) {
          const double d = box_distance(blo, bhi, &c.R[3 * J]);
          if (d < r0) local.push_back(J);
          if (d < reach) charged = true;
        }
        if (charged) {
          it_cell.push_back(cell);
          it_fn.push_back(-1);
        }
        for (size_t i = 0; i < local.size(); ++i) {
          it_cell.push_back(cell);
          it_fn.push_back(local[i]);
          for (size_t j = i; j < local.size(); ++j) {
            aa_cell.push_back(cell);
            aa_a.push_back(local[i]);
            aa_b.push_back(local[j]);
          }
        }
      }
  std::vector<double> at(4 * (size_t)nA);
  for (int J = 0; J < nA; ++J) {
    at[4 * J] = c.Z[J];
    for (int a = 0; a < 3; ++a) at[4 * J + 1 + a] = c.R[3 * J + a];
  }
  const long long n_h = c.n_h;
  const size_t vecs = (size_t)nA * n_h;
  Bufs B;
  double *d_rule, *d_at, *d_bA, *d_G, *d_ba, *d_dC, *d_AA, *d_LC, *d_X, *d_z, *d_Lz, *d_u, *d_Ap, *d_phiB, *d_nodes;
  double *d_dots, *d_xE;
  int *d_ic, *d_if, *d_ac, *d_aa, *d_ab;
  NUC_CK(B.alloc(d_rule, rule.size()), "allocating");
  NUC_CK(B.alloc(d_at, at.size()), "allocating");
  NUC_CK(B.alloc(d_bA, vecs), "allocating");
  NUC_CK(B.alloc(d_G, vecs), "allocating");
  NUC_CK(B.alloc(d_LC, vecs), "allocating");
  NUC_CK(B.alloc(d_X, vecs), "allocating");
  NUC_CK(B.alloc(d_ba, nA), "allocating");
  NUC_CK(B.alloc(d_AA, (size_t)nA * nA), "allocating");
  NUC_CK(B.alloc(d_dots, (size_t)5 * nA * nA + 3 * nA), "allocating");
  NUC_CK(B.alloc(d_xE, nA), "allocating");
  for (double** v : {&d_dC, &d_z, &d_Lz, &d_u, &d_Ap, &d_phiB}) NUC_CK(B.alloc(*v, (size_t)n_h), "allocating");
  NUC_CK(B.alloc(d_nodes, (size_t)3 * n_h), "allocating");
  NUC_CK(B.alloc(d_ic, it_cell.size()), "allocating");
  NUC_CK(B.alloc(d_if, it_fn.size()), "allocating");
  NUC_CK(B.alloc(d_ac, aa_cell.size()), "allocating");
  NUC_CK(B.alloc(d_aa, aa_a.size()), "allocating");
  NUC_CK(B.alloc(d_ab, aa_b.size()), "allocating");
  auto up = [&](void* dst, const void* src, size_t bytes) {
    return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st) : cudaSuccess;
  };
  NUC_CK(up(d_rule, rule.data(), sizeof(double) * rule.size()), "copy");
  NUC_CK(up(d_at, at.data(), sizeof(double) * at.size()), "copy");
  NUC_CK(up(d_ic, it_cell.data(), sizeof(int) * it_cell.size()), "copy");
  NUC_CK(up(d_if, it_fn.data(), sizeof(int) * it_fn.size()), "copy");
  NUC_CK(up(d_ac, aa_cell.data(), sizeof(int) * aa_cell.size()), "copy");
  NUC_CK(up(d_aa, aa_a.data(), sizeof(int) * aa_a.size()), "copy");
  NUC_CK(up(d_ab, aa_b.data(), sizeof(int) * aa_b.size()), "copy");
  for (double* v : {d_bA, d_G, d_LC})
    NUC_CK(cudaMemsetAsync(v, 0, sizeof(double) * vecs, st), "clear");
  NUC_CK(cudaMemsetAsync(d_ba, 0, sizeof(double) * nA, st), "clear");
  NUC_CK(cudaMemsetAsync(d_AA, 0, sizeof(double) * nA * nA, st), "clear");
  NUC_CK(cudaMemsetAsync(d_dC, 0, sizeof(double) * n_h, st), "clear");
  NUC_CK(cudaMemsetAsync(d_Lz, 0, sizeof(double) * n_h, st), "clear");
  // cell integrals of the atomic parts and of the charge
  const double a = 1.0 / (std::sqrt(2.0) * sigma);
  const double norm = std::pow(2.0 * kPi * sigma * sigma, -1.5);
  const double inv2s2 = 1.0 / (2.0 * sigma * sigma);
  if (!it_cell.empty()) {
    const size_t sm = sizeof(double) * (2 * (size_t)m1 * P1 + 2 * m1 + 5 * kNucThreads);
    k_nuc_cells<<<(unsigned)it_cell.size(), kNucThreads, sm, st>>>(c.mesh, d_rule, m1, d_ic, d_if, d_at, nA, a, norm,
                                                                    inv2s2, r0, s, d_bA, d_G, d_ba, d_dC);
    note_launch();
    NUC_CK(cudaGetLastError(), "cell integrals");
  }
  if (!aa_cell.empty()) {
    k_nuc_aa<<<(unsigned)aa_cell.size(), kNucThreads, 0, st>>>(c.mesh, d_rule, m1, d_ac, d_aa, d_ab, d_at, a, r0, s,
                                                                nA, d_AA);
    note_launch();
    NUC_CK(cudaGetLastError(), "atomic stiffness");
  }
  // orthogonalisation coefficients C (in place of bA), k K C_J, the dots of the enriched block
  const double k4 = 1.0 / (4.0 * kPi), lap = 1.0 / (2.0 * kPi);   // launch_laplace applies lap * (1/2) K
  double* d_C = d_bA;
  k_nuc_orth<<<nblk((long long)vecs), 256, 0, st>>>(d_C, c.d_Dsc, n_h, nA);
  note_launch();
  NUC_CK(cudaGetLastError(), "orthogonalisation");
  for (int J = 0; J < nA; ++J)
    NUC_CK(launch_laplace(c, d_C + (size_t)J * n_h, d_LC + (size_t)J * n_h, 1, 1, lap, st), "stiffness");
  double* CG = d_dots;                 // [nA][nA] C_J . G_K
  double* CLC = CG + nA * nA;          // [nA][nA] C_J . (k K C_K)
  double* AX = CLC + nA * nA;          // [nA][nA] A_IJ . X_K
  double* CdC = AX + nA * nA;          // [nA]     C_J . d
  double* Gz = CdC + nA;               // [nA]     G_J . z
  double* CLz = Gz + nA;               // [nA]     C_J . (k K z)
  auto dots = [&](const double* A, const double* Bv, int na, int nb, double* out) {
    k_nuc_dots<<<(unsigned)(na * nb), kNucThreads, 0, st>>>(A, n_h, Bv, n_h, n_h, nb, out);
    note_launch();
    return cudaGetLastError();
  };
  NUC_CK(dots(d_C, d_G, nA, nA, CG), "dots");
  NUC_CK(dots(d_C, d_LC, nA, nA, CLC), "dots");
  NUC_CK(dots(d_C, d_dC, nA, 1, CdC), "dots");
  // A_IJ (in place of k K C_J), X_J = A_II^-1 A_IJ
  k_nuc_ace<<<nblk((long long)vecs), 256, 0, st>>>(d_G, c.d_Dsc, n_h, nA, k4, d_LC);
  note_launch();
  NUC_CK(cudaGetLastError(), "coupling");
  for (int J = 0; J < nA; ++J)
    NUC_CK(fdm_solve(c, d_LC + (size_t)J * n_h, d_Ap, d_X + (size_t)J * n_h, 1, st, true), "direct solve");
  NUC_CK(dots(d_LC, d_X, nA, nA, AX), "dots");
  // classical solve with the smeared-nucleus boundary data
  NUC_CK(launch_coords(c, d_nodes, nullptr, st), "node coordinates");
  k_nuc_bc<<<nblk(n_h), 256, 0, st>>>(d_nodes, c.d_Dsc, n_h, d_at, nA, a, d_phiB);
  note_launch();
  NUC_CK(cudaGetLastError(), "boundary data");
  NUC_CK(fdm_solve(c, d_dC, d_Ap, d_z, 1, st, false, d_phiB), "direct solve");
  NUC_CK(launch_laplace(c, d_z, d_Lz, 1, 0, lap, st), "stiffness");
  NUC_CK(dots(d_G, d_z, nA, 1, Gz), "dots");
  NUC_CK(dots(d_C, d_Lz, nA, 1, CLz), "dots");
  // the enriched block on the host: S phi^E = rhs
  std::vector<double> hd((size_t)3 * nA * nA + 3 * nA), hAA((size_t)nA * nA), hba(nA);
  NUC_CK(cudaMemcpyAsync(hd.data(), d_dots, sizeof(double) * hd.size(), cudaMemcpyDeviceToHost, st), "copy");
  NUC_CK(cudaMemcpyAsync(hAA.data(), d_AA, sizeof(double) * hAA.size(), cudaMemcpyDeviceToHost, st), "copy");
  NUC_CK(cudaMemcpyAsync(hba.data(), d_ba, sizeof(double) * nA, cudaMemcpyDeviceToHost, st), "copy");
  NUC_CK(cudaStreamSynchronize(st), "set-up");
  const double* hCG = hd.data();
  const double* hCLC = hCG + nA * nA;
  const double* hAX = hCLC + nA * nA;
  const double* hCdC = hAX + nA * nA;
  const double* hGz = hCdC + nA;
  const double* hCLz = hGz + nA;
  std::vector<double> S((size_t)nA * nA), rhs(nA), x(nA);
  for (int J = 0; J < nA; ++J) {
    for (int K = 0; K < nA; ++K) {
      const double aee = k4 * (hAA[J * nA + K] - hCG[K * nA + J] - hCG[J * nA + K]) + hCLC[J * nA + K];
      S[J * nA + K] = aee - hAX[J * nA + K];
    }
    rhs[J] = (hba[J] - hCdC[J]) - k4 * hGz[J] + hCLz[J];
  }
  for (int J = 0; J < nA; ++J)
    for (int K = 0; K < J; ++K) S[J * nA + K] = S[K * nA + J] = 0.5 * (S[J * nA + K] + S[K * nA + J]);
  // Cholesky S = L L^T, then the two triangular solves
  std::vector<double> Lc((size_t)nA * nA, 0.0);
  for (int i = 0; i < nA; ++i)
    for (int j = 0; j <= i; ++j) {
      double v = S[i * nA + j];
      for (int k = 0; k < j; ++k) v -= Lc[i * nA + k] * Lc[j * nA + k];
      if (i == j) {
        if (!(v > 0.0)) {
          c.err = "nuclear enrichment: Schur complement not positive definite";
          return EFE_ERR_NOT_SPD;
        }
        Lc[i * nA + i] = std::sqrt(v);
      } else {
        Lc[i * nA + j] = v / Lc[j * nA + j];
      }
    }
  for (int i = 0; i < nA; ++i) {
    double v = rhs[i];
    for (int k = 0; k < i; ++k) v -= Lc[i * nA + k] * x[k];
    x[i] = v / Lc[i * nA + i];
  }
  for (int i = nA - 1; i >= 0; --i) {
    double v = x[i];
    for (int k = i + 1; k < nA; ++k) v -= Lc[k * nA + i] * x[k];
    x[i] = v / Lc[i * nA + i];
  }
  // v_N at the quadrature points
  NUC_CK(up(d_xE, x.data(), sizeof(double) * nA), "copy");
  k_nuc_combine<<<nblk(n_h), 256, 0, st>>>(d_z, d_X, d_C, d_xE, n_h, nA, d_u);
  note_launch();
  NUC_CK(cudaGetLastError(), "combine");
  NUC_CK(launch_interp(c, d_u, c.d_vN, 1, st), "interpolation");
  const long long npts = (long long)c.nc * c.nq;
  k_nuc_add_atomic<<<nblk(npts), 256, 0, st>>>(c.d_xq, npts, d_at, nA, a, r0, s, d_xE, c.d_vN);
  note_launch();
  NUC_CK(cudaGetLastError(), "enrichment values");
  NUC_CK(cudaStreamSynchronize(st), "set-up");
#undef NUC_CK
  if (phiE_host)
    for (int J = 0; J < nA; ++J) phiE_host[J] = x[J];
  c.state_valid = false;
  c.has_prev = false;
  return EFE_OK;
}

}  // namespace efe
