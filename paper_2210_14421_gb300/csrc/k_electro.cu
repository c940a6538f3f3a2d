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
#include <thread>
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

// Radial parts of the atomic functions.  NucRadial: one smeared nucleus,
// f = -Z erf(a r) / r.  TabRadial: the Hartree potential of an isolated
// neutral atom tabulated on r_i = rmax (i / (n - 1))^2, linear interpolation
// in r between the table points, f = n_el / r and Q = n_el beyond the table;
// df/dr = -Q(r) / r^2 with Q the enclosed charge.  atoms: [J][4] = Z, x, y, z.
struct NucRadial {
  double a;
  __device__ void operator()(const double* atoms, int J, double r, double& f, double& df) const {
    nuc_radial(atoms[4 * J], a, r, f, df);
  }
};

struct TabRadial {
  const double* r;     // [n] grid
  const double* v;     // [nA][n] potential
  const double* q;     // [nA][n] enclosed charge
  const double* nel;   // [nA] electrons (Q at the end of the table)
  int n;
  double rmax;
  __device__ void operator()(const double*, int J, double x, double& f, double& df) const {
    const double rl = r[n - 1];
    double Q;
    if (x <= rl) {
      // interval [r_j, r_j+1] holding x: guess from the grid law, then settle on the table values
      int j = (int)(sqrt(fmax(x, 0.0) / rmax) * (n - 1));
      j = min(max(j, 0), n - 2);
      while (j > 0 && r[j] > x) --j;
      while (j < n - 2 && r[j + 1] <= x) ++j;
      const double h = r[j + 1] - r[j];
      const double* vv = v + (long long)J * n;
      const double* qq = q + (long long)J * n;
      f = (vv[j + 1] - vv[j]) / h * (x - r[j]) + vv[j];
      Q = (qq[j + 1] - qq[j]) / h * (x - r[j]) + qq[j];
    } else {
      f = nel[J] / fmax(x, 1e-300);
      Q = nel[J];
    }
    df = x > 0.0 ? -Q / (x * x) : 0.0;
  }
};

// Atomic part N^A_J = f u (cutoff r0, s) at (x, y, w) and its gradient.
template <class Rad>
__device__ __forceinline__ void atomic_part(const Rad& rad, const double* atoms, int J, double r0, double s, double x,
                                            double y, double w, double& v, double g[3]) {
  const double dx = x - atoms[4 * J + 1], dy = y - atoms[4 * J + 2], dz = w - atoms[4 * J + 3];
  const double r = sqrt(dx * dx + dy * dy + dz * dz);
  double f, df, u, du;
  rad(atoms, J, r, f, df);
  cutoff(r, r0, s, u, du);
  v = f * u;
  const double radial = df * u + f * du;
  const double inv = r > 0.0 ? 1.0 / r : 0.0;
  g[0] = radial * dx * inv;
  g[1] = radial * dy * inv;
  g[2] = radial * dz * inv;
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

// Sum over the block (blockDim.x == kNucThreads), returned to every thread;
// safe to call again right away.
__device__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = kNucThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double out = red[0];
  __syncthreads();
  return out;
}

// Cell rules as lists of boxes: a box is [lo, hi]^3 in the cell's reference
// coordinates [-1, 1]^3 with the n^3 Gauss-Legendre rule on it (the uniform
// composite rule: sub^3 equal boxes; the adaptive rule: the boxes of the
// recursive refinement).  BoxRule holds, per box, the 1D Lagrange tables of the
// cell basis at its points (L, dL [3][n][P1]), the physical points (px [3][n])
// and the 1D weights including the Jacobian (pw [3][n]).
struct BoxTables {
  double L[3][8 * kMaxP1], dL[3][8 * kMaxP1], px[3][8], pw[3][8];
};

// Lagrange basis function i of the nodes and its derivative at x.
__device__ __forceinline__ double lagrange1(const double* nodes, int P1, int i, double x, double& d) {
  double v = 1.0;
  for (int j = 0; j < P1; ++j)
    if (j != i) v *= (x - nodes[j]) / (nodes[i] - nodes[j]);
  d = 0.0;
  for (int a = 0; a < P1; ++a) {
    if (a == i) continue;
    double t = 1.0 / (nodes[i] - nodes[a]);
    for (int j = 0; j < P1; ++j)
      if (j != i && j != a) t *= (x - nodes[j]) / (nodes[i] - nodes[j]);
    d += t;
  }
  return v;
}

// Fills the tables of box `box` (6 doubles: lo[3], hi[3]) for a cell with origin o and sizes h.
__device__ void box_tables(BoxTables& T, const double* box, const double* gll, int P1, const double* xg,
                           const double* wg, int n, const double o[3], const double h[3]) {
  for (int t = threadIdx.x; t < 3 * n * P1; t += blockDim.x) {
    const int a = t / (n * P1), j = (t / P1) % n, i = t % P1;
    const double mid = 0.5 * (box[a] + box[3 + a]), half = 0.5 * (box[3 + a] - box[a]);
    double d;
    T.L[a][j * P1 + i] = lagrange1(gll, P1, i, mid + xg[j] * half, d);
    T.dL[a][j * P1 + i] = d;
  }
  for (int t = threadIdx.x; t < 3 * n; t += blockDim.x) {
    const int a = t / n, j = t % n;
    const double mid = 0.5 * (box[a] + box[3 + a]), half = 0.5 * (box[3 + a] - box[a]);
    T.px[a][j] = o[a] + 0.5 * (mid + xg[j] * half + 1.0) * h[a];
    T.pw[a][j] = wg[j] * half * 0.5 * h[a];
  }
}

// Cell integrals on the item's boxes.  One block per item k: for fn[k] = J >= 0,
// over cell cells[k]
//   bA[J][g] += int N^A_J N_g,  G[J][g] += int grad N^A_J . grad N_g,  ba[J] += int b N^A_J;
// for fn[k] < 0 the charge load dC[g] += int b N_g (b from the smeared nuclei;
// with norm = 0 the charge terms vanish, as for the Hartree enrichment).  The
// cell's boxes are boxes[cb[c] .. cb[c + 1]) (cb indexed by cell).
template <class Rad>
__global__ void __launch_bounds__(kNucThreads)
k_nuc_cells(const MeshView mesh, const double* __restrict__ gll, const double* __restrict__ xg,
            const double* __restrict__ wg, int n, const long long* __restrict__ cb, const double* __restrict__ boxes,
            const int* __restrict__ cells, const int* __restrict__ fn, const double* __restrict__ atoms, int n_atoms,
            const Rad rad, double norm, double inv2s2, double r0, double s, double* __restrict__ bA,
            double* __restrict__ G, double* __restrict__ ba, double* __restrict__ dC) {
  __shared__ BoxTables T;
  __shared__ double fv[kNucThreads], gx[kNucThreads], gy[kNucThreads], gz[kNucThreads], red[kNucThreads];
  const int P1 = mesh.p + 1, nn = P1 * P1 * P1;
  const int c = cells[blockIdx.x], J = fn[blockIdx.x];
  const CellGeo cg = cell_geo(mesh, c);
  const double o[3] = {cg.ox, cg.oy, cg.oz}, h[3] = {cg.hx, cg.hy, cg.hz};
  const double sc0 = 2.0 / cg.hx, sc1 = 2.0 / cg.hy, sc2 = 2.0 / cg.hz;
  const int npts = n * n * n;
  double accB[2] = {0.0, 0.0}, accG[2] = {0.0, 0.0};
  double bacc = 0.0;
  for (long long bx = cb[c]; bx < cb[c + 1]; ++bx) {
    box_tables(T, boxes + 6 * bx, gll, P1, xg, wg, n, o, h);
    __syncthreads();
    for (int q0 = 0; q0 < npts; q0 += kNucThreads) {
      const int q = q0 + threadIdx.x;
      double v = 0.0, g[3] = {0.0, 0.0, 0.0};
      if (q < npts) {
        const int q1 = q % n, q2 = (q / n) % n, q3 = q / (n * n);
        const double x = T.px[0][q1], y = T.px[1][q2], zc = T.px[2][q3];
        const double w = T.pw[0][q1] * T.pw[1][q2] * T.pw[2][q3];
        double b = 0.0;
        for (int t = 0; t < n_atoms; ++t) {
          const double dx = x - atoms[4 * t + 1], dy = y - atoms[4 * t + 2], dz = zc - atoms[4 * t + 3];
          b -= atoms[4 * t] * norm * exp(-(dx * dx + dy * dy + dz * dz) * inv2s2);
        }
        if (J < 0) {
          v = w * b;
        } else {
          double na, gn[3];
          atomic_part(rad, atoms, J, r0, s, x, y, zc, na, gn);
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
          const int q1 = qa % n, q2 = (qa / n) % n, q3 = qa / (n * n);
          const double l1 = T.L[0][q1 * P1 + i1], l2 = T.L[1][q2 * P1 + i2], l3 = T.L[2][q3 * P1 + i3];
          ab += fv[qq] * l1 * l2 * l3;
          if (J >= 0)
            ag += sc0 * gx[qq] * T.dL[0][q1 * P1 + i1] * l2 * l3 + sc1 * gy[qq] * l1 * T.dL[1][q2 * P1 + i2] * l3 +
                  sc2 * gz[qq] * l1 * l2 * T.dL[2][q3 * P1 + i3];
        }
        accB[j] += ab;
        accG[j] += ag;
      }
      __syncthreads();
    }
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

// AA[J][K] (and AA[K][J]) += int grad N^A_J . grad N^A_K over the boxes of cell cells[k],
// J = fa[k] <= K = fb[k].
template <class Rad>
__global__ void __launch_bounds__(kNucThreads)
k_nuc_aa(const MeshView mesh, const double* __restrict__ xg, const double* __restrict__ wg, int n,
         const long long* __restrict__ cb, const double* __restrict__ boxes, const int* __restrict__ cells,
         const int* __restrict__ fa, const int* __restrict__ fb, const double* __restrict__ atoms, const Rad rad,
         double r0, double s, int nA, double* __restrict__ AA) {
  __shared__ double red[kNucThreads];
  const int c = cells[blockIdx.x], J = fa[blockIdx.x], K = fb[blockIdx.x];
  const CellGeo cg = cell_geo(mesh, c);
  const double o[3] = {cg.ox, cg.oy, cg.oz}, h[3] = {cg.hx, cg.hy, cg.hz};
  const int npts = n * n * n;
  double acc = 0.0;
  for (long long bx = cb[c]; bx < cb[c + 1]; ++bx) {
    const double* box = boxes + 6 * bx;
    for (int q = threadIdx.x; q < npts; q += blockDim.x) {
      const int qi[3] = {q % n, (q / n) % n, q / (n * n)};
      double x[3], w = 1.0;
      for (int a = 0; a < 3; ++a) {
        const double mid = 0.5 * (box[a] + box[3 + a]), half = 0.5 * (box[3 + a] - box[a]);
        x[a] = o[a] + 0.5 * (mid + xg[qi[a]] * half + 1.0) * h[a];
        w *= wg[qi[a]] * half * 0.5 * h[a];
      }
      double va, ga[3], vb, gb[3];
      atomic_part(rad, atoms, J, r0, s, x[0], x[1], x[2], va, ga);
      atomic_part(rad, atoms, K, r0, s, x[0], x[1], x[2], vb, gb);
      acc += w * (ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2]);
    }
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
template <class Rad>
__global__ void k_nuc_add_atomic(const double* __restrict__ xq, long long npts, const double* __restrict__ atoms,
                                 int nA, const Rad rad, double r0, double s, const double* __restrict__ xE,
                                 double* __restrict__ vN) {
  const long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (m >= npts) return;
  double v = 0.0;
  for (int J = 0; J < nA; ++J) {
    double na, g[3];
    atomic_part(rad, atoms, J, r0, s, xq[3 * m], xq[3 * m + 1], xq[3 * m + 2], na, g);
    v += xE[J] * na;
  }
  vN[m] += v;
}


// ---------------------------------------------------------------------------- enriched Hartree solve
// Per-solve kernels; members m < nb of the batch, nodal vectors [n_h][nb], quadrature
// fields [nb][n_cells][nq].

// dA[J][m] += sum_q w|J| rho_m N^A_J at the quadrature points of the pair's cell
template <class Rad>
__global__ void __launch_bounds__(kNucThreads)
k_hen_load(const int* __restrict__ cells, const int* __restrict__ fn, int nq, int nc, int nb,
           const double* __restrict__ xq, const double* __restrict__ wJ, const double* __restrict__ rho,
           const double* __restrict__ atoms, const Rad rad, double r0, double s, double* __restrict__ dA) {
  __shared__ double wa[kMaxNQ1 * kMaxNQ1 * kMaxNQ1];
  __shared__ double red[kNucThreads];
  const int c = cells[blockIdx.x], J = fn[blockIdx.x];
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    const long long m = (long long)c * nq + q;
    double na, g[3];
    atomic_part(rad, atoms, J, r0, s, xq[3 * m], xq[3 * m + 1], xq[3 * m + 2], na, g);
    wa[q] = wJ[m] * na;
  }
  __syncthreads();
  for (int b = 0; b < nb; ++b) {
    double acc = 0.0;
    for (int q = threadIdx.x; q < nq; q += blockDim.x) acc += wa[q] * rho[((long long)b * nc + c) * nq + q];
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) atomicAdd(&dA[J * nb + b], tot);
  }
}

// Partial dots of the right sides, spread over gridDim.y slices of the nodes:
// sums[0][J][m] += C_J . d_m, sums[1][J][m] += G_J . z_m, sums[2][J][m] += C_J . Lz_m
// (blockIdx.x = (J, m); the caller zeroes sums)
__global__ void __launch_bounds__(kNucThreads)
k_hen_dots(const double* __restrict__ C, const double* __restrict__ G, const double* __restrict__ d,
           const double* __restrict__ z, const double* __restrict__ Lz, long long n_h, int nb, int nAnb,
           double* __restrict__ sums) {
  __shared__ double red[kNucThreads];
  const int J = blockIdx.x / nb, b = blockIdx.x % nb;
  const double* cj = C + (long long)J * n_h;
  const double* gj = G + (long long)J * n_h;
  const long long chunk = (n_h + gridDim.y - 1) / gridDim.y;
  const long long g0 = (long long)blockIdx.y * chunk, g1 = min(n_h, g0 + chunk);
  double ad = 0.0, az = 0.0, al = 0.0;
  for (long long g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
    const long long i = g * nb + b;
    ad += cj[g] * d[i];
    az += gj[g] * z[i];
    al += cj[g] * Lz[i];
  }
  const double sd = block_sum(ad, red);
  const double sz = block_sum(az, red);
  const double sl = block_sum(al, red);
  if (threadIdx.x == 0) {
    atomicAdd(&sums[blockIdx.x], sd);
    atomicAdd(&sums[nAnb + blockIdx.x], sz);
    atomicAdd(&sums[2 * nAnb + blockIdx.x], sl);
  }
}

// rhs[J][m] = dA[J][m] - C_J . d_m - k G_J . z_m + C_J . Lz_m
__global__ void k_hen_rhs(const double* __restrict__ dA, const double* __restrict__ sums, int nAnb, double k,
                          double* __restrict__ rhs) {
  for (int i = threadIdx.x; i < nAnb; i += blockDim.x)
    rhs[i] = dA[i] - sums[i] - k * sums[nAnb + i] + sums[2 * nAnb + i];
}

// xE[J][m] = sum_K Sinv[J][K] rhs[K][m]
__global__ void k_hen_coef(const double* __restrict__ Sinv, const double* __restrict__ rhs, int nA, int nb,
                           double* __restrict__ xE) {
  for (int i = threadIdx.x; i < nA * nb; i += blockDim.x) {
    const int J = i / nb, b = i % nb;
    double v = 0.0;
    for (int K = 0; K < nA; ++K) v += Sinv[J * nA + K] * rhs[K * nb + b];
    xE[i] = v;
  }
}

// phi = z - sum_J xE_J X_J (in place), u = phi - sum_J xE_J C_J
__global__ void k_hen_combine(double* __restrict__ phi, double* __restrict__ u, const double* __restrict__ X,
                              const double* __restrict__ C, const double* __restrict__ xE, long long n_h, int nA,
                              int nb) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n_h * nb) return;
  const long long g = idx / nb;
  const int b = (int)(idx % nb);
  double p = phi[idx], cc = 0.0;
  for (int J = 0; J < nA; ++J) {
    const double e = xE[J * nb + b];
    p -= e * X[(long long)J * n_h + g];
    cc += e * C[(long long)J * n_h + g];
  }
  phi[idx] = p;
  u[idx] = p - cc;
}

// vH[m][pt] += sum_J xE[J][m] N^A_J(x_pt)
template <class Rad>
__global__ void k_hen_add(const double* __restrict__ xq, long long npts, int nb, const double* __restrict__ atoms,
                          int nA, const Rad rad, double r0, double s, const double* __restrict__ xE,
                          double* __restrict__ vH) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= npts * nb) return;
  const int b = (int)(idx / npts);
  const long long m = idx % npts;
  double v = 0.0;
  for (int J = 0; J < nA; ++J) {
    double na, g[3];
    atomic_part(rad, atoms, J, r0, s, xq[3 * m], xq[3 * m + 1], xq[3 * m + 2], na, g);
    v += xE[J * nb + b] * na;
  }
  vH[idx] += v;
}

// Transposed enriched Hartree map (the adjoint's v_H'(rho)^T): helpers.
// out[J] = (X_J + C_J) . h   (one block per atom)
__global__ void __launch_bounds__(kNucThreads)
k_hen_xc_dot(const double* __restrict__ X, const double* __restrict__ C, const double* __restrict__ h, long long n_h,
             double* __restrict__ out) {
  __shared__ double red[kNucThreads];
  const int J = blockIdx.x;
  const double* xj = X + (long long)J * n_h;
  const double* cj = C + (long long)J * n_h;
  double acc = 0.0;
  for (long long g = threadIdx.x; g < n_h; g += blockDim.x) acc += (xj[g] + cj[g]) * h[g];
  const double tot = block_sum(acc, red);
  if (threadIdx.x == 0) out[J] = tot;
}

// t = Sinv (sN - sX)
__global__ void k_hen_tcoef(const double* __restrict__ Sinv, const double* __restrict__ sN,
                            const double* __restrict__ sX, int nA, double* __restrict__ t) {
  for (int J = threadIdx.x; J < nA; J += blockDim.x) {
    double v = 0.0;
    for (int K = 0; K < nA; ++K) v += Sinv[J * nA + K] * (sN[K] - sX[K]);
    t[J] = v;
  }
}

// ct = sum_J t_J C_J;  r0 = sum_J t_J G_J
__global__ void k_hen_comb_t(const double* __restrict__ C, const double* __restrict__ G, const double* __restrict__ t,
                             long long n_h, int nA, double* __restrict__ ct, double* __restrict__ gt) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= n_h) return;
  double a = 0.0, b = 0.0;
  for (int J = 0; J < nA; ++J) {
    a += t[J] * C[(long long)J * n_h + g];
    b += t[J] * G[(long long)J * n_h + g];
  }
  ct[g] = a;
  gt[g] = b;
}

// r = k gt - Kc at interior nodes, 0 on the boundary (in place on gt)
__global__ void k_hen_rvec(double* __restrict__ gt, const double* __restrict__ Kc, const double* __restrict__ Dsc,
                           long long n_h, double k) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= n_h) return;
  gt[g] = Dsc[g] != 0.0 ? k * gt[g] - Kc[g] : 0.0;
}

// y = Zh - ct - Zr
__global__ void k_hen_yvec(const double* __restrict__ Zh, const double* __restrict__ ct, const double* __restrict__ Zr,
                           long long n_h, double* __restrict__ y) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= n_h) return;
  y[g] = Zh[g] - ct[g] - Zr[g];
}

// ---------------------------------------------------------------------------- host side
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

#define ENR_CK(x, what)                                                      \
  do {                                                                       \
    cudaError_t _e = (x);                                                    \
    if (_e != cudaSuccess) {                                                 \
      c.err = std::string(what) + ": " + cudaGetErrorString(_e);             \
      return _e == cudaErrorMemoryAllocation ? EFE_ERR_NOMEM : EFE_ERR_CUDA; \
    }                                                                        \
  } while (0)

// Checks shared by both problems: atoms present, 0 < s < r0, rule sizes, every
// support ball inside the box (the enrichment functions vanish on the boundary).
bool enr_args_ok(Ctx& c, double r0, double s, int sub, int& n_quad) {
  if (n_quad == 0) n_quad = c.p + 2;
  if (c.n_atoms < 1) {
    c.err = "electrostatic enrichment: the context has no atoms";
    return false;
  }
  if (!(s > 0.0) || !(r0 > s) || sub < 1 || sub > 8 || n_quad < c.p + 1 || n_quad > 8 || c.P1 > kMaxP1) {
    c.err = "electrostatic enrichment: need 0 < s < r0, sub in [1, 8], n_quad in [p + 1, 8]";
    return false;
  }
  const double lo[3] = {c.xb.front(), c.yb.front(), c.zb.front()};
  const double hi[3] = {c.xb.back(), c.yb.back(), c.zb.back()};
  for (int J = 0; J < c.n_atoms; ++J)
    for (int a = 0; a < 3; ++a)
      if (c.R[3 * J + a] - lo[a] < r0 || hi[a] - c.R[3 * J + a] < r0) {
        c.err = "electrostatic enrichment: every support (radius r0) must lie inside the box";
        return false;
      }
  return true;
}

// Work lists: (cell, atom) pairs whose cell meets the atom's support ball, cells
// within `reach` of a nucleus as charge items (fn = -1; reach 0: none), and
// (cell, atom, atom) overlaps with the first atom <= the second.
struct Lists {
  std::vector<int> it_cell, it_fn, pr_cell, pr_fn, aa_cell, aa_a, aa_b;
};

void work_lists(const Ctx& c, double r0, double reach, Lists& L) {
  std::vector<int> local;
  for (int cz = 0; cz < c.ncz; ++cz)
    for (int cy = 0; cy < c.ncy; ++cy)
      for (int cx = 0; cx < c.ncx; ++cx) {
        const int cell = cx + c.ncx * (cy + c.ncy * cz);
        const double blo[3] = {c.xb[cx], c.yb[cy], c.zb[cz]};
        const double bhi[3] = {c.xb[cx + 1], c.yb[cy + 1], c.zb[cz + 1]};
        local.clear();
        bool charged = false;
        for (int J = 0; J < c.n_atoms; ++J) {
          const double d = box_distance(blo, bhi, &c.R[3 * J]);
          if (d < r0) local.push_back(J);
          if (d < reach) charged = true;
        }
        if (charged) {
          L.it_cell.push_back(cell);
          L.it_fn.push_back(-1);
        }
        for (size_t i = 0; i < local.size(); ++i) {
          L.it_cell.push_back(cell);
          L.it_fn.push_back(local[i]);
          L.pr_cell.push_back(cell);
          L.pr_fn.push_back(local[i]);
          for (size_t j = i; j < local.size(); ++j) {
            L.aa_cell.push_back(cell);
            L.aa_a.push_back(local[i]);
            L.aa_b.push_back(local[j]);
          }
        }
      }
}

// A cell rule: n^3 Gauss-Legendre points on each of a cell's boxes (reference
// coordinates, lo[3] then hi[3]); boxes of cell c: boxes[6 cb[c] .. 6 cb[c + 1]).
// Only the cells of the work lists carry boxes (elsewhere every integrand vanishes).
struct BoxRule {
  int n = 0;
  std::vector<long long> cb;
  std::vector<double> boxes;
};

std::vector<char> listed_cells(const Ctx& c, const Lists& L) {
  std::vector<char> on(c.nc, 0);
  for (int x : L.it_cell) on[x] = 1;
  for (int x : L.aa_cell) on[x] = 1;
  return on;
}

// The uniform composite rule: sub^3 equal boxes per listed cell.
BoxRule uniform_rule(const Ctx& c, const Lists& L, int sub, int n) {
  BoxRule R;
  R.n = n;
  const std::vector<char> on = listed_cells(c, L);
  R.cb.assign(c.nc + 1, 0);
  for (int cell = 0; cell < c.nc; ++cell) {
    R.cb[cell + 1] = R.cb[cell];
    if (!on[cell]) continue;
    for (int k3 = 0; k3 < sub; ++k3)
      for (int k2 = 0; k2 < sub; ++k2)
        for (int k1 = 0; k1 < sub; ++k1) {
          const int k[3] = {k1, k2, k3};
          for (int a = 0; a < 3; ++a) R.boxes.push_back(-1.0 + 2.0 * k[a] / sub);
          for (int a = 0; a < 3; ++a) R.boxes.push_back(-1.0 + 2.0 * (k[a] + 1) / sub);
          ++R.cb[cell + 1];
        }
  }
  return R;
}

// The adaptive rule (reading Q1): a box's n^3 estimate of the trial integrals
// against the sum of the same rule on its eight half-size children; where every
// trial integral agrees to tol the children are kept, else each child is refined
// the same way, down to max_depth levels.  Trial integrands of the nuclear
// enrichment: the smeared charge b and the atomic part N^A_J of every atom
// (those that vanish on a cell contribute zero to both estimates and are skipped,
// as are the charges of nuclei beyond 40 sigma).
struct NucTrial {
  const double* R;   // [nA][3]
  const double* Z;   // [nA]
  double a, norm, inv2s2, r0, s;
  std::vector<int> local, nearb;   // atoms whose support / charge reaches the cell
  void eval(const double x[3], double* out) const {
    double b = 0.0;
    for (int t : nearb) {
      const double dx = x[0] - R[3 * t], dy = x[1] - R[3 * t + 1], dz = x[2] - R[3 * t + 2];
      b -= Z[t] * norm * std::exp(-(dx * dx + dy * dy + dz * dz) * inv2s2);
    }
    out[0] = b;
    for (size_t k = 0; k < local.size(); ++k) {
      const int J = local[k];
      const double dx = x[0] - R[3 * J], dy = x[1] - R[3 * J + 1], dz = x[2] - R[3 * J + 2];
      const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
      const double f = r > 0.0 ? -Z[J] * std::erf(a * r) / r : -Z[J] * 2.0 * a / std::sqrt(kPi);
      double u, du;
      cutoff(r, r0, s, u, du);
      out[1 + k] = f * u;
    }
  }
};

void box_integrals(const NucTrial& T, const double lo[3], const double hi[3], const double o[3], const double h[3],
                   const std::vector<double>& xg, const std::vector<double>& wg, double* acc, double* val) {
  const int n = (int)xg.size(), m = 1 + (int)T.local.size();
  for (int i = 0; i < m; ++i) acc[i] = 0.0;
  double mid[3], half[3];
  for (int a = 0; a < 3; ++a) {
    mid[a] = 0.5 * (lo[a] + hi[a]);
    half[a] = 0.5 * (hi[a] - lo[a]);
  }
  for (int k3 = 0; k3 < n; ++k3)
    for (int k2 = 0; k2 < n; ++k2)
      for (int k1 = 0; k1 < n; ++k1) {
        const int k[3] = {k1, k2, k3};
        double x[3], w = 1.0;
        for (int a = 0; a < 3; ++a) {
          x[a] = o[a] + 0.5 * (mid[a] + xg[k[a]] * half[a] + 1.0) * h[a];
          w *= wg[k[a]] * half[a] * 0.5 * h[a];
        }
        T.eval(x, val);
        for (int i = 0; i < m; ++i) acc[i] += w * val[i];
      }
}

void adapt_box(const NucTrial& T, const double lo[3], const double hi[3], int depth, int max_depth, double tol,
               const double o[3], const double h[3], const std::vector<double>& xg, const std::vector<double>& wg,
               std::vector<double>& out) {
  const int m = 1 + (int)T.local.size();
  std::vector<double> coarse(m), fine(m, 0.0), part(m), val(m);
  box_integrals(T, lo, hi, o, h, xg, wg, coarse.data(), val.data());
  double clo[8][3], chi[8][3];
  for (int i = 0; i < 8; ++i)
    for (int a = 0; a < 3; ++a) {
      const double mid = 0.5 * (lo[a] + hi[a]);
      const bool up = (i >> a) & 1;
      clo[i][a] = up ? mid : lo[a];
      chi[i][a] = up ? hi[a] : mid;
    }
  for (int i = 0; i < 8; ++i) {
    box_integrals(T, clo[i], chi[i], o, h, xg, wg, part.data(), val.data());
    for (int j = 0; j < m; ++j) fine[j] += part[j];
  }
  bool ok = depth >= max_depth;
  if (!ok) {
    ok = true;
    for (int j = 0; j < m; ++j)
      if (!(std::fabs(fine[j] - coarse[j]) <= tol)) ok = false;
  }
  if (ok) {
    for (int i = 0; i < 8; ++i) {
      out.insert(out.end(), clo[i], clo[i] + 3);
      out.insert(out.end(), chi[i], chi[i] + 3);
    }
    return;
  }
  for (int i = 0; i < 8; ++i) adapt_box(T, clo[i], chi[i], depth + 1, max_depth, tol, o, h, xg, wg, out);
}

// The adaptive boxes of one cell (origin o, sizes h) for atoms R [nA][3], Z [nA].
void adaptive_cell(const double o[3], const double h[3], const double* R, const double* Z, int nA, double sigma,
                   double r0, double s, const std::vector<double>& xg, const std::vector<double>& wg, double tol,
                   int max_depth, std::vector<double>& out) {
  const double bhi[3] = {o[0] + h[0], o[1] + h[1], o[2] + h[2]};
  NucTrial T{R, Z, 1.0 / (std::sqrt(2.0) * sigma), std::pow(2.0 * kPi * sigma * sigma, -1.5),
             1.0 / (2.0 * sigma * sigma), r0, s, {}, {}};
  for (int J = 0; J < nA; ++J) {
    const double d = box_distance(o, bhi, &R[3 * J]);
    if (d < r0) T.local.push_back(J);
    if (d < 40.0 * sigma) T.nearb.push_back(J);
  }
  const double lo[3] = {-1.0, -1.0, -1.0}, hi[3] = {1.0, 1.0, 1.0};
  adapt_box(T, lo, hi, 0, max_depth, tol, o, h, xg, wg, out);
}

BoxRule adaptive_rule(const Ctx& c, const Lists& L, int n, double tol, int max_depth, double sigma, double r0,
                      double s) {
  BoxRule R;
  R.n = n;
  std::vector<double> xg(n), wg(n);
  gauss_legendre(n, xg.data(), wg.data());
  const std::vector<char> on = listed_cells(c, L);
  std::vector<int> cells;
  for (int cell = 0; cell < c.nc; ++cell)
    if (on[cell]) cells.push_back(cell);
  std::vector<std::vector<double>> per(cells.size());
  const unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  auto work = [&](unsigned tid) {
    for (size_t i = tid; i < cells.size(); i += nt) {
      const int cell = cells[i];
      const int cx = cell % c.ncx, cy = (cell / c.ncx) % c.ncy, cz = cell / (c.ncx * c.ncy);
      const double o[3] = {c.xb[cx], c.yb[cy], c.zb[cz]};
      const double h[3] = {c.xb[cx + 1] - c.xb[cx], c.yb[cy + 1] - c.yb[cy], c.zb[cz + 1] - c.zb[cz]};
      adaptive_cell(o, h, c.R.data(), c.Z.data(), c.n_atoms, sigma, r0, s, xg, wg, tol, max_depth, per[i]);
    }
  };
  std::vector<std::thread> pool;
  for (unsigned t = 0; t < nt; ++t) pool.emplace_back(work, t);
  for (auto& t : pool) t.join();
  R.cb.assign(c.nc + 1, 0);
  size_t i = 0;
  for (int cell = 0; cell < c.nc; ++cell) {
    R.cb[cell + 1] = R.cb[cell];
    if (i < cells.size() && cells[i] == cell) {
      R.cb[cell + 1] += (long long)(per[i].size() / 6);
      R.boxes.insert(R.boxes.end(), per[i].begin(), per[i].end());
      ++i;
    }
  }
  return R;
}

// Blocks of one enrichment (module comment): C (d_C), G (d_G), A_IJ (d_LC),
// X_J = A_II^-1 A_IJ (d_X), each [nA][n_h], and on the host S = A_EE - A_EI X.
// With a charge (norm > 0) also d = int b N (d_dC) and, on the host,
// dE = int b N^A - C . d.  Synchronises st.
template <class Rad>
efe_status enr_blocks(Ctx& c, const Rad& rad, const double* d_at, double r0, double s, const BoxRule& rule,
                      double norm, double inv2s2, const Lists& L, double* d_C, double* d_G,
                      double* d_LC, double* d_X, double* d_dC, std::vector<double>& S, std::vector<double>& dE,
                      cudaStream_t st) {
  const int nA = c.n_atoms, P1 = c.P1, n = rule.n;
  const long long n_h = c.n_h;
  const size_t vecs = (size_t)nA * n_h;
  std::vector<double> tabs(P1 + 2 * n), gllw(P1);   // GLL nodes, GL points, GL weights
  gauss_lobatto(c.p, tabs.data(), gllw.data());
  gauss_legendre(n, tabs.data() + P1, tabs.data() + P1 + n);
  Bufs B;
  double *d_tabs, *d_boxes, *d_ba, *d_AA, *d_dots, *d_Ap;
  long long* d_cb;
  int *d_ic, *d_if, *d_ac, *d_aa, *d_ab;
  ENR_CK(B.alloc(d_tabs, tabs.size()), "allocating");
  ENR_CK(B.alloc(d_boxes, rule.boxes.size()), "allocating");
  ENR_CK(B.alloc(d_cb, rule.cb.size()), "allocating");
  ENR_CK(B.alloc(d_ba, nA), "allocating");
  ENR_CK(B.alloc(d_AA, (size_t)nA * nA), "allocating");
  ENR_CK(B.alloc(d_dots, (size_t)3 * nA * nA + nA), "allocating");
  ENR_CK(B.alloc(d_Ap, (size_t)n_h), "allocating");
  ENR_CK(B.alloc(d_ic, L.it_cell.size()), "allocating");
  ENR_CK(B.alloc(d_if, L.it_fn.size()), "allocating");
  ENR_CK(B.alloc(d_ac, L.aa_cell.size()), "allocating");
  ENR_CK(B.alloc(d_aa, L.aa_a.size()), "allocating");
  ENR_CK(B.alloc(d_ab, L.aa_b.size()), "allocating");
  auto up = [&](void* dst, const void* src, size_t bytes) {
    return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st) : cudaSuccess;
  };
  ENR_CK(up(d_tabs, tabs.data(), sizeof(double) * tabs.size()), "copy");
  ENR_CK(up(d_boxes, rule.boxes.data(), sizeof(double) * rule.boxes.size()), "copy");
  ENR_CK(up(d_cb, rule.cb.data(), sizeof(long long) * rule.cb.size()), "copy");
  ENR_CK(up(d_ic, L.it_cell.data(), sizeof(int) * L.it_cell.size()), "copy");
  ENR_CK(up(d_if, L.it_fn.data(), sizeof(int) * L.it_fn.size()), "copy");
  ENR_CK(up(d_ac, L.aa_cell.data(), sizeof(int) * L.aa_cell.size()), "copy");
  ENR_CK(up(d_aa, L.aa_a.data(), sizeof(int) * L.aa_a.size()), "copy");
  ENR_CK(up(d_ab, L.aa_b.data(), sizeof(int) * L.aa_b.size()), "copy");
  for (double* v : {d_C, d_G, d_LC}) ENR_CK(cudaMemsetAsync(v, 0, sizeof(double) * vecs, st), "clear");
  ENR_CK(cudaMemsetAsync(d_ba, 0, sizeof(double) * nA, st), "clear");
  ENR_CK(cudaMemsetAsync(d_AA, 0, sizeof(double) * nA * nA, st), "clear");
  if (d_dC) ENR_CK(cudaMemsetAsync(d_dC, 0, sizeof(double) * n_h, st), "clear");
  // cell integrals (bA into d_C, then scaled in place)
  const double* d_gll = d_tabs;
  const double* d_xg = d_tabs + P1;
  const double* d_wg = d_tabs + P1 + n;
  if (!L.it_cell.empty()) {
    k_nuc_cells<Rad><<<(unsigned)L.it_cell.size(), kNucThreads, 0, st>>>(c.mesh, d_gll, d_xg, d_wg, n, d_cb, d_boxes,
                                                                         d_ic, d_if, d_at, nA, rad, norm, inv2s2, r0,
                                                                         s, d_C, d_G, d_ba, d_dC);
    note_launch();
    ENR_CK(cudaGetLastError(), "cell integrals");
  }
  if (!L.aa_cell.empty()) {
    k_nuc_aa<Rad><<<(unsigned)L.aa_cell.size(), kNucThreads, 0, st>>>(c.mesh, d_xg, d_wg, n, d_cb, d_boxes, d_ac,
                                                                       d_aa, d_ab, d_at, rad, r0, s, nA, d_AA);
    note_launch();
    ENR_CK(cudaGetLastError(), "atomic stiffness");
  }
  const double k4 = 1.0 / (4.0 * kPi), lap = 1.0 / (2.0 * kPi);   // launch_laplace applies lap * (1/2) K
  k_nuc_orth<<<nblk((long long)vecs), 256, 0, st>>>(d_C, c.d_Dsc, n_h, nA);
  note_launch();
  ENR_CK(cudaGetLastError(), "orthogonalisation");
  for (int J = 0; J < nA; ++J)
    ENR_CK(launch_laplace(c, d_C + (size_t)J * n_h, d_LC + (size_t)J * n_h, 1, 1, lap, st), "stiffness");
  double* CG = d_dots;            // [nA][nA] C_J . G_K
  double* CLC = CG + nA * nA;     // [nA][nA] C_J . (k K C_K)
  double* AX = CLC + nA * nA;     // [nA][nA] A_IJ . X_K
  double* CdC = AX + nA * nA;     // [nA]     C_J . d
  auto dots = [&](const double* A, const double* Bv, int na, int nb, double* out) {
    k_nuc_dots<<<(unsigned)(na * nb), kNucThreads, 0, st>>>(A, n_h, Bv, n_h, n_h, nb, out);
    note_launch();
    return cudaGetLastError();
  };
  ENR_CK(dots(d_C, d_G, nA, nA, CG), "dots");
  ENR_CK(dots(d_C, d_LC, nA, nA, CLC), "dots");
  if (d_dC) ENR_CK(dots(d_C, d_dC, nA, 1, CdC), "dots");
  k_nuc_ace<<<nblk((long long)vecs), 256, 0, st>>>(d_G, c.d_Dsc, n_h, nA, k4, d_LC);
  note_launch();
  ENR_CK(cudaGetLastError(), "coupling");
  for (int J = 0; J < nA; ++J)
    ENR_CK(fdm_solve(c, d_LC + (size_t)J * n_h, d_Ap, d_X + (size_t)J * n_h, 1, st, true), "direct solve");
  ENR_CK(dots(d_LC, d_X, nA, nA, AX), "dots");
  std::vector<double> hd((size_t)3 * nA * nA + nA, 0.0), hAA((size_t)nA * nA), hba(nA);
  ENR_CK(cudaMemcpyAsync(hd.data(), d_dots, sizeof(double) * (3 * (size_t)nA * nA + (d_dC ? nA : 0)),
                         cudaMemcpyDeviceToHost, st), "copy");
  ENR_CK(cudaMemcpyAsync(hAA.data(), d_AA, sizeof(double) * hAA.size(), cudaMemcpyDeviceToHost, st), "copy");
  ENR_CK(cudaMemcpyAsync(hba.data(), d_ba, sizeof(double) * nA, cudaMemcpyDeviceToHost, st), "copy");
  ENR_CK(cudaStreamSynchronize(st), "set-up");
  const double* hCG = hd.data();
  const double* hCLC = hCG + nA * nA;
  const double* hAX = hCLC + nA * nA;
  const double* hCdC = hAX + nA * nA;
  S.assign((size_t)nA * nA, 0.0);
  for (int J = 0; J < nA; ++J)
    for (int K = 0; K < nA; ++K) {
      const double aee = k4 * (hAA[J * nA + K] - hCG[K * nA + J] - hCG[J * nA + K]) + hCLC[J * nA + K];
      S[J * nA + K] = aee - hAX[J * nA + K];
    }
  for (int J = 0; J < nA; ++J)
    for (int K = 0; K < J; ++K) S[J * nA + K] = S[K * nA + J] = 0.5 * (S[J * nA + K] + S[K * nA + J]);
  dE.assign(nA, 0.0);
  if (d_dC)
    for (int J = 0; J < nA; ++J) dE[J] = hba[J] - hCdC[J];
  return EFE_OK;
}

// Cholesky factor of the symmetric n x n matrix S (lower, row-major); false if not positive definite.
bool cholesky(const std::vector<double>& S, int n, std::vector<double>& L) {
  L.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      double v = S[i * n + j];
      for (int k = 0; k < j; ++k) v -= L[i * n + k] * L[j * n + k];
      if (i == j) {
        if (!(v > 0.0)) return false;
        L[i * n + i] = std::sqrt(v);
      } else {
        L[i * n + j] = v / L[j * n + j];
      }
    }
  return true;
}

// x = (L L^T)^-1 b
void chol_solve(const std::vector<double>& L, int n, const double* b, double* x) {
  for (int i = 0; i < n; ++i) {
    double v = b[i];
    for (int k = 0; k < i; ++k) v -= L[i * n + k] * x[k];
    x[i] = v / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double v = x[i];
    for (int k = i + 1; k < n; ++k) v -= L[k * n + i] * x[k];
    x[i] = v / L[i * n + i];
  }
}

// ---- radial functions of the wavefunction enrichment (host), for the atomic densities
double laguerre_h(int k, int a, double x) {
  if (k < 0) return 0.0;
  double out = 0.0, fact = 1.0, xp = 1.0;
  for (int i = 0; i <= k; ++i) {
    double binom = 1.0;   // C(k + a, k - i)
    for (int j = 1; j <= k - i; ++j) binom = binom * (a + i + j) / j;
    out += ((i & 1) ? -1.0 : 1.0) * binom * xp / fact;
    xp *= x;
    fact *= (i + 1);
  }
  return out;
}

// R_nl(r) = f(r) r^l for the radial kinds of efe_enrich_fn
double radial_value(int kind, int n, int l, double zeta, double r) {
  double f;
  if (kind == EFE_RADIAL_SLATER) {
    const int p = n - 1 - l;
    f = (p > 0 ? std::pow(r, (double)p) : 1.0) * std::exp(-zeta * r);
  } else if (kind == EFE_RADIAL_HYDROGENIC) {
    f = std::pow(zeta, (double)l) * laguerre_h(n - l - 1, 2 * l + 1, 2.0 * zeta * r / n) * std::exp(-zeta * r / n);
  } else {
    f = std::exp(-zeta * r * r);
  }
  return f * (l > 0 ? std::pow(r, (double)l) : 1.0);
}

// Cumulative integral of y dr on the grid r = rmax t^2 (trapezoid rule in t, dr = 2 rmax t dt).
std::vector<double> cum_t2(const std::vector<double>& y, const std::vector<double>& r) {
  const size_t n = r.size();
  const double rl = r[n - 1];
  std::vector<double> t(n), g(n), out(n, 0.0);
  for (size_t i = 0; i < n; ++i) {
    t[i] = std::sqrt(r[i] / rl);
    g[i] = y[i] * 2.0 * rl * t[i];
  }
  for (size_t i = 1; i < n; ++i) out[i] = out[i - 1] + 0.5 * (g[i] + g[i - 1]) * (t[i] - t[i - 1]);
  return out;
}

// The atomic Hartree potentials (one isolated neutral atom per nucleus): the shells of
// the atom's wavefunction enrichment functions (distinct radial kind, n, l, zeta, in the
// order of n, then l) are filled with Z electrons, two per orbital, in that order;
// rho(r) = sum occ R_nl^2 / (4 pi int R_nl^2 r^2 dr), Q(r) = 4 pi int_0^r rho s^2 ds,
// v(r) = Q(r) / r + 4 pi int_r^inf rho s ds, tabulated on r_i = rmax t_i^2 with t uniform
// on [0, 1] (nt points): rg [nt], V and Q [nA][nt], nel [nA] = Q at the end of the table.
void atom_tables(int nA, const double* Zs, const std::vector<efe_enrich_fn>& fns, int nt, double rmax,
                 std::vector<double>& rg, std::vector<double>& V, std::vector<double>& Q, std::vector<double>& nel) {
  rg.assign(nt, 0.0);
  for (int i = 0; i < nt; ++i) {
    const double t = i == nt - 1 ? 1.0 : i * (1.0 / (nt - 1));
    rg[i] = rmax * t * t;
  }
  V.assign((size_t)nA * nt, 0.0);
  Q.assign((size_t)nA * nt, 0.0);
  nel.assign(nA, 0.0);
  for (int J = 0; J < nA; ++J) {
    struct Shell { int kind, n, l; double zeta; };
    std::vector<Shell> sh;
    for (const efe_enrich_fn& f : fns) {
      if (f.atom != J) continue;
      bool seen = false;
      for (const Shell& x : sh)
        if (x.kind == f.radial && x.n == f.n && x.l == f.l && x.zeta == f.zeta) seen = true;
      if (!seen) sh.push_back(Shell{f.radial, f.n, f.l, f.zeta});
    }
    std::stable_sort(sh.begin(), sh.end(), [](const Shell& a, const Shell& b) {
      return a.n != b.n ? a.n < b.n : a.l < b.l;
    });
    std::vector<double> rho(nt, 0.0), R(nt), y(nt);
    double left = Zs[J];
    for (const Shell& x : sh) {
      const double occ = std::min(left, 2.0 * (2 * x.l + 1));
      if (occ <= 0.0) break;
      for (int i = 0; i < nt; ++i) {
        R[i] = radial_value(x.kind, x.n, x.l, x.zeta, rg[i]);
        y[i] = R[i] * R[i] * rg[i] * rg[i];
      }
      const double nrm = cum_t2(y, rg)[nt - 1];
      for (int i = 0; i < nt; ++i) rho[i] += occ * R[i] * R[i] / (4.0 * kPi * nrm);
      left -= occ;
    }
    for (int i = 0; i < nt; ++i) y[i] = rho[i] * rg[i] * rg[i];
    const std::vector<double> q = cum_t2(y, rg);
    for (int i = 0; i < nt; ++i) y[i] = rho[i] * rg[i];
    const std::vector<double> o = cum_t2(y, rg);
    for (int i = 0; i < nt; ++i) {
      Q[(size_t)J * nt + i] = 4.0 * kPi * q[i];
      const double outer = 4.0 * kPi * (o[nt - 1] - o[i]);
      V[(size_t)J * nt + i] = (rg[i] > 0.0 ? 4.0 * kPi * q[i] / rg[i] : 0.0) + outer;
    }
    V[(size_t)J * nt] = 4.0 * kPi * o[nt - 1];
    nel[J] = Q[(size_t)J * nt + nt - 1];
  }
}

}  // namespace

// ---------------------------------------------------------------------------- nuclear potential
efe_status nuclear_enriched(Ctx& c, double sigma, double r0, double s, int sub, int n_quad, double adapt_tol,
                            int adapt_depth, double* phiE_host, cudaStream_t st) {
  if (!(sigma > 0.0) || !(adapt_tol >= 0.0) || adapt_depth < 0 || adapt_depth > 8) {
    c.err = "nuclear enrichment: need sigma > 0, adapt_tol >= 0, adapt_depth in [0, 8]";
    return EFE_ERR_ARG;
  }
  if (adapt_tol > 0.0) sub = 1;
  if (!enr_args_ok(c, r0, s, sub, n_quad)) return EFE_ERR_ARG;
  const int nA = c.n_atoms;
  std::vector<double> at(4 * (size_t)nA);
  for (int J = 0; J < nA; ++J) {
    at[4 * J] = c.Z[J];
    for (int a = 0; a < 3; ++a) at[4 * J + 1 + a] = c.R[3 * J + a];
  }
  const long long n_h = c.n_h;
  const size_t vecs = (size_t)nA * n_h;
  Bufs B;
  double *d_at, *d_C, *d_G, *d_LC, *d_X, *d_dC, *d_z, *d_Lz, *d_u, *d_Ap, *d_phiB, *d_nodes, *d_dots, *d_xE;
  ENR_CK(B.alloc(d_at, at.size()), "allocating");
  for (double** v : {&d_C, &d_G, &d_LC, &d_X}) ENR_CK(B.alloc(*v, vecs), "allocating");
  for (double** v : {&d_dC, &d_z, &d_Lz, &d_u, &d_Ap, &d_phiB}) ENR_CK(B.alloc(*v, (size_t)n_h), "allocating");
  ENR_CK(B.alloc(d_nodes, (size_t)3 * n_h), "allocating");
  ENR_CK(B.alloc(d_dots, (size_t)2 * nA), "allocating");
  ENR_CK(B.alloc(d_xE, nA), "allocating");
  ENR_CK(cudaMemcpyAsync(d_at, at.data(), sizeof(double) * at.size(), cudaMemcpyHostToDevice, st), "copy");
  const double a = 1.0 / (std::sqrt(2.0) * sigma);
  const double norm = std::pow(2.0 * kPi * sigma * sigma, -1.5);
  const double inv2s2 = 1.0 / (2.0 * sigma * sigma);
  const NucRadial nrad{a};
  Lists L;
  work_lists(c, r0, 40.0 * sigma, L);   // exp(-40^2 / 2) underflows: no charge beyond 40 sigma
  std::vector<double> S, dE;
  const BoxRule rule = adapt_tol > 0.0 ? adaptive_rule(c, L, n_quad, adapt_tol, adapt_depth, sigma, r0, s)
                                       : uniform_rule(c, L, sub, n_quad);
  efe_status e = enr_blocks(c, nrad, d_at, r0, s, rule, norm, inv2s2, L, d_C, d_G, d_LC, d_X,
                            d_dC, S, dE, st);
  if (e != EFE_OK) return e;
  // classical solve with the smeared-nucleus boundary data
  const double k4 = 1.0 / (4.0 * kPi), lap = 1.0 / (2.0 * kPi);
  ENR_CK(launch_coords(c, d_nodes, nullptr, st), "node coordinates");
  k_nuc_bc<<<nblk(n_h), 256, 0, st>>>(d_nodes, c.d_Dsc, n_h, d_at, nA, a, d_phiB);
  note_launch();
  ENR_CK(cudaGetLastError(), "boundary data");
  ENR_CK(fdm_solve(c, d_dC, d_Ap, d_z, 1, st, false, d_phiB), "direct solve");
  ENR_CK(cudaMemsetAsync(d_Lz, 0, sizeof(double) * n_h, st), "clear");
  ENR_CK(launch_laplace(c, d_z, d_Lz, 1, 0, lap, st), "stiffness");
  k_nuc_dots<<<(unsigned)nA, kNucThreads, 0, st>>>(d_G, n_h, d_z, n_h, n_h, 1, d_dots);
  note_launch();
  k_nuc_dots<<<(unsigned)nA, kNucThreads, 0, st>>>(d_C, n_h, d_Lz, n_h, n_h, 1, d_dots + nA);
  note_launch();
  ENR_CK(cudaGetLastError(), "dots");
  std::vector<double> hd(2 * (size_t)nA);
  ENR_CK(cudaMemcpyAsync(hd.data(), d_dots, sizeof(double) * hd.size(), cudaMemcpyDeviceToHost, st), "copy");
  ENR_CK(cudaStreamSynchronize(st), "set-up");
  // S phi^E = d_E - A_EB phi_B - A_EI z on the host
  std::vector<double> rhs(nA), x(nA), Lc;
  for (int J = 0; J < nA; ++J) rhs[J] = dE[J] - k4 * hd[J] + hd[nA + J];
  if (!cholesky(S, nA, Lc)) {
    c.err = "nuclear enrichment: Schur complement not positive definite";
    return EFE_ERR_NOT_SPD;
  }
  chol_solve(Lc, nA, rhs.data(), x.data());
  // v_N at the quadrature points
  ENR_CK(cudaMemcpyAsync(d_xE, x.data(), sizeof(double) * nA, cudaMemcpyHostToDevice, st), "copy");
  k_nuc_combine<<<nblk(n_h), 256, 0, st>>>(d_z, d_X, d_C, d_xE, n_h, nA, d_u);
  note_launch();
  ENR_CK(cudaGetLastError(), "combine");
  ENR_CK(launch_interp(c, d_u, c.d_vN, 1, st), "interpolation");
  const long long npts = (long long)c.nc * c.nq;
  k_nuc_add_atomic<<<nblk(npts), 256, 0, st>>>(c.d_xq, npts, d_at, nA, nrad, r0, s, d_xE, c.d_vN);
  note_launch();
  ENR_CK(cudaGetLastError(), "enrichment values");
  ENR_CK(cudaStreamSynchronize(st), "set-up");
  if (phiE_host)
    for (int J = 0; J < nA; ++J) phiE_host[J] = x[J];
  c.state_valid = false;
  c.has_prev = false;
  return EFE_OK;
}

// ---------------------------------------------------------------------------- Hartree potential
void hen_free(HartreeEnr& h) {
  for (double** p : {&h.C, &h.G, &h.X, &h.Sinv, &h.atoms, &h.r, &h.v, &h.q, &h.nel, &h.small}) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  for (int** p : {&h.pair_cell, &h.pair_fn}) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  h.on = false;
}

// Installs the enriched Hartree solve: atomic tables, the enrichment blocks and the
// inverse of the eliminated block.
efe_status hartree_enrich_install(Ctx& c, double r0, double s, int sub, int n_quad, cudaStream_t st) {
  if (c.hartree_method != EFE_HARTREE_FDM) {
    c.err = "enriched Hartree solve: needs the direct (fast-diagonalisation) Hartree method";
    return EFE_ERR_ARG;
  }
  if (!enr_args_ok(c, r0, s, sub, n_quad)) return EFE_ERR_ARG;
  const int nA = c.n_atoms, nt = 24001;
  const double rmax = 60.0;
  std::vector<double> rg, V, Q, nel;
  atom_tables(nA, c.Z.data(), c.fns, nt, rmax, rg, V, Q, nel);
  hen_free(c.hen);
  HartreeEnr& h = c.hen;
  h.nA = nA;
  h.n_tab = nt;
  h.rmax = rmax;
  h.r0 = r0;
  h.s = s;
  std::vector<double> at(4 * (size_t)nA);
  for (int J = 0; J < nA; ++J) {
    at[4 * J] = c.Z[J];
    for (int a = 0; a < 3; ++a) at[4 * J + 1 + a] = c.R[3 * J + a];
  }
  const long long n_h = c.n_h;
  const size_t vecs = (size_t)nA * n_h;
  auto dal = [](double*& p, size_t n) { return cudaMalloc(&p, sizeof(double) * std::max<size_t>(n, 1)); };
  ENR_CK(dal(h.C, vecs), "allocating");
  ENR_CK(dal(h.G, vecs), "allocating");
  ENR_CK(dal(h.X, vecs), "allocating");
  ENR_CK(dal(h.Sinv, (size_t)nA * nA), "allocating");
  ENR_CK(dal(h.atoms, at.size()), "allocating");
  ENR_CK(dal(h.r, nt), "allocating");
  ENR_CK(dal(h.v, V.size()), "allocating");
  ENR_CK(dal(h.q, Q.size()), "allocating");
  ENR_CK(dal(h.nel, nA), "allocating");
  ENR_CK(dal(h.small, (size_t)6 * nA * c.batch), "allocating");
  ENR_CK(cudaMemcpyAsync(h.atoms, at.data(), sizeof(double) * at.size(), cudaMemcpyHostToDevice, st), "copy");
  ENR_CK(cudaMemcpyAsync(h.r, rg.data(), sizeof(double) * nt, cudaMemcpyHostToDevice, st), "copy");
  ENR_CK(cudaMemcpyAsync(h.v, V.data(), sizeof(double) * V.size(), cudaMemcpyHostToDevice, st), "copy");
  ENR_CK(cudaMemcpyAsync(h.q, Q.data(), sizeof(double) * Q.size(), cudaMemcpyHostToDevice, st), "copy");
  ENR_CK(cudaMemcpyAsync(h.nel, nel.data(), sizeof(double) * nA, cudaMemcpyHostToDevice, st), "copy");
  const TabRadial trad{h.r, h.v, h.q, h.nel, nt, rmax};
  Lists L;
  work_lists(c, r0, 0.0, L);
  Bufs B;
  double* d_LC;
  ENR_CK(B.alloc(d_LC, vecs), "allocating");
  std::vector<double> S, dE;
  const BoxRule rule = uniform_rule(c, L, sub, n_quad);
  efe_status e = enr_blocks(c, trad, h.atoms, r0, s, rule, 0.0, 0.0, L, h.C, h.G, d_LC, h.X, nullptr,
                            S, dE, st);
  if (e != EFE_OK) return e;
  std::vector<double> Lc, Sinv((size_t)nA * nA), col(nA), x(nA);
  if (!cholesky(S, nA, Lc)) {
    c.err = "enriched Hartree solve: Schur complement not positive definite";
    return EFE_ERR_NOT_SPD;
  }
  for (int K = 0; K < nA; ++K) {
    std::fill(col.begin(), col.end(), 0.0);
    col[K] = 1.0;
    chol_solve(Lc, nA, col.data(), x.data());
    for (int J = 0; J < nA; ++J) Sinv[J * nA + K] = x[J];
  }
  ENR_CK(cudaMemcpyAsync(h.Sinv, Sinv.data(), sizeof(double) * Sinv.size(), cudaMemcpyHostToDevice, st), "copy");
  h.n_pairs = (long long)L.pr_cell.size();
  ENR_CK(cudaMalloc(&h.pair_cell, sizeof(int) * std::max<size_t>(L.pr_cell.size(), 1)), "allocating");
  ENR_CK(cudaMalloc(&h.pair_fn, sizeof(int) * std::max<size_t>(L.pr_fn.size(), 1)), "allocating");
  ENR_CK(cudaMemcpyAsync(h.pair_cell, L.pr_cell.data(), sizeof(int) * L.pr_cell.size(), cudaMemcpyHostToDevice, st),
         "copy");
  ENR_CK(cudaMemcpyAsync(h.pair_fn, L.pr_fn.data(), sizeof(int) * L.pr_fn.size(), cudaMemcpyHostToDevice, st), "copy");
  ENR_CK(cudaStreamSynchronize(st), "set-up");
  h.on = true;
  c.state_valid = false;
  c.has_prev = false;
  return EFE_OK;
}

cudaError_t hartree_enriched_solve(Ctx& c, const double* rho, double* vH, const double* d, double* Ap, double* Lz,
                                   double* u, cudaStream_t s) {
  HartreeEnr& h = c.hen;
  const int nb = c.batch, nA = h.nA;
  const long long n_h = c.n_h, N = n_h * nb;
  const double k4 = 1.0 / (4.0 * kPi), lap = 1.0 / (2.0 * kPi);
  const TabRadial trad{h.r, h.v, h.q, h.nel, h.n_tab, h.rmax};
  double* dA = h.small;
  double* rhs = dA + nA * nb;
  double* xE = rhs + nA * nb;
  EFE_CUDA_TRY(fdm_solve(c, d, Ap, c.d_phi, nb, s));   // z, with the Hartree Dirichlet data
  EFE_CUDA_TRY(cudaMemsetAsync(Lz, 0, sizeof(double) * N, s));
  EFE_CUDA_TRY(launch_laplace(c, c.d_phi, Lz, nb, 0, lap, s));
  EFE_CUDA_TRY(cudaMemsetAsync(dA, 0, sizeof(double) * nA * nb, s));
  if (h.n_pairs > 0) {
    k_hen_load<TabRadial><<<(unsigned)h.n_pairs, kNucThreads, 0, s>>>(h.pair_cell, h.pair_fn, c.nq, c.nc, nb, c.d_xq,
                                                                      c.d_wJ, rho, h.atoms, trad, h.r0, h.s, dA);
    note_launch();
  }
  double* sums = h.small + 3 * nA * nb;   // [3][nA][nb]
  EFE_CUDA_TRY(cudaMemsetAsync(sums, 0, sizeof(double) * 3 * nA * nb, s));
  k_hen_dots<<<dim3((unsigned)(nA * nb), 64), kNucThreads, 0, s>>>(h.C, h.G, d, c.d_phi, Lz, n_h, nb, nA * nb, sums);
  note_launch();
  k_hen_rhs<<<1, 256, 0, s>>>(dA, sums, nA * nb, k4, rhs);
  note_launch();
  k_hen_coef<<<1, 256, 0, s>>>(h.Sinv, rhs, nA, nb, xE);
  note_launch();
  k_hen_combine<<<nblk(N), 256, 0, s>>>(c.d_phi, u, h.X, h.C, xE, n_h, nA, nb);
  note_launch();
  EFE_CUDA_TRY(cudaGetLastError());
  EFE_CUDA_TRY(launch_interp(c, u, vH, nb, s));
  const long long npts = (long long)c.nc * c.nq;
  k_hen_add<TabRadial><<<nblk(npts * nb), 256, 0, s>>>(c.d_xq, npts, nb, h.atoms, nA, trad, h.r0, h.s, xE, vH);
  note_launch();
  return cudaGetLastError();
}

// The transpose of the enriched Hartree map rho -> v_H (batch 1), as the adjoint
// needs it.  With d = L rho (load), z = Z d (homogeneous direct solve),
// d_E = A rho (enrichment loads), rhs = A rho - W L rho with
// W d = C d + k G (Z d) - C (k K Z d), phi^E = Sinv rhs and
// v_H = I (z - (X + C)^T phi^E) + N^T phi^E (I: interpolation, N: atomic values),
//   v_H^T g = L^T (Z h - W^T t) + A^T t,   h = I^T g,   t = Sinv (N g - (X + C) h),
//   W^T t = C^T t + Z (k G^T t - k K C^T t),   L^T = w I,   (A^T t)_q = w_q sum_J t_J N^A_J(q).
// gw: g / w at the quadrature points (input); out: I (Z h - W^T t) + sum_J t_J N^A_J, to be
// multiplied by w by the caller (may alias gw); s1..s6: [n_h] scratch.
cudaError_t hartree_enriched_vt(Ctx& c, const double* gw, double* out, double* s1, double* s2, double* s3, double* s4,
                                double* s5, double* s6, cudaStream_t s) {
  HartreeEnr& h = c.hen;
  const int nA = h.nA;
  const long long n_h = c.n_h;
  const double k4 = 1.0 / (4.0 * kPi), lap = 1.0 / (2.0 * kPi);
  const TabRadial trad{h.r, h.v, h.q, h.nel, h.n_tab, h.rmax};
  double* sN = h.small;
  double* sX = sN + nA;
  double* t = sX + nA;
  // h = I^T g = load(g / w);  Zh
  EFE_CUDA_TRY(cudaMemsetAsync(s1, 0, sizeof(double) * n_h, s));
  EFE_CUDA_TRY(launch_load_vector(c, gw, s1, 1, s));
  EFE_CUDA_TRY(fdm_solve(c, s1, s2, s3, 1, s, true));
  // N g (the enrichment loads of g / w) and (X + C) . h, then t
  EFE_CUDA_TRY(cudaMemsetAsync(sN, 0, sizeof(double) * nA, s));
  if (h.n_pairs > 0) {
    k_hen_load<TabRadial><<<(unsigned)h.n_pairs, kNucThreads, 0, s>>>(h.pair_cell, h.pair_fn, c.nq, c.nc, 1, c.d_xq,
                                                                      c.d_wJ, gw, h.atoms, trad, h.r0, h.s, sN);
    note_launch();
  }
  k_hen_xc_dot<<<(unsigned)nA, kNucThreads, 0, s>>>(h.X, h.C, s1, n_h, sX);
  note_launch();
  k_hen_tcoef<<<1, 256, 0, s>>>(h.Sinv, sN, sX, nA, t);
  note_launch();
  // W^T t = ct + Z (k gt - k K ct)
  k_hen_comb_t<<<nblk(n_h), 256, 0, s>>>(h.C, h.G, t, n_h, nA, s4, s5);
  note_launch();
  EFE_CUDA_TRY(cudaMemsetAsync(s6, 0, sizeof(double) * n_h, s));
  EFE_CUDA_TRY(launch_laplace(c, s4, s6, 1, 1, lap, s));
  k_hen_rvec<<<nblk(n_h), 256, 0, s>>>(s5, s6, c.d_Dsc, n_h, k4);
  note_launch();
  EFE_CUDA_TRY(cudaGetLastError());
  EFE_CUDA_TRY(fdm_solve(c, s5, s2, s6, 1, s, true));
  // y = Zh - W^T t, then out = I y + sum_J t_J N^A_J
  k_hen_yvec<<<nblk(n_h), 256, 0, s>>>(s3, s4, s6, n_h, s1);
  note_launch();
  EFE_CUDA_TRY(cudaGetLastError());
  EFE_CUDA_TRY(launch_interp(c, s1, out, 1, s));
  const long long npts = (long long)c.nc * c.nq;
  k_hen_add<TabRadial><<<nblk(npts), 256, 0, s>>>(c.d_xq, npts, 1, h.atoms, nA, trad, h.r0, h.s, t, out);
  note_launch();
  return cudaGetLastError();
}

#undef ENR_CK

}  // namespace efe

// ---------------------------------------------------------------------------- host-only diagnostics
extern "C" {

efe_status efe_atom_hartree_table(const efe_enrich_fn* fns_host, int32_t n_fn, const double* Z_host, int32_t n_atoms,
                                  int32_t n_tab, double rmax, double* r_host, double* v_host, double* q_host,
                                  double* nel_host) {
  if (!Z_host || n_atoms < 1 || n_fn < 0 || (n_fn > 0 && !fns_host) || n_tab < 2 || !(rmax > 0.0)) return EFE_ERR_ARG;
  for (int i = 0; i < n_fn; ++i)
    if (fns_host[i].atom < 0 || fns_host[i].atom >= n_atoms) return EFE_ERR_ARG;
  std::vector<efe_enrich_fn> fns(fns_host, fns_host + n_fn);
  std::vector<double> rg, V, Q, nel;
  efe::atom_tables(n_atoms, Z_host, fns, n_tab, rmax, rg, V, Q, nel);
  if (r_host) std::copy(rg.begin(), rg.end(), r_host);
  if (v_host) std::copy(V.begin(), V.end(), v_host);
  if (q_host) std::copy(Q.begin(), Q.end(), q_host);
  if (nel_host) std::copy(nel.begin(), nel.end(), nel_host);
  return EFE_OK;
}

efe_status efe_adaptive_cell_boxes(const double* origin_host, const double* size_host, const double* atoms_host,
                                   int32_t n_atoms, double sigma, double r0, double s, int32_t n_quad, double tol,
                                   int32_t max_depth, int64_t* n_boxes, double* boxes_host, int64_t capacity) {
  if (!origin_host || !size_host || (n_atoms > 0 && !atoms_host) || n_atoms < 0 || !(sigma > 0.0) || !(s > 0.0) ||
      !(r0 > s) || n_quad < 1 || n_quad > 8 || !(tol > 0.0) || max_depth < 0 || max_depth > 8 || !n_boxes)
    return EFE_ERR_ARG;
  std::vector<double> R(3 * (size_t)n_atoms), Z(n_atoms);
  for (int J = 0; J < n_atoms; ++J) {
    Z[J] = atoms_host[4 * J];
    for (int a = 0; a < 3; ++a) R[3 * J + a] = atoms_host[4 * J + 1 + a];
  }
  std::vector<double> xg(n_quad), wg(n_quad), out;
  efe::gauss_legendre(n_quad, xg.data(), wg.data());
  efe::adaptive_cell(origin_host, size_host, R.data(), Z.data(), n_atoms, sigma, r0, s, xg, wg, tol, max_depth, out);
  *n_boxes = (int64_t)(out.size() / 6);
  if (boxes_host) {
    if (capacity < *n_boxes) return EFE_ERR_ARG;
    std::copy(out.begin(), out.end(), boxes_host);
  }
  return EFE_OK;
}

}  // extern "C"
