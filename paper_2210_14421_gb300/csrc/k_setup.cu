// Set-up kernels: quadrature geometry, nuclear potential, enrichment functions
// and their orthogonalisation (Eqs. EFEAtomic, EFEOrtho, M, MSquareRoot), the
// v-independent coupling blocks, Dirichlet data of the Hartree problem.
// These run once per context; they favour plain loops over speed.
#include <cmath>

#include "efe_internal.h"
#include "radial.cuh"

namespace efe {

struct EnrDev {
  int atom, n, l, m, radial;
  double zeta;
  double cx, cy, cz;
};

// Quadrature points, weights w_q |J| and v_N = -sum Z / |x - R| (Eq. VN).
__global__ void k_geometry(const __grid_constant__ RefTables tab, const MeshView mesh, int NQ1,
                           const double* __restrict__ atoms /* [n][4] Z,x,y,z */, int n_atoms,
                           double* __restrict__ xq, double* __restrict__ wJ, double* __restrict__ vN) {
  const int nq = NQ1 * NQ1 * NQ1;
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)mesh.nc * nq) return;
  const int c = (int)(idx / nq), q = (int)(idx % nq);
  int cx, cy, cz;
  cell_ijk(mesh, c, cx, cy, cz);
  const int q1 = q % NQ1, q2 = (q / NQ1) % NQ1, q3 = q / (NQ1 * NQ1);
  const double hx = mesh.h[cx], hy = mesh.h[mesh.ncx + cy], hz = mesh.h[mesh.ncx + mesh.ncy + cz];
  const double x = mesh.x0[cx] + 0.5 * (tab.xg[q1] + 1.0) * hx;
  const double y = mesh.x0[mesh.ncx + cy] + 0.5 * (tab.xg[q2] + 1.0) * hy;
  const double z = mesh.x0[mesh.ncx + mesh.ncy + cz] + 0.5 * (tab.xg[q3] + 1.0) * hz;
  xq[idx * 3 + 0] = x;
  xq[idx * 3 + 1] = y;
  xq[idx * 3 + 2] = z;
  wJ[idx] = tab.wg[q1] * tab.wg[q2] * tab.wg[q3] * hx * hy * hz / 8.0;
  double v = 0.0;
  for (int a = 0; a < n_atoms; ++a) {
    const double dx = x - atoms[4 * a + 1], dy = y - atoms[4 * a + 2], dz = z - atoms[4 * a + 3];
    v -= atoms[4 * a] / sqrt(dx * dx + dy * dy + dz * dz);
  }
  vN[idx] = v;
}

// generalised Laguerre polynomial L_k^(a)(x) by its explicit sum
__device__ double laguerre(int k, int a, double x) {
  if (k < 0) return 0.0;
  double out = 0.0, fact = 1.0, xp = 1.0;
  for (int i = 0; i <= k; ++i) {
    // C(k + a, k - i)
    double binom = 1.0;
    for (int j = 1; j <= k - i; ++j) binom = binom * (a + i + j) / j;
    out += ((i & 1) ? -1.0 : 1.0) * binom * xp / fact;
    xp *= x;
    fact *= (i + 1);
  }
  return out;
}

// f(r) = R_nl / r^l and df/dr
__device__ void radial_fn(const EnrDev& e, double r, double& f, double& df) {
  if (e.radial == EFE_RADIAL_SLATER) {
    const int p = e.n - 1 - e.l;
    const double ex = exp(-e.zeta * r);
    const double rp = p > 0 ? pow(r, (double)p) : 1.0;
    f = rp * ex;
    df = (p > 0 ? p * pow(r, (double)(p - 1)) : 0.0) * ex - e.zeta * f;
  } else if (e.radial == EFE_RADIAL_HYDROGENIC) {
    const int k = e.n - e.l - 1;
    const double x = 2.0 * e.zeta * r / e.n;
    const double L = laguerre(k, 2 * e.l + 1, x);
    const double dL = k >= 1 ? -laguerre(k - 1, 2 * e.l + 2, x) : 0.0;
    const double ex = exp(-e.zeta * r / e.n);
    const double zl = pow(e.zeta, (double)e.l);
    f = zl * L * ex;
    df = zl * (dL * (2.0 * e.zeta / e.n) - (e.zeta / e.n) * L) * ex;
  } else {
    f = exp(-e.zeta * r * r);
    df = -2.0 * e.zeta * r * f;
  }
}

// real solid harmonic S_lm(d) and gradient
__device__ void solid(int l, int m, double x, double y, double z, double& S, double g[3]) {
  g[0] = g[1] = g[2] = 0.0;
  if (l == 0) { S = 1.0; return; }
  if (l == 1) {
    if (m == -1) { S = y; g[1] = 1.0; }
    else if (m == 0) { S = z; g[2] = 1.0; }
    else { S = x; g[0] = 1.0; }
    return;
  }
  if (m == -2) { S = x * y; g[0] = y; g[1] = x; }
  else if (m == -1) { S = y * z; g[1] = z; g[2] = y; }
  else if (m == 0) { S = 2 * z * z - x * x - y * y; g[0] = -2 * x; g[1] = -2 * y; g[2] = 4 * z; }
  else if (m == 1) { S = x * z; g[0] = z; g[2] = x; }
  else { S = x * x - y * y; g[0] = 2 * x; g[1] = -2 * y; }
}

// values and gradients of N^A for every (pair, q)
__global__ void k_enr_eval(const int* __restrict__ pair_cell, const int* __restrict__ pair_fn, long long n_pairs,
                           int nq, const double* __restrict__ xq, const EnrDev* __restrict__ fns, double r0,
                           double s, double* __restrict__ Aval, double* __restrict__ Agrad) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n_pairs * nq) return;
  const long long k = idx / nq;
  const int q = (int)(idx % nq);
  const EnrDev e = fns[pair_fn[k]];
  const double* x = xq + ((long long)pair_cell[k] * nq + q) * 3;
  const double dx = x[0] - e.cx, dy = x[1] - e.cy, dz = x[2] - e.cz;
  const double r = sqrt(dx * dx + dy * dy + dz * dz);
  double f, df, S, gS[3], u, du;
  radial_fn(e, r, f, df);
  solid(e.l, e.m, dx, dy, dz, S, gS);
  cutoff(r, r0, s, u, du);
  Aval[idx] = f * S * u;
  const double rad = (df * u + f * du) * S;
  const double inv = r > 0.0 ? 1.0 / r : 0.0;
  Agrad[idx * 3 + 0] = rad * dx * inv + f * u * gS[0];
  Agrad[idx * 3 + 1] = rad * dy * inv + f * u * gS[1];
  Agrad[idx * 3 + 2] = rad * dz * inv + f * u * gS[2];
}

__device__ __forceinline__ double basis_val(const RefTables& t, int P1, int q1, int q2, int q3, int i1, int i2, int i3) {
  return t.B1[q1 * P1 + i1] * t.B1[q2 * P1 + i2] * t.B1[q3 * P1 + i3];
}

// b[fn][g] += sum_q N_l(x_q) w_q |J| A(x_q)   (one thread per (pair, local node))
__global__ void k_enr_b(const __grid_constant__ RefTables tab, const MeshView mesh, int NQ1,
                        const int* __restrict__ pair_cell, const int* __restrict__ pair_fn, long long n_pairs,
                        const double* __restrict__ wJ, const double* __restrict__ Aval, double* __restrict__ bmat) {
  const int P1 = mesh.p + 1, nn = P1 * P1 * P1, nq = NQ1 * NQ1 * NQ1;
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n_pairs * nn) return;
  const long long k = idx / nn;
  const int l = (int)(idx % nn);
  const int c = pair_cell[k];
  const int i1 = l % P1, i2 = (l / P1) % P1, i3 = l / (P1 * P1);
  double acc = 0.0;
  for (int q = 0; q < nq; ++q) {
    const int q1 = q % NQ1, q2 = (q / NQ1) % NQ1, q3 = q / (NQ1 * NQ1);
    acc += basis_val(tab, P1, q1, q2, q3, i1, i2, i3) * wJ[(long long)c * nq + q] * Aval[k * nq + q];
  }
  int cx, cy, cz;
  cell_ijk(mesh, c, cx, cy, cz);
  const long long g = node_index(mesh, cx, cy, cz, i1, i2, i3);
  atomicAdd(&bmat[(long long)pair_fn[k] * mesh.n_h + g], acc);
}

// c = b / M on interior nodes (1/M = D^2 with D = mask / sqrt(M)), 0 on the boundary
// where no classical function exists.
__global__ void k_enr_c2(const double* __restrict__ bmat, const double* __restrict__ Dsc, double* __restrict__ cmat,
                         long long n_h, int nE) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n_h * nE) return;
  const long long g = idx % n_h;
  cmat[idx] = bmat[idx] * Dsc[g] * Dsc[g];
}

// Orthogonalised values Atil = A - sum_l c_l N_l and gradients at the pair's
// quadrature points, and KE[l] = 1/2 sum_q w|J| grad N_l . grad Atil.
// One block per pair.
__global__ void k_enr_orth(const __grid_constant__ RefTables tab, const MeshView mesh, int NQ1,
                           const int* __restrict__ pair_cell, const int* __restrict__ pair_fn, long long n_pairs,
                           const double* __restrict__ wJ, const double* __restrict__ cmat,
                           const double* __restrict__ Aval, double* __restrict__ Agrad /* in: grad A, out: grad Atil */,
                           double* __restrict__ Atil, double* __restrict__ KE) {
  extern __shared__ double sh[];
  const int P1 = mesh.p + 1, nn = P1 * P1 * P1, nq = NQ1 * NQ1 * NQ1;
  double* cl = sh;            // nn
  double* gt = sh + nn;       // nq * 3 (w|J| grad Atil)
  const long long k = blockIdx.x;
  const int c = pair_cell[k];
  int cx, cy, cz;
  cell_ijk(mesh, c, cx, cy, cz);
  const double hx = mesh.h[cx], hy = mesh.h[mesh.ncx + cy], hz = mesh.h[mesh.ncx + mesh.ncy + cz];
  const double sc[3] = {2.0 / hx, 2.0 / hy, 2.0 / hz};
  for (int l = threadIdx.x; l < nn; l += blockDim.x) {
    const int i1 = l % P1, i2 = (l / P1) % P1, i3 = l / (P1 * P1);
    cl[l] = cmat[(long long)pair_fn[k] * mesh.n_h + node_index(mesh, cx, cy, cz, i1, i2, i3)];
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    const int q1 = q % NQ1, q2 = (q / NQ1) % NQ1, q3 = q / (NQ1 * NQ1);
    double v = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
    for (int l = 0; l < nn; ++l) {
      const int i1 = l % P1, i2 = (l / P1) % P1, i3 = l / (P1 * P1);
      const double b1 = tab.B1[q1 * P1 + i1], b2 = tab.B1[q2 * P1 + i2], b3 = tab.B1[q3 * P1 + i3];
      const double d1 = tab.D1[q1 * P1 + i1], d2 = tab.D1[q2 * P1 + i2], d3 = tab.D1[q3 * P1 + i3];
      v += b1 * b2 * b3 * cl[l];
      g0 += d1 * b2 * b3 * cl[l];
      g1 += b1 * d2 * b3 * cl[l];
      g2 += b1 * b2 * d3 * cl[l];
    }
    const long long o = k * nq + q;
    Atil[o] = Aval[o] - v;
    const double a0 = Agrad[o * 3 + 0] - sc[0] * g0;
    const double a1 = Agrad[o * 3 + 1] - sc[1] * g1;
    const double a2 = Agrad[o * 3 + 2] - sc[2] * g2;
    Agrad[o * 3 + 0] = a0;
    Agrad[o * 3 + 1] = a1;
    Agrad[o * 3 + 2] = a2;
    const double w = wJ[(long long)c * nq + q];
    gt[q * 3 + 0] = w * a0;
    gt[q * 3 + 1] = w * a1;
    gt[q * 3 + 2] = w * a2;
  }
  __syncthreads();
  for (int l = threadIdx.x; l < nn; l += blockDim.x) {
    const int i1 = l % P1, i2 = (l / P1) % P1, i3 = l / (P1 * P1);
    double acc = 0.0;
    for (int q = 0; q < nq; ++q) {
      const int q1 = q % NQ1, q2 = (q / NQ1) % NQ1, q3 = q / (NQ1 * NQ1);
      const double b1 = tab.B1[q1 * P1 + i1], b2 = tab.B1[q2 * P1 + i2], b3 = tab.B1[q3 * P1 + i3];
      const double d1 = tab.D1[q1 * P1 + i1], d2 = tab.D1[q2 * P1 + i2], d3 = tab.D1[q3 * P1 + i3];
      acc += sc[0] * d1 * b2 * b3 * gt[q * 3 + 0] + sc[1] * b1 * d2 * b3 * gt[q * 3 + 1] +
             sc[2] * b1 * b2 * d3 * gt[q * 3 + 2];
    }
    KE[k * nn + l] = 0.5 * acc;
  }
}

// per cell: MAA[mu][nu] += sum_q w A_mu A_nu (raw atomic parts),
//           KEE[mu][nu] += 1/2 sum_q w grad Atil_mu . grad Atil_nu
__global__ void k_enr_gram(const int* __restrict__ pair_start, const int* __restrict__ pair_fn, int nq, int nE,
                           const double* __restrict__ wJ, const double* __restrict__ Aval,
                           const double* __restrict__ Ggrad, double* __restrict__ MAA, double* __restrict__ KEE) {
  const int c = blockIdx.x;
  const int p0 = pair_start[c], np = pair_start[c + 1] - p0;
  for (int it = threadIdx.x; it < np * np; it += blockDim.x) {
    const int a = it / np, b = it % np;
    if (b < a) continue;
    const long long ka = p0 + a, kb = p0 + b;
    double m = 0.0, kk = 0.0;
    for (int q = 0; q < nq; ++q) {
      const double w = wJ[(long long)c * nq + q];
      m += w * Aval[ka * nq + q] * Aval[kb * nq + q];
      kk += w * (Ggrad[(ka * nq + q) * 3] * Ggrad[(kb * nq + q) * 3] +
                 Ggrad[(ka * nq + q) * 3 + 1] * Ggrad[(kb * nq + q) * 3 + 1] +
                 Ggrad[(ka * nq + q) * 3 + 2] * Ggrad[(kb * nq + q) * 3 + 2]);
    }
    kk *= 0.5;
    const int ia = pair_fn[ka], ib = pair_fn[kb];
    atomicAdd(&MAA[ia * nE + ib], m);
    atomicAdd(&KEE[ia * nE + ib], kk);
    if (ia != ib) {
      atomicAdd(&MAA[ib * nE + ia], m);
      atomicAdd(&KEE[ib * nE + ia], kk);
    }
  }
}

// Mee[mu][nu] = MAA[mu][nu] - sum_i b[mu][i] b[nu][i] / M_i   (interior i);  one block per (mu, nu)
__global__ void k_mee(const double* __restrict__ bmat, const double* __restrict__ Dsc, long long n_h, int nE,
                      const double* __restrict__ MAA, double* __restrict__ Mee) {
  const int mu = blockIdx.x / nE, nu = blockIdx.x % nE;
  if (nu < mu) return;
  __shared__ double red[kThreads];
  double acc = 0.0;
  const double* bm = bmat + (long long)mu * n_h;
  const double* bn = bmat + (long long)nu * n_h;
  for (long long i = threadIdx.x; i < n_h; i += blockDim.x) {
    const double d = Dsc[i];
    acc += bm[i] * bn[i] * d * d;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double v = MAA[mu * nE + nu] - red[0];
    Mee[mu * nE + nu] = v;
    Mee[nu * nE + mu] = v;
  }
}

// ---------------------------------------------------------------------------- Poisson data
// diag of (scale) * (1/2 int grad N . grad N) per node; boundary nodes get 1.
__global__ void k_laplace_diag(const __grid_constant__ RefTables tab, const MeshView mesh, double scale,
                               double* __restrict__ diag) {
  const int P1 = mesh.p + 1, nn = P1 * P1 * P1;
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)mesh.nc * nn) return;
  const int c = (int)(idx / nn), l = (int)(idx % nn);
  int cx, cy, cz;
  cell_ijk(mesh, c, cx, cy, cz);
  const double hx = mesh.h[cx], hy = mesh.h[mesh.ncx + cy], hz = mesh.h[mesh.ncx + mesh.ncy + cz];
  const int i1 = l % P1, i2 = (l / P1) % P1, i3 = l / (P1 * P1);
  const double K1a = tab.K1[i1 * P1 + i1], K1b = tab.K1[i2 * P1 + i2], K1c = tab.K1[i3 * P1 + i3];
  const double M1a = tab.M1[i1 * P1 + i1], M1b = tab.M1[i2 * P1 + i2], M1c = tab.M1[i3 * P1 + i3];
  const double v = scale * (hy * hz / (4.0 * hx) * K1a * M1b * M1c + hx * hz / (4.0 * hy) * M1a * K1b * M1c +
                            hx * hy / (4.0 * hz) * M1a * M1b * K1c);
  atomicAdd(&diag[node_index(mesh, cx, cy, cz, i1, i2, i3)], v);
}

__global__ void k_poisson_bc(const MeshView mesh, const double* __restrict__ nodes, const double* __restrict__ Dsc,
                             const double* __restrict__ atoms, int n_atoms, double* __restrict__ phiB,
                             double* __restrict__ diag) {
  long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= mesh.n_h) return;
  if (Dsc[g] != 0.0) { phiB[g] = 0.0; return; }
  double v = 0.0;
  for (int a = 0; a < n_atoms; ++a) {
    const double dx = nodes[g * 3] - atoms[4 * a + 1], dy = nodes[g * 3 + 1] - atoms[4 * a + 2],
                 dz = nodes[g * 3 + 2] - atoms[4 * a + 3];
    v += atoms[4 * a] / sqrt(dx * dx + dy * dy + dz * dz);
  }
  phiB[g] = v;
  diag[g] = 1.0;
}

__global__ void k_node_coords(const __grid_constant__ RefTables tab, const MeshView mesh, const double* __restrict__ xi,
                              double* __restrict__ out) {
  long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= mesh.n_h) return;
  const long long ix = g % mesh.Nx, iy = (g / mesh.Nx) % mesh.Ny, iz = g / ((long long)mesh.Nx * mesh.Ny);
  const long long id[3] = {ix, iy, iz};
  const int off[3] = {0, mesh.ncx, mesh.ncx + mesh.ncy};
  const int nca[3] = {mesh.ncx, mesh.ncy, mesh.ncz};
  for (int a = 0; a < 3; ++a) {
    int cell = (int)(id[a] / mesh.p), loc = (int)(id[a] % mesh.p);
    if (cell == nca[a]) { cell -= 1; loc = mesh.p; }
    out[g * 3 + a] = mesh.x0[off[a] + cell] + 0.5 * (xi[loc] + 1.0) * mesh.h[off[a] + cell];
  }
}

// psi_bar^C_i = sqrt(M_i) sum_g coef exp(-a |x_i - c|^2) on interior nodes, replicated per member
__global__ void k_init_orb(const double* __restrict__ nodes, const double* __restrict__ Dsc, long long n_h, int n_orb,
                           int batch, int G, const double* __restrict__ centers, const double* __restrict__ expo,
                           const double* __restrict__ coef, double* __restrict__ psi, long long ld2) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n_h * n_orb) return;
  const long long g = idx / n_orb;
  const int a = (int)(idx % n_orb);
  double re = 0.0, im = 0.0;
  const double d = Dsc[g];
  if (d != 0.0) {
    for (int k = 0; k < G; ++k) {
      const double* cc = centers + ((long long)a * G + k) * 3;
      const double dx = nodes[g * 3] - cc[0], dy = nodes[g * 3 + 1] - cc[1], dz = nodes[g * 3 + 2] - cc[2];
      const double e = exp(-expo[a * G + k] * (dx * dx + dy * dy + dz * dz));
      re += coef[2 * (a * G + k)] * e;
      im += coef[2 * (a * G + k) + 1] * e;
    }
    re /= d;
    im /= d;
  }
  for (int b = 0; b < batch; ++b) {
    psi[g * ld2 + 2 * (b * n_orb + a)] = re;
    psi[g * ld2 + 2 * (b * n_orb + a) + 1] = im;
  }
}

__global__ void k_init_enr(const double* __restrict__ Shalf, const double* __restrict__ enr, long long n_h, int nE,
                           int n_orb, int batch, double* __restrict__ psi, long long ld2) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)nE * n_orb) return;
  const int nu = (int)(idx / n_orb), a = (int)(idx % n_orb);
  double re = 0.0, im = 0.0;
  for (int mu = 0; mu < nE; ++mu) {
    re += Shalf[nu * nE + mu] * enr[2 * (a * nE + mu)];
    im += Shalf[nu * nE + mu] * enr[2 * (a * nE + mu) + 1];
  }
  for (int b = 0; b < batch; ++b) {
    psi[(n_h + nu) * ld2 + 2 * (b * n_orb + a)] = re;
    psi[(n_h + nu) * ld2 + 2 * (b * n_orb + a) + 1] = im;
  }
}

// ---------------------------------------------------------------------------- host wrappers
static unsigned nblk(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_geometry(const Ctx& c, cudaStream_t s) {
  std::vector<double> at(4 * (size_t)c.n_atoms);
  for (int a = 0; a < c.n_atoms; ++a) {
    at[4 * a] = c.Z[a];
    at[4 * a + 1] = c.R[3 * a];
    at[4 * a + 2] = c.R[3 * a + 1];
    at[4 * a + 3] = c.R[3 * a + 2];
  }
  double* d_at = nullptr;
  EFE_CUDA_TRY(cudaMalloc(&d_at, sizeof(double) * std::max<size_t>(at.size(), 4)));
  EFE_CUDA_TRY(cudaMemcpyAsync(d_at, at.data(), sizeof(double) * at.size(), cudaMemcpyHostToDevice, s));
  k_geometry<<<nblk((long long)c.nc * c.nq), 256, 0, s>>>(c.tab, c.mesh, c.NQ1, d_at, c.n_atoms, c.d_xq, c.d_wJ,
                                                        c.d_vN);
  note_launch();
  EFE_CUDA_TRY(cudaGetLastError());
  EFE_CUDA_TRY(cudaStreamSynchronize(s));
  cudaFree(d_at);
  return cudaSuccess;
}

cudaError_t launch_coords(const Ctx& c, double* nodes, double* quad, cudaStream_t s) {
  if (nodes) {
    double xi[kMaxP1], w[kMaxP1];
    gauss_lobatto(c.p, xi, w);
    double* d_xi = nullptr;
    EFE_CUDA_TRY(cudaMalloc(&d_xi, sizeof(xi)));
    EFE_CUDA_TRY(cudaMemcpyAsync(d_xi, xi, sizeof(xi), cudaMemcpyHostToDevice, s));
    k_node_coords<<<nblk(c.n_h), 256, 0, s>>>(c.tab, c.mesh, d_xi, nodes);
    note_launch();
    EFE_CUDA_TRY(cudaGetLastError());
    EFE_CUDA_TRY(cudaStreamSynchronize(s));
    cudaFree(d_xi);
  }
  if (quad)
    EFE_CUDA_TRY(cudaMemcpyAsync(quad, c.d_xq, sizeof(double) * 3 * c.nc * c.nq, cudaMemcpyDeviceToDevice, s));
  return cudaSuccess;
}

cudaError_t launch_enrich_setup(Ctx& c, cudaStream_t s) {
  const int nE = c.nE;
  const long long np = c.n_pairs;
  std::vector<EnrDev> h(nE);
  for (int i = 0; i < nE; ++i) {
    const efe_enrich_fn& f = c.fns[i];
    h[i] = EnrDev{f.atom, f.n, f.l, f.m, f.radial, f.zeta, c.R[3 * f.atom], c.R[3 * f.atom + 1], c.R[3 * f.atom + 2]};
  }
  EnrDev* d_fns = nullptr;
  double *d_Aval = nullptr, *d_Agrad = nullptr, *d_b = nullptr, *d_cm = nullptr, *d_MAA = nullptr, *d_Mee = nullptr;
  EFE_CUDA_TRY(cudaMalloc(&d_fns, sizeof(EnrDev) * nE));
  EFE_CUDA_TRY(cudaMalloc(&d_Aval, sizeof(double) * std::max(np, 1LL) * c.nq));
  EFE_CUDA_TRY(cudaMalloc(&d_Agrad, sizeof(double) * std::max(np, 1LL) * c.nq * 3));
  EFE_CUDA_TRY(cudaMalloc(&d_b, sizeof(double) * c.n_h * nE));
  EFE_CUDA_TRY(cudaMalloc(&d_cm, sizeof(double) * c.n_h * nE));
  EFE_CUDA_TRY(cudaMalloc(&d_MAA, sizeof(double) * nE * nE));
  EFE_CUDA_TRY(cudaMalloc(&d_Mee, sizeof(double) * nE * nE));
  EFE_CUDA_TRY(cudaMemcpyAsync(d_fns, h.data(), sizeof(EnrDev) * nE, cudaMemcpyHostToDevice, s));
  EFE_CUDA_TRY(cudaMemsetAsync(d_b, 0, sizeof(double) * c.n_h * nE, s));
  EFE_CUDA_TRY(cudaMemsetAsync(d_MAA, 0, sizeof(double) * nE * nE, s));
  EFE_CUDA_TRY(cudaMemsetAsync(c.d_KEE, 0, sizeof(double) * nE * nE, s));
  if (np > 0) {
    k_enr_eval<<<nblk(np * c.nq), 256, 0, s>>>(c.d_pair_cell, c.d_pair_fn, np, c.nq, c.d_xq, d_fns, c.r0, c.s,
                                               d_Aval, d_Agrad);
    note_launch();
    k_enr_b<<<nblk(np * c.nn), 256, 0, s>>>(c.tab, c.mesh, c.NQ1, c.d_pair_cell, c.d_pair_fn, np, c.d_wJ, d_Aval, d_b);
    note_launch();
    EFE_CUDA_TRY(cudaGetLastError());
  }
  k_enr_c2<<<nblk(c.n_h * nE), 256, 0, s>>>(d_b, c.d_Dsc, d_cm, c.n_h, nE);
  note_launch();
  EFE_CUDA_TRY(cudaGetLastError());
  if (np > 0) {
    const size_t sm = sizeof(double) * (c.nn + 3 * c.nq);
    k_enr_orth<<<(unsigned)np, 128, sm, s>>>(c.tab, c.mesh, c.NQ1, c.d_pair_cell, c.d_pair_fn, np, c.d_wJ, d_cm,
                                             d_Aval, d_Agrad, c.d_Atil, c.d_KE);
    note_launch();
    k_enr_gram<<<c.nc, 128, 0, s>>>(c.d_pair_start, c.d_pair_fn, c.nq, nE, c.d_wJ, d_Aval, d_Agrad, d_MAA, c.d_KEE);
    note_launch();
    EFE_CUDA_TRY(cudaGetLastError());
  }
  k_mee<<<nE * nE, kThreads, 0, s>>>(d_b, c.d_Dsc, c.n_h, nE, d_MAA, d_Mee);
  note_launch();
  EFE_CUDA_TRY(cudaGetLastError());
  c.Mee.assign((size_t)nE * nE, 0.0);
  EFE_CUDA_TRY(cudaMemcpyAsync(c.Mee.data(), d_Mee, sizeof(double) * nE * nE, cudaMemcpyDeviceToHost, s));
  EFE_CUDA_TRY(cudaStreamSynchronize(s));
  cudaFree(d_fns);
  cudaFree(d_Aval);
  cudaFree(d_Agrad);
  cudaFree(d_b);
  cudaFree(d_cm);
  cudaFree(d_MAA);
  cudaFree(d_Mee);
  return cudaSuccess;
}

cudaError_t launch_poisson_setup(Ctx& c, cudaStream_t s) {
  EFE_CUDA_TRY(cudaMemsetAsync(c.d_diagA, 0, sizeof(double) * c.n_h, s));
  const double scale = 1.0 / (2.0 * 3.14159265358979323846);   // (1/4pi) int grad.grad = (1/2pi) * kinetic
  k_laplace_diag<<<nblk((long long)c.nc * c.nn), 256, 0, s>>>(c.tab, c.mesh, scale, c.d_diagA);
  note_launch();
  EFE_CUDA_TRY(cudaGetLastError());
  double* d_nodes = nullptr;
  EFE_CUDA_TRY(cudaMalloc(&d_nodes, sizeof(double) * 3 * c.n_h));
  EFE_CUDA_TRY(launch_coords(c, d_nodes, nullptr, s));
  std::vector<double> at(4 * (size_t)c.n_atoms);
  for (int a = 0; a < c.n_atoms; ++a) {
    at[4 * a] = c.Z[a];
    at[4 * a + 1] = c.R[3 * a];
    at[4 * a + 2] = c.R[3 * a + 1];
    at[4 * a + 3] = c.R[3 * a + 2];
  }
  double* d_at = nullptr;
  EFE_CUDA_TRY(cudaMalloc(&d_at, sizeof(double) * std::max<size_t>(at.size(), 4)));
  EFE_CUDA_TRY(cudaMemcpyAsync(d_at, at.data(), sizeof(double) * at.size(), cudaMemcpyHostToDevice, s));
  k_poisson_bc<<<nblk(c.n_h), 256, 0, s>>>(c.mesh, d_nodes, c.d_Dsc, d_at, c.n_atoms, c.d_phiB, c.d_diagA);
  note_launch();
  EFE_CUDA_TRY(cudaGetLastError());
  EFE_CUDA_TRY(cudaStreamSynchronize(s));
  cudaFree(d_nodes);
  cudaFree(d_at);
  return cudaSuccess;
}

cudaError_t launch_init_orbitals(const Ctx& c, double* psi, int G, const double* d_centers, const double* d_expo,
                                 const double* d_coef, const double* d_enr, cudaStream_t s) {
  double* d_nodes = nullptr;
  EFE_CUDA_TRY(cudaMalloc(&d_nodes, sizeof(double) * 3 * c.n_h));
  EFE_CUDA_TRY(launch_coords(c, d_nodes, nullptr, s));
  const long long ld2 = 2LL * c.n_orb * c.batch;
  k_init_orb<<<nblk(c.n_h * c.n_orb), 256, 0, s>>>(d_nodes, c.d_Dsc, c.n_h, c.n_orb, c.batch, G, d_centers, d_expo,
                                                  d_coef, psi, ld2);
  note_launch();
  if (c.nE > 0)
    k_init_enr<<<nblk((long long)c.nE * c.n_orb), 256, 0, s>>>(c.d_Shalf, d_enr, c.n_h, c.nE, c.n_orb, c.batch, psi,
                                                               ld2);
    note_launch();
  EFE_CUDA_TRY(cudaGetLastError());
  EFE_CUDA_TRY(cudaStreamSynchronize(s));
  cudaFree(d_nodes);
  return cudaSuccess;
}

}  // namespace efe
