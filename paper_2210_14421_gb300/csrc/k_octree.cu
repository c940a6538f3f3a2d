// Locally refined mesh with hanging-node constraints (the paper's adaptively
// refined mesh, Sec. "Enriched finite element basis"): the Hamiltonian of
// Eq. Hmn applied in the constrained space, Y = P^T (kin (1/2) K + V) P X.
//
// The mesh is one refinement level over a uniform coarse grid: chosen coarse
// cells are split into 2 x 2 x 2 leaves, so neighbouring leaves differ by at
// most one level.  Every leaf carries degree-p Lagrange functions on GLL nodes;
// coincident nodes of leaves are one node.  A node of a fine leaf that lies on
// the closed box of a coarse leaf without being one of its nodes is hanging:
// its value is the coarse leaf's interpolant there, so u_all = P u_free with P
// the interpolation weights (rows of hanging nodes) and the identity (rows of
// free nodes).  The apply is three stages: the gather x_all = P x_free, the
// per-leaf operator (kinetic and potential by sum factorisation, the
// potential at the Gauss-Legendre points) scatter-added into y_all, and
// the transposed scatter y_free = P^T y_all.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <type_traits>
#include <vector>

#include "efe_internal.h"

namespace efe {

constexpr int kOctMaxQ1 = 8;
constexpr int kOctThreads = 128;

// 1D reference tables of the leaves (passed by value): GL values of the GLL
// Lagrange basis B1[q][i], exact 1D stiffness and mass K1, M1, GL weights.
struct OctTables {
  double B1[kOctMaxQ1 * kMaxP1];
  double K1[kMaxP1 * kMaxP1];
  double M1[kMaxP1 * kMaxP1];
  double wg[kOctMaxQ1];
  int P1, NQ1;
};

struct Octree {
  std::string err;
  int p = 0, P1 = 0, NQ1 = 0, nn = 0, nq = 0;
  long long n_leaves = 0, n_all = 0, n_free = 0, n_hang = 0;
  OctTables tab{};
  std::vector<double> free_xyz, quad_xyz;   // host copies for efe_octree_coords
  std::vector<double> all_xyz;              // coordinates of all nodes
  std::vector<double> geo;                  // host copies of the device arrays
  std::vector<int> conn;
  std::vector<unsigned char> bnd;
  std::vector<double> D;                    // [n_free] mask / sqrt(lumped constrained mass)
  std::vector<double> Kdiag;                // [n_free] diagonal of P^T K P (Jacobi preconditioner)
  std::vector<long long> rs;                // host copy of P (CSR over all nodes)
  std::vector<int> col;
  std::vector<double> val;
  double* d_geo = nullptr;                  // [n_leaves][6] origin, size
  int* d_conn = nullptr;                    // [n_leaves][nn] node ids
  long long* d_rs = nullptr;                // [n_all + 1] row starts of P
  int* d_col = nullptr;                     // free index per entry
  double* d_val = nullptr;                  // weight per entry
  unsigned char* d_bnd = nullptr;           // [n_free] 1 on the domain boundary
  double* d_D = nullptr;                    // [n_free] Loewdin scaling
  double* d_Kdiag = nullptr;                // [n_free] diagonal of the constrained stiffness
  double* d_xall = nullptr;                 // [n_all][cols] scratch
  double* d_yall = nullptr;
  long long ws_cols = 0;
  ~Octree() {
    for (void* q : {(void*)d_geo, (void*)d_conn, (void*)d_rs, (void*)d_col, (void*)d_val, (void*)d_bnd,
                    (void*)d_D, (void*)d_Kdiag, (void*)d_xall, (void*)d_yall})
      if (q) cudaFree(q);
  }
};

namespace {

// x_all[n][c] = sum_k val_k x_free[col_k][c] over row n of P (boundary free values as 0 when masked)
// (with scale: x_free scaled by scale[f] first, the Loewdin D that is 0 on the boundary)
__global__ void k_oct_expand(const long long* __restrict__ rs, const int* __restrict__ col,
                             const double* __restrict__ val, const unsigned char* __restrict__ bnd,
                             const double* __restrict__ scale, const double* __restrict__ xf, long long n_all,
                             int ncols, int mask, double* __restrict__ xa) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n_all * ncols) return;
  const long long n = idx / ncols;
  const int c = (int)(idx % ncols);
  double v = 0.0;
  for (long long k = rs[n]; k < rs[n + 1]; ++k) {
    const int f = col[k];
    if (mask && bnd[f]) continue;
    v += val[k] * (scale ? scale[f] : 1.0) * xf[(long long)f * ncols + c];
  }
  xa[idx] = v;
}

// y_free[col_k][c] += val_k y_all[n][c] over row n of P (boundary rows skipped when masked)
// (with scale: each contribution scaled by scale[f])
__global__ void k_oct_reduce(const long long* __restrict__ rs, const int* __restrict__ col,
                             const double* __restrict__ val, const unsigned char* __restrict__ bnd,
                             const double* __restrict__ scale, const double* __restrict__ ya, long long n_all,
                             int ncols, int mask, double* __restrict__ yf) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n_all * ncols) return;
  const long long n = idx / ncols;
  const int c = (int)(idx % ncols);
  const double y = ya[idx];
  for (long long k = rs[n]; k < rs[n + 1]; ++k) {
    const int f = col[k];
    if (mask && bnd[f]) continue;
    atomicAdd(&yf[(long long)f * ncols + c], val[k] * (scale ? scale[f] : 1.0) * y);
  }
}

// One block per (leaf, column): y_all += (kin (1/2) K_leaf + V_leaf) x_leaf, v at the leaf's GL points.
__global__ void __launch_bounds__(kOctThreads)
k_oct_apply(const OctTables T, const double* __restrict__ geo, const int* __restrict__ conn,
            const double* __restrict__ vq, double kin, const double* __restrict__ xa, int ncols,
            double* __restrict__ ya) {
  __shared__ double x[kMaxP1 * kMaxP1 * kMaxP1];
  __shared__ double A[kOctMaxQ1 * kMaxP1 * kMaxP1];
  __shared__ double Bq[kOctMaxQ1 * kOctMaxQ1 * kMaxP1];
  __shared__ double Cq[kOctMaxQ1 * kOctMaxQ1 * kOctMaxQ1];
  __shared__ double ka[kMaxP1 * kMaxP1 * kMaxP1], kb[kMaxP1 * kMaxP1 * kMaxP1];
  __shared__ double kc[kMaxP1 * kMaxP1 * kMaxP1], kd[kMaxP1 * kMaxP1 * kMaxP1], ke[kMaxP1 * kMaxP1 * kMaxP1];
  const int P1 = T.P1, Q = T.NQ1, nn = P1 * P1 * P1, nq = Q * Q * Q;
  const long long leaf = blockIdx.x;
  const int c = blockIdx.y;
  const double hx = geo[6 * leaf + 3], hy = geo[6 * leaf + 4], hz = geo[6 * leaf + 5];
  const int* cl = conn + leaf * nn;
  for (int l = threadIdx.x; l < nn; l += blockDim.x) x[l] = xa[(long long)cl[l] * ncols + c];
  __syncthreads();
  // potential (skipped when vq is NULL: v = 0): values at the GL points (axis 1, 2, 3), times
  // w |J| v, back (axis 3, 2, 1)
  const bool pot = vq != nullptr;   // uniform over the block
  if (pot) {
  for (int t = threadIdx.x; t < Q * P1 * P1; t += blockDim.x) {   // A[q1][i2][i3]
    const int q1 = t % Q, i2 = (t / Q) % P1, i3 = t / (Q * P1);
    double s = 0.0;
    for (int i1 = 0; i1 < P1; ++i1) s += T.B1[q1 * P1 + i1] * x[i1 + P1 * (i2 + P1 * i3)];
    A[t] = s;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < Q * Q * P1; t += blockDim.x) {    // Bq[q1][q2][i3]
    const int q1 = t % Q, q2 = (t / Q) % Q, i3 = t / (Q * Q);
    double s = 0.0;
    for (int i2 = 0; i2 < P1; ++i2) s += T.B1[q2 * P1 + i2] * A[q1 + Q * (i2 + P1 * i3)];
    Bq[t] = s;
  }
  __syncthreads();
  const double detJ = hx * hy * hz / 8.0;
  for (int t = threadIdx.x; t < nq; t += blockDim.x) {            // Cq[q1][q2][q3]
    const int q1 = t % Q, q2 = (t / Q) % Q, q3 = t / (Q * Q);
    double s = 0.0;
    for (int i3 = 0; i3 < P1; ++i3) s += T.B1[q3 * P1 + i3] * Bq[q1 + Q * (q2 + Q * i3)];
    Cq[t] = s * T.wg[q1] * T.wg[q2] * T.wg[q3] * detJ * vq[leaf * nq + t];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < Q * Q * P1; t += blockDim.x) {    // Bq[q1][q2][i3] = sum_q3
    const int q1 = t % Q, q2 = (t / Q) % Q, i3 = t / (Q * Q);
    double s = 0.0;
    for (int q3 = 0; q3 < Q; ++q3) s += T.B1[q3 * P1 + i3] * Cq[q1 + Q * (q2 + Q * q3)];
    Bq[t] = s;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < Q * P1 * P1; t += blockDim.x) {   // A[q1][i2][i3] = sum_q2
    const int q1 = t % Q, i2 = (t / Q) % P1, i3 = t / (Q * P1);
    double s = 0.0;
    for (int q2 = 0; q2 < Q; ++q2) s += T.B1[q2 * P1 + i2] * Bq[q1 + Q * (q2 + Q * i3)];
    A[t] = s;
  }
  __syncthreads();
  }
  // kinetic by sum factorisation: with a = M1 x, b = K1 x along axis 3, then c = M1 a, d = K1 a,
  // e = M1 b along axis 2, y = ax K1 c + ay M1 d + az M1 e along axis 1 (ax = kin hy hz / (4 hx), ...)
  for (int l = threadIdx.x; l < nn; l += blockDim.x) {   // a, b [i1][i2][i3] from x along axis 3
    const int i1 = l % P1, i2 = (l / P1) % P1, i3 = l / (P1 * P1);
    double sa = 0.0, sb = 0.0;
    for (int j3 = 0; j3 < P1; ++j3) {
      const double v = x[i1 + P1 * (i2 + P1 * j3)];
      sa += T.M1[i3 * P1 + j3] * v;
      sb += T.K1[i3 * P1 + j3] * v;
    }
    ka[l] = sa;
    kb[l] = sb;
  }
  __syncthreads();
  for (int l = threadIdx.x; l < nn; l += blockDim.x) {   // c, d, e along axis 2
    const int i1 = l % P1, i2 = (l / P1) % P1, i3 = l / (P1 * P1);
    double sc = 0.0, sd = 0.0, se = 0.0;
    for (int j2 = 0; j2 < P1; ++j2) {
      const int m = i1 + P1 * (j2 + P1 * i3);
      sc += T.M1[i2 * P1 + j2] * ka[m];
      sd += T.K1[i2 * P1 + j2] * ka[m];
      se += T.M1[i2 * P1 + j2] * kb[m];
    }
    kc[l] = sc;
    kd[l] = sd;
    ke[l] = se;
  }
  __syncthreads();
  const double ax = kin * hy * hz / (4.0 * hx), ay = kin * hx * hz / (4.0 * hy), az = kin * hx * hy / (4.0 * hz);
  for (int l = threadIdx.x; l < nn; l += blockDim.x) {   // axis 1, plus the last potential axis; scatter-add
    const int i1 = l % P1, i2 = (l / P1) % P1, i3 = l / (P1 * P1);
    double y = 0.0;
    if (pot)
      for (int q1 = 0; q1 < Q; ++q1) y += T.B1[q1 * P1 + i1] * A[q1 + Q * (i2 + P1 * i3)];
    double k1 = 0.0, k2 = 0.0, k3 = 0.0;
    for (int j1 = 0; j1 < P1; ++j1) {
      const int m = j1 + P1 * (i2 + P1 * i3);
      k1 += T.K1[i1 * P1 + j1] * kc[m];
      k2 += T.M1[i1 * P1 + j1] * kd[m];
      k3 += T.M1[i1 * P1 + j1] * ke[m];
    }
    atomicAdd(&ya[(long long)cl[l] * ncols + c], y + ax * k1 + ay * k2 + az * k3);
  }
}

// rho[leaf][q] = sum_a occ_a |psi_a(x_q)|^2 from x_all [n_all][2 n_orb] (re, im per orbital), one
// block per leaf: each component interpolated to the GL points by three sum-factorisation passes.
__global__ void __launch_bounds__(kOctThreads)
k_oct_density(const OctTables T, const int* __restrict__ conn, const double* __restrict__ xa, int n_orb,
              const double* __restrict__ occ, double* __restrict__ rho) {
  __shared__ double x[kMaxP1 * kMaxP1 * kMaxP1];
  __shared__ double A[kOctMaxQ1 * kMaxP1 * kMaxP1];
  __shared__ double Bq[kOctMaxQ1 * kOctMaxQ1 * kMaxP1];
  __shared__ double acc[kOctMaxQ1 * kOctMaxQ1 * kOctMaxQ1];
  const int P1 = T.P1, Q = T.NQ1, nn = P1 * P1 * P1, nq = Q * Q * Q;
  const long long leaf = blockIdx.x;
  const int* cl = conn + leaf * nn;
  const int ncols = 2 * n_orb;
  for (int t = threadIdx.x; t < nq; t += blockDim.x) acc[t] = 0.0;
  for (int col = 0; col < ncols; ++col) {
    __syncthreads();
    for (int l = threadIdx.x; l < nn; l += blockDim.x) x[l] = xa[(long long)cl[l] * ncols + col];
    __syncthreads();
    for (int t = threadIdx.x; t < Q * P1 * P1; t += blockDim.x) {
      const int q1 = t % Q, i2 = (t / Q) % P1, i3 = t / (Q * P1);
      double s = 0.0;
      for (int i1 = 0; i1 < P1; ++i1) s += T.B1[q1 * P1 + i1] * x[i1 + P1 * (i2 + P1 * i3)];
      A[t] = s;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < Q * Q * P1; t += blockDim.x) {
      const int q1 = t % Q, q2 = (t / Q) % Q, i3 = t / (Q * Q);
      double s = 0.0;
      for (int i2 = 0; i2 < P1; ++i2) s += T.B1[q2 * P1 + i2] * A[q1 + Q * (i2 + P1 * i3)];
      Bq[t] = s;
    }
    __syncthreads();
    const double o = occ[col / 2];
    for (int t = threadIdx.x; t < nq; t += blockDim.x) {
      const int q1 = t % Q, q2 = (t / Q) % Q, q3 = t / (Q * Q);
      double s = 0.0;
      for (int i3 = 0; i3 < P1; ++i3) s += T.B1[q3 * P1 + i3] * Bq[q1 + Q * (q2 + Q * i3)];
      acc[t] += o * s * s;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nq; t += blockDim.x) rho[leaf * nq + t] = acc[t];
}

// out[c][leaf][q] = sum_l N_l(x_q) x_all[conn[leaf][l]][c]: values at the leaves' GL points of ncols
// real nodal columns (one block per leaf, three sum-factorisation passes per column)
__global__ void __launch_bounds__(kOctThreads)
k_oct_interp(const OctTables T, const int* __restrict__ conn, const double* __restrict__ xa, int ncols,
             long long n_leaves, double* __restrict__ out) {
  __shared__ double x[kMaxP1 * kMaxP1 * kMaxP1];
  __shared__ double A[kOctMaxQ1 * kMaxP1 * kMaxP1];
  __shared__ double Bq[kOctMaxQ1 * kOctMaxQ1 * kMaxP1];
  const int P1 = T.P1, Q = T.NQ1, nn = P1 * P1 * P1, nq = Q * Q * Q;
  const long long leaf = blockIdx.x;
  const int* cl = conn + leaf * nn;
  for (int col = 0; col < ncols; ++col) {
    __syncthreads();
    for (int l = threadIdx.x; l < nn; l += blockDim.x) x[l] = xa[(long long)cl[l] * ncols + col];
    __syncthreads();
    for (int t = threadIdx.x; t < Q * P1 * P1; t += blockDim.x) {
      const int q1 = t % Q, i2 = (t / Q) % P1, i3 = t / (Q * P1);
      double s = 0.0;
      for (int i1 = 0; i1 < P1; ++i1) s += T.B1[q1 * P1 + i1] * x[i1 + P1 * (i2 + P1 * i3)];
      A[t] = s;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < Q * Q * P1; t += blockDim.x) {
      const int q1 = t % Q, q2 = (t / Q) % Q, i3 = t / (Q * Q);
      double s = 0.0;
      for (int i2 = 0; i2 < P1; ++i2) s += T.B1[q2 * P1 + i2] * A[q1 + Q * (i2 + P1 * i3)];
      Bq[t] = s;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nq; t += blockDim.x) {
      const int q1 = t % Q, q2 = (t / Q) % Q, q3 = t / (Q * Q);
      double s = 0.0;
      for (int i3 = 0; i3 < P1; ++i3) s += T.B1[q3 * P1 + i3] * Bq[q1 + Q * (q2 + Q * i3)];
      out[((long long)col * n_leaves + leaf) * nq + t] = s;
    }
  }
}

// v = vN + vH + vxc + vf (pointwise), rho_mid = (a + b) / 2, y = c x
__global__ void k_oct_vsum(const double* __restrict__ vN, const double* __restrict__ vH, const double* __restrict__ vxc,
                           const double* __restrict__ vf, long long n, double* __restrict__ v) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) v[i] = vN[i] + vH[i] + vxc[i] + vf[i];
}
__global__ void k_oct_axpby(const double* a, const double* b, double ca, double cb, long long n, double* out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = ca * a[i] + cb * b[i];
}

unsigned oblk(long long n) { return (unsigned)((n + 255) / 256); }

// Per complex column c of [n][2C] arrays (re, im interleaved): out[c] += Re sum_i conj(a_ic) b_ic over the
// block's slice of rows (blockIdx.x = column, gridDim.y slices; the caller zeroes out)
__global__ void __launch_bounds__(256) k_oct_cdot(const double* __restrict__ a, const double* __restrict__ b,
                                                  long long n, int C, double* __restrict__ out) {
  __shared__ double red[256];
  const int c = blockIdx.x;
  const long long chunk = (n + gridDim.y - 1) / gridDim.y;
  const long long i0 = (long long)blockIdx.y * chunk, i1 = min(n, i0 + chunk);
  double acc = 0.0;
  for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const long long o = i * 2 * C + 2 * c;
    acc += a[o] * b[o] + a[o + 1] * b[o + 1];
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(&out[c], red[0]);
}

// boundary rows of a [n][2C] array set to 0 (the Dirichlet space)
__global__ void k_oct_zero_bnd(double* __restrict__ x, const unsigned char* __restrict__ bnd, long long n, int C) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n * 2 * C) return;
  if (bnd[idx / (2 * C)]) x[idx] = 0.0;
}

// y[:, c] = s[c] x[:, c] (complex column c, real scalar; y may be x)
__global__ void k_oct_cscale(const double* x, const double* __restrict__ sc, long long n, int C, double* y) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n * 2 * C) return;
  y[idx] = sc[(idx % (2 * C)) / 2] * x[idx];
}

// w[:, c] -= a[c] q[:, c] + b[c] qm[:, c]   (qm may be NULL)
__global__ void k_oct_lz_update(double* __restrict__ w, const double* __restrict__ q, const double* __restrict__ qm,
                                const double* __restrict__ a, const double* __restrict__ b, long long n, int C) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n * 2 * C) return;
  const int c = (int)((idx % (2 * C)) / 2);
  double v = w[idx] - a[c] * q[idx];
  if (qm) v -= b[c] * qm[idx];
  w[idx] = v;
}

// psi[:, c] = sum_j y[c][j] Q_j[:, c] with complex y ([C][k][2]); Q_j = Q + j n 2C
// psi = sum_{j < k} y_j Q_j per column, y [C][ks][2] (only the first k basis vectors were formed)
__global__ void k_oct_lz_combine(const double* __restrict__ Q, const double* __restrict__ y, int k, int ks, long long n,
                                 int C, double* __restrict__ psi) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n * C) return;
  const long long i = idx / C;
  const int c = (int)(idx % C);
  double re = 0.0, im = 0.0;
  for (int j = 0; j < k; ++j) {
    const double* q = Q + (long long)j * n * 2 * C + i * 2 * C + 2 * c;
    const double yr = y[(c * ks + j) * 2], yi = y[(c * ks + j) * 2 + 1];
    re += yr * q[0] - yi * q[1];
    im += yr * q[1] + yi * q[0];
  }
  psi[i * 2 * C + 2 * c] = re;
  psi[i * 2 * C + 2 * c + 1] = im;
}

// *out += a . b (the caller zeroes *out)
__global__ void __launch_bounds__(256) k_oct_dot(const double* __restrict__ a, const double* __restrict__ b,
                                                 long long n, double* __restrict__ out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc += a[i] * b[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, red[0]);
}

// gB = g on the boundary free nodes, 0 inside; ones = 1
__global__ void k_oct_bc(const double* __restrict__ g, const unsigned char* __restrict__ bnd, long long n,
                         double* __restrict__ gB, double* __restrict__ ones) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  gB[i] = bnd[i] ? g[i] : 0.0;
  ones[i] = 1.0;
}

// r = F - y inside, 0 on the boundary; z = p = r / diag; u = 0
__global__ void k_oct_cg_start(const double* __restrict__ F, const double* __restrict__ y,
                               const unsigned char* __restrict__ bnd, const double* __restrict__ diag, long long n,
                               double* __restrict__ r, double* __restrict__ z, double* __restrict__ p,
                               double* __restrict__ u) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = bnd[i] ? 0.0 : F[i] - y[i];
  r[i] = v;
  z[i] = bnd[i] ? 0.0 : v / diag[i];
  p[i] = z[i];
  u[i] = 0.0;
}

// z = r / diag inside (0 on the boundary)
__global__ void k_oct_precond(const double* __restrict__ r, const double* __restrict__ diag,
                              const unsigned char* __restrict__ bnd, long long n, double* __restrict__ z) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  z[i] = bnd[i] ? 0.0 : r[i] / diag[i];
}

// u += alpha p, r -= alpha Ap
__global__ void k_oct_cg_step(double* __restrict__ u, double* __restrict__ r, const double* __restrict__ p,
                              const double* __restrict__ Ap, double alpha, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  u[i] += alpha * p[i];
  r[i] -= alpha * Ap[i];
}

// p = z + beta p
__global__ void k_oct_cg_dir(double* __restrict__ p, const double* __restrict__ r, double beta, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  p[i] = r[i] + beta * p[i];
}

// u = g on the boundary free nodes
__global__ void k_oct_cg_finish(double* __restrict__ u, const double* __restrict__ g,
                                const unsigned char* __restrict__ bnd, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (bnd[i]) u[i] = g[i];
}

}  // namespace

// Builds the mesh, the constraints and the tables (host), then copies them to the device.
// Host side of the set-up: leaves, nodes, constraints, tables (no device work).
static efe_status octree_host(Octree& o, const double* lo, const double* hi, int nc, int p, int n_quad,
                              const int32_t* refine, int n_refine) {
  if (nc < 1 || p < 1 || p + 1 > kMaxP1 || n_quad < p + 1 || n_quad > kOctMaxQ1 || n_refine < 0 ||
      (n_refine > 0 && !refine)) {
    o.err = "octree: need nc >= 1, degree in [1, 5], n_quad in [p + 1, 8]";
    return EFE_ERR_ARG;
  }
  for (int a = 0; a < 3; ++a)
    if (!(hi[a] > lo[a])) {
      o.err = "octree: empty box";
      return EFE_ERR_ARG;
    }
  std::vector<char> ref((size_t)nc * nc * nc, 0);
  for (int r = 0; r < n_refine; ++r) {
    const int i = refine[3 * r], j = refine[3 * r + 1], k = refine[3 * r + 2];
    if (i < 0 || j < 0 || k < 0 || i >= nc || j >= nc || k >= nc) {
      o.err = "octree: refined cell outside the coarse grid";
      return EFE_ERR_ARG;
    }
    ref[i + (size_t)nc * (j + (size_t)nc * k)] = 1;
  }
  o.p = p;
  o.P1 = p + 1;
  o.NQ1 = n_quad;
  o.nn = o.P1 * o.P1 * o.P1;
  o.nq = n_quad * n_quad * n_quad;
  const int P1 = o.P1, nn = o.nn;
  double hc[3], hmin = 1e300;
  for (int a = 0; a < 3; ++a) {
    hc[a] = (hi[a] - lo[a]) / nc;
    hmin = std::min(hmin, hc[a]);
  }
  // leaves: coarse cells in x-fastest order, a refined cell as its 8 children (bit a of the child: upper half on axis a)
  struct Leaf { double x0[3], h[3]; bool coarse; };
  std::vector<Leaf> leaves;
  std::vector<long long> coarse_leaf((size_t)nc * nc * nc, -1);   // leaf of an unrefined coarse cell
  for (int k = 0; k < nc; ++k)
    for (int j = 0; j < nc; ++j)
      for (int i = 0; i < nc; ++i) {
        const int ijk[3] = {i, j, k};
        Leaf L;
        for (int a = 0; a < 3; ++a) L.x0[a] = lo[a] + ijk[a] * hc[a];
        if (ref[i + (size_t)nc * (j + (size_t)nc * k)]) {
          for (int ch = 0; ch < 8; ++ch) {
            Leaf S;
            for (int a = 0; a < 3; ++a) {
              S.x0[a] = L.x0[a] + 0.5 * ((ch >> a) & 1) * hc[a];
              S.h[a] = 0.5 * hc[a];
            }
            S.coarse = false;
            leaves.push_back(S);
          }
        } else {
          for (int a = 0; a < 3; ++a) L.h[a] = hc[a];
          L.coarse = true;
          coarse_leaf[i + (size_t)nc * (j + (size_t)nc * k)] = (long long)leaves.size();
          leaves.push_back(L);
        }
      }
  std::vector<double> xi(P1), wl(P1);
  gauss_lobatto(p, xi.data(), wl.data());
  // nodes merged by position (integer keys on a lattice much finer than any node spacing)
  const double scale = 1.0 / (hmin * 1e-9);
  std::map<std::array<long long, 3>, int> key_of;
  std::vector<double> xyz;
  std::vector<int> conn(leaves.size() * (size_t)nn);
  std::vector<char> fine_node;
  for (size_t li = 0; li < leaves.size(); ++li)
    for (int l = 0; l < nn; ++l) {
      const int loc[3] = {l % P1, (l / P1) % P1, l / (P1 * P1)};
      double X[3];
      std::array<long long, 3> key;
      for (int a = 0; a < 3; ++a) {
        X[a] = leaves[li].x0[a] + 0.5 * (xi[loc[a]] + 1.0) * leaves[li].h[a];
        key[a] = std::llround(X[a] * scale);
      }
      auto it = key_of.find(key);
      int id;
      if (it == key_of.end()) {
        id = (int)(xyz.size() / 3);
        key_of.emplace(key, id);
        xyz.insert(xyz.end(), X, X + 3);
        fine_node.push_back(0);
      } else {
        id = it->second;
      }
      if (!leaves[li].coarse) fine_node[id] = 1;
      conn[li * nn + l] = id;
    }
  const long long n_all = (long long)(xyz.size() / 3);
  // hanging nodes: nodes of fine leaves on the closed box of a coarse leaf that are not its nodes
  const double tol = 1e-9 * hmin;
  std::vector<std::vector<std::pair<int, double>>> hang((size_t)n_all);
  std::vector<char> is_hang((size_t)n_all, 0);
  std::vector<double> L1(P1), dL1(P1);
  for (long long nd = 0; nd < n_all; ++nd) {
    if (!fine_node[nd]) continue;
    const double* X = &xyz[3 * nd];
    // the coarse cells whose closed box holds X
    int lo_i[3], hi_i[3];
    for (int a = 0; a < 3; ++a) {
      lo_i[a] = std::max(0, (int)std::floor((X[a] - lo[a] - tol) / hc[a]));
      hi_i[a] = std::min(nc - 1, (int)std::floor((X[a] - lo[a] + tol) / hc[a]));
    }
    for (int k = lo_i[2]; k <= hi_i[2] && !is_hang[nd]; ++k)
      for (int j = lo_i[1]; j <= hi_i[1] && !is_hang[nd]; ++j)
        for (int i = lo_i[0]; i <= hi_i[0] && !is_hang[nd]; ++i) {
          const long long lc = coarse_leaf[i + (size_t)nc * (j + (size_t)nc * k)];
          if (lc < 0) continue;   // refined cell
          const size_t li = (size_t)lc;
          const Leaf& C = leaves[li];
          bool inside = true, own = false;
          for (int a = 0; a < 3; ++a)
            if (X[a] < C.x0[a] - tol || X[a] > C.x0[a] + C.h[a] + tol) inside = false;
          for (int l = 0; l < nn && inside; ++l)
            if (conn[li * nn + l] == nd) own = true;
          if (!inside || own) continue;
          std::vector<double> Lv[3];
          for (int a = 0; a < 3; ++a) {
            const double r = 2.0 * (X[a] - C.x0[a]) / C.h[a] - 1.0;
            lagrange_tables(P1, xi.data(), 1, &r, L1.data(), dL1.data());
            Lv[a] = L1;
          }
          for (int l = 0; l < nn; ++l) {
            const double w = Lv[0][l % P1] * Lv[1][(l / P1) % P1] * Lv[2][l / (P1 * P1)];
            if (std::fabs(w) > 1e-14) hang[nd].push_back({conn[li * nn + l], w});
          }
          is_hang[nd] = 1;
        }
  }
  // free numbering and P in CSR over all nodes
  std::vector<int> free_of((size_t)n_all, -1);
  long long n_free = 0;
  for (long long nd = 0; nd < n_all; ++nd)
    if (!is_hang[nd]) free_of[nd] = (int)n_free++;
  std::vector<long long>& rs = o.rs;
  std::vector<int>& col = o.col;
  std::vector<double>& val = o.val;
  rs.assign((size_t)n_all + 1, 0);
  col.clear();
  val.clear();
  for (long long nd = 0; nd < n_all; ++nd) {
    if (is_hang[nd]) {
      for (auto& mw : hang[nd]) {
        if (is_hang[mw.first]) {
          o.err = "octree: a master node is hanging (more than one level between neighbours)";
          return EFE_ERR_ARG;
        }
        col.push_back(free_of[mw.first]);
        val.push_back(mw.second);
      }
    } else {
      col.push_back(free_of[nd]);
      val.push_back(1.0);
    }
    rs[nd + 1] = (long long)col.size();
  }
  std::vector<unsigned char> bnd((size_t)n_free, 0);
  o.free_xyz.assign((size_t)3 * n_free, 0.0);
  for (long long nd = 0; nd < n_all; ++nd) {
    if (is_hang[nd]) continue;
    const long long f = free_of[nd];
    for (int a = 0; a < 3; ++a) {
      o.free_xyz[3 * f + a] = xyz[3 * nd + a];
      if (std::fabs(xyz[3 * nd + a] - lo[a]) < tol || std::fabs(xyz[3 * nd + a] - hi[a]) < tol) bnd[f] = 1;
    }
  }
  // lumped mass of the constrained space: P^T m_all, m_all the GLL-lumped weights of all nodes
  {
    std::vector<double> m_all((size_t)n_all, 0.0);
    for (size_t li = 0; li < leaves.size(); ++li) {
      const double J = leaves[li].h[0] * leaves[li].h[1] * leaves[li].h[2] / 8.0;
      for (int l = 0; l < nn; ++l)
        m_all[conn[li * nn + l]] += wl[l % P1] * wl[(l / P1) % P1] * wl[l / (P1 * P1)] * J;
    }
    std::vector<double> m_c((size_t)n_free, 0.0);
    for (long long nd = 0; nd < n_all; ++nd)
      for (long long k = rs[nd]; k < rs[nd + 1]; ++k) m_c[col[k]] += val[k] * m_all[nd];
    o.D.assign((size_t)n_free, 0.0);
    for (long long f = 0; f < n_free; ++f) o.D[f] = bnd[f] ? 0.0 : 1.0 / std::sqrt(m_c[f]);
  }
  // tables
  std::vector<double> xg(n_quad), wg(n_quad), B(n_quad * P1), D(n_quad * P1);
  gauss_legendre(n_quad, xg.data(), wg.data());
  lagrange_tables(P1, xi.data(), n_quad, xg.data(), B.data(), D.data());
  o.tab.P1 = P1;
  o.tab.NQ1 = n_quad;
  for (int q = 0; q < n_quad; ++q) {
    o.tab.wg[q] = wg[q];
    for (int i = 0; i < P1; ++i) o.tab.B1[q * P1 + i] = B[q * P1 + i];
  }
  for (int i = 0; i < P1; ++i)
    for (int j = 0; j < P1; ++j) {
      double k = 0.0, m = 0.0;
      for (int q = 0; q < n_quad; ++q) {
        k += wg[q] * D[q * P1 + i] * D[q * P1 + j];
        m += wg[q] * B[q * P1 + i] * B[q * P1 + j];
      }
      o.tab.K1[i * P1 + j] = k;
      o.tab.M1[i * P1 + j] = m;
    }
  // diagonal of the constrained stiffness P^T K P: per leaf, sum over local pairs whose P rows share a free index
  o.Kdiag.assign((size_t)n_free, 0.0);
  {
    std::vector<std::vector<std::pair<int, double>>> rows(nn);
    for (size_t li = 0; li < leaves.size(); ++li) {
      const double hx = leaves[li].h[0], hy = leaves[li].h[1], hz = leaves[li].h[2];
      const double ax = hy * hz / (2.0 * hx), ay = hx * hz / (2.0 * hy), az = hx * hy / (2.0 * hz);
      for (int l = 0; l < nn; ++l) {
        rows[l].clear();
        const int nd = conn[li * nn + l];
        for (long long k = rs[nd]; k < rs[nd + 1]; ++k) rows[l].push_back({col[k], val[k]});
      }
      auto Ke = [&](int l, int m) {
        const int i1 = l % P1, i2 = (l / P1) % P1, i3 = l / (P1 * P1);
        const int j1 = m % P1, j2 = (m / P1) % P1, j3 = m / (P1 * P1);
        const double* K1 = o.tab.K1;
        const double* M1 = o.tab.M1;
        return ax * K1[i1 * P1 + j1] * M1[i2 * P1 + j2] * M1[i3 * P1 + j3] +
               ay * M1[i1 * P1 + j1] * K1[i2 * P1 + j2] * M1[i3 * P1 + j3] +
               az * M1[i1 * P1 + j1] * M1[i2 * P1 + j2] * K1[i3 * P1 + j3];
      };
      // group the leaf's (local node, weight) pairs by free index: diag[f] += sum over pairs of w w' K_e
      std::map<int, std::vector<std::pair<int, double>>> by_f;
      for (int l = 0; l < nn; ++l)
        for (const auto& a : rows[l]) by_f[a.first].push_back({l, a.second});
      for (const auto& kv : by_f)
        for (const auto& a : kv.second)
          for (const auto& b : kv.second) o.Kdiag[kv.first] += a.second * b.second * Ke(a.first, b.first);
    }
  }
  std::vector<double> geo(6 * leaves.size());
  o.quad_xyz.assign(leaves.size() * (size_t)o.nq * 3, 0.0);
  for (size_t li = 0; li < leaves.size(); ++li) {
    for (int a = 0; a < 3; ++a) {
      geo[6 * li + a] = leaves[li].x0[a];
      geo[6 * li + 3 + a] = leaves[li].h[a];
    }
    for (int q = 0; q < o.nq; ++q) {
      const int qi[3] = {q % n_quad, (q / n_quad) % n_quad, q / (n_quad * n_quad)};
      for (int a = 0; a < 3; ++a)
        o.quad_xyz[(li * o.nq + q) * 3 + a] = leaves[li].x0[a] + 0.5 * (xg[qi[a]] + 1.0) * leaves[li].h[a];
    }
  }
  o.all_xyz = xyz;
  o.n_leaves = (long long)leaves.size();
  o.n_all = n_all;
  o.n_free = n_free;
  o.n_hang = n_all - n_free;
  o.geo = std::move(geo);
  o.conn = std::move(conn);
  o.bnd = std::move(bnd);
  return EFE_OK;
}

// Host set-up, then the device copies.
static efe_status octree_build(Octree& o, const double* lo, const double* hi, int nc, int p, int n_quad,
                               const int32_t* refine, int n_refine) {
  efe_status st = octree_host(o, lo, hi, nc, p, n_quad, refine, n_refine);
  if (st != EFE_OK) return st;
  const std::vector<double>& geo = o.geo;
  const std::vector<int>& conn = o.conn;
  const std::vector<long long>& rs = o.rs;
  const std::vector<int>& col = o.col;
  const std::vector<double>& val = o.val;
  const std::vector<unsigned char>& bnd = o.bnd;
  auto up = [](auto*& dst, const auto& v) -> cudaError_t {
    using T = typename std::remove_reference<decltype(v)>::type::value_type;
    cudaError_t e = cudaMalloc((void**)&dst, sizeof(T) * std::max<size_t>(v.size(), 1));
    if (e != cudaSuccess) return e;
    return v.empty() ? cudaSuccess : cudaMemcpy(dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
  };
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = up(o.d_geo, geo);
  if (e == cudaSuccess) e = up(o.d_conn, conn);
  if (e == cudaSuccess) e = up(o.d_rs, rs);
  if (e == cudaSuccess) e = up(o.d_col, col);
  if (e == cudaSuccess) e = up(o.d_val, val);
  if (e == cudaSuccess) e = up(o.d_bnd, bnd);
  if (e == cudaSuccess) e = up(o.d_D, o.D);
  if (e == cudaSuccess) e = up(o.d_Kdiag, o.Kdiag);
  if (e != cudaSuccess) {
    o.err = std::string("octree set-up: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? EFE_ERR_NOMEM : EFE_ERR_CUDA;
  }
  return EFE_OK;
}

}  // namespace efe

namespace efe {
efe_status octree_apply(Octree& o, const double* vq_dev, double kin, const double* X_dev, double* Y_dev,
                        long long n_cols, int mask_boundary, cudaStream_t s);
}  // namespace efe

struct efe_octree {
  efe::Octree o;
};

static thread_local std::string g_oct_err;

extern "C" {

efe_status efe_octree_setup(const double* lo_host, const double* hi_host, int32_t nc, int32_t degree, int32_t n_quad,
                            const int32_t* refine_host, int32_t n_refine, efe_octree** out) {
  if (!out || !lo_host || !hi_host) return EFE_ERR_ARG;
  *out = nullptr;
  efe_octree* h = new efe_octree();
  efe_status st = efe::octree_build(h->o, lo_host, hi_host, nc, degree, n_quad, refine_host, n_refine);
  if (st != EFE_OK) {
    g_oct_err = h->o.err;
    delete h;
    return st;
  }
  *out = h;
  return EFE_OK;
}

efe_status efe_octree_constraints(const double* lo_host, const double* hi_host, int32_t nc, int32_t degree,
                                  int32_t n_quad, const int32_t* refine_host, int32_t n_refine, int64_t* n_all,
                                  int64_t* n_free, int64_t* nnz, int64_t* row_start, int32_t* col, double* val,
                                  double* all_xyz, double* free_xyz) {
  if (!lo_host || !hi_host) return EFE_ERR_ARG;
  efe::Octree o;
  efe_status st = efe::octree_host(o, lo_host, hi_host, nc, degree, n_quad, refine_host, n_refine);
  if (st != EFE_OK) {
    g_oct_err = o.err;
    return st;
  }
  if (n_all) *n_all = o.n_all;
  if (n_free) *n_free = o.n_free;
  if (nnz) *nnz = (int64_t)o.col.size();
  if (row_start) std::copy(o.rs.begin(), o.rs.end(), row_start);
  if (col) std::copy(o.col.begin(), o.col.end(), col);
  if (val) std::copy(o.val.begin(), o.val.end(), val);
  if (all_xyz) std::copy(o.all_xyz.begin(), o.all_xyz.end(), all_xyz);
  if (free_xyz) std::copy(o.free_xyz.begin(), o.free_xyz.end(), free_xyz);
  return EFE_OK;
}

efe_status efe_octree_destroy(efe_octree* oct) {
  delete oct;
  return EFE_OK;
}

const char* efe_octree_last_error(const efe_octree* oct) { return oct ? oct->o.err.c_str() : g_oct_err.c_str(); }

efe_status efe_octree_sizes(const efe_octree* oct, int64_t* n_free, int64_t* n_all, int64_t* n_leaves, int64_t* n_q,
                            int64_t* n_hanging) {
  if (!oct) return EFE_ERR_ARG;
  const efe::Octree& o = oct->o;
  if (n_free) *n_free = o.n_free;
  if (n_all) *n_all = o.n_all;
  if (n_leaves) *n_leaves = o.n_leaves;
  if (n_q) *n_q = o.nq;
  if (n_hanging) *n_hanging = o.n_hang;
  return EFE_OK;
}

efe_status efe_octree_coords(const efe_octree* oct, double* free_xyz_host, double* quad_xyz_host,
                             uint8_t* boundary_host) {
  if (!oct) return EFE_ERR_ARG;
  const efe::Octree& o = oct->o;
  if (free_xyz_host) std::copy(o.free_xyz.begin(), o.free_xyz.end(), free_xyz_host);
  if (quad_xyz_host) std::copy(o.quad_xyz.begin(), o.quad_xyz.end(), quad_xyz_host);
  if (boundary_host && cudaMemcpy(boundary_host, o.d_bnd, (size_t)o.n_free, cudaMemcpyDeviceToHost) != cudaSuccess)
    return EFE_ERR_CUDA;
  return EFE_OK;
}

efe_status efe_octree_apply(efe_octree* oct, const double* vq_dev, double kin, const double* X_dev, double* Y_dev,
                            int64_t n_cols, int32_t mask_boundary, void* stream) {
  if (!oct || !vq_dev || !X_dev || !Y_dev || n_cols < 1 || n_cols > 65535 || mask_boundary < 0 || mask_boundary > 2)
    return EFE_ERR_ARG;
  return efe::octree_apply(oct->o, vq_dev, kin, X_dev, Y_dev, n_cols, mask_boundary,
                           reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace efe {

// Y = P^T (kin K/2 + V) P X (V = 0 when vq is NULL).
efe_status octree_apply(Octree& o, const double* vq_dev, double kin, const double* X_dev, double* Y_dev,
                        long long n_cols, int mask_boundary, cudaStream_t s) {
  if (o.ws_cols < n_cols) {
    if (o.d_xall) cudaFree(o.d_xall);
    if (o.d_yall) cudaFree(o.d_yall);
    o.d_xall = o.d_yall = nullptr;
    o.ws_cols = 0;
    if (cudaMalloc(&o.d_xall, sizeof(double) * o.n_all * n_cols) != cudaSuccess ||
        cudaMalloc(&o.d_yall, sizeof(double) * o.n_all * n_cols) != cudaSuccess) {
      o.err = "octree apply: out of device memory";
      return EFE_ERR_NOMEM;
    }
    o.ws_cols = n_cols;
  }
  const int nc = (int)n_cols;
  const long long N = o.n_all * n_cols;
  const double* scale = mask_boundary == 2 ? o.d_D : nullptr;   // Loewdin: D = mask / sqrt(m_c) both sides
  const int mask = mask_boundary != 0;
  efe::k_oct_expand<<<efe::oblk(N), 256, 0, s>>>(o.d_rs, o.d_col, o.d_val, o.d_bnd, scale, X_dev, o.n_all, nc,
                                                 mask, o.d_xall);
  efe::note_launch();
  cudaMemsetAsync(o.d_yall, 0, sizeof(double) * N, s);
  dim3 grid((unsigned)o.n_leaves, (unsigned)nc);
  efe::k_oct_apply<<<grid, efe::kOctThreads, 0, s>>>(o.tab, o.d_geo, o.d_conn, vq_dev, kin, o.d_xall, nc, o.d_yall);
  efe::note_launch();
  cudaMemsetAsync(Y_dev, 0, sizeof(double) * o.n_free * n_cols, s);
  efe::k_oct_reduce<<<efe::oblk(N), 256, 0, s>>>(o.d_rs, o.d_col, o.d_val, o.d_bnd, scale, o.d_yall, o.n_all, nc,
                                                 mask, Y_dev);
  efe::note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    o.err = std::string("octree apply: ") + cudaGetErrorString(e);
    return EFE_ERR_CUDA;
  }
  return EFE_OK;
}

// -lap u = f with u = g on the boundary free nodes: K_II u_I = F_I - K_IB g_B, F = P^T int f N
// (F = P^T V P 1 with v = f: the constants are in the constrained space and the basis sums to 1),
// by conjugate gradients with the Jacobi preconditioner (the diagonal of P^T K P) to
// |r| <= tol |F_I - K_IB g_B|.
efe_status octree_poisson(Octree& o, const double* fq, const double* g, double* u, double tol, int max_it,
                          int* iters, cudaStream_t s) {
  const long long n = o.n_free;
  double* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * (7 * n + 4)) != cudaSuccess) {
    o.err = "octree Poisson: out of device memory";
    return EFE_ERR_NOMEM;
  }
  double *gB = buf, *ones = buf + n, *F = buf + 2 * n, *r = buf + 3 * n, *p = buf + 4 * n, *Ap = buf + 5 * n;
  double* z = buf + 6 * n;
  double* dots = buf + 7 * n;
  std::vector<double> hd(2);
  efe_status st = EFE_OK;
  auto fail = [&](cudaError_t e) {
    o.err = std::string("octree Poisson: ") + cudaGetErrorString(e);
    return EFE_ERR_CUDA;
  };
  auto dot = [&](const double* a, const double* b, double* out) {
    k_oct_dot<<<(unsigned)std::min<long long>(oblk(n), 1024), 256, 0, s>>>(a, b, n, out);
    note_launch();
  };
  int it = 0;
  bool conv = false;
  do {
    k_oct_bc<<<oblk(n), 256, 0, s>>>(g, o.d_bnd, n, gB, ones);
    note_launch();
    if ((st = octree_apply(o, fq, 0.0, ones, F, 1, 0, s)) != EFE_OK) break;    // F = P^T int f N
    if ((st = octree_apply(o, nullptr, 2.0, gB, Ap, 1, 0, s)) != EFE_OK) break; // K g_B
    k_oct_cg_start<<<oblk(n), 256, 0, s>>>(F, Ap, o.d_bnd, o.d_Kdiag, n, r, z, p, u);
    note_launch();
    cudaMemsetAsync(dots, 0, sizeof(double) * 4, s);
    dot(r, r, dots);
    dot(r, z, dots + 2);
    hd.resize(4);
    cudaError_t e = cudaMemcpyAsync(hd.data(), dots, sizeof(double) * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      st = fail(e);
      break;
    }
    const double rr0 = hd[0];
    double rz = hd[2];
    conv = rr0 == 0.0;
    while (!conv && it < max_it) {
      if ((st = octree_apply(o, nullptr, 2.0, p, Ap, 1, 1, s)) != EFE_OK) break;   // K_II p
      cudaMemsetAsync(dots, 0, sizeof(double), s);
      dot(p, Ap, dots);
      e = cudaMemcpyAsync(hd.data(), dots, sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess || !(hd[0] > 0.0)) {
        if (e != cudaSuccess) st = fail(e);
        else { o.err = "octree Poisson: the operator is not positive definite"; st = EFE_ERR_NOT_SPD; }
        break;
      }
      const double alpha = rz / hd[0];
      k_oct_cg_step<<<oblk(n), 256, 0, s>>>(u, r, p, Ap, alpha, n);
      note_launch();
      k_oct_precond<<<oblk(n), 256, 0, s>>>(r, o.d_Kdiag, o.d_bnd, n, z);
      note_launch();
      cudaMemsetAsync(dots + 1, 0, sizeof(double) * 3, s);
      dot(r, r, dots + 1);
      dot(r, z, dots + 3);
      e = cudaMemcpyAsync(hd.data() + 1, dots + 1, sizeof(double) * 3, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        st = fail(e);
        break;
      }
      const double rr_new = hd[1], rz_new = hd[3];
      ++it;
      conv = std::sqrt(rr_new) <= tol * std::sqrt(rr0);
      k_oct_cg_dir<<<oblk(n), 256, 0, s>>>(p, z, rz_new / rz, n);
      note_launch();
      rz = rz_new;
    }
    if (st != EFE_OK) break;
    k_oct_cg_finish<<<oblk(n), 256, 0, s>>>(u, g, o.d_bnd, n);
    note_launch();
    e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) st = fail(e);
  } while (false);
  cudaFree(buf);
  if (iters) *iters = it;
  if (st == EFE_OK && !conv) {
    o.err = "octree Poisson: no convergence within max_it";
    st = EFE_ERR_CG_NOCONV;
  }
  return st;
}

}  // namespace efe

extern "C" {

efe_status efe_octree_poisson(efe_octree* oct, const double* f_q_dev, const double* g_free_dev, double* u_dev,
                              double tol, int32_t max_it, int32_t* iters_host, void* stream) {
  if (!oct || !f_q_dev || !g_free_dev || !u_dev || !(tol > 0.0) || max_it < 1) return EFE_ERR_ARG;
  int its = 0;
  efe_status st = efe::octree_poisson(oct->o, f_q_dev, g_free_dev, u_dev, tol, max_it, &its,
                                      reinterpret_cast<cudaStream_t>(stream));
  if (iters_host) *iters_host = its;
  return st;
}

}  // extern "C"

extern "C" {

efe_status efe_octree_density(efe_octree* oct, const double* psi_bar_dev, int32_t n_orb, const double* occ_host,
                              double* rho_dev, void* stream) {
  if (!oct || !psi_bar_dev || !occ_host || !rho_dev || n_orb < 1 || 2 * n_orb > 65535) return EFE_ERR_ARG;
  efe::Octree& o = oct->o;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const long long nc2 = 2LL * n_orb;
  if (o.ws_cols < nc2) {
    if (o.d_xall) cudaFree(o.d_xall);
    if (o.d_yall) cudaFree(o.d_yall);
    o.d_xall = o.d_yall = nullptr;
    o.ws_cols = 0;
    if (cudaMalloc(&o.d_xall, sizeof(double) * o.n_all * nc2) != cudaSuccess ||
        cudaMalloc(&o.d_yall, sizeof(double) * o.n_all * nc2) != cudaSuccess) {
      o.err = "octree density: out of device memory";
      return EFE_ERR_NOMEM;
    }
    o.ws_cols = nc2;
  }
  double* d_occ = nullptr;
  if (cudaMalloc(&d_occ, sizeof(double) * n_orb) != cudaSuccess) {
    o.err = "octree density: out of device memory";
    return EFE_ERR_NOMEM;
  }
  cudaMemcpyAsync(d_occ, occ_host, sizeof(double) * n_orb, cudaMemcpyHostToDevice, s);
  const long long N = o.n_all * nc2;
  efe::k_oct_expand<<<efe::oblk(N), 256, 0, s>>>(o.d_rs, o.d_col, o.d_val, o.d_bnd, o.d_D, psi_bar_dev, o.n_all,
                                                 (int)nc2, 1, o.d_xall);
  efe::note_launch();
  efe::k_oct_density<<<(unsigned)o.n_leaves, efe::kOctThreads, 0, s>>>(o.tab, o.d_conn, o.d_xall, n_orb, d_occ,
                                                                       rho_dev);
  efe::note_launch();
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaFree(d_occ);
  if (e != cudaSuccess) {
    o.err = std::string("octree density: ") + cudaGetErrorString(e);
    return EFE_ERR_CUDA;
  }
  return EFE_OK;
}

}  // extern "C"

namespace efe {

// y = exp(-i dt T_m) e_1 for the m x m tridiagonal matrix (diagonal a, off-diagonal b) of one column
// by its eigendecomposition; false if the eigensolver did not converge
static bool tri_exp_host(int m, const double* a, const double* b, double dt, std::vector<double>& yre,
                         std::vector<double>& yim) {
  std::vector<double> T((size_t)m * m, 0.0), V, lam;
  for (int i = 0; i < m; ++i) {
    T[(size_t)i * m + i] = a[i];
    if (i + 1 < m) T[(size_t)i * m + i + 1] = T[(size_t)(i + 1) * m + i] = b[i];
  }
  if (!jacobi_eigen(m, T, V, lam)) return false;
  yre.assign(m, 0.0);
  yim.assign(m, 0.0);
  for (int i = 0; i < m; ++i)
    for (int q = 0; q < m; ++q) {
      const double v0 = V[(size_t)0 * m + q], vi = V[(size_t)i * m + q];
      yre[i] += vi * std::cos(-dt * lam[q]) * v0;
      yim[i] += vi * std::sin(-dt * lam[q]) * v0;
    }
  return true;
}

// psi <- exp(-i dt Hbar) psi per complex column by Lanczos steps (Eqs. AdaptiveKrylov,
// AdaptiveKrylovErr): Hbar = D P^T H P D (octree_apply mode 2), three-term recurrence, the exponential
// of the tridiagonal matrix by its eigendecomposition on the host, psi = |psi| Q_m y.  tol <= 0: every
// column takes k steps; tol > 0: a column stops at the first m <= k whose estimate
// eps_m = |dt| beta_m |psi| |[exp(-i dt T_m) e_1]_m| is at most tol (or whose recurrence breaks
// down), the others at k (counted in *caps); *k_used receives the largest m.
efe_status octree_kexp(Octree& o, const double* vq, double kin, double* psi, int C, double dt, int k, double tol,
                       int* k_used, int* caps, cudaStream_t s) {
  const long long n = o.n_free, N2 = n * 2 * C;
  double* Q = nullptr;
  double* small = nullptr;   // nrm[C], a[C], b[C], scratch[C], y[C][k][2]
  if (cudaMalloc(&Q, sizeof(double) * N2 * (k + 1)) != cudaSuccess ||
      cudaMalloc(&small, sizeof(double) * (4 * C + 2 * (size_t)C * k)) != cudaSuccess) {
    if (Q) cudaFree(Q);
    o.err = "octree exponential: out of device memory";
    return EFE_ERR_NOMEM;
  }
  double *nrm = small, *a = small + C, *b = small + 2 * C, *tmp = small + 3 * C, *ydev = small + 4 * C;
  std::vector<double> h_nrm(C), h_a((size_t)C * k), h_b((size_t)C * k), hv(C);
  efe_status st = EFE_OK;
  const dim3 dg((unsigned)C, 64);
  auto cdot = [&](const double* x, const double* y, double* out) {
    cudaMemsetAsync(out, 0, sizeof(double) * C, s);
    k_oct_cdot<<<dg, 256, 0, s>>>(x, y, n, C, out);
    note_launch();
  };
  auto to_host = [&](const double* d, std::vector<double>& h) {
    cudaError_t e = cudaMemcpyAsync(h.data(), d, sizeof(double) * C, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
  };
  do {
    // q_0 = psi / |psi| (boundary rows of psi zeroed first: they are not part of the space)
    k_oct_zero_bnd<<<oblk(N2), 256, 0, s>>>(psi, o.d_bnd, n, C);
    note_launch();
    cdot(psi, psi, nrm);
    if (to_host(nrm, h_nrm) != cudaSuccess) { st = EFE_ERR_CUDA; break; }
    for (int c = 0; c < C; ++c) {
      h_nrm[c] = std::sqrt(h_nrm[c]);
      hv[c] = h_nrm[c] > 0.0 ? 1.0 / h_nrm[c] : 0.0;
    }
    cudaMemcpyAsync(tmp, hv.data(), sizeof(double) * C, cudaMemcpyHostToDevice, s);
    k_oct_cscale<<<oblk(N2), 256, 0, s>>>(psi, tmp, n, C, Q);
    note_launch();
    // per column: the Lanczos dimension it stops at (0: still running) and its y at that point
    std::vector<int> mc(C, 0);
    std::vector<std::vector<double>> yre_c(C), yim_c(C);
    int n_run = C;
    for (int j = 0; j < k && st == EFE_OK && n_run > 0; ++j) {
      double* qj = Q + (long long)j * N2;
      double* w = Q + (long long)(j + 1) * N2;
      if ((st = octree_apply(o, vq, kin, qj, w, 2 * C, 2, s)) != EFE_OK) break;
      cdot(qj, w, a);
      if (to_host(a, hv) != cudaSuccess) { st = EFE_ERR_CUDA; break; }
      for (int c = 0; c < C; ++c) h_a[(size_t)c * k + j] = hv[c];
      k_oct_lz_update<<<oblk(N2), 256, 0, s>>>(w, qj, j > 0 ? Q + (long long)(j - 1) * N2 : nullptr, a, b, n, C);
      note_launch();
      cdot(w, w, tmp);
      if (to_host(tmp, hv) != cudaSuccess) { st = EFE_ERR_CUDA; break; }
      for (int c = 0; c < C; ++c) {
        const double beta = std::sqrt(std::max(hv[c], 0.0));
        h_b[(size_t)c * k + j] = beta;
        hv[c] = beta > 1e-300 ? 1.0 / beta : 0.0;   // invariant subspace: the rest of the basis is zero
      }
      if (tol > 0.0) {
        // the estimate of each running column at m = j + 1
        for (int c = 0; c < C && st == EFE_OK; ++c) {
          if (mc[c] != 0) continue;
          const int m = j + 1;
          const double bm = h_b[(size_t)c * k + j];
          std::vector<double> yr, yi;
          if (!tri_exp_host(m, &h_a[(size_t)c * k], &h_b[(size_t)c * k], dt, yr, yi)) {
            o.err = "octree exponential: tridiagonal eigensolver did not converge";
            st = EFE_ERR_CUDA;
            break;
          }
          const double eps = std::fabs(dt) * bm * h_nrm[c] * std::hypot(yr[m - 1], yi[m - 1]);
          if (eps <= tol || bm <= 1e-300 || h_nrm[c] == 0.0) {
            mc[c] = m;
            yre_c[c] = yr;
            yim_c[c] = yi;
            --n_run;
          }
        }
        if (st != EFE_OK) break;
      }
      std::vector<double> bj(C);
      for (int c = 0; c < C; ++c) bj[c] = h_b[(size_t)c * k + j];
      cudaMemcpyAsync(b, bj.data(), sizeof(double) * C, cudaMemcpyHostToDevice, s);
      cudaMemcpyAsync(tmp, hv.data(), sizeof(double) * C, cudaMemcpyHostToDevice, s);
      if (j + 1 < k) {
        k_oct_cscale<<<oblk(N2), 256, 0, s>>>(w, tmp, n, C, w);
        note_launch();
      }
    }
    if (st != EFE_OK) break;
    // y = |psi| exp(-i dt T_m) e_1 for each column's m x m tridiagonal matrix (zero past m), columns
    // that did not stop taking m = k
    std::vector<double> y((size_t)C * k * 2, 0.0);
    int kmax = 0, ncap = 0;
    for (int c = 0; c < C; ++c) {
      if (mc[c] == 0) {
        mc[c] = k;
        if (tol > 0.0) ++ncap;
        if (!tri_exp_host(k, &h_a[(size_t)c * k], &h_b[(size_t)c * k], dt, yre_c[c], yim_c[c])) {
          o.err = "octree exponential: tridiagonal eigensolver did not converge";
          st = EFE_ERR_CUDA;
          break;
        }
      }
      kmax = std::max(kmax, mc[c]);
      for (int i = 0; i < mc[c]; ++i) {
        y[((size_t)c * k + i) * 2] = h_nrm[c] * yre_c[c][i];
        y[((size_t)c * k + i) * 2 + 1] = h_nrm[c] * yim_c[c][i];
      }
    }
    if (st != EFE_OK) break;
    if (k_used) *k_used = kmax;
    if (caps) *caps = ncap;
    cudaMemcpyAsync(ydev, y.data(), sizeof(double) * y.size(), cudaMemcpyHostToDevice, s);
    k_oct_lz_combine<<<oblk(n * C), 256, 0, s>>>(Q, ydev, kmax, k, n, C, psi);
    note_launch();
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) st = EFE_ERR_CUDA;
  } while (false);
  if (st == EFE_ERR_CUDA && o.err.empty()) o.err = "octree exponential: CUDA error";
  cudaFree(Q);
  cudaFree(small);
  return st;
}

}  // namespace efe

extern "C" {

efe_status efe_octree_kexp(efe_octree* oct, const double* vq_dev, double kin, double* psi_bar_dev, int32_t n_cols,
                           double dt, int32_t k, double tol, int32_t* k_used_host, void* stream) {
  if (!oct || !vq_dev || !psi_bar_dev || n_cols < 1 || 2 * n_cols > 65535 || k < 1 || k > 64 || !std::isfinite(tol))
    return EFE_ERR_ARG;
  int ku = 0, caps = 0;
  const efe_status st = efe::octree_kexp(oct->o, vq_dev, kin, psi_bar_dev, n_cols, dt, k, tol, &ku, &caps,
                                         reinterpret_cast<cudaStream_t>(stream));
  if (k_used_host) *k_used_host = ku;
  if (st == EFE_OK && caps > 0) return EFE_WARN_KRYLOV_CAP;
  return st;
}

}  // extern "C"

extern "C" {

efe_status efe_octree_interp(efe_octree* oct, const double* u_free_dev, int32_t n_cols, double* out_q_dev,
                             void* stream) {
  if (!oct || !u_free_dev || !out_q_dev || n_cols < 1 || n_cols > 65535) return EFE_ERR_ARG;
  efe::Octree& o = oct->o;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (o.ws_cols < n_cols) {
    if (o.d_xall) cudaFree(o.d_xall);
    if (o.d_yall) cudaFree(o.d_yall);
    o.d_xall = o.d_yall = nullptr;
    o.ws_cols = 0;
    if (cudaMalloc(&o.d_xall, sizeof(double) * o.n_all * n_cols) != cudaSuccess ||
        cudaMalloc(&o.d_yall, sizeof(double) * o.n_all * n_cols) != cudaSuccess) {
      o.err = "octree interpolation: out of device memory";
      return EFE_ERR_NOMEM;
    }
    o.ws_cols = n_cols;
  }
  const long long N = o.n_all * n_cols;
  efe::k_oct_expand<<<efe::oblk(N), 256, 0, s>>>(o.d_rs, o.d_col, o.d_val, o.d_bnd, nullptr, u_free_dev, o.n_all,
                                                 n_cols, 0, o.d_xall);
  efe::note_launch();
  efe::k_oct_interp<<<(unsigned)o.n_leaves, efe::kOctThreads, 0, s>>>(o.tab, o.d_conn, o.d_xall, n_cols, o.n_leaves,
                                                                      out_q_dev);
  efe::note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    o.err = std::string("octree interpolation: ") + cudaGetErrorString(e);
    return EFE_ERR_CUDA;
  }
  return EFE_OK;
}

}  // extern "C"

extern "C" efe_status efe_lda_points(const double* rho_dev, double* vxc_dev, double* exc_dev, int64_t n, int32_t xc,
                                     void* stream);
extern "C" efe_status efe_octree_density(efe_octree* oct, const double* psi_bar_dev, int32_t n_orb,
                                         const double* occ_host, double* rho_dev, void* stream);
extern "C" efe_status efe_octree_interp(efe_octree* oct, const double* u_free_dev, int32_t n_cols, double* out_q_dev,
                                        void* stream);

namespace efe {

// One predictor-corrector step (Eq. ApproxMagnus) on the locally refined mesh with the field E at the
// mid-point and a fixed Krylov dimension: psi_p = exp(-i dt Hbar[v(rho_n)]) psi_n,
// rho_mid = (rho_n + rho(psi_p)) / 2, psi_n+1 = exp(-i dt Hbar[v(rho_mid)]) psi_n, with
// v = -sum Z / |x - R| + v_H + v_xc - E . x at the leaves' Gauss-Legendre points and v_H from
// -lap v_H = 4 pi rho with the Dirichlet data sum Z / |x - R|.
static efe_status octree_step(efe_octree* oct, double* psi, int n_orb, const double* occ, const double* atoms,
                              int n_atoms, const double E[3], double dt, int k, double ktol, double cg_tol, int xc,
                              cudaStream_t s) {
  Octree& o = oct->o;
  const long long nq = o.n_leaves * o.nq, nf = o.n_free, N2 = nf * 2 * n_orb;
  // host: v_N and the field potential at the points, the Dirichlet data at the free nodes
  std::vector<double> vNf(2 * (size_t)nq), g((size_t)nf, 0.0);
  for (long long m = 0; m < nq; ++m) {
    const double* x = &o.quad_xyz[3 * m];
    double v = 0.0;
    for (int a = 0; a < n_atoms; ++a) {
      const double dx = x[0] - atoms[4 * a + 1], dy = x[1] - atoms[4 * a + 2], dz = x[2] - atoms[4 * a + 3];
      v -= atoms[4 * a] / std::sqrt(dx * dx + dy * dy + dz * dz);
    }
    vNf[m] = v;
    vNf[nq + m] = -(E[0] * x[0] + E[1] * x[1] + E[2] * x[2]);
  }
  for (long long f = 0; f < nf; ++f) {
    double v = 0.0;
    for (int a = 0; a < n_atoms; ++a) {
      const double dx = o.free_xyz[3 * f] - atoms[4 * a + 1], dy = o.free_xyz[3 * f + 1] - atoms[4 * a + 2],
                   dz = o.free_xyz[3 * f + 2] - atoms[4 * a + 3];
      v += atoms[4 * a] / std::sqrt(dx * dx + dy * dy + dz * dz);
    }
    g[f] = v;
  }
  double* buf = nullptr;
  const size_t nbuf = 8 * (size_t)nq + 2 * (size_t)nf + (size_t)N2;
  if (cudaMalloc(&buf, sizeof(double) * nbuf) != cudaSuccess) {
    o.err = "octree step: out of device memory";
    return EFE_ERR_NOMEM;
  }
  double *vN = buf, *vf = buf + nq, *rho_n = buf + 2 * nq, *rho = buf + 3 * nq, *vH = buf + 4 * nq;
  double *vxc = buf + 5 * nq, *v = buf + 6 * nq, *fq = buf + 7 * nq, *gd = buf + 8 * nq, *u = gd + nf;
  double* psi_p = u + nf;
  efe_status st = EFE_OK;
  auto potential = [&](const double* r) -> efe_status {
    k_oct_axpby<<<oblk(nq), 256, 0, s>>>(r, r, 4.0 * 3.14159265358979323846, 0.0, nq, fq);
    note_launch();
    int its = 0;
    efe_status e = octree_poisson(o, fq, gd, u, cg_tol, 100000, &its, s);
    if (e != EFE_OK) return e;
    if ((e = efe_octree_interp(oct, u, 1, vH, s)) != EFE_OK) return e;
    if ((e = efe_lda_points(r, vxc, nullptr, nq, xc, s)) != EFE_OK) return e;
    k_oct_vsum<<<oblk(nq), 256, 0, s>>>(vN, vH, vxc, vf, nq, v);
    note_launch();
    return EFE_OK;
  };
  cudaError_t ce = cudaSuccess;
  do {
    if ((ce = cudaMemcpyAsync(vN, vNf.data(), sizeof(double) * 2 * nq, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (ce = cudaMemcpyAsync(gd, g.data(), sizeof(double) * nf, cudaMemcpyHostToDevice, s)) != cudaSuccess)
      break;
    if ((st = efe_octree_density(oct, psi, n_orb, occ, rho_n, s)) != EFE_OK) break;
    if ((st = potential(rho_n)) != EFE_OK) break;
    if ((ce = cudaMemcpyAsync(psi_p, psi, sizeof(double) * N2, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) break;
    if ((st = octree_kexp(o, v, 1.0, psi_p, n_orb, dt, k, ktol, nullptr, nullptr, s)) != EFE_OK) break;
    if ((st = efe_octree_density(oct, psi_p, n_orb, occ, rho, s)) != EFE_OK) break;
    k_oct_axpby<<<oblk(nq), 256, 0, s>>>(rho_n, rho, 0.5, 0.5, nq, rho);
    note_launch();
    if ((st = potential(rho)) != EFE_OK) break;
    st = octree_kexp(o, v, 1.0, psi, n_orb, dt, k, ktol, nullptr, nullptr, s);
  } while (false);
  // the host vectors vNf and g must outlive the copies, and a kernel fault of the last launches
  // surfaces only here: both need the synchronisation before the status is final
  const cudaError_t se = cudaStreamSynchronize(s);
  if (ce == cudaSuccess) ce = se;
  if (ce == cudaSuccess) ce = cudaGetLastError();
  cudaFree(buf);
  if (st == EFE_OK && ce != cudaSuccess) {
    o.err = std::string("octree step: ") + cudaGetErrorString(ce);
    st = EFE_ERR_CUDA;
  }
  return st;
}

}  // namespace efe

extern "C" efe_status efe_octree_magnus_step(efe_octree* oct, double* psi_bar_dev, int32_t n_orb, const double* occ_host,
                                             const double* atoms_host, int32_t n_atoms, const double* field_host,
                                             double dt, int32_t k, double krylov_tol, double cg_tol, int32_t xc,
                                             void* stream) {
  if (!oct) return EFE_ERR_ARG;
  if (!psi_bar_dev || !occ_host || (n_atoms > 0 && !atoms_host) || n_atoms < 0 || !field_host || n_orb < 1 ||
      2 * n_orb > 65535 || k < 1 || k > 64 || !(cg_tol > 0.0) || !std::isfinite(dt) || !(dt > 0.0) ||
      !std::isfinite(krylov_tol) || (xc != EFE_XC_PW92 && xc != EFE_XC_PZ81)) {
    oct->o.err = "efe_octree_magnus_step: bad arguments (null pointer, n_orb outside 1..32767, k outside 1..64, "
                 "cg_tol <= 0, dt not finite and > 0, krylov_tol not finite, or an unknown xc)";
    return EFE_ERR_ARG;
  }
  return efe::octree_step(oct, psi_bar_dev, n_orb, occ_host, atoms_host, n_atoms, field_host, dt, k, krylov_tol,
                          cg_tol, xc, reinterpret_cast<cudaStream_t>(stream));
}
