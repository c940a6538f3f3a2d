// Direct Hartree solve by fast diagonalisation (Eqs. Hartree_possion,
// DiscretePoisson).
//
// On a rectilinear mesh with tensor-product GLL bases the exact stiffness is a
// Kronecker sum, A = (1/4pi)(K_x (x) M_y (x) M_z + M_x (x) K_y (x) M_z +
// M_x (x) M_y (x) K_z), with K_a, M_a the assembled 1D stiffness and
// (consistent) mass matrices restricted to interior nodes.  With the 1D
// generalised eigenvectors V_a^T K_a V_a = diag(lam_a), V_a^T M_a V_a = I,
//   A^-1 = (V_x (x) V_y (x) V_z) diag(4pi / (lam_x + lam_y + lam_z)) (V_x (x) V_y (x) V_z)^T,
// so the interior system A_II phi_I = d_I - A_IB phi_B is solved exactly (to
// rounding) by six dense mode products and one diagonal scaling: the same
// discrete problem the Jacobi-PCG path iterates on.
#include <cmath>
#include <vector>

#include "efe_internal.h"

namespace efe {

// ---------------------------------------------------------------------------- batched DGEMM
// C[b] = opA(A[b]) opB(B[b]); opA[m][k] = TA ? A[k lda + m] : A[m lda + k]; opB likewise.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_dgemm(int M, int N, int K, const double* __restrict__ A, long long lda,
                                               long long sA, const double* __restrict__ B, long long ldb,
                                               long long sB, double* __restrict__ C, long long ldc, long long sC) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int b = blockIdx.z;
  A += b * sA;
  B += b * sB;
  C += b * sC;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int i = threadIdx.x; i < BK * BM; i += 256) {
      int kk, mm;
      if (TA) { mm = i % BM; kk = i / BM; } else { kk = i % BK; mm = i / BK; }
      const int m = m0 + mm, k = k0 + kk;
      double v = 0.0;
      if (m < M && k < K) v = TA ? A[(long long)k * lda + m] : A[(long long)m * lda + k];
      As[kk][mm] = v;
    }
    for (int i = threadIdx.x; i < BK * BN; i += 256) {
      int kk, nn;
      if (TB) { kk = i % BK; nn = i / BK; } else { nn = i % BN; kk = i / BN; }
      const int n = n0 + nn, k = k0 + kk;
      double v = 0.0;
      if (n < N && k < K) v = TB ? B[(long long)n * ldb + k] : B[(long long)k * ldb + n];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n < N) C[(long long)m * ldc + n] = acc[i][j];
    }
  }
}

template <bool TA, bool TB>
static cudaError_t dgemm(int M, int N, int K, const double* A, long long lda, long long sA, const double* B,
                         long long ldb, long long sB, double* C, long long ldc, long long sC, int batch,
                         cudaStream_t s) {
  dim3 grid((N + 63) / 64, (M + 63) / 64, batch);
  k_dgemm<TA, TB><<<grid, 256, 0, s>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------- gather / scatter
// t[m][iz][iy][ix] = r[g(interior ix, iy, iz)][m], interior grid nx*ny*nz
__global__ void k_fdm_gather(const double* __restrict__ d, const double* __restrict__ Ap, long long Nx, long long Ny,
                             int nx, int ny, int nz, int nb, double* __restrict__ t) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n = (long long)nx * ny * nz;
  if (idx >= n * nb) return;
  const int m = (int)(idx / n);
  const long long i = idx % n;
  const long long ix = i % nx, iy = (i / nx) % ny, iz = i / ((long long)nx * ny);
  const long long g = (ix + 1) + Nx * ((iy + 1) + Ny * (iz + 1));
  t[idx] = d[g * nb + m] - Ap[g * nb + m];
}

__global__ void k_fdm_scale(double* __restrict__ t, const double* __restrict__ lx, const double* __restrict__ ly,
                            const double* __restrict__ lz, int nx, int ny, int nz, int nb, double four_pi) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n = (long long)nx * ny * nz;
  if (idx >= n * nb) return;
  const long long i = idx % n;
  const int ix = (int)(i % nx), iy = (int)((i / nx) % ny), iz = (int)(i / ((long long)nx * ny));
  t[idx] *= four_pi / (lx[ix] + ly[iy] + lz[iz]);
}

// phi[g][m] = phiB[g] on boundary nodes, u[m][interior index] inside
__global__ void k_fdm_scatter(const double* __restrict__ u, const double* __restrict__ phiB, long long n_h,
                              long long Nx, long long Ny, int nx, int ny, int nz, int nb, double* __restrict__ phi) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n_h * nb) return;
  const long long g = idx / nb;
  const int m = (int)(idx % nb);
  const long long ix = g % Nx, iy = (g / Nx) % Ny, iz = g / (Nx * Ny);
  double v = phiB ? phiB[g] : 0.0;
  if (ix > 0 && iy > 0 && iz > 0 && ix < nx + 1 && iy < ny + 1 && iz < nz + 1) {
    const long long i = (ix - 1) + nx * ((iy - 1) + (long long)ny * (iz - 1));
    v = u[(long long)m * nx * ny * nz + i];
  }
  phi[idx] = v;
}

// ---------------------------------------------------------------------------- set-up
// 1D assembled stiffness / mass on one axis, restricted to interior nodes,
// and the generalised eigendecomposition K V = M V diag(lam), V^T M V = I.
static bool axis_eigen(const Ctx& c, const std::vector<double>& b, std::vector<double>& V, std::vector<double>& lam) {
  const int ncell = (int)b.size() - 1;
  const int N = ncell * c.p + 1;
  const int n = N - 2;
  std::vector<double> K((size_t)N * N, 0.0), M((size_t)N * N, 0.0);
  for (int k = 0; k < ncell; ++k) {
    const double h = b[k + 1] - b[k];
    for (int i = 0; i < c.P1; ++i)
      for (int j = 0; j < c.P1; ++j) {
        const int gi = k * c.p + i, gj = k * c.p + j;
        K[(size_t)gi * N + gj] += 2.0 / h * c.tab.K1[i * c.P1 + j];
        M[(size_t)gi * N + gj] += 0.5 * h * c.tab.M1[i * c.P1 + j];
      }
  }
  std::vector<double> Ki((size_t)n * n), Mi((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      Ki[(size_t)i * n + j] = K[(size_t)(i + 1) * N + (j + 1)];
      Mi[(size_t)i * n + j] = M[(size_t)(i + 1) * N + (j + 1)];
    }
  // Cholesky M = L L^T
  std::vector<double> L((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = Mi[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) s -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      if (i == j) {
        if (!(s > 0.0)) return false;
        L[(size_t)i * n + i] = std::sqrt(s);
      } else {
        L[(size_t)i * n + j] = s / L[(size_t)j * n + j];
      }
    }
  // W = L^-1 K, then C = W L^-T (forward substitution on rows and columns)
  std::vector<double> W((size_t)n * n), Cm((size_t)n * n);
  for (int col = 0; col < n; ++col)
    for (int i = 0; i < n; ++i) {
      double s = Ki[(size_t)i * n + col];
      for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * W[(size_t)k * n + col];
      W[(size_t)i * n + col] = s / L[(size_t)i * n + i];
    }
  for (int row = 0; row < n; ++row)
    for (int j = 0; j < n; ++j) {
      double s = W[(size_t)row * n + j];
      for (int k = 0; k < j; ++k) s -= Cm[(size_t)row * n + k] * L[(size_t)j * n + k];
      Cm[(size_t)row * n + j] = s / L[(size_t)j * n + j];
    }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) {
      const double a = 0.5 * (Cm[(size_t)i * n + j] + Cm[(size_t)j * n + i]);
      Cm[(size_t)i * n + j] = Cm[(size_t)j * n + i] = a;
    }
  std::vector<double> U;
  if (!jacobi_eigen(n, Cm, U, lam)) return false;
  // V = L^-T U (back substitution per column)
  V.assign((size_t)n * n, 0.0);
  for (int col = 0; col < n; ++col)
    for (int i = n - 1; i >= 0; --i) {
      double s = U[(size_t)i * n + col];
      for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * V[(size_t)k * n + col];
      V[(size_t)i * n + col] = s / L[(size_t)i * n + i];
    }
  return true;
}

cudaError_t setup_fdm(Ctx& c) {
  const std::vector<double>* bb[3] = {&c.xb, &c.yb, &c.zb};
  for (int a = 0; a < 3; ++a) {
    std::vector<double> V, lam;
    if (!axis_eigen(c, *bb[a], V, lam)) return cudaErrorInvalidValue;
    c.fdm_n[a] = (int)lam.size();
    EFE_CUDA_TRY(cudaMalloc(&c.d_fdmV[a], sizeof(double) * V.size()));
    EFE_CUDA_TRY(cudaMalloc(&c.d_fdmL[a], sizeof(double) * lam.size()));
    EFE_CUDA_TRY(cudaMemcpy(c.d_fdmV[a], V.data(), sizeof(double) * V.size(), cudaMemcpyHostToDevice));
    EFE_CUDA_TRY(cudaMemcpy(c.d_fdmL[a], lam.data(), sizeof(double) * lam.size(), cudaMemcpyHostToDevice));
  }
  const long long n = (long long)c.fdm_n[0] * c.fdm_n[1] * c.fdm_n[2];
  EFE_CUDA_TRY(cudaMalloc(&c.d_fdmT, sizeof(double) * 2 * n * c.batch));
  return cudaSuccess;
}

// phi (n_h x nb) <- solution of the Dirichlet problem for the load vector d;
// Ap is scratch (n_h x nb).  Boundary data: zero if homogeneous, else phiB
// (n_h, nb == 1) when given, else the context's Hartree data.
cudaError_t fdm_solve(Ctx& c, const double* d, double* Ap, double* phi, int nb, cudaStream_t s, bool homogeneous,
                      const double* phiB) {
  if (phiB && nb != 1) return cudaErrorInvalidValue;
  const double scale = 1.0 / (2.0 * 3.14159265358979323846);
  const int nx = c.fdm_n[0], ny = c.fdm_n[1], nz = c.fdm_n[2];
  const long long n = (long long)nx * ny * nz;
  double* t0 = c.d_fdmT;
  double* t1 = c.d_fdmT + n * nb;
  const double *Vx = c.d_fdmV[0], *Vy = c.d_fdmV[1], *Vz = c.d_fdmV[2];
  // Ap = A phi_B (output on interior nodes only)
  EFE_CUDA_TRY(cudaMemsetAsync(Ap, 0, sizeof(double) * c.n_h * nb, s));
  if (!homogeneous) EFE_CUDA_TRY(launch_laplace(c, phiB ? phiB : c.d_phiB_nb, Ap, nb, 0, scale, s));
  const unsigned g1 = (unsigned)((n * nb + 255) / 256);
  k_fdm_gather<<<g1, 256, 0, s>>>(d, Ap, c.Nx, c.Ny, nx, ny, nz, nb, t0);
  note_launch();
  EFE_CUDA_TRY(cudaGetLastError());
  for (int m = 0; m < nb; ++m) {
    double* a = t0 + m * n;
    double* b = t1 + m * n;
    // forward: hat = (Vx (x) Vy (x) Vz)^T r
    EFE_CUDA_TRY((dgemm<false, false>(ny * nz, nx, nx, a, nx, 0, Vx, nx, 0, b, nx, 0, 1, s)));          // x
    EFE_CUDA_TRY((dgemm<true, false>(ny, nx, ny, Vy, ny, 0, b, nx, (long long)ny * nx, a, nx, (long long)ny * nx,
                                     nz, s)));                                                          // y
    EFE_CUDA_TRY((dgemm<true, false>(nz, nx * ny, nz, Vz, nz, 0, a, (long long)nx * ny, 0, b, (long long)nx * ny,
                                     0, 1, s)));                                                        // z
    k_fdm_scale<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(b, c.d_fdmL[0], c.d_fdmL[1], c.d_fdmL[2], nx, ny, nz,
                                                          1, 4.0 * 3.14159265358979323846);
    note_launch();
    // backward: u = (Vx (x) Vy (x) Vz) hat
    EFE_CUDA_TRY((dgemm<false, false>(nz, nx * ny, nz, Vz, nz, 0, b, (long long)nx * ny, 0, a, (long long)nx * ny,
                                      0, 1, s)));                                                       // z
    EFE_CUDA_TRY((dgemm<false, false>(ny, nx, ny, Vy, ny, 0, a, nx, (long long)ny * nx, b, nx, (long long)ny * nx,
                                      nz, s)));                                                         // y
    EFE_CUDA_TRY((dgemm<false, true>(ny * nz, nx, nx, b, nx, 0, Vx, nx, 0, a, nx, 0, 1, s)));           // x
  }
  k_fdm_scatter<<<(unsigned)((c.n_h * nb + 255) / 256), 256, 0, s>>>(t0, homogeneous ? nullptr : (phiB ? phiB : c.d_phiB), c.n_h,
                                                                    c.Nx, c.Ny, nx, ny, nz, nb, phi);
  note_launch();
  return cudaGetLastError();
}

}  // namespace efe
