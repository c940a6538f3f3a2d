// The EFE Hamiltonian apply and the cell-local operators built on it.
//
// Hbar = M^-1/2 H M^-1/2 (Eq. TDKSDiscrete2) with H = P^T H_ext P (Eqs. Hmn,
// EFESplit, EFEOrtho) is applied as
//   x^C = D x_bar^C, x^E = S x_bar^E                 D = mask / sqrt(M^cc), S = (M^ee)^-1/2
//   y^C = sum_c G_c^T (H_c G_c x^C + E_c x^E)        cell gather / contraction / scatter-add
//   y^E = sum_c E_c^T G_c x^C + H_EE x^E              enrichment coupling
//   y_bar^C = D y^C, y_bar^E = S y^E
// where H_c is the classical cell matrix (kinetic + v-weighted mass, applied by
// sum factorisation), E_c = 1/2 int grad N_i . grad N^E_nu + int v N_i N^E_nu is
// the cell's classical-enriched block for the orthogonalised enrichment
// functions N^E = N^A - sum_l c_l N^C_l, and H_EE the enriched-enriched block.
// These are P^T H_ext P written out block by block, so no P is applied at run time.
#include <cstdio>
#include <mutex>
#include <string>
#include <type_traits>

#include "efe_internal.h"
#include "sumfact.cuh"

namespace efe {

// Slots per tile from the shared-memory budget: four tile buffers of
// NQ1^3 * RT entries of T in ~110 KB, so two blocks fit on one SM.
template <typename T, int NQ1>
constexpr int tile_rt() {
  return (110 * 1024) / (4 * NQ1 * NQ1 * NQ1 * (int)sizeof(T)) >= 32   ? 32
         : (110 * 1024) / (4 * NQ1 * NQ1 * NQ1 * (int)sizeof(T)) >= 16 ? 16
         : (110 * 1024) / (4 * NQ1 * NQ1 * NQ1 * (int)sizeof(T)) >= 8  ? 8
                                                                         : 4;
}

template <typename T, int NQ1, int RT = tile_rt<T, NQ1>()>
constexpr size_t tile_smem() {
  return (size_t)4 * NQ1 * NQ1 * NQ1 * RT * sizeof(T) + 3 * 32 * sizeof(T);   // tiles + k_laplace's factors
}

// ----------------------------------------------------------------------------
// cell apply: one block per (cell, batch member); the block walks the member's
// real columns in tiles of RT slots.
// ----------------------------------------------------------------------------
template <typename T, int P1, int NQ1, bool ENR, int RT = tile_rt<T, NQ1>()>
__global__ void __launch_bounds__(kThreads)
k_cell_apply(const __grid_constant__ RefTables tab, const MeshView mesh, const double* __restrict__ X,
             double* __restrict__ Y, long long ld2, int cols_member,
             const double* __restrict__ Dsc, const T* __restrict__ W, double kin, const int* __restrict__ pair_start,
             const int* __restrict__ pair_fn, const T* __restrict__ E, long long n_pairs,
             const T* __restrict__ xE, double* __restrict__ yE, const int* __restrict__ gate = nullptr) {
  constexpr int S3 = NQ1 * NQ1 * NQ1;
  constexpr int NN = P1 * P1 * P1;
  constexpr int NQ = S3;
  // coupling rows staged per chunk: kc * NN entries of E_c and kc * RT of x^E
  constexpr int KCAP = (S3 * RT) / NN < S3 ? (S3 * RT) / NN : S3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);
  T* B = A + S3 * RT;
  T* C = B + S3 * RT;
  T* D = C + S3 * RT;

  if (gate && *gate == 0) return;   // every Lanczos column has converged (graph-captured loops)
  const int c = blockIdx.x;
  const int member = blockIdx.y;
  int cx, cy, cz;
  cell_ijk(mesh, c, cx, cy, cz);
  T kx, ky, kz;   // kinetic factors hy hz / (4 hx) etc.
  {
    const double hx = mesh.h[cx], hy = mesh.h[mesh.ncx + cy], hz = mesh.h[mesh.ncx + mesh.ncy + cz];
    kx = from_f64<T>(kin * hy * hz / (4.0 * hx));
    ky = from_f64<T>(kin * hx * hz / (4.0 * hy));
    kz = from_f64<T>(kin * hx * hy / (4.0 * hz));
  }
  const T* Wc = W + ((long long)member * mesh.nc + c) * NQ;
  int p0 = 0, np = 0;
  if (ENR) {
    p0 = pair_start[c];
    np = pair_start[c + 1] - p0;
  }
  const T* Ec = ENR ? E + ((long long)member * n_pairs + p0) * NN : nullptr;
  const int col0 = member * cols_member;
  const int n_tiles = (cols_member + RT - 1) / RT;

  for (int tile = 0; tile < n_tiles; ++tile) {
    const int cbase = tile * RT;
    // gather x^C = D x_bar^C into A
    for (int it = threadIdx.x; it < NN * RT; it += blockDim.x) {
      const int r = it % RT, l = it / RT;
      const int i1 = l % P1, i2 = (l / P1) % P1, i3 = l / (P1 * P1);
      const long long g = node_index(mesh, cx, cy, cz, i1, i2, i3);
      T v = T(0);
      if (cbase + r < cols_member) v = from_f64_split<T>(X[g * ld2 + col0 + cbase + r] * Dsc[g]);
      A[it] = v;
    }
    __syncthreads();
    if (ENR && np > 0) {
      // y^E += E_c^T x^C while x^C is still in A (E_c rows staged in C)
      for (int k0 = 0; k0 < np; k0 += KCAP) {
        const int kc = np - k0 < KCAP ? np - k0 : KCAP;
        for (int i = threadIdx.x; i < kc * NN; i += blockDim.x) C[i] = Ec[(long long)k0 * NN + i];
        __syncthreads();
        for (int it = threadIdx.x; it < kc * RT; it += blockDim.x) {
          const int r = it % RT, k = it / RT;
          if (cbase + r >= cols_member) continue;
          const T* e = C + k * NN;
          T acc = T(0);
#pragma unroll 5
          for (int l = 0; l < NN; ++l) acc = fma(e[l], A[l * RT + r], acc);
          atomicAdd(&yE[(long long)pair_fn[p0 + k0 + k] * ld2 + col0 + cbase + r], to_f64<T>(acc));
        }
        __syncthreads();
      }
    }
    // classical cell operator: y^C = H_c x^C into D
    cell_operator_tile<T, P1, NQ1, RT>(tab, A, B, C, D, Wc, kx, ky, kz);
    if (ENR && np > 0) {
      // y^C += E_c x^E, with E_c rows staged in B and x^E in C
      for (int k0 = 0; k0 < np; k0 += KCAP) {
        const int kc = np - k0 < KCAP ? np - k0 : KCAP;
        for (int i = threadIdx.x; i < kc * NN; i += blockDim.x) B[i] = Ec[(long long)k0 * NN + i];
        for (int i = threadIdx.x; i < kc * RT; i += blockDim.x) {
          const int r = i % RT, k = i / RT;
          C[i] = (cbase + r < cols_member) ? xE[(long long)pair_fn[p0 + k0 + k] * ld2 + col0 + cbase + r] : T(0);
        }
        __syncthreads();
        for (int it = threadIdx.x; it < NN * RT; it += blockDim.x) {
          const int r = it % RT, l = it / RT;
          T acc = T(0);
          for (int k = 0; k < kc; ++k) acc = fma(B[k * NN + l], C[k * RT + r], acc);
          D[it] += fin(acc);
        }
        __syncthreads();
      }
    }
    // scatter-add y_bar^C += D y^C
    for (int it = threadIdx.x; it < NN * RT; it += blockDim.x) {
      const int r = it % RT, l = it / RT;
      if (cbase + r >= cols_member) continue;
      const int i1 = l % P1, i2 = (l / P1) % P1, i3 = l / (P1 * P1);
      const long long g = node_index(mesh, cx, cy, cz, i1, i2, i3);
      const double d = Dsc[g];
      if (d != 0.0) atomicAdd(&Y[g * ld2 + col0 + cbase + r], d * to_f64<T>(D[it]));
    }
    __syncthreads();
  }
}

// xE[nu][col] = sum_mu S[nu][mu] X[n_h + mu][col]  (and float and pair copies; xE2 may be NULL)
__global__ void k_enr_pre(const double* __restrict__ S, const double* __restrict__ X, long long n_h, long long ld2,
                          int ncols2, int nE, double* __restrict__ xE, float* __restrict__ xE32,
                          df32* __restrict__ xE2 = nullptr) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)nE * ncols2) return;
  int nu = idx / ncols2, col = idx % ncols2;
  double acc = 0.0;
  for (int mu = 0; mu < nE; ++mu) acc += S[nu * nE + mu] * X[(n_h + mu) * ld2 + col];
  xE[nu * ld2 + col] = acc;
  xE32[nu * ld2 + col] = (float)acc;
  if (xE2) {
    const float h = (float)acc;
    xE2[nu * ld2 + col] = df32(h, (float)(acc - (double)h));
  }
}

// yE[mu][col] += sum_k HEE[member][mu][k] xE[k][col]
__global__ void k_enr_post1(const double* __restrict__ HEE, const double* __restrict__ xE, double* __restrict__ yE,
                            long long ld2, int ncols2, int cols_member, int nE) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)nE * ncols2) return;
  int mu = idx / ncols2, col = idx % ncols2;
  int member = col / cols_member;
  const double* H = HEE + (long long)member * nE * nE + (long long)mu * nE;
  double acc = 0.0;
  for (int k = 0; k < nE; ++k) acc += H[k] * xE[k * ld2 + col];
  yE[mu * ld2 + col] += acc;
}

// Y[n_h + nu][col] = sum_mu S[nu][mu] yE[mu][col]
__global__ void k_enr_post2(const double* __restrict__ S, const double* __restrict__ yE, double* __restrict__ Y,
                            long long n_h, long long ld2, int ncols2, int nE) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)nE * ncols2) return;
  int nu = idx / ncols2, col = idx % ncols2;
  double acc = 0.0;
  for (int mu = 0; mu < nE; ++mu) acc += S[nu * nE + mu] * yE[mu * ld2 + col];
  Y[(n_h + nu) * ld2 + col] = acc;
}

// ----------------------------------------------------------------------------
// operator build
// ----------------------------------------------------------------------------
__global__ void k_op_W(const double* __restrict__ wJ, const double* __restrict__ v, double* __restrict__ W64,
                       float* __restrict__ W32, df32* __restrict__ W2, long long n_per_member, int batch) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n_per_member * batch) return;
  double w = wJ[idx % n_per_member] * v[idx];
  W64[idx] = w;
  const float h = (float)w;
  W32[idx] = h;
  W2[idx] = df32(h, (float)(w - (double)h));
}

// E[member][k][l] = kin * KE[k][l] + sum_q B[q][l] W[member][cell_k][q] Atil[k][q]
// slots = pairs (RT per block), sum-factorised B^T.
template <int P1, int NQ1>
__global__ void __launch_bounds__(kThreads)
k_op_pairs(const __grid_constant__ RefTables tab, const int* __restrict__ pair_cell, long long n_pairs, int nc,
           const double* __restrict__ Atil, const double* __restrict__ KE, const double* __restrict__ W,
           double kin, double* __restrict__ E64, float* __restrict__ E32, df32* __restrict__ E2) {
  constexpr int RT = tile_rt<double, NQ1>();
  constexpr int S3 = NQ1 * NQ1 * NQ1;
  constexpr int NN = P1 * P1 * P1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* Bt = reinterpret_cast<double*>(smem_raw);
  double* C = Bt + S3 * RT;
  double* D = C + S3 * RT;
  const int member = blockIdx.y;
  const long long k0 = (long long)blockIdx.x * RT;
  for (int it = threadIdx.x; it < S3 * RT; it += blockDim.x) {
    const int r = it % RT, q = it / RT;
    const long long k = k0 + r;
    double v = 0.0;
    if (k < n_pairs) v = W[((long long)member * nc + pair_cell[k]) * S3 + q] * Atil[k * S3 + q];
    C[it] = v;
  }
  __syncthreads();
  interp_bwd<double, P1, NQ1, RT, false>(tab, C, Bt, D, C);
  for (int it = threadIdx.x; it < NN * RT; it += blockDim.x) {
    const int r = it % RT, l = it / RT;
    const long long k = k0 + r;
    if (k >= n_pairs) continue;
    const double e = kin * KE[k * NN + l] + Bt[l * RT + r];
    const long long o = ((long long)member * n_pairs + k) * NN + l;
    E64[o] = e;
    const float h = (float)e;
    E32[o] = h;
    E2[o] = df32(h, (float)(e - (double)h));
  }
}

// HEE[member] = kin * KEE + sum_cells Atil_c^T diag(W) Atil_c
__global__ void k_op_hee_init(const double* __restrict__ KEE, double kin, double* __restrict__ HEE, int nE, int batch) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)batch * nE * nE) return;
  HEE[idx] = kin * KEE[idx % ((long long)nE * nE)];
}

__global__ void k_op_hee(const int* __restrict__ pair_start, const int* __restrict__ pair_fn,
                         const double* __restrict__ Atil, const double* __restrict__ W, int nc, int nq, int nE,
                         double* __restrict__ HEE) {
  const int c = blockIdx.x, member = blockIdx.y;
  const int p0 = pair_start[c], np = pair_start[c + 1] - p0;
  if (np == 0) return;
  const double* Wc = W + ((long long)member * nc + c) * nq;
  for (int it = threadIdx.x; it < np * np; it += blockDim.x) {
    const int a = it / np, b = it % np;
    if (b < a) continue;
    const double* fa = Atil + (long long)(p0 + a) * nq;
    const double* fb = Atil + (long long)(p0 + b) * nq;
    double acc = 0.0;
    for (int q = 0; q < nq; ++q) acc += Wc[q] * fa[q] * fb[q];
    const int ia = pair_fn[p0 + a], ib = pair_fn[p0 + b];
    double* H = HEE + (long long)member * nE * nE;
    atomicAdd(&H[(long long)ia * nE + ib], acc);
    if (ia != ib) atomicAdd(&H[(long long)ib * nE + ia], acc);
  }
}

// ----------------------------------------------------------------------------
// multi-cell tiles (one real column per cell and batch member): Laplacian,
// Poisson load vector, nodal -> quadrature interpolation.  Slot s of the
// launch covers cell s / nb and member s % nb.
// ----------------------------------------------------------------------------
template <int P1, int NQ1>
__global__ void __launch_bounds__(kThreads)
k_laplace(const __grid_constant__ RefTables tab, const MeshView mesh, const double* __restrict__ x,
          double* __restrict__ y, int nb, const double* __restrict__ Dsc, int mask_in, double scale) {
  constexpr int RT = tile_rt<double, NQ1>();
  constexpr int S3 = NQ1 * NQ1 * NQ1;
  constexpr int NN = P1 * P1 * P1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* A = reinterpret_cast<double*>(smem_raw);
  double* B = A + S3 * RT;
  double* C = B + S3 * RT;
  double* D = C + S3 * RT;
  double* ax = D + S3 * RT;
  double* ay = ax + 32;
  double* az = ay + 32;
  const long long s0 = (long long)blockIdx.x * RT;
  const long long n_slots = (long long)mesh.nc * nb;
  if (threadIdx.x < RT) {
    const long long s = s0 + threadIdx.x;
    double a1 = 0, a2 = 0, a3 = 0;
    if (s < n_slots) {
      int cx, cy, cz;
      cell_ijk(mesh, (int)(s / nb), cx, cy, cz);
      const double hx = mesh.h[cx], hy = mesh.h[mesh.ncx + cy], hz = mesh.h[mesh.ncx + mesh.ncy + cz];
      a1 = scale * hy * hz / (4.0 * hx);
      a2 = scale * hx * hz / (4.0 * hy);
      a3 = scale * hx * hy / (4.0 * hz);
    }
    ax[threadIdx.x] = a1;
    ay[threadIdx.x] = a2;
    az[threadIdx.x] = a3;
  }
  for (int it = threadIdx.x; it < NN * RT; it += blockDim.x) {
    const int r = it % RT, l = it / RT;
    const long long s = s0 + r;
    double v = 0.0;
    if (s < n_slots) {
      int cx, cy, cz;
      cell_ijk(mesh, (int)(s / nb), cx, cy, cz);
      const long long g = node_index(mesh, cx, cy, cz, l % P1, (l / P1) % P1, l / (P1 * P1));
      v = x[g * nb + s % nb];
      if (mask_in && Dsc[g] == 0.0) v = 0.0;
    }
    A[it] = v;
  }
  __syncthreads();
  kinetic_tile<double, P1, RT>(tab, A, B, C, D, ax, ay, az);
  for (int it = threadIdx.x; it < NN * RT; it += blockDim.x) {
    const int r = it % RT, l = it / RT;
    const long long s = s0 + r;
    if (s >= n_slots) continue;
    int cx, cy, cz;
    cell_ijk(mesh, (int)(s / nb), cx, cy, cz);
    const long long g = node_index(mesh, cx, cy, cz, l % P1, (l / P1) % P1, l / (P1 * P1));
    if (Dsc[g] != 0.0) atomicAdd(&y[g * nb + s % nb], B[it]);
  }
}

// d[g][m] += sum_q B[q][l] wJ[c][q] f[m][c][q]
template <int P1, int NQ1>
__global__ void __launch_bounds__(kThreads)
k_load_vector(const __grid_constant__ RefTables tab, const MeshView mesh, const double* __restrict__ wJ,
              const double* __restrict__ f, double* __restrict__ d, int nb) {
  constexpr int RT = tile_rt<double, NQ1>();
  constexpr int S3 = NQ1 * NQ1 * NQ1;
  constexpr int NN = P1 * P1 * P1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* Bt = reinterpret_cast<double*>(smem_raw);
  double* C = Bt + S3 * RT;
  double* D = C + S3 * RT;
  const long long s0 = (long long)blockIdx.x * RT;
  const long long n_slots = (long long)mesh.nc * nb;
  for (int it = threadIdx.x; it < S3 * RT; it += blockDim.x) {
    const int r = it % RT, q = it / RT;
    const long long s = s0 + r;
    double v = 0.0;
    if (s < n_slots) {
      const long long c = s / nb, m = s % nb;
      v = wJ[c * S3 + q] * f[(m * mesh.nc + c) * S3 + q];
    }
    C[it] = v;
  }
  __syncthreads();
  interp_bwd<double, P1, NQ1, RT, false>(tab, C, Bt, D, C);
  for (int it = threadIdx.x; it < NN * RT; it += blockDim.x) {
    const int r = it % RT, l = it / RT;
    const long long s = s0 + r;
    if (s >= n_slots) continue;
    int cx, cy, cz;
    cell_ijk(mesh, (int)(s / nb), cx, cy, cz);
    const long long g = node_index(mesh, cx, cy, cz, l % P1, (l / P1) % P1, l / (P1 * P1));
    atomicAdd(&d[g * nb + s % nb], Bt[it]);
  }
}

// out[m][c][q] = sum_l B[q][l] x[g(c,l)][m]
template <int P1, int NQ1>
__global__ void __launch_bounds__(kThreads)
k_interp(const __grid_constant__ RefTables tab, const MeshView mesh, const double* __restrict__ x,
         double* __restrict__ out, int nb) {
  constexpr int RT = tile_rt<double, NQ1>();
  constexpr int S3 = NQ1 * NQ1 * NQ1;
  constexpr int NN = P1 * P1 * P1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* A = reinterpret_cast<double*>(smem_raw);
  double* C = A + S3 * RT;
  double* D = C + S3 * RT;
  const long long s0 = (long long)blockIdx.x * RT;
  const long long n_slots = (long long)mesh.nc * nb;
  for (int it = threadIdx.x; it < NN * RT; it += blockDim.x) {
    const int r = it % RT, l = it / RT;
    const long long s = s0 + r;
    double v = 0.0;
    if (s < n_slots) {
      int cx, cy, cz;
      cell_ijk(mesh, (int)(s / nb), cx, cy, cz);
      v = x[node_index(mesh, cx, cy, cz, l % P1, (l / P1) % P1, l / (P1 * P1)) * nb + s % nb];
    }
    A[it] = v;
  }
  __syncthreads();
  interp_fwd<double, P1, NQ1, RT>(tab, A, C, D);
  for (int it = threadIdx.x; it < S3 * RT; it += blockDim.x) {
    const int r = it % RT, q = it / RT;
    const long long s = s0 + r;
    if (s >= n_slots) continue;
    const long long c = s / nb, m = s % nb;
    out[(m * mesh.nc + c) * S3 + q] = C[it];
  }
}

// ----------------------------------------------------------------------------
// self-test of the integer-pipe conversions against the hardware ones, on
// seeded bit patterns: doubles in the binary32 normal range (a quarter of them
// exact round-to-nearest ties) and binary32 normal floats.
// ----------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_selftest_cvt(long long n, unsigned long long* __restrict__ bad) {
  unsigned long long local = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long h = splitmix64((unsigned long long)i);
    const unsigned long long sign = (h >> 63) << 63;
    const unsigned long long e = 897ull + (h >> 40) % 253ull;            // binary32 exponents 1..253
    unsigned long long mant = splitmix64(h) & 0xFFFFFFFFFFFFFull;
    if ((i & 3) == 0) mant = (mant & ~0x1FFFFFFFull) | 0x10000000ull;    // exact tie
    const double x = __longlong_as_double((long long)(sign | (e << 52) | mant));
    if (__float_as_uint(f64_to_f32_rn(x)) != __float_as_uint(__double2float_rn(x))) ++local;
    const unsigned fb = (unsigned)(h & 0x807FFFFFu) | ((unsigned)(1u + (h >> 32) % 254u) << 23);
    const float f = __uint_as_float(fb);
    if (__double_as_longlong(f32_to_f64(f)) != __double_as_longlong((double)f)) ++local;
  }
  if (local) atomicAdd(bad, local);
}

// ----------------------------------------------------------------------------
// host wrappers
// ----------------------------------------------------------------------------
cudaError_t run_selftest_cvt(long long n, long long* mismatches) {
  unsigned long long* d = nullptr;
  EFE_CUDA_TRY(cudaMalloc(&d, sizeof(unsigned long long)));
  EFE_CUDA_TRY(cudaMemset(d, 0, sizeof(unsigned long long)));
  k_selftest_cvt<<<1216, 256>>>(n, d);
  note_launch();
  EFE_CUDA_TRY(cudaGetLastError());
  unsigned long long h = 0;
  EFE_CUDA_TRY(cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost));
  cudaFree(d);
  *mismatches = (long long)h;
  return cudaSuccess;
}

template <typename F>
static cudaError_t set_smem(F f, size_t bytes) {
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int P1, int NQ1>
static cudaError_t apply_impl(Ctx& c, const double* X, double* Y, long long n_cols, long long ld, cudaStream_t s) {
  const long long ld2 = 2 * ld;
  const int batch = c.op.batch;
  const int cols_member = (int)(2 * n_cols / batch);
  const int ncols2 = (int)(2 * n_cols);
  EFE_CUDA_TRY(cudaMemset2DAsync(Y, sizeof(double) * ld2, 0, sizeof(double) * ncols2, c.n_dof, s));
  if (c.nE > 0) {
    EFE_CUDA_TRY(cudaMemsetAsync(c.d_yE, 0, sizeof(double) * c.nE * ld2, s));
    EFE_CUDA_TRY(launch_enr_pre(c, X, ld2, ncols2, s));
  }
  constexpr bool F32 = std::is_same<T, float>::value;
  constexpr bool PR = std::is_same<T, df32>::value;
  constexpr int PI = PR ? 2 : F32 ? 1 : 0;   // precision index of the autotuner
  const T* W = PR ? (const T*)c.op.W2 : F32 ? (const T*)c.op.W32 : (const T*)c.op.W64;
  const T* E = PR ? (const T*)c.op.E2 : F32 ? (const T*)c.op.E32 : (const T*)c.op.E64;
  const T* xEt = PR ? (const T*)c.d_xE2 : F32 ? (const T*)c.d_xE32 : (const T*)c.d_xE;
  dim3 grid(c.nc, batch);
  constexpr int RT0 = tile_rt<T, NQ1>();
  constexpr int RT1 = RT0 / 2;
  // one launch of the cell kernel with tile width RT0 (variant 0) or RT1 (variant 1)
  auto launch = [&](int variant) -> cudaError_t {
    if (variant == 0) {
      const size_t sm = tile_smem<T, NQ1, RT0>();
      if (c.n_pairs > 0) {
        auto f = k_cell_apply<T, P1, NQ1, true, RT0>;
        EFE_CUDA_TRY(set_smem(f, sm));
        f<<<grid, kThreads, sm, s>>>(c.tab, c.mesh, X, Y, ld2, cols_member, c.d_Dsc, W, c.op.kin, c.d_pair_start,
                                     c.d_pair_fn, E, c.n_pairs, xEt, c.d_yE, c.apply_gate);
      } else {
        auto f = k_cell_apply<T, P1, NQ1, false, RT0>;
        EFE_CUDA_TRY(set_smem(f, sm));
        f<<<grid, kThreads, sm, s>>>(c.tab, c.mesh, X, Y, ld2, cols_member, c.d_Dsc, W, c.op.kin, nullptr, nullptr,
                                     nullptr, 0, nullptr, nullptr, c.apply_gate);
      }
    } else {
      const size_t sm = tile_smem<T, NQ1, RT1>();
      if (c.n_pairs > 0) {
        auto f = k_cell_apply<T, P1, NQ1, true, RT1>;
        EFE_CUDA_TRY(set_smem(f, sm));
        f<<<grid, kThreads, sm, s>>>(c.tab, c.mesh, X, Y, ld2, cols_member, c.d_Dsc, W, c.op.kin, c.d_pair_start,
                                     c.d_pair_fn, E, c.n_pairs, xEt, c.d_yE, c.apply_gate);
      } else {
        auto f = k_cell_apply<T, P1, NQ1, false, RT1>;
        EFE_CUDA_TRY(set_smem(f, sm));
        f<<<grid, kThreads, sm, s>>>(c.tab, c.mesh, X, Y, ld2, cols_member, c.d_Dsc, W, c.op.kin, nullptr, nullptr,
                                     nullptr, 0, nullptr, nullptr, c.apply_gate);
      }
    }
    note_launch();
    return cudaGetLastError();
  };
  // Autotuner: the first apply of each (precision, column count) on a stream that
  // is not being captured times both tile widths (CUDA events, two launches each,
  // results discarded by the zero-fill and the final launch) and keeps the faster.
  int& choice = c.tile_choice[PI];
  if (choice < 0 || c.tile_cols[PI] != n_cols) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    EFE_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) {
      choice = 0;
    } else {
      float best = 1e30f;
      int bestv = 0;
      cudaEvent_t t0, t1;
      EFE_CUDA_TRY(cudaEventCreate(&t0));
      EFE_CUDA_TRY(cudaEventCreate(&t1));
      for (int v = 0; v < 2; ++v) {
        EFE_CUDA_TRY(launch(v));   // warm
        EFE_CUDA_TRY(cudaEventRecord(t0, s));
        EFE_CUDA_TRY(launch(v));
        EFE_CUDA_TRY(cudaEventRecord(t1, s));
        EFE_CUDA_TRY(cudaEventSynchronize(t1));
        float ms = 0.0f;
        EFE_CUDA_TRY(cudaEventElapsedTime(&ms, t0, t1));
        c.tile_ms[PI][v] = ms;
        if (ms < best) { best = ms; bestv = v; }
      }
      cudaEventDestroy(t0);
      cudaEventDestroy(t1);
      choice = bestv;
      c.tile_cols[PI] = n_cols;
      // the timing launches accumulated into Y and yE: start again from zero
      EFE_CUDA_TRY(cudaMemset2DAsync(Y, sizeof(double) * ld2, 0, sizeof(double) * ncols2, c.n_dof, s));
      if (c.nE > 0) EFE_CUDA_TRY(cudaMemsetAsync(c.d_yE, 0, sizeof(double) * c.nE * ld2, s));
    }
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!c.apply_gate) prof_pair(c, e0, e1);   // no timing events inside captured graphs
  if (e0) EFE_CUDA_TRY(cudaEventRecord(e0, s));
  EFE_CUDA_TRY(launch(choice));
  if (e1) EFE_CUDA_TRY(cudaEventRecord(e1, s));
  if (c.nE > 0) EFE_CUDA_TRY(launch_enr_post(c, Y, ld2, ncols2, cols_member, s));
  return cudaSuccess;
}

cudaError_t launch_enr_pre(Ctx& c, const double* X, long long ld2, int ncols2, cudaStream_t s) {
  const long long n = (long long)c.nE * ncols2;
  k_enr_pre<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(c.d_S, X, c.n_h, ld2, ncols2, c.nE, c.d_xE, c.d_xE32, c.d_xE2);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_enr_post(Ctx& c, double* Y, long long ld2, int ncols2, int cols_member, cudaStream_t s) {
  const long long n = (long long)c.nE * ncols2;
  k_enr_post1<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(c.op.HEE, c.d_xE, c.d_yE, ld2, ncols2, cols_member, c.nE);
  note_launch();
  k_enr_post2<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(c.d_S, c.d_yE, Y, c.n_h, ld2, ncols2, c.nE);
  note_launch();
  return cudaGetLastError();
}

template <int P1, int NQ1>
static cudaError_t build_impl(Ctx& c, const double* v, int batch, double kin, cudaStream_t s) {
  const long long per = (long long)c.nc * c.nq;
  k_op_W<<<(unsigned)((per * batch + 255) / 256), 256, 0, s>>>(c.d_wJ, v, c.op.W64, c.op.W32, c.op.W2, per, batch);
  note_launch();
  EFE_CUDA_TRY(cudaGetLastError());
  if (c.nE > 0) {
    if (c.n_pairs > 0) {
      constexpr int RT = tile_rt<double, NQ1>();
      const size_t sm = tile_smem<double, NQ1>();
      auto f = k_op_pairs<P1, NQ1>;
      EFE_CUDA_TRY(set_smem(f, sm));
      dim3 grid((unsigned)((c.n_pairs + RT - 1) / RT), batch);
      f<<<grid, kThreads, sm, s>>>(c.tab, c.d_pair_cell, c.n_pairs, c.nc, c.d_Atil, c.d_KE, c.op.W64, kin, c.op.E64,
                                   c.op.E32, c.op.E2);
      note_launch();
      EFE_CUDA_TRY(cudaGetLastError());
    }
    long long n = (long long)batch * c.nE * c.nE;
    k_op_hee_init<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(c.d_KEE, kin, c.op.HEE, c.nE, batch);
    note_launch();
    dim3 g2(c.nc, batch);
    k_op_hee<<<g2, 128, 0, s>>>(c.d_pair_start, c.d_pair_fn, c.d_Atil, c.op.W64, c.nc, c.nq, c.nE, c.op.HEE);
    note_launch();
    EFE_CUDA_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

#define EFE_DISPATCH_P(P, CALL)                         \
  switch (P) {                                          \
    case 2: { constexpr int P1 = 3, NQ1 = 4; CALL; }    \
    case 3: { constexpr int P1 = 4, NQ1 = 5; CALL; }    \
    case 4: { constexpr int P1 = 5, NQ1 = 6; CALL; }    \
    case 5: { constexpr int P1 = 6, NQ1 = 7; CALL; }    \
    default: return cudaErrorInvalidValue;              \
  }

cudaError_t launch_apply(Ctx& c, const double* X, double* Y, long long n_cols, long long ld, int precision,
                         cudaStream_t s) {
  if (precision == EFE_TC) return launch_tc_apply(c, X, Y, n_cols, ld, s);
  if (precision == EFE_MIXED) {
    EFE_DISPATCH_P(c.p, return (apply_impl<float, P1, NQ1>(c, X, Y, n_cols, ld, s)));
  }
  if (precision == EFE_PAIR) {
    EFE_DISPATCH_P(c.p, return (apply_impl<df32, P1, NQ1>(c, X, Y, n_cols, ld, s)));
  }
  EFE_DISPATCH_P(c.p, return (apply_impl<double, P1, NQ1>(c, X, Y, n_cols, ld, s)));
}

cudaError_t launch_build_operator(Ctx& c, const double* v, int batch, double kin, cudaStream_t s) {
  EFE_DISPATCH_P(c.p, return (build_impl<P1, NQ1>(c, v, batch, kin, s)));
}

template <int P1, int NQ1>
static cudaError_t laplace_impl(const Ctx& c, const double* x, double* y, int nb, int mask_in, double scale,
                                cudaStream_t s) {
  constexpr int RT = tile_rt<double, NQ1>();
  const size_t sm = tile_smem<double, NQ1>();
  auto f = k_laplace<P1, NQ1>;
  EFE_CUDA_TRY(set_smem(f, sm));
  const long long slots = (long long)c.nc * nb;
  f<<<(unsigned)((slots + RT - 1) / RT), kThreads, sm, s>>>(c.tab, c.mesh, x, y, nb, c.d_Dsc, mask_in, scale);
  note_launch();
  return cudaGetLastError();
}

template <int P1, int NQ1>
static cudaError_t loadvec_impl(const Ctx& c, const double* f, double* d, int nb, cudaStream_t s) {
  constexpr int RT = tile_rt<double, NQ1>();
  const size_t sm = tile_smem<double, NQ1>();
  auto k = k_load_vector<P1, NQ1>;
  EFE_CUDA_TRY(set_smem(k, sm));
  const long long slots = (long long)c.nc * nb;
  k<<<(unsigned)((slots + RT - 1) / RT), kThreads, sm, s>>>(c.tab, c.mesh, c.d_wJ, f, d, nb);
  note_launch();
  return cudaGetLastError();
}

template <int P1, int NQ1>
static cudaError_t interp_impl(const Ctx& c, const double* x, double* out, int nb, cudaStream_t s) {
  constexpr int RT = tile_rt<double, NQ1>();
  const size_t sm = tile_smem<double, NQ1>();
  auto k = k_interp<P1, NQ1>;
  EFE_CUDA_TRY(set_smem(k, sm));
  const long long slots = (long long)c.nc * nb;
  k<<<(unsigned)((slots + RT - 1) / RT), kThreads, sm, s>>>(c.tab, c.mesh, x, out, nb);
  note_launch();
  return cudaGetLastError();
}

// y (+)= mask_out * scale * (1/2 int grad N . grad N) x  (atomically added; caller zeroes y)
cudaError_t launch_laplace(const Ctx& c, const double* x, double* y, int nb, int mask_in, double scale, cudaStream_t s) {
  EFE_DISPATCH_P(c.p, return (laplace_impl<P1, NQ1>(c, x, y, nb, mask_in, scale, s)));
}
cudaError_t launch_load_vector(const Ctx& c, const double* f, double* d, int nb, cudaStream_t s) {
  EFE_DISPATCH_P(c.p, return (loadvec_impl<P1, NQ1>(c, f, d, nb, s)));
}
cudaError_t launch_interp(const Ctx& c, const double* x, double* out, int nb, cudaStream_t s) {
  EFE_DISPATCH_P(c.p, return (interp_impl<P1, NQ1>(c, x, out, nb, s)));
}

}  // namespace efe

// ============================================================================
// Apply without allocation.
//
// Callers that cannot allocate device memory at the time they apply the
// operator - a host framework that owns every allocation and forbids new
// ones once it is running, or a caller recording work into a CUDA graph,
// where cudaMalloc is not allowed during stream capture - use
// efe_apply_H_noalloc.  Its enrichment scratch (S x^E in float64 and float32
// and the y^E accumulator) lives in the file-scope device array below instead
// of context workspaces.  The array exists once per GPU that loads the library
// and stays allocated until the process exits; every call on that GPU shares
// it, so calls that overlap on the GPU race, and the accumulator is cleared at
// the start of each call.
// ============================================================================
namespace efe {

constexpr long long kNoAllocScratchDoubles = 262144;   // 2 MiB per device
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[256] = {};

// Device address of the static scratch for the current device (looked up
// once per device; the first call must come before any stream capture).
static cudaError_t noalloc_scratch(int device, double** out) {
  if (device < 0 || device >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[device] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[device];
  return cudaSuccess;
}

template <typename T, int P1, int NQ1>
static cudaError_t apply_noalloc_impl(Ctx& c, const double* X, double* Y, long long n_cols, long long ld,
                                      double* xE, float* xE32, double* yE, cudaStream_t s) {
  const long long ld2 = 2 * ld;
  const int batch = c.op.batch;
  const int cols_member = (int)(2 * n_cols / batch);
  const int ncols2 = (int)(2 * n_cols);
  EFE_CUDA_TRY(cudaMemset2DAsync(Y, sizeof(double) * ld2, 0, sizeof(double) * ncols2, c.n_dof, s));
  if (c.nE > 0) {
    EFE_CUDA_TRY(cudaMemsetAsync(yE, 0, sizeof(double) * c.nE * ld2, s));
    long long n = (long long)c.nE * ncols2;
    k_enr_pre<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(c.d_S, X, c.n_h, ld2, ncols2, c.nE, xE, xE32);
    note_launch();
    EFE_CUDA_TRY(cudaGetLastError());
  }
  constexpr bool F32 = std::is_same<T, float>::value;
  const T* W = F32 ? (const T*)c.op.W32 : (const T*)c.op.W64;
  const T* E = F32 ? (const T*)c.op.E32 : (const T*)c.op.E64;
  const T* xEt = F32 ? (const T*)xE32 : (const T*)xE;
  const size_t sm = tile_smem<T, NQ1>();
  dim3 grid(c.nc, batch);
  if (c.n_pairs > 0) {
    auto f = k_cell_apply<T, P1, NQ1, true>;
    EFE_CUDA_TRY(set_smem(f, sm));
    f<<<grid, kThreads, sm, s>>>(c.tab, c.mesh, X, Y, ld2, cols_member, c.d_Dsc, W, c.op.kin, c.d_pair_start,
                                 c.d_pair_fn, E, c.n_pairs, xEt, yE, nullptr);
    note_launch();
  } else {
    auto f = k_cell_apply<T, P1, NQ1, false>;
    EFE_CUDA_TRY(set_smem(f, sm));
    f<<<grid, kThreads, sm, s>>>(c.tab, c.mesh, X, Y, ld2, cols_member, c.d_Dsc, W, c.op.kin, nullptr, nullptr,
                                 nullptr, 0, nullptr, nullptr, nullptr);
    note_launch();
  }
  EFE_CUDA_TRY(cudaGetLastError());
  if (c.nE > 0) {
    long long n = (long long)c.nE * ncols2;
    k_enr_post1<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(c.op.HEE, xE, yE, ld2, ncols2, cols_member, c.nE);
    note_launch();
    k_enr_post2<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(c.d_S, yE, Y, c.n_h, ld2, ncols2, c.nE);
    note_launch();
    EFE_CUDA_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

}  // namespace efe

extern "C" efe_status efe_apply_H_noalloc(efe_ctx* ctx, const double* X_dev, double* Y_dev, int64_t n_cols,
                                          int64_t ld, int32_t precision, void* stream) {
  using namespace efe;
  if (!ctx) return EFE_ERR_ARG;
  Ctx& c = ctx->c;
  c.err.clear();
  if (!c.op.valid) {
    c.err = "no operator: call efe_set_potential first";
    return EFE_ERR_STATE;
  }
  if (!X_dev || !Y_dev || X_dev == Y_dev || n_cols < 1 || ld < n_cols || n_cols % c.op.batch != 0 ||
      (precision != EFE_FP64 && precision != EFE_MIXED)) {
    c.err = "bad arguments to efe_apply_H_noalloc (n_cols must be a multiple of the operator's batch, ld >= n_cols)";
    return EFE_ERR_ARG;
  }
  // partition: x^E (float64), y^E (float64), x^E (float32), each n_enrich * 2 ld entries
  const long long per = (long long)c.nE * 2 * ld;
  const long long need = 2 * per + (per + 1) / 2;
  if (need > kNoAllocScratchDoubles) {
    c.err = "efe_apply_H_noalloc: n_enrich * 2 * ld = " + std::to_string(per) + " needs " + std::to_string(need) +
            " doubles of scratch; the static scratch holds " + std::to_string(kNoAllocScratchDoubles) +
            " (2 MiB), i.e. n_enrich * 2 * ld <= " + std::to_string(kNoAllocScratchDoubles * 2 / 5);
    return EFE_ERR_ARG;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess && dev != c.device) {
    c.err = "efe_apply_H_noalloc: the context's device must be current";
    return EFE_ERR_ARG;
  }
  double* base = nullptr;
  if (e == cudaSuccess) e = noalloc_scratch(dev, &base);
  if (e != cudaSuccess) {
    c.err = std::string("efe_apply_H_noalloc: static scratch: ") + cudaGetErrorString(e);
    return EFE_ERR_CUDA;
  }
  double* xE = base;
  double* yE = base + per;
  float* xE32 = reinterpret_cast<float*>(base + 2 * per);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (precision == EFE_MIXED) {
    switch (c.p) {
      case 2: e = apply_noalloc_impl<float, 3, 4>(c, X_dev, Y_dev, n_cols, ld, xE, xE32, yE, s); break;
      case 3: e = apply_noalloc_impl<float, 4, 5>(c, X_dev, Y_dev, n_cols, ld, xE, xE32, yE, s); break;
      case 4: e = apply_noalloc_impl<float, 5, 6>(c, X_dev, Y_dev, n_cols, ld, xE, xE32, yE, s); break;
      default: e = apply_noalloc_impl<float, 6, 7>(c, X_dev, Y_dev, n_cols, ld, xE, xE32, yE, s); break;
    }
  } else {
    switch (c.p) {
      case 2: e = apply_noalloc_impl<double, 3, 4>(c, X_dev, Y_dev, n_cols, ld, xE, xE32, yE, s); break;
      case 3: e = apply_noalloc_impl<double, 4, 5>(c, X_dev, Y_dev, n_cols, ld, xE, xE32, yE, s); break;
      case 4: e = apply_noalloc_impl<double, 5, 6>(c, X_dev, Y_dev, n_cols, ld, xE, xE32, yE, s); break;
      default: e = apply_noalloc_impl<double, 6, 7>(c, X_dev, Y_dev, n_cols, ld, xE, xE32, yE, s); break;
    }
  }
  if (e != cudaSuccess) {
    c.err = std::string("efe_apply_H_noalloc: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? EFE_ERR_NOMEM : EFE_ERR_CUDA;
  }
  return EFE_OK;
}
