// Lanczos exponential (Eqs. AdaptiveKrylov, AdaptiveKrylovErr), density
// (Sec. "Time dependent Kohn-Sham equations"), LDA, dipole, potential
// assembly and the Hartree PCG (Eqs. Hartree_possion, DiscretePoisson).
// Everything here is float64 and bound by HBM bandwidth or by the FP64 pipe.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "efe_internal.h"
#include "sumfact.cuh"

namespace efe {

cudaError_t launch_laplace(const Ctx& c, const double* x, double* y, int nb, int mask_in, double scale,
                           cudaStream_t s);
cudaError_t launch_load_vector(const Ctx& c, const double* f, double* d, int nb, cudaStream_t s);
cudaError_t launch_interp(const Ctx& c, const double* x, double* out, int nb, cudaStream_t s);

static unsigned nblk(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// Lanczos scalar layout in Ctx::d_lz for C complex columns.
struct LzView {
  double *nrm, *alpha, *beta, *yre, *yim, *eps, *red, *red2, *dt, *dts_in;
  df32* wp;     // [kMaxK][C][2] combination weights nrm y_j as float32 pairs (re, im)
  double* hre;  // [kMaxK][2][C] reorthogonalisation coefficients <V_i, W> (re, im)
  int *active, *kused, *cap, *n_active;
};
static LzView lz_view(const Ctx& c, long long C) {
  LzView v;
  double* b = c.d_lz;
  v.nrm = b;
  v.alpha = b + C;
  v.beta = v.alpha + kMaxK * C;
  v.yre = v.beta + kMaxK * C;
  v.yim = v.yre + kMaxK * C;
  v.eps = v.yim + kMaxK * C;
  v.red = v.eps + C;
  v.red2 = v.red + C;
  v.dt = v.red2 + C;
  v.dts_in = v.dt + C;
  v.wp = reinterpret_cast<df32*>(v.dts_in + C);
  v.hre = reinterpret_cast<double*>(v.wp + 2 * kMaxK * C);
  int* ib = c.d_lzi;
  v.active = ib;
  v.kused = ib + C;
  v.cap = ib + 2 * C;
  v.n_active = ib + 3 * C;
  return v;
}

// Flat grid over (row, column) with a fixed column per thread: the thread
// count used is the largest multiple of C not above the launch size.
struct FlatIter {
  long long row0, rstride;
  int col;
  bool ok;
};
__device__ __forceinline__ FlatIter flat_iter(int C) {
  const long long T = (long long)gridDim.x * blockDim.x;
  const long long Tc = (T / C) * C;
  const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  FlatIter f;
  f.ok = gt < Tc;
  f.col = (int)(gt % C);
  f.row0 = gt / C;
  f.rstride = Tc / C;
  return f;
}

// block-level reduction of one value per thread into out[col] (atomics)
__device__ __forceinline__ void block_col_reduce(double v, int col, bool ok, int C, double* sred, double* out) {
  for (int i = threadIdx.x; i < C; i += blockDim.x) sred[i] = 0.0;
  __syncthreads();
  if (ok && v != 0.0) atomicAdd(&sred[col], v);
  __syncthreads();
  for (int i = threadIdx.x; i < C; i += blockDim.x)
    if (sred[i] != 0.0) atomicAdd(&out[i], sred[i]);
}

// out[col] += sum_rows |X[row][col]|^2 (complex)
__global__ void k_norm2(const double* __restrict__ X, long long n_rows, int C, long long ld2, double* __restrict__ out) {
  extern __shared__ double sred[];
  FlatIter f = flat_iter(C);
  double acc = 0.0;
  if (f.ok)
    for (long long r = f.row0; r < n_rows; r += f.rstride) {
      const double2 v = *reinterpret_cast<const double2*>(X + r * ld2 + 2 * f.col);
      acc += v.x * v.x + v.y * v.y;
    }
  block_col_reduce(acc, f.col, f.ok, C, sred, out);
}

// Q0 = X / nrm, set up the per-column state
__global__ void k_lz_init(const double* __restrict__ X, double* __restrict__ Q0, long long n_rows, int C, long long ld2,
                          const double* __restrict__ red) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n_rows * C) return;
  const long long r = idx / C;
  const int col = (int)(idx % C);
  const double n = sqrt(red[col]);
  const double inv = n > 0.0 ? 1.0 / n : 0.0;
  const double2 v = *reinterpret_cast<const double2*>(X + r * ld2 + 2 * col);
  *reinterpret_cast<double2*>(Q0 + r * 2 * C + 2 * col) = make_double2(v.x * inv, v.y * inv);
}

__global__ void k_lz_state(LzView v, int C, const double* __restrict__ dts) {
  int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col == 0) *v.n_active = C;   // lets the first (gated) apply run
  if (col >= C) return;
  const double n = sqrt(v.red[col]);
  v.nrm[col] = n;
  v.active[col] = n > 0.0 ? 1 : 0;
  v.kused[col] = 0;
  v.cap[col] = 0;
  v.eps[col] = 0.0;
  v.dt[col] = dts[col];
}

// red[col] += Re <Qj, W>
__global__ void k_lz_dot(const double* __restrict__ Qj, const double* __restrict__ W, long long n_rows, int C,
                         const int* __restrict__ active, double* __restrict__ out) {
  extern __shared__ double sred[];
  FlatIter f = flat_iter(C);
  double acc = 0.0;
  if (f.ok && active[f.col])
    for (long long r = f.row0; r < n_rows; r += f.rstride) {
      const double2 a = *reinterpret_cast<const double2*>(Qj + r * 2 * C + 2 * f.col);
      const double2 b = *reinterpret_cast<const double2*>(W + r * 2 * C + 2 * f.col);
      acc += a.x * b.x + a.y * b.y;
    }
  block_col_reduce(acc, f.col, f.ok, C, sred, out);
}

// The basis is stored unnormalised: V_0 = Q_0 and V_{j+1} = w_j, the Lanczos residual of
// iteration j, so V_j = s_j Q_j with s_0 = 1 and s_j = beta_{j-1}; no scaling pass is needed.
// Iteration j, after the apply W = Hbar V_j and the dot red = <V_j, W> = s_j^2 alpha_j:
//   w = (W - alpha_j V_j) / s_j - beta_{j-1} V_{j-1} / s_{j-1},   red2[col] += |w|^2,
// written over W (it becomes V_{j+1}).  Columns that have stopped get zeros, so the applies of
// later iterations (graph mode runs all k_max) see a zero vector.
__device__ __forceinline__ double lz_norm_of_basis(const double* beta, int j, int C, int col) {
  return j <= 0 ? 1.0 : beta[(long long)(j - 1) * C + col];
}
__global__ void k_lz_update(double* __restrict__ W, const double* __restrict__ Vj, const double* __restrict__ Vjm1,
                            long long n_rows, int C, const int* __restrict__ active, const double* __restrict__ dotv,
                            const double* __restrict__ beta, int j, double* __restrict__ out) {
  extern __shared__ double sred[];
  FlatIter f = flat_iter(C);
  double acc = 0.0;
  if (f.ok && active[f.col]) {
    const double sj = lz_norm_of_basis(beta, j, C, f.col);
    const double c1 = 1.0 / sj;
    const double c2 = dotv[f.col] / (sj * sj) * c1;   // alpha_j / s_j
    const double c3 = Vjm1 ? beta[(long long)(j - 1) * C + f.col] / lz_norm_of_basis(beta, j - 1, C, f.col) : 0.0;
    for (long long r = f.row0; r < n_rows; r += f.rstride) {
      const long long o = r * 2 * C + 2 * f.col;
      double2 w = *reinterpret_cast<double2*>(W + o);
      const double2 q = *reinterpret_cast<const double2*>(Vj + o);
      w.x = c1 * w.x - c2 * q.x;
      w.y = c1 * w.y - c2 * q.y;
      if (Vjm1) {
        const double2 p = *reinterpret_cast<const double2*>(Vjm1 + o);
        w.x -= c3 * p.x;
        w.y -= c3 * p.y;
      }
      *reinterpret_cast<double2*>(W + o) = w;
      acc += w.x * w.x + w.y * w.y;
    }
  } else if (f.ok) {
    for (long long r = f.row0; r < n_rows; r += f.rstride)
      *reinterpret_cast<double2*>(W + r * 2 * C + 2 * f.col) = make_double2(0.0, 0.0);
  }
  block_col_reduce(acc, f.col, f.ok, C, sred, out);
}

// Reorthogonalisation (option krylov_reorth, classical Gram-Schmidt applied twice): the new
// Lanczos vector W (= V_{j+1}) loses its components along q_0 .. q_j, q_i = V_i / s_i.
// k_lz_mdot: h[i][col] = <V_i, W> (complex, i <= j), eight basis vectors per pass over W.
__global__ void k_lz_mdot(const double* __restrict__ W, const double* __restrict__ Q, long long qstride,
                          long long n_rows, int C, const int* __restrict__ active, int j, double* __restrict__ h) {
  extern __shared__ double sred[];
  FlatIter f = flat_iter(C);
  const bool on = f.ok && active[f.col];
  for (int i0 = 0; i0 <= j; i0 += 8) {
    double re[8], im[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) re[t] = im[t] = 0.0;
    if (on)
      for (long long r = f.row0; r < n_rows; r += f.rstride) {
        const long long o = r * 2 * C + 2 * f.col;
        const double2 w = *reinterpret_cast<const double2*>(W + o);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          if (i0 + t <= j) {
            const double2 q = *reinterpret_cast<const double2*>(Q + (long long)(i0 + t) * qstride + o);
            re[t] += q.x * w.x + q.y * w.y;   // conj(q) w
            im[t] += q.x * w.y - q.y * w.x;
          }
        }
      }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      if (i0 + t > j) break;
      block_col_reduce(re[t], f.col, on, C, sred, h + (long long)(2 * (i0 + t)) * C);
      __syncthreads();
      block_col_reduce(im[t], f.col, on, C, sred, h + (long long)(2 * (i0 + t) + 1) * C);
      __syncthreads();
    }
  }
}
// W <- W - sum_{i <= j} (h_i / s_i^2) V_i, and out[col] += |W|^2
__global__ void k_lz_maxpy(double* __restrict__ W, const double* __restrict__ Q, long long qstride, long long n_rows,
                           int C, const int* __restrict__ active, int j, const double* __restrict__ h,
                           const double* __restrict__ beta, double* __restrict__ out) {
  extern __shared__ double sred[];
  FlatIter f = flat_iter(C);
  double acc = 0.0;
  if (f.ok && active[f.col]) {
    double cr[kMaxK], ci[kMaxK];
    for (int i = 0; i <= j; ++i) {
      const double si = lz_norm_of_basis(beta, i, C, f.col);
      const double inv = 1.0 / (si * si);
      cr[i] = h[(long long)(2 * i) * C + f.col] * inv;
      ci[i] = h[(long long)(2 * i + 1) * C + f.col] * inv;
    }
    for (long long r = f.row0; r < n_rows; r += f.rstride) {
      const long long o = r * 2 * C + 2 * f.col;
      double2 w = *reinterpret_cast<double2*>(W + o);
      for (int i = 0; i <= j; ++i) {
        const double2 q = *reinterpret_cast<const double2*>(Q + (long long)i * qstride + o);
        w.x -= cr[i] * q.x - ci[i] * q.y;
        w.y -= cr[i] * q.y + ci[i] * q.x;
      }
      *reinterpret_cast<double2*>(W + o) = w;
      acc += w.x * w.x + w.y * w.y;
    }
  }
  block_col_reduce(acc, f.col, f.ok && active[f.col], C, sred, out);
}

// y = exp(-i dt T) e_1 for the real symmetric m x m tridiagonal T (diagonal al,
// off-diagonal be[0..m-2]) of one column, by one warp; y goes to v.yre/v.yim
// and its last component to u0[0] (re) and u1[0] (im).
// The exponential is the Chebyshev (Jacobi-Anger) series on the Gershgorin
// interval [c - e, c + e] of T:
//   exp(-i dt T) = exp(-i dt c) [J_0(z) + 2 sum_k (-i)^k J_k(z) T_k((T - c)/e)],  z = dt e,
// with the Bessel values J_k(z) from Miller's backward recurrence (normalised
// by J_0 + 2 sum J_2k = 1) and T_k(.) e_1 from the three-term recurrence, so a
// step costs O(K m) with K ~ 1.3 z + 40 terms (truncation below 1e-17).
constexpr int kMaxBessel = 1200;
struct TriScratch {
  double* u0;   // [kMaxK + 2] T_{k-1} e1 (padded)
  double* u1;   // [kMaxK + 2] T_k e1
  double* jb;   // [kMaxBessel] Bessel values
  double* sc;   // [4]
  int* sK;
};
__device__ void tri_exp_warp(const double* al, const double* be, int m, double dt, TriScratch t, LzView v, int col,
                             int C) {
  const int lane = threadIdx.x;
  double* u0 = t.u0;
  double* u1 = t.u1;
  double* jb = t.jb;
  if (lane == 0) {
    double lo = 1e300, hi = -1e300;
    for (int r = 0; r < m; ++r) {
      const double off = (r > 0 ? fabs(be[r - 1]) : 0.0) + (r + 1 < m ? fabs(be[r]) : 0.0);
      lo = fmin(lo, al[r] - off);
      hi = fmax(hi, al[r] + off);
    }
    const double c = 0.5 * (hi + lo), e = fmax(0.5 * (hi - lo), 1e-300);
    const double z = fabs(dt) * e;
    int K = (int)(1.3 * z + 40.0);
    if (K > kMaxBessel - 40) K = kMaxBessel - 40;
    // Miller: J_{n-1} = (2n / z) J_n - J_{n+1} from n0 well above K, then normalise
    if (z < 1e-280) {
      for (int n = 0; n < K; ++n) jb[n] = (n == 0) ? 1.0 : 0.0;
    } else {
      const int n0 = K + 30;
      double jp1 = 0.0, jn = 1e-300, norm = 0.0;
      for (int n = n0; n >= 1; --n) {
        const double jm1 = (2.0 * n / z) * jn - jp1;
        jp1 = jn;
        jn = jm1;
        if (n - 1 < K) jb[n - 1] = jn;
        if (((n - 1) & 1) == 0) norm += ((n - 1) == 0 ? 1.0 : 2.0) * jn;
        if (fabs(jn) > 1e250) {   // rescale the running values
          jp1 *= 1e-250;
          jn *= 1e-250;
          norm *= 1e-250;
          for (int q = n - 1; q < K; ++q) jb[q] *= 1e-250;
        }
      }
      const double inv = 1.0 / norm;
      for (int n = 0; n < K; ++n) jb[n] *= inv;
    }
    t.sc[0] = c;
    t.sc[1] = e;
    t.sc[2] = z;
    *t.sK = K;
  }
  __syncwarp();
  const double c = t.sc[0], e = t.sc[1];
  const int K = *t.sK;
  const double sgn = dt >= 0 ? 1.0 : -1.0;    // exp(-i dt T): for dt < 0 the series of |dt| with conjugated phases
  // lane-owned components r = lane, lane + 32
  double yr[2] = {0.0, 0.0}, yi[2] = {0.0, 0.0};
  for (int q = 0; q < 2; ++q) {
    const int r = lane + 32 * q;
    if (r < m) {
      u0[r + 1] = (r == 0) ? 1.0 : 0.0;
      u1[r + 1] = 0.0;
    }
  }
  if (lane == 0) { u0[0] = u0[m + 1] = 0.0; u1[0] = u1[m + 1] = 0.0; }
  __syncwarp();
  // k = 0 term
  for (int q = 0; q < 2; ++q) {
    const int r = lane + 32 * q;
    if (r < m) yr[q] += jb[0] * u0[r + 1];
  }
  // T_1 e1 = ((T - c) / e) e1
  for (int q = 0; q < 2; ++q) {
    const int r = lane + 32 * q;
    if (r < m) {
      const double bl = r > 0 ? be[r - 1] : 0.0, br = r + 1 < m ? be[r] : 0.0;
      u1[r + 1] = ((al[r] - c) * u0[r + 1] + bl * u0[r] + br * u0[r + 2]) / e;
    }
  }
  __syncwarp();
  for (int k = 1; k < K; ++k) {
    // coefficient 2 (-i)^k J_k (sign of the imaginary unit follows dt)
    const double cf = 2.0 * jb[k];
    const int ph = k & 3;   // (-i)^k: 1, -i, -1, i
    for (int q = 0; q < 2; ++q) {
      const int r = lane + 32 * q;
      if (r < m) {
        const double w = cf * u1[r + 1];
        if (ph == 0) yr[q] += w;
        else if (ph == 1) yi[q] -= sgn * w;
        else if (ph == 2) yr[q] -= w;
        else yi[q] += sgn * w;
      }
    }
    // next: T_{k+1} = 2 X T_k - T_{k-1}, stored in u0
    double nx[2] = {0.0, 0.0};
    for (int q = 0; q < 2; ++q) {
      const int r = lane + 32 * q;
      if (r < m) {
        const double bl = r > 0 ? be[r - 1] : 0.0, br = r + 1 < m ? be[r] : 0.0;
        nx[q] = 2.0 * ((al[r] - c) * u1[r + 1] + bl * u1[r] + br * u1[r + 2]) / e - u0[r + 1];
      }
    }
    __syncwarp();
    for (int q = 0; q < 2; ++q) {
      const int r = lane + 32 * q;
      if (r < m) {
        u0[r + 1] = u1[r + 1];
        u1[r + 1] = nx[q];
      }
    }
    __syncwarp();
  }
  // global phase exp(-i dt c)
  double sp, cp;
  sincos(dt * c, &sp, &cp);
  for (int q = 0; q < 2; ++q) {
    const int r = lane + 32 * q;
    if (r < m) {
      const double re = yr[q] * cp + yi[q] * sp;
      const double im = yi[q] * cp - yr[q] * sp;
      v.yre[(long long)r * C + col] = re;
      v.yim[(long long)r * C + col] = im;
      if (r == m - 1) { u0[0] = re; u1[0] = im; }
    }
  }
  __syncwarp();
}

// Iteration j of one column: record alpha_j, beta_j, evaluate exp(-i dt T_{j+1}) e_1
// and the error estimate of Eq. AdaptiveKrylovErr, and decide whether to stop.
__global__ void k_lz_tri(LzView v, int C, int j, int k_max, int fixed_k, double tol) {
  extern __shared__ double tri_sh[];
  const int col = blockIdx.x;
  const int lane = threadIdx.x;   // 32 lanes
  if (col >= C) return;
  if (!v.active[col]) return;
  const int m = j + 1;
  double* al = tri_sh;            // [kMaxK]
  double* be = al + kMaxK;        // [kMaxK]
  __shared__ double sc[4];
  __shared__ int sK;
  TriScratch t{be + kMaxK, be + 2 * kMaxK + 2, be + 3 * kMaxK + 4, sc, &sK};
  if (lane == 0) {
    const double sj = lz_norm_of_basis(v.beta, j, C, col);
    v.alpha[(long long)j * C + col] = v.red[col] / (sj * sj);
    v.beta[(long long)j * C + col] = sqrt(v.red2[col]);
  }
  __syncwarp();
  for (int r = lane; r < m; r += 32) {
    al[r] = v.alpha[(long long)r * C + col];
    be[r] = v.beta[(long long)r * C + col];   // be[m-1] = beta_j (not part of T_m)
  }
  __syncwarp();
  const double dt = v.dt[col];
  tri_exp_warp(al, be, m, dt, t, v, col, C);
  if (lane != 0) return;
  const double b_j = be[m - 1];
  const double eps = fabs(dt) * b_j * v.nrm[col] * sqrt(t.u0[0] * t.u0[0] + t.u1[0] * t.u1[0]);
  v.eps[col] = eps;
  bool stop = false;
  if (fixed_k > 0) {
    stop = (m >= fixed_k);
  } else if (eps <= tol || b_j == 0.0) {
    stop = true;
  }
  if (!stop && m >= k_max) {
    stop = true;
    if (fixed_k <= 0) v.cap[col] = 1;
  }
  if (stop) {
    v.active[col] = 0;
    v.kused[col] = m;
  } else {
    atomicAdd(v.n_active, 1);
  }
}

// After a finished exponential: y = exp(-i dts[col] T) e_1 with the column's final
// T (kused rows), for recombining the same Krylov basis at another time step.
__global__ void k_lz_eval(LzView v, int C, const double* __restrict__ dts) {
  extern __shared__ double tri_sh[];
  const int col = blockIdx.x;
  const int lane = threadIdx.x;
  if (col >= C) return;
  const int m = v.kused[col];
  if (m <= 0) return;
  double* al = tri_sh;
  double* be = al + kMaxK;
  __shared__ double sc[4];
  __shared__ int sK;
  TriScratch t{be + kMaxK, be + 2 * kMaxK + 2, be + 3 * kMaxK + 4, sc, &sK};
  for (int r = lane; r < m; r += 32) {
    al[r] = v.alpha[(long long)r * C + col];
    be[r] = v.beta[(long long)r * C + col];
  }
  __syncwarp();
  tri_exp_warp(al, be, m, dts[col], t, v, col, C);
}

// y_j <- y_j / s_j for j < kused: the weights of the unnormalised basis vectors V_j = s_j Q_j
__global__ void k_lz_wscale(LzView v, int C, int K) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= K * C) return;
  const int j = i / C, col = i % C;
  if (j >= v.kused[col]) return;
  const double inv = 1.0 / lz_norm_of_basis(v.beta, j, C, col);
  v.yre[i] *= inv;
  v.yim[i] *= inv;
}

// out = nrm * sum_{j < kused} y_j V_j (weights already divided by s_j).  One thread per complex entry; the basis
// vectors are read eight at a time (independent loads in flight) with
// streaming hints, since each is touched once.
__global__ void __launch_bounds__(256) k_lz_combine(const double* __restrict__ Q, long long qstride,
                                                    long long n_rows, int C, LzView v, double* __restrict__ out,
                                                    long long ld2) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n_rows * C) return;
  const long long r = idx / C;
  const int col = (int)(idx % C);
  const int k = v.kused[col];
  const double2* q = reinterpret_cast<const double2*>(Q) + idx;
  const long long qs = qstride / 2;
  const double* yr = v.yre + col;
  const double* yi = v.yim + col;
  double re = 0.0, im = 0.0;
  int j = 0;
  for (; j + 8 <= k; j += 8) {
    double2 a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = __ldcs(q + (long long)(j + u) * qs);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const double cr = yr[(long long)(j + u) * C], ci = yi[(long long)(j + u) * C];
      re += cr * a[u].x - ci * a[u].y;
      im += cr * a[u].y + ci * a[u].x;
    }
  }
  for (; j < k; ++j) {
    const double2 a = __ldcs(q + (long long)j * qs);
    const double cr = yr[(long long)j * C], ci = yi[(long long)j * C];
    re += cr * a.x - ci * a.y;
    im += cr * a.y + ci * a.x;
  }
  const double n = v.nrm[col];
  *reinterpret_cast<double2*>(out + r * ld2 + 2 * col) = make_double2(n * re, n * im);
}

// Weights of the pair combination: wp[j][col] = split(nrm y_j) for j < kused, zero beyond.
__global__ void k_lz_wpair(LzView v, int C, int K) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= K * C) return;
  const int j = i / C, col = i % C;
  const double w = j < v.kused[col] ? v.nrm[col] : 0.0;
  v.wp[2 * i] = split_f64(w * v.yre[i]);
  v.wp[2 * i + 1] = split_f64(w * v.yim[i]);
}

// out = sum_{j < kused} wp_j Q_j in float32 pairs on the FP32 pipe (the float64 form needs four
// FP64 FMA per entry and basis vector and is bound by the FP64 pipe, not by HBM).
__global__ void __launch_bounds__(256) k_lz_combine_pair(const double* __restrict__ Q, long long qstride,
                                                         long long n_rows, int C, LzView v,
                                                         double* __restrict__ out, long long ld2) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n_rows * C) return;
  const long long r = idx / C;
  const int col = (int)(idx % C);
  const int k = v.kused[col];
  const double2* q = reinterpret_cast<const double2*>(Q) + idx;
  const long long qs = qstride / 2;
  const float4* wp = reinterpret_cast<const float4*>(v.wp) + col;
  df32 re(0.0f), im(0.0f);
  int j = 0;
  for (; j + 4 <= k; j += 4) {
    double2 a[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) a[u] = __ldcs(q + (long long)(j + u) * qs);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float4 w = wp[(long long)(j + u) * C];
      const df32 wr(w.x, w.y), wi(w.z, w.w), mwi(-w.z, -w.w);
      const df32 ar = split_f64(a[u].x), ai = split_f64(a[u].y);
      re = fma(wr, ar, re);
      re = fma(mwi, ai, re);
      im = fma(wr, ai, im);
      im = fma(wi, ar, im);
    }
  }
  for (; j < k; ++j) {
    const double2 a = __ldcs(q + (long long)j * qs);
    const float4 w = wp[(long long)j * C];
    const df32 wr(w.x, w.y), wi(w.z, w.w), mwi(-w.z, -w.w);
    const df32 ar = split_f64(a.x), ai = split_f64(a.y);
    re = fma(wr, ar, re);
    re = fma(mwi, ai, re);
    im = fma(wr, ai, im);
    im = fma(wi, ar, im);
  }
  *reinterpret_cast<double2*>(out + r * ld2 + 2 * col) =
      make_double2(to_f64<df32>(fin(re)), to_f64<df32>(fin(im)));
}

// The Krylov combination in the precision of the run: float64 for EFE_FP64, float32 pairs otherwise.
static cudaError_t launch_combine(const Ctx& c, const LzView& v, long long n, long long C, double* out, long long ld2,
                                  int precision, cudaStream_t s) {
  k_lz_wscale<<<nblk((long long)c.k_max * C), 256, 0, s>>>(v, (int)C, c.k_max);
  note_launch();
  if (precision == EFE_FP64) {
    k_lz_combine<<<nblk(n * C), 256, 0, s>>>(c.d_Q, n * 2 * C, n, (int)C, v, out, ld2);
    note_launch();
  } else {
    k_lz_wpair<<<nblk((long long)c.k_max * C), 256, 0, s>>>(v, (int)C, c.k_max);
    note_launch();
    k_lz_combine_pair<<<nblk(n * C), 256, 0, s>>>(c.d_Q, n * 2 * C, n, (int)C, v, out, ld2);
    note_launch();
  }
  return cudaGetLastError();
}

__global__ void k_lz_stats(LzView v, int C, int* __restrict__ stats_i, double* __restrict__ stats_d) {
  // stats_i: [max k, cap hits]; stats_d: [max eps]  (single block)
  __shared__ int smax, scap;
  __shared__ double seps;
  if (threadIdx.x == 0) { smax = 0; scap = 0; seps = 0.0; }
  __syncthreads();
  for (int col = threadIdx.x; col < C; col += blockDim.x) {
    atomicMax(&smax, v.kused[col]);
    atomicAdd(&scap, v.cap[col]);
    const double e = v.eps[col];
    unsigned long long* a = reinterpret_cast<unsigned long long*>(&seps);
    unsigned long long old = *a, assumed;
    do {
      assumed = old;
      if (__longlong_as_double(assumed) >= e) break;
      old = atomicCAS(a, assumed, __double_as_longlong(e));
    } while (old != assumed);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    stats_i[0] = smax;
    stats_i[1] = scap;
    stats_d[0] = seps;
  }
}

static size_t red_smem(long long C) { return sizeof(double) * (size_t)C; }
static unsigned red_grid(long long n_rows, long long C) {
  long long want = (n_rows * C + 255) / 256;
  long long cap = 152LL * 8;
  long long g = want < cap ? want : cap;
  if (g * 256 < C) g = (C + 255) / 256;
  return (unsigned)(g < 1 ? 1 : g);
}

// The Lanczos loop for the C columns at in / out (row stride ld2 doubles): eager (host checks
// the active count after every iteration and stops when it reaches zero) or graph body (all
// k_max iterations, finished columns skipped on the device, no host synchronisation).  The
// Krylov basis is contiguous ([k_max + 1][n][C]).
static cudaError_t kexp_body(Ctx& c, const double* in, double* out, long long C, long long ld2, int precision,
                             cudaStream_t s, bool eager) {
  const long long n = c.n_dof;
  const long long qstride = n * 2 * C;
  LzView v = lz_view(c, C);
  EFE_CUDA_TRY(cudaMemsetAsync(v.red, 0, sizeof(double) * C, s));
  const unsigned rg = red_grid(n, C);
  const size_t rs = red_smem(C);
  k_norm2<<<rg, 256, rs, s>>>(in, n, (int)C, ld2, v.red);
  note_launch();
  k_lz_init<<<nblk(n * C), 256, 0, s>>>(in, c.d_Q, n, (int)C, ld2, v.red);
  note_launch();
  k_lz_state<<<nblk(C), 256, 0, s>>>(v, (int)C, v.dts_in);
  note_launch();
  EFE_CUDA_TRY(cudaGetLastError());
  c.apply_gate = eager ? nullptr : v.n_active;
  for (int j = 0; j < c.k_max; ++j) {
    double* Qj = c.d_Q + j * qstride;
    double* W = c.d_Q + (j + 1) * qstride;
    cudaError_t e = launch_apply(c, Qj, W, C, C, precision, s);
    if (e != cudaSuccess) { c.apply_gate = nullptr; return e; }
    EFE_CUDA_TRY(cudaMemsetAsync(v.red, 0, sizeof(double) * 2 * C, s));   // red and red2
    EFE_CUDA_TRY(cudaMemsetAsync(v.n_active, 0, sizeof(int), s));
    k_lz_dot<<<rg, 256, rs, s>>>(Qj, W, n, (int)C, v.active, v.red);
    note_launch();
    k_lz_update<<<rg, 256, rs, s>>>(W, Qj, j > 0 ? c.d_Q + (j - 1) * qstride : nullptr, n, (int)C, v.active, v.red,
                                    v.beta, j, v.red2);
    note_launch();
    if (c.reorth) {
      for (int pass = 0; pass < 2; ++pass) {
        EFE_CUDA_TRY(cudaMemsetAsync(v.hre, 0, sizeof(double) * 2 * (j + 1) * C, s));
        EFE_CUDA_TRY(cudaMemsetAsync(v.red2, 0, sizeof(double) * C, s));
        k_lz_mdot<<<rg, 256, rs, s>>>(W, c.d_Q, qstride, n, (int)C, v.active, j, v.hre);
        note_launch();
        k_lz_maxpy<<<rg, 256, rs, s>>>(W, c.d_Q, qstride, n, (int)C, v.active, j, v.hre, v.beta, v.red2);
        note_launch();
      }
    }
    k_lz_tri<<<(unsigned)C, 32, sizeof(double) * (4 * kMaxK + 4 + kMaxBessel), s>>>(v, (int)C, j, c.k_max, c.fixed_k,
                                                                            c.krylov_tol);
    note_launch();
    EFE_CUDA_TRY(cudaGetLastError());
    if (eager) {
      EFE_CUDA_TRY(cudaMemcpyAsync(c.h_flag, v.n_active, sizeof(int), cudaMemcpyDeviceToHost, s));
      EFE_CUDA_TRY(cudaStreamSynchronize(s));
      if (*c.h_flag == 0) break;
    }
  }
  c.apply_gate = nullptr;
  EFE_CUDA_TRY(launch_combine(c, v, n, C, out, ld2, precision, s));
  int* d_si = v.n_active;   // reuse: [0] max k, [1] caps
  double* d_sd = v.red;
  k_lz_stats<<<1, 256, 0, s>>>(v, (int)C, d_si, d_sd);
  note_launch();
  return cudaGetLastError();
}

// One Lanczos run over the columns [col0, col0 + C) of in / out (ld2: their row stride).
static cudaError_t kexp_block(Ctx& c, const double* in, double* out, long long C, long long ld2, const double* h_dts,
                              int precision, int* kmax_used, int* cap_hits, double* eps_max, cudaStream_t s,
                              bool need_stats) {
  LzView v = lz_view(c, C);
  c.lz_last_C = C;
  // per-column time steps; they reach k_lz_state through dts_in (outside any graph)
  EFE_CUDA_TRY(cudaMemcpyAsync(v.dts_in, h_dts, sizeof(double) * C, cudaMemcpyHostToDevice, s));
  bool done = false;
  if (c.use_graphs) {
    Ctx::KexpGraph key{in, out, precision, C, c.op.kin, c.ws_gen, nullptr};
    auto same = [&](const Ctx::KexpGraph& g) {
      return g.in == key.in && g.out == key.out && g.precision == key.precision && g.C == key.C && g.kin == key.kin &&
             g.gen == key.gen;
    };
    cudaGraphExec_t exec = nullptr;
    for (auto& g : c.graphs)
      if (same(g)) exec = g.exec;
    bool seen = false;
    for (auto& g : c.graph_seen)
      if (same(g)) seen = true;
    if (!exec && seen) {
      // capture on the context's own stream, ordered after the work already on s
      cudaEvent_t ev;
      EFE_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      EFE_CUDA_TRY(cudaEventRecord(ev, s));
      EFE_CUDA_TRY(cudaStreamWaitEvent(c.cap_stream, ev, 0));
      EFE_CUDA_TRY(cudaStreamSynchronize(c.cap_stream));
      cudaEventDestroy(ev);
      EFE_CUDA_TRY(cudaStreamBeginCapture(c.cap_stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = kexp_body(c, in, out, C, ld2, precision, c.cap_stream, false);
      cudaGraph_t graph = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(c.cap_stream, &graph);
      if (e != cudaSuccess) return e;
      EFE_CUDA_TRY(e2);
      EFE_CUDA_TRY(cudaGraphInstantiate(&exec, graph, 0));
      cudaGraphDestroy(graph);
      key.exec = exec;
      c.graphs.push_back(key);
    }
    if (exec) {
      EFE_CUDA_TRY(cudaGraphLaunch(exec, s));
      done = true;
    } else {
      c.graph_seen.push_back(key);   // first time: run eagerly (this also tunes the apply)
    }
  }
  if (!done) EFE_CUDA_TRY(kexp_body(c, in, out, C, ld2, precision, s, true));
  if (!need_stats) return cudaSuccess;
  int hi[2];
  double hd;
  EFE_CUDA_TRY(cudaMemcpyAsync(hi, v.n_active, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
  EFE_CUDA_TRY(cudaMemcpyAsync(&hd, v.red, sizeof(double), cudaMemcpyDeviceToHost, s));
  EFE_CUDA_TRY(cudaStreamSynchronize(s));
  if (kmax_used) *kmax_used = hi[0];
  if (cap_hits) *cap_hits = hi[1];
  if (eps_max) *eps_max = hd;
  return cudaSuccess;
}

// out = Kexp(-i dt_col Hbar) in for all n_orb * batch columns, in blocks of at most c.kblock
// columns (one Lanczos run each; the columns are independent).  Statistics: the largest k, the
// cap hits and the largest estimate over the blocks.
// The operator of batch members [m0, m0 + nb) as the whole operator: per-member arrays offset,
// batch = nb (the apply then runs on those members' columns alone).
static void view_members(Ctx& c, int m0, int nb) {
  const long long pq = (long long)c.nc * c.nq, pe = c.n_pairs * (long long)c.nn, ph = (long long)c.nE * c.nE;
  Operator& o = c.op;
  if (o.W64) o.W64 += m0 * pq;
  if (o.W32) o.W32 += m0 * pq;
  if (o.W2) o.W2 += m0 * pq;
  if (o.E64) o.E64 += m0 * pe;
  if (o.E32) o.E32 += m0 * pe;
  if (o.E2) o.E2 += m0 * pe;
  if (o.HEE) o.HEE += m0 * ph;
  o.batch = nb;
  TcState& t = c.tc;
  if (t.H) {
    t.H += (size_t)m0 * c.nc * 4 * 128 * 128 * 2;
    t.rexp += (size_t)m0 * c.nc * 128;
    t.rexpE += (size_t)m0 * t.n_items * 128;
    t.E += (size_t)m0 * (t.e_total > 0 ? t.e_total : 1) * 2048;
    t.hexp += (size_t)m0 * (c.n_pairs > 0 ? c.n_pairs : 1);
    t.batch = nb;
  }
}

cudaError_t run_kexp_cols(Ctx& c, const double* in, double* out, const double* h_dts, int precision, int* kmax_used,
                          int* cap_hits, double* eps_max, cudaStream_t s, bool need_stats) {
  if (ensure_krylov(c) != EFE_OK) return cudaErrorMemoryAllocation;
  const int batch = c.op.batch;
  const long long C = (long long)c.n_orb * batch;
  long long blk = (c.kblock > 0 && c.kblock < C) ? c.kblock : C;
  if (batch > 1 && blk < C) blk = std::max<long long>(1, blk / c.n_orb) * c.n_orb;   // whole members
  int km = 0, caps = 0;
  double em = 0.0;
  for (long long off = 0; off < C; off += blk) {
    const long long Cb = std::min(blk, C - off);
    int k = 0, cp = 0;
    double e = 0.0;
    cudaError_t err;
    if (batch > 1 && Cb < C) {
      const Operator op_all = c.op;
      const TcState tc_all = c.tc;
      view_members(c, (int)(off / c.n_orb), (int)(Cb / c.n_orb));
      err = kexp_block(c, in + 2 * off, out + 2 * off, Cb, 2 * C, h_dts + off, precision, &k, &cp, &e, s,
                       need_stats);
      c.op = op_all;
      c.tc = tc_all;
    } else {
      err = kexp_block(c, in + 2 * off, out + 2 * off, Cb, 2 * C, h_dts + off, precision, &k, &cp, &e, s,
                       need_stats);
    }
    EFE_CUDA_TRY(err);
    km = std::max(km, k);
    caps += cp;
    em = std::max(em, e);
  }
  if (kmax_used) *kmax_used = km;
  if (cap_hits) *cap_hits = caps;
  if (eps_max) *eps_max = em;
  return cudaSuccess;
}

// out = nrm V exp(-i dts[col] T) e_1 with the Krylov basis V and tridiagonal T left by the
// last run_kexp_cols (same columns): the exponential of the same start vector at another
// time step of no larger magnitude, without new operator applies.
void lz_last_views(const Ctx& c, const double** norms, const int** kused) {
  const LzView v = lz_view(c, c.lz_last_C);
  *norms = v.beta;   // the norm of V_j is beta_{j-1}
  *kused = v.kused;
}

cudaError_t run_kexp_recombine(Ctx& c, double* out, const double* h_dts, cudaStream_t s) {
  const long long C = (long long)c.n_orb * c.op.batch;
  const long long n = c.n_dof;
  LzView v = lz_view(c, C);
  EFE_CUDA_TRY(cudaMemcpyAsync(v.dts_in, h_dts, sizeof(double) * C, cudaMemcpyHostToDevice, s));
  k_lz_eval<<<(unsigned)C, 32, sizeof(double) * (4 * kMaxK + 4 + kMaxBessel), s>>>(v, (int)C, v.dts_in);
  note_launch();
  return launch_combine(c, v, n, C, out, 2 * C, c.precision == EFE_FP64 ? EFE_FP64 : EFE_PAIR, s);
}

// ---------------------------------------------------------------------------- density
// rho_q = sum_a f_a |psi_a(x_q)|^2.  The classical values Phi^C psi are interpolated in T
// (float64, or float32 pairs: both 8 bytes, so a tile entry of T is overwritten in place by
// the float64 value), the enrichment values and the squares are float64.
template <typename T, int P1, int NQ1>
__global__ void __launch_bounds__(kThreads)
k_density(const __grid_constant__ RefTables tab, const MeshView mesh, const double* __restrict__ X, long long ld2,
          int n_orb, const double* __restrict__ occ, const double* __restrict__ Dsc,
          const int* __restrict__ pair_start, const int* __restrict__ pair_fn, const double* __restrict__ Atil,
          const double* __restrict__ xE, double* __restrict__ rho) {
  static_assert(sizeof(T) == sizeof(double), "tile entries are reused as float64");
  constexpr int RT = 16;
  constexpr int S3 = NQ1 * NQ1 * NQ1;
  constexpr int NN = P1 * P1 * P1;
  extern __shared__ __align__(16) double dsm[];
  T* A = reinterpret_cast<T*>(dsm);
  T* Ct = A + S3 * RT;
  T* D = Ct + S3 * RT;
  double* C = reinterpret_cast<double*>(Ct);
  double* racc = dsm + 3 * S3 * RT;
  const int c = blockIdx.x, member = blockIdx.y;
  int cx, cy, cz;
  cell_ijk(mesh, c, cx, cy, cz);
  const int cols_member = 2 * n_orb;
  const int col0 = member * cols_member;
  const int p0 = pair_start ? pair_start[c] : 0;
  const int np = pair_start ? pair_start[c + 1] - p0 : 0;
  for (int q = threadIdx.x; q < S3; q += blockDim.x) racc[q] = 0.0;
  for (int cbase = 0; cbase < cols_member; cbase += RT) {
    for (int it = threadIdx.x; it < NN * RT; it += blockDim.x) {
      const int r = it % RT, l = it / RT;
      const long long g = node_index(mesh, cx, cy, cz, l % P1, (l / P1) % P1, l / (P1 * P1));
      A[it] = from_f64<T>((cbase + r < cols_member) ? Dsc[g] * X[g * ld2 + col0 + cbase + r] : 0.0);
    }
    __syncthreads();
    interp_fwd<T, P1, NQ1, RT>(tab, A, Ct, D);
    for (int it = threadIdx.x; it < S3 * RT; it += blockDim.x) {
      const int r = it % RT, q = it / RT;
      if (cbase + r >= cols_member) continue;
      double acc = to_f64<T>(Ct[it]);
      for (int k = 0; k < np; ++k)
        acc += Atil[(long long)(p0 + k) * S3 + q] * xE[(long long)pair_fn[p0 + k] * ld2 + col0 + cbase + r];
      C[it] = acc;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < S3; q += blockDim.x) {
      double s = 0.0;
      for (int r = 0; r < RT; ++r) {
        if (cbase + r >= cols_member) break;
        const double u = C[q * RT + r];
        s += occ[((cbase + r) / 2) % n_orb] * u * u;
      }
      racc[q] += s;
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < S3; q += blockDim.x) rho[((long long)member * mesh.nc + c) * S3 + q] = racc[q];
}

__global__ void k_enr_pre_d(const double* __restrict__ S, const double* __restrict__ X, long long n_h, long long ld2,
                            int ncols2, int nE, double* __restrict__ xE) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)nE * ncols2) return;
  int nu = idx / ncols2, col = idx % ncols2;
  double acc = 0.0;
  for (int mu = 0; mu < nE; ++mu) acc += S[nu * nE + mu] * X[(n_h + mu) * ld2 + col];
  xE[nu * ld2 + col] = acc;
}

template <typename T, int P1, int NQ1>
static cudaError_t density_impl(Ctx& c, const double* psi, double* rho, cudaStream_t s) {
  const long long C = (long long)c.n_orb * c.batch;
  const long long ld2 = 2 * C;
  if (c.nE > 0) {
    long long n = (long long)c.nE * ld2;
    k_enr_pre_d<<<nblk(n), 256, 0, s>>>(c.d_S, psi, c.n_h, ld2, (int)ld2, c.nE, c.d_xE);
    note_launch();
  }
  dim3 grid(c.nc, c.batch);
  const size_t sm = sizeof(double) * (3 * 16 * NQ1 * NQ1 * NQ1 + NQ1 * NQ1 * NQ1);
  EFE_CUDA_TRY(cudaFuncSetAttribute(k_density<T, P1, NQ1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_density<T, P1, NQ1><<<grid, kThreads, sm, s>>>(c.tab, c.mesh, psi, ld2, c.n_orb, c.d_occ, c.d_Dsc,
                                                c.n_pairs ? c.d_pair_start : nullptr, c.d_pair_fn, c.d_Atil, c.d_xE,
                                                rho);
  note_launch();
  return cudaGetLastError();
}

// Float32 pairs for the interpolation unless the context computes in float64.
cudaError_t launch_density(Ctx& c, const double* psi, double* rho, cudaStream_t s) {
  if (c.precision != EFE_FP64) {
    switch (c.p) {
      case 2: return density_impl<df32, 3, 4>(c, psi, rho, s);
      case 3: return density_impl<df32, 4, 5>(c, psi, rho, s);
      case 4: return density_impl<df32, 5, 6>(c, psi, rho, s);
      case 5: return density_impl<df32, 6, 7>(c, psi, rho, s);
    }
    return cudaErrorInvalidValue;
  }
  switch (c.p) {
    case 2: return density_impl<double, 3, 4>(c, psi, rho, s);
    case 3: return density_impl<double, 4, 5>(c, psi, rho, s);
    case 4: return density_impl<double, 5, 6>(c, psi, rho, s);
    case 5: return density_impl<double, 6, 7>(c, psi, rho, s);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------- LDA
// Slater exchange plus PW92 (kind EFE_XC_PW92) or Perdew-Zunger 1981 (EFE_XC_PZ81)
// unpolarised correlation; zero below rho = 1e-14.
__global__ void k_lda(const double* __restrict__ rho, double* __restrict__ vxc, double* __restrict__ exc, long long n,
                      int kind) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double r = rho[i];
  double e = 0.0, v = 0.0;
  if (r > 1e-14) {
    const double pi = 3.14159265358979323846;
    const double c13 = cbrt(3.0 * r / pi);
    const double ex = -0.75 * c13, vx = -c13;
    const double rs = cbrt(3.0 / (4.0 * pi * r));
    const double srs = sqrt(rs);
    double ec, dec;
    if (kind == EFE_XC_PZ81) {
      if (rs >= 1.0) {
        const double g = -0.1423, b1 = 1.0529, b2 = 0.3334;
        const double den = 1.0 + b1 * srs + b2 * rs;
        ec = g / den;
        dec = -g * (0.5 * b1 / srs + b2) / (den * den);
      } else {
        const double A = 0.0311, B = -0.048, C = 0.0020, D = -0.0116;
        const double lr = log(rs);
        ec = A * lr + B + C * rs * lr + D * rs;
        dec = A / rs + C * (lr + 1.0) + D;
      }
    } else {
      const double A = 0.031091, a1 = 0.21370, b1 = 7.5957, b2 = 3.5876, b3 = 1.6382, b4 = 0.49294;
      const double Q = 2.0 * A * (b1 * srs + b2 * rs + b3 * rs * srs + b4 * rs * rs);
      const double dQ = 2.0 * A * (0.5 * b1 / srs + b2 + 1.5 * b3 * srs + 2.0 * b4 * rs);
      const double lg = log1p(1.0 / Q);
      ec = -2.0 * A * (1.0 + a1 * rs) * lg;
      dec = -2.0 * A * a1 * lg + 2.0 * A * (1.0 + a1 * rs) * dQ / (Q * (Q + 1.0));
    }
    const double vc = ec - rs / 3.0 * dec;
    e = ex + ec;
    v = vx + vc;
  }
  if (vxc) vxc[i] = v;
  if (exc) exc[i] = e;
}

cudaError_t launch_lda(const Ctx& c, const double* rho, double* vxc, double* exc, long long n, cudaStream_t s) {
  k_lda<<<nblk(n), 256, 0, s>>>(rho, vxc, exc, n, c.xc);
  note_launch();
  return cudaGetLastError();
}

}  // namespace efe

// Context-free LDA at n points (the potential assembly of meshes without an efe_ctx,
// e.g. the locally refined mesh).
extern "C" efe_status efe_lda_points(const double* rho_dev, double* vxc_dev, double* exc_dev, int64_t n, int32_t xc,
                                     void* stream) {
  if (!rho_dev || n < 0 || (xc != EFE_XC_PW92 && xc != EFE_XC_PZ81)) return EFE_ERR_ARG;
  if (n == 0) return EFE_OK;
  efe::k_lda<<<efe::nblk(n), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(rho_dev, vxc_dev, exc_dev, n, xc);
  efe::note_launch();
  return cudaGetLastError() == cudaSuccess ? EFE_OK : EFE_ERR_CUDA;
}

namespace efe {

// ---------------------------------------------------------------------------- dipole
__global__ void k_dipole(const double* __restrict__ rho, const double* __restrict__ wJ, const double* __restrict__ xq,
                         long long npts, double* __restrict__ mu) {
  const int member = blockIdx.y;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    const double w = wJ[i] * rho[member * npts + i];
    a0 += w * xq[3 * i];
    a1 += w * xq[3 * i + 1];
    a2 += w * xq[3 * i + 2];
  }
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_down_sync(0xffffffffu, a0, o);
    a1 += __shfl_down_sync(0xffffffffu, a1, o);
    a2 += __shfl_down_sync(0xffffffffu, a2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&mu[member * 3 + 0], -a0);
    atomicAdd(&mu[member * 3 + 1], -a1);
    atomicAdd(&mu[member * 3 + 2], -a2);
  }
}

__global__ void k_dipole_init(double* mu, int batch, double n0, double n1, double n2) {
  int m = threadIdx.x;
  if (m < batch) {
    mu[3 * m] = n0;
    mu[3 * m + 1] = n1;
    mu[3 * m + 2] = n2;
  }
}

cudaError_t launch_dipole(const Ctx& c, const double* rho, double* mu, cudaStream_t s) {
  double n[3] = {0, 0, 0};
  for (int a = 0; a < c.n_atoms; ++a)
    for (int k = 0; k < 3; ++k) n[k] += c.Z[a] * c.R[3 * a + k];
  for (int b0 = 0; b0 < c.batch; b0 += 1024) {
    int nb = std::min(1024, c.batch - b0);
    k_dipole_init<<<1, 1024, 0, s>>>(mu + 3 * b0, nb, n[0], n[1], n[2]);
    note_launch();
  }
  const long long npts = (long long)c.nc * c.nq;
  dim3 grid(std::min<long long>(nblk(npts), 608), c.batch);
  k_dipole<<<grid, 256, 0, s>>>(rho, c.d_wJ, c.d_xq, npts, mu);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------- potentials
__global__ void k_potential(const double* __restrict__ vN, const double* __restrict__ vH, const double* __restrict__ vxc,
                            const double* __restrict__ xq, const double* __restrict__ E, long long npts, int batch,
                            double* __restrict__ v) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= npts * batch) return;
  const long long i = idx % npts;
  const int m = (int)(idx / npts);
  double val = vN ? vN[i] : 0.0;
  if (vH) val += vH[idx];
  if (vxc) val += vxc[idx];
  val -= E[3 * m] * xq[3 * i] + E[3 * m + 1] * xq[3 * i + 1] + E[3 * m + 2] * xq[3 * i + 2];
  v[idx] = val;
}

double field_amp(const efe_field& f, double t) {
  const double pi = 3.14159265358979323846;
  switch (f.kind) {
    case EFE_FIELD_GAUSS: return f.amp * std::exp(-(t - f.t0) * (t - f.t0) / (2.0 * f.sigma * f.sigma));
    case EFE_FIELD_SINE_GAUSS:
      return f.amp * std::sin(f.omega * t) * std::exp(-(t - f.t0) * (t - f.t0) / (2.0 * f.sigma * f.sigma));
    case EFE_FIELD_SINE_TRAP: {
      if (t < 0.0 || t > f.period) return 0.0;
      double env = 1.0;
      if (f.ramp > 0.0) env = std::min(1.0, std::min(t / f.ramp, (f.period - t) / f.ramp));
      if (env < 0.0) env = 0.0;
      return f.amp * std::sin(f.omega * t) * env;
    }
    case EFE_FIELD_SINE_SINE:
      if (t < 0.0 || t > f.period) return 0.0;
      return f.amp * std::sin(pi * t / f.period) * std::sin(f.omega * t);
    default: return 0.0;
  }
}

struct FieldVec {
  double e[3 * 64];
};

__global__ void k_potential_v(const double* __restrict__ vN, const double* __restrict__ vH,
                              const double* __restrict__ vxc, const double* __restrict__ xq, const FieldVec E,
                              long long npts, int batch, double* __restrict__ v) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= npts * batch) return;
  const long long i = idx % npts;
  const int m = (int)(idx / npts);
  double val = vN ? vN[i] : 0.0;
  if (vH) val += vH[idx];
  if (vxc) val += vxc[idx];
  val -= E.e[3 * m] * xq[3 * i] + E.e[3 * m + 1] * xq[3 * i + 1] + E.e[3 * m + 2] * xq[3 * i + 2];
  v[idx] = val;
}

// v[m] = (nuclear ? v_N : 0) + vH[m] + vxc[m] - E[m] . x   (vH / vxc may be NULL); E_host [batch][3]
cudaError_t launch_potential_sum(const Ctx& c, const double* vH, const double* vxc, const double* E_host,
                                 bool nuclear, double* v, cudaStream_t s) {
  const long long npts = (long long)c.nc * c.nq;
  if (c.batch <= 64) {
    FieldVec E{};
    for (int k = 0; k < 3 * c.batch; ++k) E.e[k] = E_host[k];
    k_potential_v<<<nblk(npts * c.batch), 256, 0, s>>>(nuclear ? c.d_vN : nullptr, vH, vxc, c.d_xq, E, npts,
                                                       c.batch, v);
    note_launch();
    return cudaGetLastError();
  }
  EFE_CUDA_TRY(cudaMemcpyAsync(c.d_red, E_host, sizeof(double) * 3 * c.batch, cudaMemcpyHostToDevice, s));
  k_potential<<<nblk(npts * c.batch), 256, 0, s>>>(nuclear ? c.d_vN : nullptr, vH, vxc, c.d_xq, c.d_red, npts,
                                                   c.batch, v);
  note_launch();
  EFE_CUDA_TRY(cudaGetLastError());
  return cudaStreamSynchronize(s);
}

__global__ void k_axpby(double* __restrict__ y, const double* __restrict__ a, const double* __restrict__ b, double ca,
                        double cb, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) y[i] = ca * a[i] + cb * b[i];
}

cudaError_t launch_axpby(double* y, const double* a, const double* b, double ca, double cb, long long n, cudaStream_t s) {
  k_axpby<<<nblk(n), 256, 0, s>>>(y, a, b, ca, cb, n);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------- Hartree PCG
// vectors are [n_h][nb]; per-member scalars
__global__ void k_coldot(const double* __restrict__ a, const double* __restrict__ b, long long n_rows, int C,
                         double* __restrict__ out) {
  extern __shared__ double sred[];
  FlatIter f = flat_iter(C);
  double acc = 0.0;
  if (f.ok)
    for (long long r = f.row0; r < n_rows; r += f.rstride) acc += a[r * C + f.col] * b[r * C + f.col];
  block_col_reduce(acc, f.col, f.ok, C, sred, out);
}

// phi boundary values <- phiB (once, or after a reset)
__global__ void k_cg_bc(double* __restrict__ phi, const double* __restrict__ phiB, const double* __restrict__ Dsc,
                        long long n_h, int nb) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n_h * nb) return;
  const long long g = idx / nb;
  if (Dsc[g] == 0.0) phi[idx] = phiB[g];
}

// r = d - Ap (interior), z = r / diag, p = z; zero on the boundary
__global__ void k_cg_start(const double* __restrict__ d, const double* __restrict__ Ap, const double* __restrict__ diag,
                           const double* __restrict__ Dsc, long long n_h, int nb, double* __restrict__ r,
                           double* __restrict__ z, double* __restrict__ p, double* __restrict__ dm) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n_h * nb) return;
  const long long g = idx / nb;
  if (Dsc[g] == 0.0) {
    r[idx] = z[idx] = p[idx] = 0.0;
    dm[idx] = 0.0;
    return;
  }
  const double rr = d[idx] - Ap[idx];
  r[idx] = rr;
  z[idx] = rr / diag[g];
  p[idx] = z[idx];
  dm[idx] = d[idx];
}

// scalars per member: [0] rz, [1] rz_new, [2] pAp, [3] rr, [4] dd
__global__ void k_cg_update(double* __restrict__ phi, double* __restrict__ r, double* __restrict__ z,
                            const double* __restrict__ p, const double* __restrict__ Ap, const double* __restrict__ diag,
                            const double* __restrict__ Dsc, long long n_h, int nb, const double* __restrict__ sc,
                            double* __restrict__ rz_new, double* __restrict__ rr) {
  extern __shared__ double sred[];   // 2 * nb
  FlatIter f = flat_iter(nb);
  double a_rz = 0.0, a_rr = 0.0;
  if (f.ok) {
    const double pAp = sc[2 * nb + f.col];
    const double alpha = pAp != 0.0 ? sc[0 * nb + f.col] / pAp : 0.0;
    for (long long g = f.row0; g < n_h; g += f.rstride) {
      const long long i = g * nb + f.col;
      if (Dsc[g] == 0.0) continue;
      phi[i] += alpha * p[i];
      const double rv = r[i] - alpha * Ap[i];
      r[i] = rv;
      const double zv = rv / diag[g];
      z[i] = zv;
      a_rz += rv * zv;
      a_rr += rv * rv;
    }
  }
  block_col_reduce(a_rz, f.col, f.ok, nb, sred, rz_new);
  __syncthreads();
  block_col_reduce(a_rr, f.col, f.ok, nb, sred, rr);
}

__global__ void k_cg_dir(double* __restrict__ p, const double* __restrict__ z, long long n, int nb,
                         const double* __restrict__ sc) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n * nb) return;
  const int m = (int)(idx % nb);
  const double rz = sc[m], rzn = sc[nb + m];
  const double beta = rz != 0.0 ? rzn / rz : 0.0;
  p[idx] = z[idx] + beta * p[idx];
}

__global__ void k_cg_rot(double* sc, int nb) {
  int m = threadIdx.x + blockIdx.x * blockDim.x;
  if (m >= nb) return;
  sc[m] = sc[nb + m];   // rz <- rz_new
  sc[nb + m] = 0.0;
  sc[2 * nb + m] = 0.0;  // pAp (rr is cleared before each update)
}

efe_status run_hartree(Ctx& c, const double* rho, double* vH, double tol, int max_it, int* iters, cudaStream_t s) {
  const int nb = c.batch;
  const long long n = c.n_h;
  const long long N = n * nb;
  double* d = c.d_cg;
  double* r = d + N;
  double* z = r + N;
  double* p = z + N;
  double* Ap = p + N;
  double* dm = Ap + N;
  double* sc = dm + N;   // 5 * nb scalars
  const double scale = 1.0 / (2.0 * 3.14159265358979323846);
  const size_t rs = sizeof(double) * nb;
  const unsigned rg = red_grid(n, nb);
#define CK(x)                                              \
  do {                                                     \
    cudaError_t _e = (x);                                  \
    if (_e != cudaSuccess) {                               \
      c.err = std::string("CUDA: ") + cudaGetErrorString(_e); \
      return EFE_ERR_CUDA;                                 \
    }                                                      \
  } while (0)
  CK(cudaMemsetAsync(d, 0, sizeof(double) * N, s));
  CK(launch_load_vector(c, rho, d, nb, s));
  if (c.hartree_method == EFE_HARTREE_FDM && c.hen.on) {
    CK(hartree_enriched_solve(c, rho, vH, d, Ap, r, z, s));
    if (iters) *iters = 1;
    return EFE_OK;
  }
  if (c.hartree_method == EFE_HARTREE_FDM) {
    CK(fdm_solve(c, d, Ap, c.d_phi, nb, s));
    CK(launch_interp(c, c.d_phi, vH, nb, s));
    if (iters) *iters = 1;
    return EFE_OK;
  }
  k_cg_bc<<<nblk(N), 256, 0, s>>>(c.d_phi, c.d_phiB, c.d_Dsc, n, nb);
  note_launch();
  CK(cudaMemsetAsync(Ap, 0, sizeof(double) * N, s));
  CK(launch_laplace(c, c.d_phi, Ap, nb, 0, scale, s));
  k_cg_start<<<nblk(N), 256, 0, s>>>(d, Ap, c.d_diagA, c.d_Dsc, n, nb, r, z, p, dm);
  note_launch();
  CK(cudaMemsetAsync(sc, 0, sizeof(double) * 5 * nb, s));
  k_coldot<<<rg, 256, rs, s>>>(r, z, n, nb, sc);            // rz
  k_coldot<<<rg, 256, rs, s>>>(r, r, n, nb, sc + 3 * nb);   // rr
  k_coldot<<<rg, 256, rs, s>>>(dm, dm, n, nb, sc + 4 * nb); // dd
  CK(cudaGetLastError());
  note_launch();
  std::vector<double> hs(5 * (size_t)nb);
  int it = 0;
  bool conv = false;
  for (;;) {
    if (it % 8 == 0 || it >= max_it) {
      CK(cudaMemcpyAsync(hs.data(), sc, sizeof(double) * 5 * nb, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      conv = true;
      for (int m = 0; m < nb; ++m)
        if (!(std::sqrt(hs[3 * nb + m]) <= tol * std::sqrt(hs[4 * nb + m]) || hs[3 * nb + m] == 0.0)) conv = false;
      if (conv || it >= max_it) break;
    }
    CK(cudaMemsetAsync(Ap, 0, sizeof(double) * N, s));
    CK(launch_laplace(c, p, Ap, nb, 1, scale, s));
    k_coldot<<<rg, 256, rs, s>>>(p, Ap, n, nb, sc + 2 * nb);
    note_launch();
    CK(cudaMemsetAsync(sc + 3 * nb, 0, sizeof(double) * nb, s));
    k_cg_update<<<rg, 256, rs, s>>>(c.d_phi, r, z, p, Ap, c.d_diagA, c.d_Dsc, n, nb, sc, sc + nb, sc + 3 * nb);
    note_launch();
    k_cg_dir<<<nblk(N), 256, 0, s>>>(p, z, n, nb, sc);
    note_launch();
    k_cg_rot<<<1, 1024, 0, s>>>(sc, nb);
    note_launch();
    CK(cudaGetLastError());
    ++it;
  }
  CK(launch_interp(c, c.d_phi, vH, nb, s));
  if (iters) *iters = it;
#undef CK
  return conv ? EFE_OK : EFE_ERR_CG_NOCONV;
}

}  // namespace efe
