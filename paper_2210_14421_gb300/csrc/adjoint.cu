// Adjoint of the Magnus predictor-corrector step: gradient of a window-averaged
// dipole signal with respect to the external-field parameters (amp, omega,
// sigma).  The paper has no adjoint; this is the reverse sweep of the forward
// step of efe_magnus_step (Eq. ApproxMagnus with the predictor-corrector
// reading):
//   forward  v1 = V(rho_n) + f_n, psi^p = U(v1) psi_n, rho_m = (rho_n + rho(psi^p)) / 2,
//            v2 = V(rho_m) + f_n, psi_n+1 = U(v2) psi_n,   U(v) = exp(-i dt Hbar[v])
//   reverse  psi_bar_n  = U(v2)^H lam + U(v1)^H lam_p            (Lanczos with -dt)
//            v_bar(v)_q = w_q dt int_0^1 Im sum_a conj(Phi a_a(s))_q (Phi b_a(s))_q ds,
//                         a(s) = exp(+i (1-s) dt Hbar) lam, b(s) = exp(-i s dt Hbar) psi_n
//                         (Frechet derivative of the exponential; Gauss-Legendre in s)
//            rho_bar   += V'(rho)^T v_bar = w * Interp(A_II^-1 Interp^T v_bar) + f_xc(rho) v_bar
//            lam_p      = 2 occ Phi^T (rho_bar_p * Phi psi^p)   (the potential-only operator)
//            theta_bar += -(dE/dtheta)(t_mid) . sum_q x_q (v_bar1 + v_bar2)_q
// with checkpoints of psi every K steps and the states of a segment recomputed
// before its reverse sweep.  Applies in float64, or in float32 pairs when the
// context's precision is EFE_PAIR; everything else in float64.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "efe_internal.h"
#include "sumfact.cuh"

namespace efe {

static unsigned nb256(long long n) { return (unsigned)((n + 255) / 256); }

// out[c][q] += scale * wJ[c][q] * sum_a Im(conj(Phi a_a)(x_q) (Phi b_a)(x_q))   (batch member 0).
// The classical values are interpolated in T (float64, or float32 pairs: 8 bytes either way, a
// tile entry of T is overwritten in place by its float64 value); enrichment values and the
// products are float64.
template <typename T, int P1, int NQ1>
__global__ void __launch_bounds__(kThreads)
k_cross_density(const __grid_constant__ RefTables tab, const MeshView mesh, const double* __restrict__ Xa,
                const double* __restrict__ Xb, long long ld2, int n_orb, const double* __restrict__ Dsc,
                const int* __restrict__ pair_start, const int* __restrict__ pair_fn, const double* __restrict__ Atil,
                const double* __restrict__ xEa, const double* __restrict__ xEb, const double* __restrict__ wJ,
                double scale, double* __restrict__ out) {
  constexpr int RT = 16;
  constexpr int S3 = NQ1 * NQ1 * NQ1;
  constexpr int NN = P1 * P1 * P1;
  static_assert(sizeof(T) == sizeof(double), "tile entries are reused as float64");
  extern __shared__ __align__(16) double xsm[];
  T* A = reinterpret_cast<T*>(xsm);
  double* Ca = xsm + S3 * RT;
  T* D = reinterpret_cast<T*>(xsm + 2 * S3 * RT);
  double* Cb = xsm + 3 * S3 * RT;
  double* racc = xsm + 4 * S3 * RT;
  const int c = blockIdx.x;
  int cx, cy, cz;
  cell_ijk(mesh, c, cx, cy, cz);
  const int cols = 2 * n_orb;
  const int p0 = pair_start ? pair_start[c] : 0;
  const int np = pair_start ? pair_start[c + 1] - p0 : 0;
  for (int q = threadIdx.x; q < S3; q += blockDim.x) racc[q] = 0.0;
  for (int cbase = 0; cbase < cols; cbase += RT) {
    for (int pass = 0; pass < 2; ++pass) {
      const double* X = pass == 0 ? Xa : Xb;
      const double* xE = pass == 0 ? xEa : xEb;
      double* Cq = pass == 0 ? Ca : Cb;
      for (int it = threadIdx.x; it < NN * RT; it += blockDim.x) {
        const int r = it % RT, l = it / RT;
        const long long g = node_index(mesh, cx, cy, cz, l % P1, (l / P1) % P1, l / (P1 * P1));
        A[it] = from_f64<T>((cbase + r < cols) ? Dsc[g] * X[g * ld2 + cbase + r] : 0.0);
      }
      __syncthreads();
      interp_fwd<T, P1, NQ1, RT>(tab, A, reinterpret_cast<T*>(Cq), D);
      for (int it = threadIdx.x; it < S3 * RT; it += blockDim.x) {
        const int r = it % RT, q = it / RT;
        if (cbase + r >= cols) continue;
        double acc = to_f64<T>(reinterpret_cast<const T*>(Cq)[it]);
        for (int k = 0; k < np; ++k)
          acc += Atil[(long long)(p0 + k) * S3 + q] * xE[(long long)pair_fn[p0 + k] * ld2 + cbase + r];
        Cq[it] = acc;
      }
      __syncthreads();
    }
    for (int q = threadIdx.x; q < S3; q += blockDim.x) {
      double s = 0.0;
      for (int r = 0; r + 1 < RT; r += 2) {
        if (cbase + r >= cols) break;
        const double ar = Ca[q * RT + r], ai = Ca[q * RT + r + 1];
        const double br = Cb[q * RT + r], bi = Cb[q * RT + r + 1];
        s += ar * bi - ai * br;
      }
      racc[q] += s;
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < S3; q += blockDim.x)
    out[(long long)c * S3 + q] += scale * wJ[(long long)c * S3 + q] * racc[q];
}

// d v_xc / d rho of Slater exchange + PW92 correlation; out (+)= f_xc(rho) g
__device__ double fxc_lda(double rho) {
  if (!(rho > 1e-14)) return 0.0;
  const double pi = 3.14159265358979323846;
  const double dvx = -(1.0 / 3.0) * cbrt(3.0 / pi) * pow(rho, -2.0 / 3.0);
  const double A = 0.031091, a1 = 0.21370, b1 = 7.5957, b2 = 3.5876, b3 = 1.6382, b4 = 0.49294;
  const double rs = cbrt(3.0 / (4.0 * pi * rho));
  const double srs = sqrt(rs);
  const double Q = 2.0 * A * (b1 * srs + b2 * rs + b3 * rs * srs + b4 * rs * rs);
  const double dQ = 2.0 * A * (0.5 * b1 / srs + b2 + 1.5 * b3 * srs + 2.0 * b4 * rs);
  const double d2Q = 2.0 * A * (-0.25 * b1 / (rs * srs) + 0.75 * b3 / srs + 2.0 * b4);
  const double L = log1p(1.0 / Q);
  const double QQ = Q * (Q + 1.0);
  const double dL = -dQ / QQ;
  const double d2L = -d2Q / QQ + dQ * dQ * (2.0 * Q + 1.0) / (QQ * QQ);
  const double dG = -2.0 * A * a1 * L - 2.0 * A * (1.0 + a1 * rs) * dL;
  const double d2G = -4.0 * A * a1 * dL - 2.0 * A * (1.0 + a1 * rs) * d2L;
  const double dvc = ((2.0 / 3.0) * dG - rs / 3.0 * d2G) * (-rs / (3.0 * rho));
  return dvx + dvc;
}

// out = w * u + f_xc(rho) g   (u: interpolated homogeneous Poisson solution)
__global__ void k_vt_finish(const double* __restrict__ u, const double* __restrict__ wJ,
                            const double* __restrict__ rho, const double* __restrict__ g, double* __restrict__ out,
                            long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = wJ[i] * u[i] + fxc_lda(rho[i]) * g[i];
}

__global__ void k_div_w(const double* __restrict__ g, const double* __restrict__ wJ, double* __restrict__ out,
                        double scale, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = scale * g[i] / wJ[i];
}

__global__ void k_axpy_q(double* __restrict__ y, const double* __restrict__ x, double a, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) y[i] += a * x[i];
}

// rho_bar += coef * w_q (d . x_q)
__global__ void k_window_term(double* __restrict__ rho_bar, const double* __restrict__ wJ,
                              const double* __restrict__ xq, double d0, double d1, double d2, double coef,
                              long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) rho_bar[i] += coef * wJ[i] * (d0 * xq[3 * i] + d1 * xq[3 * i + 1] + d2 * xq[3 * i + 2]);
}

// out3 += sum_q g_q x_q
__global__ void k_xdot(const double* __restrict__ g, const double* __restrict__ xq, long long n,
                       double* __restrict__ out3) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    a0 += g[i] * xq[3 * i];
    a1 += g[i] * xq[3 * i + 1];
    a2 += g[i] * xq[3 * i + 2];
  }
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_down_sync(0xffffffffu, a0, o);
    a1 += __shfl_down_sync(0xffffffffu, a1, o);
    a2 += __shfl_down_sync(0xffffffffu, a2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out3[0], a0);
    atomicAdd(&out3[1], a1);
    atomicAdd(&out3[2], a2);
  }
}

// y[row][col] += 2 occ[col % n_orb] x[row][col]  (complex, C columns)
__global__ void k_occ_axpy(double* __restrict__ y, const double* __restrict__ x, const double* __restrict__ occ,
                           long long n_rows, int C, int n_orb) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n_rows * C) return;
  const double a = 2.0 * occ[(int)(idx % C) % n_orb];
  y[2 * idx] += a * x[2 * idx];
  y[2 * idx + 1] += a * x[2 * idx + 1];
}

__global__ void k_scale(double* __restrict__ y, double a, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) y[i] *= a;
}

__global__ void k_avg(double* __restrict__ y, const double* __restrict__ a, const double* __restrict__ b,
                      long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) y[i] = 0.5 * (a[i] + b[i]);
}

__global__ void k_enr_vals(const double* __restrict__ S, const double* __restrict__ X, long long n_h, long long ld2,
                           int nE, double* __restrict__ xE) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)nE * ld2) return;
  int nu = (int)(idx / ld2), col = (int)(idx % ld2);
  double acc = 0.0;
  for (int mu = 0; mu < nE; ++mu) acc += S[nu * nE + mu] * X[(n_h + mu) * ld2 + col];
  xE[idx] = acc;
}

// ---------------------------------------------------------------------------- host side
namespace {

struct Fail {
  efe_status st;
};

// throws Fail with the context's error text set
void ck(Ctx& c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return;
  c.err = std::string(what) + ": " + cudaGetErrorString(e);
  throw Fail{e == cudaErrorMemoryAllocation ? EFE_ERR_NOMEM : EFE_ERR_CUDA};
}
void ck(efe_status st) {
  if (st != EFE_OK) throw Fail{st};
}

struct Buffers {
  std::vector<double*> owned;
  double* get(Ctx& c, size_t n) {
    double* p = nullptr;
    ck(c, cudaMalloc((void**)&p, sizeof(double) * (n ? n : 1)), "allocating adjoint buffers");
    owned.push_back(p);
    return p;
  }
  ~Buffers() {
    for (double* p : owned) cudaFree(p);
  }
};

template <typename T, int P1, int NQ1>
cudaError_t cross_impl(Ctx& c, const double* a, const double* b, double scale, double* out, cudaStream_t s) {
  const long long ld2 = 2LL * c.n_orb;
  if (c.nE > 0) {
    const long long n = (long long)c.nE * ld2;
    k_enr_vals<<<nb256(n), 256, 0, s>>>(c.d_S, a, c.n_h, ld2, c.nE, c.d_xE);
    note_launch();
    k_enr_vals<<<nb256(n), 256, 0, s>>>(c.d_S, b, c.n_h, ld2, c.nE, c.d_yE);
    note_launch();
  }
  constexpr int S3 = NQ1 * NQ1 * NQ1;
  const size_t sm = sizeof(double) * (4 * 16 * S3 + S3);
  EFE_CUDA_TRY(cudaFuncSetAttribute(k_cross_density<T, P1, NQ1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_cross_density<T, P1, NQ1><<<c.nc, kThreads, sm, s>>>(c.tab, c.mesh, a, b, ld2, c.n_orb, c.d_Dsc,
                                                     c.n_pairs ? c.d_pair_start : nullptr, c.d_pair_fn, c.d_Atil,
                                                     c.d_xE, c.d_yE, c.d_wJ, scale, out);
  note_launch();
  return cudaGetLastError();
}

// out += scale * w Im(conj(Phi a) Phi b), summed over the orbitals
cudaError_t cross_density(Ctx& c, const double* a, const double* b, double scale, double* out, cudaStream_t s) {
  if (c.precision != EFE_FP64) {
    switch (c.p) {
      case 2: return cross_impl<df32, 3, 4>(c, a, b, scale, out, s);
      case 3: return cross_impl<df32, 4, 5>(c, a, b, scale, out, s);
      case 4: return cross_impl<df32, 5, 6>(c, a, b, scale, out, s);
      case 5: return cross_impl<df32, 6, 7>(c, a, b, scale, out, s);
    }
    return cudaErrorInvalidValue;
  }
  switch (c.p) {
    case 2: return cross_impl<double, 3, 4>(c, a, b, scale, out, s);
    case 3: return cross_impl<double, 4, 5>(c, a, b, scale, out, s);
    case 4: return cross_impl<double, 5, 6>(c, a, b, scale, out, s);
    case 5: return cross_impl<double, 6, 7>(c, a, b, scale, out, s);
  }
  return cudaErrorInvalidValue;
}

void field_derivs(const efe_field& f, double t, double E[3], double dE[3][3]) {
  double a = 0.0, da[3] = {0.0, 0.0, 0.0};
  const double u = t - f.t0;
  const double g = std::exp(-u * u / (2.0 * f.sigma * f.sigma));
  const double gs = u * u / (f.sigma * f.sigma * f.sigma);   // d/dsigma of the exponent
  if (f.kind == EFE_FIELD_SINE_GAUSS) {
    const double sn = std::sin(f.omega * t), cs = std::cos(f.omega * t);
    a = f.amp * sn * g;
    da[0] = sn * g;
    da[1] = f.amp * t * cs * g;
    da[2] = a * gs;
  } else {   // EFE_FIELD_GAUSS
    a = f.amp * g;
    da[0] = g;
    da[2] = a * gs;
  }
  for (int k = 0; k < 3; ++k) {
    E[k] = a * f.dir[k];
    for (int p = 0; p < 3; ++p) dE[p][k] = da[p] * f.dir[k];
  }
}

// The reverse sweep and its forward recomputation.  The Frechet derivative of
// exp(-i dt Hbar) needs exp(-i s dt Hbar) psi and exp(+i (1 - s) dt Hbar) lam at the
// n_s Gauss-Legendre nodes s_k; each family comes from one Krylov basis (that of
// psi, resp. lam, for the full step) recombined at the scaled time steps.
class Sweep {
 public:
  Sweep(Ctx& c, cudaStream_t s, int n_s) : c_(c), s_(s) {
    prec_ = c.precision == EFE_PAIR ? EFE_PAIR : EFE_FP64;
    C_ = c.n_orb;
    nqt_ = (long long)c.nc * c.nq;
    blk_ = c.n_dof * 2 * C_;
    for (double** p : {&rho0_, &rhop_, &rhom_, &v1_, &v2_, &vb1_, &vb2_, &rbar_, &rbm_, &tq_, &tq2_})
      *p = buf_.get(c, nqt_);
    for (double** p : {&psip_, &lam_, &lam_new_, &lamp_, &ba_, &tmp_}) *p = buf_.get(c, blk_);
    red_ = buf_.get(c, 3);
    std::vector<double> x((size_t)n_s), w((size_t)n_s);
    gauss_legendre(n_s, x.data(), w.data());
    for (int k = 0; k < n_s; ++k) {
      sk_.push_back(0.5 * (x[k] + 1.0));
      wk_.push_back(0.5 * w[k]);
      b1_.push_back(buf_.get(c, blk_));
      b2_.push_back(buf_.get(c, blk_));
    }
  }

  double* block() { return buf_.get(c_, blk_); }
  double* scratch(size_t n) { return buf_.get(c_, n); }
  long long blk() const { return blk_; }
  long long cap_hits() const { return cap_hits_; }

  // forward step psi -> out (intermediates kept: rho0, v1, psip, rhop, rhom, v2);
  // the corrector is skipped when out is NULL; with nodes, exp(-i s_k dt H1) psi
  // goes to the node buffers b1
  void forward(const double* psi, double* out, const double E[3], double dt, bool nodes = false) {
    ck(c_, launch_density(c_, psi, rho0_, s_), "density");
    potential(rho0_, E, v1_);
    ck(build_op(c_, v1_, 1, 1.0, s_));
    ck(c_, kexp(psi, psip_, dt), "predictor");
    if (nodes)
      for (size_t k = 0; k < sk_.size(); ++k) ck(c_, recombine(b1_[k], sk_[k] * dt), "Frechet node");
    ck(c_, launch_density(c_, psip_, rhop_, s_), "density");
    k_avg<<<nb256(nqt_), 256, 0, s_>>>(rhom_, rho0_, rhop_, nqt_);
    note_launch();
    potential(rhom_, E, v2_);
    if (out) {
      ck(build_op(c_, v2_, 1, 1.0, s_));
      ck(c_, kexp(psi, out, dt), "corrector");
    }
  }

  // mu (3 doubles, device) of the state psi
  void dipole(const double* psi, double* mu) {
    ck(c_, launch_density(c_, psi, tq_, s_), "density");
    ck(c_, launch_dipole(c_, tq_, mu, s_), "dipole");
  }

  void zero_cotangents() {
    ck(c_, cudaMemsetAsync(lam_, 0, sizeof(double) * blk_, s_), "memset");
    ck(c_, cudaMemsetAsync(rbar_, 0, sizeof(double) * nqt_, s_), "memset");
  }

  // cotangent of rho_n from the objective: -w (d . x) / |W|
  void window_term(const double d[3], double coef) {
    k_window_term<<<nb256(nqt_), 256, 0, s_>>>(rbar_, c_.d_wJ, c_.d_xq, d[0], d[1], d[2], coef, nqt_);
    note_launch();
  }

  // psi_n -> rho_n: lam += 2 occ Phi^T (rho_bar Phi psi_n), rho_bar reset
  void density_to_lam(const double* psi_n) {
    density_vjp(psi_n, rbar_, lam_);
    ck(c_, cudaMemsetAsync(rbar_, 0, sizeof(double) * nqt_, s_), "memset");
  }

  // reverse of the step psi -> psi_next (lam holds psi_next's cotangent on entry,
  // psi's on exit; rho_bar receives rho_n's); theta_bar accumulated
  void reverse_step(const double* psi, const double E[3], const double dE[3][3], double dt,
                    double theta_bar[3]) {
    forward(psi, nullptr, E, dt, true);
    // corrector psi_next = U(v2) psi
    ck(build_op(c_, v2_, 1, 1.0, s_));
    ck(c_, kexp(psi, tmp_, dt), "corrector");
    for (size_t k = 0; k < sk_.size(); ++k) ck(c_, recombine(b2_[k], sk_[k] * dt), "Frechet node");
    ck(c_, kexp(lam_, lam_new_, -dt), "adjoint corrector");
    frechet(b2_, dt, vb2_);
    vt(rhom_, vb2_, rbm_);
    k_axpy_q<<<nb256(nqt_), 256, 0, s_>>>(rbar_, rbm_, 0.5, nqt_);   // rho_m = (rho_n + rho^p) / 2
    note_launch();
    // predictor psi^p = U(v1) psi, reached through rho^p
    k_scale<<<nb256(nqt_), 256, 0, s_>>>(rbm_, 0.5, nqt_);
    note_launch();
    ck(c_, cudaMemsetAsync(lamp_, 0, sizeof(double) * blk_, s_), "memset");
    density_vjp(psip_, rbm_, lamp_);
    ck(build_op(c_, v1_, 1, 1.0, s_));
    ck(c_, kexp(lamp_, tmp_, -dt), "adjoint predictor");
    k_axpy_q<<<nb256(blk_), 256, 0, s_>>>(lam_new_, tmp_, 1.0, blk_);
    note_launch();
    frechet(b1_, dt, vb1_);
    vt(rho0_, vb1_, tq_);
    k_axpy_q<<<nb256(nqt_), 256, 0, s_>>>(rbar_, tq_, 1.0, nqt_);
    note_launch();
    // field: v = ... - E . x in both potentials
    k_axpy_q<<<nb256(nqt_), 256, 0, s_>>>(vb1_, vb2_, 1.0, nqt_);
    note_launch();
    ck(c_, cudaMemsetAsync(red_, 0, sizeof(double) * 3, s_), "memset");
    k_xdot<<<(unsigned)std::min<long long>(nb256(nqt_), 608), 256, 0, s_>>>(vb1_, c_.d_xq, nqt_, red_);
    note_launch();
    double xs[3];
    ck(c_, cudaMemcpyAsync(xs, red_, sizeof(xs), cudaMemcpyDeviceToHost, s_), "reading the field cotangent");
    ck(c_, cudaStreamSynchronize(s_), "adjoint step");
    for (int p = 0; p < 3; ++p) theta_bar[p] -= dE[p][0] * xs[0] + dE[p][1] * xs[1] + dE[p][2] * xs[2];
    std::swap(lam_, lam_new_);
  }

 private:
  cudaError_t kexp(const double* in, double* out, double dt) {
    std::vector<double> dts((size_t)C_, dt);
    int k = 0, caps = 0;
    double eps = 0.0;
    cudaError_t e = run_kexp_cols(c_, in, out, dts.data(), prec_, &k, &caps, &eps, s_, true);
    cap_hits_ += caps;
    return e;
  }

  // v = v_N + v_H[rho] + v_xc(rho) - E . x
  void potential(const double* rho, const double E[3], double* v) {
    ck(c_, launch_lda(c_, rho, c_.d_vxc, nullptr, nqt_, s_), "LDA");
    int its = 0;
    ck(run_hartree(c_, rho, c_.d_vH, c_.cg_tol, c_.cg_max_it, &its, s_));
    ck(c_, launch_potential_sum(c_, c_.d_vH, c_.d_vxc, E, true, v, s_), "potential");
  }

  // out = V'(rho)^T g = w Interp(A_II^-1 Interp^T g) + f_xc(rho) g, where Interp^T g
  // is the load vector of g / w and A_II^-1 the direct solve with zero boundary data
  void vt(const double* rho, const double* g, double* out) {
    double* d = c_.d_cg;
    double* phi = c_.d_cg + c_.n_h;
    double* Ap = c_.d_cg + 2 * c_.n_h;
    k_div_w<<<nb256(nqt_), 256, 0, s_>>>(g, c_.d_wJ, tq2_, 1.0, nqt_);
    note_launch();
    if (c_.hen.on) {   // enriched Hartree solve: its own transpose
      double* w = c_.d_cg;
      ck(c_, hartree_enriched_vt(c_, tq2_, tq2_, w, w + c_.n_h, w + 2 * c_.n_h, w + 3 * c_.n_h, w + 4 * c_.n_h,
                                 w + 5 * c_.n_h, s_), "enriched Hartree transpose");
    } else {
      ck(c_, cudaMemsetAsync(d, 0, sizeof(double) * c_.n_h, s_), "memset");
      ck(c_, launch_load_vector(c_, tq2_, d, 1, s_), "load vector");
      ck(c_, fdm_solve(c_, d, Ap, phi, 1, s_, true), "Hartree transpose");
      ck(c_, launch_interp(c_, phi, tq2_, 1, s_), "interpolation");
    }
    k_vt_finish<<<nb256(nqt_), 256, 0, s_>>>(tq2_, c_.d_wJ, rho, g, out, nqt_);
    note_launch();
  }

  // acc += 2 occ Phi^T (rho_bar Phi psi) with the potential-only operator v = rho_bar / w
  void density_vjp(const double* psi, const double* rho_bar, double* acc) {
    k_div_w<<<nb256(nqt_), 256, 0, s_>>>(rho_bar, c_.d_wJ, tq2_, 1.0, nqt_);
    note_launch();
    ck(build_op(c_, tq2_, 1, 0.0, s_));
    ck(c_, launch_apply(c_, psi, tmp_, C_, C_, prec_, s_), "apply");
    k_occ_axpy<<<nb256(c_.n_dof * C_), 256, 0, s_>>>(acc, tmp_, c_.d_occ, c_.n_dof, (int)C_, c_.n_orb);
    note_launch();
  }

  // vbar = w dt int_0^1 Im sum_a conj(Phi a_a(s)) Phi b_a(s) ds by the Gauss-Legendre nodes,
  // b(s_k) = exp(-i s_k dt Hbar) psi given, a(s) = exp(+i (1-s) dt Hbar) lam recombined from
  // the Krylov basis of lam just built (for -dt)
  void frechet(const std::vector<double*>& b, double dt, double* vbar) {
    ck(c_, cudaMemsetAsync(vbar, 0, sizeof(double) * nqt_, s_), "memset");
    for (size_t k = 0; k < sk_.size(); ++k) {
      ck(c_, recombine(ba_, -(1.0 - sk_[k]) * dt), "Frechet node");
      ck(c_, cross_density(c_, ba_, b[k], wk_[k] * dt, vbar, s_), "cross density");
    }
  }

  cudaError_t recombine(double* out, double dt) {
    std::vector<double> dts((size_t)C_, dt);
    return run_kexp_recombine(c_, out, dts.data(), s_);
  }

  Ctx& c_;
  cudaStream_t s_;
  int prec_ = EFE_FP64;
  long long C_ = 0, nqt_ = 0, blk_ = 0, cap_hits_ = 0;
  Buffers buf_;
  double *rho0_, *rhop_, *rhom_, *v1_, *v2_, *vb1_, *vb2_, *rbar_, *rbm_, *tq_, *tq2_;
  double *psip_, *lam_, *lam_new_, *lamp_, *ba_, *tmp_, *red_;
  std::vector<double> sk_, wk_;
  std::vector<double*> b1_, b2_;   // exp(-i s_k dt H1) psi, exp(-i s_k dt H2) psi
};

}  // namespace

efe_status adjoint_dipole(Ctx& c, const double* psi0, int n_steps, double dt, const efe_field& f, const double dir[3],
                          int w_first, int w_last, int K, int n_s, double* J_out, double grad[3], cudaStream_t s) {
  const bool graphs = c.use_graphs;
  c.use_graphs = false;   // the exponentials run on operators rebuilt between calls
  efe_status st = EFE_OK;
  try {
    ck(ensure_ws(c, c.n_orb, c.n_orb));
    ck(ensure_krylov(c));
    if (c.kblock < c.n_orb) {   // the reverse sweep recombines one Krylov basis of every column
      c.err = "efe_adjoint_dipole needs the Krylov basis of all orbitals at once (krylov_block too small for them)";
      c.use_graphs = graphs;
      return EFE_ERR_ARG;
    }
    Sweep sw(c, s, n_s);
    const long long blk = sw.blk();
    const int n_ck = (n_steps + K - 1) / K;
    const int nW = w_last - w_first + 1;
    std::vector<double*> ck_psi((size_t)n_ck), seg((size_t)K + 1);
    for (auto& p : ck_psi) p = sw.block();
    for (auto& p : seg) p = sw.block();
    double* mu_dev = sw.scratch(3 * (size_t)nW);   // [nW][3] window dipoles
    std::vector<double> mus_h(3 * (size_t)nW);
    double E[3], dE[3][3];
    // forward with a checkpoint every K steps and the dipoles of the window
    ck(c, cudaMemcpyAsync(seg[0], psi0, sizeof(double) * blk, cudaMemcpyDeviceToDevice, s), "copy");
    for (int n = 0; n < n_steps; ++n) {
      double* cur = seg[n % 2];
      double* nxt = seg[(n + 1) % 2];
      if (n % K == 0) ck(c, cudaMemcpyAsync(ck_psi[n / K], cur, sizeof(double) * blk, cudaMemcpyDeviceToDevice, s), "copy");
      field_derivs(f, n * dt + 0.5 * dt, E, dE);
      sw.forward(cur, nxt, E, dt);
      if (n + 1 >= w_first && n + 1 <= w_last) {
        sw.dipole(nxt, mu_dev + 3 * (n + 1 - w_first));
      }
    }
    ck(c, cudaMemcpyAsync(mus_h.data(), mu_dev, sizeof(double) * mus_h.size(), cudaMemcpyDeviceToHost, s),
       "reading the dipoles");
    ck(c, cudaStreamSynchronize(s), "forward");
    double J = 0.0;
    for (int i = 0; i < nW; ++i) J += (dir[0] * mus_h[3 * i] + dir[1] * mus_h[3 * i + 1] + dir[2] * mus_h[3 * i + 2]) / nW;
    *J_out = J;
    // reverse sweep, one checkpoint segment at a time (its states recomputed first)
    grad[0] = grad[1] = grad[2] = 0.0;
    sw.zero_cotangents();
    for (int k = n_ck - 1; k >= 0; --k) {
      const int n0 = k * K, n1 = std::min(n0 + K, n_steps);
      ck(c, cudaMemcpyAsync(seg[0], ck_psi[k], sizeof(double) * blk, cudaMemcpyDeviceToDevice, s), "copy");
      for (int n = n0; n < n1; ++n) {
        field_derivs(f, n * dt + 0.5 * dt, E, dE);
        sw.forward(seg[n - n0], seg[n - n0 + 1], E, dt);
      }
      for (int n = n1; n > n0; --n) {
        if (n >= w_first && n <= w_last) sw.window_term(dir, -1.0 / nW);
        sw.density_to_lam(seg[n - n0]);
        field_derivs(f, (n - 1) * dt + 0.5 * dt, E, dE);
        sw.reverse_step(seg[n - 1 - n0], E, dE, dt, grad);
      }
    }
    ck(c, cudaStreamSynchronize(s), "reverse sweep");
    if (sw.cap_hits() > 0) st = EFE_WARN_KRYLOV_CAP;
  } catch (const Fail& e) {
    st = e.st;
  }
  c.use_graphs = graphs;
  c.state_valid = false;
  c.has_prev = false;
  c.op.valid = false;
  return st;
}

}  // namespace efe
