// Spectra from dipole traces (Sec. Results: the absorption spectrum of the
// weak-perturbation study and the power spectrum of the high-harmonic study).
// Samples f_n = f(t_n), t_n = n dt, n = 0..N; time integrals are the trapezoid
// rule, F[f](w) = dt sum_n c_n f_n e^{i w t_n}, c_0 = c_N = 1/2.  One block per
// frequency; its threads stride over the samples and reduce in shared memory.
#include <cmath>

#include "efe_internal.h"

namespace efe {

constexpr int kSpecThreads = 128;

// sum over the block of NV values per thread; the result is valid in thread 0
template <int NV>
__device__ void block_sum(double (&v)[NV], double* sh) {
  for (int o = 16; o > 0; o >>= 1)
    for (int k = 0; k < NV; ++k) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
    for (int k = 0; k < NV; ++k) sh[warp * NV + k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      for (int k = 0; k < NV; ++k) v[k] += sh[w * NV + k];
}

// S(w) = (4 w / (3 pi)) sum_j Im( F[g (mu_j^(j) - mu_j^(j)(0))](w) / F[E_0](w) ),  g = e^{-t/tau};
// mu[j * sdir + n * st + j]; F[E_0] from the field samples E, or = kick when E is NULL
__global__ void __launch_bounds__(kSpecThreads)
k_absorption(const double* __restrict__ mu, long long n_t, long long sdir, long long st, double dt,
             const double* __restrict__ E, double kick, const double* __restrict__ om, double tau,
             double* __restrict__ S) {
  __shared__ double sh[8 * (kSpecThreads / 32)];
  const long long w = blockIdx.x;
  const double omega = om[w];
  double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // (re, im) of the three traces and of the field
  for (long long n = threadIdx.x; n < n_t; n += blockDim.x) {
    const double t = (double)n * dt;
    const double c = (n == 0 || n == n_t - 1) ? 0.5 : 1.0;
    double sn, cs;
    sincos(omega * t, &sn, &cs);
    const double g = c * exp(-t / tau);
    for (int j = 0; j < 3; ++j) {
      const double d = (mu[j * sdir + n * st + j] - mu[j * sdir + j]) * g;
      v[2 * j] += d * cs;
      v[2 * j + 1] += d * sn;
    }
    if (E) {
      v[6] += c * E[n] * cs;
      v[7] += c * E[n] * sn;
    }
  }
  block_sum<8>(v, sh);
  if (threadIdx.x != 0) return;
  const double fr = E ? dt * v[6] : kick, fi = E ? dt * v[7] : 0.0;
  const double den = fr * fr + fi * fi;
  double im = 0.0;
  for (int j = 0; j < 3; ++j) im += (dt * v[2 * j + 1] * fr - dt * v[2 * j] * fi) / den;
  S[w] = 4.0 * omega / (3.0 * 3.14159265358979323846) * im;
}

// P(w) = | dt sum_{n=1}^{N-1} e^{-i w t_n} a_n e^{-t_n^2/tau} |^2,  a_n the central second
// difference of mu[n * st]
__global__ void __launch_bounds__(kSpecThreads)
k_power(const double* __restrict__ mu, long long n_t, long long st, double dt, const double* __restrict__ om,
        double tau, double* __restrict__ P) {
  __shared__ double sh[2 * (kSpecThreads / 32)];
  const long long w = blockIdx.x;
  const double omega = om[w];
  double v[2] = {0, 0};
  for (long long n = 1 + threadIdx.x; n < n_t - 1; n += blockDim.x) {
    const double t = (double)n * dt;
    const double a = (mu[(n + 1) * st] - 2.0 * mu[n * st] + mu[(n - 1) * st]) / (dt * dt);
    const double x = a * exp(-t * t / tau);
    double sn, cs;
    sincos(omega * t, &sn, &cs);
    v[0] += x * cs;
    v[1] -= x * sn;
  }
  block_sum<2>(v, sh);
  if (threadIdx.x != 0) return;
  P[w] = dt * dt * (v[0] * v[0] + v[1] * v[1]);
}

cudaError_t launch_absorption(const double* mu, long long n_t, long long sdir, long long st, double dt,
                              const double* E, double kick, const double* om, long long n_om, double tau, double* S,
                              cudaStream_t s) {
  k_absorption<<<(unsigned)n_om, kSpecThreads, 0, s>>>(mu, n_t, sdir, st, dt, E, kick, om, tau, S);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_power(const double* mu, long long n_t, long long st, double dt, const double* om, long long n_om,
                         double tau, double* P, cudaStream_t s) {
  k_power<<<(unsigned)n_om, kSpecThreads, 0, s>>>(mu, n_t, st, dt, om, tau, P);
  note_launch();
  return cudaGetLastError();
}

}  // namespace efe
