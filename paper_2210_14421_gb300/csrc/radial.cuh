// Smooth truncation of the atom-centred enrichment functions, shared by the
// set-up kernels of the wavefunction and the electrostatic enrichment.  The
// paper leaves the truncation unspecified: u = 1 for r <= r0 - s, u = 0 for
// r >= r0, and a C-infinity step in between.
#pragma once

namespace efe {

// smooth cutoff u(r) = 1 - S(t), t = (r - r0 + s)/s, S(t) = g(t)/(g(t)+g(1-t)), g = exp(-1/t)
__host__ __device__ __forceinline__ void cutoff(double r, double r0, double s, double& u, double& du) {
  const double t = (r - (r0 - s)) / s;
  if (t <= 0.0) { u = 1.0; du = 0.0; return; }
  if (t >= 1.0) { u = 0.0; du = 0.0; return; }
  const double g1 = exp(-1.0 / t), g2 = exp(-1.0 / (1.0 - t));
  const double den = g1 + g2;
  const double dg1 = g1 / (t * t), dg2 = g2 / ((1.0 - t) * (1.0 - t));
  u = 1.0 - g1 / den;
  du = -((dg1 * g2 + g1 * dg2) / (den * den)) / s;
}

}  // namespace efe
