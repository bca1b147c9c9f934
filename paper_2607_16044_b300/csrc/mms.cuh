// Manufactured-solution source of Sec. 5.1.1 (the MMS of Gassner et al.) on
// the device: U_e = (s+4, s+4, s+4, (s+4)^2), s = sin(phi),
// phi = pi (kx x + ky y) - omega pi t, 2D, i.e. rho = s + 4, u = v = 1,
// rho E = rho^2, p = (gamma-1)(rho^2 - rho).  With u, v constant the stress
// vanishes and the heat flux is -(gamma mu / Pr) grad e with e = rho - 1, so
// S = dU_e/dt + div(F^c - F^nu)(U_e) is (c = cos phi, p' = (gamma-1)(2 rho - 1))
//   S_rho   = pi c (kx + ky - omega)
//   S_rho u = pi c (kx (1 + p') + ky - omega)
//   S_rho v = pi c (kx + ky (1 + p') - omega)
//   S_rho E = pi c ((kx + ky)(2 rho + p') - 2 rho omega) + (gamma mu / Pr) pi^2 (kx^2 + ky^2) s.
// Evaluated in FP64 at the Gauss nodes of box elements and added to dU/dt.
#pragma once
#include <cuda_runtime.h>

namespace dgx {

struct MmsNodes {
  double xi[6];  // the 1D Gauss nodes on [-1, 1]
};

template <typename S>
__global__ void __launch_bounds__(256) k_mms_source(int E, int n, MmsNodes nodes, const double* __restrict__ lo,
                                                    const double* __restrict__ size, double t, double kx, double ky,
                                                    double omega, double gm1, double kcv, S* __restrict__ out) {
  const int N = n * n;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long long)E * N) return;
  const int e = (int)(gid / N), q = (int)(gid % N);
  const double pi = 3.14159265358979323846;
  const double x = lo[e * 2] + 0.5 * (1.0 + nodes.xi[q % n]) * size[e * 2];
  const double y = lo[e * 2 + 1] + 0.5 * (1.0 + nodes.xi[q / n]) * size[e * 2 + 1];
  const double phi = pi * (kx * x + ky * y) - omega * pi * t;
  const double s = sin(phi), c = cos(phi);
  const double rho = s + 4.0;
  const double dp = gm1 * (2.0 * rho - 1.0);
  S* o = out + (size_t)e * 4 * N + q;
  o[0] += (S)(pi * c * (kx + ky - omega));
  o[N] += (S)(pi * c * (kx * (1.0 + dp) + ky - omega));
  o[2 * N] += (S)(pi * c * (kx + ky * (1.0 + dp) - omega));
  o[3 * N] += (S)(pi * c * ((kx + ky) * (2.0 * rho + dp) - 2.0 * rho * omega) + kcv * pi * pi * (kx * kx + ky * ky) * s);
}

}  // namespace dgx
