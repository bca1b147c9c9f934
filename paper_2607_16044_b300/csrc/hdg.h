// Element-local HDG-IP Newton blocks (see hdg.cu): host interface.
#pragma once
#include <cuda_runtime.h>

#include "physics.cuh"

namespace dgx {

struct HdgArgs {
  int E;
  const double* rh;   // [E][2] 2/h_a
  const double* il;   // [E] 1/l = |dT| / |T|
  const int* nb;      // [E][4] neighbour or -(1+tag)
  double tk2;         // alpha (k+1)^2, alpha = 10 for HDG-IP
  double w[6];        // 1D Gauss weights
  double Uinf[4];     // farfield state
  Gas<double> gas;
};

cudaError_t hdg_jacobian(int P, const HdgArgs& a, const double* U, const double* Uh, double gamma, double* K,
                         double* C, double* Dm, double* A33, double* Rv, double* hv, cudaStream_t st);
cudaError_t hdg_condense(int E, int NU, int NH, const double* K, const double* C, const double* Dm, const double* A33,
                         double* X, double* S, double* W, cudaStream_t st);

}  // namespace dgx
