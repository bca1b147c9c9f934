// Element-local HDG-IP Newton blocks (see hdg.cu): host interface.
#pragma once
#include <cuda_runtime.h>

#include "physics.cuh"

namespace dgx {

struct HdgArgs {
  int E;
  const double* rh;   // boxes: [E][2] 2/h_a (nullptr on curved meshes)
  const double* il;   // [E] 1/l = |dT| / |T|
  // curved meshes (nullptr on boxes): Ja [E][2][2][N] = J dxi_a/dx_c, iJ [E][N],
  // SnE [E][4][2][nfp] own area normals, JaF [E][4][2][2][nfp] and iJF [E][4][nfp]
  // the metric terms traced to the own face points
  const double* Ja;
  const double* iJ;
  const double* SnE;
  const double* JaF;
  const double* iJF;
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
