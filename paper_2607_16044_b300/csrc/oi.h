// Over-integration of the DG-IP operator by an M-point Gauss rule (see oi.cu):
// host interface of the tensor-product transfer between the solution nodes
// and the quadrature points.
#pragma once
#include <cuda_runtime.h>

namespace dgx {

constexpr int OI_MAXQ = 8;  // points per direction (the DG-IP kernels' largest degree + 1)

// out[e][f] = (A x A [x A]) in[e][f]: the [no][ni] matrix A applied along
// every reference direction of each element's nodal field ([E][nf][ni^D] in,
// [E][nf][no^D] out, direction 0 fastest).  a is row-major in FP64.  With
// pre and post ([E][ni^D] and [E][no^D], the working precision; both or
// neither) the input points are scaled by pre and the output points by post:
// out = post . A (pre . in), the Jacobian weights of curved elements.
cudaError_t oi_apply(int D, bool fp64, const void* in, void* out, int E, int nf, int ni, int no, const double* a,
                     const void* pre, const void* post, int nsm, cudaStream_t st);

}  // namespace dgx
