// Persistent batched ARK step: host-side interface (see batchp.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"
#include "ops.cuh"

namespace dgx {

// One instance group of a batch, as the persistent kernels see it: its
// concatenated mesh, degree, physics, workspace views and the per-stage
// inputs and outputs of one ARK step (what the group's own ARK step would
// pass to its kernels).
template <typename S>
struct BGroup {
  Mesh<S> M;
  int P, visc;
  Work w;                      // TU, FF, G, Q of the group's workspace slice
  const double* U64;           // the group's FP64 state
  S* first;                    // FP32: rounded copy of U_n written by the first trace; FP64: nullptr
  const S* Uin[MAXSTAGES];     // stage input state
  Stage<S> st[MAXSTAGES];      // stage update (coefficients, pointers, per-element dt)
};

// Work item of a phase: (group, tile) for the tile phases, (group, block of
// 256 unique face points) for the face phase.
struct BItem {
  int g, unit;
};

// Launch one phase over all items (grid: min(items, SMs x resident CTAs)).
// phase: 0 first traces (FP64 state in), 1 BR1, 2 face, 3 element + stage update.
template <typename S>
cudaError_t batch_phase(int phase, int stage, const BGroup<S>* groups, const BItem* items, int nitems, int nsm,
                        cudaStream_t st);

// Elements per tile of degree P (the 256-thread CTA tile, 2D).
int batch_tile_elems(int P);

}  // namespace dgx
