// Type-erased entry points into the per-(D, P, S) launch layer.  Every
// generated translation unit registers one table; the host code picks the
// table for the handle's dimension, degree and precision.
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "ops.cuh"

namespace dgx {

struct Table {
  cudaError_t (*rhs)(const void* M, bool visc, bool curv, const void* U, void* out, const Work& w, cudaStream_t st);
  cudaError_t (*trace_from64)(const void* M, const double* U, void* TU, void* shadow, cudaStream_t st);
  cudaError_t (*stage)(const void* M, bool visc, bool curv, const void* U, const Work& w, const void* stage,
                       cudaStream_t st);
  cudaError_t (*vjp)(const void* M, bool visc, bool curv, const void* U, const void* lam, void* g, const void* vw,
                     cudaStream_t st);  // nullptr until the adjoint kernels are compiled in
};

// Defined in the generated units: table for (D, P, S) or nullptr.
const Table* table_d2_f64(int P);
const Table* table_d3_f64(int P);
const Table* table_d2_f32(int P);
const Table* table_d3_f32(int P);

}  // namespace dgx
