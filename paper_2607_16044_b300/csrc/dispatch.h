// Type-erased entry points into the per-(D, P, S) launch layer.  Every
// generated translation unit registers one table; the host code picks the
// table for the handle's dimension, degree and precision.
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "ops.cuh"

namespace dgx {

struct Table {
  // Individual kernel launches (the host composes residuals, stages and
  // adjoints); V selects the tile variant of tile kernels.
  cudaError_t (*trace)(const void* M, int V, const void* U, void* TU, cudaStream_t st);
  cudaError_t (*trace_from64)(const void* M, int V, const double* U, void* TU, void* shadow, cudaStream_t st);
  cudaError_t (*br1)(const void* M, int V, bool curv, const void* U, const Work& w, cudaStream_t st);
  cudaError_t (*face)(const void* M, bool visc, bool curv, const Work& w, cudaStream_t st);
  cudaError_t (*elem)(const void* M, int V, bool visc, bool curv, const void* U, const Work& w, void* out,
                      cudaStream_t st);
  cudaError_t (*elem_stage)(const void* M, int V, bool visc, bool curv, const void* U, const Work& w,
                            const void* stage, cudaStream_t st);
  // persistent TMA-fed element kernel; *used = false when it cannot run (nothing launched)
  cudaError_t (*elem_pipe)(const void* M, int V, bool visc, bool curv, const void* U, const Work& w, void* out,
                           const void* stage, int nsm, cudaStream_t st, bool* used);
  // tensor-core element kernel (FP32 tables only, else nullptr): tc = 1 TF32, 3 3xTF32;
  // stage == nullptr writes f to out, otherwise performs the ARK stage update
  cudaError_t (*elem_tc)(const void* M, int tc, bool visc, bool curv, const void* U, const Work& w, void* out,
                         const void* stage, cudaStream_t st);
  size_t (*smem)(int kind, int V);  // tile kernels: 0 trace, 1 br1, 2 elem
  const void* vjp;                   // adjoint launch table (VjpTable) or nullptr
  const void* dgip;                  // DG-IP scheme launch table (DgipTable) or nullptr
};

// Defined in the generated units: table for (D, P, S) or nullptr.
const Table* table_d2_f64(int P);
const Table* table_d3_f64(int P);
const Table* table_d2_f32(int P);
const Table* table_d3_f32(int P);

// DG-IP launch table (a DgipTable) alone for degrees 6 and 7, the point
// operator of over-integration with 7 or 8 points per direction; else nullptr.
const void* dgip_only_d2_f64(int P);
const void* dgip_only_d3_f64(int P);
const void* dgip_only_d2_f32(int P);
const void* dgip_only_d3_f32(int P);

}  // namespace dgx
