// Arithmetic-throughput probe for roofline denominators (measurement only; no
// counterpart in the paper).  Every thread runs eight independent chains of
// fused multiply-adds x <- x * m + c in the requested precision, so the
// FMA pipe is never waiting on one chain's latency; the final values are
// stored so that nothing is optimised away.  One launch performs exactly
// 2 * 8 * iters * threads flops; the caller times it with CUDA events.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/dgx.h"

namespace {
template <typename S>
__global__ void __launch_bounds__(256) k_fma_chain(int64_t iters, S m, S c, S* __restrict__ out) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  S x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = S(1) + S(1e-3) * (S)((tid + k) & 255);
  // four iterations per trip so loop control takes a negligible share of issue slots
  int64_t i = 0;
  for (; i + 4 <= iters; i += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = fma(x[k], m, c);
  }
  for (; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], m, c);
  }
  S s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[tid] = s;
}
}  // namespace

extern "C" dgx_status dgx_probe_fma(int32_t precision, int64_t iters, void* out, int64_t threads, double* flops,
                                    void* stream) {
  if (!out || iters < 1 || threads < 256 || threads % 256 != 0 || threads / 256 > 0x7fffffff) return DGX_EINVAL;
  if (precision != DGX_FP64 && precision != DGX_FP32) return DGX_EINVAL;
  const int blocks = (int)(threads / 256);
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == DGX_FP64)
    k_fma_chain<double><<<blocks, 256, 0, st>>>(iters, 0.9999999, 1e-7, (double*)out);
  else
    k_fma_chain<float><<<blocks, 256, 0, st>>>(iters, 0.9999f, 1e-4f, (float*)out);
  if (cudaGetLastError() != cudaSuccess) return DGX_ECUDA;
  if (flops) *flops = 2.0 * 8.0 * (double)iters * (double)threads;
  return DGX_OK;
}
