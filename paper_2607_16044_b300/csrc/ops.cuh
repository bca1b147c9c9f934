// Launch layer: one Ops<D, P, S> per (dimension, degree, precision), explicitly
// instantiated in generated translation units so the templates compile in
// parallel.  Each entry enqueues one kernel on a stream and returns the launch
// status; nothing here allocates or synchronises.  The host runtime composes
// residuals, ARK stages and adjoints from these launches.
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace dgx {

struct Work {            // caller-owned scratch, in the handle's precision
  void* TU;              // [E][2D][nf][nfp]
  void* FF;              // [E][2D][nf][nfp]
  void* G;               // [E][2D][nf][nfp]   (viscous)
  void* Q;               // [E][D][nf][N]      (viscous)
};

template <int D, int P, typename S>
struct Ops {
  using H = Sh<D, P>;
  static size_t smem_trace() { return sizeof(S) * (H::T * H::STATE + 2 * H::n); }
  static size_t smem_br1() {
    return sizeof(S) * (H::T * H::STATE + H::T * H::FACE + H::T * D * H::STATE + H::n * H::n + 4 * H::n);
  }
  static size_t smem_elem() { return sizeof(S) * (H::T * D * H::STATE + H::T * H::FACE + H::n * H::n + 4 * H::n); }
  static int blocks(int E) { return (E + H::T - 1) / H::T; }

  template <typename K>
  static void allow_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  }

  template <typename Sin>
  static cudaError_t trace(const Mesh<S>& M, const Sin* U, S* TU, S* shadow, cudaStream_t st) {
    auto k = k_trace<D, P, S, Sin>;
    allow_smem(k, smem_trace());
    k<<<blocks(M.E), H::THREADS, smem_trace(), st>>>(M.E, U, TU, shadow, M.tabs);
    return cudaGetLastError();
  }

  static cudaError_t br1(const Mesh<S>& M, bool curv, const S* U, const Work& w, cudaStream_t st) {
    if (curv) {
      auto k = k_br1<D, P, S, true>;
      allow_smem(k, smem_br1());
      k<<<blocks(M.E), H::THREADS, smem_br1(), st>>>(M, U, (const S*)w.TU, (S*)w.Q, (S*)w.G);
    } else {
      auto k = k_br1<D, P, S, false>;
      allow_smem(k, smem_br1());
      k<<<blocks(M.E), H::THREADS, smem_br1(), st>>>(M, U, (const S*)w.TU, (S*)w.Q, (S*)w.G);
    }
    return cudaGetLastError();
  }

  static cudaError_t face(const Mesh<S>& M, bool visc, bool curv, const Work& w, cudaStream_t st) {
    const int total = M.nFaces * H::nfp;
    const int nb = (total + 255) / 256;
    if (total == 0) return cudaSuccess;
    const S* TU = (const S*)w.TU;
    const S* G = (const S*)w.G;
    S* FF = (S*)w.FF;
    if (visc) {
      if (curv) k_face<D, P, S, true, true><<<nb, 256, 0, st>>>(M, TU, G, FF);
      else k_face<D, P, S, true, false><<<nb, 256, 0, st>>>(M, TU, G, FF);
    } else {
      if (curv) k_face<D, P, S, false, true><<<nb, 256, 0, st>>>(M, TU, G, FF);
      else k_face<D, P, S, false, false><<<nb, 256, 0, st>>>(M, TU, G, FF);
    }
    return cudaGetLastError();
  }

  template <int MODE>
  static cudaError_t elem(const Mesh<S>& M, bool visc, bool curv, const S* U, const Work& w, S* out,
                          const Stage<S>& sa, cudaStream_t st) {
    const size_t sm = smem_elem();
    const S* Q = (const S*)w.Q;
    const S* FF = (const S*)w.FF;
#define DGX_ELEM(V, C)                                   \
  {                                                      \
    auto k = k_elem<D, P, S, V, C, MODE>;                \
    allow_smem(k, sm);                                   \
    k<<<blocks(M.E), H::THREADS, sm, st>>>(M, U, Q, FF, out, sa); \
  }
    if (visc) {
      if (curv) DGX_ELEM(true, true) else DGX_ELEM(true, false)
    } else {
      if (curv) DGX_ELEM(false, true) else DGX_ELEM(false, false)
    }
#undef DGX_ELEM
    return cudaGetLastError();
  }

};

}  // namespace dgx
