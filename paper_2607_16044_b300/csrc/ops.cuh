// Launch layer: one Ops<D, P, S> per (dimension, degree, precision), explicitly
// instantiated in generated translation units so the templates compile in
// parallel.  Each entry enqueues one kernel on a stream and returns the launch
// status; nothing here allocates or synchronises.  The host runtime composes
// residuals, ARK stages and adjoints from these launches and picks a tile
// variant (about 128 / 256 / 512 threads per CTA) per kernel.
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

constexpr size_t SMEM_LIMIT = 227 * 1024;  // opt-in shared memory per CTA on sm_103a

// Raise a kernel's dynamic shared-memory limit once (first launch); later
// launches -- including ones inside a stream capture -- skip the call.
template <typename K>
inline void allow_smem_once(K kernel, size_t bytes, bool& done) {
  if (!done) {
    if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    done = true;
  }
}

template <int D, int P, typename S>
struct Ops {
  template <int V>
  using H = Sh<D, P, V>;
  template <int V>
  static size_t smem_trace() {
    return sizeof(S) * (H<V>::T * H<V>::STATE + 2 * H<V>::n);
  }
  template <int V>
  static size_t smem_br1() {
    using h = H<V>;
    return sizeof(S) * (h::T * h::STATE + h::T * h::FACE + h::T * D * h::STATE + h::n * h::n + 4 * h::n);
  }
  template <int V>
  static size_t smem_elem() {
    using h = H<V>;
    return sizeof(S) * (h::T * D * h::STATE + h::T * h::FACE + h::n * h::n + 4 * h::n);
  }
  template <int V>
  static int blocks(int E) {
    return (E + H<V>::T - 1) / H<V>::T;
  }
  // shared memory of a tile kernel kind (0 trace, 1 br1, 2 elem) for variant V
  static size_t smem(int kind, int V) {
    switch (V) {
      case 0: return kind == 0 ? smem_trace<0>() : kind == 1 ? smem_br1<0>() : smem_elem<0>();
      case 1: return kind == 0 ? smem_trace<1>() : kind == 1 ? smem_br1<1>() : smem_elem<1>();
      default: return kind == 0 ? smem_trace<2>() : kind == 1 ? smem_br1<2>() : smem_elem<2>();
    }
  }

  template <typename Sin, int V>
  static cudaError_t trace_v(const Mesh<S>& M, const Sin* U, S* TU, S* shadow, cudaStream_t st) {
    static bool done = false;
    auto k = k_trace<D, P, S, Sin, V>;
    allow_smem_once(k, smem_trace<V>(), done);
    k<<<blocks<V>(M.E), H<V>::THREADS, smem_trace<V>(), st>>>(M.E, U, TU, shadow, M.tabs);
    return cudaGetLastError();
  }
  template <typename Sin>
  static cudaError_t trace(const Mesh<S>& M, int V, const Sin* U, S* TU, S* shadow, cudaStream_t st) {
    if (V == 0) return trace_v<Sin, 0>(M, U, TU, shadow, st);
    if (V == 1) return trace_v<Sin, 1>(M, U, TU, shadow, st);
    return trace_v<Sin, 2>(M, U, TU, shadow, st);
  }

  template <bool CURV, int V>
  static cudaError_t br1_v(const Mesh<S>& M, const S* U, const Work& w, cudaStream_t st) {
    static bool done = false;
    auto k = k_br1<D, P, S, CURV, V>;
    allow_smem_once(k, smem_br1<V>(), done);
    k<<<blocks<V>(M.E), H<V>::THREADS, smem_br1<V>(), st>>>(M, U, (const S*)w.TU, (S*)w.Q, (S*)w.G);
    return cudaGetLastError();
  }
  static cudaError_t br1(const Mesh<S>& M, int V, bool curv, const S* U, const Work& w, cudaStream_t st) {
    if (curv) {
      if (V == 0) return br1_v<true, 0>(M, U, w, st);
      if (V == 1) return br1_v<true, 1>(M, U, w, st);
      return br1_v<true, 2>(M, U, w, st);
    }
    if (V == 0) return br1_v<false, 0>(M, U, w, st);
    if (V == 1) return br1_v<false, 1>(M, U, w, st);
    return br1_v<false, 2>(M, U, w, st);
  }

  static cudaError_t face(const Mesh<S>& M, bool visc, bool curv, const Work& w, cudaStream_t st) {
    const int total = M.nFaces * Sh<D, P>::nfp;
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

  template <int MODE, bool VISC, bool CURV, int V>
  static cudaError_t elem_v(const Mesh<S>& M, const S* U, const Work& w, S* out, const Stage<S>& sa,
                            cudaStream_t st) {
    static bool done = false;
    auto k = k_elem<D, P, S, VISC, CURV, MODE, V>;
    allow_smem_once(k, smem_elem<V>(), done);
    k<<<blocks<V>(M.E), H<V>::THREADS, smem_elem<V>(), st>>>(M, U, (const S*)w.Q, (const S*)w.FF, out, sa);
    return cudaGetLastError();
  }
  template <int MODE, bool VISC, bool CURV>
  static cudaError_t elem_c(const Mesh<S>& M, int V, const S* U, const Work& w, S* out, const Stage<S>& sa,
                            cudaStream_t st) {
    if (V == 0) return elem_v<MODE, VISC, CURV, 0>(M, U, w, out, sa, st);
    if (V == 1) return elem_v<MODE, VISC, CURV, 1>(M, U, w, out, sa, st);
    return elem_v<MODE, VISC, CURV, 2>(M, U, w, out, sa, st);
  }
  template <int MODE>
  static cudaError_t elem(const Mesh<S>& M, int V, bool visc, bool curv, const S* U, const Work& w, S* out,
                          const Stage<S>& sa, cudaStream_t st) {
    if (visc) {
      if (curv) return elem_c<MODE, true, true>(M, V, U, w, out, sa, st);
      return elem_c<MODE, true, false>(M, V, U, w, out, sa, st);
    }
    if (curv) return elem_c<MODE, false, true>(M, V, U, w, out, sa, st);
    return elem_c<MODE, false, false>(M, V, U, w, out, sa, st);
  }
};

}  // namespace dgx
