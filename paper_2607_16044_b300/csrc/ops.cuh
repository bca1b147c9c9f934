// Launch layer: one Ops<D, P, S> per (dimension, degree, precision), explicitly
// instantiated in generated translation units so the templates compile in
// parallel.  Each entry enqueues one kernel on a stream and returns the launch
// status; nothing here allocates or synchronises.  The host runtime composes
// residuals, ARK stages and adjoints from these launches and picks a tile
// variant (about 128 / 256 / 512 threads per CTA) per kernel.
#pragma once
#include <cuda_runtime.h>

#include <atomic>

#include "kernels.cuh"
#include "kernels_p.cuh"

namespace dgx {

struct Work {            // caller-owned scratch, in the handle's precision
  void* TU;              // [E][2D][nf][nfp]
  void* FF;              // [E][2D][nf][nfp]
  void* G;               // [E][2D][nf][nfp]   (viscous)
  void* Q;               // [E][D][nf][N]      (viscous)
  void* TQ = nullptr;    // [E][2D][D][nf][nfp] traces of Q, stored by k_br1 when set (FP64 stage checkpoints)
};

constexpr size_t SMEM_LIMIT = 227 * 1024;  // opt-in shared memory per CTA on sm_103a

// Raise a kernel's dynamic shared-memory limit once per device (the
// attribute is per device): the first launch on each device sets it, later
// launches -- including ones inside a stream capture -- skip the call.  The
// gate keeps one bit per device ordinal (0..63) and reports the attribute
// call's error.
struct SmemGate {
  std::atomic<unsigned long long> done{0};
};
inline int current_device_bit() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
  return dev & 63;
}
template <typename K>
inline cudaError_t allow_smem_once(K kernel, size_t bytes, SmemGate& gate) {
  const unsigned long long bit = 1ull << current_device_bit();
  if (gate.done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  if (bytes > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
  }
  gate.done.fetch_or(bit, std::memory_order_acq_rel);
  return cudaSuccess;
}

template <int D, int P, typename S>
struct Ops {
  template <int V>
  using H = Sh<D, P, V>;
  // dynamic shared memory of one CTA (all of its element groups)
  template <int V>
  static size_t smem_trace() {
    return H<V>::GROUPS * smem_trace_g<D, P, S, V>();
  }
  template <int V>
  static size_t smem_br1() {
    return H<V>::GROUPS * smem_br1_g<D, P, S, V>();
  }
  template <int V>
  static size_t smem_elem() {
    return H<V>::GROUPS * smem_elem_g<D, P, S, V>();
  }
  template <int V>
  static int blocks(int E) {
    return H<V>::WARP ? (E + WPB - 1) / WPB : (E + H<V>::T - 1) / H<V>::T;
  }
  // shared memory of a tile kernel kind (0 trace, 1 br1, 2 elem) for variant V;
  // a variant that cannot run here reports SIZE_MAX
  template <int V>
  static size_t smem_v(int kind) {
    if (!H<V>::VALID) return (size_t)-1;
    return kind == 0 ? smem_trace<V>() : kind == 1 ? smem_br1<V>() : smem_elem<V>();
  }
  static size_t smem(int kind, int V) {
    switch (V) {
      case 0: return smem_v<0>(kind);
      case 1: return smem_v<1>(kind);
      case 2: return smem_v<2>(kind);
      default: return smem_v<3>(kind);
    }
  }

  template <typename Sin, int V>
  static cudaError_t trace_v(const Mesh<S>& M, const Sin* U, S* TU, S* shadow, cudaStream_t st) {
    static SmemGate done;
    auto k = k_trace<D, P, S, Sin, V>;
    if (const cudaError_t e = allow_smem_once(k, smem_trace<V>(), done)) return e;
    k<<<blocks<V>(M.E), H<V>::THREADS, smem_trace<V>(), st>>>(M.E, U, TU, shadow, M.tabs);
    return cudaGetLastError();
  }
  template <typename Sin>
  static cudaError_t trace(const Mesh<S>& M, int V, const Sin* U, S* TU, S* shadow, cudaStream_t st) {
    if (V == 0) return trace_v<Sin, 0>(M, U, TU, shadow, st);
    if (V == 1) return trace_v<Sin, 1>(M, U, TU, shadow, st);
    if (V == 2) return trace_v<Sin, 2>(M, U, TU, shadow, st);
    return trace_v<Sin, 3>(M, U, TU, shadow, st);
  }

  template <bool CURV, int V>
  static cudaError_t br1_v(const Mesh<S>& M, const S* U, const Work& w, cudaStream_t st) {
    static SmemGate done;
    auto k = k_br1<D, P, S, CURV, V>;
    if (const cudaError_t e = allow_smem_once(k, smem_br1<V>(), done)) return e;
    k<<<blocks<V>(M.E), H<V>::THREADS, smem_br1<V>(), st>>>(M, U, (const S*)w.TU, (S*)w.Q, (S*)w.G, (S*)w.TQ);
    return cudaGetLastError();
  }
  static cudaError_t br1(const Mesh<S>& M, int V, bool curv, const S* U, const Work& w, cudaStream_t st) {
    if (curv) {
      if (V == 0) return br1_v<true, 0>(M, U, w, st);
      if (V == 1) return br1_v<true, 1>(M, U, w, st);
      if (V == 2) return br1_v<true, 2>(M, U, w, st);
      return br1_v<true, 3>(M, U, w, st);
    }
    if (V == 0) return br1_v<false, 0>(M, U, w, st);
    if (V == 1) return br1_v<false, 1>(M, U, w, st);
    if (V == 2) return br1_v<false, 2>(M, U, w, st);
    return br1_v<false, 3>(M, U, w, st);
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
    static SmemGate done;
    auto k = k_elem<D, P, S, VISC, CURV, MODE, V>;
    if (const cudaError_t e = allow_smem_once(k, smem_elem<V>(), done)) return e;
    k<<<blocks<V>(M.E), H<V>::THREADS, smem_elem<V>(), st>>>(M, U, (const S*)w.Q, (const S*)w.FF, out, sa);
    return cudaGetLastError();
  }
  template <int MODE, bool VISC, bool CURV>
  static cudaError_t elem_c(const Mesh<S>& M, int V, const S* U, const Work& w, S* out, const Stage<S>& sa,
                            cudaStream_t st) {
    if (V == 0) return elem_v<MODE, VISC, CURV, 0>(M, U, w, out, sa, st);
    if (V == 1) return elem_v<MODE, VISC, CURV, 1>(M, U, w, out, sa, st);
    if (V == 2) return elem_v<MODE, VISC, CURV, 2>(M, U, w, out, sa, st);
    return elem_v<MODE, VISC, CURV, 3>(M, U, w, out, sa, st);
  }
  // ---- persistent TMA-fed element kernel
  template <int MODE, bool VISC, bool CURV, int V>
  static cudaError_t elem_p_v(const Mesh<S>& M, const TileIn& in, S* out, const Stage<S>& sa, int nsm,
                              cudaStream_t st, bool& used) {
    using h = H<V>;
    const size_t smem =
        2 * (size_t)h::T * in.bytes_per_elem + sizeof(S) * h::T * elem_flux_stride<D, P, V>();
    if (smem + sizeof(PipeState) > SMEM_LIMIT) {  // static pipeline state shares the per-CTA limit
      used = false;
      return cudaSuccess;
    }
    auto k = k_elem_p<D, P, S, VISC, CURV, MODE, V>;
    static size_t raised[64] = {};  // dynamic shared memory allowed so far for this kernel, per device
    const int dv = current_device_bit();
    if (smem > 48 * 1024 && smem > raised[dv]) {
      if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        used = false;
        return cudaSuccess;
      }
      raised[dv] = smem;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, h::THREADS, smem) != cudaSuccess || occ < 1) {
      used = false;
      return cudaSuccess;
    }
    const int ntiles = blocks<V>(M.E);
    const int grid = ntiles < nsm * occ ? ntiles : nsm * occ;
    k<<<grid, h::THREADS, smem, st>>>(M, in, out, sa, ntiles);
    used = true;
    return cudaGetLastError();
  }
  template <int MODE, bool VISC, bool CURV>
  static cudaError_t elem_p_c(const Mesh<S>& M, int V, const TileIn& in, S* out, const Stage<S>& sa, int nsm,
                              cudaStream_t st, bool& used) {
    if (V == 0) return elem_p_v<MODE, VISC, CURV, 0>(M, in, out, sa, nsm, st, used);
    if (V == 1) return elem_p_v<MODE, VISC, CURV, 1>(M, in, out, sa, nsm, st, used);
    if (V == 2) return elem_p_v<MODE, VISC, CURV, 2>(M, in, out, sa, nsm, st, used);
    used = false;  // the warp-per-element variant has no persistent form
    return cudaSuccess;
  }
  // Tries the persistent kernel; used = false (nothing launched) when a block
  // cannot be streamed or the buffers do not fit.
  template <int MODE>
  static cudaError_t elem_pipe(const Mesh<S>& M, int V, bool visc, bool curv, const S* U, const Work& w, S* out,
                               const Stage<S>& sa, int nsm, cudaStream_t st, bool& used) {
    using h = Sh<D, P>;
    const size_t s = sizeof(S);
    TileIn in{};
    bool ok = tilein_add(in, U, h::STATE * s);
    if (visc) ok = ok && tilein_add(in, w.Q, D * h::STATE * s);
    ok = ok && tilein_add(in, w.FF, h::FACE * s);
    if (curv) ok = ok && tilein_add(in, M.geo.Ja, D * D * h::N * s) && tilein_add(in, M.geo.iJ, h::N * s);
    if (MODE == 1) {
      ok = ok && tilein_add(in, sa.base, h::STATE * s);
      for (int j = 0; j < sa.i; ++j) ok = ok && tilein_add(in, sa.k[j], h::STATE * s);
      if (sa.last) ok = ok && tilein_add(in, sa.Un, h::STATE * sizeof(double));
    }
    used = false;
    if (!ok) return cudaSuccess;
    if (visc) {
      if (curv) return elem_p_c<MODE, true, true>(M, V, in, out, sa, nsm, st, used);
      return elem_p_c<MODE, true, false>(M, V, in, out, sa, nsm, st, used);
    }
    if (curv) return elem_p_c<MODE, false, true>(M, V, in, out, sa, nsm, st, used);
    return elem_p_c<MODE, false, false>(M, V, in, out, sa, nsm, st, used);
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
