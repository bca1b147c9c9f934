// Persistent batched ARK step of an instance ensemble (2D box meshes).
//
// An ensemble's instances are grouped by degree and physics (each group one
// concatenated mesh, see host.cu).  Instead of one launch per group, kernel
// and stage, one persistent kernel per phase of the stage (first traces,
// BR1 gradient, face fluxes, element + stage update) covers every group: a
// grid of SMs x resident CTAs walks a list of work items (group, tile)
// ordered by decreasing degree and calls, for each item, the same tile
// function the group's own kernels run (trace_tile, br1_tile, face_point,
// elem_tile of kernels.cuh, 256-thread tiles), dispatched on the group's
// degree.  So a step is 1 + 3 s launches however many groups there are, every
// SM works on whichever instance has work left, and the arithmetic is that
// of the per-group kernels bit for bit.
#include "batchp.h"

namespace dgx {

namespace {

constexpr int BV = 1;  // tile variant of the persistent path (about 256 threads)

template <typename S>
constexpr size_t smax(size_t a, size_t b) {
  return a > b ? a : b;
}

template <typename S>
constexpr size_t batch_smem() {
  size_t m = 0;
  m = smax<S>(m, smem_trace_g<2, 1, S, BV>());
  m = smax<S>(m, smem_trace_g<2, 2, S, BV>());
  m = smax<S>(m, smem_trace_g<2, 3, S, BV>());
  m = smax<S>(m, smem_trace_g<2, 4, S, BV>());
  m = smax<S>(m, smem_trace_g<2, 5, S, BV>());
  m = smax<S>(m, smem_br1_g<2, 1, S, BV>());
  m = smax<S>(m, smem_br1_g<2, 2, S, BV>());
  m = smax<S>(m, smem_br1_g<2, 3, S, BV>());
  m = smax<S>(m, smem_br1_g<2, 4, S, BV>());
  m = smax<S>(m, smem_br1_g<2, 5, S, BV>());
  m = smax<S>(m, smem_elem_g<2, 1, S, BV>());
  m = smax<S>(m, smem_elem_g<2, 2, S, BV>());
  m = smax<S>(m, smem_elem_g<2, 3, S, BV>());
  m = smax<S>(m, smem_elem_g<2, 4, S, BV>());
  m = smax<S>(m, smem_elem_g<2, 5, S, BV>());
  return m;
}

template <typename S, int P, int PHASE>
__device__ __forceinline__ void run_item(int stage, const BGroup<S>& g, int unit, unsigned char* smem) {
  constexpr int phase = PHASE;
  if (phase == 0) {
    trace_tile<2, P, S, double, BV>(unit, smem, g.M.E, g.U64, (S*)g.w.TU, g.first);
  } else if (phase == 1) {
    br1_tile<2, P, S, false, BV>(unit, smem, g.M, g.Uin[stage], (const S*)g.w.TU, (S*)g.w.Q, (S*)g.w.G);
  } else if (phase == 2) {
    if (g.visc) face_point<2, P, S, true, false>(unit * 256 + (int)threadIdx.x, g.M, (const S*)g.w.TU,
                                                 (const S*)g.w.G, (S*)g.w.FF);
    else face_point<2, P, S, false, false>(unit * 256 + (int)threadIdx.x, g.M, (const S*)g.w.TU, nullptr,
                                           (S*)g.w.FF);
  } else {
    if (g.visc)
      elem_tile<2, P, S, true, false, 1, BV>(unit, smem, g.M, g.Uin[stage], (const S*)g.w.Q, (const S*)g.w.FF,
                                             nullptr, g.st[stage]);
    else
      elem_tile<2, P, S, false, false, 1, BV>(unit, smem, g.M, g.Uin[stage], nullptr, (const S*)g.w.FF, nullptr,
                                              g.st[stage]);
  }
}

template <typename S, int PHASE>
__global__ void __launch_bounds__(256) k_batch_phase(int stage, const BGroup<S>* __restrict__ groups,
                                                     const BItem* __restrict__ items, int nitems) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    __syncthreads();  // the previous item's last shared-memory reads are done
    const BItem w = items[it];
    const BGroup<S>& g = groups[w.g];
    switch (g.P) {
      case 1: run_item<S, 1, PHASE>(stage, g, w.unit, smem_raw); break;
      case 2: run_item<S, 2, PHASE>(stage, g, w.unit, smem_raw); break;
      case 3: run_item<S, 3, PHASE>(stage, g, w.unit, smem_raw); break;
      case 4: run_item<S, 4, PHASE>(stage, g, w.unit, smem_raw); break;
      default: run_item<S, 5, PHASE>(stage, g, w.unit, smem_raw); break;
    }
  }
}

}  // namespace

int batch_tile_elems(int P) {
  switch (P) {
    case 1: return Sh<2, 1, BV>::T;
    case 2: return Sh<2, 2, BV>::T;
    case 3: return Sh<2, 3, BV>::T;
    case 4: return Sh<2, 4, BV>::T;
    default: return Sh<2, 5, BV>::T;
  }
}

template <typename S, int PHASE>
cudaError_t launch_phase(int stage, const BGroup<S>* groups, const BItem* items, int nitems, int nsm,
                         cudaStream_t st) {
  constexpr size_t smem = batch_smem<S>();
  static SmemGate done;
  static int occ[64] = {};
  auto k = k_batch_phase<S, PHASE>;
  if (const cudaError_t e = allow_smem_once(k, smem, done)) return e;
  const int dv = current_device_bit();
  if (occ[dv] == 0) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, 256, smem) != cudaSuccess || o < 1) o = 1;
    occ[dv] = o;
  }
  const int grid = nitems < nsm * occ[dv] ? nitems : nsm * occ[dv];
  k<<<grid, 256, smem, st>>>(stage, groups, items, nitems);
  return cudaGetLastError();
}

template <typename S>
cudaError_t batch_phase(int phase, int stage, const BGroup<S>* groups, const BItem* items, int nitems, int nsm,
                        cudaStream_t st) {
  if (nitems == 0) return cudaSuccess;
  switch (phase) {
    case 0: return launch_phase<S, 0>(stage, groups, items, nitems, nsm, st);
    case 1: return launch_phase<S, 1>(stage, groups, items, nitems, nsm, st);
    case 2: return launch_phase<S, 2>(stage, groups, items, nitems, nsm, st);
    default: return launch_phase<S, 3>(stage, groups, items, nitems, nsm, st);
  }
}

template cudaError_t batch_phase<float>(int, int, const BGroup<float>*, const BItem*, int, int, cudaStream_t);
template cudaError_t batch_phase<double>(int, int, const BGroup<double>*, const BItem*, int, int, cudaStream_t);

}  // namespace dgx
