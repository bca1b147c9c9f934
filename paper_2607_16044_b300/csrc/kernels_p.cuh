// Persistent, TMA-fed variants of the tile kernels (see pipe.cuh).
//
// Same arithmetic as kernels.cuh, but every contiguous per-tile input arrives
// by cp.async.bulk into a double buffer while the previous tile is computed;
// used whenever each block's bytes per element are a multiple of 16 (always
// in 2D; in 3D for an even node count N).
#pragma once
#include "kernels.cuh"
#include "pipe.cuh"

namespace dgx {

// Bounded-wait step shared by the persistent kernels: returns false (all
// threads) if the copy of buffer b did not complete within `polls` polls; then
// the kernel flags a timeout and returns after waiting (with the default
// bound, whatever `polls` is) for the copies still in flight into both
// buffers, so that no CTA leaves with a bulk copy outstanding.
__device__ __forceinline__ bool pipe_acquire(PipeState& ps, int b, uint32_t& par, bool other_pending,
                                             uint32_t other_par, unsigned* flags, uint32_t polls) {
  if (threadIdx.x == 0) ps.abort = !mbar_wait_bounded(&ps.bar[b], par, polls);
  __syncthreads();
  if (ps.abort) {
    if (threadIdx.x == 0) {
      atomicOr(flags, 2u);
      mbar_wait_bounded(&ps.bar[b], par);
      if (other_pending) mbar_wait_bounded(&ps.bar[b ^ 1], other_par);
    }
    return false;
  }
  mbar_try(&ps.bar[b], par);  // acquire the completed phase in every thread
  par ^= 1u;
  return true;
}

// ---------------------------------------------------------------------------
// k_elem_p: persistent k_elem.  Buffer layout per tile (T-element strides):
//   U [nf][N] | Q [D][nf][N] (VISC) | FF [NF][nf][nfp] | geometry (CURV: Ja, iJ)
//   | stage: base [nf][N] | k_0 .. k_{i-1} | U_n (double, last stage)
// ---------------------------------------------------------------------------
template <int D, int P, typename S, bool VISC, bool CURV, int MODE, int V>
__global__ void __launch_bounds__(Sh<D, P, V>::THREADS) k_elem_p(Mesh<S> M, TileIn in, S* __restrict__ out,
                                                                 Stage<S> st, int ntiles) {
  using H = Sh<D, P, V>;
  constexpr int n = H::n, N = H::N, nf = H::nf, nfp = H::nfp, NF = H::NF, T = H::T;
  constexpr Tab1<S> tb = make_tab1<S>(P);  // compile-time 1D tables
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ PipeState ps;
  const uint32_t buf_bytes = in.bytes_per_elem * T;
  auto buf = [&](int b) { return smem_raw + (size_t)b * buf_bytes; };  // the two tile buffers
  constexpr int FES = elem_flux_stride<D, P, V>(), SES = elem_state_stride<D, P, V>();
  S* fs = reinterpret_cast<S*>(smem_raw + 2 * buf_bytes);  // [T][D][nf][N] (stride FES), then [T][nf][N] (stride SES)
  if (threadIdx.x == 0) {
    mbar_init(&ps.bar[0], 1);
    mbar_init(&ps.bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  int tile = blockIdx.x;
  if (threadIdx.x == 0 && tile < ntiles) tile_issue(in, tile * T, min(T, M.E - tile * T), T, buf(0), &ps.bar[0]);
  uint32_t par[2] = {0u, 0u};
  for (int k = 0; tile < ntiles; ++k, tile += gridDim.x) {
    const int b = k & 1;
    const int next = tile + gridDim.x;
    if (threadIdx.x == 0 && next < ntiles)
      tile_issue(in, next * T, min(T, M.E - next * T), T, buf(b ^ 1), &ps.bar[b ^ 1]);
    if (!pipe_acquire(ps, b, par[b], next < ntiles, par[b ^ 1], M.flags, M.wait_polls)) return;
    const int e0 = tile * T;
    const int nel = min(T, M.E - e0);
    // views into the buffer
    const S* Us = reinterpret_cast<const S*>(buf(b));
    const S* Qs = Us + T * H::STATE;
    const S* FFs = VISC ? Qs + T * D * H::STATE : Qs;
    const S* geo = FFs + T * H::FACE;
    const S* Jas = geo;                                   // [T][D][D][N]
    const S* iJs = geo + T * D * D * N;                   // [T][N]
    const S* stg = CURV ? iJs + T * N : geo;
    const S* bases = stg;
    const S* kss = bases + T * H::STATE;                  // k_j: [i][T][nf][N]
    const double* Uns = reinterpret_cast<const double*>(kss + (size_t)st.i * T * H::STATE);
    const int t = threadIdx.x / N, q = threadIdx.x % N;
    const bool active = t < nel;
    const int e = e0 + t;
    S pre[nf];
    double pre64[nf];
    if (MODE == 1 && active) {
      const int off = t * H::STATE + q;
      stage_prefix<nf, S>(
          st, e, [&](int f) { return bases[off + f * N]; },
          [&](int j, int f) { return kss[(size_t)j * T * H::STATE + off + f * N]; },
          [&](int f) { return Uns[off + f * N]; }, pre, pre64);
    }
    if (active) {
      S Uq[nf];
#pragma unroll
      for (int f = 0; f < nf; ++f) Uq[f] = Us[t * H::STATE + f * N + q];
      S Fa[D][nf];
      node_flux<D, S, VISC, CURV>(
          M.gas, Uq, [&](int c, int f) { return Qs[t * D * H::STATE + (c * nf + f) * N + q]; },
          [&](int a, int c) { return Jas[((t * D + a) * D + c) * N + q]; }, Fa);
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int f = 0; f < nf; ++f) fs[t * FES + (a * nf + f) * N + q] = Fa[a][f];
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < D; ++a) {
      for (int i = threadIdx.x; i < nel * nf * nfp; i += blockDim.x) {
        int tt, f, line;
        line_item<nf, nfp>(i, tt, f, line);
        S* v = fs + tt * FES + (a * nf + f) * N;
        S x[n];
#pragma unroll
        for (int m = 0; m < n; ++m) x[m] = v[H::node(m, line, a)];
        const S ffm = FFs[((tt * NF + 2 * a) * nf + f) * nfp + line];
        const S ffp = FFs[((tt * NF + 2 * a + 1) * nf + f) * nfp + line];
        const S r = CURV ? S(1) : M.geo.rh[(e0 + tt) * D + a];
#pragma unroll
        for (int kk = 0; kk < n; ++kk) {
          S s = 0;
#pragma unroll
          for (int m = 0; m < n; ++m) s += tb.Dh[kk][m] * x[m];
          v[H::node(kk, line, a)] = r * (s - tb.Lm[kk] * ffm - tb.Lp[kk] * ffp);
        }
      }
    }
    __syncthreads();
    S res[nf];
#pragma unroll
    for (int f = 0; f < nf; ++f) res[f] = S(0);
    if (active) {
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int f = 0; f < nf; ++f) res[f] += fs[t * FES + (a * nf + f) * N + q];
      if (CURV) {
        const S iJ = iJs[t * N + q];
#pragma unroll
        for (int f = 0; f < nf; ++f) res[f] *= iJ;
      }
      flag_nonfinite<nf>(res, M.flags);
    }
    if (MODE == 0) {
      if (active) {
        S* op = out + (size_t)e * H::STATE + q;
#pragma unroll
        for (int f = 0; f < nf; ++f) op[f * N] = res[f];
      }
      __syncthreads();  // buffer and fs free for the next tile
      continue;
    }
    S y[nf];
    if (active)
      stage_update<nf, S>(st, e, (size_t)e * H::STATE + q, N, res, pre, pre64, y);
    __syncthreads();  // everyone is done with fs
    if (active) {
#pragma unroll
      for (int f = 0; f < nf; ++f) fs[t * SES + f * N + q] = y[f];
    }
    __syncthreads();
    tile_traces<D, P, S, V, SES>(fs, nel, st.TU + (size_t)e0 * H::FACE);
    __syncthreads();  // buffer and fs free for the next tile
  }
}

}  // namespace dgx
