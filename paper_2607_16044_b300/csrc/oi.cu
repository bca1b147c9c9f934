// Tensor-product transfer between the (k+1)-point solution nodes and the
// M-point quadrature points of the over-integrated DG-IP operator (Sec. 5:
// the nonlinear terms are integrated by a rule of order 3k).
//
// The over-integrated residual is f = Pi f'(I U): I interpolates the degree-k
// state to the M Gauss points, f' is the collocated DG-IP operator there (the
// degree-(M-1) kernels, with the penalty of the true degree), and
// Pi[q][m] = omega_m l_q(z_m) / w_q projects the result back (exact, because
// every degree-k test function lies in the degree-(M-1) space of the M
// points).  The adjoint uses the transposes.  This file holds the one kernel
// that applies such a 1D matrix along every direction.
//
// One CTA takes a tile of TE consecutive elements.  Their input block is
// contiguous in global memory and is copied coalesced into shared memory;
// each direction is one pass between two shared buffers in which a thread
// takes whole lines (the NI values of one fibre along the direction in,
// its NO values out: sum factorisation, NO x NI multiply-adds per line, the
// matrix entries compile-time indices into the kernel parameters); the last
// pass writes the tile's contiguous output block, consecutive threads on
// consecutive addresses.  Sizes are template parameters, so every index is
// a constant multiply.  The kernel moves nf (NI^D + NO^D) values per element;
// in FP64 its multiply-adds (1220 per element and field for 3D, 4 -> 5
// points) bound it on the FP64 pipe, in FP32 the traffic does.
//
// On curved elements the projection carries the Jacobians: with the
// collocated mass w_q J_q at the nodes and J' at the M points,
// f = J^-1 Pi (J' f'), and its transpose J' Pi^T (J^-1 lam) in the adjoint.
// The weighted form of the kernel scales every input point by a per-point
// factor as the tile is loaded and every output point by another before the
// store (the last pass then goes through shared memory, so the store stays
// one contiguous block).
#include <cuda_runtime.h>

#include "oi.h"

namespace dgx {

namespace {

template <typename S>
struct OiMat {
  S a[OI_MAXQ * OI_MAXQ];  // [no][ni]
};

constexpr int OI_THREADS = 256;

template <int B, int E>
struct Pow {
  static constexpr int v = B * Pow<B, E - 1>::v;
};
template <int B>
struct Pow<B, 0> {
  static constexpr int v = 1;
};

template <int D, int NI, int NO, typename S>
struct OiShape {
  static constexpr int nf = D + 2;
  static constexpr int MX = NI > NO ? NI : NO;
  static constexpr int ROW = Pow<MX, D>::v;  // largest extent of one (element, field) row
  // elements per tile: about 8 KB per shared buffer
  static constexpr int TE0 = 8192 / (nf * ROW * (int)sizeof(S));
  static constexpr int TE = TE0 < 1 ? 1 : (TE0 > 32 ? 32 : TE0);
  static constexpr int CAP = TE * nf * ROW;  // values per buffer
};

// Pass A of the tensor product: direction A goes from NI to NO values;
// directions < A already have NO, directions > A still NI.
template <int D, int NI, int NO, int A, typename S>
__device__ __forceinline__ void oi_pass(const S* __restrict__ x, S* __restrict__ y, int rows, const OiMat<S>& M) {
  constexpr int LO = Pow<NO, A>::v;               // extent of the directions before A
  constexpr int HI = Pow<NI, D - 1 - A>::v;       // extent of the directions after A
  constexpr int SZ_IN = LO * NI * HI, SZ_OUT = LO * NO * HI;
  constexpr int LINES = LO * HI;
  for (int i = threadIdx.x; i < rows * LINES; i += blockDim.x) {
    const int r = i / LINES, l = i - r * LINES;
    const int below = l % LO, above = l / LO;  // below fastest: consecutive threads, consecutive addresses
    const S* xs = x + r * SZ_IN + below + above * LO * NI;
    S v[NI];
#pragma unroll
    for (int k = 0; k < NI; ++k) v[k] = xs[k * LO];
    S* ys = y + r * SZ_OUT + below + above * LO * NO;
#pragma unroll
    for (int j = 0; j < NO; ++j) {
      S s = 0;
#pragma unroll
      for (int k = 0; k < NI; ++k) s += M.a[j * NI + k] * v[k];
      ys[j * LO] = s;
    }
  }
}

// W: scale the input points by pre[e][point] and the output points by
// post[e][point] (curved elements); otherwise pre and post are unused.
template <int D, int NI, int NO, bool W, typename S>
__global__ void __launch_bounds__(OI_THREADS) k_oi_apply(const S* __restrict__ in, S* __restrict__ out, int E,
                                                         OiMat<S> M, const S* __restrict__ pre,
                                                         const S* __restrict__ post) {
  using H = OiShape<D, NI, NO, S>;
  constexpr int nf = H::nf, TE = H::TE, RI = Pow<NI, D>::v, RO = Pow<NO, D>::v;
  __shared__ __align__(16) S buf[2][H::CAP];
  for (int e0 = blockIdx.x * TE; e0 < E; e0 += gridDim.x * TE) {
    const int nel = min(TE, E - e0);
    const int rows = nel * nf;
    const S* src = in + (size_t)e0 * nf * RI;
    if constexpr (W) {
      const S* pw = pre + (size_t)e0 * RI;
      for (int i = threadIdx.x; i < rows * RI; i += OI_THREADS) {
        const int r = i / RI, q = i - r * RI;
        buf[0][i] = src[i] * pw[(r / nf) * RI + q];
      }
    } else if (nel == TE) {  // full tile: a compile-time trip count, every load issued before the stores
#pragma unroll 4
      for (int i = threadIdx.x; i < TE * nf * RI; i += OI_THREADS) buf[0][i] = src[i];
    } else {
      for (int i = threadIdx.x; i < rows * RI; i += OI_THREADS) buf[0][i] = src[i];
    }
    __syncthreads();
    S* dst = out + (size_t)e0 * nf * RO;
    // the last pass writes the output block directly, or (W) the free buffer
    S* last = W ? buf[D == 2 ? 0 : 1] : dst;
    if constexpr (D == 2) {
      oi_pass<D, NI, NO, 0, S>(buf[0], buf[1], rows, M);
      __syncthreads();
      oi_pass<D, NI, NO, 1, S>(buf[1], last, rows, M);
    } else {
      oi_pass<D, NI, NO, 0, S>(buf[0], buf[1], rows, M);
      __syncthreads();
      oi_pass<D, NI, NO, 1, S>(buf[1], buf[0], rows, M);
      __syncthreads();
      oi_pass<D, NI, NO, 2, S>(buf[0], last, rows, M);
    }
    if constexpr (W) {
      __syncthreads();
      const S* qw = post + (size_t)e0 * RO;
      for (int i = threadIdx.x; i < rows * RO; i += OI_THREADS) {
        const int r = i / RO, q = i - r * RO;
        dst[i] = last[i] * qw[(r / nf) * RO + q];
      }
    }
    __syncthreads();
  }
}

template <int D, typename S, int NI, int NO>
cudaError_t run(const void* in, void* out, int E, const double* a, const void* pre, const void* post, int nsm,
                cudaStream_t st) {
  OiMat<S> M{};
  for (int i = 0; i < NO * NI; ++i) M.a[i] = (S)a[i];
  constexpr int TE = OiShape<D, NI, NO, S>::TE;
  const int tiles = (E + TE - 1) / TE;
  const int grid = tiles < nsm * 16 ? tiles : nsm * 16;
  if (pre)
    k_oi_apply<D, NI, NO, true, S>
        <<<grid, OI_THREADS, 0, st>>>((const S*)in, (S*)out, E, M, (const S*)pre, (const S*)post);
  else
    k_oi_apply<D, NI, NO, false, S><<<grid, OI_THREADS, 0, st>>>((const S*)in, (S*)out, E, M, nullptr, nullptr);
  return cudaGetLastError();
}

// (ni, no) pairs: the nodes have at most 6 points per direction (p <= 5), the
// quadrature points at most 8; one side of every transfer is the nodes.
template <int D, typename S, int NI>
cudaError_t by_no(int no, const void* in, void* out, int E, const double* a, const void* pre, const void* post,
                  int nsm, cudaStream_t st) {
  switch (no) {
    case 2: return run<D, S, NI, 2>(in, out, E, a, pre, post, nsm, st);
    case 3: return run<D, S, NI, 3>(in, out, E, a, pre, post, nsm, st);
    case 4: return run<D, S, NI, 4>(in, out, E, a, pre, post, nsm, st);
    case 5: return run<D, S, NI, 5>(in, out, E, a, pre, post, nsm, st);
    case 6: return run<D, S, NI, 6>(in, out, E, a, pre, post, nsm, st);
    case 7:
      if constexpr (NI <= 6) return run<D, S, NI, 7>(in, out, E, a, pre, post, nsm, st);
      return cudaErrorInvalidValue;
    case 8:
      if constexpr (NI <= 6) return run<D, S, NI, 8>(in, out, E, a, pre, post, nsm, st);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

template <int D, typename S>
cudaError_t by_ni(int ni, int no, const void* in, void* out, int E, const double* a, const void* pre,
                  const void* post, int nsm, cudaStream_t st) {
  switch (ni) {
    case 2: return by_no<D, S, 2>(no, in, out, E, a, pre, post, nsm, st);
    case 3: return by_no<D, S, 3>(no, in, out, E, a, pre, post, nsm, st);
    case 4: return by_no<D, S, 4>(no, in, out, E, a, pre, post, nsm, st);
    case 5: return by_no<D, S, 5>(no, in, out, E, a, pre, post, nsm, st);
    case 6: return by_no<D, S, 6>(no, in, out, E, a, pre, post, nsm, st);
    case 7:
      if (no <= 6) return by_no<D, S, 7>(no, in, out, E, a, pre, post, nsm, st);
      return cudaErrorInvalidValue;
    case 8:
      if (no <= 6) return by_no<D, S, 8>(no, in, out, E, a, pre, post, nsm, st);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t oi_apply(int D, bool fp64, const void* in, void* out, int E, int nf, int ni, int no, const double* a,
                     const void* pre, const void* post, int nsm, cudaStream_t st) {
  if (E <= 0) return cudaSuccess;
  if (nf != D + 2 || ni < 2 || no < 2 || ni > OI_MAXQ || no > OI_MAXQ || (D != 2 && D != 3) || (!pre != !post))
    return cudaErrorInvalidValue;
  if (D == 2)
    return fp64 ? by_ni<2, double>(ni, no, in, out, E, a, pre, post, nsm, st)
                : by_ni<2, float>(ni, no, in, out, E, a, pre, post, nsm, st);
  return fp64 ? by_ni<3, double>(ni, no, in, out, E, a, pre, post, nsm, st)
              : by_ni<3, float>(ni, no, in, out, E, a, pre, post, nsm, st);
}

}  // namespace dgx
