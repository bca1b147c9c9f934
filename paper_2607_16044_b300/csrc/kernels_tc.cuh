// Tensor-core (tcgen05, kind::tf32 or kind::f16) variant of the element kernel, FP32 only.
//
// The weak divergence plus lift of k_elem is, for every (direction a, element,
// field, line along a), the same small affine map of the line's values
//   out_k = sum_m Dh[k][m] x_m - Lm[k] Fhat^- - Lp[k] Fhat^+,   k < n,
// i.e. one row of a GEMM  OUT[rows x n] = X[rows x (n + 2)] * B^T with the
// fixed operand B = [Dh | -Lm | -Lp].  With n + 2 <= 8 one kind::tf32 MMA
// (M = 128, N = 16, K = 8) covers 128 rows; a tile of T elements has
// D * T * nf * nfp rows, processed by ceil(rows / 128) MMAs issued by one
// thread into a tensor-memory accumulator (16 columns per block of rows).
//
// Flow of one CTA: every node thread computes its volume fluxes and stores
// them straight into the K-major operand rows (column = position along a);
// the face fluxes fill columns n and n + 1; thread 0 issues the MMAs and
// commits them to an mbarrier (bounded wait, timeout -> flag bit 1); the
// warps read the accumulator back with tcgen05.ld (warp w sees TMEM lanes
// 32 (w % 4) ..), scale by 2/h_a and scatter to the node layout for the same
// per-node epilogue as k_elem (sum over directions, 1/J, stage update,
// traces of the next stage state).
//
// TC = 1: operands rounded to TF32 (about 11 significant bits).
// TC = 2: operands rounded to BF16 (8 significant bits), kind::f16 MMAs with
//         K = 16 (columns n + 2 .. 15 zero), FP32 accumulation.
// TC = 3: 3xTF32, x = hi + lo with both parts TF32; hi*hi + hi*lo + lo*hi
//         accumulated in FP32 recovers (nearly) FP32 accuracy.
#pragma once
#include <cuda_bf16.h>

#include "ops.cuh"
#include "umma.cuh"

namespace dgx {

constexpr int TC_V = 1;  // tile shape of the tensor-core element kernel (about 256 threads)

template <int D, int P, int TC>
struct TcShape {
  using H = Sh<D, P, TC_V>;
  static constexpr int ES = TC == 2 ? 2 : 4;               // operand element bytes (BF16 / TF32)
  static constexpr int K = 32 / ES;                        // K per MMA: 8 (kind::tf32), 16 (kind::f16)
  static constexpr int PADK = K - (H::n + 2);              // zero columns after the lift columns
  static constexpr int ROWS = D * H::T * H::nf * H::nfp;   // (direction, element, field, line)
  static constexpr int BLOCKS = (ROWS + 127) / 128;        // M = 128 rows per MMA
  static constexpr int COLS = 16 * BLOCKS;                 // N = 16 accumulator columns per block
  static constexpr uint32_t TMEM_COLS = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128 : COLS <= 256 ? 256 : 512;
  static constexpr int SPLIT = TC == 3 ? 2 : 1;            // 3xTF32 keeps hi and lo operands
  static constexpr size_t BLOCK_BYTES = 128 * K * ES;
  static constexpr size_t A_BYTES = (size_t)BLOCKS * BLOCK_BYTES;
  static constexpr size_t B_BYTES = 16 * K * ES;
  static constexpr size_t SMEM = SPLIT * (A_BYTES + B_BYTES) + r16(sizeof(float) * 2 * H::n) + 16;
  static_assert(PADK >= 0, "line length plus two lift columns must fit one MMA K step");
  static_assert(COLS <= 512, "accumulator exceeds tensor memory");
  static_assert(H::THREADS >= 128, "four warps are needed to read every TMEM lane quarter");
  static_assert(A_BYTES >= sizeof(float) * H::T * D * H::STATE, "node layout reuses the operand region");
};

template <int D, int P, bool VISC, bool CURV, int MODE, int TC>
__global__ void __launch_bounds__(Sh<D, P, TC_V>::THREADS)
    k_elem_tc(Mesh<float> M, const float* U, const float* __restrict__ Q, const float* __restrict__ FF,
              float* __restrict__ out, Stage<float> st) {
  using S = float;
  using H = Sh<D, P, TC_V>;
  using C = TcShape<D, P, TC>;
  constexpr int n = H::n, N = H::N, nf = H::nf, nfp = H::nfp, T = H::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* Ah = smem_raw;                                // [BLOCKS x 128 rows][K], K-major
  unsigned char* Al = smem_raw + C::A_BYTES;                   // lo parts (TC = 3)
  unsigned char* Bh = smem_raw + C::SPLIT * C::A_BYTES;        // [16 rows][K]
  unsigned char* Bl = Bh + C::B_BYTES;
  S* lm = reinterpret_cast<S*>(Bh + C::SPLIT * C::B_BYTES);
  S* lp = lm + n;
  unsigned char* ctl = reinterpret_cast<unsigned char*>(lm) + r16(sizeof(S) * 2 * n);
  uint64_t* bar = reinterpret_cast<uint64_t*>(ctl);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(ctl + 8);
  int* abort_flag = reinterpret_cast<int*>(ctl + 12);
  S* fs = reinterpret_cast<S*>(smem_raw);  // [T][D][nf][N] once the MMAs are done (reuses the operands)
  const int tid = threadIdx.x;
  const int e0 = blockIdx.x * T;
  const int nel = min(T, M.E - e0);

  if (tid < 32) tmem_alloc(tslot, C::TMEM_COLS);
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  // one operand element: BF16 (round to nearest even) or TF32 hi (and lo for 3xTF32)
  auto store = [&](unsigned char* hi_base, unsigned char* lo_base, uint32_t o, float v) {
    if constexpr (TC == 2) {
      *reinterpret_cast<__nv_bfloat16*>(hi_base + o) = __float2bfloat16_rn(v);
    } else {
      const float hi = tf32_rna(v);
      *reinterpret_cast<float*>(hi_base + o) = hi;
      if (TC == 3) *reinterpret_cast<float*>(lo_base + o) = tf32_rna(v - hi);
    }
  };
  auto put = [&](int row, int k, float v) { store(Ah, Al, umma_off32<C::ES>(row, k), v); };
  // rows are independent, so only the padding columns need defined (zero) values
  if constexpr (C::PADK > 0) {
    for (int i = tid; i < C::BLOCKS * 128 * C::PADK; i += blockDim.x) put(i / C::PADK, n + 2 + i % C::PADK, 0.f);
  }
  {
    const Tab<S>& tb = M.tabs[P];
    for (int i = tid; i < 16 * C::K; i += blockDim.x) {
      const int k = i / C::K, m = i % C::K;
      S v = 0;
      if (k < n) v = m < n ? tb.Dh[k * 6 + m] : (m == n ? -tb.Lm[k] : (m == n + 1 ? -tb.Lp[k] : S(0)));
      store(Bh, Bl, umma_off32<C::ES>(k, m), v);
    }
    for (int i = tid; i < n; i += blockDim.x) {
      lm[i] = tb.lm[i];
      lp[i] = tb.lp[i];
    }
  }
  const int t = tid / N, q = tid % N;
  const bool active = t < nel;
  const int e = e0 + t;
  S pre[nf];
  double pre64[nf];
  if (MODE == 1 && active) {
    const size_t off = (size_t)e * H::STATE + q;
    stage_prefix<nf, S>(
        st, e, [&](int f) { return st.base[off + f * N]; },
        [&](int j, int f) { return st.k[j][off + f * N]; }, [&](int f) { return st.Un[off + f * N]; }, pre, pre64);
  }
  if (active) {
    const S* up = U + (size_t)e * H::STATE + q;
    S Uq[nf];
#pragma unroll
    for (int f = 0; f < nf; ++f) Uq[f] = up[f * N];
    S Fa[D][nf];
    node_flux<D, S, VISC, CURV>(
        M.gas, Uq, [&](int c, int f) { return Q[(size_t)e * D * H::STATE + (c * nf + f) * N + q]; },
        [&](int a, int c) { return M.geo.Ja[(((size_t)e * D + a) * D + c) * N + q]; }, Fa);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int f = 0; f < nf; ++f) put(((a * T + t) * nf + f) * nfp + H::fpoint(q, a), H::qa(q, a), Fa[a][f]);
  }
  {  // face fluxes: column n takes the face at -1 of direction a, column n + 1 the face at +1
    const S* src = FF + (size_t)e0 * H::FACE;
    for (int i = tid; i < nel * H::FACE; i += blockDim.x) {
      const int tt = i / H::FACE, r = i % H::FACE;
      const int face = r / (nf * nfp), f = (r / nfp) % nf, line = r % nfp;
      put((((face >> 1) * T + tt) * nf + f) * nfp + line, n + (face & 1), src[i]);
    }
  }
  fence_proxy_async();  // generic-proxy operand stores -> visible to the tensor core
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  if (tid == 0) {
    const uint32_t idesc = TC == 2 ? umma_idesc_bf16(128, 16) : umma_idesc_tf32(128, 16);
    const uint64_t bh = umma_smem_desc(smem_u32(Bh), 128, 256);
    const uint64_t bl = umma_smem_desc(smem_u32(Bl), 128, 256);
    for (int b = 0; b < C::BLOCKS; ++b) {
      const uint32_t d = tmem + 16 * b;
      const uint64_t ah = umma_smem_desc(smem_u32(Ah + b * C::BLOCK_BYTES), 128, 256);
      if (TC == 2)
        umma_bf16(d, ah, bh, idesc, 0u);
      else
        umma_tf32(d, ah, bh, idesc, 0u);
      if (TC == 3) {
        const uint64_t al = umma_smem_desc(smem_u32(Al + b * C::BLOCK_BYTES), 128, 256);
        umma_tf32(d, ah, bl, idesc, 1u);
        umma_tf32(d, al, bh, idesc, 1u);
      }
    }
    umma_commit(bar);
    *abort_flag = !mbar_wait_bounded(bar, 0);
  }
  __syncthreads();
  const bool ok = *abort_flag == 0;  // CTA-uniform
  if (ok) {
    mbar_try(bar, 0);
    tc_fence_after();
    const int w = tid >> 5, lane = tid & 31, j = w & 3;
    const int nw = blockDim.x >> 5;
    const int cnt = (nw - j + 3) >> 2;  // warps that read lane quarter j
    for (int b = w >> 2; b < C::BLOCKS; b += cnt) {
      float v[8];
      tmem_ld8(tmem + ((uint32_t)(32 * j) << 16) + (uint32_t)(16 * b), v);
      const int row = 128 * b + 32 * j + lane;  // ((a T + tt) nf + f) nfp + line
      const int line = row % nfp, f = (row / nfp) % nf, tt = (row / (nf * nfp)) % T, a = row / (T * nf * nfp);
      if (row < C::ROWS && tt < nel) {
        const S r = CURV ? S(1) : M.geo.rh[(e0 + tt) * D + a];
        S* o = fs + ((tt * D + a) * nf + f) * N;
#pragma unroll
        for (int k = 0; k < n; ++k) o[H::node(k, line, a)] = r * v[k];
      }
    }
  } else if (tid == 0) {
    atomicOr(M.flags, 2u);
    mbar_wait_bounded(bar, 0);  // let the MMAs drain before the accumulator is freed
  }
  tc_fence_before();
  __syncthreads();
  if (tid < 32) {
    tc_fence_after();
    tmem_dealloc(tmem, C::TMEM_COLS);
  }
  if (!ok) return;
  S res[nf];
#pragma unroll
  for (int f = 0; f < nf; ++f) res[f] = S(0);
  if (active) {
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int f = 0; f < nf; ++f) res[f] += fs[((t * D + a) * nf + f) * N + q];
    if (CURV) {
      const S iJ = M.geo.iJ[(size_t)e * N + q];
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
    return;
  }
  S y[nf];
  if (active)
    stage_update<nf, S>(st, e, (size_t)e * H::STATE + q, N, res, pre, pre64, y);
  __syncthreads();  // everyone is done with fs
  if (active) {
#pragma unroll
    for (int f = 0; f < nf; ++f) fs[(t * nf + f) * N + q] = y[f];
  }
  __syncthreads();
  tile_traces<D, P, S, TC_V>(fs, nel, st.TU + (size_t)e0 * H::FACE);
}

// Launch layer of the tensor-core element kernel (FP32 handles only).
template <int D, int P>
struct TcOps {
  template <int MODE, bool VISC, bool CURV, int TC>
  static cudaError_t run(const Mesh<float>& M, const float* U, const Work& w, float* out, const Stage<float>& sa,
                         cudaStream_t st) {
    using C = TcShape<D, P, TC>;
    using H = Sh<D, P, TC_V>;
    static SmemGate done;
    auto k = k_elem_tc<D, P, VISC, CURV, MODE, TC>;
    if (const cudaError_t e = allow_smem_once(k, C::SMEM, done)) return e;
    const int blocks = (M.E + H::T - 1) / H::T;
    if (blocks == 0) return cudaSuccess;
    k<<<blocks, H::THREADS, C::SMEM, st>>>(M, U, (const float*)w.Q, (const float*)w.FF, out, sa);
    return cudaGetLastError();
  }
  template <int MODE, int TC>
  static cudaError_t mode_tc(const Mesh<float>& M, bool visc, bool curv, const float* U, const Work& w, float* out,
                             const Stage<float>& sa, cudaStream_t st) {
    if (visc) {
      if (curv) return run<MODE, true, true, TC>(M, U, w, out, sa, st);
      return run<MODE, true, false, TC>(M, U, w, out, sa, st);
    }
    if (curv) return run<MODE, false, true, TC>(M, U, w, out, sa, st);
    return run<MODE, false, false, TC>(M, U, w, out, sa, st);
  }
  // tc: 1 = TF32, 2 = BF16, 3 = 3xTF32; stage == nullptr writes f to out, otherwise the ARK stage update
  static cudaError_t elem(const Mesh<float>& M, int tc, bool visc, bool curv, const float* U, const Work& w,
                          float* out, const Stage<float>* stage, cudaStream_t st) {
    if (tc != 1 && tc != 2 && tc != 3) return cudaErrorInvalidValue;
    if (stage) {
      if (tc == 1) return mode_tc<1, 1>(M, visc, curv, U, w, nullptr, *stage, st);
      if (tc == 2) return mode_tc<1, 2>(M, visc, curv, U, w, nullptr, *stage, st);
      return mode_tc<1, 3>(M, visc, curv, U, w, nullptr, *stage, st);
    }
    Stage<float> none{};
    if (tc == 1) return mode_tc<0, 1>(M, visc, curv, U, w, out, none, st);
    if (tc == 2) return mode_tc<0, 2>(M, visc, curv, U, w, out, none, st);
    return mode_tc<0, 3>(M, visc, curv, U, w, out, none, st);
  }
};

}  // namespace dgx
