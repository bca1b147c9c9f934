// Forward kernels of the explicit DG right-hand side (sm_103a).
//
// One CTA owns a tile of T consecutive elements, one thread per node
// (T * N threads rounded up to whole warps).  Element data is contiguous in
// HBM (U[E][nf][N]), so a tile is one contiguous block that is staged into
// shared memory with linear (fully coalesced) copies; every face quantity is
// stored per element and face ([E][2d][nf][n^(d-1)]) so that a tile's face
// data is contiguous too.
//
// Pipeline per residual (Sec. 3.3 weak form; LLF/BR1 reading):
//   k_trace  U -> TU            face traces of U (Gauss nodes: full-line dot products)
//   k_br1    U, TU -> Q, G      BR1 lifted gradient, its traces, each side's viscous
//                               normal flux G = F^nu(U_f, Q_f) . n_own     (NS only)
//   k_face   TU, G -> FF        one thread per unique face point: LLF flux minus the
//                               central viscous flux, written to both sides
//   k_elem   U, Q, FF -> f      volume flux, sum-factorised weak divergence, lift,
//                               inverse mass; optionally the ARK stage update and the
//                               face traces of the next stage state (fused epilogue)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "basis1d.h"
#include "physics.cuh"

namespace dgx {

constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

// Tile variants (chosen per kernel by the autotuner).  V = 0, 1, 2: one CTA
// per tile of T = max(1, 64 * 2^(V+1) / N) elements (about 128 / 256 / 512
// threads), phases separated by __syncthreads.  V = 3 (elements of at most 32
// nodes): one warp per element, WPB warps per CTA, each warp with its own
// shared-memory slice and __syncwarp between phases -- no CTA barriers.
constexpr int NVARIANTS = 4;
constexpr int WARP_VARIANT = 3;
constexpr int WPB = 8;
constexpr int variant_threads(int V) { return 64 << (V + 1); }

template <int D, int P, int V = 1>
struct Sh {
  static constexpr int n = P + 1;
  static constexpr int N = ipow(n, D);
  static constexpr int nf = D + 2;
  static constexpr int nfp = ipow(n, D - 1);
  static constexpr int NF = 2 * D;
  static constexpr bool WARP = (V == WARP_VARIANT);
  static constexpr int T = WARP ? 1 : ((variant_threads(V) / N) > 0 ? (variant_threads(V) / N) : 1);
  static constexpr int THREADS = WARP ? 32 * WPB : ((T * N + 31) / 32) * 32;
  static constexpr int GROUPS = WARP ? WPB : 1;  // independent element groups per CTA
  static constexpr bool VALID = !WARP || N <= 32;
  static constexpr int FACE = NF * nf * nfp;  // face values per element
  static constexpr int STATE = nf * N;        // state values per element
  __host__ __device__ static constexpr int pw(int a) { return a == 0 ? 1 : (a == 1 ? n : (a == 2 ? n * n : n * n * n)); }
  // face-point index of node q on the faces normal to direction a
  __device__ static __forceinline__ int fpoint(int q, int a) { return q % pw(a) + (q / pw(a + 1)) * pw(a); }
  // node at position m along direction a through face point fp
  __device__ static __forceinline__ int node(int m, int fp, int a) {
    return fp % pw(a) + m * pw(a) + (fp / pw(a)) * pw(a + 1);
  }
  __device__ static __forceinline__ int qa(int q, int a) { return (q / pw(a)) % n; }
};

// Thread-group primitives: a group is the whole CTA (V < 3) or one warp (V = 3).
template <int V>
__device__ __forceinline__ int g_tid() {
  return V == WARP_VARIANT ? (int)(threadIdx.x & 31) : (int)threadIdx.x;
}
template <int V>
__device__ __forceinline__ int g_size() {
  return V == WARP_VARIANT ? 32 : (int)blockDim.x;
}
template <int V>
__device__ __forceinline__ int g_index() {
  return V == WARP_VARIANT ? (int)(blockIdx.x * WPB + (threadIdx.x >> 5)) : (int)blockIdx.x;
}
template <int V>
__device__ __forceinline__ void g_sync() {
  if (V == WARP_VARIANT) __syncwarp();
  else __syncthreads();
}
template <int V>
__device__ __forceinline__ unsigned char* g_smem(unsigned char* base, size_t group_bytes) {
  return V == WARP_VARIANT ? base + (threadIdx.x >> 5) * group_bytes : base;
}

// Own face point -> neighbour face point (orientation code, see dgx.h).
template <int D, int n>
__device__ __forceinline__ int orient_map(int code, int fp) {
  if (D == 2) return (code & 1) ? (n - 1 - fp) : fp;
  int s = fp % n, t = fp / n;
  if (code & 4) {
    const int tmp = s;
    s = t;
    t = tmp;
  }
  const int u = (code & 1) ? (n - 1 - s) : s;
  const int v = (code & 2) ? (n - 1 - t) : t;
  return u + n * v;
}

// 1D tables for one degree (n <= 6): D[i][j] = l_j'(x_i), Dh[i][m] = w_m D[m][i] / w_i,
// lm/lp = l_j(-1)/l_j(+1), Lm/Lp = l_j(-1)/w_j, l_j(+1)/w_j.
template <typename S>
struct Tab {
  S D[36], Dh[36], lm[6], lp[6], Lm[6], Lp[6];
};

template <typename S>
struct Geo {
  const S* rh;   // boxes: [E][D] 2 / h_a
  const S* Ja;   // curvilinear: [E][D][D][N], Ja[a][c] = J dxi_a / dx_c
  const S* iJ;   // curvilinear: [E][N] 1 / J
  const S* SnE;  // curvilinear: [E][2D][D][nfp] own outward area normal
  const S* SnF;  // curvilinear: [F][D][nfp] averaged area normal of each unique face
};

template <typename S>
struct Mesh {
  int E, nFaces;
  const int* nb;       // [E][2D]
  const int8_t* nbf;   // [E][2D]
  const int8_t* ori;   // [E][2D]
  const int4* faces;   // [nFaces]: x = owner element, y = other element or -(1+tag),
                       //           z = owner face | other face << 8 | orient << 16
  Geo<S> geo;
  const Tab<S>* tabs;  // indexed by p
  Gas<S> gas;
  unsigned* flags;     // bit 0: non-finite residual, bit 1: a bounded device wait gave up
  uint32_t wait_polls; // bound of the persistent kernels' consumer waits (polls)
};

constexpr int MAXSTAGES = 8;

template <typename S>
struct Stage {
  const S* k[MAXSTAGES];   // k_0 .. k_{i-1}
  // Stage coefficients in the working precision, formed as products of S
  // values (S(dt) * S(a)) so that per-element and uniform time steps give
  // identical numbers and FP32 kernels do no FP64 arithmetic (FP64 runs at
  // ~1/64 of the FP32 rate on this part):
  S caf[MAXSTAGES];        // S(dt) S(a_{i+1, j}), j <= i      (uniform dt)
  S cbf[MAXSTAGES];        // S(dt) S(b_j)  (last stage)      (uniform dt)
  S ca[MAXSTAGES];         // S(a_{i+1, j})                    (with dte)
  S cb[MAXSTAGES];         // S(b_j)                           (with dte)
  const S* dte;            // per-element time step in S (batched instances) or nullptr
  int i;                   // this stage (0-based)
  int last;
  const S* base;           // y = base + sum ca_j k_j (FP64: U_n itself, FP32: fl32(U_n))
  double* Un;              // FP64 master state (updated at the last stage)
  S* Y;                    // next stage state (may alias the stage input)
  S* Kout;                 // k_i
  S* shadow;               // FP32 only: fl32(U_{n+1}) written at the last stage
  S* TU;                   // traces of the next stage state
};

template <typename S, int V = 1>
__device__ __forceinline__ void load_tab(const Tab<S>* tabs, int P, S* slm, S* slp, S* sLm, S* sLp, int n) {
  const Tab<S>& t = tabs[P];
  for (int i = g_tid<V>(); i < n; i += g_size<V>()) {
    if (slm) slm[i] = t.lm[i];
    if (slp) slp[i] = t.lp[i];
    if (sLm) sLm[i] = t.Lm[i];
    if (sLp) sLp[i] = t.Lp[i];
  }
}

// Shared-memory bytes of one element group (rounded to 16) for each tile kernel.
constexpr size_t r16(size_t b) { return (b + 15) & ~(size_t)15; }
template <int D, int P, typename S, int V>
constexpr size_t smem_trace_g() {
  using h = Sh<D, P, V>;
  return r16(sizeof(S) * h::T * h::STATE);
}
template <int D, int P, typename S, int V>
constexpr size_t smem_br1_g() {
  using h = Sh<D, P, V>;
  return r16(sizeof(S) * (h::T * h::STATE + h::T * h::FACE + h::T * D * h::STATE + h::T * h::NF * D * h::nf * h::nfp +
                          2 * h::n));
}
// Element strides (in scalars) of the element kernels' shared tiles, padded so
// that the line passes of neighbouring elements fall in different banks: the
// [T][D][nf][N] flux tile and the [T][nf][N] state tile whose traces are
// emitted.  Pads minimise the mean wavefronts per warp access of the line
// passes (threads over (element, field, line), line fastest) for each tile
// shape of the CTA variants, found by enumerating the 32 residues.
template <int D, int P, int V>
constexpr int flux_pad() {
  if (V > 2) return 0;  // one element per warp: nothing to separate
  constexpr int p2[6] = {0, 1, 28, 5, 28, 15};
  constexpr int p3[6] = {0, 15, 18, 5, 30, 15};
  return D == 2 ? p2[P] : (P == 4 && V == 0) || (P == 5 && V < 2) ? 0 : p3[P];
}
template <int D, int P, int V>
constexpr int state_pad() {
  if (V > 2) return 0;
  return (D == 2 && (P == 3 || P == 5)) ? (P == 3 ? 5 : 1) : (D == 3 && (P == 1 || P == 3)) ? (P == 1 ? 1 : 5) : 0;
}
template <int D, int P, int V>
constexpr int elem_flux_stride() {
  return D * Sh<D, P, V>::STATE + flux_pad<D, P, V>();
}
template <int D, int P, int V>
constexpr int elem_state_stride() {
  return Sh<D, P, V>::STATE + state_pad<D, P, V>();
}
template <int D, int P, typename S, int V>
constexpr size_t smem_elem_g() {
  using h = Sh<D, P, V>;
  return r16(sizeof(S) * (h::T * elem_flux_stride<D, P, V>() + h::T * h::FACE));
}

// Work items of a line pass along direction a: (element t, field f, line), the
// line being the face-point index of the faces normal to a.
template <int nf, int nfp>
__device__ __forceinline__ void line_item(int i, int& t, int& f, int& line) {
  line = i % nfp;
  f = (i / nfp) % nf;
  t = i / (nfp * nf);
}

// Tile staging, one thread per node (rows of [T][ROWS][N] tile arrays) or per
// face point (rows of [T][NF][nf][nfp]): each thread issues all of its loads
// before its first store, so their latencies overlap.
template <int D, int P, typename S, int V, int ROWS, typename Sin>
__device__ __forceinline__ void stage_nodes(S* dst, const Sin* src, int nel, S* copy = nullptr) {
  using H = Sh<D, P, V>;
  constexpr int N = H::N;
  const int t = g_tid<V>() / N, q = g_tid<V>() % N;
  if (t >= nel) return;
  S v[ROWS];
#pragma unroll
  for (int r = 0; r < ROWS; ++r) v[r] = (S)src[(t * ROWS + r) * N + q];
#pragma unroll
  for (int r = 0; r < ROWS; ++r) dst[(t * ROWS + r) * N + q] = v[r];
  if (copy) {
#pragma unroll
    for (int r = 0; r < ROWS; ++r) copy[(t * ROWS + r) * N + q] = v[r];
  }
}

template <int D, int P, typename S, int V>
__device__ __forceinline__ void stage_faces(S* dst, const S* src, int nel) {
  using H = Sh<D, P, V>;
  constexpr int nf = H::nf, nfp = H::nfp, NF = H::NF;
  for (int i = g_tid<V>(); i < nel * NF * nfp; i += g_size<V>()) {
    const int fp = i % nfp, tf = i / nfp;  // tf = t * NF + face
    S v[nf];
#pragma unroll
    for (int f = 0; f < nf; ++f) v[f] = src[(tf * nf + f) * nfp + fp];
#pragma unroll
    for (int f = 0; f < nf; ++f) dst[(tf * nf + f) * nfp + fp] = v[f];
  }
}

// Traces of a staged tile (us[t][f][q]): one thread per (element, field, line)
// and direction loads the line once and writes both end values.
template <int D, int P, typename S, int V, int ES = Sh<D, P, V>::STATE>
__device__ __forceinline__ void tile_traces(const S* us, int nel, S* dst) {  // us: [T][nf][N], element stride ES
  using H = Sh<D, P, V>;
  constexpr int n = H::n, nf = H::nf, nfp = H::nfp, N = H::N;
  constexpr Tab1<S> tb = make_tab1<S>(P);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    for (int i = g_tid<V>(); i < nel * nf * nfp; i += g_size<V>()) {
      int t, f, line;
      line_item<nf, nfp>(i, t, f, line);
      const S* v = us + t * ES + f * N;
      S sm = 0, sp = 0;
#pragma unroll
      for (int m = 0; m < n; ++m) {
        const S x = v[H::node(m, line, a)];
        sm += tb.lm[m] * x;
        sp += tb.lp[m] * x;
      }
      S* o = dst + (size_t)t * H::FACE + f * nfp + line;
      o[(2 * a) * nf * nfp] = sm;
      o[(2 * a + 1) * nf * nfp] = sp;
    }
  }
}

// ---------------------------------------------------------------------------
// k_trace: TU = traces of U (input may be double while S is float: the FP32
// ARK path converts the FP64 master state here and keeps the rounded copy).
// ---------------------------------------------------------------------------
// One element tile (also the unit of work of the persistent batched kernels).
template <int D, int P, typename S, typename Sin, int V>
__device__ __forceinline__ void trace_tile(int tile, unsigned char* smem_raw, int E, const Sin* __restrict__ U,
                                           S* __restrict__ TU, S* __restrict__ shadow) {
  using H = Sh<D, P, V>;
  S* us = reinterpret_cast<S*>(g_smem<V>(smem_raw, smem_trace_g<D, P, S, V>()));
  const int e0 = tile * H::T;
  const int nel = min(H::T, E - e0);
  stage_nodes<D, P, S, V, H::nf>(us, U + (size_t)e0 * H::STATE, nel,
                                  shadow ? shadow + (size_t)e0 * H::STATE : nullptr);
  g_sync<V>();
  tile_traces<D, P, S, V>(us, nel, TU + (size_t)e0 * H::FACE);
}

template <int D, int P, typename S, typename Sin, int V>
__global__ void __launch_bounds__(Sh<D, P, V>::THREADS) k_trace(int E, const Sin* __restrict__ U,
                                                                S* __restrict__ TU, S* __restrict__ shadow,
                                                                const Tab<S>* tabs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  trace_tile<D, P, S, Sin, V>(g_index<V>(), smem_raw, E, U, TU, shadow);
}

// ---------------------------------------------------------------------------
// k_br1: BR1 lifted gradient (conservative variables)
//   Q_c(q) = (1/J) sum_b Ja[b][c] (D_b U)(q) + sum_faces l_{q_a}(+-1)/(w_{q_a} J) (Uhat - U^-) Sn_c
// Uhat = (U^- + U^+)/2 inside, U_w on walls.  Writes Q and each own face's
// viscous normal flux G = F^nu(U_f, Q_f) . n (wall: adiabatic wall flux).
// Boxes use unit normals (the element kernel applies 2/h_a).  Contractions run
// one thread per line: the line is loaded once and all n outputs produced.
// ---------------------------------------------------------------------------
template <int D, int P, typename S, bool CURV, int V>
__device__ __forceinline__ void br1_tile(int tile, unsigned char* smem_raw, const Mesh<S>& M, const S* __restrict__ U,
                                         const S* __restrict__ TU, S* __restrict__ Q, S* __restrict__ G,
                                         S* __restrict__ TQg = nullptr) {
  using H = Sh<D, P, V>;
  constexpr int n = H::n, N = H::N, nf = H::nf, nfp = H::nfp, NF = H::NF, T = H::T;
  constexpr Tab1<S> tb = make_tab1<S>(P);  // compile-time 1D tables
    S* us = reinterpret_cast<S*>(g_smem<V>(smem_raw, smem_br1_g<D, P, S, V>()));     // [T][nf][N]
  S* js = us + T * H::STATE;                   // [T][NF][nf][nfp]     jumps
  S* qs = js + T * H::FACE;                    // [T][D][nf][N]        Q
  S* tq = qs + T * D * H::STATE;               // [T][NF][D][nf][nfp]  traces of Q
  S* Lm = tq + T * NF * D * nf * nfp;         // node-indexed lift weights (curvilinear)
  S* Lp = Lm + n;
  const int e0 = tile * T;
  const int nel = min(T, M.E - e0);
  stage_nodes<D, P, S, V, nf>(us, U + (size_t)e0 * H::STATE, nel);
  load_tab<S, V>(M.tabs, P, nullptr, nullptr, Lm, Lp, n);  // node-indexed lift (curvilinear)
  // jumps Uhat - U^- at every own face point.  When one thread covers one face
  // point, it keeps that point's trace U^- and neighbour for the flux phase.
  constexpr bool ONE = T * NF * nfp <= (H::WARP ? 32 : H::THREADS);
  auto load_face = [&](int i, S (&UL)[nf], int& nbe) {
    const int e = e0 + i / (nfp * NF), face = (i / nfp) % NF;
    const S* tl = TU + ((size_t)e * NF + face) * nf * nfp + i % nfp;
#pragma unroll
    for (int f = 0; f < nf; ++f) UL[f] = tl[f * nfp];
    nbe = M.nb[e * NF + face];
  };
  auto jump_at = [&](int i, const S (&UL)[nf], int nbe) {
    const int fp = i % nfp;
    const int face = (i / nfp) % NF;
    const int t = i / (nfp * NF);
    const int e = e0 + t;
    S* jd = js + (t * NF + face) * nf * nfp + fp;
    if (nbe >= 0) {
      const int fpn = orient_map<D, n>(M.ori[e * NF + face], fp);
      const S* tr = TU + ((size_t)nbe * NF + M.nbf[e * NF + face]) * nf * nfp + fpn;
#pragma unroll
      for (int f = 0; f < nf; ++f) jd[f * nfp] = S(0.5) * (tr[f * nfp] - UL[f]);
    } else {
      S W[nf];
      wall_state<D, S>(UL, W);
#pragma unroll
      for (int f = 0; f < nf; ++f) jd[f * nfp] = W[f] - UL[f];
    }
  };
  S pUL[nf];
  int pnb = -1;
  const bool has1 = ONE && g_tid<V>() < nel * NF * nfp;
  if (ONE) {
    if (has1) {
      load_face(g_tid<V>(), pUL, pnb);
      jump_at(g_tid<V>(), pUL, pnb);
    }
  } else {
    for (int i = g_tid<V>(); i < nel * NF * nfp; i += g_size<V>()) {
      S UL[nf];
      int nbe;
      load_face(i, UL, nbe);
      jump_at(i, UL, nbe);
    }
  }
  g_sync<V>();
  // derivative lines along each direction (boxes: the Q_a of this direction, lift included)
#pragma unroll
  for (int a = 0; a < D; ++a) {
    for (int i = g_tid<V>(); i < nel * nf * nfp; i += g_size<V>()) {
      int t, f, line;
      line_item<nf, nfp>(i, t, f, line);
      const S* v = us + (t * nf + f) * N;
      S x[n];
#pragma unroll
      for (int m = 0; m < n; ++m) x[m] = v[H::node(m, line, a)];
      S* qo = qs + ((t * D + a) * nf + f) * N;
      S* qg = Q + ((size_t)(e0 + t) * D + a) * H::STATE + f * N;  // the same row in global memory
      if (!CURV) {
        const S r = M.geo.rh[(e0 + t) * D + a];
        const S jm = js[((t * NF + 2 * a) * nf + f) * nfp + line];
        const S jp = js[((t * NF + 2 * a + 1) * nf + f) * nfp + line];
        S sm = 0, sp = 0;
#pragma unroll
        for (int k = 0; k < n; ++k) {
          S d = 0;
#pragma unroll
          for (int m = 0; m < n; ++m) d += tb.D[k][m] * x[m];
          const S qk = r * (d + tb.Lp[k] * jp - tb.Lm[k] * jm);
          qo[H::node(k, line, a)] = qk;
          qg[H::node(k, line, a)] = qk;
          sm += tb.lm[k] * qk;
          sp += tb.lp[k] * qk;
        }
        // this line ends on the two faces normal to a: the traces of Q_a there
        tq[(((t * NF + 2 * a) * D + a) * nf + f) * nfp + line] = sm;
        tq[(((t * NF + 2 * a + 1) * D + a) * nf + f) * nfp + line] = sp;
      } else {
#pragma unroll
        for (int k = 0; k < n; ++k) {
          S d = 0;
#pragma unroll
          for (int m = 0; m < n; ++m) d += tb.D[k][m] * x[m];
          qo[H::node(k, line, a)] = d;  // D_a U, combined below
        }
      }
    }
  }
  g_sync<V>();
  if (CURV) {  // Q_c = (1/J) (sum_b Ja[b][c] D_b U + sum_faces lift (Uhat - U) Sn_c), per node
    const int t = g_tid<V>() / N, q = g_tid<V>() % N;
    const bool act = t < nel;
    S Qv[D][nf];
    if (act) {
      const int e = e0 + t;
      const S iJ = M.geo.iJ[(size_t)e * N + q];
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int f = 0; f < nf; ++f) {
          S s = 0;
#pragma unroll
          for (int b = 0; b < D; ++b)
            s += M.geo.Ja[(((size_t)e * D + b) * D + c) * N + q] * qs[((t * D + b) * nf + f) * N + q];
          Qv[c][f] = s;
        }
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int fp = H::fpoint(q, a), qa = H::qa(q, a);
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          const int face = 2 * a + side;
          const S L = side ? Lp[qa] : Lm[qa];
          const S* jd = js + (t * NF + face) * nf * nfp + fp;
#pragma unroll
          for (int c = 0; c < D; ++c) {
            const S sn = M.geo.SnE[(((size_t)e * NF + face) * D + c) * nfp + fp];
#pragma unroll
            for (int f = 0; f < nf; ++f) Qv[c][f] += L * jd[f * nfp] * sn;
          }
        }
      }
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int f = 0; f < nf; ++f) Qv[c][f] *= iJ;
    }
    g_sync<V>();  // every D_b U has been read
    if (act) {
      S* qg = Q + (size_t)(e0 + t) * D * H::STATE + q;
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int f = 0; f < nf; ++f) {
          qs[((t * D + c) * nf + f) * N + q] = Qv[c][f];
          qg[(c * nf + f) * N] = Qv[c][f];
        }
    }
    g_sync<V>();
  }
  // traces of Q: one thread per (face direction a, component c, field, line);
  // on boxes the component c = a came out of the derivative lines already
  constexpr int NC = CURV ? D : D - 1;  // components per face direction left to trace
#pragma unroll
  for (int a = 0; a < D; ++a) {
    for (int i = g_tid<V>(); i < nel * NC * nf * nfp; i += g_size<V>()) {
      const int line = i % nfp;
      const int f = (i / nfp) % nf;
      const int cc = (i / (nfp * nf)) % NC;
      const int c = CURV ? cc : cc + (cc >= a);
      const int t = i / (nfp * nf * NC);
      const S* v = qs + ((t * D + c) * nf + f) * N;
      S sm = 0, sp = 0;
#pragma unroll
      for (int m = 0; m < n; ++m) {
        const S x = v[H::node(m, line, a)];
        sm += tb.lm[m] * x;
        sp += tb.lp[m] * x;
      }
      tq[(((t * NF + 2 * a) * D + c) * nf + f) * nfp + line] = sm;
      tq[(((t * NF + 2 * a + 1) * D + c) * nf + f) * nfp + line] = sp;
    }
  }
  g_sync<V>();
  if (TQg) {  // keep the traces of Q for the adjoint (the tile's block is contiguous)
    constexpr int TQS = NF * D * nf * nfp;
    S* dst = TQg + (size_t)e0 * TQS;
    for (int i = g_tid<V>(); i < nel * TQS; i += g_size<V>()) dst[i] = tq[i];
  }
  // own-face viscous fluxes
  auto flux_at = [&](int i, const S (&UL)[nf], int nbe) {
    const int fp = i % nfp;
    const int face = (i / nfp) % NF;
    const int t = i / (nfp * NF);
    const int e = e0 + t;
    const int a = face >> 1;
    S TQ[D][nf], nv[D];
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int f = 0; f < nf; ++f) TQ[c][f] = tq[(((t * NF + face) * D + c) * nf + f) * nfp + fp];
    if (CURV) {
#pragma unroll
      for (int c = 0; c < D; ++c) nv[c] = M.geo.SnE[(((size_t)e * NF + face) * D + c) * nfp + fp];
    } else {
#pragma unroll
      for (int c = 0; c < D; ++c) nv[c] = (c == a) ? ((face & 1) ? S(1) : S(-1)) : S(0);
    }
    S Gv[nf];
    if (nbe < 0)
      wall_visc_flux<D, S>(UL, TQ, nv, M.gas, Gv);
    else if (CURV)
      visc_flux_normal<D, S>(UL, TQ, nv, M.gas, Gv);
    else  // axis normal: the one row of the flux
      visc_flux_axis_rt<D, S>(UL, TQ, a, (face & 1) ? S(1) : S(-1), M.gas, Gv);
    S* gd = G + ((size_t)e * NF + face) * nf * nfp + fp;
#pragma unroll
    for (int f = 0; f < nf; ++f) gd[f * nfp] = Gv[f];
  };
  if (ONE) {
    if (has1) flux_at(g_tid<V>(), pUL, pnb);
  } else {
    for (int i = g_tid<V>(); i < nel * NF * nfp; i += g_size<V>()) {
      S UL[nf];
      int nbe;
      load_face(i, UL, nbe);
      flux_at(i, UL, nbe);
    }
  }
}

template <int D, int P, typename S, bool CURV, int V>
__global__ void __launch_bounds__(Sh<D, P, V>::THREADS) k_br1(Mesh<S> M, const S* __restrict__ U,
                                                              const S* __restrict__ TU, S* __restrict__ Q,
                                                              S* __restrict__ G, S* __restrict__ TQ) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  br1_tile<D, P, S, CURV, V>(g_index<V>(), smem_raw, M, U, TU, Q, G, TQ);
}

// ---------------------------------------------------------------------------
// k_face: one thread per unique face point.  Fhat = LLF(U^-, U^+; n) - Fhat^nu,
// Fhat^nu = (G^- - G^+)/2 inside, G^- on walls; written as +Fhat to the owner
// side and -Fhat to the other side.  Boxes: unit normals; curvilinear: the
// averaged area normal of the face.
// ---------------------------------------------------------------------------
template <int D, int P, typename S, bool VISC, bool CURV>
__device__ __forceinline__ void face_point(int gid, const Mesh<S>& M, const S* __restrict__ TU,
                                           const S* __restrict__ G, S* __restrict__ FF) {
  using H = Sh<D, P>;
  constexpr int n = H::n, nf = H::nf, nfp = H::nfp, NF = H::NF;
  if (gid >= M.nFaces * nfp) return;
  const int F = gid / nfp, fp = gid % nfp;
  const int4 rec = M.faces[F];
  const int em = rec.x, ep = rec.y;
  const int fm = rec.z & 0xff, fo = (rec.z >> 8) & 0xff, code = (rec.z >> 16) & 0xff;
  S nv[D];
  if (CURV) {
#pragma unroll
    for (int c = 0; c < D; ++c) nv[c] = M.geo.SnF[((size_t)F * D + c) * nfp + fp];
  } else {
#pragma unroll
    for (int c = 0; c < D; ++c) nv[c] = (c == (fm >> 1)) ? ((fm & 1) ? S(1) : S(-1)) : S(0);
  }
  S UL[nf], UR[nf];
  const S* tl = TU + ((size_t)em * NF + fm) * nf * nfp + fp;
#pragma unroll
  for (int f = 0; f < nf; ++f) UL[f] = tl[f * nfp];
  int fpn = 0;
  if (ep >= 0) {
    fpn = orient_map<D, n>(code, fp);
    const S* tr = TU + ((size_t)ep * NF + fo) * nf * nfp + fpn;
#pragma unroll
    for (int f = 0; f < nf; ++f) UR[f] = tr[f * nfp];
  } else {
    mirror_state<D, S>(UL, nv, UR);
  }
  S Fc[nf];
  llf_flux<D, S, !CURV>(UL, UR, nv, M.gas, Fc);
  if (VISC) {
    const S* gl = G + ((size_t)em * NF + fm) * nf * nfp + fp;
    if (ep >= 0) {
      const S* gr = G + ((size_t)ep * NF + fo) * nf * nfp + fpn;
#pragma unroll
      for (int f = 0; f < nf; ++f) Fc[f] -= S(0.5) * (gl[f * nfp] - gr[f * nfp]);
    } else {
#pragma unroll
      for (int f = 0; f < nf; ++f) Fc[f] -= gl[f * nfp];
    }
  }
  S* ol = FF + ((size_t)em * NF + fm) * nf * nfp + fp;
#pragma unroll
  for (int f = 0; f < nf; ++f) ol[f * nfp] = Fc[f];
  if (ep >= 0) {
    S* orr = FF + ((size_t)ep * NF + fo) * nf * nfp + fpn;
#pragma unroll
    for (int f = 0; f < nf; ++f) orr[f * nfp] = -Fc[f];
  }
}

template <int D, int P, typename S, bool VISC, bool CURV>
__global__ void __launch_bounds__(256) k_face(Mesh<S> M, const S* __restrict__ TU, const S* __restrict__ G,
                                              S* __restrict__ FF) {
  face_point<D, P, S, VISC, CURV>(blockIdx.x * blockDim.x + threadIdx.x, M, TU, G, FF);
}

// ---------------------------------------------------------------------------
// Per-node pieces shared by the element kernels (k_elem, k_elem_p, k_elem_tc).
// ---------------------------------------------------------------------------

// ARK stage inputs of one node, read before the flux work so their latency
// overlaps it: pre = base + sum_{j<i} dt a_{i+1,j} k_j, or at the last stage
// pre64 = U_n (FP64 path: + sum_{j<i} dt b_j k_j) and pre = the FP32
// increment sum_{j<i} dt b_j k_j.  base(f), kj(j, f), un(f) fetch the inputs;
// each k_j term is added in the same order (j ascending) for every field.
template <int nf, typename S, typename Base, typename Kj, typename Un>
__device__ __forceinline__ void stage_prefix(const Stage<S>& st, int e, Base base, Kj kj, Un un, S (&pre)[nf],
                                             double (&pre64)[nf]) {
  const S dte = st.dte ? st.dte[e] : S(0);
  // FP32: a fixed trip count (stages beyond i predicated off) puts every k_j
  // load of the node in flight together; FP64 is bound by its arithmetic
  constexpr int JMAX = sizeof(S) == 4 ? MAXSTAGES - 1 : 0;
  if (!st.last) {
#pragma unroll
    for (int f = 0; f < nf; ++f) pre[f] = base(f);
    if (JMAX) {
#pragma unroll
      for (int j = 0; j < JMAX; ++j) {
        if (j < st.i) {
          const S c = st.dte ? dte * st.ca[j] : st.caf[j];
#pragma unroll
          for (int f = 0; f < nf; ++f) pre[f] += c * kj(j, f);
        }
      }
    } else {
      for (int j = 0; j < st.i; ++j) {
        const S c = st.dte ? dte * st.ca[j] : st.caf[j];
#pragma unroll
        for (int f = 0; f < nf; ++f) pre[f] += c * kj(j, f);
      }
    }
  } else {
#pragma unroll
    for (int f = 0; f < nf; ++f) {
      pre64[f] = un(f);
      pre[f] = S(0);
    }
    if (JMAX) {
#pragma unroll
      for (int j = 0; j < JMAX; ++j) {
        if (j < st.i) {
          const S c = st.dte ? dte * st.cb[j] : st.cbf[j];
#pragma unroll
          for (int f = 0; f < nf; ++f) pre[f] += c * kj(j, f);
        }
      }
    } else {
      for (int j = 0; j < st.i; ++j) {
        const S c = st.dte ? dte * st.cb[j] : st.cbf[j];
#pragma unroll
        for (int f = 0; f < nf; ++f) pre64[f] += (double)c * (double)kj(j, f);
      }
    }
  }
}

// Volume flux of one node along each reference direction a:
// Fa[a] = sum_c Ja[a][c] (F^c - F^nu)_c (boxes: Fa[a] = (F^c - F^nu)_a).
// q(c, f) fetches the lifted gradient, ja(a, c) the metric term.
template <int D, typename S, bool VISC, bool CURV, typename Qf, typename Jf>
__device__ __forceinline__ void node_flux(const Gas<S>& gas, const S (&Uq)[D + 2], Qf q, Jf ja, S (&Fa)[D][D + 2]) {
  constexpr int nf = D + 2;
  S F[D][nf];
  conv_flux_all<D, S>(Uq, gas, F);
  if (VISC) {
    S Qv[D][nf], Fv[D][nf];
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int f = 0; f < nf; ++f) Qv[c][f] = q(c, f);
    visc_flux_all<D, S>(Uq, Qv, gas, Fv);
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int f = 0; f < nf; ++f) F[c][f] -= Fv[c][f];
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    if (!CURV) {
#pragma unroll
      for (int f = 0; f < nf; ++f) Fa[a][f] = F[a][f];
    } else {
      S j[D];
#pragma unroll
      for (int c = 0; c < D; ++c) j[c] = ja(a, c);
#pragma unroll
      for (int f = 0; f < nf; ++f) {
        S s = 0;
#pragma unroll
        for (int c = 0; c < D; ++c) s += j[c] * F[c][f];
        Fa[a][f] = s;
      }
    }
  }
}

// ARK stage update of one node (Sec. 4.2): k_i = res; y_{i+1} = pre + dt a_{i+1,i} k_i,
// or at the last stage U_{n+1} = U_n + sum_j dt b_j k_j accumulated in FP64.
// off is the node's offset in the global [E][nf][N] arrays; returns y.
template <int nf, typename S>
__device__ __forceinline__ void stage_update(const Stage<S>& st, int e, size_t off, int N, const S (&res)[nf],
                                             const S (&pre)[nf], const double (&pre64)[nf], S (&y)[nf]) {
  const S dte = st.dte ? st.dte[e] : S(0);
  if (!st.last) {
    const S ci = st.dte ? dte * st.ca[st.i] : st.caf[st.i];
#pragma unroll
    for (int f = 0; f < nf; ++f) {
      const S acc = pre[f] + ci * res[f];
      y[f] = acc;
      st.Kout[off + f * N] = res[f];
      st.Y[off + f * N] = acc;
    }
  } else {
    const S cbi = st.dte ? dte * st.cb[st.i] : st.cbf[st.i];
#pragma unroll
    for (int f = 0; f < nf; ++f) {
      double un = pre64[f];
      if (sizeof(S) == 8) {
        un += (double)cbi * (double)res[f];
      } else {
        const S inc = pre[f] + cbi * res[f];
        un += (double)inc;
      }
      st.Un[off + f * N] = un;
      y[f] = (S)un;
      if (st.shadow) st.shadow[off + f * N] = y[f];
    }
  }
}

// non-finite check of a node's residual (flag bit 0)
template <int nf, typename S>
__device__ __forceinline__ void flag_nonfinite(const S (&res)[nf], unsigned* flags) {
  bool bad = false;
#pragma unroll
  for (int f = 0; f < nf; ++f) bad |= !isfinite(res[f]);
  if (bad) atomicOr(flags, 1u);
}

// ---------------------------------------------------------------------------
// k_elem: f_q = (1/J) [ sum_a sum_m Dh[q_a][m] (F^c - F^nu)~_a(m) - sum_faces L_{q_a}(+-1) Fhat ]
// (boxes: (F^c - F^nu)~_a = F_a with the factor 2/h_a applied per direction).
// MODE 0 writes f; MODE 1 performs the ARK stage update and emits the next
// stage state's traces.
// ---------------------------------------------------------------------------
template <int D, int P, typename S, bool VISC, bool CURV, int MODE, int V>
__device__ __forceinline__ void elem_tile(int tile, unsigned char* smem_raw, const Mesh<S>& M, const S* U,
                                          const S* __restrict__ Q, const S* __restrict__ FF, S* __restrict__ out,
                                          const Stage<S>& st) {
  using H = Sh<D, P, V>;
  constexpr int n = H::n, N = H::N, nf = H::nf, nfp = H::nfp, NF = H::NF, T = H::T;
  constexpr Tab1<S> tb = make_tab1<S>(P);  // compile-time 1D tables
  constexpr int FES = elem_flux_stride<D, P, V>(), SES = elem_state_stride<D, P, V>();
  S* fs = reinterpret_cast<S*>(g_smem<V>(smem_raw, smem_elem_g<D, P, S, V>()));   // [T][D][nf][N] (stride FES), then the next state [T][nf][N] (stride SES)
  S* ffs = fs + T * FES;                     // [T][NF][nf][nfp]
  const int e0 = tile * T;
  const int nel = min(T, M.E - e0);
  stage_faces<D, P, S, V>(ffs, FF + (size_t)e0 * H::FACE, nel);
  const int t = g_tid<V>() / N, q = g_tid<V>() % N;
  const bool active = t < nel;
  const int e = e0 + t;
  // stage-update inputs, read early so their latency overlaps the flux work:
  // pre = base + sum_{j<i} dt a_{i+1,j} k_j (or, at the last stage, the FP64
  // state and sum_{j<i} dt b_j k_j), summed in the same order as before
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
      for (int f = 0; f < nf; ++f) fs[t * FES + (a * nf + f) * N + q] = Fa[a][f];
  }
  g_sync<V>();
  // weak divergence + lift, one thread per line and direction, in place in fs
#pragma unroll
  for (int a = 0; a < D; ++a) {
    for (int i = g_tid<V>(); i < nel * nf * nfp; i += g_size<V>()) {
      int tt, f, line;
      line_item<nf, nfp>(i, tt, f, line);
      S* v = fs + tt * FES + (a * nf + f) * N;
      S x[n];
#pragma unroll
      for (int m = 0; m < n; ++m) x[m] = v[H::node(m, line, a)];
      const S ffm = ffs[((tt * NF + 2 * a) * nf + f) * nfp + line];
      const S ffp = ffs[((tt * NF + 2 * a + 1) * nf + f) * nfp + line];
      const S r = CURV ? S(1) : M.geo.rh[(e0 + tt) * D + a];
#pragma unroll
      for (int k = 0; k < n; ++k) {
        S s = 0;
#pragma unroll
        for (int m = 0; m < n; ++m) s += tb.Dh[k][m] * x[m];
        v[H::node(k, line, a)] = r * (s - tb.Lm[k] * ffm - tb.Lp[k] * ffp);
      }
    }
  }
  g_sync<V>();
  S res[nf];
#pragma unroll
  for (int f = 0; f < nf; ++f) res[f] = S(0);
  if (active) {
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int f = 0; f < nf; ++f) res[f] += fs[t * FES + (a * nf + f) * N + q];
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
  // ---- ARK stage update (Sec. 4.2): k_i = f(y_i); y_{i+1} = base + sum_{j<=i} dt a_{i+1,j} k_j;
  //      last stage: U_{n+1} = U_n + sum_j dt b_j k_j in FP64.
  S y[nf];
  if (active)
    stage_update<nf, S>(st, e, (size_t)e * H::STATE + q, N, res, pre, pre64, y);
  g_sync<V>();  // everyone is done with fs
  if (active) {
#pragma unroll
    for (int f = 0; f < nf; ++f) fs[t * SES + f * N + q] = y[f];
  }
  g_sync<V>();
  tile_traces<D, P, S, V, SES>(fs, nel, st.TU + (size_t)e0 * H::FACE);
}

template <int D, int P, typename S, bool VISC, bool CURV, int MODE, int V>
__global__ void __launch_bounds__(Sh<D, P, V>::THREADS) k_elem(Mesh<S> M, const S* U,
                                                               const S* __restrict__ Q, const S* __restrict__ FF,
                                                               S* __restrict__ out, Stage<S> st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  elem_tile<D, P, S, VISC, CURV, MODE, V>(g_index<V>(), smem_raw, M, U, Q, FF, out, st);
}

}  // namespace dgx
