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

#include "physics.cuh"

namespace dgx {

constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

// Tile variants (chosen per kernel by the autotuner): about 128, 256 or 512
// threads per CTA, i.e. T = max(1, 64 * 2^(V+1) / N) elements per tile.
constexpr int NVARIANTS = 3;
constexpr int variant_threads(int V) { return 64 << (V + 1); }

template <int D, int P, int V = 1>
struct Sh {
  static constexpr int n = P + 1;
  static constexpr int N = ipow(n, D);
  static constexpr int nf = D + 2;
  static constexpr int nfp = ipow(n, D - 1);
  static constexpr int NF = 2 * D;
  static constexpr int T = (variant_threads(V) / N) > 0 ? (variant_threads(V) / N) : 1;
  static constexpr int THREADS = ((T * N + 31) / 32) * 32;
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
  unsigned* flags;     // bit 0: non-finite residual
};

constexpr int MAXSTAGES = 8;

template <typename S>
struct Stage {
  const S* k[MAXSTAGES];   // k_0 .. k_{i-1}
  double ca[MAXSTAGES];    // a_{i+1, j}, j <= i
  double cb[MAXSTAGES];    // b_j (last stage)
  double dt;               // time step, unless dte is given
  const double* dte;       // per-element time step (batched instances) or nullptr
  int i;                   // this stage (0-based)
  int last;
  const S* base;           // y = base + sum ca_j k_j (FP64: U_n itself, FP32: fl32(U_n))
  double* Un;              // FP64 master state (updated at the last stage)
  S* Y;                    // next stage state (may alias the stage input)
  S* Kout;                 // k_i
  S* shadow;               // FP32 only: fl32(U_{n+1}) written at the last stage
  S* TU;                   // traces of the next stage state
};

template <typename S>
__device__ __forceinline__ void load_tab(const Tab<S>* tabs, int P, S* sD, S* sDh, S* slm, S* slp, S* sLm, S* sLp,
                                         int n) {
  const Tab<S>& t = tabs[P];
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    const int r = i / n, c = i % n;
    if (sD) sD[i] = t.D[r * 6 + c];
    if (sDh) sDh[i] = t.Dh[r * 6 + c];
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (slm) slm[i] = t.lm[i];
    if (slp) slp[i] = t.lp[i];
    if (sLm) sLm[i] = t.Lm[i];
    if (sLp) sLp[i] = t.Lp[i];
  }
}

// Traces of a staged tile (us[t][f][q]) written in output order (coalesced).
template <int D, int P, typename S, int V>
__device__ __forceinline__ void tile_traces(const S* us, const S* lm, const S* lp, int nel, S* dst) {
  using H = Sh<D, P, V>;
  const int tot = nel * H::FACE;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    const int fp = i % H::nfp;
    int r = i / H::nfp;
    const int f = r % H::nf;
    r /= H::nf;
    const int face = r % H::NF;
    const int t = r / H::NF;
    const int a = face >> 1;
    const S* l = (face & 1) ? lp : lm;
    const S* v = us + (t * H::nf + f) * H::N;
    S acc = 0;
#pragma unroll
    for (int m = 0; m < H::n; ++m) acc += l[m] * v[H::node(m, fp, a)];
    dst[i] = acc;
  }
}

// ---------------------------------------------------------------------------
// k_trace: TU = traces of U (input may be double while S is float: the FP32
// ARK path converts the FP64 master state here and keeps the rounded copy).
// ---------------------------------------------------------------------------
template <int D, int P, typename S, typename Sin, int V>
__global__ void __launch_bounds__(Sh<D, P, V>::THREADS) k_trace(int E, const Sin* __restrict__ U,
                                                                S* __restrict__ TU, S* __restrict__ shadow,
                                                                const Tab<S>* tabs) {
  using H = Sh<D, P, V>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S* us = reinterpret_cast<S*>(smem_raw);
  S* lm = us + H::T * H::STATE;
  S* lp = lm + H::n;
  const int e0 = blockIdx.x * H::T;
  const int nel = min(H::T, E - e0);
  const Sin* src = U + (size_t)e0 * H::STATE;
  S* sh = shadow ? shadow + (size_t)e0 * H::STATE : nullptr;
  for (int i = threadIdx.x; i < nel * H::STATE; i += blockDim.x) {
    const S v = (S)src[i];
    us[i] = v;
    if (sh) sh[i] = v;
  }
  load_tab<S>(tabs, P, nullptr, nullptr, lm, lp, nullptr, nullptr, H::n);
  __syncthreads();
  tile_traces<D, P, S, V>(us, lm, lp, nel, TU + (size_t)e0 * H::FACE);
}

// ---------------------------------------------------------------------------
// k_br1: BR1 lifted gradient (conservative variables)
//   Q_c(q) = (1/J) sum_b Ja[b][c] (D_b U)(q) + sum_faces l_{q_a}(+-1)/(w_{q_a} J) (Uhat - U^-) Sn_c
// Uhat = (U^- + U^+)/2 inside, U_w on walls.  Writes Q and each own face's
// viscous normal flux G = F^nu(U_f, Q_f) . n (wall: adiabatic wall flux).
// Boxes use unit normals (the element kernel applies 2/h_a).
// ---------------------------------------------------------------------------
template <int D, int P, typename S, bool CURV, int V>
__global__ void __launch_bounds__(Sh<D, P, V>::THREADS) k_br1(Mesh<S> M, const S* __restrict__ U,
                                                              const S* __restrict__ TU, S* __restrict__ Q,
                                                              S* __restrict__ G) {
  using H = Sh<D, P, V>;
  constexpr int n = H::n, N = H::N, nf = H::nf, nfp = H::nfp, NF = H::NF, T = H::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S* us = reinterpret_cast<S*>(smem_raw);     // [T][nf][N]
  S* js = us + T * H::STATE;                   // [T][NF][nf][nfp]
  S* qs = js + T * H::FACE;                    // [T][D][nf][N]
  S* sD = qs + T * D * H::STATE;
  S* lm = sD + n * n;
  S* lp = lm + n;
  S* Lm = lp + n;
  S* Lp = Lm + n;
  const int e0 = blockIdx.x * T;
  const int nel = min(T, M.E - e0);
  {
    const S* src = U + (size_t)e0 * H::STATE;
    for (int i = threadIdx.x; i < nel * H::STATE; i += blockDim.x) us[i] = src[i];
  }
  load_tab<S>(M.tabs, P, sD, nullptr, lm, lp, Lm, Lp, n);
  // jumps Uhat - U^- at every own face point
  for (int i = threadIdx.x; i < nel * NF * nfp; i += blockDim.x) {
    const int fp = i % nfp;
    const int face = (i / nfp) % NF;
    const int t = i / (nfp * NF);
    const int e = e0 + t;
    const S* tl = TU + ((size_t)e * NF + face) * nf * nfp + fp;
    S UL[nf];
#pragma unroll
    for (int f = 0; f < nf; ++f) UL[f] = tl[f * nfp];
    const int nbe = M.nb[e * NF + face];
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
  }
  __syncthreads();
  const int t = threadIdx.x / N, q = threadIdx.x % N;
  if (t < nel) {
    const int e = e0 + t;
    S dU[D][nf];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int fp = H::fpoint(q, a), qa = H::qa(q, a);
#pragma unroll
      for (int f = 0; f < nf; ++f) {
        const S* v = us + (t * nf + f) * N;
        S s = 0;
#pragma unroll
        for (int m = 0; m < n; ++m) s += sD[qa * n + m] * v[H::node(m, fp, a)];
        dU[a][f] = s;
      }
    }
    S Qv[D][nf];
    if (!CURV) {
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const S r = M.geo.rh[e * D + c];
        const int fp = H::fpoint(q, c), qc = H::qa(q, c);
        const S* jm = js + (t * NF + 2 * c) * nf * nfp + fp;
        const S* jp = js + (t * NF + 2 * c + 1) * nf * nfp + fp;
#pragma unroll
        for (int f = 0; f < nf; ++f) Qv[c][f] = r * (dU[c][f] + Lp[qc] * jp[f * nfp] - Lm[qc] * jm[f * nfp]);
      }
    } else {
      const S iJ = M.geo.iJ[(size_t)e * N + q];
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int f = 0; f < nf; ++f) {
          S s = 0;
#pragma unroll
          for (int b = 0; b < D; ++b) s += M.geo.Ja[(((size_t)e * D + b) * D + c) * N + q] * dU[b][f];
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
    S* qd = Q + (size_t)e * D * H::STATE + q;
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int f = 0; f < nf; ++f) {
        qs[((t * D + c) * nf + f) * N + q] = Qv[c][f];
        qd[(c * nf + f) * N] = Qv[c][f];
      }
  }
  __syncthreads();
  // own-face viscous fluxes
  for (int i = threadIdx.x; i < nel * NF * nfp; i += blockDim.x) {
    const int fp = i % nfp;
    const int face = (i / nfp) % NF;
    const int tt = i / (nfp * NF);
    const int e = e0 + tt;
    const int a = face >> 1;
    const S* l = (face & 1) ? lp : lm;
    S UL[nf], TQ[D][nf], nv[D];
    const S* tl = TU + ((size_t)e * NF + face) * nf * nfp + fp;
#pragma unroll
    for (int f = 0; f < nf; ++f) UL[f] = tl[f * nfp];
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int f = 0; f < nf; ++f) {
        const S* v = qs + ((tt * D + c) * nf + f) * N;
        S s = 0;
#pragma unroll
        for (int m = 0; m < n; ++m) s += l[m] * v[H::node(m, fp, a)];
        TQ[c][f] = s;
      }
    if (CURV) {
#pragma unroll
      for (int c = 0; c < D; ++c) nv[c] = M.geo.SnE[(((size_t)e * NF + face) * D + c) * nfp + fp];
    } else {
#pragma unroll
      for (int c = 0; c < D; ++c) nv[c] = (c == a) ? ((face & 1) ? S(1) : S(-1)) : S(0);
    }
    S Gv[nf];
    if (M.nb[e * NF + face] >= 0)
      visc_flux_normal<D, S>(UL, TQ, nv, M.gas, Gv);
    else
      wall_visc_flux<D, S>(UL, TQ, nv, M.gas, Gv);
    S* gd = G + ((size_t)e * NF + face) * nf * nfp + fp;
#pragma unroll
    for (int f = 0; f < nf; ++f) gd[f * nfp] = Gv[f];
  }
}

// ---------------------------------------------------------------------------
// k_face: one thread per unique face point.  Fhat = LLF(U^-, U^+; n) - Fhat^nu,
// Fhat^nu = (G^- - G^+)/2 inside, G^- on walls; written as +Fhat to the owner
// side and -Fhat to the other side.  Boxes: unit normals; curvilinear: the
// averaged area normal of the face.
// ---------------------------------------------------------------------------
template <int D, int P, typename S, bool VISC, bool CURV>
__global__ void __launch_bounds__(256) k_face(Mesh<S> M, const S* __restrict__ TU, const S* __restrict__ G,
                                              S* __restrict__ FF) {
  using H = Sh<D, P>;
  constexpr int n = H::n, nf = H::nf, nfp = H::nfp, NF = H::NF;
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
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

// ---------------------------------------------------------------------------
// k_elem: f_q = (1/J) [ sum_a sum_m Dh[q_a][m] (F^c - F^nu)~_a(m) - sum_faces L_{q_a}(+-1) Fhat ]
// (boxes: (F^c - F^nu)~_a = F_a with the factor 2/h_a applied per direction).
// MODE 0 writes f; MODE 1 performs the ARK stage update and emits the next
// stage state's traces.
// ---------------------------------------------------------------------------
template <int D, int P, typename S, bool VISC, bool CURV, int MODE, int V>
__global__ void __launch_bounds__(Sh<D, P, V>::THREADS) k_elem(Mesh<S> M, const S* U,
                                                               const S* __restrict__ Q, const S* __restrict__ FF,
                                                               S* __restrict__ out, Stage<S> st) {
  using H = Sh<D, P, V>;
  constexpr int n = H::n, N = H::N, nf = H::nf, nfp = H::nfp, NF = H::NF, T = H::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S* fs = reinterpret_cast<S*>(smem_raw);   // [T][D][nf][N]  (reused for the next state's traces)
  S* ffs = fs + T * D * H::STATE;            // [T][NF][nf][nfp]
  S* sDh = ffs + T * H::FACE;
  S* lm = sDh + n * n;
  S* lp = lm + n;
  S* Lm = lp + n;
  S* Lp = Lm + n;
  const int e0 = blockIdx.x * T;
  const int nel = min(T, M.E - e0);
  {
    const S* src = FF + (size_t)e0 * H::FACE;
    for (int i = threadIdx.x; i < nel * H::FACE; i += blockDim.x) ffs[i] = src[i];
  }
  load_tab<S>(M.tabs, P, nullptr, sDh, lm, lp, Lm, Lp, n);
  const int t = threadIdx.x / N, q = threadIdx.x % N;
  const bool active = t < nel;
  const int e = e0 + t;
  S Uq[nf];
  if (active) {
    const S* up = U + (size_t)e * H::STATE + q;
#pragma unroll
    for (int f = 0; f < nf; ++f) Uq[f] = up[f * N];
    S F[D][nf];
    conv_flux_all<D, S>(Uq, M.gas, F);
    if (VISC) {
      S Qv[D][nf], Fv[D][nf];
      const S* qp = Q + (size_t)e * D * H::STATE + q;
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int f = 0; f < nf; ++f) Qv[c][f] = qp[(c * nf + f) * N];
      visc_flux_all<D, S>(Uq, Qv, M.gas, Fv);
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int f = 0; f < nf; ++f) F[c][f] -= Fv[c][f];
    }
    if (!CURV) {
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int f = 0; f < nf; ++f) fs[((t * D + a) * nf + f) * N + q] = F[a][f];
    } else {
#pragma unroll
      for (int a = 0; a < D; ++a) {
        S ja[D];
#pragma unroll
        for (int c = 0; c < D; ++c) ja[c] = M.geo.Ja[(((size_t)e * D + a) * D + c) * N + q];
#pragma unroll
        for (int f = 0; f < nf; ++f) {
          S s = 0;
#pragma unroll
          for (int c = 0; c < D; ++c) s += ja[c] * F[c][f];
          fs[((t * D + a) * nf + f) * N + q] = s;
        }
      }
    }
  }
  __syncthreads();
  S res[nf];
#pragma unroll
  for (int f = 0; f < nf; ++f) res[f] = S(0);
  if (active) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int fp = H::fpoint(q, a), qa = H::qa(q, a);
      const S cm = Lm[qa], cp = Lp[qa];
      const S r = CURV ? S(1) : M.geo.rh[e * D + a];
#pragma unroll
      for (int f = 0; f < nf; ++f) {
        const S* v = fs + ((t * D + a) * nf + f) * N;
        S s = 0;
#pragma unroll
        for (int m = 0; m < n; ++m) s += sDh[qa * n + m] * v[H::node(m, fp, a)];
        s -= cm * ffs[((t * NF + 2 * a) * nf + f) * nfp + fp];
        s -= cp * ffs[((t * NF + 2 * a + 1) * nf + f) * nfp + fp];
        res[f] += r * s;
      }
    }
    if (CURV) {
      const S iJ = M.geo.iJ[(size_t)e * N + q];
#pragma unroll
      for (int f = 0; f < nf; ++f) res[f] *= iJ;
    }
    bool bad = false;
#pragma unroll
    for (int f = 0; f < nf; ++f) bad |= !isfinite(res[f]);
    if (bad) atomicOr(M.flags, 1u);
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
  if (active) {
    const size_t off = (size_t)e * H::STATE + q;
    const double dt = st.dte ? st.dte[e] : st.dt;
    if (!st.last) {
      S ca[MAXSTAGES];
      for (int j = 0; j <= st.i; ++j) ca[j] = (S)(dt * st.ca[j]);
#pragma unroll
      for (int f = 0; f < nf; ++f) {
        S acc = st.base[off + f * N];
        for (int j = 0; j < st.i; ++j) acc += ca[j] * st.k[j][off + f * N];
        acc += ca[st.i] * res[f];
        y[f] = acc;
        st.Kout[off + f * N] = res[f];
        st.Y[off + f * N] = acc;
      }
    } else {
#pragma unroll
      for (int f = 0; f < nf; ++f) {
        double un = st.Un[off + f * N];
        if (sizeof(S) == 8) {
          for (int j = 0; j < st.i; ++j) un += (dt * st.cb[j]) * (double)st.k[j][off + f * N];
          un += (dt * st.cb[st.i]) * (double)res[f];
        } else {
          S inc = S(0);
          for (int j = 0; j < st.i; ++j) inc += (S)(dt * st.cb[j]) * st.k[j][off + f * N];
          inc += (S)(dt * st.cb[st.i]) * res[f];
          un += (double)inc;
        }
        st.Un[off + f * N] = un;
        y[f] = (S)un;
        if (st.shadow) st.shadow[off + f * N] = y[f];
      }
    }
  }
  __syncthreads();  // everyone is done with fs
  if (active) {
#pragma unroll
    for (int f = 0; f < nf; ++f) fs[(t * nf + f) * N + q] = y[f];
  }
  __syncthreads();
  tile_traces<D, P, S, V>(fs, lm, lp, nel, st.TU + (size_t)e0 * H::FACE);
}

}  // namespace dgx
