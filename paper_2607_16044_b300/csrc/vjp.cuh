// Adjoint (vector-Jacobian product) kernels of the explicit DG residual.
//
// g = (df/dU)^T lambda, obtained by running the forward pipeline of
// kernels.cuh backwards (each step's transpose, derived by hand):
//   k_vjp_elem    lambda -> Fhat_bar (transposed lift), U_bar (transposed
//                 weak-divergence contraction and flux Jacobians^T), Q_bar
//   k_vjp_face    per unique face point: LLF (and mirror-state) adjoint, written
//                 to both sides' trace cotangents
//   k_vjp_br1     (NS) viscous face-flux adjoint (its cotangent formed from both
//                 sides' Fhat_bar), transposed Q traces, transposed
//                 derivative contraction and BR1 lift adjoint; the neighbour's
//                 share of each jump cotangent goes to a per-face buffer
//   k_vjp_gather  transposed traces: g += sum_faces l(+-1) TU_bar (+ neighbours'
//                 jump shares)
// Every output location is written by exactly one thread (no atomics): face
// quantities are per element and face, and the unique-face kernel writes both
// sides of its face.
//
// For the ARK adjoint (reverse stage recurrence) the element kernel can form
// its cotangent as  mu = c_lam * lam + sum_j c_j nu_j  on the fly, and the
// gather kernel can finish lam_n = lam + sum_j nu_j in FP64.
#pragma once
#include "ops.cuh"

namespace dgx {

struct VjpWork {
  void* TU;   // forward traces                  [E][2D][nf][nfp]
  void* FFb;  // lift cotangent (Fhat_bar)        [E][2D][nf][nfp]
  void* G;    // forward viscous face flux (unused by the adjoint, written by k_br1)
  void* Q;    // forward BR1 gradient            [E][D][nf][N]
  void* TUb;  // trace cotangents                 [E][2D][nf][nfp]
  void* JB;   // BR1 jump cotangents, stored in the layout of the element that receives them:
              // [E][2D][nf][nfp] at (e, face, fp) holds the cotangent of the jump seen by the
              // neighbour across that face (zero on walls)
  void* Qb;   // gradient cotangents              [E][D][nf][N]
  void* TQ;   // forward traces of Q [E][2D][D][nf][nfp] when the forward stored them (else nullptr:
              // k_vjp_br1 traces Q itself)
};

// Element strides (in scalars) of k_vjp_elem's [T][nf][N] cotangent tile and
// [T][D][nf][N] flux-cotangent tile, padded so that the line passes and node
// phases of neighbouring elements fall in different banks (pads minimise the
// mean wavefronts per warp access over both phases for each CTA tile shape,
// found by enumerating the 32 x 32 residue pairs; one element per tile needs none).
template <int D, int P, int V>
constexpr int vjp_mu_stride() {
  constexpr int p2[6] = {0, 1, 0, 5, 0, 1}, p3[6] = {0, 0, 20, 5, 0, 0};
  const int pad = V > 2 ? 0 : D == 2 ? (P == 2 ? (V == 0 ? 1 : V == 1 ? 17 : 7) : p2[P]) : p3[P];
  return Sh<D, P, V>::STATE + pad;
}
template <int D, int P, int V>
constexpr int vjp_fb_stride() {
  constexpr int p2[6] = {0, 3, 0, 5, 17, 15}, p3[6] = {0, 16, 6, 5, 10, 16};
  const int pad = V > 2 ? 0 : D == 2 ? (P == 2 ? (V == 1 ? 13 : 3) : p2[P]) : p3[P];
  return D * Sh<D, P, V>::STATE + pad;
}
template <int D, int P, typename S, int V>
constexpr size_t smem_velem_g() {
  using h = Sh<D, P, V>;
  return r16(sizeof(S) * (h::T * (vjp_mu_stride<D, P, V>() + vjp_fb_stride<D, P, V>()) + 2 * h::n));
}
// k_vjp_br1's shared memory per element group: the Q_bar staging tile only on
// curvilinear meshes (boxes read each Q_bar line straight from global memory)
template <int D, int P, typename S, int V, bool CURV = true>
constexpr size_t smem_vbr1_g() {
  using h = Sh<D, P, V>;
  return r16(sizeof(S) * ((CURV ? 2 : 1) * h::T * D * h::STATE + 2 * h::T * h::NF * D * h::nf * h::nfp +
                          h::T * h::FACE + 2 * h::n));
}
template <int D, int P, typename S, int V>
constexpr size_t smem_vgather_g() {
  using h = Sh<D, P, V>;
  return r16(sizeof(S) * (h::T * h::FACE + 2 * h::n));
}

// Cotangent source of the element kernel: mu = c_lam * lam + sum_j c_j nu_j.
template <typename S>
struct Cot {
  const S* lam;        // cotangent in the handle's precision (plain VJP; FP32 ARK adjoint after
                       // its first reverse stage: the FP32 copy of lambda_{n+1}), or nullptr
  const double* lam64; // ARK adjoint: lambda_{n+1} (double), or nullptr
  S* lam_out;          // FP32 ARK adjoint, first reverse stage: S(lambda_{n+1}) is written here
  S c_lam;             // coefficients rounded to S on the host (FP32 kernels do no FP64 math
  const S* nu[MAXSTAGES];  // in the combination: FP64 is ~1/64 of the FP32 rate here)
  S c_nu[MAXSTAGES];
  int n_nu;
  // ARK adjoint finish (gather kernel of the last reverse stage):
  // lam64_out = lam64 + g + sum_j nu_j
  double* lam64_out;
  const S* nu_all[MAXSTAGES];
  int n_all;
  // ARK adjoint, fused gather (k_vjp_elem<GATHER>): nu_prev = the previous reverse
  // stage's partial nu (volume part, finished here with its trace cotangents and
  // written back), entering mu with coefficient c_prev
  S* nu_prev;
  S c_prev;
};

// ---------------------------------------------------------------------------
// GATHER (ARK adjoint, every reverse stage but the first): the kernel first
// finishes the previous reverse stage's nu (the gather of k_vjp_gather, from
// TUb and JB of that stage, which are still in the workspace) and uses it
// directly in this stage's mu.
template <int D, int P, typename S, bool VISC, bool CURV, int V, bool GATHER>
__global__ void __launch_bounds__(Sh<D, P, V>::THREADS) k_vjp_elem(Mesh<S> M, const S* __restrict__ U,
                                                                   const S* __restrict__ Q, Cot<S> cot,
                                                                   S* __restrict__ FFb, S* __restrict__ Ub,
                                                                   S* __restrict__ Qb, const S* __restrict__ TUbp,
                                                                   const S* __restrict__ JBp) {
  using H = Sh<D, P, V>;
  constexpr int n = H::n, N = H::N, nf = H::nf, nfp = H::nfp, NF = H::NF, T = H::T;
  constexpr Tab1<S> tb = make_tab1<S>(P);  // compile-time 1D tables
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int MS = vjp_mu_stride<D, P, V>(), FBS = vjp_fb_stride<D, P, V>();
  S* mus = reinterpret_cast<S*>(g_smem<V>(smem_raw, smem_velem_g<D, P, S, V>()));  // [T][nf][N] (stride MS)  cotangent / J
  S* fb = mus + T * MS;                      // [T][D][nf][N] (stride FBS)  contravariant flux cotangents
  S* tubs = fb;                              // GATHER: [T][NF][nf][nfp] trace cotangents (before fb is written)
  S* lms = fb + T * FBS;                     // node-indexed trace weights (GATHER)
  S* lps = lms + n;
  const int e0 = g_index<V>() * T;
  const int nel = min(T, M.E - e0);
  // per-node inputs of the pointwise adjoint, read first (latency overlaps the contractions)
  const int tn = g_tid<V>() / N, qn = g_tid<V>() % N;
  S Uq[nf], Qv[VISC ? D : 1][nf];
  if (tn < nel) {
    const S* up = U + (size_t)(e0 + tn) * H::STATE + qn;
#pragma unroll
    for (int f = 0; f < nf; ++f) Uq[f] = up[f * N];
    if (VISC) {
      const S* qp = Q + (size_t)(e0 + tn) * D * H::STATE + qn;
#pragma unroll
      for (int c = 0; c < (VISC ? D : 1); ++c)
#pragma unroll
        for (int f = 0; f < nf; ++f) Qv[c][f] = qp[(c * nf + f) * N];
    }
  }
  // mu = c_lam lambda + sum_j c_j nu_j at this node, every field's loads issued
  // together and ahead of the gather phase, whose latency they overlap
  S s[nf];
#pragma unroll
  for (int f = 0; f < nf; ++f) s[f] = S(0);
  if (tn < nel) {
    const size_t off = (size_t)(e0 + tn) * H::STATE + qn;
    if (cot.lam) {
#pragma unroll
      for (int f = 0; f < nf; ++f) s[f] = cot.lam[off + f * N];
    } else if (cot.lam64 && (cot.c_lam != S(0) || cot.lam_out)) {
#pragma unroll
      for (int f = 0; f < nf; ++f) s[f] = (S)cot.lam64[off + f * N];
      if (cot.lam_out) {
#pragma unroll
        for (int f = 0; f < nf; ++f) cot.lam_out[off + f * N] = s[f];
      }
    }
#pragma unroll
    for (int f = 0; f < nf; ++f) s[f] *= cot.c_lam;
    if (sizeof(S) == 4) {  // FP32: fixed trip count, every nu load of the node in flight together
#pragma unroll
      for (int j = 0; j < MAXSTAGES - 1; ++j) {
        if (j < cot.n_nu) {
          const S c = cot.c_nu[j];
          const S* nu = cot.nu[j] + off;
#pragma unroll
          for (int f = 0; f < nf; ++f) s[f] += c * nu[f * N];
        }
      }
    } else {  // FP64: bound by its arithmetic, the plain loop
      for (int j = 0; j < cot.n_nu; ++j) {
        const S c = cot.c_nu[j];
        const S* nu = cot.nu[j] + off;
#pragma unroll
        for (int f = 0; f < nf; ++f) s[f] += c * nu[f * N];
      }
    }
  }
  S nuq[nf];  // GATHER: the finished nu of the previous reverse stage at this node
  if (GATHER) {
    const size_t off = (size_t)(e0 + tn) * H::STATE + qn;
    if (tn < nel) {
#pragma unroll
      for (int f = 0; f < nf; ++f) nuq[f] = cot.nu_prev[off + f * N];
    }
    load_tab<S, V>(M.tabs, P, lms, lps, nullptr, nullptr, n);
    // own trace cotangent plus half the jump cotangent the neighbour scattered here
    const S* tsrc = TUbp + (size_t)e0 * H::FACE;
    const S* jsrc = JBp + (size_t)e0 * H::FACE;
    for (int i = g_tid<V>(); i < nel * NF * nfp; i += g_size<V>()) {
      const int fp = i % nfp, tf = i / nfp;  // tf = t * NF + face
      S a[nf], c[nf];
#pragma unroll
      for (int f = 0; f < nf; ++f) {
        a[f] = tsrc[(tf * nf + f) * nfp + fp];
        c[f] = VISC ? jsrc[(tf * nf + f) * nfp + fp] : S(0);
      }
#pragma unroll
      for (int f = 0; f < nf; ++f) tubs[(tf * nf + f) * nfp + fp] = a[f] + S(0.5) * c[f];
    }
    g_sync<V>();
    if (tn < nel) {
      S lmq[D], lpq[D];
      int fpq[D];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int qa = H::qa(qn, a);
        lmq[a] = lms[qa];
        lpq[a] = lps[qa];
        fpq[a] = H::fpoint(qn, a);
      }
#pragma unroll
      for (int f = 0; f < nf; ++f) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
          nuq[f] += lmq[a] * tubs[((tn * NF + 2 * a) * nf + f) * nfp + fpq[a]];
          nuq[f] += lpq[a] * tubs[((tn * NF + 2 * a + 1) * nf + f) * nfp + fpq[a]];
        }
        cot.nu_prev[off + f * N] = nuq[f];
      }
    }
  }
  if (tn < nel) {
    if (GATHER) {
#pragma unroll
      for (int f = 0; f < nf; ++f) s[f] += cot.c_prev * nuq[f];
    }
    const S ij = CURV ? M.geo.iJ[(size_t)(e0 + tn) * N + qn] : S(1);
#pragma unroll
    for (int f = 0; f < nf; ++f) mus[tn * MS + f * N + qn] = CURV ? s[f] * ij : s[f];
  }
  g_sync<V>();
  // one thread per line and direction: transposed weak divergence
  //   Ft_bar_a(m) = rr_a sum_k Dh[k][m] mu(k)   -> fb
  // and transposed lift  Fhat_bar(a, side) = -rr_a sum_k L_side[k] mu(k) -> FFb
#pragma unroll
  for (int a = 0; a < D; ++a) {
    for (int i = g_tid<V>(); i < nel * nf * nfp; i += g_size<V>()) {
      int tt, f, line;
      line_item<nf, nfp>(i, tt, f, line);
      const S* v = mus + tt * MS + f * N;
      S x[n];
#pragma unroll
      for (int k = 0; k < n; ++k) x[k] = v[H::node(k, line, a)];
      const S rr = CURV ? S(1) : M.geo.rh[(e0 + tt) * D + a];
      S* fo = fb + tt * FBS + (a * nf + f) * N;
      S sm = 0, sp = 0;
#pragma unroll
      for (int m = 0; m < n; ++m) {
        S acc = 0;
#pragma unroll
        for (int k = 0; k < n; ++k) acc += tb.Dh[k][m] * x[k];
        fo[H::node(m, line, a)] = rr * acc;
        sm += tb.Lm[m] * x[m];
        sp += tb.Lp[m] * x[m];
      }
      S* dst = FFb + (size_t)(e0 + tt) * H::FACE + f * nfp + line;
      dst[(2 * a) * nf * nfp] = -rr * sm;
      dst[(2 * a + 1) * nf * nfp] = -rr * sp;
    }
  }
  g_sync<V>();
  const int t = g_tid<V>() / N, q = g_tid<V>() % N;
  if (t >= nel) return;
  const int e = e0 + t;
  S Fb[D][nf];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int f = 0; f < nf; ++f) Fb[a][f] = fb[t * FBS + (a * nf + f) * N + q];
  if (CURV) {  // physical flux cotangent F_bar_c = sum_a Ja[a][c] Ft_bar_a
    S Fc[D][nf];
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int f = 0; f < nf; ++f) Fc[c][f] = S(0);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const S ja = M.geo.Ja[(((size_t)e * D + a) * D + c) * N + q];
#pragma unroll
        for (int f = 0; f < nf; ++f) Fc[c][f] += ja * Fb[a][f];
      }
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int f = 0; f < nf; ++f) Fb[c][f] = Fc[c][f];
  }
  S Ubq[nf];
#pragma unroll
  for (int f = 0; f < nf; ++f) Ubq[f] = S(0);
  conv_flux_all_vjp<D, S>(Uq, Fb, M.gas, Ubq);
  if (VISC) {  // F = F^c - F^nu
    S Qbv[D][nf], Fm[D][nf], Qd[D][nf];
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int f = 0; f < nf; ++f) {
        Qd[c][f] = Qv[VISC ? c : 0][f];
        Qbv[c][f] = S(0);
        Fm[c][f] = -Fb[c][f];
      }
    visc_flux_all_vjp<D, S>(Uq, Qd, Fm, M.gas, Ubq, Qbv);
    S* qb = Qb + (size_t)e * D * H::STATE + q;
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int f = 0; f < nf; ++f) qb[(c * nf + f) * N] = Qbv[c][f];
  }
  S* ub = Ub + (size_t)e * H::STATE + q;
#pragma unroll
  for (int f = 0; f < nf; ++f) ub[f * N] = Ubq[f];
}

// ---------------------------------------------------------------------------
template <int D, int P, typename S, bool CURV>
__global__ void __launch_bounds__(256, sizeof(S) == 8 ? 2 : 6) k_vjp_face(Mesh<S> M, const S* __restrict__ TU, const S* __restrict__ FFb,
                                                  S* __restrict__ TUb) {
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
  const size_t oL = ((size_t)em * NF + fm) * nf * nfp + fp;
  S UL[nf], UR[nf], sig[nf];
#pragma unroll
  for (int f = 0; f < nf; ++f) {
    UL[f] = TU[oL + f * nfp];
    sig[f] = FFb[oL + f * nfp];
  }
  int fpn = 0;
  size_t oR = 0;
  if (ep >= 0) {
    fpn = orient_map<D, n>(code, fp);
    oR = ((size_t)ep * NF + fo) * nf * nfp + fpn;
#pragma unroll
    for (int f = 0; f < nf; ++f) {
      UR[f] = TU[oR + f * nfp];
      sig[f] -= FFb[oR + f * nfp];
    }
  } else {
    mirror_state<D, S>(UL, nv, UR);
  }
  S ULb[nf], URb[nf];
#pragma unroll
  for (int f = 0; f < nf; ++f) ULb[f] = URb[f] = S(0);
  llf_flux_vjp<D, S, !CURV>(UL, UR, nv, sig, M.gas, ULb, URb);
  if (ep >= 0) {
#pragma unroll
    for (int f = 0; f < nf; ++f) {
      TUb[oL + f * nfp] = ULb[f];
      TUb[oR + f * nfp] = URb[f];
    }
  } else {
    mirror_state_vjp<D, S>(nv, URb, ULb);
#pragma unroll
    for (int f = 0; f < nf; ++f) TUb[oL + f * nfp] = ULb[f];
  }
}

// ---------------------------------------------------------------------------
template <int D, int P, typename S, bool CURV, int V>
__global__ void __launch_bounds__(Sh<D, P, V>::THREADS) k_vjp_br1(Mesh<S> M, const S* __restrict__ TU,
                                                                  const S* __restrict__ Q, const S* __restrict__ FFb,
                                                                  S* __restrict__ Qb, S* __restrict__ TUb,
                                                                  S* __restrict__ JB, S* __restrict__ Ub,
                                                                  const S* __restrict__ TQg) {
  using H = Sh<D, P, V>;
  constexpr int n = H::n, N = H::N, nf = H::nf, nfp = H::nfp, NF = H::NF, T = H::T;
  constexpr Tab1<S> tb = make_tab1<S>(P);  // compile-time 1D tables
  constexpr int TQS = NF * D * nf * nfp;      // traces of Q per element
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S* qs = reinterpret_cast<S*>(g_smem<V>(smem_raw, smem_vbr1_g<D, P, S, V, CURV>()));  // [T][D][nf][N]  dU_bar and D^T dU_bar
  S* qbs = qs + T * D * H::STATE;            // [T][D][nf][N]  Q_bar (total), later P (curvilinear only)
  S* tq = CURV ? qbs + T * D * H::STATE : qbs;  // [T][NF][D][nf][nfp] traces of Q, later J_bar [T][NF][nf][nfp]
  S* tqb = tq + T * TQS;                     // [T][NF][D][nf][nfp] TQ_bar
  S* tub = tqb + T * TQS;                    // [T][NF][nf][nfp] own TU_bar
  S* lm = tub + T * H::FACE;                 // node-indexed trace weights
  S* lp = lm + n;
  S* js = tq;
  const int e0 = g_index<V>() * T;
  const int nel = min(T, M.E - e0);
  load_tab<S, V>(M.tabs, P, lm, lp, nullptr, nullptr, n);  // node-indexed traces
  // Cotangent of the own viscous face flux G at a face point.  The face flux
  // is Fhat = LLF - (G_own - G_nb) / 2 (wall: LLF - G_own), so with the lift
  // cotangents of both sides G_own_bar = -(FFb_own - FFb_nb) / 2 (wall: -FFb_own).
  auto g_bar = [&](const S (&own)[nf], int nbe, int nbf, int ori, int fp, S (&gb)[nf]) {
    if (nbe >= 0) {
      const S* fn = FFb + ((size_t)nbe * NF + nbf) * nf * nfp + orient_map<D, n>(ori, fp);
#pragma unroll
      for (int f = 0; f < nf; ++f) gb[f] = -S(0.5) * (own[f] - fn[f * nfp]);
    } else {
#pragma unroll
      for (int f = 0; f < nf; ++f) gb[f] = -own[f];
    }
  };
  // When every own face point of the tile has a thread of its own, that
  // thread's inputs of the face phase (1) are requested now, so their latency
  // overlaps the staging and the trace pass.
  constexpr bool ONE = T * NF * nfp <= (H::WARP ? 32 : H::THREADS);
  S pUL[nf], pgb[nf], pub[nf];
  int pnb = -1, pnbf = 0, pori = 0;  // neighbour, its face, orientation (reused by phase 6)
  const bool has1 = ONE && g_tid<V>() < nel * NF * nfp;
  if (has1) {
    const int i = g_tid<V>();
    const int e = e0 + i / (nfp * NF), face = (i / nfp) % NF;
    const size_t o = ((size_t)e * NF + face) * nf * nfp + i % nfp;
    S own[nf];
#pragma unroll
    for (int f = 0; f < nf; ++f) {
      pUL[f] = TU[o + f * nfp];
      own[f] = FFb[o + f * nfp];
      pub[f] = TUb[o + f * nfp];
    }
    pnb = M.nb[e * NF + face];
    pnbf = M.nbf[e * NF + face];
    pori = M.ori[e * NF + face];
    g_bar(own, pnb, pnbf, pori, i % nfp, pgb);
  }
  // Q_bar: curvilinear meshes combine its components node by node (staged
  // tile); on boxes each line of Q_bar_b is read once, from global memory
  if (CURV) stage_nodes<D, P, S, V, D * nf>(qbs, Qb + (size_t)e0 * D * H::STATE, nel);
  // 0. traces of Q (the forward Q is needed only here): copied when the
  //    forward stored them (TQg), else traced.  2D: each line read straight
  //    from global memory (every value is read twice); 3D: every value is
  //    read three times, so Q is staged once into qs (scratch for the later
  //    phases) and the lines are read from there.
  const S* qsrc = Q + (size_t)e0 * D * H::STATE;
  if (TQg) {
    const S* src = TQg + (size_t)e0 * TQS;
    for (int i = g_tid<V>(); i < nel * TQS; i += g_size<V>()) tq[i] = src[i];
  } else if (D == 3) {
    stage_nodes<D, P, S, V, D * nf>(qs, qsrc, nel);
    g_sync<V>();
    qsrc = qs;
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    if (TQg) break;
    for (int i = g_tid<V>(); i < nel * D * nf * nfp; i += g_size<V>()) {
      const int line = i % nfp;
      const int f = (i / nfp) % nf;
      const int c = (i / (nfp * nf)) % D;
      const int t = i / (nfp * nf * D);
      const S* v = qsrc + (size_t)t * D * H::STATE + (c * nf + f) * N;
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
  // 1. viscous face-flux adjoint at every own face point
  auto face_vjp = [&](int i, S (&UL)[nf], S (&gb)[nf], S (&ubf)[nf], int nbe) {
    const int fp = i % nfp;
    const int face = (i / nfp) % NF;
    const int t = i / (nfp * NF);
    const int e = e0 + t;
    const int a = face >> 1;
    S TQ[D][nf], nv[D], tqbv[D][nf];
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int f = 0; f < nf; ++f) {
        TQ[c][f] = tq[(((t * NF + face) * D + c) * nf + f) * nfp + fp];
        tqbv[c][f] = S(0);
      }
    if (CURV) {
#pragma unroll
      for (int c = 0; c < D; ++c) nv[c] = M.geo.SnE[(((size_t)e * NF + face) * D + c) * nfp + fp];
    } else {
#pragma unroll
      for (int c = 0; c < D; ++c) nv[c] = (c == a) ? ((face & 1) ? S(1) : S(-1)) : S(0);
    }
    if (nbe < 0)
      wall_visc_flux_vjp<D, S>(UL, TQ, nv, gb, M.gas, ubf, tqbv);
    else if (CURV)
      visc_flux_normal_vjp<D, S>(UL, TQ, nv, gb, M.gas, ubf, tqbv);
    else  // axis normal: the one row of the flux
      visc_flux_axis_vjp_rt<D, S>(UL, TQ, a, (face & 1) ? S(1) : S(-1), gb, M.gas, ubf, tqbv);
#pragma unroll
    for (int f = 0; f < nf; ++f) tub[((t * NF + face) * nf + f) * nfp + fp] = ubf[f];
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int f = 0; f < nf; ++f) tqb[(((t * NF + face) * D + c) * nf + f) * nfp + fp] = tqbv[c][f];
  };
  if (ONE) {
    if (has1) face_vjp(g_tid<V>(), pUL, pgb, pub, pnb);
  } else {
    for (int i = g_tid<V>(); i < nel * NF * nfp; i += g_size<V>()) {
      const int e = e0 + i / (nfp * NF), face = (i / nfp) % NF;
      const size_t o = ((size_t)e * NF + face) * nf * nfp + i % nfp;
      S UL[nf], own[nf], gb[nf], ubf[nf];
#pragma unroll
      for (int f = 0; f < nf; ++f) {
        UL[f] = TU[o + f * nfp];
        own[f] = FFb[o + f * nfp];
        ubf[f] = TUb[o + f * nfp];
      }
      const int nbe = M.nb[e * NF + face];
      g_bar(own, nbe, M.nbf[e * NF + face], M.ori[e * NF + face], i % nfp, gb);
      face_vjp(i, UL, gb, ubf, nbe);
    }
  }
  g_sync<V>();
  // 2. (curvilinear) Q_bar += transposed traces of TQ_bar; then P = iJ Q_bar in place
  const int t = g_tid<V>() / N, q = g_tid<V>() % N;
  const bool active = t < nel;
  const int e = e0 + t;
  if (CURV && active) {
    const S iJ = CURV ? M.geo.iJ[(size_t)e * N + q] : S(1);
    S lmq[D], lpq[D];
    int fpq[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int qa = H::qa(q, a);
      lmq[a] = lm[qa];
      lpq[a] = lp[qa];
      fpq[a] = H::fpoint(q, a);
    }
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int f = 0; f < nf; ++f) {
        S s = qbs[((t * D + c) * nf + f) * N + q];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          s += lmq[a] * tqb[(((t * NF + 2 * a) * D + c) * nf + f) * nfp + fpq[a]];
          s += lpq[a] * tqb[(((t * NF + 2 * a + 1) * D + c) * nf + f) * nfp + fpq[a]];
        }
        qbs[((t * D + c) * nf + f) * N + q] = s * iJ;
      }
  }
  if (CURV) g_sync<V>();
  if (!CURV) {
    // 2+3+4 (boxes): only component b of P feeds direction b, so each line of
    // P_b = Q_bar_b + (transposed traces of TQ_bar)_b is assembled where it is
    // used; one pass then gives r_b D_b^T P_b (-> qs) and the jump
    // cotangents J_bar = -+r_b sum_m L(-+)[m] P_b(m)
    // on the two faces normal to b.  Along a line the index in every other
    // direction a is constant, so each such face contributes one weight pair.
#pragma unroll
    for (int b = 0; b < D; ++b) {
      for (int i = g_tid<V>(); i < nel * nf * nfp; i += g_size<V>()) {
        int tt, f, line;
        line_item<nf, nfp>(i, tt, f, line);
        const S* pb = Qb + (size_t)(e0 + tt) * D * H::STATE + (b * nf + f) * N;
        S* v = qs + ((tt * D + b) * nf + f) * N;
        const S r = M.geo.rh[(e0 + tt) * D + b];
        auto tqb_at = [&](int face, int fp) { return tqb[(((tt * NF + face) * D + b) * nf + f) * nfp + fp]; };
        const S tbm = tqb_at(2 * b, line), tbp = tqb_at(2 * b + 1, line);
        S x[n];
#pragma unroll
        for (int k = 0; k < n; ++k) x[k] = pb[H::node(k, line, b)] + tb.lm[k] * tbm + tb.lp[k] * tbp;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          if (a == b) continue;
          const int qa = H::qa(H::node(0, line, b), a);
          const S wm = lm[qa], wp = lp[qa];
#pragma unroll
          for (int k = 0; k < n; ++k) {
            const int fpk = H::fpoint(H::node(k, line, b), a);
            x[k] += wm * tqb_at(2 * a, fpk) + wp * tqb_at(2 * a + 1, fpk);
          }
        }
        S sm = 0, sp = 0;
#pragma unroll
        for (int m = 0; m < n; ++m) {
          S acc = 0;
#pragma unroll
          for (int k = 0; k < n; ++k) acc += tb.D[k][m] * x[k];
          v[H::node(m, line, b)] = r * acc;
          sm += tb.Lm[m] * x[m];
          sp += tb.Lp[m] * x[m];
        }
        js[((tt * NF + 2 * b) * nf + f) * nfp + line] = -r * sm;
        js[((tt * NF + 2 * b + 1) * nf + f) * nfp + line] = r * sp;
      }
    }
  } else {
  // 3. dU_bar_b(q) = sum_c Ja[b][c] P_c   -> qs
  if (active) {
#pragma unroll
    for (int b = 0; b < D; ++b)
#pragma unroll
      for (int f = 0; f < nf; ++f) {
        S s = 0;
#pragma unroll
        for (int c = 0; c < D; ++c)
          s += M.geo.Ja[(((size_t)e * D + b) * D + c) * N + q] * qbs[((t * D + c) * nf + f) * N + q];
        qs[((t * D + b) * nf + f) * N + q] = s;
      }
  }
  g_sync<V>();
  // 4. line passes: D_b^T dU_bar_b in place (qs), and the jump cotangents J_bar (js)
#pragma unroll
  for (int b = 0; b < D; ++b) {
    for (int i = g_tid<V>(); i < nel * nf * nfp; i += g_size<V>()) {
      int tt, f, line;
      line_item<nf, nfp>(i, tt, f, line);
      S* v = qs + ((tt * D + b) * nf + f) * N;
      S x[n];
#pragma unroll
      for (int k = 0; k < n; ++k) x[k] = v[H::node(k, line, b)];
#pragma unroll
      for (int m = 0; m < n; ++m) {
        S acc = 0;
#pragma unroll
        for (int k = 0; k < n; ++k) acc += tb.D[k][m] * x[k];
        v[H::node(m, line, b)] = acc;
      }
      // J_bar on the two faces normal to b: sum_c Sn_c sum_m L(+-)[m] P_c(m)
      S jm = 0, jp = 0;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const S* pc = qbs + ((tt * D + c) * nf + f) * N;
        S sm = 0, sp = 0;
#pragma unroll
        for (int m = 0; m < n; ++m) {
          const S y = pc[H::node(m, line, b)];
          sm += tb.Lm[m] * y;
          sp += tb.Lp[m] * y;
        }
        const size_t ge = (size_t)(e0 + tt) * NF;
        jm += M.geo.SnE[((ge + 2 * b) * D + c) * nfp + line] * sm;
        jp += M.geo.SnE[((ge + 2 * b + 1) * D + c) * nfp + line] * sp;
      }
      js[((tt * NF + 2 * b) * nf + f) * nfp + line] = jm;
      js[((tt * NF + 2 * b + 1) * nf + f) * nfp + line] = jp;
    }
  }
  }
  g_sync<V>();
  // 5. U_bar += sum_b D_b^T dU_bar_b
  if (active) {
    S* ub = Ub + (size_t)e * H::STATE + q;
#pragma unroll
    for (int f = 0; f < nf; ++f) {
      S s = 0;
#pragma unroll
      for (int b = 0; b < D; ++b) s += qs[((t * D + b) * nf + f) * N + q];
      ub[f * N] += s;
    }
  }
  // 6. the own trace cotangent and the neighbour's share of each jump
  auto finish_at = [&](int i, int nbe, int nbf, int ori, const S* ULw) {
    const int fp = i % nfp;
    const int face = (i / nfp) % NF;
    const int tt = i / (nfp * NF);
    const int ee = e0 + tt;
    const size_t o = ((size_t)ee * NF + face) * nf * nfp + fp;
    S jb[nf], ubf[nf];
#pragma unroll
    for (int f = 0; f < nf; ++f) {
      jb[f] = js[((tt * NF + face) * nf + f) * nfp + fp];
      ubf[f] = tub[((tt * NF + face) * nf + f) * nfp + fp];
    }
    if (nbe >= 0) {  // scatter into the neighbour's own face slot (its gather reads it there)
      const size_t on = ((size_t)nbe * NF + nbf) * nf * nfp + orient_map<D, n>(ori, fp);
#pragma unroll
      for (int f = 0; f < nf; ++f) {
        ubf[f] -= S(0.5) * jb[f];
        JB[on + f * nfp] = jb[f];
      }
    } else {
      S UL[nf];
#pragma unroll
      for (int f = 0; f < nf; ++f) {
        UL[f] = ULw ? ULw[f] : TU[o + f * nfp];
        ubf[f] -= jb[f];
        JB[o + f * nfp] = S(0);
      }
      wall_state_vjp<D, S>(UL, jb, ubf);
    }
#pragma unroll
    for (int f = 0; f < nf; ++f) TUb[o + f * nfp] = ubf[f];
  };
  if (ONE) {
    if (has1) finish_at(g_tid<V>(), pnb, pnbf, pori, pUL);
  } else {
    for (int i = g_tid<V>(); i < nel * NF * nfp; i += g_size<V>()) {
      const int k = (e0 + i / (nfp * NF)) * NF + (i / nfp) % NF;
      finish_at(i, M.nb[k], M.nbf[k], M.ori[k], nullptr);
    }
  }
}

// ---------------------------------------------------------------------------
template <int D, int P, typename S, bool VISC, int V>
__global__ void __launch_bounds__(Sh<D, P, V>::THREADS) k_vjp_gather(Mesh<S> M, const S* __restrict__ TUb,
                                                                     const S* __restrict__ JB, S* g, Cot<S> cot) {
  using H = Sh<D, P, V>;
  constexpr int n = H::n, N = H::N, nf = H::nf, nfp = H::nfp, NF = H::NF, T = H::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S* tub = reinterpret_cast<S*>(g_smem<V>(smem_raw, smem_vgather_g<D, P, S, V>()));  // [T][NF][nf][nfp]
  S* lm = tub + T * H::FACE;
  S* lp = lm + n;
  const int e0 = g_index<V>() * T;
  const int nel = min(T, M.E - e0);
  load_tab<S, V>(M.tabs, P, lm, lp, nullptr, nullptr, n);
  // this thread's node: its running cotangent is read first (latency overlaps the face phase)
  const int t = g_tid<V>() / N, q = g_tid<V>() % N;
  const bool act = t < nel;
  const size_t off = (size_t)(e0 + t) * H::STATE + q;
  S gq[nf];
  double l64[nf];  // ARK adjoint: lambda_{n+1} and the sum of the other stages' nu, read early too
  S nsum[nf];
  if (act) {
#pragma unroll
    for (int f = 0; f < nf; ++f) gq[f] = g[off + f * N];
    if (cot.lam64_out) {
#pragma unroll
      for (int f = 0; f < nf; ++f) {
        l64[f] = cot.lam64_out[off + f * N];
        nsum[f] = S(0);
      }
      if (sizeof(S) != 8) {
#pragma unroll
        for (int j = 0; j < MAXSTAGES - 1; ++j) {
          if (j < cot.n_all) {
#pragma unroll
            for (int f = 0; f < nf; ++f) nsum[f] += cot.nu_all[j][off + f * N];
          }
        }
      }
    }
  }
  {
    const S* src = TUb + (size_t)e0 * H::FACE;
    if (!VISC) {
      stage_faces<D, P, S, V>(tub, src, nel);
    } else {
      // own trace cotangent plus half the jump cotangent the neighbour scattered here
      for (int i = g_tid<V>(); i < nel * NF * nfp; i += g_size<V>()) {
        const int fp = i % nfp, tf = i / nfp;  // tf = t * NF + face
        const S* jb = JB + (size_t)e0 * H::FACE;
        S a[nf], c[nf];
#pragma unroll
        for (int f = 0; f < nf; ++f) {
          a[f] = src[(tf * nf + f) * nfp + fp];
          c[f] = jb[(tf * nf + f) * nfp + fp];
        }
#pragma unroll
        for (int f = 0; f < nf; ++f) tub[(tf * nf + f) * nfp + fp] = a[f] + S(0.5) * c[f];
      }
    }
  }
  g_sync<V>();
  if (!act) return;
  S lmq[D], lpq[D];
  int fpq[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const int qa = H::qa(q, a);
    lmq[a] = lm[qa];
    lpq[a] = lp[qa];
    fpq[a] = H::fpoint(q, a);
  }
#pragma unroll
  for (int f = 0; f < nf; ++f) {
    S s = gq[f];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      s += lmq[a] * tub[((t * NF + 2 * a) * nf + f) * nfp + fpq[a]];
      s += lpq[a] * tub[((t * NF + 2 * a + 1) * nf + f) * nfp + fpq[a]];
    }
    g[off + f * N] = s;
    if (cot.lam64_out) {  // ARK adjoint: lambda_n = lambda_{n+1} + sum_j nu_j, accumulated in FP64
      if (sizeof(S) == 8) {
        double acc = l64[f] + (double)s;
        for (int j = 0; j < cot.n_all; ++j) acc += (double)cot.nu_all[j][off + f * N];
        cot.lam64_out[off + f * N] = acc;
      } else {  // FP32 increment, one FP64 add (as the forward's last stage)
        cot.lam64_out[off + f * N] = l64[f] + (double)(s + nsum[f]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
template <int D, int P, typename S>
struct VjpOps {
  template <int V>
  using H = Sh<D, P, V>;
  template <int V>
  static size_t smem_elem() {
    return H<V>::GROUPS * smem_velem_g<D, P, S, V>();
  }
  template <int V, bool CURV = true>  // the curvilinear size bounds both
  static size_t smem_br1() {
    return H<V>::GROUPS * smem_vbr1_g<D, P, S, V, CURV>();
  }
  template <int V>
  static size_t smem_gather() {
    return H<V>::GROUPS * smem_vgather_g<D, P, S, V>();
  }
  template <int V>
  static int blocks(int E) {
    return H<V>::WARP ? (E + WPB - 1) / WPB : (E + H<V>::T - 1) / H<V>::T;
  }
  // 0 elem, 1 br1, 2 gather; SIZE_MAX if the variant cannot run here
  template <int V>
  static size_t smem_v(int kind) {
    if (!H<V>::VALID) return (size_t)-1;
    return kind == 0 ? smem_elem<V>() : kind == 1 ? smem_br1<V>() : smem_gather<V>();
  }
  static size_t smem(int kind, int V) {
    switch (V) {
      case 0: return smem_v<0>(kind);
      case 1: return smem_v<1>(kind);
      case 2: return smem_v<2>(kind);
      default: return smem_v<3>(kind);
    }
  }

  template <bool VISC, bool CURV, int V>
  static cudaError_t elem_v(const Mesh<S>& M, const S* U, const VjpWork& w, const Cot<S>& c, S* Ub,
                            cudaStream_t st) {
    if (c.nu_prev) {
      static SmemGate done;
      auto k = k_vjp_elem<D, P, S, VISC, CURV, V, true>;
      if (const cudaError_t e = allow_smem_once(k, smem_elem<V>(), done)) return e;
      k<<<blocks<V>(M.E), H<V>::THREADS, smem_elem<V>(), st>>>(M, U, (const S*)w.Q, c, (S*)w.FFb, Ub, (S*)w.Qb,
                                                               (const S*)w.TUb, (const S*)w.JB);
    } else {
      static SmemGate done;
      auto k = k_vjp_elem<D, P, S, VISC, CURV, V, false>;
      if (const cudaError_t e = allow_smem_once(k, smem_elem<V>(), done)) return e;
      k<<<blocks<V>(M.E), H<V>::THREADS, smem_elem<V>(), st>>>(M, U, (const S*)w.Q, c, (S*)w.FFb, Ub, (S*)w.Qb,
                                                               nullptr, nullptr);
    }
    return cudaGetLastError();
  }
  template <bool VISC, bool CURV>
  static cudaError_t elem_c(const Mesh<S>& M, int V, const S* U, const VjpWork& w, const Cot<S>& c, S* Ub,
                            cudaStream_t st) {
    if (V == 0) return elem_v<VISC, CURV, 0>(M, U, w, c, Ub, st);
    if (V == 1) return elem_v<VISC, CURV, 1>(M, U, w, c, Ub, st);
    if (V == 2) return elem_v<VISC, CURV, 2>(M, U, w, c, Ub, st);
    return elem_v<VISC, CURV, 3>(M, U, w, c, Ub, st);
  }
  static cudaError_t elem(const Mesh<S>& M, int V, bool visc, bool curv, const S* U, const VjpWork& w,
                          const Cot<S>& c, S* Ub, cudaStream_t st) {
    if (visc) return curv ? elem_c<true, true>(M, V, U, w, c, Ub, st) : elem_c<true, false>(M, V, U, w, c, Ub, st);
    return curv ? elem_c<false, true>(M, V, U, w, c, Ub, st) : elem_c<false, false>(M, V, U, w, c, Ub, st);
  }

  static cudaError_t face(const Mesh<S>& M, bool /*visc*/, bool curv, const VjpWork& w, cudaStream_t st) {
    const int total = M.nFaces * Sh<D, P>::nfp;
    if (total == 0) return cudaSuccess;
    const int nb = (total + 255) / 256;
    const S* TU = (const S*)w.TU;
    const S* FFb = (const S*)w.FFb;
    S* TUb = (S*)w.TUb;
    if (curv) k_vjp_face<D, P, S, true><<<nb, 256, 0, st>>>(M, TU, FFb, TUb);
    else k_vjp_face<D, P, S, false><<<nb, 256, 0, st>>>(M, TU, FFb, TUb);
    return cudaGetLastError();
  }

  template <bool CURV, int V>
  static cudaError_t br1_v(const Mesh<S>& M, const VjpWork& w, S* Ub, cudaStream_t st) {
    static SmemGate done;
    auto k = k_vjp_br1<D, P, S, CURV, V>;
    if (const cudaError_t e = allow_smem_once(k, smem_br1<V, CURV>(), done)) return e;
    k<<<blocks<V>(M.E), H<V>::THREADS, smem_br1<V, CURV>(), st>>>(M, (const S*)w.TU, (const S*)w.Q, (const S*)w.FFb,
                                                             (S*)w.Qb, (S*)w.TUb, (S*)w.JB, Ub, (const S*)w.TQ);
    return cudaGetLastError();
  }
  static cudaError_t br1(const Mesh<S>& M, int V, bool curv, const VjpWork& w, S* Ub, cudaStream_t st) {
    if (curv) {
      if (V == 0) return br1_v<true, 0>(M, w, Ub, st);
      if (V == 1) return br1_v<true, 1>(M, w, Ub, st);
      if (V == 2) return br1_v<true, 2>(M, w, Ub, st);
      return br1_v<true, 3>(M, w, Ub, st);
    }
    if (V == 0) return br1_v<false, 0>(M, w, Ub, st);
    if (V == 1) return br1_v<false, 1>(M, w, Ub, st);
    if (V == 2) return br1_v<false, 2>(M, w, Ub, st);
    return br1_v<false, 3>(M, w, Ub, st);
  }

  template <bool VISC, int V>
  static cudaError_t gather_v(const Mesh<S>& M, const VjpWork& w, S* g, const Cot<S>& c, cudaStream_t st) {
    static SmemGate done;
    auto k = k_vjp_gather<D, P, S, VISC, V>;
    if (const cudaError_t e = allow_smem_once(k, smem_gather<V>(), done)) return e;
    k<<<blocks<V>(M.E), H<V>::THREADS, smem_gather<V>(), st>>>(M, (const S*)w.TUb, (const S*)w.JB, g, c);
    return cudaGetLastError();
  }
  static cudaError_t gather(const Mesh<S>& M, int V, bool visc, const VjpWork& w, S* g, const Cot<S>& c,
                            cudaStream_t st) {
    if (visc) {
      if (V == 0) return gather_v<true, 0>(M, w, g, c, st);
      if (V == 1) return gather_v<true, 1>(M, w, g, c, st);
      if (V == 2) return gather_v<true, 2>(M, w, g, c, st);
      return gather_v<true, 3>(M, w, g, c, st);
    }
    if (V == 0) return gather_v<false, 0>(M, w, g, c, st);
    if (V == 1) return gather_v<false, 1>(M, w, g, c, st);
    if (V == 2) return gather_v<false, 2>(M, w, g, c, st);
    return gather_v<false, 3>(M, w, g, c, st);
  }
};

// Type-erased adjoint launch table (one per (D, P, S)); V = tile variant.
struct VjpTable {
  cudaError_t (*elem)(const void* M, int V, bool visc, bool curv, const void* U, const VjpWork& w, const void* cot,
                      void* Ub, cudaStream_t st);
  cudaError_t (*face)(const void* M, bool visc, bool curv, const VjpWork& w, cudaStream_t st);
  cudaError_t (*br1)(const void* M, int V, bool curv, const VjpWork& w, void* Ub, cudaStream_t st);
  cudaError_t (*gather)(const void* M, int V, bool visc, const VjpWork& w, void* g, const void* cot,
                        cudaStream_t st);
  size_t (*smem)(int kind, int V);  // 0 elem, 1 br1, 2 gather
};

template <int D, int P, typename S>
const void* vjp_table() {
  struct R {
    static cudaError_t elem(const void* M, int V, bool v, bool c, const void* U, const VjpWork& w, const void* cot,
                            void* Ub, cudaStream_t st) {
      return VjpOps<D, P, S>::elem(*(const Mesh<S>*)M, V, v, c, (const S*)U, w, *(const Cot<S>*)cot, (S*)Ub, st);
    }
    static cudaError_t face(const void* M, bool v, bool c, const VjpWork& w, cudaStream_t st) {
      return VjpOps<D, P, S>::face(*(const Mesh<S>*)M, v, c, w, st);
    }
    static cudaError_t br1(const void* M, int V, bool c, const VjpWork& w, void* Ub, cudaStream_t st) {
      return VjpOps<D, P, S>::br1(*(const Mesh<S>*)M, V, c, w, (S*)Ub, st);
    }
    static cudaError_t gather(const void* M, int V, bool v, const VjpWork& w, void* g, const void* cot,
                              cudaStream_t st) {
      return VjpOps<D, P, S>::gather(*(const Mesh<S>*)M, V, v, w, (S*)g, *(const Cot<S>*)cot, st);
    }
    static size_t smem(int kind, int V) { return VjpOps<D, P, S>::smem(kind, V); }
  };
  static const VjpTable t = {&R::elem, &R::face, &R::br1, &R::gather, &R::smem};
  return &t;
}

}  // namespace dgx
