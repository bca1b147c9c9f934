// Kernels of the paper's own explicit operator, DG-IP (sm_103a): the
// Vijayasundaram convective flux and the symmetric interior-penalty viscous
// terms of Sec. 3.3 (B_I of Eq. bilinear_form_interior_sdg, penalty
// tau = alpha (k+1)^2 / l of Eq. penalty_coefficient_ip), the farfield and
// adiabatic-wall forms of App. B.1 and the DG side of the geometry-split
// interface of Sec. 4.1.1 (Eq. interface_bilinearform_explicit), on
// axis-aligned box meshes with the collocated Gauss-node basis.
//
// Per residual:
//   k_dgip_trace  U -> TU, G     face traces of U and each own face's viscous
//                                normal flux G = F^nu(U_f, grad U_f).n with the
//                                element's own (broken) gradient at the face
//   k_dgip_face   TU, G -> FF, HA  one thread per unique face point: the
//                                numerical flux (written +- to both sides) and
//                                each side's adjoint-consistency vector
//                                H = c K(U)(delta (x) n) (all directions)
//   k_dgip_elem   U, FF, HA -> f volume flux F^c - F^nu(U, grad U) (gradient
//                                from the element's own lines, never stored),
//                                weak divergence, lift of FF, the adjoint-
//                                consistency term (normal part lifted with
//                                l'(+-1)/w, tangential part folded into the
//                                volume flux before the divergence), inverse
//                                mass; optionally the ARK stage update.
// With unit normals on boxes (r_a = 2/h_a), node q of an element gets
//   f_q = sum_a r_a [ sum_m Dh[q_a][m] Fa(m) - L(-)[q_a] FF(2a) - L(+)[q_a] FF(2a+1)
//                     + r_a (dL(-)[q_a] H_a(2a) + dL(+)[q_a] H_a(2a+1)) ],
//   Fa(r) = (F^c - F^nu)_a(r) + sum_{a0 != a} r_a0 sum_side L(side)[r_a0] H_a(face(a0, side), r),
// L = l(+-1)/w, dL = l'(+-1)/w; this is the oracle's
//   (1/(w_q J)) sum_faces sum_f w_f grad l_q(x_f) . H(f)
// written out for boxes.  The adjoint kernels reverse the three steps; the
// face step is differentiated exactly with forward-mode dual numbers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "dgip_physics.cuh"
#include "kernels.cuh"
#include "ops.cuh"

namespace dgx {

template <typename S>
struct Dgip {
  const S* il;          // [E] 1/l = |dT| / |T| of every element (boxes: 2 sum_a 1/h_a)
  // curvilinear meshes (nullptr on boxes): the metric terms and 1/J traced to
  // every own face point, JaF[E][2D][a][c][nfp] = (J dxi_a/dx_c)(x_f), iJF[E][2D][nfp]
  const S* JaF;
  const S* iJF;
  S tk2;                // alpha (k+1)^2
  const int8_t* mask;   // [E] 1 = explicit element; nullptr: every element explicit
  const S* Uim;         // states of the implicit elements ([E][nf][N] layout) or nullptr
  S Uinf[5];            // farfield state (conservative)
};

template <int D, int P>
using HD = Sh<D, P, 1>;  // one CTA of ~256 threads per tile of T elements

template <typename S>
__device__ __forceinline__ bool dgip_explicit(const Dgip<S>& dp, int e) {
  return !dp.mask || dp.mask[e] != 0;
}

// stride of tangential direction c inside the face-point index of faces normal to a0
template <int D, int P>
__device__ __forceinline__ int tan_stride(int c, int a0) {
  return c < a0 ? HD<D, P>::pw(c) : HD<D, P>::pw(c - 1);
}

// f(std::integral_constant<int, v>) for a runtime v in [I, N): face and
// direction numbers become compile-time constants, so the node and face-point
// index arithmetic that depends on them is constant multiplies (a runtime
// face number makes every such index an integer division).
template <int I, int N, typename F>
__device__ __forceinline__ void with_const(int v, F&& f) {
  if constexpr (I < N) {
    if (v == I) f(std::integral_constant<int, I>{});
    else with_const<I + 1, N>(v, f);
  }
}

// Face quantities of a staged tile (us[t][f][q]), one thread per (element,
// field, line) and direction: the traces tu[t][face][f][fp] at both ends of
// every line and, for the viscous terms, the normal derivative of the
// element's polynomial there, qf[t][face][a][f][fp] = (2/h_a) l'(+-1) . line
// (face normal to a).  TUg (or nullptr) receives the traces in global memory.
template <int D, int P, typename S, bool VISC, bool CURV = false>
__device__ __forceinline__ void face_lines(const S* us, S* tu, S* qf, const S* rh, int e0, int nel, S* TUg) {
  using H = HD<D, P>;
  constexpr int n = H::n, N = H::N, nf = H::nf, nfp = H::nfp, NF = H::NF, STATE = H::STATE, FACE = H::FACE;
  constexpr Tab1<S> tb = make_tab1<S>(P);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    for (int i = threadIdx.x; i < nel * nf * nfp; i += blockDim.x) {
      int t, f, line;
      line_item<nf, nfp>(i, t, f, line);
      const S* v = us + t * STATE + f * N;
      S x[n];
#pragma unroll
      for (int m = 0; m < n; ++m) x[m] = v[H::node(m, line, a)];
      S sm = 0, sp = 0, dm = 0, dq = 0;
#pragma unroll
      for (int m = 0; m < n; ++m) {
        sm += tb.lm[m] * x[m];
        sp += tb.lp[m] * x[m];
        if (VISC) {
          dm += tb.dlm[m] * x[m];
          dq += tb.dlp[m] * x[m];
        }
      }
      const int om = (t * NF + 2 * a) * nf * nfp + f * nfp + line, op = om + nf * nfp;
      tu[om] = sm;
      tu[op] = sp;
      if (TUg) {
        TUg[(size_t)e0 * FACE + om] = sm;
        TUg[(size_t)e0 * FACE + op] = sp;
      }
      if (VISC) {  // boxes: physical (2/h_a); curvilinear: reference derivatives
        const S r = CURV ? S(1) : rh[(e0 + t) * D + a];
        qf[((t * NF + 2 * a) * D + a) * nf * nfp + f * nfp + line] = r * dm;
        qf[((t * NF + 2 * a + 1) * D + a) * nf * nfp + f * nfp + line] = r * dq;
      }
    }
  }
}

// The tangential derivatives on every face from its traced values, one thread
// per (element, face, tangential direction, field, face line): the line's n
// values in, the derivative at its n points out (rows of D as compile-time
// constants), qf[t][face][c][f][fp] = (2/h_c) (D y)(fp).
template <int D, int P, typename S, bool CURV = false>
__device__ __forceinline__ void face_tangential(const S* tu, S* qf, const S* rh, int e0, int nel) {
  using H = HD<D, P>;
  constexpr int n = H::n, nf = H::nf, nfp = H::nfp, NF = H::NF;
  constexpr int NL = nfp / n;  // lines of one tangential direction on a face
  constexpr int ITEMS = NF * (D - 1) * nf * NL;
  constexpr Tab1<S> tb = make_tab1<S>(P);
  for (int i = threadIdx.x; i < nel * ITEMS; i += blockDim.x) {
    const int fl = i % NL, f = (i / NL) % nf, ci = (i / (NL * nf)) % (D - 1);
    const int face = (i / (NL * nf * (D - 1))) % NF, t = i / ITEMS;
    const int a0 = face >> 1, c = ci + (ci >= a0);
    const int st = tan_stride<D, P>(c, a0);
    const int base = (D == 2) ? 0 : (st == 1 ? fl * n : fl);
    const S* y = tu + (t * NF + face) * nf * nfp + f * nfp + base;
    S yv[n];
#pragma unroll
    for (int k = 0; k < n; ++k) yv[k] = y[k * st];
    const S r = CURV ? S(1) : rh[(e0 + t) * D + c];
    S* o = qf + ((t * NF + face) * D + c) * nf * nfp + f * nfp + base;
#pragma unroll
    for (int j = 0; j < n; ++j) {
      S s = 0;
#pragma unroll
      for (int k = 0; k < n; ++k) s += tb.D[j][k] * yv[k];
      o[j * st] = r * s;
    }
  }
}

// Transposed face_tangential for one tangential direction index ci:
// tub[t][face][f] += (2/h_c) D^T qfb[t][face][c][f] along every face line.
template <int D, int P, typename S, bool CURV = false>
__device__ __forceinline__ void face_tangential_t(const S* qfb, S* tub, const S* rh, int e0, int nel, int ci) {
  using H = HD<D, P>;
  constexpr int n = H::n, nf = H::nf, nfp = H::nfp, NF = H::NF;
  constexpr int NL = nfp / n;
  constexpr int ITEMS = NF * nf * NL;
  constexpr Tab1<S> tb = make_tab1<S>(P);
  for (int i = threadIdx.x; i < nel * ITEMS; i += blockDim.x) {
    const int fl = i % NL, f = (i / NL) % nf, face = (i / (NL * nf)) % NF, t = i / ITEMS;
    const int a0 = face >> 1, c = ci + (ci >= a0);
    const int st = tan_stride<D, P>(c, a0);
    const int base = (D == 2) ? 0 : (st == 1 ? fl * n : fl);
    const S* z = qfb + ((t * NF + face) * D + c) * nf * nfp + f * nfp + base;
    S zv[n];
#pragma unroll
    for (int j = 0; j < n; ++j) zv[j] = z[j * st];
    const S r = CURV ? S(1) : rh[(e0 + t) * D + c];
    S* o = tub + (t * NF + face) * nf * nfp + f * nfp + base;
#pragma unroll
    for (int k = 0; k < n; ++k) {
      S s = 0;
#pragma unroll
      for (int j = 0; j < n; ++j) s += tb.D[j][k] * zv[j];
      o[k * st] += r * s;
    }
  }
}

template <int D, typename S>
__device__ __forceinline__ void unit_normal(int face, S (&nv)[D]) {
#pragma unroll
  for (int c = 0; c < D; ++c) nv[c] = (c == (face >> 1)) ? ((face & 1) ? S(1) : S(-1)) : S(0);
}

template <typename S>
__device__ __forceinline__ Gas<S> gas_no_heat(const Gas<S>& g) {
  Gas<S> w = g;
  w.kcv = S(0);
  return w;
}

// ---------------------------------------------------------------------------
// k_dgip_trace: TU = traces of U; G = each own face's viscous normal flux
// (interior: F^nu(U_f, grad U_f).n; wall: the same with kappa = 0 (q.n = 0);
// farfield: F^nu(U_inf, grad U_f).n).
// ---------------------------------------------------------------------------
template <int D, int P, typename S, bool VISC, bool CURV>
__global__ void __launch_bounds__(HD<D, P>::THREADS) k_dgip_trace(Mesh<S> M, Dgip<S> dp, const S* __restrict__ U,
                                                                  S* __restrict__ TU, S* __restrict__ G,
                                                                  S* __restrict__ QF) {
  using H = HD<D, P>;
  constexpr int n = H::n, N = H::N, nf = H::nf, nfp = H::nfp, NF = H::NF, T = H::T, STATE = H::STATE,
                FACE = H::FACE;
  constexpr Tab1<S> tb = make_tab1<S>(P);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S* us = reinterpret_cast<S*>(smem_raw);  // [T][nf][N]
  S* tu = us + T * STATE;                  // [T][NF][nf][nfp]
  S* qf = tu + T * FACE;                   // [T][NF][D][nf][nfp] face gradients (viscous)
  const int e0 = blockIdx.x * T;
  const int nel = min(T, M.E - e0);
  const int tid = threadIdx.x;
  {
    const int t = tid / N, q = tid % N;
    if (t < nel) {
      const int e = e0 + t;
      const S* src = (dgip_explicit(dp, e) ? U : dp.Uim) + (size_t)e * STATE + q;
      S v[nf];
#pragma unroll
      for (int f = 0; f < nf; ++f) v[f] = src[f * N];
#pragma unroll
      for (int f = 0; f < nf; ++f) us[t * STATE + f * N + q] = v[f];
    }
  }
  __syncthreads();
  face_lines<D, P, S, VISC, CURV>(us, tu, qf, M.geo.rh, e0, nel, TU);
  if (!VISC) return;
  __syncthreads();
  face_tangential<D, P, S, CURV>(tu, qf, M.geo.rh, e0, nel);
  __syncthreads();
  if (QF) {  // keep the face gradients for the adjoint (the tile's block is contiguous)
    constexpr int QS = NF * D * nf * nfp;
    S* dst = QF + (size_t)e0 * QS;
    for (int i = tid; i < nel * QS; i += blockDim.x) dst[i] = qf[i];
  }
  const Gas<S> gw = gas_no_heat(M.gas);
  for (int i = tid; i < nel * NF * nfp; i += blockDim.x) {
    const int fp = i % nfp, face = (i / nfp) % NF, t = i / (nfp * NF);
    const int e = e0 + t;
    const S* tf = tu + (t * NF + face) * nf * nfp;
    const S* qg = qf + (t * NF + face) * D * nf * nfp + fp;
    S Uf[nf], Q[D][nf], nv[D], Gv[nf];
#pragma unroll
    for (int f = 0; f < nf; ++f) Uf[f] = tf[f * nfp + fp];
    if (CURV) {  // grad U = (1/J) sum_b (J dxi_b/dx) d/dxi_b U with the traced metric; own area normal
      const size_t fo = (size_t)e * NF + face;
      const S ij = dp.iJF[fo * nfp + fp];
      S ja[D][D];
#pragma unroll
      for (int b = 0; b < D; ++b)
#pragma unroll
        for (int c = 0; c < D; ++c) ja[b][c] = dp.JaF[((fo * D + b) * D + c) * nfp + fp];
#pragma unroll
      for (int c = 0; c < D; ++c) {
        nv[c] = M.geo.SnE[(fo * D + c) * nfp + fp];
#pragma unroll
        for (int f = 0; f < nf; ++f) {
          S v = 0;
#pragma unroll
          for (int b = 0; b < D; ++b) v += ja[b][c] * qg[(b * nf + f) * nfp];
          Q[c][f] = ij * v;
        }
      }
    } else {
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int f = 0; f < nf; ++f) Q[c][f] = qg[(c * nf + f) * nfp];
      unit_normal<D, S>(face, nv);
    }
    const int nbk = M.nb[e * NF + face];
    // boxes: the axis normal selects one row of the flux
    auto vflux = [&](const S (&Us)[nf], const Gas<S>& gg) {
      if (CURV) visc_flux_normal<D, S>(Us, Q, nv, gg, Gv);
      else visc_flux_axis_rt<D, S>(Us, Q, face >> 1, (face & 1) ? S(1) : S(-1), gg, Gv);
    };
    if (nbk >= 0) {
      vflux(Uf, M.gas);
    } else if (nbk == -1) {
      vflux(Uf, gw);
    } else {
      S Ui[nf];
#pragma unroll
      for (int f = 0; f < nf; ++f) Ui[f] = dp.Uinf[f];
      vflux(Ui, M.gas);
    }
    S* gd = G + ((size_t)e * NF + face) * nf * nfp + fp;
#pragma unroll
    for (int f = 0; f < nf; ++f) gd[f * nfp] = Gv[f];
  }
}

// ---------------------------------------------------------------------------
// k_dgip_face: one thread per unique face point (unit normals on boxes).
// ---------------------------------------------------------------------------
template <int D, int P, typename S, bool VISC, bool CURV>
__global__ void __launch_bounds__(128) k_dgip_face(Mesh<S> M, Dgip<S> dp, const S* __restrict__ TU,
                                                   const S* __restrict__ G, S* __restrict__ FF, S* __restrict__ HA) {
  using H = HD<D, P>;
  constexpr int n = H::n, nf = H::nf, nfp = H::nfp, NF = H::NF;
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= M.nFaces * nfp) return;
  const int F = gid / nfp, fp = gid % nfp;
  const int4 rec = M.faces[F];
  const int em = rec.x, ep = rec.y;
  const int fm = rec.z & 0xff, fo = (rec.z >> 8) & 0xff, code = (rec.z >> 16) & 0xff;
  const bool exm = dgip_explicit(dp, em);
  const bool exp_ = ep >= 0 && dgip_explicit(dp, ep);
  if (!exm && !exp_) return;
  S nv[D];
  S isJ = S(1);  // 1 / |area normal| (the penalty term is tau K(..).n / |n|)
  if (CURV) {    // averaged area normal (own one on boundary faces)
    S n2 = 0;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      nv[c] = M.geo.SnF[((size_t)F * D + c) * nfp + fp];
      n2 += nv[c] * nv[c];
    }
    isJ = S(1) / sqrt(n2);
  } else {
    unit_normal<D, S>(fm, nv);
  }
  S UL[nf], UR[nf], Fv[nf], HL[D][nf], HR[D][nf];
  const S* tl = TU + ((size_t)em * NF + fm) * nf * nfp + fp;
#pragma unroll
  for (int f = 0; f < nf; ++f) UL[f] = tl[f * nfp];
  const Gas<S> gw = gas_no_heat(M.gas);
  int fpn = 0;
  if (ep >= 0) {
    fpn = orient_map<D, n>(code, fp);
    const S* tr = TU + ((size_t)ep * NF + fo) * nf * nfp + fpn;
#pragma unroll
    for (int f = 0; f < nf; ++f) UR[f] = tr[f * nfp];
    const S tau = dp.tk2 * fmax(dp.il[em], dp.il[ep]) * isJ;
    dgip_face_fn<D, S, S, VISC, DGIP_INTERIOR, !CURV, !CURV && sizeof(S) == 8>(UL, UR, nv, M.gas, gw, tau, exm && !exp_, exp_ && !exm, Fv, HL, HR);
    if (VISC) {
      const S* gl = G + ((size_t)em * NF + fm) * nf * nfp + fp;
      const S* gr = G + ((size_t)ep * NF + fo) * nf * nfp + fpn;
#pragma unroll
      for (int f = 0; f < nf; ++f) Fv[f] -= S(0.5) * (gl[f * nfp] - gr[f * nfp]);
    }
  } else {
    const S tau = dp.tk2 * dp.il[em] * isJ;
    if (ep == -1) {
      dgip_face_fn<D, S, S, VISC, DGIP_WALL, !CURV, !CURV && sizeof(S) == 8>(UL, UL, nv, M.gas, gw, tau, false, false, Fv, HL, HR);
    } else {
#pragma unroll
      for (int f = 0; f < nf; ++f) UR[f] = dp.Uinf[f];
      dgip_face_fn<D, S, S, VISC, DGIP_FARFIELD, !CURV, !CURV && sizeof(S) == 8>(UL, UR, nv, M.gas, gw, tau, false, false, Fv, HL, HR);
    }
    if (VISC) {
      const S* gl = G + ((size_t)em * NF + fm) * nf * nfp + fp;
#pragma unroll
      for (int f = 0; f < nf; ++f) Fv[f] -= gl[f * nfp];
    }
  }
  if (exm) {
    S* ol = FF + ((size_t)em * NF + fm) * nf * nfp + fp;
#pragma unroll
    for (int f = 0; f < nf; ++f) ol[f * nfp] = Fv[f];
    if (VISC) {
      S* hl = HA + ((size_t)em * NF + fm) * D * nf * nfp + fp;
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int f = 0; f < nf; ++f) hl[(c * nf + f) * nfp] = HL[c][f];
    }
  }
  if (exp_) {
    S* orr = FF + ((size_t)ep * NF + fo) * nf * nfp + fpn;
#pragma unroll
    for (int f = 0; f < nf; ++f) orr[f * nfp] = -Fv[f];
    if (VISC) {
      S* hr = HA + ((size_t)ep * NF + fo) * D * nf * nfp + fpn;
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int f = 0; f < nf; ++f) hr[(c * nf + f) * nfp] = HR[c][f];
    }
  }
}

template <int D, int P, typename S, bool VISC>
constexpr size_t smem_dgip_elem() {
  using H = HD<D, P>;
  return r16(sizeof(S) * (H::T * H::STATE + (VISC ? 2 : 1) * H::T * D * H::STATE + H::T * H::FACE +
                          (VISC ? H::T * D * H::FACE : 0)));
}

// ---------------------------------------------------------------------------
// k_dgip_elem: residual of every explicit element (0 on implicit ones).
// MODE 0 writes f; MODE 1 performs the ARK stage update (Sec. 4.2).
// ---------------------------------------------------------------------------
template <int D, int P, typename S, bool VISC, int MODE, bool CURV>
__global__ void __launch_bounds__(HD<D, P>::THREADS) k_dgip_elem(Mesh<S> M, Dgip<S> dp, const S* __restrict__ U,
                                                                 const S* __restrict__ FF, const S* __restrict__ HA,
                                                                 S* __restrict__ out, Stage<S> st) {
  using H = HD<D, P>;
  constexpr int n = H::n, N = H::N, nf = H::nf, nfp = H::nfp, NF = H::NF, T = H::T, STATE = H::STATE,
                FACE = H::FACE;
  constexpr Tab1<S> tb = make_tab1<S>(P);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S* us = reinterpret_cast<S*>(smem_raw);        // [T][nf][N]
  S* fs = us + T * STATE;                        // [T][D][nf][N]  flux, then divergence lines
  S* gs = fs + T * D * STATE;                    // [T][D][nf][N]  gradient (viscous)
  S* ffs = gs + (VISC ? T * D * STATE : 0);      // [T][NF][nf][nfp]
  S* has = ffs + T * FACE;                       // [T][NF][D][nf][nfp] (viscous)
  const int e0 = blockIdx.x * T;
  const int nel = min(T, M.E - e0);
  const int tid = threadIdx.x;
  const int t = tid / N, q = tid % N;
  const bool active = t < nel;
  const int e = e0 + t;
  const bool expl = active && dgip_explicit(dp, e);
  // face inputs, one thread per face point: all of its loads before its stores
  for (int i = tid; i < nel * NF * nfp; i += blockDim.x) {
    const int fp = i % nfp, tf = i / nfp;  // tf = element-in-tile * NF + face
    const bool x = dgip_explicit(dp, e0 + tf / NF);
    S v[nf];
    const S* ff = FF + ((size_t)e0 * NF + tf) * nf * nfp + fp;
#pragma unroll
    for (int f = 0; f < nf; ++f) v[f] = x ? ff[f * nfp] : S(0);
    if (VISC) {
      S hv[D][nf];
      const S* ha = HA + ((size_t)e0 * NF + tf) * D * nf * nfp + fp;
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int f = 0; f < nf; ++f) hv[c][f] = x ? ha[(c * nf + f) * nfp] : S(0);
      if (CURV) {  // contravariant components (1/J) sum_c (J dxi_a/dx_c) H_c at the face point
        const size_t fo = (size_t)e0 * NF + tf;
        const S ij = dp.iJF[fo * nfp + fp];
        S ht[D][nf];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          S ja[D];
#pragma unroll
          for (int c = 0; c < D; ++c) ja[c] = dp.JaF[((fo * D + a) * D + c) * nfp + fp];
#pragma unroll
          for (int f = 0; f < nf; ++f) {
            S v = 0;
#pragma unroll
            for (int c = 0; c < D; ++c) v += ja[c] * hv[c][f];
            ht[a][f] = ij * v;
          }
        }
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int f = 0; f < nf; ++f) hv[a][f] = ht[a][f];
      }
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int f = 0; f < nf; ++f) has[(tf * D + c) * nf * nfp + f * nfp + fp] = hv[c][f];
    }
#pragma unroll
    for (int f = 0; f < nf; ++f) ffs[(tf * nf + f) * nfp + fp] = v[f];
  }
  S Uq[nf];
  if (active) {
    const S* src = (dgip_explicit(dp, e) ? U : dp.Uim) + (size_t)e * STATE + q;
#pragma unroll
    for (int f = 0; f < nf; ++f) {
      Uq[f] = src[f * N];
      us[t * STATE + f * N + q] = Uq[f];
    }
  }
  S pre[nf];
  double pre64[nf];
  if (MODE == 1 && active) {
    const size_t off = (size_t)e * STATE + q;
    stage_prefix<nf, S>(
        st, e, [&](int f) { return st.base[off + f * N]; }, [&](int j, int f) { return st.k[j][off + f * N]; },
        [&](int f) { return st.Un[off + f * N]; }, pre, pre64);
  }
  __syncthreads();
  if (VISC) {  // broken gradient: one thread per (element, field, line) and direction
#pragma unroll
    for (int a = 0; a < D; ++a) {
      for (int i = tid; i < nel * nf * nfp; i += blockDim.x) {
        int tt, f, line;
        line_item<nf, nfp>(i, tt, f, line);
        const S* v = us + tt * STATE + f * N;
        S x[n];
#pragma unroll
        for (int m = 0; m < n; ++m) x[m] = v[H::node(m, line, a)];
        const S r = CURV ? S(1) : M.geo.rh[(e0 + tt) * D + a];  // curvilinear: reference derivative
        S* o = gs + (tt * D + a) * STATE + f * N;
#pragma unroll
        for (int k = 0; k < n; ++k) {
          S s = 0;
#pragma unroll
          for (int m = 0; m < n; ++m) s += tb.D[k][m] * x[m];
          o[H::node(k, line, a)] = r * s;
        }
      }
    }
    __syncthreads();
  }
  if (active) {
    S Fa[D][nf];
    if (CURV) {  // grad U = (1/J) sum_b Ja[b] d/dxi_b U; contravariant flux sum_c Ja[a][c] F_c
      const S* ja = M.geo.Ja + (size_t)e * D * D * N + q;
      const S ij = M.geo.iJ[(size_t)e * N + q];
      node_flux<D, S, VISC, true>(
          M.gas, Uq,
          [&](int c, int f) {
            S v = 0;
#pragma unroll
            for (int b = 0; b < D; ++b) v += ja[(b * D + c) * N] * gs[(t * D + b) * STATE + f * N + q];
            return ij * v;
          },
          [&](int a, int c) { return ja[(a * D + c) * N]; }, Fa);
    } else {
      node_flux<D, S, VISC, false>(
          M.gas, Uq, [&](int c, int f) { return gs[(t * D + c) * STATE + f * N + q]; },
          [&](int, int) { return S(0); }, Fa);
    }
    if (VISC) {  // tangential part of the adjoint-consistency term
#pragma unroll
      for (int a0 = 0; a0 < D; ++a0) {
        const S r0 = M.geo.rh[e * D + a0];
        const int fp = H::fpoint(q, a0), k0 = H::qa(q, a0);
        S Lm0 = tb.Lm[0], Lp0 = tb.Lp[0];  // L(-+1) at node k0 by selects (no runtime table index)
#pragma unroll
        for (int k = 1; k < n; ++k) {
          Lm0 = (k0 == k) ? tb.Lm[k] : Lm0;
          Lp0 = (k0 == k) ? tb.Lp[k] : Lp0;
        }
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          const S L = (CURV ? S(1) : r0) * (side ? Lp0 : Lm0);
          const S* hf = has + (t * NF + 2 * a0 + side) * D * nf * nfp + fp;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            if (a == a0) continue;
#pragma unroll
            for (int f = 0; f < nf; ++f) Fa[a][f] += L * hf[(a * nf + f) * nfp];
          }
        }
      }
    }
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int f = 0; f < nf; ++f) fs[(t * D + a) * STATE + f * N + q] = Fa[a][f];
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < D; ++a) {
    for (int i = tid; i < nel * nf * nfp; i += blockDim.x) {
      int tt, f, line;
      line_item<nf, nfp>(i, tt, f, line);
      S* v = fs + (tt * D + a) * STATE + f * N;
      S x[n];
#pragma unroll
      for (int m = 0; m < n; ++m) x[m] = v[H::node(m, line, a)];
      const S ffm = ffs[((tt * NF + 2 * a) * nf + f) * nfp + line];
      const S ffp = ffs[((tt * NF + 2 * a + 1) * nf + f) * nfp + line];
      S hm = 0, hp = 0;
      if (VISC) {
        hm = has[(((tt * NF + 2 * a) * D + a) * nf + f) * nfp + line];
        hp = has[(((tt * NF + 2 * a + 1) * D + a) * nf + f) * nfp + line];
      }
      // boxes: the 2/h_a factors here; curvilinear: the contravariant fluxes
      // and face vectors carry the metric, and 1/J comes at the node
      const S r = CURV ? S(1) : M.geo.rh[(e0 + tt) * D + a];
#pragma unroll
      for (int k = 0; k < n; ++k) {
        S s = 0;
#pragma unroll
        for (int m = 0; m < n; ++m) s += tb.Dh[k][m] * x[m];
        S val = s - tb.Lm[k] * ffm - tb.Lp[k] * ffp;
        if (VISC) val += r * (tb.dLm[k] * hm + tb.dLp[k] * hp);
        v[H::node(k, line, a)] = r * val;
      }
    }
  }
  __syncthreads();
  if (!active) return;
  S res[nf];
  const S ijq = CURV ? M.geo.iJ[(size_t)e * N + q] : S(1);
#pragma unroll
  for (int f = 0; f < nf; ++f) {
    S s = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) s += fs[(t * D + a) * STATE + f * N + q];
    res[f] = expl ? (CURV ? ijq * s : s) : S(0);
  }
  if (expl) flag_nonfinite<nf>(res, M.flags);
  if (MODE == 0) {
    S* op = out + (size_t)e * STATE + q;
#pragma unroll
    for (int f = 0; f < nf; ++f) op[f * N] = res[f];
    return;
  }
  S y[nf];
  stage_update<nf, S>(st, e, (size_t)e * STATE + q, N, res, pre, pre64, y);
}

// ===========================================================================
// Adjoint (vector-Jacobian product g = (df/dU)^T lambda), every element explicit.
// ===========================================================================

template <int D, int P, typename S, bool VISC>
constexpr size_t smem_dgip_vjp_elem() {
  using H = HD<D, P>;
  return r16(sizeof(S) * (2 * H::T * H::STATE + (VISC ? 3 : 1) * H::T * D * H::STATE));
}

// k_dgip_vjp_elem: from lambda, the cotangents of the face quantities (FFb, HAb)
// and the element-local part of g (volume flux and gradient).
template <int D, int P, typename S, bool VISC, bool CURV>
__global__ void __launch_bounds__(HD<D, P>::THREADS) k_dgip_vjp_elem(Mesh<S> M, const S* __restrict__ U,
                                                                     const S* __restrict__ lam, S* __restrict__ gpart,
                                                                     S* __restrict__ FFb, S* __restrict__ HAb) {
  using H = HD<D, P>;
  constexpr int n = H::n, N = H::N, nf = H::nf, nfp = H::nfp, NF = H::NF, T = H::T, STATE = H::STATE,
                FACE = H::FACE;
  constexpr Tab1<S> tb = make_tab1<S>(P);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S* us = reinterpret_cast<S*>(smem_raw);   // [T][nf][N]
  S* ls = us + T * STATE;                   // [T][nf][N]  lambda, later the cotangent of U
  S* fb = ls + T * STATE;                   // [T][D][nf][N]  cotangent of the volume flux
  S* gs = fb + T * D * STATE;               // [T][D][nf][N]  gradient (viscous)
  S* qb = gs + (VISC ? T * D * STATE : 0);  // [T][D][nf][N]  its cotangent (viscous)
  const int e0 = blockIdx.x * T;
  const int nel = min(T, M.E - e0);
  const int tid = threadIdx.x;
  const int t = tid / N, q = tid % N;
  const bool active = t < nel;
  const int e = e0 + t;
  S Uq[nf];
  if (active) {
    // curvilinear: f = (1/J) (...) at the node, so the cotangent entering the
    // transposed passes is lambda / J
    const S ijq = CURV ? M.geo.iJ[(size_t)e * N + q] : S(1);
#pragma unroll
    for (int f = 0; f < nf; ++f) {
      Uq[f] = U[(size_t)e * STATE + f * N + q];
      us[t * STATE + f * N + q] = Uq[f];
      ls[t * STATE + f * N + q] = ijq * lam[(size_t)e * STATE + f * N + q];
    }
  }
  __syncthreads();
  // transposed divergence / lift / normal adjoint-term lines along each direction
#pragma unroll
  for (int a = 0; a < D; ++a) {
    for (int i = tid; i < nel * nf * nfp; i += blockDim.x) {
      int tt, f, line;
      line_item<nf, nfp>(i, tt, f, line);
      const S* v = ls + tt * STATE + f * N;
      S y[n];
#pragma unroll
      for (int k = 0; k < n; ++k) y[k] = v[H::node(k, line, a)];
      const S r = CURV ? S(1) : M.geo.rh[(e0 + tt) * D + a];
      S* o = fb + (tt * D + a) * STATE + f * N;
      S sm = 0, sp = 0, dm = 0, dpp = 0;
#pragma unroll
      for (int k = 0; k < n; ++k) {
        sm += tb.Lm[k] * y[k];
        sp += tb.Lp[k] * y[k];
        dm += tb.dLm[k] * y[k];
        dpp += tb.dLp[k] * y[k];
      }
#pragma unroll
      for (int m = 0; m < n; ++m) {
        S s = 0;
#pragma unroll
        for (int k = 0; k < n; ++k) s += tb.Dh[k][m] * y[k];
        o[H::node(m, line, a)] = r * s;
      }
      const size_t fo = ((size_t)(e0 + tt) * NF + 2 * a) * nf * nfp + f * nfp + line;
      FFb[fo] = -r * sm;
      FFb[fo + nf * nfp] = -r * sp;
      if (VISC) {
        const size_t ho = (((size_t)(e0 + tt) * NF + 2 * a) * D + a) * nf * nfp + f * nfp + line;
        HAb[ho] = r * r * dm;
        HAb[ho + D * nf * nfp] = r * r * dpp;
      }
    }
  }
  if (VISC) {  // forward gradient of the element (for the viscous flux adjoint)
#pragma unroll
    for (int a = 0; a < D; ++a) {
      for (int i = tid; i < nel * nf * nfp; i += blockDim.x) {
        int tt, f, line;
        line_item<nf, nfp>(i, tt, f, line);
        const S* v = us + tt * STATE + f * N;
        S x[n];
#pragma unroll
        for (int m = 0; m < n; ++m) x[m] = v[H::node(m, line, a)];
        const S r = CURV ? S(1) : M.geo.rh[(e0 + tt) * D + a];
        S* o = gs + (tt * D + a) * STATE + f * N;
#pragma unroll
        for (int k = 0; k < n; ++k) {
          S s = 0;
#pragma unroll
          for (int m = 0; m < n; ++m) s += tb.D[k][m] * x[m];
          o[H::node(k, line, a)] = r * s;
        }
      }
    }
  }
  __syncthreads();
  if (VISC) {  // tangential adjoint-term cotangents: HAb[a0,side][a] = r_a0 sum_k L(side)[k] Fb_a(line along a0)
    constexpr int ITEMS = D * (D - 1) * nf * nfp;  // (a0, a != a0, f, fp): both sides from one line
    for (int i = tid; i < nel * ITEMS; i += blockDim.x) {
      const int fp = i % nfp;
      const int f = (i / nfp) % nf;
      const int pair = (i / (nfp * nf)) % (D * (D - 1));
      const int tt = i / ITEMS;
      with_const<0, D * (D - 1)>(pair, [&](auto PC) {
        constexpr Tab1<S> tbl = make_tab1<S>(P);
        constexpr int a0 = decltype(PC)::value / (D - 1), ai = decltype(PC)::value % (D - 1);
        constexpr int a = ai + (ai >= a0);
        const S r0 = CURV ? S(1) : M.geo.rh[(e0 + tt) * D + a0];
        const S* v = fb + (tt * D + a) * STATE + f * N;
        S sm = 0, sp = 0;
#pragma unroll
        for (int k = 0; k < n; ++k) {
          const S x = v[H::node(k, fp, a0)];
          sm += tbl.Lm[k] * x;
          sp += tbl.Lp[k] * x;
        }
        S* ho = HAb + ((((size_t)(e0 + tt) * NF + 2 * a0) * D + a) * nf + f) * nfp + fp;
        ho[0] = r0 * sm;
        ho[D * nf * nfp] = r0 * sp;
      });
    }
  }
  // pointwise flux adjoint: F = F^c - F^nu(U, Q)
  S Ub[nf];
  if (active) {
    S Fb[D][nf];
    const S* jaq = CURV ? M.geo.Ja + (size_t)e * D * D * N + q : nullptr;
    const S ijq = CURV ? M.geo.iJ[(size_t)e * N + q] : S(1);
    if (CURV) {  // cotangent of F_c from those of the contravariant fluxes sum_c Ja[a][c] F_c
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int f = 0; f < nf; ++f) {
          S v = 0;
#pragma unroll
          for (int a = 0; a < D; ++a) v += jaq[(a * D + c) * N] * fb[(t * D + a) * STATE + f * N + q];
          Fb[c][f] = v;
        }
    } else {
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int f = 0; f < nf; ++f) Fb[a][f] = fb[(t * D + a) * STATE + f * N + q];
    }
#pragma unroll
    for (int f = 0; f < nf; ++f) Ub[f] = S(0);
    conv_flux_all_vjp<D, S>(Uq, Fb, M.gas, Ub);
    if (VISC) {
      S Q[D][nf], Fn[D][nf], Qb[D][nf];
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int f = 0; f < nf; ++f) {
          if (CURV) {  // physical gradient (1/J) sum_b Ja[b][c] d/dxi_b U
            S v = 0;
#pragma unroll
            for (int b = 0; b < D; ++b) v += jaq[(b * D + c) * N] * gs[(t * D + b) * STATE + f * N + q];
            Q[c][f] = ijq * v;
          } else {
            Q[c][f] = gs[(t * D + c) * STATE + f * N + q];
          }
          Fn[c][f] = -Fb[c][f];
          Qb[c][f] = S(0);
        }
      visc_flux_all_vjp<D, S>(Uq, Q, Fn, M.gas, Ub, Qb);
#pragma unroll
      for (int b = 0; b < D; ++b)
#pragma unroll
        for (int f = 0; f < nf; ++f) {
          S v = Qb[b][f];
          if (CURV) {  // cotangent of the reference derivative d/dxi_b U
            v = 0;
#pragma unroll
            for (int c = 0; c < D; ++c) v += jaq[(b * D + c) * N] * Qb[c][f];
            v *= ijq;
          }
          qb[(t * D + b) * STATE + f * N + q] = v;
        }
    }
  }
  __syncthreads();  // everyone is done with ls (lambda) and the line reads
  if (active) {
#pragma unroll
    for (int f = 0; f < nf; ++f) ls[t * STATE + f * N + q] = Ub[f];
  }
  if (VISC) {  // gradient adjoint: Ub += r_a D_a^T Qb_a, one direction per pass
#pragma unroll
    for (int a = 0; a < D; ++a) {
      __syncthreads();
      for (int i = tid; i < nel * nf * nfp; i += blockDim.x) {
        int tt, f, line;
        line_item<nf, nfp>(i, tt, f, line);
        const S* v = qb + (tt * D + a) * STATE + f * N;
        S x[n];
#pragma unroll
        for (int m = 0; m < n; ++m) x[m] = v[H::node(m, line, a)];
        const S r = CURV ? S(1) : M.geo.rh[(e0 + tt) * D + a];
        S* o = ls + tt * STATE + f * N;
#pragma unroll
        for (int k = 0; k < n; ++k) {
          S s = 0;
#pragma unroll
          for (int m = 0; m < n; ++m) s += tb.D[m][k] * x[m];
          o[H::node(k, line, a)] += r * s;
        }
      }
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int f = 0; f < nf; ++f) gpart[(size_t)e * STATE + f * N + q] = ls[t * STATE + f * N + q];
  }
}

// Cotangents of one face point's inputs: interior faces by the hand-written
// reverse mode (dgip_face_interior_vjp); boundary faces by forward-mode
// differentiation of dgip_face_fn, one dual pass per input component.
template <int D, typename S, bool VISC, int KIND, bool AXIS = false, bool KAXIS = AXIS>
__device__ __forceinline__ void dgip_face_fn_vjp(const S (&UL)[D + 2], const S (&UR)[D + 2], const S (&nv)[D],
                                                 const Gas<S>& g, const Gas<S>& gw, S tau, bool ifL, bool ifR,
                                                 const S (&Fb)[D + 2], const S (&HLb)[D][D + 2],
                                                 const S (&HRb)[D][D + 2], S (&ULb)[D + 2], S (&URb)[D + 2]) {
  constexpr int nf = D + 2;
  if constexpr (KIND == DGIP_INTERIOR) {
#pragma unroll
    for (int f = 0; f < nf; ++f) ULb[f] = URb[f] = S(0);
    dgip_face_interior_vjp<D, S, VISC, AXIS, KAXIS>(UL, UR, nv, g, tau, ifL, ifR, Fb, HLb, HRb, ULb, URb);
    return;
  }
  using T = Dual<S, 1>;
  const Gas<T> gd = gas_as<T, S>(g), gwd = gas_as<T, S>(gw);
#pragma unroll 1
  for (int k = 0; k < nf; ++k) {
    T L[nf], R[nf], F[nf], HL[D][nf], HR[D][nf];
#pragma unroll
    for (int f = 0; f < nf; ++f) {
      L[f] = T(UL[f]);
      R[f] = T(UR[f]);
    }
    L[k].d[0] = S(1);
    dgip_face_fn<D, T, S, VISC, KIND, AXIS, KAXIS>(L, R, nv, gd, gwd, tau, ifL, ifR, F, HL, HR);
    S s = 0;
#pragma unroll
    for (int f = 0; f < nf; ++f) s += F[f].d[0] * Fb[f];
    if (VISC) {
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int f = 0; f < nf; ++f) s += HL[c][f].d[0] * HLb[c][f];
    }
    ULb[k] = s;
  }
}

// Host twin of dgip_face_fn_vjp (interior box face: unit normal, no
// interface; KAX: the axis K-products of the FP64 kernels) for the
// operation-counting work model.
template <int D, typename S, bool VISC, bool KAX = true>
inline void dgip_face_fn_vjp_host(const S (&UL)[D + 2], const S (&UR)[D + 2], const S (&nv)[D], const Gas<S>& g,
                                  S tau, const S (&Fb)[D + 2], const S (&HLb)[D][D + 2], const S (&HRb)[D][D + 2],
                                  S (&ULb)[D + 2], S (&URb)[D + 2]) {
  for (int f = 0; f < D + 2; ++f) ULb[f] = URb[f] = S(0);
  dgip_face_interior_vjp<D, S, VISC, true, KAX>(UL, UR, nv, g, tau, false, false, Fb, HLb, HRb, ULb, URb);
}

// k_dgip_vjp_face: one thread per unique face point: cotangents of both sides'
// traces (TUb) and viscous normal fluxes (Gb) from those of FF and HA.
template <int D, int P, typename S, bool VISC, bool CURV>
__global__ void __launch_bounds__(128) k_dgip_vjp_face(Mesh<S> M, Dgip<S> dp, const S* __restrict__ TU,
                                                       const S* __restrict__ FFb, const S* __restrict__ HAb,
                                                       S* __restrict__ TUb, S* __restrict__ Gb) {
  using H = HD<D, P>;
  constexpr int n = H::n, nf = H::nf, nfp = H::nfp, NF = H::NF;
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= M.nFaces * nfp) return;
  const int F = gid / nfp, fp = gid % nfp;
  const int4 rec = M.faces[F];
  const int em = rec.x, ep = rec.y;
  const int fm = rec.z & 0xff, fo = (rec.z >> 8) & 0xff, code = (rec.z >> 16) & 0xff;
  S nv[D];
  S isJ = S(1);
  if (CURV) {
    S n2 = 0;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      nv[c] = M.geo.SnF[((size_t)F * D + c) * nfp + fp];
      n2 += nv[c] * nv[c];
    }
    isJ = S(1) / sqrt(n2);
  } else {
    unit_normal<D, S>(fm, nv);
  }
  // curvilinear: HAb holds the cotangents of the contravariant vectors
  // (1/J_f) sum_c Ja_f[a][c] H_c; back to those of H_c by the transpose
  auto to_physical = [&](size_t fo_, int fp_, S (&hb)[D][D + 2]) {
    if (!CURV) return;
    const S ij = dp.iJF[fo_ * nfp + fp_];
    S out[D][D + 2];
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int f = 0; f < nf; ++f) {
        S v = 0;
#pragma unroll
        for (int a = 0; a < D; ++a) v += dp.JaF[((fo_ * D + a) * D + c) * nfp + fp_] * hb[a][f];
        out[c][f] = ij * v;
      }
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int f = 0; f < nf; ++f) hb[c][f] = out[c][f];
  };
  const Gas<S> gw = gas_no_heat(M.gas);
  const size_t ol = ((size_t)em * NF + fm) * nf * nfp + fp;
  S UL[nf], UR[nf], Fbar[nf], HLb[D][nf], HRb[D][nf], ULb[nf], URb[nf];
#pragma unroll
  for (int f = 0; f < nf; ++f) {
    UL[f] = TU[ol + f * nfp];
    Fbar[f] = FFb[ol + f * nfp];
  }
#pragma unroll
  for (int c = 0; c < D; ++c)
#pragma unroll
    for (int f = 0; f < nf; ++f) {
      HLb[c][f] = VISC ? HAb[((size_t)em * NF + fm) * D * nf * nfp + (c * nf + f) * nfp + fp] : S(0);
      HRb[c][f] = S(0);
    }
  if (VISC) to_physical((size_t)em * NF + fm, fp, HLb);
  if (ep >= 0) {
    const int fpn = orient_map<D, n>(code, fp);
    const size_t orr = ((size_t)ep * NF + fo) * nf * nfp + fpn;
#pragma unroll
    for (int f = 0; f < nf; ++f) {
      UR[f] = TU[orr + f * nfp];
      Fbar[f] -= FFb[orr + f * nfp];  // FF_R = -F
    }
    if (VISC) {
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int f = 0; f < nf; ++f) HRb[c][f] = HAb[((size_t)ep * NF + fo) * D * nf * nfp + (c * nf + f) * nfp + fpn];
      to_physical((size_t)ep * NF + fo, fpn, HRb);
    }
    const S tau = dp.tk2 * fmax(dp.il[em], dp.il[ep]) * isJ;
    dgip_face_fn_vjp<D, S, VISC, DGIP_INTERIOR, !CURV, !CURV && sizeof(S) == 8>(UL, UR, nv, M.gas, gw, tau, false, false, Fbar, HLb, HRb, ULb, URb);
#pragma unroll
    for (int f = 0; f < nf; ++f) {
      TUb[ol + f * nfp] = ULb[f];
      TUb[orr + f * nfp] = URb[f];
      if (VISC) {
        Gb[ol + f * nfp] = -S(0.5) * Fbar[f];
        Gb[orr + f * nfp] = S(0.5) * Fbar[f];
      }
    }
  } else {
    const S tau = dp.tk2 * dp.il[em] * isJ;
    if (ep == -1) {
      dgip_face_fn_vjp<D, S, VISC, DGIP_WALL, !CURV, !CURV && sizeof(S) == 8>(UL, UL, nv, M.gas, gw, tau, false, false, Fbar, HLb, HRb, ULb, URb);
    } else {
#pragma unroll
      for (int f = 0; f < nf; ++f) UR[f] = dp.Uinf[f];
      dgip_face_fn_vjp<D, S, VISC, DGIP_FARFIELD, !CURV, !CURV && sizeof(S) == 8>(UL, UR, nv, M.gas, gw, tau, false, false, Fbar, HLb, HRb, ULb,
                                                 URb);
    }
#pragma unroll
    for (int f = 0; f < nf; ++f) {
      TUb[ol + f * nfp] = ULb[f];
      if (VISC) Gb[ol + f * nfp] = -Fbar[f];
    }
  }
}

template <int D, int P, typename S, bool VISC>
constexpr size_t smem_dgip_gather() {
  using H = HD<D, P>;
  return r16(sizeof(S) * (2 * H::T * H::STATE + 2 * H::T * H::FACE + (VISC ? H::T * D * H::FACE : 0)));
}

// k_dgip_vjp_gather: g = gpart + the adjoint of the traces and of each own
// face's viscous normal flux G = F^nu(U_f, grad U_f).n.
template <int D, int P, typename S, bool VISC, bool CURV>
__global__ void __launch_bounds__(HD<D, P>::THREADS) k_dgip_vjp_gather(Mesh<S> M, Dgip<S> dp, const S* __restrict__ U,
                                                                       const S* __restrict__ TUb,
                                                                       const S* __restrict__ Gb,
                                                                       const S* __restrict__ gpart,
                                                                       S* __restrict__ g,
                                                                       const S* __restrict__ TUg,
                                                                       const S* __restrict__ QFg) {
  using H = HD<D, P>;
  constexpr int n = H::n, N = H::N, nf = H::nf, nfp = H::nfp, NF = H::NF, T = H::T, STATE = H::STATE,
                FACE = H::FACE;
  constexpr Tab1<S> tb = make_tab1<S>(P);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S* us = reinterpret_cast<S*>(smem_raw);   // [T][nf][N]   U
  S* ub = us + T * STATE;                   // [T][nf][N]   g being assembled
  S* tu = ub + T * STATE;                   // [T][NF][nf][nfp]  traces of U
  S* tub = tu + T * FACE;                   // [T][NF][nf][nfp]  trace cotangents
  S* qfb = tub + T * FACE;                  // [T][NF][D][nf][nfp]  face-gradient cotangents (viscous)
  const int e0 = blockIdx.x * T;
  const int nel = min(T, M.E - e0);
  const int tid = threadIdx.x;
  {
    const int t = tid / N, q = tid % N;
    if (t < nel) {
      const size_t off = (size_t)(e0 + t) * STATE + q;
#pragma unroll
      for (int f = 0; f < nf; ++f) {
        if (!QFg) us[t * STATE + f * N + q] = U[off + f * N];
        ub[t * STATE + f * N + q] = gpart[off + f * N];
      }
    }
  }
  for (int i = tid; i < nel * NF * nfp; i += blockDim.x) {  // one thread per face point, loads before stores
    const int fp = i % nfp, tf = i / nfp;
    S v[nf];
#pragma unroll
    for (int f = 0; f < nf; ++f) v[f] = TUb[((size_t)e0 * NF + tf) * nf * nfp + f * nfp + fp];
#pragma unroll
    for (int f = 0; f < nf; ++f) tub[(tf * nf + f) * nfp + fp] = v[f];
  }
  __syncthreads();
  if (VISC) {
    if (QFg) {  // the forward's traces and face gradients (stage checkpoints)
      constexpr int QS = NF * D * nf * nfp;
      const S* tsrc = TUg + (size_t)e0 * FACE;
      const S* qsrc = QFg + (size_t)e0 * QS;
      for (int i = tid; i < nel * FACE; i += blockDim.x) tu[i] = tsrc[i];
      for (int i = tid; i < nel * QS; i += blockDim.x) qfb[i] = qsrc[i];
      __syncthreads();
    } else {
      face_lines<D, P, S, true, CURV>(us, tu, qfb, M.geo.rh, e0, nel, nullptr);
      __syncthreads();
      face_tangential<D, P, S, CURV>(tu, qfb, M.geo.rh, e0, nel);
      __syncthreads();
    }
    const Gas<S> gw = gas_no_heat(M.gas);
    // adjoint of G at every own face point: its U_f part goes to the trace
    // cotangent (own entry), its gradient part replaces the gradient in qfb
    // (each thread reads and then overwrites only its own face point's entries)
    for (int i = tid; i < nel * NF * nfp; i += blockDim.x) {
      const int fp = i % nfp, face = (i / nfp) % NF, t = i / (nfp * NF);
      const int e = e0 + t;
      const S* tf = tu + (t * NF + face) * nf * nfp;
      S* qg = qfb + (t * NF + face) * D * nf * nfp + fp;
      S Uf[nf], Q[D][nf], nv[D], Gbar[nf], Ufb[nf], Qb[D][nf];
#pragma unroll
      for (int f = 0; f < nf; ++f) {
        Uf[f] = tf[f * nfp + fp];
        Gbar[f] = Gb[((size_t)e * NF + face) * nf * nfp + f * nfp + fp];
        Ufb[f] = S(0);
      }
      const size_t fo = (size_t)e * NF + face;
      S ij = S(1), ja[D][D];
      if (CURV) {
        ij = dp.iJF[fo * nfp + fp];
#pragma unroll
        for (int b = 0; b < D; ++b)
#pragma unroll
          for (int c = 0; c < D; ++c) ja[b][c] = dp.JaF[((fo * D + b) * D + c) * nfp + fp];
      }
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int f = 0; f < nf; ++f) {
          if (CURV) {  // physical gradient from the reference derivatives
            S v = 0;
#pragma unroll
            for (int b = 0; b < D; ++b) v += ja[b][c] * qg[(b * nf + f) * nfp];
            Q[c][f] = ij * v;
          } else {
            Q[c][f] = qg[(c * nf + f) * nfp];
          }
          Qb[c][f] = S(0);
        }
      if (CURV) {
#pragma unroll
        for (int c = 0; c < D; ++c) nv[c] = M.geo.SnE[(fo * D + c) * nfp + fp];
      } else {
        unit_normal<D, S>(face, nv);
      }
      const int nbk = M.nb[e * NF + face];
      // boxes: the axis normal selects one row of the flux
      auto vflux_vjp = [&](const S (&Us)[nf], const Gas<S>& gg, S (&Usb)[nf]) {
        if (CURV) visc_flux_normal_vjp<D, S>(Us, Q, nv, Gbar, gg, Usb, Qb);
        else visc_flux_axis_vjp_rt<D, S>(Us, Q, face >> 1, (face & 1) ? S(1) : S(-1), Gbar, gg, Usb, Qb);
      };
      if (nbk >= 0) {
        vflux_vjp(Uf, M.gas, Ufb);
      } else if (nbk == -1) {
        vflux_vjp(Uf, gw, Ufb);
      } else {
        S Ui[nf], Uib[nf];
#pragma unroll
        for (int f = 0; f < nf; ++f) {
          Ui[f] = dp.Uinf[f];
          Uib[f] = S(0);
        }
        vflux_vjp(Ui, M.gas, Uib);
      }
      S* tb_ = tub + (t * NF + face) * nf * nfp + fp;
#pragma unroll
      for (int f = 0; f < nf; ++f) tb_[f * nfp] += Ufb[f];
      if (CURV) {  // cotangents of the reference derivatives: the transposed metric
        S rb[D][nf];
#pragma unroll
        for (int b = 0; b < D; ++b)
#pragma unroll
          for (int f = 0; f < nf; ++f) {
            S v = 0;
#pragma unroll
            for (int c = 0; c < D; ++c) v += ja[b][c] * Qb[c][f];
            rb[b][f] = ij * v;
          }
#pragma unroll
        for (int b = 0; b < D; ++b)
#pragma unroll
          for (int f = 0; f < nf; ++f) qg[(b * nf + f) * nfp] = rb[b][f];
      } else {
#pragma unroll
        for (int c = 0; c < D; ++c)
#pragma unroll
          for (int f = 0; f < nf; ++f) qg[(c * nf + f) * nfp] = Qb[c][f];
      }
    }
    // tangential face derivatives, transposed: one tangential direction per
    // pass (lines of different directions share face points)
#pragma unroll
    for (int ci = 0; ci < D - 1; ++ci) {
      __syncthreads();
      face_tangential_t<D, P, S, CURV>(qfb, tub, M.geo.rh, e0, nel, ci);
    }
  }
  __syncthreads();
  // transposed traces (and the normal face-gradient part), one direction per pass
#pragma unroll
  for (int a = 0; a < D; ++a) {
    for (int i = tid; i < nel * nf * nfp; i += blockDim.x) {
      int t, f, line;
      line_item<nf, nfp>(i, t, f, line);
      const S bm = tub[(t * NF + 2 * a) * nf * nfp + f * nfp + line];
      const S bp = tub[(t * NF + 2 * a + 1) * nf * nfp + f * nfp + line];
      S qm = 0, qp = 0;
      if (VISC) {
        const S r = CURV ? S(1) : M.geo.rh[(e0 + t) * D + a];
        qm = r * qfb[((t * NF + 2 * a) * D + a) * nf * nfp + f * nfp + line];
        qp = r * qfb[((t * NF + 2 * a + 1) * D + a) * nf * nfp + f * nfp + line];
      }
      S* o = ub + t * STATE + f * N;
#pragma unroll
      for (int j = 0; j < n; ++j) {
        S v = tb.lm[j] * bm + tb.lp[j] * bp;
        if (VISC) v += tb.dlm[j] * qm + tb.dlp[j] * qp;
        o[H::node(j, line, a)] += v;
      }
    }
    __syncthreads();
  }
  {
    const int t = tid / N, q = tid % N;
    if (t < nel) {
      const size_t off = (size_t)(e0 + t) * STATE + q;
#pragma unroll
      for (int f = 0; f < nf; ++f) g[off + f * N] = ub[t * STATE + f * N + q];
    }
  }
}

}  // namespace dgx

namespace dgx {

// ---------------------------------------------------------------------------
// Launch layer of the DG-IP kernels for one (D, P, S).
// ---------------------------------------------------------------------------
struct DgipWork {       // caller-owned scratch, in the handle's precision
  void* TU;             // [E][2D][nf][nfp]  traces of U
  void* G;              // [E][2D][nf][nfp]  own-face viscous normal fluxes
  void* FF;             // [E][2D][nf][nfp]  numerical flux      (VJP: its cotangent)
  void* HA;             // [E][2D][D][nf][nfp] adjoint-term vectors (VJP: their cotangents)
  void* TUb;            // VJP: trace cotangents
  void* Gb;             // VJP: cotangents of G
  void* gpart;          // VJP: element-local part of g [E][nf][N]
  void* QF = nullptr;   // [E][2D][D][nf][nfp] face gradients: stored by the viscous trace kernel
                        // when set, read by the gather instead of recomputing them (with TU)
};

template <int D, int P, typename S>
struct DgipOps {
  using H = HD<D, P>;
  static int blocks(int E) { return (E + H::T - 1) / H::T; }
  template <bool VISC>
  static size_t smem_trace() {
    return r16(sizeof(S) * (H::T * H::STATE + H::T * H::FACE + (VISC ? H::T * D * H::FACE : 0)));
  }

  template <bool VISC, bool CURV>
  static cudaError_t trace_v(const Mesh<S>& M, const Dgip<S>& dp, const S* U, const DgipWork& w, cudaStream_t st) {
    static SmemGate done;
    auto k = k_dgip_trace<D, P, S, VISC, CURV>;
    if (const cudaError_t e = allow_smem_once(k, smem_trace<VISC>(), done)) return e;
    k<<<blocks(M.E), H::THREADS, smem_trace<VISC>(), st>>>(M, dp, U, (S*)w.TU, (S*)w.G, (S*)w.QF);
    return cudaGetLastError();
  }
  // curvilinear meshes are recognised by their face metric (dp.JaF)
  static cudaError_t trace(const void* M, const void* dp, bool visc, const void* U, const DgipWork& w,
                           cudaStream_t st) {
    const Mesh<S>& m = *(const Mesh<S>*)M;
    const Dgip<S>& p = *(const Dgip<S>*)dp;
    if (p.JaF)
      return visc ? trace_v<true, true>(m, p, (const S*)U, w, st) : trace_v<false, true>(m, p, (const S*)U, w, st);
    return visc ? trace_v<true, false>(m, p, (const S*)U, w, st) : trace_v<false, false>(m, p, (const S*)U, w, st);
  }
  static cudaError_t face(const void* M, const void* dp, bool visc, const DgipWork& w, cudaStream_t st) {
    const Mesh<S>& m = *(const Mesh<S>*)M;
    const Dgip<S>& p = *(const Dgip<S>*)dp;
    const int total = m.nFaces * H::nfp;
    if (total == 0) return cudaSuccess;
    const int nb = (total + 127) / 128;
    const S* TU = (const S*)w.TU;
    const S* G = (const S*)w.G;
    S* FF = (S*)w.FF;
    S* HA = (S*)w.HA;
    if (p.JaF) {
      if (visc) k_dgip_face<D, P, S, true, true><<<nb, 128, 0, st>>>(m, p, TU, G, FF, HA);
      else k_dgip_face<D, P, S, false, true><<<nb, 128, 0, st>>>(m, p, TU, G, FF, HA);
    } else {
      if (visc) k_dgip_face<D, P, S, true, false><<<nb, 128, 0, st>>>(m, p, TU, G, FF, HA);
      else k_dgip_face<D, P, S, false, false><<<nb, 128, 0, st>>>(m, p, TU, G, FF, HA);
    }
    return cudaGetLastError();
  }
  template <bool VISC, int MODE, bool CURV>
  static cudaError_t elem_vc(const Mesh<S>& M, const Dgip<S>& dp, const S* U, const DgipWork& w, S* out,
                             const Stage<S>& sa, cudaStream_t st) {
    static SmemGate done;
    auto k = k_dgip_elem<D, P, S, VISC, MODE, CURV>;
    constexpr size_t sm = smem_dgip_elem<D, P, S, VISC>();
    if (const cudaError_t e = allow_smem_once(k, sm, done)) return e;
    k<<<blocks(M.E), H::THREADS, sm, st>>>(M, dp, U, (const S*)w.FF, (const S*)w.HA, out, sa);
    return cudaGetLastError();
  }
  template <bool VISC, int MODE>
  static cudaError_t elem_v(const Mesh<S>& M, const Dgip<S>& dp, const S* U, const DgipWork& w, S* out,
                            const Stage<S>& sa, cudaStream_t st) {
    return dp.JaF ? elem_vc<VISC, MODE, true>(M, dp, U, w, out, sa, st)
                  : elem_vc<VISC, MODE, false>(M, dp, U, w, out, sa, st);
  }
  // stage == nullptr: write f to out; otherwise the ARK stage update
  static cudaError_t elem(const void* M, const void* dp, bool visc, const void* U, const DgipWork& w, void* out,
                          const void* stage, cudaStream_t st) {
    const Mesh<S>& m = *(const Mesh<S>*)M;
    const Dgip<S>& p = *(const Dgip<S>*)dp;
    if (stage) {
      const Stage<S>& sa = *(const Stage<S>*)stage;
      return visc ? elem_v<true, 1>(m, p, (const S*)U, w, nullptr, sa, st)
                  : elem_v<false, 1>(m, p, (const S*)U, w, nullptr, sa, st);
    }
    Stage<S> none{};
    return visc ? elem_v<true, 0>(m, p, (const S*)U, w, (S*)out, none, st)
                : elem_v<false, 0>(m, p, (const S*)U, w, (S*)out, none, st);
  }
  template <bool VISC, bool CURV>
  static cudaError_t vjp_elem_v(const Mesh<S>& M, const S* U, const S* lam, const DgipWork& w, cudaStream_t st) {
    static SmemGate done;
    auto k = k_dgip_vjp_elem<D, P, S, VISC, CURV>;
    constexpr size_t sm = smem_dgip_vjp_elem<D, P, S, VISC>();
    if (const cudaError_t e = allow_smem_once(k, sm, done)) return e;
    k<<<blocks(M.E), H::THREADS, sm, st>>>(M, U, lam, (S*)w.gpart, (S*)w.FF, (S*)w.HA);
    return cudaGetLastError();
  }
  // the element adjoint reads the metric from the mesh (geo.Ja set on curved meshes)
  static cudaError_t vjp_elem(const void* M, bool visc, const void* U, const void* lam, const DgipWork& w,
                              cudaStream_t st) {
    const Mesh<S>& m = *(const Mesh<S>*)M;
    if (m.geo.Ja)
      return visc ? vjp_elem_v<true, true>(m, (const S*)U, (const S*)lam, w, st)
                  : vjp_elem_v<false, true>(m, (const S*)U, (const S*)lam, w, st);
    return visc ? vjp_elem_v<true, false>(m, (const S*)U, (const S*)lam, w, st)
                : vjp_elem_v<false, false>(m, (const S*)U, (const S*)lam, w, st);
  }
  static cudaError_t vjp_face(const void* M, const void* dp, bool visc, const DgipWork& w, cudaStream_t st) {
    const Mesh<S>& m = *(const Mesh<S>*)M;
    const Dgip<S>& p = *(const Dgip<S>*)dp;
    const int total = m.nFaces * H::nfp;
    if (total == 0) return cudaSuccess;
    const int nb = (total + 127) / 128;
    const S* TU = (const S*)w.TU;
    const S* FFb = (const S*)w.FF;
    const S* HAb = (const S*)w.HA;
    if (p.JaF) {
      if (visc) k_dgip_vjp_face<D, P, S, true, true><<<nb, 128, 0, st>>>(m, p, TU, FFb, HAb, (S*)w.TUb, (S*)w.Gb);
      else k_dgip_vjp_face<D, P, S, false, true><<<nb, 128, 0, st>>>(m, p, TU, FFb, HAb, (S*)w.TUb, (S*)w.Gb);
    } else {
      if (visc) k_dgip_vjp_face<D, P, S, true, false><<<nb, 128, 0, st>>>(m, p, TU, FFb, HAb, (S*)w.TUb, (S*)w.Gb);
      else k_dgip_vjp_face<D, P, S, false, false><<<nb, 128, 0, st>>>(m, p, TU, FFb, HAb, (S*)w.TUb, (S*)w.Gb);
    }
    return cudaGetLastError();
  }
  template <bool VISC, bool CURV>
  static cudaError_t gather_v(const Mesh<S>& M, const Dgip<S>& dp, const S* U, const DgipWork& w, S* g,
                              cudaStream_t st) {
    static SmemGate done;
    auto k = k_dgip_vjp_gather<D, P, S, VISC, CURV>;
    constexpr size_t sm = smem_dgip_gather<D, P, S, VISC>();
    if (const cudaError_t e = allow_smem_once(k, sm, done)) return e;
    k<<<blocks(M.E), H::THREADS, sm, st>>>(M, dp, U, (const S*)w.TUb, (const S*)w.Gb, (const S*)w.gpart, g,
                                           (const S*)w.TU, (const S*)w.QF);
    return cudaGetLastError();
  }
  static cudaError_t vjp_gather(const void* M, const void* dp, bool visc, const void* U, const DgipWork& w, void* g,
                                cudaStream_t st) {
    const Mesh<S>& m = *(const Mesh<S>*)M;
    const Dgip<S>& p = *(const Dgip<S>*)dp;
    if (p.JaF)
      return visc ? gather_v<true, true>(m, p, (const S*)U, w, (S*)g, st)
                  : gather_v<false, true>(m, p, (const S*)U, w, (S*)g, st);
    return visc ? gather_v<true, false>(m, p, (const S*)U, w, (S*)g, st)
                : gather_v<false, false>(m, p, (const S*)U, w, (S*)g, st);
  }
};

// Linear combinations of state vectors for the composed ARK adjoint:
// out = (S)(c_lam lam + sum_j c_j in_j) (sums in FP64), and/or
// acc64 += sum_j c_j in_j in FP64.
template <typename S>
struct LinComb {
  size_t n;
  const double* lam;   // FP64 input (or nullptr)
  double c_lam;
  int m;
  const S* in[MAXSTAGES];
  double c[MAXSTAGES];
  S* out;              // or nullptr
  double* acc64;       // or nullptr
};

template <typename S>
__global__ void __launch_bounds__(256) k_lincomb(LinComb<S> a) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (size_t)gridDim.x * blockDim.x) {
    double v = a.lam ? a.c_lam * a.lam[i] : 0.0;
    for (int j = 0; j < a.m; ++j) v += a.c[j] * (double)a.in[j][i];
    if (a.out) a.out[i] = (S)v;
    if (a.acc64) a.acc64[i] += v;
  }
}

template <typename S>
inline cudaError_t lincomb(const LinComb<S>& a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  const size_t blocks = (a.n + 255) / 256;
  k_lincomb<S><<<(unsigned)(blocks < 148 * 16 ? blocks : 148 * 16), 256, 0, st>>>(a);
  return cudaGetLastError();
}

struct DgipTable {
  cudaError_t (*trace)(const void* M, const void* dp, bool visc, const void* U, const DgipWork& w, cudaStream_t st);
  cudaError_t (*face)(const void* M, const void* dp, bool visc, const DgipWork& w, cudaStream_t st);
  cudaError_t (*elem)(const void* M, const void* dp, bool visc, const void* U, const DgipWork& w, void* out,
                      const void* stage, cudaStream_t st);
  cudaError_t (*vjp_elem)(const void* M, bool visc, const void* U, const void* lam, const DgipWork& w,
                          cudaStream_t st);
  cudaError_t (*vjp_face)(const void* M, const void* dp, bool visc, const DgipWork& w, cudaStream_t st);
  cudaError_t (*vjp_gather)(const void* M, const void* dp, bool visc, const void* U, const DgipWork& w, void* g,
                            cudaStream_t st);
};

template <int D, int P, typename S>
const DgipTable* dgip_table() {
  using O = DgipOps<D, P, S>;
  static const DgipTable t = {&O::trace, &O::face, &O::elem, &O::vjp_elem, &O::vjp_face, &O::vjp_gather};
  return &t;
}

}  // namespace dgx
