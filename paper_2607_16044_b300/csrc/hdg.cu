// Element-local blocks of the implicit region's HDG-IP Newton system
// (Sec. 3.4 element and facet forms, Sec. 4.3 static condensation), FP64,
// 2D box and curved meshes.
//
// k_hdg_jacobian: one thread per (element, group of KC input columns).  The
// element's residual R_T (the HDG-IP element form tested with each nodal
// basis function) and facet residual h_T (the transmission form tested with
// each facet basis function) are evaluated serially by that thread with
// forward-mode dual numbers carrying KC tangents, one seeded on each of its
// columns (element or facet DOFs; the primal part is computed once for all
// KC), which yields columns j of
//   K = M + gamma dR/dU,  C = gamma dR/dUhat,  D = dh/dU,  A33_T = dh/dUhat.
// With unit normals on boxes (r_a = 2/h_a, J = prod h_a/2, area factor
// J r_a0 on a face normal to a0) the element form is written like the DG-IP
// element kernel's strong form f, R = -M f, with, per own face point,
//   FF = Fhat*_n(U_f, Uhat) - F^nu(Uhat, grad U_f).n + tau F^nu(Uhat; (U_f - Uhat) (x) n).n,
//   H  = F^nu(Uhat; (U_f - Uhat) (x) n)      (weight 1; walls with kappa = 0),
//   Fhat*_n = F_n(Uhat) + A_n^+(Uhat)(U_f - Uhat)  (= A^+ U_f + A^- Uhat),
// tau = 10 (k+1)^2 / l of the element, and the facet residual (face weight w_f,
// area factor s_J) -w_f s_J FF inside, w_f s_J (Uhat - U_w(U_f)) on walls,
// w_f s_J (A^+(Uhat)(Uhat - U_f) - A^-(Uhat)(Uhat - U_inf)) on farfield faces.
//
// k_hdg_condense_lu: one CTA per element: LU factorisation of K with partial
// pivoting in shared memory, the columns of C solved in shared-memory panels
// (K^{-1} C), then S_T = A33_T - D K^{-1} C.  k_hdg_condense (Gauss-Jordan
// elimination of [K | C] in global memory) serves where K does not fit in
// shared memory.
#include <cuda_runtime.h>

#include "dgip_physics.cuh"
#include "hdg.h"
#include "kernels.cuh"

namespace dgx {
namespace {

// columns of the Newton blocks one thread differentiates at once (tangents
// of its dual numbers): the primal evaluation is shared by that many columns
constexpr int HDG_COLUMNS_PER_THREAD = 8;

template <typename T, typename S, int D>
__device__ __forceinline__ void split_apply(const T (&Us)[D + 2], const T (&dU)[D + 2], const S (&nh)[D],
                                            const Gas<T>& g, int sign, T (&out)[D + 2]) {
  // A_n^+ dU (sign > 0), A_n^- dU (sign < 0) or A_n dU (sign == 0) at the state Us
  constexpr int nf = D + 2;
  const Waves<D, T, S> w(Us, dU, nh, g);
  T rm[nf], rp[nf];
  w.r(-1, nh, rm);
  w.r(1, nh, rp);
  // positive / negative part; at x = 0 exactly the value 0 with the mean of
  // the one-sided derivatives (x / 2)
  auto part = [&](const T& x) {
    if (sign == 0) return x;
    if (sign > 0) return x > T(0) ? x : (x < T(0) ? T(0) : T(0.5) * x);
    return x < T(0) ? x : (x > T(0) ? T(0) : T(0.5) * x);
  };
  const T l0 = part(w.un), lm = part(w.un - w.c), lp = part(w.un + w.c);
#pragma unroll
  for (int f = 0; f < nf; ++f) out[f] = l0 * dU[f] + (lm - l0) * w.am * rm[f] + (lp - l0) * w.ap * rp[f];
}

// CURV: the element's metric terms come from the arrays of HdgArgs (curved
// or general affine elements); FF is then the area-weighted flux through the
// own area normal Sn (|Sn| = s_J), HA the contravariant adjoint-consistency
// vector (1/J_f) sum_c (J dxi_a/dx_c)_f H_c of H = F^nu(Uhat; (U_f - Uhat) (x) Sn),
// and R = -w_q (sum_a Dh_a(Ja_a . (F - F^nu) + tangential H parts) - lift(FF)
// + normal H parts).  On boxes both reduce to the unit-normal forms above.
// FACET: the tangents of a column group seeded on facet DOFs alone (the bits
// of fmask: the faces holding them).  The forms depend on Uhat only through
// the face quantities of the face the DOF sits on, so only those faces are
// evaluated (the others' FF, HA and h have zero tangents) and the element
// residual takes no volume flux (its tangent is zero): what remains is the
// lift of FF and the adjoint-consistency terms of HA.  The values are then
// not the forms' values (they come from the full evaluation).
template <int P, bool CURV, bool FACET, typename T>
__device__ void hdg_forms(const HdgArgs& a, int e, const T* u, const T* uh, T* R, T* hres, int fmask = 0xf) {
  constexpr int D = 2, n = P + 1, N = n * n, nf = 4, nfp = n, NF = 4;
  using H = Sh<D, P, 1>;
  constexpr Tab1<double> tb = make_tab1<double>(P);
  double rh[2] = {0.0, 0.0}, J = 0.0;
  if constexpr (!CURV) {
    rh[0] = a.rh[e * 2];
    rh[1] = a.rh[e * 2 + 1];
    J = 1.0 / (rh[0] * rh[1]);  // prod(h_a / 2) = 1 / prod(r_a)
  }
  const double tau = a.tk2 * a.il[e];
  const Gas<T> g = gas_as<T, double>(a.gas);
  Gas<double> gw0 = a.gas;
  gw0.kcv = 0.0;
  const Gas<T> gw = gas_as<T, double>(gw0);
  // traces of U
  T TU[NF][nf][nfp];
  for (int face = 0; face < NF; ++face)
    for (int f = 0; f < nf; ++f)
      for (int fp = 0; fp < nfp; ++fp) {
        T s = T(0);
        for (int m = 0; m < n; ++m) s += T((face & 1) ? tb.lp[m] : tb.lm[m]) * u[f * N + H::node(m, fp, face >> 1)];
        TU[face][f][fp] = s;
      }
  // face quantities
  T FF[NF][nf][nfp], HA[NF][D][nf][nfp];
  for (int face = 0; face < NF; ++face) {
    const int a0 = face >> 1, side = face & 1, c = 1 - a0;
    const int kind = a.nb[e * NF + face];
    if (FACET && !((fmask >> face) & 1)) {  // no seeded DOF on this face: zero tangents
      for (int f = 0; f < nf; ++f)
        for (int fp = 0; fp < nfp; ++fp) {
          FF[face][f][fp] = T(0);
          for (int aa = 0; aa < D; ++aa) HA[face][aa][f][fp] = T(0);
          hres[(face * nf + f) * nfp + fp] = T(0);
        }
      continue;
    }
    for (int fp = 0; fp < nfp; ++fp) {
      double nv[D] = {0.0, 0.0}, sJ, iJf = 0.0, JF[D][D] = {};
      if constexpr (CURV) {
        for (int cc = 0; cc < D; ++cc) nv[cc] = a.SnE[(((size_t)e * NF + face) * D + cc) * nfp + fp];
        sJ = sqrt(nv[0] * nv[0] + nv[1] * nv[1]);
        iJf = a.iJF[((size_t)e * NF + face) * nfp + fp];
        for (int aa = 0; aa < D; ++aa)
          for (int cc = 0; cc < D; ++cc) JF[aa][cc] = a.JaF[((((size_t)e * NF + face) * D + aa) * D + cc) * nfp + fp];
      } else {
        nv[a0] = side ? 1.0 : -1.0;
        sJ = J * rh[a0];
      }
      T Uf[nf], Uhf[nf], Q[D][nf], dl[nf];
      for (int f = 0; f < nf; ++f) {
        Uf[f] = TU[face][f][fp];
        Uhf[f] = uh[(face * nf + f) * nfp + fp];
        dl[f] = Uf[f] - Uhf[f];
        T sn = T(0), st = T(0);
        for (int j = 0; j < n; ++j) sn += T(side ? tb.dlp[j] : tb.dlm[j]) * u[f * N + H::node(j, fp, a0)];
        for (int m = 0; m < n; ++m) st += T(tb.D[fp][m]) * TU[face][f][m];
        if constexpr (CURV) {  // grad U = (1/J_f) sum_b (J dxi_b/dx)_f d_b U
          for (int cc = 0; cc < D; ++cc) Q[cc][f] = T(iJf) * (T(JF[a0][cc]) * sn + T(JF[c][cc]) * st);
        } else {
          Q[a0][f] = T(rh[a0]) * sn;
          Q[c][f] = T(rh[c]) * st;
        }
      }
      // the characteristic split takes the unit normal: A^+-(Sn) = s_J A^+-(n)
      double nu[D];
      for (int cc = 0; cc < D; ++cc) nu[cc] = CURV ? nv[cc] / sJ : nv[cc];
      const T sa = T(CURV ? sJ : 1.0);
      const Gas<T>& gk = (kind == -1) ? gw : g;
      T Fn[nf], Ad[nf], Vg[D][nf], Kd[D][nf], Qd[D][nf];
      conv_flux_normal<D, T, double>(Uhf, nv, g, Fn);
      split_apply<T, double, D>(Uhf, dl, nu, g, 1, Ad);
      for (int f = 0; f < nf; ++f) Ad[f] *= sa;
      visc_flux_all<D, T>(Uhf, Q, gk, Vg);
      for (int cc = 0; cc < D; ++cc)
        for (int f = 0; f < nf; ++f) Qd[cc][f] = T(nv[cc]) * dl[f];
      visc_flux_all<D, T>(Uhf, Qd, gk, Kd);
      const double tpen = CURV ? tau / sJ : tau;
      T ff[nf];
      for (int f = 0; f < nf; ++f) {
        T vn = T(0), kn = T(0);
        for (int cc = 0; cc < D; ++cc) {
          vn += Vg[cc][f] * T(nv[cc]);
          kn += Kd[cc][f] * T(nv[cc]);
        }
        ff[f] = Fn[f] + Ad[f] - vn + T(tpen) * kn;
        FF[face][f][fp] = ff[f];
        for (int aa = 0; aa < D; ++aa) {
          if constexpr (CURV) {
            T ht = T(0);
            for (int cc = 0; cc < D; ++cc) ht += T(JF[aa][cc]) * Kd[cc][f];
            HA[face][aa][f][fp] = T(iJf) * ht;
          } else {
            HA[face][aa][f][fp] = Kd[aa][f];
          }
        }
      }
      // facet residual
      const double wf = CURV ? a.w[fp] : a.w[fp] * sJ;
      T hv[nf];
      if (kind >= 0) {
        for (int f = 0; f < nf; ++f) hv[f] = -ff[f];
      } else if (kind == -1) {
        T Uw[nf];
        wall_state<D, T>(Uf, Uw);
        for (int f = 0; f < nf; ++f) hv[f] = (CURV ? T(sJ) : T(1)) * (Uhf[f] - Uw[f]);
      } else {
        T d1[nf], d2[nf], p1[nf], m2[nf];
        for (int f = 0; f < nf; ++f) {
          d1[f] = Uhf[f] - Uf[f];
          d2[f] = Uhf[f] - T(a.Uinf[f]);
        }
        split_apply<T, double, D>(Uhf, d1, nu, g, 1, p1);
        split_apply<T, double, D>(Uhf, d2, nu, g, -1, m2);
        for (int f = 0; f < nf; ++f) hv[f] = sa * (p1[f] - m2[f]);
      }
      for (int f = 0; f < nf; ++f) hres[(face * nf + f) * nfp + fp] = T(wf) * hv[f];
    }
  }
  // element residual: the DG-IP strong form with these face quantities, R = -M f
  T Fa[D][nf][N];
  if constexpr (FACET) {  // the volume flux has zero tangent: only the tangential H parts
    for (int q = 0; q < N; ++q)
      for (int aa = 0; aa < D; ++aa)
        for (int f = 0; f < nf; ++f) {
          const int a0 = 1 - aa;
          const int fp = H::fpoint(q, a0), k0 = H::qa(q, a0);
          const double r0 = CURV ? 1.0 : rh[a0];
          Fa[aa][f][q] = T(r0 * tb.Lm[k0]) * HA[2 * a0][aa][f][fp] + T(r0 * tb.Lp[k0]) * HA[2 * a0 + 1][aa][f][fp];
        }
  } else {
  T Q[D][nf][N];
  for (int cc = 0; cc < D; ++cc)
    for (int f = 0; f < nf; ++f)
      for (int q = 0; q < N; ++q) {
        const int line = H::fpoint(q, cc), k = H::qa(q, cc);
        T s = T(0);
        for (int m = 0; m < n; ++m) s += T(tb.D[k][m]) * u[f * N + H::node(m, line, cc)];
        Q[cc][f][q] = CURV ? s : T(rh[cc]) * s;  // curved: reference derivatives, mapped below
      }
  for (int q = 0; q < N; ++q) {
    double Ja[D][D] = {}, iJ = 0.0;
    if constexpr (CURV) {
      iJ = a.iJ[(size_t)e * N + q];
      for (int aa = 0; aa < D; ++aa)
        for (int cc = 0; cc < D; ++cc) Ja[aa][cc] = a.Ja[(((size_t)e * D + aa) * D + cc) * N + q];
    }
    T Uq[nf], Qq[D][nf], F[D][nf], V[D][nf];
    for (int f = 0; f < nf; ++f) {
      Uq[f] = u[f * N + q];
      if constexpr (CURV) {
        for (int cc = 0; cc < D; ++cc) Qq[cc][f] = T(iJ) * (T(Ja[0][cc]) * Q[0][f][q] + T(Ja[1][cc]) * Q[1][f][q]);
      } else {
        for (int cc = 0; cc < D; ++cc) Qq[cc][f] = Q[cc][f][q];
      }
    }
    conv_flux_all<D, T>(Uq, g, F);
    visc_flux_all<D, T>(Uq, Qq, g, V);
    for (int aa = 0; aa < D; ++aa)
      for (int f = 0; f < nf; ++f) {
        T x;
        if constexpr (CURV) {
          x = T(0);
          for (int cc = 0; cc < D; ++cc) x += T(Ja[aa][cc]) * (F[cc][f] - V[cc][f]);
        } else {
          x = F[aa][f] - V[aa][f];
        }
        const int a0 = 1 - aa;  // the other direction's faces carry the tangential part
        const int fp = H::fpoint(q, a0), k0 = H::qa(q, a0);
        const double r0 = CURV ? 1.0 : rh[a0];
        x += T(r0 * tb.Lm[k0]) * HA[2 * a0][aa][f][fp] + T(r0 * tb.Lp[k0]) * HA[2 * a0 + 1][aa][f][fp];
        Fa[aa][f][q] = x;
      }
  }
  }
  for (int q = 0; q < N; ++q)
    for (int f = 0; f < nf; ++f) {
      T s = T(0);
      for (int aa = 0; aa < D; ++aa) {
        const int line = H::fpoint(q, aa), k = H::qa(q, aa);
        const double ra = CURV ? 1.0 : rh[aa];
        T v = T(0);
        for (int m = 0; m < n; ++m) v += T(tb.Dh[k][m]) * Fa[aa][f][H::node(m, line, aa)];
        v -= T(tb.Lm[k]) * FF[2 * aa][f][line] + T(tb.Lp[k]) * FF[2 * aa + 1][f][line];
        v += T(ra) * (T(tb.dLm[k]) * HA[2 * aa][aa][f][line] + T(tb.dLp[k]) * HA[2 * aa + 1][aa][f][line]);
        s += T(ra) * v;
      }
      const double wq = a.w[q % n] * a.w[q / n];
      R[f * N + q] = -T(CURV ? wq : wq * J) * s;
    }
}

// Column groups of KC columns: the first NGE cover the element DOFs (the
// last of them may reach into the facet DOFs), the remaining NGF hold facet
// DOFs only.  One launch takes both sets, the element groups in its first
// EB blocks and the facet groups after them, so that a warp never mixes the
// full evaluation with the facet-only one.
template <int P, int KC>
struct HdgGroups {
  static constexpr int n = P + 1, NU = 4 * n * n, NH = 16 * n, NCOL = NU + NH;
  static constexpr int NGE = (NU + KC - 1) / KC;
  static constexpr int NGF = (NCOL - NGE * KC + KC - 1) / KC;
};

template <int P, int KC, bool CURV>
__global__ void __launch_bounds__(128) k_hdg_jacobian(HdgArgs a, const double* __restrict__ U,
                                                      const double* __restrict__ Uh, double gamma, double* K,
                                                      double* C, double* Dm, double* A33, double* Rv, double* hv,
                                                      int EB) {
  using G = HdgGroups<P, KC>;
  constexpr int n = P + 1, N = n * n, nf = 4, NU = nf * N, NH = 4 * nf * n;
  constexpr int NCOL = NU + NH;
  using T = Dual<double, KC>;
  const bool facet = (int)blockIdx.x >= EB;  // uniform over the block
  const int NG = facet ? G::NGF : G::NGE;    // column groups per element in this part
  const long long gid = (long long)(facet ? blockIdx.x - EB : blockIdx.x) * blockDim.x + threadIdx.x;
  if (gid >= (long long)a.E * NG) return;
  const int e = (int)(gid / NG), c0 = (facet ? G::NGE * KC : 0) + (int)(gid % NG) * KC;
  T u[NU], uh[NH], R[NU], h[NH];
  for (int i = 0; i < NU; ++i) u[i] = T(U[(size_t)e * NU + i]);
  for (int i = 0; i < NH; ++i) uh[i] = T(Uh[(size_t)e * NH + i]);
#pragma unroll
  for (int k = 0; k < KC; ++k) {
    const int col = c0 + k;
    if (col < NU) u[col].d[k] = 1.0;
    else if (col < NCOL) uh[col - NU].d[k] = 1.0;
  }
  if (facet) {  // facet columns only: the faces that hold them
    int fmask = 0;
    for (int k = 0; k < KC; ++k)
      if (c0 + k < NCOL) fmask |= 1 << ((c0 + k - NU) / (nf * n));
    hdg_forms<P, CURV, true, T>(a, e, u, uh, R, h, fmask);
  } else {
    hdg_forms<P, CURV, false, T>(a, e, u, uh, R, h);
  }
  if (c0 == 0 && Rv) {  // the forms' values (the value part of any group)
    for (int i = 0; i < NU; ++i) Rv[(size_t)e * NU + i] = R[i].v;
    for (int k = 0; k < NH; ++k) hv[(size_t)e * NH + k] = h[k].v;
  }
  const double J = CURV ? 0.0 : 1.0 / (a.rh[e * 2] * a.rh[e * 2 + 1]);
#pragma unroll
  for (int k = 0; k < KC; ++k) {
    const int col = c0 + k;
    if (col < NU) {
      for (int i = 0; i < NU; ++i) {
        const int q = i % N;
        const double Jq = CURV ? 1.0 / a.iJ[(size_t)e * N + q] : J;
        const double m = (i == col) ? a.w[q % n] * a.w[q / n] * Jq : 0.0;
        K[((size_t)e * NU + i) * NU + col] = m + gamma * R[i].d[k];
      }
      for (int r = 0; r < NH; ++r) Dm[((size_t)e * NH + r) * NU + col] = h[r].d[k];
    } else if (col < NCOL) {
      const int j = col - NU;
      for (int i = 0; i < NU; ++i) C[((size_t)e * NU + i) * NH + j] = gamma * R[i].d[k];
      for (int r = 0; r < NH; ++r) A33[((size_t)e * NH + r) * NH + j] = h[r].d[k];
    }
  }
}

// Gauss-Jordan with partial pivoting of [W | X] (W = K copied into the
// workspace, X = C copied into KinvC), then S = A33 - D X.
__global__ void __launch_bounds__(256) k_hdg_condense(int E, int NU, int NH, const double* __restrict__ K,
                                                      const double* __restrict__ C, const double* __restrict__ Dm,
                                                      const double* __restrict__ A33, double* __restrict__ X,
                                                      double* __restrict__ S, double* __restrict__ Wbuf) {
  const int e = blockIdx.x;
  if (e >= E) return;
  double* W = Wbuf + (size_t)e * NU * NU;
  double* Xe = X + (size_t)e * NU * NH;
  const double* Ke = K + (size_t)e * NU * NU;
  const double* Ce = C + (size_t)e * NU * NH;
  for (int i = threadIdx.x; i < NU * NU; i += blockDim.x) W[i] = Ke[i];
  for (int i = threadIdx.x; i < NU * NH; i += blockDim.x) Xe[i] = Ce[i];
  __shared__ double sval[256];
  __shared__ int sidx[256];
  __shared__ double piv_inv;
  __syncthreads();
  for (int k = 0; k < NU; ++k) {
    // pivot: the largest |W[i][k]| over i >= k
    double best = -1.0;
    int bi = k;
    for (int i = k + threadIdx.x; i < NU; i += blockDim.x) {
      const double v = fabs(W[(size_t)i * NU + k]);
      if (v > best) {
        best = v;
        bi = i;
      }
    }
    sval[threadIdx.x] = best;
    sidx[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        const double o = sval[threadIdx.x + s];
        const int oi = sidx[threadIdx.x + s];
        if (o > sval[threadIdx.x] || (o == sval[threadIdx.x] && oi < sidx[threadIdx.x])) {
          sval[threadIdx.x] = o;
          sidx[threadIdx.x] = oi;
        }
      }
      __syncthreads();
    }
    const int p = sidx[0];
    if (p != k) {  // swap rows k and p of W (columns >= k) and X
      for (int j = k + threadIdx.x; j < NU; j += blockDim.x) {
        const double t = W[(size_t)k * NU + j];
        W[(size_t)k * NU + j] = W[(size_t)p * NU + j];
        W[(size_t)p * NU + j] = t;
      }
      for (int j = threadIdx.x; j < NH; j += blockDim.x) {
        const double t = Xe[(size_t)k * NH + j];
        Xe[(size_t)k * NH + j] = Xe[(size_t)p * NH + j];
        Xe[(size_t)p * NH + j] = t;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) piv_inv = 1.0 / W[(size_t)k * NU + k];
    __syncthreads();
    const double pinv = piv_inv;
    for (int j = k + threadIdx.x; j < NU; j += blockDim.x) W[(size_t)k * NU + j] *= pinv;
    for (int j = threadIdx.x; j < NH; j += blockDim.x) Xe[(size_t)k * NH + j] *= pinv;
    __syncthreads();
    // eliminate column k from every other row
    const int cols = (NU - k - 1) + NH;
    for (int t = threadIdx.x; t < (NU - 1) * cols; t += blockDim.x) {
      int i = t / cols;
      if (i >= k) ++i;  // skip the pivot row
      const int jj = t % cols;
      const double f = W[(size_t)i * NU + k];
      if (jj < NU - k - 1) {
        const int j = k + 1 + jj;
        W[(size_t)i * NU + j] -= f * W[(size_t)k * NU + j];
      } else {
        const int j = jj - (NU - k - 1);
        Xe[(size_t)i * NH + j] -= f * Xe[(size_t)k * NH + j];
      }
    }
    __syncthreads();
  }
  // S = A33 - D X
  const double* De = Dm + (size_t)e * NH * NU;
  const double* Ae = A33 + (size_t)e * NH * NH;
  double* Se = S + (size_t)e * NH * NH;
  for (int t = threadIdx.x; t < NH * NH; t += blockDim.x) {
    const int r = t / NH, c = t % NH;
    double s = Ae[t];
    for (int m = 0; m < NU; ++m) s -= De[(size_t)r * NU + m] * Xe[(size_t)m * NH + c];
    Se[t] = s;
  }
}

// The same blocks by LU factorisation in shared memory: K (nu x nu) is
// copied into shared memory and factorised in place with partial pivoting
// (full-row swaps, unit lower triangle below the diagonal); the columns of C
// are then solved in panels of pc columns held in shared memory (the row
// swaps, forward substitution with L, back substitution with U) and stored as
// K^{-1} C; S = A33 - D K^{-1} C follows from global memory (the CTA's own,
// L2-resident writes).  One CTA per element; the FP64 arithmetic works on
// shared memory only, where the global Gauss-Jordan form streams its
// nu x (nu + nh) working set through L2 at every elimination step.
template <int NT>
__device__ __forceinline__ void argmax_abs(double v, int i, double* rv, int* ri, double& best, int& bi) {
  // block-wide max of |v| (ties: the smaller index); every thread gets the result
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_down_sync(0xffffffffu, v, o);
    const int oi = __shfl_down_sync(0xffffffffu, i, o);
    if (ov > v || (ov == v && oi < i)) {
      v = ov;
      i = oi;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    rv[warp] = v;
    ri[warp] = i;
  }
  __syncthreads();
  if (warp == 0) {
    constexpr int NW = NT / 32;
    v = lane < NW ? rv[lane] : -1.0;
    i = lane < NW ? ri[lane] : 0x7fffffff;
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, v, o);
      const int oi = __shfl_down_sync(0xffffffffu, i, o);
      if (ov > v || (ov == v && oi < i)) {
        v = ov;
        i = oi;
      }
    }
    if (lane == 0) {
      rv[0] = v;
      ri[0] = i;
    }
  }
  __syncthreads();
  best = rv[0];
  bi = ri[0];
}

template <int NT>
__global__ void __launch_bounds__(NT) k_hdg_condense_lu(int E, int NU, int NH, int PC,
                                                                    const double* __restrict__ K,
                                                                    const double* __restrict__ C,
                                                                    const double* __restrict__ Dm,
                                                                    const double* __restrict__ A33,
                                                                    double* __restrict__ X, double* __restrict__ S) {
  extern __shared__ __align__(16) double sm_lu[];
  double* W = sm_lu;                      // [NU][NU]
  double* Pn = W + (size_t)NU * NU;       // [NU][PC] panel of C, then of K^{-1} C
  int* piv = (int*)(Pn + (size_t)NU * PC);
  __shared__ double rv[NT / 32];
  __shared__ int ri[NT / 32];
  constexpr int NWARP = NT / 32;
  const int e = blockIdx.x;
  if (e >= E) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const double* Ke = K + (size_t)e * NU * NU;
  const double* Ce = C + (size_t)e * NU * NH;
  double* Xe = X + (size_t)e * NU * NH;
  for (int i = tid; i < NU * NU; i += NT) W[i] = Ke[i];
  __syncthreads();
  for (int k = 0; k < NU; ++k) {
    double best = -1.0;
    int bi = k;
    for (int i = k + tid; i < NU; i += NT) {
      const double v = fabs(W[(size_t)i * NU + k]);
      if (v > best) {
        best = v;
        bi = i;
      }
    }
    argmax_abs<NT>(best, bi, rv, ri, best, bi);
    const int p = bi;
    if (tid == 0) piv[k] = p;
    if (p != k)
      for (int j = tid; j < NU; j += NT) {
        const double t = W[(size_t)k * NU + j];
        W[(size_t)k * NU + j] = W[(size_t)p * NU + j];
        W[(size_t)p * NU + j] = t;
      }
    __syncthreads();
    const double inv = 1.0 / W[(size_t)k * NU + k];
    for (int i = k + 1 + tid; i < NU; i += NT) W[(size_t)i * NU + k] *= inv;
    __syncthreads();
    // trailing update: rows over warps, columns over lanes (no index division)
    for (int i = k + 1 + warp; i < NU; i += NWARP) {
      const double l = W[(size_t)i * NU + k];
      for (int j = k + 1 + lane; j < NU; j += 32) W[(size_t)i * NU + j] -= l * W[(size_t)k * NU + j];
    }
    __syncthreads();
  }
  for (int c0 = 0; c0 < NH; c0 += PC) {
    const int pc = min(PC, NH - c0);
    for (int t = tid; t < NU * pc; t += NT) {
      const int i = t / pc, j = t % pc;
      Pn[(size_t)i * PC + j] = Ce[(size_t)i * NH + c0 + j];
    }
    __syncthreads();
    for (int j = tid; j < pc; j += NT)  // the row swaps, in order, one thread per column
      for (int k = 0; k < NU; ++k) {
        const int p = piv[k];
        if (p != k) {
          const double t = Pn[(size_t)k * PC + j];
          Pn[(size_t)k * PC + j] = Pn[(size_t)p * PC + j];
          Pn[(size_t)p * PC + j] = t;
        }
      }
    __syncthreads();
    for (int k = 0; k + 1 < NU; ++k) {  // L y = P c
      for (int i = k + 1 + warp; i < NU; i += NWARP) {
        const double l = W[(size_t)i * NU + k];
        for (int j = lane; j < pc; j += 32) Pn[(size_t)i * PC + j] -= l * Pn[(size_t)k * PC + j];
      }
      __syncthreads();
    }
    for (int k = NU - 1; k >= 0; --k) {  // U x = y
      const double d = 1.0 / W[(size_t)k * NU + k];
      for (int j = tid; j < pc; j += NT) Pn[(size_t)k * PC + j] *= d;
      __syncthreads();
      for (int i = warp; i < k; i += NWARP) {
        const double u = W[(size_t)i * NU + k];
        for (int j = lane; j < pc; j += 32) Pn[(size_t)i * PC + j] -= u * Pn[(size_t)k * PC + j];
      }
      __syncthreads();
    }
    for (int t = tid; t < NU * pc; t += NT) {
      const int i = t / pc, j = t % pc;
      Xe[(size_t)i * NH + c0 + j] = Pn[(size_t)i * PC + j];
    }
    __syncthreads();
  }
  // S = A33 - D X, with X staged in the shared memory the factors held
  // (nu nh <= nu nu doubles: nh <= nu for every degree here; else from global)
  const double* De = Dm + (size_t)e * NH * NU;
  const double* Ae = A33 + (size_t)e * NH * NH;
  double* Se = S + (size_t)e * NH * NH;
  const bool staged = NH <= NU;
  if (staged)
    for (int i = tid; i < NU * NH; i += NT) W[i] = Xe[i];
  __syncthreads();
  const double* Xs = staged ? W : Xe;
  for (int t = tid; t < NH * NH; t += NT) {
    const int r = t / NH, c = t % NH;
    double s = Ae[t];
    for (int m = 0; m < NU; ++m) s -= De[(size_t)r * NU + m] * Xs[(size_t)m * NH + c];
    Se[t] = s;
  }
}

template <int P>
cudaError_t launch_jac(const HdgArgs& a, const double* U, const double* Uh, double gamma, double* K, double* C,
                       double* Dm, double* A33, double* Rv, double* hv, cudaStream_t st) {
  constexpr int KC = HDG_COLUMNS_PER_THREAD;
  using G = HdgGroups<P, KC>;
  const int ge = (int)(((long long)a.E * G::NGE + 127) / 128), gf = (int)(((long long)a.E * G::NGF + 127) / 128);
  if (a.Ja)
    k_hdg_jacobian<P, KC, true><<<ge + gf, 128, 0, st>>>(a, U, Uh, gamma, K, C, Dm, A33, Rv, hv, ge);
  else
    k_hdg_jacobian<P, KC, false><<<ge + gf, 128, 0, st>>>(a, U, Uh, gamma, K, C, Dm, A33, Rv, hv, ge);
  return cudaGetLastError();
}

// One launch of the shared-memory LU kernel, or cudaErrorNotSupported when
// its shared memory cannot be had here (the caller then takes Gauss-Jordan).
template <int NT>
cudaError_t condense_lu(int E, int NU, int NH, const double* K, const double* C, const double* Dm,
                        const double* A33, double* X, double* S, cudaStream_t st) {
  int dev = 0, optin = 0;
  cudaFuncAttributes fa{};
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, k_hdg_condense_lu<NT>) != cudaSuccess) {
    cudaGetLastError();
    return cudaErrorNotSupported;
  }
  const size_t budget = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
  const size_t fixed = (size_t)NU * NU * 8 + (size_t)NU * 4 + 16;
  if (budget <= fixed) return cudaErrorNotSupported;
  int PC = fixed + (size_t)NU * NH * 8 <= budget / 2 ? NH : (int)((budget - fixed) / ((size_t)NU * 8));
  PC = PC > NH ? NH : PC;
  if (PC < 8) return cudaErrorNotSupported;
  const size_t smem = fixed + (size_t)NU * PC * 8;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(k_hdg_condense_lu<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess) {
    cudaGetLastError();
    return cudaErrorNotSupported;
  }
  k_hdg_condense_lu<NT><<<E, NT, smem, st>>>(E, NU, NH, PC, K, C, Dm, A33, X, S);
  return cudaGetLastError();
}

}  // namespace

cudaError_t hdg_jacobian(int P, const HdgArgs& a, const double* U, const double* Uh, double gamma, double* K,
                         double* C, double* Dm, double* A33, double* Rv, double* hv, cudaStream_t st) {
  switch (P) {
    case 1: return launch_jac<1>(a, U, Uh, gamma, K, C, Dm, A33, Rv, hv, st);
    case 2: return launch_jac<2>(a, U, Uh, gamma, K, C, Dm, A33, Rv, hv, st);
    case 3: return launch_jac<3>(a, U, Uh, gamma, K, C, Dm, A33, Rv, hv, st);
    case 4: return launch_jac<4>(a, U, Uh, gamma, K, C, Dm, A33, Rv, hv, st);
    default: return launch_jac<5>(a, U, Uh, gamma, K, C, Dm, A33, Rv, hv, st);
  }
}

cudaError_t hdg_condense(int E, int NU, int NH, const double* K, const double* C, const double* Dm, const double* A33,
                         double* X, double* S, double* W, cudaStream_t st) {
  if (E == 0) return cudaSuccess;
  // shared-memory LU (nu >= 64, p >= 3 in 2D; smaller K are faster with the
  // global Gauss-Jordan kernel) when K and a panel of at least 8 columns of C
  // fit next to the kernel's static shared memory; the panel takes all of C
  // when the whole [K | C] fits in half the limit (two CTAs per SM), else as
  // many columns as fit.  512 threads from nu = 100 (one CTA per SM), 256 below.
  if (NU >= 64) {
    const cudaError_t e = NU >= 100 ? condense_lu<512>(E, NU, NH, K, C, Dm, A33, X, S, st)
                                    : condense_lu<256>(E, NU, NH, K, C, Dm, A33, X, S, st);
    if (e != cudaErrorNotSupported) return e;
  }
  k_hdg_condense<<<E, 256, 0, st>>>(E, NU, NH, K, C, Dm, A33, X, S, W);
  return cudaGetLastError();
}

}  // namespace dgx
