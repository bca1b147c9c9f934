// Pointwise compressible-flow physics on the device (Sec. 2 of the paper).
//
// State U = (rho, m_1..m_D, rho E), m = rho u; ideal gas p = (gamma-1)(rho E - |m|^2/(2 rho)).
// Convective flux F^c_i = (m_i, m_i u_j + p delta_ij, (rho E + p) u_i).
// Viscous flux F^nu_i = (0, tau_ij, tau_ij u_j - q_i), tau = mu (grad u + grad u^T)
// + lambda (div u) I, lambda = -2 mu / 3, q = -kappa grad theta.  With the
// nondimensionalisation rho_ref = |u_ref| = L_ref = 1, theta_inf = 1 one has
// kappa grad theta = (gamma mu / Pr) grad e, e = E - |u|^2/2, so the operator
// needs only gamma, mu and kcv = gamma mu / Pr.
// Gradients are of the conservative variables: Q[a][f] = d U_f / d x_a.
#pragma once
#include <cuda_runtime.h>

namespace dgx {

template <typename S>
struct Gas {
  S gamma, gm1, mu, lam, kcv;
};

template <typename S>
__device__ __forceinline__ S dsqrt(S x) { return sqrt(x); }

// Physical convective fluxes in all D directions: F[i][f].
template <int D, typename S>
__device__ __forceinline__ void conv_flux_all(const S (&U)[D + 2], const Gas<S>& g, S (&F)[D][D + 2]) {
  const S ir = S(1) / U[0];
  S u[D];
  S mm = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    u[i] = U[1 + i] * ir;
    mm += U[1 + i] * u[i];
  }
  const S p = g.gm1 * (U[D + 1] - S(0.5) * mm);
  const S h = U[D + 1] + p;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    F[i][0] = U[1 + i];
#pragma unroll
    for (int j = 0; j < D; ++j) F[i][1 + j] = U[1 + j] * u[i] + (i == j ? p : S(0));
    F[i][D + 1] = h * u[i];
  }
}

// Viscous fluxes in all D directions from U and Q = grad U.
template <int D, typename S>
__device__ __forceinline__ void visc_flux_all(const S (&U)[D + 2], const S (&Q)[D][D + 2], const Gas<S>& g,
                                              S (&F)[D][D + 2]) {
  const S ir = S(1) / U[0];
  S u[D];
#pragma unroll
  for (int i = 0; i < D; ++i) u[i] = U[1 + i] * ir;
  const S Et = U[D + 1] * ir;
  S gu[D][D];  // gu[a][i] = d_a u_i
  S ge[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    S s = 0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      gu[a][i] = (Q[a][1 + i] - u[i] * Q[a][0]) * ir;
      s += u[i] * gu[a][i];
    }
    ge[a] = (Q[a][D + 1] - Et * Q[a][0]) * ir - s;
  }
  S div = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) div += gu[i][i];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    F[i][0] = S(0);
    S w = 0;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const S tau = g.mu * (gu[i][j] + gu[j][i]) + (i == j ? g.lam * div : S(0));
      F[i][1 + j] = tau;
      w += tau * u[j];
    }
    F[i][D + 1] = w + g.kcv * ge[i];
  }
}

// Viscous flux through the vector nv:  G = sum_i F^nu_i nv_i.
template <int D, typename S>
__device__ __forceinline__ void visc_flux_normal(const S (&U)[D + 2], const S (&Q)[D][D + 2], const S (&nv)[D],
                                                 const Gas<S>& g, S (&G)[D + 2]) {
  S F[D][D + 2];
  visc_flux_all<D, S>(U, Q, g, F);
#pragma unroll
  for (int f = 0; f < D + 2; ++f) {
    S s = 0;
#pragma unroll
    for (int i = 0; i < D; ++i) s += F[i][f] * nv[i];
    G[f] = s;
  }
}

// Adiabatic no-slip wall: F^nu(U_w, Q).nv with U_w = (rho, 0, rho e_i) and q.n = 0,
// i.e. (0, tau(U_w, Q) nv, 0) where d_a u_i = Q[a][1+i] / rho.
template <int D, typename S>
__device__ __forceinline__ void wall_visc_flux(const S (&U)[D + 2], const S (&Q)[D][D + 2], const S (&nv)[D],
                                               const Gas<S>& g, S (&G)[D + 2]) {
  const S ir = S(1) / U[0];
  S gu[D][D];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int i = 0; i < D; ++i) gu[a][i] = Q[a][1 + i] * ir;
  S div = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) div += gu[i][i];
  G[0] = S(0);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    S s = 0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const S tau = g.mu * (gu[i][j] + gu[j][i]) + (i == j ? g.lam * div : S(0));
      s += tau * nv[i];
    }
    G[1 + j] = s;
  }
  G[D + 1] = S(0);
}

// Mirror (reflected) state across a wall with normal nv: (rho, m - 2 (m.n) n, rho E).
template <int D, typename S>
__device__ __forceinline__ void mirror_state(const S (&U)[D + 2], const S (&nv)[D], S (&R)[D + 2]) {
  S n2 = 0, mn = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    n2 += nv[i] * nv[i];
    mn += U[1 + i] * nv[i];
  }
  const S c = S(2) * mn / n2;
  R[0] = U[0];
#pragma unroll
  for (int i = 0; i < D; ++i) R[1 + i] = U[1 + i] - c * nv[i];
  R[D + 1] = U[D + 1];
}

// No-slip wall state U_w = (rho, 0, .., 0, rho E - |m|^2 / (2 rho)).
template <int D, typename S>
__device__ __forceinline__ void wall_state(const S (&U)[D + 2], S (&W)[D + 2]) {
  S mm = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) mm += U[1 + i] * U[1 + i];
  W[0] = U[0];
#pragma unroll
  for (int i = 0; i < D; ++i) W[1 + i] = S(0);
  W[D + 1] = U[D + 1] - S(0.5) * mm / U[0];
}

// Local Lax-Friedrichs flux through the (area-weighted) normal nv, own side L:
// F* = (F(UL) + F(UR)).nv / 2 - lam (UR - UL) / 2,
// lam = max(|uL.nv| + cL |nv|, |uR.nv| + cR |nv|).
template <int D, typename S, bool UNIT>
__device__ __forceinline__ void llf_flux(const S (&UL)[D + 2], const S (&UR)[D + 2], const S (&nv)[D],
                                         const Gas<S>& g, S (&F)[D + 2]) {
  S sJ = S(1);
  if (!UNIT) {
    S n2 = 0;
#pragma unroll
    for (int i = 0; i < D; ++i) n2 += nv[i] * nv[i];
    sJ = dsqrt(n2);
  }
  S lamv[2];
  S Fn[2][D + 2];
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const S(&V)[D + 2] = side ? UR : UL;
    const S ir = S(1) / V[0];
    S un = 0, mm = 0, mn = 0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const S ui = V[1 + i] * ir;
      un += ui * nv[i];
      mm += V[1 + i] * ui;
      mn += V[1 + i] * nv[i];
    }
    const S p = g.gm1 * (V[D + 1] - S(0.5) * mm);
    const S c = dsqrt(g.gamma * p * ir);
    lamv[side] = fabs(un) + c * sJ;
    Fn[side][0] = mn;
#pragma unroll
    for (int j = 0; j < D; ++j) Fn[side][1 + j] = V[1 + j] * un + p * nv[j];
    Fn[side][D + 1] = (V[D + 1] + p) * un;
  }
  const S lam = lamv[0] >= lamv[1] ? lamv[0] : lamv[1];
#pragma unroll
  for (int f = 0; f < D + 2; ++f) F[f] = S(0.5) * (Fn[0][f] + Fn[1][f]) - S(0.5) * lam * (UR[f] - UL[f]);
}

}  // namespace dgx
