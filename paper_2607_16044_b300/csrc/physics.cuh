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
__host__ __device__ __forceinline__ S dsqrt(S x) {
  using ::sqrt;
  return sqrt(x);
}
using ::fabs;

// Physical convective fluxes in all D directions: F[i][f].
template <int D, typename S>
__host__ __device__ __forceinline__ void conv_flux_all(const S (&U)[D + 2], const Gas<S>& g, S (&F)[D][D + 2]) {
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
__host__ __device__ __forceinline__ void visc_flux_all(const S (&U)[D + 2], const S (&Q)[D][D + 2], const Gas<S>& g,
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
__host__ __device__ __forceinline__ void visc_flux_normal(const S (&U)[D + 2], const S (&Q)[D][D + 2], const S (&nv)[D],
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

// The same through an axis normal, nv = sgn e_A (box faces normal to A):
// G = sgn F^nu_A, the one row of the flux.  It needs the velocity gradients
// of row A, of column A and of the diagonal (for div u) and the energy
// gradient along A only, about half the arithmetic of the full flux.
template <int D, int A, typename S>
__host__ __device__ __forceinline__ void visc_flux_axis(const S (&U)[D + 2], const S (&Q)[D][D + 2], S sgn,
                                                        const Gas<S>& g, S (&G)[D + 2]) {
  const S ir = S(1) / U[0];
  S u[D];
#pragma unroll
  for (int i = 0; i < D; ++i) u[i] = U[1 + i] * ir;
  const S Et = U[D + 1] * ir;
  S row[D], col[D], s = 0;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    row[j] = (Q[A][1 + j] - u[j] * Q[A][0]) * ir;  // d_A u_j
    s += u[j] * row[j];
  }
  S div = row[A];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    if (j == A) {
      col[j] = row[A];
    } else {
      col[j] = (Q[j][1 + A] - u[A] * Q[j][0]) * ir;  // d_j u_A
      div += (Q[j][1 + j] - u[j] * Q[j][0]) * ir;    // d_j u_j
    }
  }
  const S geA = (Q[A][D + 1] - Et * Q[A][0]) * ir - s;
  G[0] = S(0);
  S w = 0;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const S tau = g.mu * (row[j] + col[j]) + (j == A ? g.lam * div : S(0));
    G[1 + j] = sgn * tau;
    w += tau * u[j];
  }
  G[D + 1] = sgn * (w + g.kcv * geA);
}

// get(s) for the run-time shift s = A (0 .. D-1), each candidate formed with
// s fixed at compile time and the result chosen by selects, not branches.
template <int D, typename Get>
__host__ __device__ __forceinline__ auto by_shift(int A, Get get) -> decltype(get(0)) {
  if (D == 2) return A == 0 ? get(0) : get(1);
  return A == 0 ? get(0) : (A == 1 ? get(1) : get(D > 2 ? 2 : 1));
}

// Axes relabelled i -> (i + A) mod D, so that axis A becomes axis 0.  The
// viscous flux is isotropic (it commutes with every orthogonal change of
// axes, permutations included), so the row along A of the original equals
// the row along 0 of the relabelled state and gradient, its momentum
// components relabelled back.
template <int D, typename S>
__host__ __device__ __forceinline__ void relabel_state(const S (&U)[D + 2], int A, S (&Ur)[D + 2]) {
  Ur[0] = U[0];
  Ur[D + 1] = U[D + 1];
#pragma unroll
  for (int i = 0; i < D; ++i) Ur[1 + i] = by_shift<D>(A, [&](int s) { return U[1 + (i + s) % D]; });
}
// the same for a gradient-shaped array Q[c][f] (direction c, field f)
template <int D, typename S>
__host__ __device__ __forceinline__ void relabel_grad(const S (&Q)[D][D + 2], int A, S (&Qr)[D][D + 2]) {
#pragma unroll
  for (int c = 0; c < D; ++c) {
    Qr[c][0] = by_shift<D>(A, [&](int s) { return Q[(c + s) % D][0]; });
    Qr[c][D + 1] = by_shift<D>(A, [&](int s) { return Q[(c + s) % D][D + 1]; });
#pragma unroll
    for (int i = 0; i < D; ++i) Qr[c][1 + i] = by_shift<D>(A, [&](int s) { return Q[(c + s) % D][1 + (i + s) % D]; });
  }
}
template <int D, typename S>
__host__ __device__ __forceinline__ void axis_relabel(const S (&U)[D + 2], const S (&Q)[D][D + 2], int A,
                                                      S (&Ur)[D + 2], S (&Qr)[D][D + 2]) {
  relabel_state<D, S>(U, A, Ur);
  relabel_grad<D, S>(Q, A, Qr);
}

// visc_flux_axis with the axis A given at run time (0 .. D-1).  Lanes of one
// warp often hold faces of different axes (a face's points do not fill whole
// warps).  In FP64, where the kernels are bound by the FP64 pipe, branching to
// the instance for A would run two instances in those warps, so the state and
// gradient are relabelled to put A first (selects on the integer pipe) and
// the instance for axis 0 runs on every lane.  FP32 kernels are bound by
// memory and issue instead; there the relabelling's extra instructions and
// registers cost more than the divergence, and the branch is kept.
template <int D, typename S>
__host__ __device__ __forceinline__ void visc_flux_axis_rt(const S (&U)[D + 2], const S (&Q)[D][D + 2], int A, S sgn,
                                                           const Gas<S>& g, S (&G)[D + 2]) {
  if constexpr (sizeof(S) == 4) {
    if (A == 0) visc_flux_axis<D, 0, S>(U, Q, sgn, g, G);
    else if (D == 2 || A == 1) visc_flux_axis<D, 1, S>(U, Q, sgn, g, G);
    else visc_flux_axis<D, (D > 2 ? 2 : 1), S>(U, Q, sgn, g, G);
    return;
  }
  S Ur[D + 2], Qr[D][D + 2], Gr[D + 2];
  axis_relabel<D, S>(U, Q, A, Ur, Qr);
  visc_flux_axis<D, 0, S>(Ur, Qr, sgn, g, Gr);
  G[0] = Gr[0];
  G[D + 1] = Gr[D + 1];
#pragma unroll
  for (int j = 0; j < D; ++j) G[1 + j] = by_shift<D>(A, [&](int s) { return Gr[1 + (j + D - s) % D]; });
}

// Adiabatic no-slip wall: F^nu(U_w, Q).nv with U_w = (rho, 0, rho e_i) and q.n = 0,
// i.e. (0, tau(U_w, Q) nv, 0) where d_a u_i = Q[a][1+i] / rho.
template <int D, typename S>
__host__ __device__ __forceinline__ void wall_visc_flux(const S (&U)[D + 2], const S (&Q)[D][D + 2], const S (&nv)[D],
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
__host__ __device__ __forceinline__ void mirror_state(const S (&U)[D + 2], const S (&nv)[D], S (&R)[D + 2]) {
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
__host__ __device__ __forceinline__ void wall_state(const S (&U)[D + 2], S (&W)[D + 2]) {
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
__host__ __device__ __forceinline__ void llf_flux(const S (&UL)[D + 2], const S (&UR)[D + 2], const S (&nv)[D],
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

// ===========================================================================
// Reverse-mode (vector-Jacobian) counterparts, derived by hand from the
// forward formulas above.  Each *_vjp adds (d out / d in)^T * out_bar into the
// input cotangents (callers zero them first).  Conventions: d|x|/dx = sign(x)
// with sign(0) = 0; at a tie of the LLF wave speeds the interior side (L) is
// differentiated.
// ===========================================================================
namespace dgx {

template <typename S>
__host__ __device__ __forceinline__ S sgn(S x) { return x > S(0) ? S(1) : (x < S(0) ? S(-1) : S(0)); }

// Convective fluxes in all directions: Ub += (dF/dU)^T Fb.
template <int D, typename S>
__host__ __device__ __forceinline__ void conv_flux_all_vjp(const S (&U)[D + 2], const S (&Fb)[D][D + 2], const Gas<S>& g,
                                                  S (&Ub)[D + 2]) {
  const S ir = S(1) / U[0];
  S u[D], mm = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    u[i] = U[1 + i] * ir;
    mm += U[1 + i] * u[i];
  }
  const S p = g.gm1 * (U[D + 1] - S(0.5) * mm);
  const S h = U[D + 1] + p;
  S mb[D], ub[D], pb = 0, hb = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    mb[i] = Fb[i][0];
    ub[i] = S(0);
  }
#pragma unroll
  for (int i = 0; i < D; ++i) {
#pragma unroll
    for (int j = 0; j < D; ++j) {
      mb[j] += Fb[i][1 + j] * u[i];
      ub[i] += Fb[i][1 + j] * U[1 + j];
    }
    pb += Fb[i][1 + i];
    hb += Fb[i][D + 1] * u[i];
    ub[i] += Fb[i][D + 1] * h;
  }
  S Eb = hb;
  pb += hb;
  Eb += g.gm1 * pb;
  const S mmb = -S(0.5) * g.gm1 * pb;
  S irb = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    mb[i] += mmb * u[i];
    ub[i] += mmb * U[1 + i];
    mb[i] += ub[i] * ir;
    irb += ub[i] * U[1 + i];
  }
  Ub[0] += -irb * ir * ir;
#pragma unroll
  for (int i = 0; i < D; ++i) Ub[1 + i] += mb[i];
  Ub[D + 1] += Eb;
}

// Viscous fluxes in all directions: Ub += (dF/dU)^T Fb, Qb += (dF/dQ)^T Fb.
template <int D, typename S>
__host__ __device__ __forceinline__ void visc_flux_all_vjp(const S (&U)[D + 2], const S (&Q)[D][D + 2], const S (&Fb)[D][D + 2],
                                                  const Gas<S>& g, S (&Ub)[D + 2], S (&Qb)[D][D + 2]) {
  const S ir = S(1) / U[0];
  S u[D];
#pragma unroll
  for (int i = 0; i < D; ++i) u[i] = U[1 + i] * ir;
  const S Et = U[D + 1] * ir;
  S gu[D][D];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int i = 0; i < D; ++i) gu[a][i] = (Q[a][1 + i] - u[i] * Q[a][0]) * ir;
  S div = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) div += gu[i][i];
  // forward tau (needed for u_bar)
  S tau[D][D];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) tau[i][j] = g.mu * (gu[i][j] + gu[j][i]) + (i == j ? g.lam * div : S(0));
  // reverse
  S ub[D], gub[D][D], geb[D];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    ub[i] = S(0);
#pragma unroll
    for (int j = 0; j < D; ++j) gub[i][j] = S(0);
  }
  S divb = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const S we = Fb[i][D + 1];
    geb[i] = g.kcv * we;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const S taub = Fb[i][1 + j] + we * u[j];
      ub[j] += we * tau[i][j];
      gub[i][j] += g.mu * taub;
      gub[j][i] += g.mu * taub;
      if (i == j) divb += g.lam * taub;
    }
  }
#pragma unroll
  for (int i = 0; i < D; ++i) gub[i][i] += divb;
  S irb = 0, Etb = 0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    // ge[a] = (Q[a][E] - Et Q[a][0]) ir - sum_i u_i gu[a][i]
    Qb[a][D + 1] += geb[a] * ir;
    Qb[a][0] += -geb[a] * Et * ir;
    Etb += -geb[a] * Q[a][0] * ir;
    irb += geb[a] * (Q[a][D + 1] - Et * Q[a][0]);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      ub[i] += -geb[a] * gu[a][i];
      gub[a][i] += -geb[a] * u[i];
    }
  }
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int i = 0; i < D; ++i) {
      // gu[a][i] = (Q[a][1+i] - u_i Q[a][0]) ir
      Qb[a][1 + i] += gub[a][i] * ir;
      Qb[a][0] += -gub[a][i] * u[i] * ir;
      ub[i] += -gub[a][i] * Q[a][0] * ir;
      irb += gub[a][i] * (Q[a][1 + i] - u[i] * Q[a][0]);
    }
  Ub[D + 1] += Etb * ir;
  irb += Etb * U[D + 1];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    Ub[1 + i] += ub[i] * ir;
    irb += ub[i] * U[1 + i];
  }
  Ub[0] += -irb * ir * ir;
}

// G = sum_i F^nu_i nv_i: cotangent Gb -> (Ub, Qb).
template <int D, typename S>
__host__ __device__ __forceinline__ void visc_flux_normal_vjp(const S (&U)[D + 2], const S (&Q)[D][D + 2], const S (&nv)[D],
                                                     const S (&Gb)[D + 2], const Gas<S>& g, S (&Ub)[D + 2],
                                                     S (&Qb)[D][D + 2]) {
  S Fb[D][D + 2];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int f = 0; f < D + 2; ++f) Fb[i][f] = Gb[f] * nv[i];
  visc_flux_all_vjp<D, S>(U, Q, Fb, g, Ub, Qb);
}

// Cotangent of visc_flux_axis: Gb -> (Ub, Qb), accumulated; the reverse of
// its steps in the opposite order.
template <int D, int A, typename S>
__host__ __device__ __forceinline__ void visc_flux_axis_vjp(const S (&U)[D + 2], const S (&Q)[D][D + 2], S sgn,
                                                            const S (&Gb)[D + 2], const Gas<S>& g, S (&Ub)[D + 2],
                                                            S (&Qb)[D][D + 2]) {
  const S ir = S(1) / U[0];
  S u[D];
#pragma unroll
  for (int i = 0; i < D; ++i) u[i] = U[1 + i] * ir;
  const S Et = U[D + 1] * ir;
  // forward values needed by the reverse
  S nrow[D], ncol[D], ndia[D], row[D], col[D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    nrow[j] = Q[A][1 + j] - u[j] * Q[A][0];
    row[j] = nrow[j] * ir;
  }
  S div = row[A];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    if (j == A) {
      ncol[j] = ndia[j] = S(0);
      col[j] = row[A];
    } else {
      ncol[j] = Q[j][1 + A] - u[A] * Q[j][0];
      col[j] = ncol[j] * ir;
      ndia[j] = Q[j][1 + j] - u[j] * Q[j][0];
      div += ndia[j] * ir;
    }
  }
  const S ngeA = Q[A][D + 1] - Et * Q[A][0];
  // G[D+1] = sgn (sum_j tau_j u_j + kcv geA),  G[1+j] = sgn tau_j
  const S gE = sgn * Gb[D + 1];
  S ub[D], rowb[D], colb[D], diab[D], divb = 0;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    ub[j] = S(0);
    rowb[j] = colb[j] = diab[j] = S(0);
  }
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const S tau = g.mu * (row[j] + col[j]) + (j == A ? g.lam * div : S(0));
    const S taub = sgn * Gb[1 + j] + gE * u[j];
    ub[j] += gE * tau;
    rowb[j] += g.mu * taub;
    if (j == A) {
      rowb[A] += g.mu * taub;  // col[A] is row[A]
      divb += g.lam * taub;
    } else {
      colb[j] += g.mu * taub;
    }
  }
  const S geAb = gE * g.kcv;
  // div = row[A] + sum_{j != A} ndia[j] ir
  rowb[A] += divb;
#pragma unroll
  for (int j = 0; j < D; ++j)
    if (j != A) diab[j] += divb;
  // geA = ngeA ir - sum_j u_j row_j
  S irb = geAb * ngeA;
  const S cge = geAb * ir;
  Qb[A][D + 1] += cge;
  Qb[A][0] -= Et * cge;
  const S Etb = -Q[A][0] * cge;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    ub[j] -= geAb * row[j];
    rowb[j] -= geAb * u[j];
  }
  // row_j = (Q[A][1+j] - u_j Q[A][0]) ir
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const S r = rowb[j] * ir;
    Qb[A][1 + j] += r;
    Qb[A][0] -= u[j] * r;
    ub[j] -= Q[A][0] * r;
    irb += rowb[j] * nrow[j];
  }
  // col_j = (Q[j][1+A] - u_A Q[j][0]) ir and dia_j = (Q[j][1+j] - u_j Q[j][0]) ir, j != A
#pragma unroll
  for (int j = 0; j < D; ++j) {
    if (j == A) continue;
    const S rc = colb[j] * ir, rd = diab[j] * ir;
    Qb[j][1 + A] += rc;
    Qb[j][0] -= u[A] * rc + u[j] * rd;
    ub[A] -= Q[j][0] * rc;
    Qb[j][1 + j] += rd;
    ub[j] -= Q[j][0] * rd;
    irb += colb[j] * ncol[j] + diab[j] * ndia[j];
  }
  // u_i = U[1+i] ir, Et = U[D+1] ir, ir = 1 / U[0]
#pragma unroll
  for (int i = 0; i < D; ++i) {
    Ub[1 + i] += ub[i] * ir;
    irb += ub[i] * U[1 + i];
  }
  Ub[D + 1] += Etb * ir;
  irb += Etb * U[D + 1];
  Ub[0] -= irb * ir * ir;
}

template <int D, typename S>
__host__ __device__ __forceinline__ void visc_flux_axis_vjp_rt(const S (&U)[D + 2], const S (&Q)[D][D + 2], int A,
                                                               S sgn, const S (&Gb)[D + 2], const Gas<S>& g,
                                                               S (&Ub)[D + 2], S (&Qb)[D][D + 2]) {
  // the same choice as visc_flux_axis_rt (branch in FP32, relabel in FP64);
  // the accumulators are relabelled in and back out, so nothing is added
  // beyond what the axis-0 adjoint adds
  if constexpr (sizeof(S) == 4) {
    if (A == 0) visc_flux_axis_vjp<D, 0, S>(U, Q, sgn, Gb, g, Ub, Qb);
    else if (D == 2 || A == 1) visc_flux_axis_vjp<D, 1, S>(U, Q, sgn, Gb, g, Ub, Qb);
    else visc_flux_axis_vjp<D, (D > 2 ? 2 : 1), S>(U, Q, sgn, Gb, g, Ub, Qb);
    return;
  }
  S Ur[D + 2], Qr[D][D + 2], Gbr[D + 2], Ubr[D + 2], Qbr[D][D + 2];
  axis_relabel<D, S>(U, Q, A, Ur, Qr);
  axis_relabel<D, S>(Ub, Qb, A, Ubr, Qbr);
  Gbr[0] = Gb[0];
  Gbr[D + 1] = Gb[D + 1];
#pragma unroll
  for (int i = 0; i < D; ++i) Gbr[1 + i] = by_shift<D>(A, [&](int s) { return Gb[1 + (i + s) % D]; });
  visc_flux_axis_vjp<D, 0, S>(Ur, Qr, sgn, Gbr, g, Ubr, Qbr);
  // inverse relabelling: shift by (D - A) mod D
  const int Ai = (D - A) % D;
  axis_relabel<D, S>(Ubr, Qbr, Ai, Ub, Qb);
}

// Adiabatic wall flux (0, tau(U_w, Q) nv, 0), d_a u_i = Q[a][1+i] / rho.
template <int D, typename S>
__host__ __device__ __forceinline__ void wall_visc_flux_vjp(const S (&U)[D + 2], const S (&Q)[D][D + 2], const S (&nv)[D],
                                                   const S (&Gb)[D + 2], const Gas<S>& g, S (&Ub)[D + 2],
                                                   S (&Qb)[D][D + 2]) {
  const S ir = S(1) / U[0];
  S gub[D][D];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) gub[i][j] = S(0);
  S divb = 0;
#pragma unroll
  for (int j = 0; j < D; ++j)
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const S taub = Gb[1 + j] * nv[i];
      gub[i][j] += g.mu * taub;
      gub[j][i] += g.mu * taub;
      if (i == j) divb += g.lam * taub;
    }
#pragma unroll
  for (int i = 0; i < D; ++i) gub[i][i] += divb;
  S irb = 0;
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int i = 0; i < D; ++i) {
      Qb[a][1 + i] += gub[a][i] * ir;
      irb += gub[a][i] * Q[a][1 + i];
    }
  Ub[0] += -irb * ir * ir;
}

// Mirror state R = (rho, m - 2 (m.n) n / |n|^2, rho E): linear and symmetric in m.
template <int D, typename S>
__host__ __device__ __forceinline__ void mirror_state_vjp(const S (&nv)[D], const S (&Rb)[D + 2], S (&Ub)[D + 2]) {
  S n2 = 0, rn = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    n2 += nv[i] * nv[i];
    rn += Rb[1 + i] * nv[i];
  }
  const S c = S(2) * rn / n2;
  Ub[0] += Rb[0];
#pragma unroll
  for (int i = 0; i < D; ++i) Ub[1 + i] += Rb[1 + i] - c * nv[i];
  Ub[D + 1] += Rb[D + 1];
}

// Wall state W = (rho, 0, rho E - |m|^2 / (2 rho)).
template <int D, typename S>
__host__ __device__ __forceinline__ void wall_state_vjp(const S (&U)[D + 2], const S (&Wb)[D + 2], S (&Ub)[D + 2]) {
  const S ir = S(1) / U[0];
  S mm = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) mm += U[1 + i] * U[1 + i];
  Ub[0] += Wb[0] + Wb[D + 1] * S(0.5) * mm * ir * ir;
#pragma unroll
  for (int i = 0; i < D; ++i) Ub[1 + i] += -Wb[D + 1] * U[1 + i] * ir;
  Ub[D + 1] += Wb[D + 1];
}

// LLF flux: cotangent Fb -> (ULb, URb).
template <int D, typename S, bool UNIT>
__host__ __device__ __forceinline__ void llf_flux_vjp(const S (&UL)[D + 2], const S (&UR)[D + 2], const S (&nv)[D],
                                             const S (&Fb)[D + 2], const Gas<S>& g, S (&ULb)[D + 2],
                                             S (&URb)[D + 2]) {
  S sJ = S(1);
  if (!UNIT) {
    S n2 = 0;
#pragma unroll
    for (int i = 0; i < D; ++i) n2 += nv[i] * nv[i];
    sJ = dsqrt(n2);
  }
  // forward quantities per side
  S lamv[2], unv[2], cv[2], pv[2], irv[2];
  S uv[2][D];
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const S(&V)[D + 2] = side ? UR : UL;
    const S ir = S(1) / V[0];
    S un = 0, mm = 0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      uv[side][i] = V[1 + i] * ir;
      un += uv[side][i] * nv[i];
      mm += V[1 + i] * uv[side][i];
    }
    const S p = g.gm1 * (V[D + 1] - S(0.5) * mm);
    cv[side] = dsqrt(g.gamma * p * ir);
    lamv[side] = fabs(un) + cv[side] * sJ;
    unv[side] = un;
    pv[side] = p;
    irv[side] = ir;
  }
  const bool left = lamv[0] >= lamv[1];
  const S lam = left ? lamv[0] : lamv[1];
  S lamb = 0;
#pragma unroll
  for (int f = 0; f < D + 2; ++f) {
    lamb += -S(0.5) * Fb[f] * (UR[f] - UL[f]);
    URb[f] += -S(0.5) * lam * Fb[f];
    ULb[f] += S(0.5) * lam * Fb[f];
  }
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const S(&V)[D + 2] = side ? UR : UL;
    S(&Vb)[D + 2] = side ? URb : ULb;
    const S ir = irv[side], un = unv[side], p = pv[side], c = cv[side];
    const S sideLam = (left == (side == 0)) ? lamb : S(0);
    // lam_side = |un| + c sJ
    S unb = sideLam * sgn(un);
    const S cb = sideLam * sJ;
    // c = sqrt(gamma p ir)
    S pb = 0, irb = 0;
    if (c > S(0)) {  // dc = gamma (ir dp + p dir) / (2 c), one division for both
      const S h2c = cb * g.gamma / (S(2) * c);
      pb += h2c * ir;
      irb += h2c * p;
    }
    // Fn = (m.n, m_j un + p n_j, (E + p) un) with cotangent Fb/2
    S mb[D];
    S Eb = S(0);
    const S h = S(0.5);
#pragma unroll
    for (int i = 0; i < D; ++i) mb[i] = h * Fb[0] * nv[i];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      mb[j] += h * Fb[1 + j] * un;
      unb += h * Fb[1 + j] * V[1 + j];
      pb += h * Fb[1 + j] * nv[j];
    }
    Eb += h * Fb[D + 1] * un;
    pb += h * Fb[D + 1] * un;
    unb += h * Fb[D + 1] * (V[D + 1] + p);
    // un = u . n
    S ub[D];
#pragma unroll
    for (int i = 0; i < D; ++i) ub[i] = unb * nv[i];
    // p = gm1 (E - mm / 2), mm = m . u
    Eb += g.gm1 * pb;
    const S mmb = -S(0.5) * g.gm1 * pb;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      mb[i] += mmb * uv[side][i];
      ub[i] += mmb * V[1 + i];
      mb[i] += ub[i] * ir;
      irb += ub[i] * V[1 + i];
    }
    Vb[0] += -irb * ir * ir;
#pragma unroll
    for (int i = 0; i < D; ++i) Vb[1 + i] += mb[i];
    Vb[D + 1] += Eb;
  }
}

}  // namespace dgx
