// Pointwise physics of the paper's DG-IP operator (device and host).
//
// * vij_flux: the Vijayasundaram flux of Sec. 3.3 (Eq.
//   upwinding_Vijayasundaram_sdg), A_n^+(Ubar) U^+ + A_n^-(Ubar) U^-,
//   Ubar = (U^+ + U^-)/2, with the characteristic splitting of Sec. 3.2.  Since
//   the Euler flux is homogeneous of degree one, A_n(Ubar) Ubar = F_n(Ubar), and
//   A^+ U^+ + A^- U^- = F_n(Ubar) + |A_n(Ubar)| (U^+ - U^-) / 2.  |A_n| dU is
//   evaluated as the sum over characteristic waves |lambda_k| alpha_k r_k,
//   alpha_k = l_k . dU: the two acoustic waves (lambda = u.n -+ c, wave
//   strengths alpha_-+ = (dp -+ rho c du_n) / (2 c^2) with the pressure and
//   normal-velocity jumps linearised at Ubar, eigenvectors
//   r_-+ = (1, u -+ c n, H -+ c u_n)) and the d-fold wave lambda = u.n, whose
//   part of dU is what the acoustic waves leave:
//   |A| dU = |u_n| dU + (|u_n - c| - |u_n|) alpha_- r_- + (|u_n + c| - |u_n|) alpha_+ r_+.
// * farfield_state: U_Gamma of App. B.1.1, A_n(U) U_Gamma = A_n^+(U) U +
//   A_n^-(U) U_inf: the waves with lambda_k >= 0 of U - U_inf kept, so
//   U_Gamma = U_inf + [u_n - c >= 0] alpha_- r_- + [u_n + c >= 0] alpha_+ r_+
//            + [u_n >= 0] (dU - alpha_- r_- - alpha_+ r_+),  dU = U - U_inf.
// * K-products: the viscous flux is linear in its gradient argument, so
//   K(U)(delta (x) n) = F^nu(U, grad U := n (x) delta) (visc_flux_all with
//   Q[c][f] = n_c delta_f).  On adiabatic walls K_w removes the normal heat
//   flux; for a gradient argument delta (x) n the heat flux is parallel to n,
//   so K_w(U)(delta (x) n) is the viscous flux with kappa = 0, and so is the
//   normal component of F^{nu,w}(U, grad U).
// * Dual<S, K>: forward-mode dual numbers (value + K tangents) used by the
//   adjoint face kernel to differentiate the face function exactly.
#pragma once
#include <cuda_runtime.h>

#include "physics.cuh"

namespace dgx {

template <typename S, int K>
struct Dual {
  S v;
  S d[K];
  __host__ __device__ Dual() : v(0) {
#pragma unroll
    for (int k = 0; k < K; ++k) d[k] = S(0);
  }
  template <typename X>
  __host__ __device__ Dual(X x) : v((S)x) {
#pragma unroll
    for (int k = 0; k < K; ++k) d[k] = S(0);
  }
  friend __host__ __device__ __forceinline__ Dual operator+(const Dual& a, const Dual& b) {
    Dual r;
    r.v = a.v + b.v;
#pragma unroll
    for (int k = 0; k < K; ++k) r.d[k] = a.d[k] + b.d[k];
    return r;
  }
  friend __host__ __device__ __forceinline__ Dual operator-(const Dual& a, const Dual& b) {
    Dual r;
    r.v = a.v - b.v;
#pragma unroll
    for (int k = 0; k < K; ++k) r.d[k] = a.d[k] - b.d[k];
    return r;
  }
  friend __host__ __device__ __forceinline__ Dual operator-(const Dual& a) {
    Dual r;
    r.v = -a.v;
#pragma unroll
    for (int k = 0; k < K; ++k) r.d[k] = -a.d[k];
    return r;
  }
  friend __host__ __device__ __forceinline__ Dual operator*(const Dual& a, const Dual& b) {
    Dual r;
    r.v = a.v * b.v;
#pragma unroll
    for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
  }
  friend __host__ __device__ __forceinline__ Dual operator/(const Dual& a, const Dual& b) {
    Dual r;
    const S ib = S(1) / b.v;
    r.v = a.v * ib;
#pragma unroll
    for (int k = 0; k < K; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
    return r;
  }
  __host__ __device__ __forceinline__ Dual& operator+=(const Dual& b) { return *this = *this + b; }
  __host__ __device__ __forceinline__ Dual& operator-=(const Dual& b) { return *this = *this - b; }
  __host__ __device__ __forceinline__ Dual& operator*=(const Dual& b) { return *this = *this * b; }
  friend __host__ __device__ __forceinline__ bool operator>(const Dual& a, const Dual& b) { return a.v > b.v; }
  friend __host__ __device__ __forceinline__ bool operator>=(const Dual& a, const Dual& b) { return a.v >= b.v; }
  friend __host__ __device__ __forceinline__ bool operator<(const Dual& a, const Dual& b) { return a.v < b.v; }
  friend __host__ __device__ __forceinline__ Dual sqrt(const Dual& a) {
    Dual r;
    using ::sqrt;
    r.v = sqrt(a.v);
    const S h = S(0.5) / r.v;
#pragma unroll
    for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * h;
    return r;
  }
  // d|x|/dx = sign(x), sign(0) = 0
  friend __host__ __device__ __forceinline__ Dual fabs(const Dual& a) {
    const S s = a.v > S(0) ? S(1) : (a.v < S(0) ? S(-1) : S(0));
    Dual r;
    r.v = a.v < S(0) ? -a.v : a.v;
#pragma unroll
    for (int k = 0; k < K; ++k) r.d[k] = s * a.d[k];
    return r;
  }
};

template <typename T, typename S>
__host__ __device__ __forceinline__ Gas<T> gas_as(const Gas<S>& g) {
  Gas<T> r;
  r.gamma = T(g.gamma);
  r.gm1 = T(g.gm1);
  r.mu = T(g.mu);
  r.lam = T(g.lam);
  r.kcv = T(g.kcv);
  return r;
}

// Normal convective flux F^c . nv.
template <int D, typename T, typename N>
__host__ __device__ __forceinline__ void conv_flux_normal(const T (&U)[D + 2], const N (&nv)[D], const Gas<T>& g,
                                                          T (&F)[D + 2]) {
  const T ir = T(1) / U[0];
  T un = T(0), mm = T(0), mn = T(0);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const T ui = U[1 + i] * ir;
    un += ui * T(nv[i]);
    mm += U[1 + i] * ui;
    mn += U[1 + i] * T(nv[i]);
  }
  const T p = g.gm1 * (U[D + 1] - T(0.5) * mm);
  F[0] = mn;
#pragma unroll
  for (int j = 0; j < D; ++j) F[1 + j] = U[1 + j] * un + p * T(nv[j]);
  F[D + 1] = (U[D + 1] + p) * un;
}

// |nv| and the unit normal nv / |nv| (one reciprocal); UNIT: nv is a unit
// vector already (box faces) and is taken as it is.
template <int D, typename N, bool UNIT>
__host__ __device__ __forceinline__ void unit_of(const N (&nv)[D], N& sJ, N (&nh)[D]) {
  if (UNIT) {
    sJ = N(1);
#pragma unroll
    for (int i = 0; i < D; ++i) nh[i] = nv[i];
  } else {
    using ::sqrt;
    N n2 = N(0);
#pragma unroll
    for (int i = 0; i < D; ++i) n2 += nv[i] * nv[i];
    sJ = sqrt(n2);
    const N isJ = N(1) / sJ;
#pragma unroll
    for (int i = 0; i < D; ++i) nh[i] = nv[i] * isJ;
  }
}

// Characteristic quantities of a state along the unit normal nh and the two
// acoustic wave strengths of a jump dU (see the header comment).
template <int D, typename T, typename N>
struct Waves {
  T u[D], un, c, H, am, ap;
  __host__ __device__ __forceinline__ Waves(const T (&U)[D + 2], const T (&dU)[D + 2], const N (&nh)[D],
                                            const Gas<T>& g) {
    const T rho = U[0];
    const T ir = T(1) / rho;
    T q2 = T(0);
    un = T(0);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      u[i] = U[1 + i] * ir;
      q2 += u[i] * u[i];
      un += u[i] * T(nh[i]);
    }
    const T p = g.gm1 * (U[D + 1] - T(0.5) * rho * q2);
    const T c2 = g.gamma * p * ir;
    c = dsqrt(c2);
    H = (U[D + 1] + p) * ir;
    T udm = T(0), ndm = T(0);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      udm += u[i] * dU[1 + i];
      ndm += T(nh[i]) * dU[1 + i];
    }
    const T dp = g.gm1 * (T(0.5) * q2 * dU[0] - udm + dU[D + 1]);
    const T rdun = ndm - un * dU[0];  // rho * (linearised normal-velocity jump)
    const T i2c2 = T(0.5) / c2;
    am = (dp - c * rdun) * i2c2;
    ap = (dp + c * rdun) * i2c2;
  }
  // r_s for s = -1 / +1
  __host__ __device__ __forceinline__ void r(int s, const N (&nh)[D], T (&R)[D + 2]) const {
    const T sc = s > 0 ? c : -c;
    R[0] = T(1);
#pragma unroll
    for (int i = 0; i < D; ++i) R[1 + i] = u[i] + sc * T(nh[i]);
    R[D + 1] = H + sc * un;
  }
};

// Vijayasundaram flux through the area normal nv (own side UL outward).
// UNIT: nv is known to be a unit vector (box faces), so |nv| is not formed.
template <int D, typename T, typename N, bool UNIT = false>
__host__ __device__ __forceinline__ void vij_flux(const T (&UL)[D + 2], const T (&UR)[D + 2], const N (&nv)[D],
                                                  const Gas<T>& g, T (&F)[D + 2]) {
  constexpr int nf = D + 2;
  N sJ = N(1), nh[D];
  unit_of<D, N, UNIT>(nv, sJ, nh);
  T Ub[nf], dU[nf];
#pragma unroll
  for (int f = 0; f < nf; ++f) {
    Ub[f] = T(0.5) * (UL[f] + UR[f]);
    dU[f] = UL[f] - UR[f];
  }
  conv_flux_normal<D, T, N>(Ub, nv, g, F);
  const Waves<D, T, N> w(Ub, dU, nh, g);
  const T l0 = fabs(w.un), lm = fabs(w.un - w.c), lp = fabs(w.un + w.c);
  T rm[nf], rp[nf];
  w.r(-1, nh, rm);
  w.r(1, nh, rp);
  const T cm = (lm - l0) * w.am, cp = (lp - l0) * w.ap;
  const T hs = T(0.5) * T(sJ);
#pragma unroll
  for (int f = 0; f < nf; ++f) F[f] += hs * (l0 * dU[f] + cm * rm[f] + cp * rp[f]);
}

// Farfield boundary state U_Gamma (App. B.1.1) for the area normal nv.
template <int D, typename T, typename N, bool UNIT = false>
__host__ __device__ __forceinline__ void farfield_state(const T (&U)[D + 2], const T (&Ui)[D + 2], const N (&nv)[D],
                                                        const Gas<T>& g, T (&UG)[D + 2]) {
  constexpr int nf = D + 2;
  N sJ = N(1), nh[D];
  unit_of<D, N, UNIT>(nv, sJ, nh);
  T dU[nf];
#pragma unroll
  for (int f = 0; f < nf; ++f) dU[f] = U[f] - Ui[f];
  const Waves<D, T, N> w(U, dU, nh, g);
  T rm[nf], rp[nf];
  w.r(-1, nh, rm);
  w.r(1, nh, rp);
  const bool om = !(w.un - w.c < T(0)), o0 = !(w.un < T(0)), op = !(w.un + w.c < T(0));
#pragma unroll
  for (int f = 0; f < nf; ++f) {
    const T am = w.am * rm[f], ap = w.ap * rp[f];
    T v = Ui[f];
    if (om) v += am;
    if (op) v += ap;
    if (o0) v += dU[f] - am - ap;
    UG[f] = v;
  }
}

// K(U)(delta (x) nv) in every direction: F^nu(U, Q[c][f] = nv_c delta_f).
template <int D, typename T, typename N>
__host__ __device__ __forceinline__ void k_product(const T (&U)[D + 2], const T (&delta)[D + 2], const N (&nv)[D],
                                                   const Gas<T>& g, T (&K)[D][D + 2]) {
  T Q[D][D + 2];
#pragma unroll
  for (int c = 0; c < D; ++c)
#pragma unroll
    for (int f = 0; f < D + 2; ++f) Q[c][f] = T(nv[c]) * delta[f];
  visc_flux_all<D, T>(U, Q, g, K);
}

// The axis A and sign s of a box normal nv = s e_A (its other components are
// exactly zero), chosen by selects.
template <int D, typename N>
__host__ __device__ __forceinline__ int axis_of(const N (&nv)[D]) {
  int A = 0;
#pragma unroll
  for (int i = 1; i < D; ++i) A = nv[i] != N(0) ? i : A;
  return A;
}

// K(U)(delta (x) nv) for the axis normal nv = s e_0: the gradient n (x) delta
// has one non-zero row, d_0 u_i = s (delta_{1+i} - u_i delta_0) / rho =: d_i,
// so div u = d_0, tau = mu (d e_0^T + e_0 d^T) + lambda d_0 I, and the energy
// gradient is non-zero along 0 only.  About a quarter of the arithmetic of
// the full flux at a general gradient.
template <int D, typename T>
__host__ __device__ __forceinline__ void k_product_axis0(const T (&U)[D + 2], const T (&delta)[D + 2], T s,
                                                         const Gas<T>& g, T (&K)[D][D + 2]) {
  const T ir = T(1) / U[0];
  T u[D], d[D], ud = T(0);
#pragma unroll
  for (int i = 0; i < D; ++i) u[i] = U[1 + i] * ir;
  const T Et = U[D + 1] * ir;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    d[i] = s * (delta[1 + i] - u[i] * delta[0]) * ir;
    ud += u[i] * d[i];
  }
  const T ge = s * (delta[D + 1] - Et * delta[0]) * ir - ud;
  const T t00 = g.mu * (d[0] + d[0]) + g.lam * d[0];
  K[0][0] = T(0);
  K[0][1] = t00;
  T w = t00 * u[0];
#pragma unroll
  for (int j = 1; j < D; ++j) {
    const T t = g.mu * d[j];
    K[0][1 + j] = t;
    w += t * u[j];
  }
  K[0][D + 1] = w + g.kcv * ge;
  const T ld = g.lam * d[0];
#pragma unroll
  for (int i = 1; i < D; ++i) {
    const T t = g.mu * d[i];
    K[i][0] = T(0);
    K[i][1] = t;
#pragma unroll
    for (int j = 1; j < D; ++j) K[i][1 + j] = j == i ? ld : T(0);
    K[i][D + 1] = t * u[0] + ld * u[i];
  }
}

// k_product for a box normal nv = s e_A given at run time: the axes are
// relabelled so that A becomes 0 (selects, no branches), k_product_axis0 is
// applied and the result is relabelled back.
template <int D, typename T, typename N>
__host__ __device__ __forceinline__ void k_product_axis(const T (&U)[D + 2], const T (&delta)[D + 2], const N (&nv)[D],
                                                        const Gas<T>& g, T (&K)[D][D + 2]) {
  const int A = axis_of<D, N>(nv);
  const T s = T(by_shift<D>(A, [&](int k) { return nv[k]; }));
  T Ur[D + 2], dr[D + 2], Kr[D][D + 2];
  relabel_state<D, T>(U, A, Ur);
  relabel_state<D, T>(delta, A, dr);
  k_product_axis0<D, T>(Ur, dr, s, g, Kr);
  relabel_grad<D, T>(Kr, (D - A) % D, K);
}

// Cotangent of k_product_axis0: Kb -> Ub, deltab (accumulated), the reverse
// of its steps.
template <int D, typename S>
__host__ __device__ __forceinline__ void k_product_axis0_vjp(const S (&U)[D + 2], const S (&delta)[D + 2], S s,
                                                             const S (&Kb)[D][D + 2], const Gas<S>& g,
                                                             S (&Ub)[D + 2], S (&deltab)[D + 2]) {
  const S ir = S(1) / U[0];
  S u[D], nd[D], d[D];
#pragma unroll
  for (int i = 0; i < D; ++i) u[i] = U[1 + i] * ir;
  const S Et = U[D + 1] * ir;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    nd[i] = s * (delta[1 + i] - u[i] * delta[0]);
    d[i] = nd[i] * ir;
  }
  const S nge = s * (delta[D + 1] - Et * delta[0]);
  const S t00 = g.mu * (d[0] + d[0]) + g.lam * d[0];
  // K[0][1] = t00, K[0][1+j] = mu d_j, K[0][D+1] = t00 u_0 + sum_j mu d_j u_j + kcv ge,
  // K[i][1] = mu d_i, K[i][1+i] = lam d_0, K[i][D+1] = mu d_i u_0 + lam d_0 u_i
  const S e0 = Kb[0][D + 1];
  const S geb = g.kcv * e0;
  const S t00b = Kb[0][1] + e0 * u[0];
  S db[D], ub[D];
  ub[0] = e0 * t00;
  db[0] = g.mu * (t00b + t00b) + g.lam * t00b;
#pragma unroll
  for (int j = 1; j < D; ++j) {
    const S ej = Kb[j][D + 1];
    db[j] = g.mu * (Kb[0][1 + j] + e0 * u[j] + Kb[j][1] + ej * u[0]);
    ub[j] = g.mu * e0 * d[j] + g.lam * ej * d[0];
    ub[0] += g.mu * ej * d[j];
    db[0] += g.lam * (Kb[j][1 + j] + ej * u[j]);
  }
  // ge = nge ir - sum_i u_i d_i, nge = s (delta_E - Et delta_0)
  S irb = geb * nge;
  const S cg = geb * s * ir;
  deltab[D + 1] += cg;
  deltab[0] -= Et * cg;
  const S Etb = -delta[0] * cg;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    ub[i] -= geb * d[i];
    db[i] -= geb * u[i];
  }
  // d_i = nd_i ir, nd_i = s (delta_{1+i} - u_i delta_0)
#pragma unroll
  for (int i = 0; i < D; ++i) {
    irb += db[i] * nd[i];
    const S rs = s * db[i] * ir;
    deltab[1 + i] += rs;
    deltab[0] -= u[i] * rs;
    ub[i] -= delta[0] * rs;
  }
  // u_i = m_i ir, Et = E ir, ir = 1 / rho
#pragma unroll
  for (int i = 0; i < D; ++i) {
    Ub[1 + i] += ub[i] * ir;
    irb += ub[i] * U[1 + i];
  }
  Ub[D + 1] += Etb * ir;
  irb += Etb * U[D + 1];
  Ub[0] -= irb * ir * ir;
}

// Cotangent of k_product_axis: Ub += (dK/dU)^T Kb, deltab += (dK/ddelta)^T Kb.
template <int D, typename S>
__host__ __device__ __forceinline__ void k_product_axis_vjp(const S (&U)[D + 2], const S (&delta)[D + 2],
                                                            const S (&nv)[D], const S (&Kb)[D][D + 2],
                                                            const Gas<S>& g, S (&Ub)[D + 2], S (&deltab)[D + 2]) {
  constexpr int nf = D + 2;
  const int A = axis_of<D, S>(nv);
  const S s = by_shift<D>(A, [&](int k) { return nv[k]; });
  S Ur[nf], dr[nf], Kbr[D][nf], Ubr[nf], dbr[nf], t[nf];
  relabel_state<D, S>(U, A, Ur);
  relabel_state<D, S>(delta, A, dr);
  relabel_grad<D, S>(Kb, A, Kbr);
#pragma unroll
  for (int f = 0; f < nf; ++f) Ubr[f] = dbr[f] = S(0);
  k_product_axis0_vjp<D, S>(Ur, dr, s, Kbr, g, Ubr, dbr);
  const int Ai = (D - A) % D;
  relabel_state<D, S>(Ubr, Ai, t);
#pragma unroll
  for (int f = 0; f < nf; ++f) Ub[f] += t[f];
  relabel_state<D, S>(dbr, Ai, t);
#pragma unroll
  for (int f = 0; f < nf; ++f) deltab[f] += t[f];
}

// Mirror state (rho, m - 2 (m.n) n, rho E) for a normal of another scalar type.
template <int D, typename T, typename N>
__host__ __device__ __forceinline__ void mirror_state_n(const T (&U)[D + 2], const N (&nv)[D], T (&R)[D + 2]) {
  N n2 = N(0);
  T mn = T(0);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    n2 += nv[i] * nv[i];
    mn += U[1 + i] * T(nv[i]);
  }
  const T c = T(2) * mn / T(n2);
  R[0] = U[0];
#pragma unroll
  for (int i = 0; i < D; ++i) R[1 + i] = U[1 + i] - c * T(nv[i]);
  R[D + 1] = U[D + 1];
}

// Kinds of face for the face function.
enum { DGIP_INTERIOR = 0, DGIP_WALL = 1, DGIP_FARFIELD = 2 };

// The state-dependent part of the DG-IP numerical flux of one face point and
// the adjoint-consistency vectors of both sides (unit or area normal nv, own
// side L outward), excluding the viscous average -(G^L - G^R)/2 (linear in the
// gradient traces, added by the callers):
//   interior: F = Vij(UL, UR) + tau (K(UL) + K(UR))(delta (x) n).n / (2|n|),
//             HL = cL K(UL)(delta (x) n) (interface: (K(UL) + K(UR))/2 ...),
//   wall:     F = Vij(UL, mirror(UL)) + tau K_w(UL)(dw (x) n).n / |n|, HL = K_w(UL)(dw (x) n),
//   farfield: F = F^c(U_Gamma).n + tau K(U_inf)(di (x) n).n / |n|, HL = K(U_inf)(di (x) n),
// delta = UL - UR, dw = UL - U_w(UL), di = UL - U_inf.  gw: the gas with kappa = 0.
// AXIS: nv = +-e_A (box faces), so |nv| is not formed; KAXIS (with AXIS):
// the K-products also take the rank-one axis form (FP64 kernels, bound by
// the FP64 pipe; in FP32 its selects and registers cost more than the
// arithmetic it saves).
template <int D, typename T, typename N, bool VISC, int KIND, bool AXIS = false, bool KAXIS = AXIS>
__host__ __device__ __forceinline__ void dgip_face_fn(const T (&UL)[D + 2], const T (&UR)[D + 2], const N (&nv)[D],
                                                      const Gas<T>& g, const Gas<T>& gw, N tau_over_s, bool ifL,
                                                      bool ifR, T (&F)[D + 2], T (&HL)[D][D + 2],
                                                      T (&HR)[D][D + 2]) {
  constexpr int nf = D + 2;
  if (KIND == DGIP_INTERIOR) {
    vij_flux<D, T, N, AXIS>(UL, UR, nv, g, F);
    if (VISC) {
      T dl[nf];
#pragma unroll
      for (int f = 0; f < nf; ++f) dl[f] = UL[f] - UR[f];
      T KL[D][nf], KR[D][nf];
      if (KAXIS) {
        k_product_axis<D, T, N>(UL, dl, nv, g, KL);
        k_product_axis<D, T, N>(UR, dl, nv, g, KR);
      } else {
        k_product<D, T, N>(UL, dl, nv, g, KL);
        k_product<D, T, N>(UR, dl, nv, g, KR);
      }
      const T h = T(0.5) * T(tau_over_s);
#pragma unroll
      for (int f = 0; f < nf; ++f) {
        T s = T(0);
#pragma unroll
        for (int c = 0; c < D; ++c) s += (KL[c][f] + KR[c][f]) * T(nv[c]);
        F[f] += h * s;
      }
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int f = 0; f < nf; ++f) {
          const T avg = T(0.5) * (KL[c][f] + KR[c][f]);
          HL[c][f] = ifL ? avg : T(0.5) * KL[c][f];
          HR[c][f] = ifR ? avg : T(0.5) * KR[c][f];
        }
    }
  } else if (KIND == DGIP_WALL) {
    T Um[nf];
    mirror_state_n<D, T, N>(UL, nv, Um);
    vij_flux<D, T, N, AXIS>(UL, Um, nv, g, F);
    if (VISC) {
      T Uw[nf], dw[nf];
      wall_state<D, T>(UL, Uw);
#pragma unroll
      for (int f = 0; f < nf; ++f) dw[f] = UL[f] - Uw[f];
      if (KAXIS) k_product_axis<D, T, N>(UL, dw, nv, gw, HL);
      else k_product<D, T, N>(UL, dw, nv, gw, HL);
#pragma unroll
      for (int f = 0; f < nf; ++f) {
        T s = T(0);
#pragma unroll
        for (int c = 0; c < D; ++c) s += HL[c][f] * T(nv[c]);
        F[f] += T(tau_over_s) * s;
      }
    }
  } else {  // farfield: UR holds U_inf
    T UG[nf];
    farfield_state<D, T, N, AXIS>(UL, UR, nv, g, UG);
    conv_flux_normal<D, T, N>(UG, nv, g, F);
    if (VISC) {
      T di[nf];
#pragma unroll
      for (int f = 0; f < nf; ++f) di[f] = UL[f] - UR[f];
      if (KAXIS) k_product_axis<D, T, N>(UR, di, nv, g, HL);
      else k_product<D, T, N>(UR, di, nv, g, HL);
#pragma unroll
      for (int f = 0; f < nf; ++f) {
        T s = T(0);
#pragma unroll
        for (int c = 0; c < D; ++c) s += HL[c][f] * T(nv[c]);
        F[f] += T(tau_over_s) * s;
      }
    }
  }
}


// Reverse-mode adjoint of dgip_face_fn on an interior face: given the
// cotangents Fb of F and HLb, HRb of the adjoint-consistency vectors,
// ULb += (dF/dUL)^T Fb + (dHL/dUL)^T HLb + (dHR/dUL)^T HRb and likewise URb.
// Written statement by statement against vij_flux (F_n(Ubar) through
// conv_flux_all_vjp, then the wave sum |A| dU / 2 reversed through the
// characteristic quantities of Waves) and the K-products (visc_flux_all_vjp at
// the rank-one gradient nv (x) delta; KAXIS: k_product_axis_vjp).  d|x|/dx = sign(x), sign(0) = 0, as the
// dual numbers take it.
template <int D, typename S, bool VISC, bool AXIS = false, bool KAXIS = AXIS>
__host__ __device__ __forceinline__ void dgip_face_interior_vjp(const S (&UL)[D + 2], const S (&UR)[D + 2],
                                                                const S (&nv)[D], const Gas<S>& g, S tau_over_s,
                                                                bool ifL, bool ifR, const S (&Fb)[D + 2],
                                                                const S (&HLb)[D][D + 2], const S (&HRb)[D][D + 2],
                                                                S (&ULb)[D + 2], S (&URb)[D + 2]) {
  constexpr int nf = D + 2;
  S sJ = S(1), nh[D];
  unit_of<D, S, AXIS>(nv, sJ, nh);
  S Ub[nf], dU[nf];
#pragma unroll
  for (int f = 0; f < nf; ++f) {
    Ub[f] = S(0.5) * (UL[f] + UR[f]);
    dU[f] = UL[f] - UR[f];
  }
  // forward: characteristic quantities at Ubar
  const S rho = Ub[0], ir = S(1) / rho;
  S u[D], q2 = S(0), un = S(0), udm = S(0), ndm = S(0);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    u[i] = Ub[1 + i] * ir;
    q2 += u[i] * u[i];
    un += u[i] * nh[i];
  }
  const S p = g.gm1 * (Ub[D + 1] - S(0.5) * rho * q2);
  const S c2 = g.gamma * p * ir;
  const S c = sqrt(c2);
  const S H = (Ub[D + 1] + p) * ir;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    udm += u[i] * dU[1 + i];
    ndm += nh[i] * dU[1 + i];
  }
  const S dp = g.gm1 * (S(0.5) * q2 * dU[0] - udm + dU[D + 1]);
  const S rdun = ndm - un * dU[0];
  const S i2c2 = S(0.5) / c2;
  const S am = (dp - c * rdun) * i2c2, ap = (dp + c * rdun) * i2c2;
  const S l0 = fabs(un), lm = fabs(un - c), lp = fabs(un + c);
  const S cm = (lm - l0) * am, cp = (lp - l0) * ap;
  // reverse of F += hs (l0 dU + cm rm + cp rp)
  const S hs = S(0.5) * sJ;
  S dUb[nf], l0b = S(0), cmb = S(0), cpb = S(0), Hb = S(0), unb = S(0), cb = S(0), ub[D];
  {
    S G[nf];
#pragma unroll
    for (int f = 0; f < nf; ++f) {
      G[f] = hs * Fb[f];
      dUb[f] = l0 * G[f];
      l0b += G[f] * dU[f];
    }
    // rm = (1, u - c nh, H - c un), rp = (1, u + c nh, H + c un)
    cmb = G[0];
    cpb = G[0];
    S nr = S(0);  // sum_i nh_i (G_{1+i} cp - G_{1+i} cm) folded below
#pragma unroll
    for (int i = 0; i < D; ++i) {
      cmb += G[1 + i] * (u[i] - c * nh[i]);
      cpb += G[1 + i] * (u[i] + c * nh[i]);
      ub[i] = (cm + cp) * G[1 + i];
      nr += nh[i] * G[1 + i];
    }
    cmb += G[D + 1] * (H - c * un);
    cpb += G[D + 1] * (H + c * un);
    Hb = (cm + cp) * G[D + 1];
    cb = (cp - cm) * (nr + un * G[D + 1]);
    unb = c * (cp - cm) * G[D + 1];
  }
  // cm = (lm - l0) am, cp = (lp - l0) ap
  const S lmb = cmb * am, lpb = cpb * ap;
  l0b -= cmb * am + cpb * ap;
  const S amb = cmb * (lm - l0), apb = cpb * (lp - l0);
  // l0 = |un|, lm = |un - c|, lp = |un + c|
  const S sm = sgn(un - c), sp = sgn(un + c);
  unb += sgn(un) * l0b + sm * lmb + sp * lpb;
  cb += sp * lpb - sm * lmb;
  // am = (dp - c rdun) i2c2, ap = (dp + c rdun) i2c2
  const S dpb = (amb + apb) * i2c2;
  const S rdunb = c * (apb - amb) * i2c2;
  cb += rdun * (apb - amb) * i2c2;
  const S i2c2b = amb * (dp - c * rdun) + apb * (dp + c * rdun);
  S c2b = -S(2) * i2c2b * i2c2 * i2c2;  // d(1/(2 c2)) = -2 (1/(2 c2))^2 dc2
  // rdun = ndm - un dU0
  const S ndmb = rdunb;
  unb -= dU[0] * rdunb;
  dUb[0] -= un * rdunb;
  // dp = gm1 (q2 dU0 / 2 - udm + dU_E)
  S q2b = g.gm1 * S(0.5) * dU[0] * dpb;
  dUb[0] += g.gm1 * S(0.5) * q2 * dpb;
  const S udmb = -g.gm1 * dpb;
  dUb[D + 1] += g.gm1 * dpb;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    ub[i] += udmb * dU[1 + i];
    dUb[1 + i] += udmb * u[i] + ndmb * nh[i];
  }
  // c = sqrt(c2), c2 = gamma p ir, H = (E + p) ir
  c2b += cb * S(0.5) / c;
  const S pb0 = Hb * ir + c2b * g.gamma * ir;
  S Eb = Hb * ir;
  S irb = Hb * (Ub[D + 1] + p) + c2b * g.gamma * p;
  // p = gm1 (E - rho q2 / 2)
  Eb += g.gm1 * pb0;
  S rhob = -g.gm1 * S(0.5) * q2 * pb0;
  q2b -= g.gm1 * S(0.5) * rho * pb0;
  // un = u . nh, q2 = u . u, u = m ir
  S Ubb[nf];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    ub[i] += nh[i] * unb + S(2) * u[i] * q2b;
    Ubb[1 + i] = ub[i] * ir;
    irb += ub[i] * Ub[1 + i];
  }
  rhob -= irb * ir * ir;
  Ubb[0] = rhob;
  Ubb[D + 1] = Eb;
  {  // F_n(Ubar) = sum_c nv_c F_c(Ubar)
    S Fcb[D][nf];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int f = 0; f < nf; ++f) Fcb[a][f] = nv[a] * Fb[f];
    conv_flux_all_vjp<D, S>(Ub, Fcb, g, Ubb);
  }
#pragma unroll
  for (int f = 0; f < nf; ++f) {
    ULb[f] += S(0.5) * Ubb[f] + dUb[f];
    URb[f] += S(0.5) * Ubb[f] - dUb[f];
  }
  if (VISC) {
    // F += (tau / 2) sum_c (KL + KR)[c] nv_c; HL = KL / 2 (+ KR / 2 at an
    // interface), HR = KR / 2 (+ KL / 2); K(U) = F^nu(U, nv (x) delta)
    const S h = S(0.5) * tau_over_s;
    S KLb[D][nf], KRb[D][nf];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int f = 0; f < nf; ++f) {
        const S fb = h * nv[a] * Fb[f];
        KLb[a][f] = fb + S(0.5) * HLb[a][f] + (ifR ? S(0.5) * HRb[a][f] : S(0));
        KRb[a][f] = fb + S(0.5) * HRb[a][f] + (ifL ? S(0.5) * HLb[a][f] : S(0));
      }
    S db[nf];
#pragma unroll
    for (int f = 0; f < nf; ++f) db[f] = S(0);
    if constexpr (KAXIS) {
      k_product_axis_vjp<D, S>(UL, dU, nv, KLb, g, ULb, db);
      k_product_axis_vjp<D, S>(UR, dU, nv, KRb, g, URb, db);
    } else {
      S Q[D][nf], QLb[D][nf], QRb[D][nf];
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int f = 0; f < nf; ++f) {
          Q[a][f] = nv[a] * dU[f];
          QLb[a][f] = S(0);
          QRb[a][f] = S(0);
        }
      visc_flux_all_vjp<D, S>(UL, Q, KLb, g, ULb, QLb);
      visc_flux_all_vjp<D, S>(UR, Q, KRb, g, URb, QRb);
#pragma unroll
      for (int f = 0; f < nf; ++f)
#pragma unroll
        for (int a = 0; a < D; ++a) db[f] += nv[a] * (QLb[a][f] + QRb[a][f]);
    }
#pragma unroll
    for (int f = 0; f < nf; ++f) {
      ULb[f] += db[f];
      URb[f] -= db[f];
    }
  }
}

}  // namespace dgx
