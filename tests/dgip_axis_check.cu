// Host check (no GPU) of the box-face form of the DG-IP face function of
// dgip_physics.cuh: with an axis normal +-e_A the face function takes the
// rank-one axis K-products (relabelled to axis 0) and skips |n|; its values,
// their forward-mode derivatives (dual numbers, as the boundary adjoint uses
// them) and the hand-derived interior adjoint must equal the general form's
// on random states, every axis and both orientations, 2D and 3D.
#include <cmath>
#include <cstdio>
#include <random>
#include "dgip_physics.cuh"
using namespace dgx;

template <int D, int KIND>
double forward_diff(std::mt19937& rng, const Gas<double>& g, const Gas<double>& gw, double& worst_d) {
  constexpr int nf = D + 2;
  using T = Dual<double, 1>;
  std::uniform_real_distribution<double> d(-1.0, 1.0);
  double worst = 0;
  for (int trial = 0; trial < 500; ++trial) {
    double UL[nf], UR[nf];
    UL[0] = 1.0 + 0.5 * d(rng);
    UR[0] = 1.0 + 0.5 * d(rng);
    for (int i = 0; i < D; ++i) {
      UL[1 + i] = 0.5 * d(rng);
      UR[1 + i] = 0.5 * d(rng);
    }
    UL[D + 1] = 3.0 + d(rng);
    UR[D + 1] = 3.0 + d(rng);
    for (int A = 0; A < D; ++A)
      for (int sg = -1; sg <= 1; sg += 2) {
        double nv[D] = {};
        nv[A] = sg;
        for (int ifl = 0; ifl < 2; ++ifl) {
          double F1[nf], F2[nf], HL1[D][nf], HL2[D][nf], HR1[D][nf], HR2[D][nf];
          dgip_face_fn<D, double, double, true, KIND, false>(UL, UR, nv, g, gw, 7.0, ifl, false, F1, HL1, HR1);
          dgip_face_fn<D, double, double, true, KIND, true>(UL, UR, nv, g, gw, 7.0, ifl, false, F2, HL2, HR2);
          for (int f = 0; f < nf; ++f) worst = fmax(worst, fabs(F1[f] - F2[f]));
          for (int c = 0; c < D; ++c)
            for (int f = 0; f < nf; ++f) {
              worst = fmax(worst, fabs(HL1[c][f] - HL2[c][f]));
              if (KIND == 0) worst = fmax(worst, fabs(HR1[c][f] - HR2[c][f]));
            }
        }
        // tangents along each input component of the own side
        for (int k = 0; k < nf; ++k) {
          T L[nf], R[nf], F1[nf], F2[nf], HL1[D][nf], HL2[D][nf], HR1[D][nf], HR2[D][nf];
          for (int f = 0; f < nf; ++f) {
            L[f] = T(UL[f]);
            R[f] = T(UR[f]);
          }
          L[k].d[0] = 1.0;
          const Gas<T> gd = gas_as<T, double>(g), gwd = gas_as<T, double>(gw);
          dgip_face_fn<D, T, double, true, KIND, false>(L, R, nv, gd, gwd, 7.0, false, false, F1, HL1, HR1);
          dgip_face_fn<D, T, double, true, KIND, true>(L, R, nv, gd, gwd, 7.0, false, false, F2, HL2, HR2);
          for (int f = 0; f < nf; ++f) worst_d = fmax(worst_d, fabs(F1[f].d[0] - F2[f].d[0]));
          for (int c = 0; c < D; ++c)
            for (int f = 0; f < nf; ++f) worst_d = fmax(worst_d, fabs(HL1[c][f].d[0] - HL2[c][f].d[0]));
        }
      }
  }
  return worst;
}

template <int D>
double adjoint_diff(std::mt19937& rng, const Gas<double>& g) {
  constexpr int nf = D + 2;
  std::uniform_real_distribution<double> d(-1.0, 1.0);
  double worst = 0;
  for (int trial = 0; trial < 500; ++trial) {
    double UL[nf], UR[nf], Fb[nf], HLb[D][nf], HRb[D][nf];
    UL[0] = 1.0 + 0.5 * d(rng);
    UR[0] = 1.0 + 0.5 * d(rng);
    for (int i = 0; i < D; ++i) {
      UL[1 + i] = 0.5 * d(rng);
      UR[1 + i] = 0.5 * d(rng);
    }
    UL[D + 1] = 3.0 + d(rng);
    UR[D + 1] = 3.0 + d(rng);
    for (int f = 0; f < nf; ++f) {
      Fb[f] = d(rng);
      for (int c = 0; c < D; ++c) {
        HLb[c][f] = d(rng);
        HRb[c][f] = d(rng);
      }
    }
    for (int A = 0; A < D; ++A)
      for (int sg = -1; sg <= 1; sg += 2)
        for (int ifc = 0; ifc < 3; ++ifc) {
          double nv[D] = {};
          nv[A] = sg;
          const bool ifL = ifc == 1, ifR = ifc == 2;
          double ULb1[nf] = {}, URb1[nf] = {}, ULb2[nf] = {}, URb2[nf] = {};
          dgip_face_interior_vjp<D, double, true, false>(UL, UR, nv, g, 7.0, ifL, ifR, Fb, HLb, HRb, ULb1, URb1);
          dgip_face_interior_vjp<D, double, true, true>(UL, UR, nv, g, 7.0, ifL, ifR, Fb, HLb, HRb, ULb2, URb2);
          for (int f = 0; f < nf; ++f) {
            worst = fmax(worst, fabs(ULb1[f] - ULb2[f]));
            worst = fmax(worst, fabs(URb1[f] - URb2[f]));
          }
        }
  }
  return worst;
}

template <int D>
int run(std::mt19937& rng) {
  Gas<double> g{};
  g.gamma = 1.4; g.gm1 = 0.4; g.mu = 0.013; g.lam = -2.0 * 0.013 / 3; g.kcv = 1.4 * 0.013 / 0.72;
  Gas<double> gw = g;
  gw.kcv = 0.0;
  double wd = 0;
  const double fi = forward_diff<D, DGIP_INTERIOR>(rng, g, gw, wd);
  const double fw = forward_diff<D, DGIP_WALL>(rng, g, gw, wd);
  const double ff = forward_diff<D, DGIP_FARFIELD>(rng, g, gw, wd);
  const double ad = adjoint_diff<D>(rng, g);
  printf("D=%d interior %.3e wall %.3e farfield %.3e tangents %.3e adjoint %.3e\n", D, fi, fw, ff, wd, ad);
  return fi < 1e-12 && fw < 1e-12 && ff < 1e-12 && wd < 1e-11 && ad < 1e-11 ? 0 : 1;
}

int main() {
  std::mt19937 rng(11);
  const int r = run<2>(rng) + run<3>(rng);
  printf(r ? "FAIL\n" : "OK\n");
  return r;
}
