// Host check (no GPU) of the axis-normal viscous flux of physics.cuh: the
// one row visc_flux_axis and its hand-derived adjoint visc_flux_axis_vjp
// against the full flux visc_flux_normal (and its adjoint) through the same
// axis normal, on random states and gradients, 2D and 3D, both orientations.
#include <cstdio>
#include <cmath>
#include <random>
#include "physics.cuh"
using namespace dgx;
template <int D>
int run(std::mt19937& rng) {
  std::uniform_real_distribution<double> d(-1.0, 1.0);
  Gas<double> g{};
  g.gamma = 1.4; g.gm1 = 0.4; g.mu = 0.013; g.lam = -2.0 * 0.013 / 3; g.kcv = 1.4 * 0.013 / 0.72;
  double worst = 0, worstb = 0;
  for (int trial = 0; trial < 2000; ++trial) {
    double U[D + 2], Q[D][D + 2], Gb[D + 2];
    U[0] = 1.0 + 0.5 * d(rng);
    for (int i = 0; i < D; ++i) U[1 + i] = d(rng);
    U[D + 1] = 3.0 + d(rng);
    for (int a = 0; a < D; ++a) for (int f = 0; f < D + 2; ++f) Q[a][f] = d(rng);
    for (int f = 0; f < D + 2; ++f) Gb[f] = d(rng);
    for (int A = 0; A < D; ++A) for (int sg = -1; sg <= 1; sg += 2) {
      double nv[D] = {};
      nv[A] = sg;
      double G1[D + 2], G2[D + 2];
      visc_flux_normal<D, double>(U, Q, nv, g, G1);
      visc_flux_axis_rt<D, double>(U, Q, A, (double)sg, g, G2);
      for (int f = 0; f < D + 2; ++f) worst = fmax(worst, fabs(G1[f] - G2[f]));
      double Ub1[D + 2] = {}, Ub2[D + 2] = {}, Qb1[D][D + 2] = {}, Qb2[D][D + 2] = {};
      visc_flux_normal_vjp<D, double>(U, Q, nv, Gb, g, Ub1, Qb1);
      visc_flux_axis_vjp_rt<D, double>(U, Q, A, (double)sg, Gb, g, Ub2, Qb2);
      for (int f = 0; f < D + 2; ++f) worstb = fmax(worstb, fabs(Ub1[f] - Ub2[f]));
      for (int a = 0; a < D; ++a) for (int f = 0; f < D + 2; ++f) worstb = fmax(worstb, fabs(Qb1[a][f] - Qb2[a][f]));
    }
  }
  printf("D=%d forward max diff %.3e, vjp max diff %.3e\n", D, worst, worstb);
  return worst < 1e-13 && worstb < 1e-12 ? 0 : 1;
}
int main() {
  std::mt19937 rng(7);
  int r = run<2>(rng) + run<3>(rng);
  printf(r ? "FAIL\n" : "OK\n");
  return r;
}
