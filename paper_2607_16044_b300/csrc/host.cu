// Host runtime of the dgx library: handle, 1D basis, geometry (FP64), mesh
// validation, unique-face list, workspace layout and the C ABI of dgx.h.
//
// Everything that depends only on the mesh is computed once here in FP64 and
// uploaded in the handle's precision; the compute entry points only enqueue
// kernels on the caller's stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <new>
#include <vector>

#include "../../include/dgx.h"
#include "dispatch.h"
#include "flops.h"
#include "vjp.cuh"
#include "dgip.cuh"
#include "mms.cuh"
#include "batchp.h"
#include "hdg.h"
#include "oi.h"

using dgx::Tab;

struct dgx_handle {
  dgx_problem_desc desc;
  int d, p, n, N, nf, nfp, NF, E, T;
  bool viscous, fp64;
  size_t s;  // bytes per scalar
  const dgx::Table* tab;
  void* d_tabs = nullptr;      // Tab<S>[6]
  unsigned* d_flags = nullptr;
  // mesh
  bool has_mesh = false, curv = false;
  bool geo_override = false;  // metrics given by dgx_set_geometry (not derivable from the host mesh copies)
  int nFaces = 0;
  int* d_nb = nullptr;
  int8_t* d_nbf = nullptr;
  int8_t* d_ori = nullptr;
  int4* d_faces = nullptr;
  void* d_rh = nullptr;
  void* d_Ja = nullptr;
  void* d_iJ = nullptr;
  void* d_SnE = nullptr;
  void* d_SnF = nullptr;
  dgx::Mesh<double> mesh64{};   // device views passed to the launch table
  dgx::Mesh<float> mesh32{};
  int nsm = 148;          // SMs of the device (persistent grids)
  int dev = 0;            // device that was current at dgx_create (owns every device table)
  uint32_t wait_polls = 1u << 22;  // consumer-wait bound of the persistent kernels
  bool pipeline = true;   // persistent TMA-fed kernels where the layout allows
  int contraction = DGX_CONTRACT_CUDA_CORE;  // engine of the forward element kernel
  // second stream and fork / join events of dgx_ark_step_adjoint
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // tile variant per kernel kind (autotuned; 1 = about 256 threads per CTA)
  int var[DGX_KERNEL_KINDS] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};  // 0..2: CTA tiles, 3: warp per element
  // per-kernel event profiler (tracing)
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<int> ev_kind;
  int64_t prof_launches[DGX_KERNEL_KINDS] = {};
  double prof_ms[DGX_KERNEL_KINDS] = {};
  // host copies of the mesh description (the batch runtime concatenates them)
  std::vector<int> h_nb;
  std::vector<int8_t> h_nbf, h_ori;
  std::vector<double> h_lo, h_size, h_xyz;
  // the paper's DG-IP scheme (Vijayasundaram + SIPG), box meshes
  bool dgip = false;
  double alpha = 1.0;          // SIPG penalty factor
  void* d_il = nullptr;        // [E] 1/l = |dT| / |T|, handle precision
  void* d_JaF = nullptr;       // curvilinear DG-IP: [E][2d][d][d][nfp] metric at the own face points
  void* d_iJF = nullptr;       // curvilinear DG-IP: [E][2d][nfp] 1/J there
  double* d_lo = nullptr;      // [E][d] box corners and sizes, FP64 (node coordinates)
  double* d_size = nullptr;
  bool has_farfield = false;   // the mesh has farfield faces (tag 1)
  bool has_uinf = false;
  double Uinf[5] = {};
  int8_t* d_mask = nullptr;    // explicit-element mask of the geometry split
  const dgx::DgipTable* dtab = nullptr;
  int pen_k = -1;              // degree k of tau = alpha (k+1)^2 / l (-1: this handle's p)
  // over-integration by an M-point rule: the degree-(M-1) DG-IP handle that
  // evaluates the collocated operator at the M points, and the 1D transfers
  dgx_handle* inner = nullptr;
  int Mq = 0;
  double oiI[dgx::OI_MAXQ * dgx::OI_MAXQ] = {};   // [M][n]  l_j(z_m)
  double oiP[dgx::OI_MAXQ * dgx::OI_MAXQ] = {};   // [n][M]  omega_m l_q(z_m) / w_q
  double oiPT[dgx::OI_MAXQ * dgx::OI_MAXQ] = {};  // [M][n]  Pi^T
  double oiIT[dgx::OI_MAXQ * dgx::OI_MAXQ] = {};  // [n][M]  I^T
  void* d_oiJq = nullptr;  // curved elements: [E][M^d] J at the M points (handle precision)
  // tableau
  int stages = 0;
  double A[dgx::MAXSTAGES * dgx::MAXSTAGES], b[dgx::MAXSTAGES], c[dgx::MAXSTAGES];
};

namespace {

// ---------------------------------------------------------------- 1D basis
// The compile-time basis of basis1d.h (the kernels use the same tables).
struct Basis {
  int n;
  std::vector<double> x, w, D, lm, lp;
};

Basis make_basis(int p) {
  const dgx::Basis1 b = dgx::make_basis1(p);
  Basis B;
  const int n = b.n;
  B.n = n;
  B.x.assign(b.x, b.x + n);
  B.w.assign(b.w, b.w + n);
  B.lm.assign(b.lm, b.lm + n);
  B.lp.assign(b.lp, b.lp + n);
  B.D.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) B.D[i * n + j] = b.D[i][j];
  return B;
}

template <typename S>
void fill_tab(int p, Tab<S>& t) {
  std::memset(&t, 0, sizeof(t));
  const dgx::Tab1<S> c = dgx::make_tab1<S>(p);
  constexpr int W = 6;  // Tab<S> holds degrees up to 5
  for (int i = 0; i < W; ++i)
    for (int j = 0; j < W; ++j) {
      t.D[i * W + j] = c.D[i][j];
      t.Dh[i * W + j] = c.Dh[i][j];
    }
  for (int j = 0; j < W; ++j) {
    t.lm[j] = c.lm[j];
    t.lp[j] = c.lp[j];
    t.Lm[j] = c.Lm[j];
    t.Lp[j] = c.Lp[j];
  }
}

int ipow(int b, int e) {
  int r = 1;
  while (e-- > 0) r *= b;
  return r;
}

int omap(int code, int fp, int n, int d) {
  if (d == 2) return (code & 1) ? n - 1 - fp : fp;
  int s = fp % n, t = fp / n;
  if (code & 4) std::swap(s, t);
  const int u = (code & 1) ? n - 1 - s : s;
  const int v = (code & 2) ? n - 1 - t : t;
  return u + n * v;
}

int pw(int n, int a) { return a == 0 ? 1 : (a == 1 ? n : (a == 2 ? n * n : n * n * n)); }
int node_of(int n, int m, int fp, int a) { return fp % pw(n, a) + m * pw(n, a) + (fp / pw(n, a)) * pw(n, a + 1); }
int fpoint_of(int n, int q, int a) { return q % pw(n, a) + (q / pw(n, a + 1)) * pw(n, a); }

template <typename T>
dgx_status upload(const std::vector<T>& v, void** dst) {
  if (*dst) cudaFree(*dst);
  *dst = nullptr;
  if (v.empty()) return DGX_OK;
  if (cudaMalloc(dst, v.size() * sizeof(T)) != cudaSuccess) return DGX_ENOMEM;
  if (cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) return DGX_ECUDA;
  return DGX_OK;
}

dgx_status upload_real(dgx_handle* h, const std::vector<double>& v, void** dst) {
  if (h->fp64) return upload(v, dst);
  std::vector<float> f(v.size());
  for (size_t i = 0; i < v.size(); ++i) f[i] = (float)v[i];
  return upload(f, dst);
}

void free_mesh(dgx_handle* h) {
  void* ptrs[] = {h->d_nb, h->d_nbf, h->d_ori, h->d_faces, h->d_rh, h->d_Ja, h->d_iJ, h->d_SnE, h->d_SnF,
                  h->d_il, h->d_lo, h->d_size, h->d_JaF, h->d_iJF, h->d_oiJq};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  h->d_il = nullptr;
  h->d_oiJq = nullptr;
  h->d_JaF = h->d_iJF = nullptr;
  h->d_lo = h->d_size = nullptr;
  h->has_farfield = false;
  h->d_nb = nullptr;
  h->d_nbf = nullptr;
  h->d_ori = nullptr;
  h->d_faces = nullptr;
  h->d_rh = h->d_Ja = h->d_iJ = h->d_SnE = h->d_SnF = nullptr;
  h->has_mesh = false;
}

// Element metrics Ja[E][a][c][N] = J dxi_a/dx_c and iJ[E][N] = 1/J (host, FP64)
// to the device, with the face normals they imply: each element's own
// outward area normals +-Ja_a traced to xi_a = +-1, and on every unique face
// the average (Sn^- - Sn^+)/2 of both sides' (the owner's face-point order).
dgx_status upload_metrics(dgx_handle* h, const std::vector<double>& Ja, const std::vector<double>& iJ,
                          const std::vector<int4>& faces) {
  const int E = h->E, d = h->d, n = h->n, N = h->N, NF = h->NF, nfp = h->nfp;
  const dgx::Basis1 B = dgx::make_basis1(h->p);
  std::vector<double> SnE((size_t)E * NF * d * nfp);
  for (int e = 0; e < E; ++e) {
    const double* JaE = &Ja[(size_t)e * d * d * N];
    for (int face = 0; face < NF; ++face) {
      const int a = face >> 1;
      const double* l = (face & 1) ? B.lp : B.lm;
      const double sgn = (face & 1) ? 1.0 : -1.0;
      for (int c = 0; c < d; ++c)
        for (int fp = 0; fp < nfp; ++fp) {
          double s = 0.0;
          for (int m = 0; m < n; ++m) s += l[m] * JaE[(a * d + c) * N + node_of(n, m, fp, a)];
          SnE[(((size_t)e * NF + face) * d + c) * nfp + fp] = sgn * s;
        }
    }
  }
  std::vector<double> SnF(faces.size() * d * nfp);
  for (size_t F = 0; F < faces.size(); ++F) {
    const int4 r = faces[F];
    const int em = r.x, ep = r.y, fm = r.z & 0xff, fo = (r.z >> 8) & 0xff, code = (r.z >> 16) & 0xff;
    for (int c = 0; c < d; ++c)
      for (int fp = 0; fp < nfp; ++fp) {
        const double own = SnE[(((size_t)em * NF + fm) * d + c) * nfp + fp];
        double v = own;
        if (ep >= 0) v = 0.5 * (own - SnE[(((size_t)ep * NF + fo) * d + c) * nfp + omap(code, fp, n, d)]);
        SnF[(F * d + c) * nfp + fp] = v;
      }
  }
  dgx_status st;
  if ((st = upload_real(h, Ja, &h->d_Ja)) != DGX_OK) return st;
  if ((st = upload_real(h, iJ, &h->d_iJ)) != DGX_OK) return st;
  if ((st = upload_real(h, SnE, &h->d_SnE)) != DGX_OK) return st;
  return upload_real(h, SnF, &h->d_SnF);
}

// DG-IP on curvilinear meshes: the metric terms and J traced to every own face
// point (JaF[E][2d][a][c][nfp], iJF = 1 / trace of J, as the face gradients
// and the contravariant adjoint-consistency vectors need them) and the
// characteristic length of the penalty, 1/l = |dT| / |T| with
// |T| = sum_q w_q J_q and |dT| = sum over faces of w_f |J dxi_a0/dx| (Gauss rules).
dgx_status upload_dgip_metrics(dgx_handle* h, const std::vector<double>& Ja, const std::vector<double>& iJ) {
  const int E = h->E, d = h->d, n = h->n, N = h->N, NF = h->NF, nfp = h->nfp;
  const dgx::Basis1 B = dgx::make_basis1(h->p);
  std::vector<double> JaF((size_t)E * NF * d * d * nfp), iJF((size_t)E * NF * nfp), il(E);
  for (int e = 0; e < E; ++e) {
    double vol = 0.0, area = 0.0;
    for (int q = 0; q < N; ++q) {
      double wq = 1.0;
      for (int a = 0; a < d; ++a) wq *= B.w[(q / pw(n, a)) % n];
      vol += wq / iJ[(size_t)e * N + q];
    }
    for (int face = 0; face < NF; ++face) {
      const int a0 = face >> 1;
      const double* l = (face & 1) ? B.lp : B.lm;
      const size_t fo = (size_t)e * NF + face;
      for (int fp = 0; fp < nfp; ++fp) {
        double Jf = 0.0;
        for (int m = 0; m < n; ++m) Jf += l[m] / iJ[(size_t)e * N + node_of(n, m, fp, a0)];
        iJF[fo * nfp + fp] = 1.0 / Jf;
        for (int a = 0; a < d; ++a)
          for (int c = 0; c < d; ++c) {
            double s = 0.0;
            for (int m = 0; m < n; ++m) s += l[m] * Ja[(((size_t)e * d + a) * d + c) * N + node_of(n, m, fp, a0)];
            JaF[((fo * d + a) * d + c) * nfp + fp] = s;
          }
        double wf = 1.0, sn = 0.0;  // tangential weights, |area normal|
        for (int a = 0, k = 0; a < d; ++a)
          if (a != a0) wf *= B.w[(fp / pw(n, k++)) % n];
        for (int c = 0; c < d; ++c) {
          const double v = JaF[((fo * d + a0) * d + c) * nfp + fp];
          sn += v * v;
        }
        area += wf * std::sqrt(sn);
      }
    }
    il[e] = area / vol;
  }
  dgx_status st;
  if ((st = upload_real(h, JaF, &h->d_JaF)) != DGX_OK) return st;
  if ((st = upload_real(h, iJF, &h->d_iJF)) != DGX_OK) return st;
  return upload_real(h, il, &h->d_il);
}

// Connectivity checks shared by both mesh kinds; builds the unique-face list.
dgx_status check_connectivity(dgx_handle* h, const int32_t* nb, const int8_t* nbf, const int8_t* ori,
                              std::vector<int4>& faces) {
  const int E = h->E, NF = h->NF, n = h->n, d = h->d, nfp = h->nfp;
  const int maxcode = d == 2 ? 2 : 8;
  faces.clear();
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < NF; ++f) {
      const int k = e * NF + f;
      const int o = nb[k];
      if (o < 0) {
        // tag 0 (adiabatic wall); tag 1 (farfield) with the DG-IP scheme only
        if (o != -1 && !(o == -2 && h->dgip)) return DGX_EUNSUPPORTED;
        faces.push_back(make_int4(e, o, f, 0));
        continue;
      }
      if (o >= E) return DGX_EINVAL;
      const int of = nbf[k];
      if (of < 0 || of >= NF || ori[k] < 0 || ori[k] >= maxcode) return DGX_EINVAL;
      const int k2 = o * NF + of;
      if (nb[k2] != e || nbf[k2] != f) return DGX_EINVAL;  // not reciprocal
      for (int fp = 0; fp < nfp; ++fp)
        if (omap(ori[k2], omap(ori[k], fp, n, d), n, d) != fp) return DGX_EINVAL;
      if (e < o || (e == o && f < of)) faces.push_back(make_int4(e, o, f | (of << 8) | (ori[k] << 16), 0));
    }
  return DGX_OK;
}

dgx_status upload_connectivity(dgx_handle* h, const int32_t* nb, const int8_t* nbf, const int8_t* ori,
                               const std::vector<int4>& faces) {
  const size_t m = (size_t)h->E * h->NF;
  std::vector<int> vnb(nb, nb + m);
  std::vector<int8_t> vnbf(nbf, nbf + m), vori(ori, ori + m);
  h->h_nb = vnb;
  h->h_nbf = vnbf;
  h->h_ori = vori;
  dgx_status s;
  if ((s = upload(vnb, (void**)&h->d_nb)) != DGX_OK) return s;
  if ((s = upload(vnbf, (void**)&h->d_nbf)) != DGX_OK) return s;
  if ((s = upload(vori, (void**)&h->d_ori)) != DGX_OK) return s;
  if ((s = upload(faces, (void**)&h->d_faces)) != DGX_OK) return s;
  h->nFaces = (int)faces.size();
  h->has_farfield = false;
  for (const int4& r : faces) h->has_farfield |= (r.y == -2);
  return DGX_OK;
}

template <typename S>
dgx::Mesh<S> mesh_view(const dgx_handle* h) {
  dgx::Mesh<S> M;
  M.E = h->E;
  M.nFaces = h->nFaces;
  M.nb = h->d_nb;
  M.nbf = h->d_nbf;
  M.ori = h->d_ori;
  M.faces = h->d_faces;
  M.geo.rh = (const S*)h->d_rh;
  M.geo.Ja = (const S*)h->d_Ja;
  M.geo.iJ = (const S*)h->d_iJ;
  M.geo.SnE = (const S*)h->d_SnE;
  M.geo.SnF = (const S*)h->d_SnF;
  M.tabs = (const Tab<S>*)h->d_tabs;
  const double g = h->desc.gamma;
  const double mu = h->viscous ? 1.0 / h->desc.Re : 0.0;
  M.gas.gamma = (S)g;
  M.gas.gm1 = (S)(g - 1.0);
  M.gas.mu = (S)mu;
  M.gas.lam = (S)(-2.0 * mu / 3.0);
  M.gas.kcv = (S)(h->viscous ? g * mu / h->desc.Pr : 0.0);
  M.flags = h->d_flags;
  M.wait_polls = h->wait_polls;
  return M;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Enqueue one kernel; with profiling on, bracket it by two events on its stream.
template <typename F>
cudaError_t launch(dgx_handle* h, int kind, cudaStream_t st, F&& f) {
  if (!h->prof || h->ev_used + 2 > h->ev_pool.size()) return f();
  cudaEvent_t a = h->ev_pool[h->ev_used], b = h->ev_pool[h->ev_used + 1];
  cudaEventRecord(a, st);
  const cudaError_t err = f();
  cudaEventRecord(b, st);
  h->ev_used += 2;
  h->ev_kind.push_back(kind);
  return err;
}

void profile_collect(dgx_handle* h) {
  for (size_t i = 0; i < h->ev_kind.size(); ++i) {
    float ms = 0.f;
    cudaEventSynchronize(h->ev_pool[2 * i + 1]);
    if (cudaEventElapsedTime(&ms, h->ev_pool[2 * i], h->ev_pool[2 * i + 1]) == cudaSuccess) {
      h->prof_ms[h->ev_kind[i]] += ms;
      h->prof_launches[h->ev_kind[i]] += 1;
    }
  }
  h->ev_kind.clear();
  h->ev_used = 0;
}

struct Layout {
  size_t TU, FF, G, Q, Y, K, SH, TUb, JB, Qb, NU, LAM, HA, GB, GP, TQ, total;
};

// FP64 viscous LLF/BR1 handles keep the face traces of Q from the forward BR1
// kernel for the adjoint (in the VJP workspace and in each stage checkpoint):
// the adjoint then reads them instead of tracing Q again, which saves FP64
// arithmetic on an FP64-bound path for 3 state vectors of writes (at p = 5 in
// 3D the traces are as large as Q).  FP32 handles trace Q again: there the
// extra writes would cost more than the arithmetic.
bool keep_tq(const dgx_handle* h) { return h->fp64 && h->viscous && !h->dgip; }
bool keep_dgip_faces(const dgx_handle* h) { return h->fp64 && h->viscous && h->dgip && !h->inner; }

// DG-IP scheme: TU, FF (+ G, HA viscous); the VJP adds TUb (+ Gb) and the
// element-local part of g; the ARK step adds Y, k_0..k_{s-2} and the FP32 shadow.
Layout layout_dgip(const dgx_handle* h, int op) {
  Layout L{};
  const size_t face = (size_t)h->E * h->NF * h->nf * h->nfp * h->s;
  const size_t state = (size_t)h->E * h->nf * h->N * h->s;
  size_t off = 0;
  L.TU = off;
  off += align256(face);
  L.FF = off;
  off += align256(face);
  if (h->viscous) {
    L.G = off;
    off += align256(face);
    L.HA = off;
    off += align256(face * h->d);
  }
  if (op == DGX_OP_VJP || op == DGX_OP_ARK_ADJOINT) {
    L.TUb = off;
    off += align256(face);
    if (h->viscous) {
      L.GB = off;
      off += align256(face);
    }
    L.GP = off;
    off += align256(state);
  }
  if (op == DGX_OP_ARK_ADJOINT) {  // nu_0 .. nu_{s-1}, then mu
    L.NU = off;
    off += align256(state) * (h->stages > 0 ? h->stages : 1);
    L.LAM = off;
    off += align256(state);
  }
  if (op == DGX_OP_ARK) {
    L.Y = off;
    off += align256(state);
    L.K = off;
    off += align256(state) * (h->stages > 1 ? h->stages - 1 : 0);
    if (!h->fp64) {
      L.SH = off;
      off += align256(state);
    }
  }
  L.total = off;
  return L;
}

dgx::DgipWork dgip_work_at(const dgx_handle* h, void* ws, const Layout& L) {
  char* b = (char*)ws;
  dgx::DgipWork w{};
  w.TU = b + L.TU;
  w.FF = b + L.FF;
  w.G = h->viscous ? b + L.G : nullptr;
  w.HA = h->viscous ? b + L.HA : nullptr;
  w.TUb = L.TUb ? b + L.TUb : nullptr;
  w.Gb = (L.GB && h->viscous) ? b + L.GB : nullptr;
  w.gpart = L.GP ? b + L.GP : nullptr;
  return w;
}

template <typename S>
dgx::Dgip<S> dgip_params(const dgx_handle* h, const int8_t* mask, const void* Uim) {
  dgx::Dgip<S> p{};
  p.il = (const S*)h->d_il;
  p.JaF = (const S*)h->d_JaF;
  p.iJF = (const S*)h->d_iJF;
  const int k = h->pen_k >= 0 ? h->pen_k : h->p;
  p.tk2 = (S)(h->alpha * (k + 1) * (k + 1));
  p.mask = mask;
  p.Uim = (const S*)Uim;
  for (int f = 0; f < 5; ++f) p.Uinf[f] = (S)h->Uinf[f];
  return p;
}

Layout layout(const dgx_handle* h, int op) {
  if (h->dgip) return layout_dgip(h, op);
  Layout L{};
  const size_t face = (size_t)h->E * h->NF * h->nf * h->nfp * h->s;
  const size_t state = (size_t)h->E * h->nf * h->N * h->s;
  size_t off = 0;
  L.TU = off;
  off += align256(face);
  L.FF = off;
  off += align256(face);
  if (h->viscous) {
    L.G = off;
    off += align256(face);
    L.Q = off;
    off += align256(state * h->d);
  }
  if (op == DGX_OP_VJP || op == DGX_OP_ARK_ADJOINT) {
    L.TUb = off;
    off += align256(face);
    if (h->viscous) {
      L.JB = off;
      off += align256(face);
      L.Qb = off;
      off += align256(state * h->d);
    }
    if (op == DGX_OP_VJP && keep_tq(h)) {  // the recomputed forward's traces of Q
      L.TQ = off;
      off += align256(face * h->d);
    }
  }
  if (op == DGX_OP_ARK_ADJOINT) {
    L.NU = off;
    off += align256(state) * (h->stages > 0 ? h->stages : 1);
    if (!h->fp64) {  // lambda_{n+1} rounded to FP32 once per adjoint step
      L.LAM = off;
      off += align256(state);
    }
  }
  if (op == DGX_OP_ARK) {
    L.Y = off;
    off += align256(state);
    L.K = off;
    off += align256(state) * (h->stages > 1 ? h->stages - 1 : 0);
    if (!h->fp64) {
      L.SH = off;
      off += align256(state);
    }
  }
  L.total = off;
  return L;
}

// Stage-checkpoint slot: y_i | TU_i | Q_i (viscous) | traces of Q_i (FP64 viscous);
// DG-IP: y_i (| TU_i | face gradients of y_i, viscous).
struct Slot {
  size_t y, TU, Q, TQ, QF, bytes;
};

Slot slot_layout(const dgx_handle* h) {
  const size_t face = (size_t)h->E * h->NF * h->nf * h->nfp * h->s;
  const size_t state = (size_t)h->E * h->nf * h->N * h->s;
  Slot S{};
  S.y = 0;
  if (h->dgip) {
    // FP64 viscous: the forward stage's traces and face gradients, which the
    // adjoint's face and gather kernels read instead of recomputing them
    // (FP64-bound arithmetic saved for bandwidth to spare; in FP32 the extra
    // traffic cost more than it saved, and Euler and over-integrated handles
    // keep the stage states only: their adjoint traces them again)
    S.TU = S.Q = S.TQ = S.QF = 0;
    S.bytes = align256(state);
    if (keep_dgip_faces(h)) {
      S.TU = S.bytes;
      S.QF = S.TU + align256(face);
      S.bytes = S.QF + align256(face * h->d);
    }
    return S;
  }
  S.TU = align256(state);
  S.Q = S.TU + align256(face);
  S.TQ = S.Q + (h->viscous ? align256(state * h->d) : 0);
  S.bytes = S.TQ + (keep_tq(h) ? align256(face * h->d) : 0);
  return S;
}

dgx::Work work_at(const dgx_handle* h, void* ws, const Layout& L) {
  char* b = (char*)ws;
  dgx::Work w;
  w.TU = b + L.TU;
  w.FF = b + L.FF;
  w.G = h->viscous ? b + L.G : nullptr;
  w.Q = h->viscous ? b + L.Q : nullptr;
  return w;
}

dgx::VjpWork vjp_work_at(const dgx_handle* h, void* ws, const Layout& L) {
  char* b = (char*)ws;
  dgx::VjpWork w{};
  w.TU = b + L.TU;
  w.FFb = b + L.FF;
  w.G = h->viscous ? b + L.G : nullptr;
  w.Q = h->viscous ? b + L.Q : nullptr;
  w.TUb = b + L.TUb;
  w.JB = h->viscous ? b + L.JB : nullptr;
  w.Qb = h->viscous ? b + L.Qb : nullptr;
  w.TQ = keep_tq(h) && L.TQ ? b + L.TQ : nullptr;
  return w;
}

dgx_status cuda_status(cudaError_t e) { return e == cudaSuccess ? DGX_OK : DGX_ECUDA; }

// Forward recompute (traces, BR1) then the four adjoint kernels.  g receives
// nu = (df/dU)(U)^T mu with mu described by cot (see dgx::Cot).
template <typename S>
// One VJP of the residual: [traces, BR1 gradient,] element, face, BR1 adjoint and
// (unless gather == false: the ARK adjoint defers it into the next reverse
// stage's element kernel) the gather that finishes g.
cudaError_t vjp_chain(dgx_handle* h, const void* U, const dgx::Cot<S>& cot, const dgx::Cot<S>& fin, void* g,
                      const dgx::VjpWork& vw, cudaStream_t st, bool have_forward = false, bool gather = true) {
  const void* M = h->fp64 ? (const void*)&h->mesh64 : (const void*)&h->mesh32;
  const dgx::Table* t = h->tab;
  const dgx::VjpTable* v = (const dgx::VjpTable*)t->vjp;
  dgx::Work w{vw.TU, vw.FFb, vw.G, vw.Q, vw.TQ};
  cudaError_t err = cudaSuccess;
  if (!have_forward) {  // recompute the forward traces and BR1 gradient
    err = launch(h, DGX_K_TRACE, st, [&] { return t->trace(M, h->var[DGX_K_TRACE], U, w.TU, st); });
    if (err == cudaSuccess && h->viscous)
      err = launch(h, DGX_K_BR1, st, [&] { return t->br1(M, h->var[DGX_K_BR1], h->curv, U, w, st); });
  }
  if (err == cudaSuccess)
    err = launch(h, DGX_K_VJP_ELEM, st, [&] { return v->elem(M, h->var[DGX_K_VJP_ELEM], h->viscous, h->curv, U, vw, &cot, g, st); });
  if (err == cudaSuccess)
    err = launch(h, DGX_K_VJP_FACE, st, [&] { return v->face(M, h->viscous, h->curv, vw, st); });
  if (err == cudaSuccess && h->viscous)
    err = launch(h, DGX_K_VJP_BR1, st, [&] { return v->br1(M, h->var[DGX_K_VJP_BR1], h->curv, vw, g, st); });
  if (err == cudaSuccess && gather)
    err = launch(h, DGX_K_VJP_GATHER, st, [&] { return v->gather(M, h->var[DGX_K_VJP_GATHER], h->viscous, vw, g, &fin, st); });
  return err;
}

// One ARK step.  With fork set, the last stage's face and element kernels (the
// ones that form U_{n+1}) go to the handle's second stream after an event on
// st; the caller joins it through h->ev_join.
template <typename S>
dgx_status ark_impl(dgx_handle* h, double* U64, double dt, void* stages, void* workspace, cudaStream_t st,
                    const S* dte = nullptr, bool fork = false) {
  const Layout L = layout(h, DGX_OP_ARK);
  const dgx::Work w = work_at(h, workspace, L);
  char* base = (char*)workspace;
  S* Y = (S*)(base + L.Y);
  const size_t state = align256((size_t)h->E * h->nf * h->N * h->s);
  S* shadow = h->fp64 ? nullptr : (S*)(base + L.SH);
  const Slot SL = slot_layout(h);
  char* ck = (char*)stages;  // optional stage checkpoints (slots)
  auto slot_y = [&](int i) { return (S*)(ck + SL.bytes * i + SL.y); };
  auto slot_tu = [&](int i) { return (void*)(ck + SL.bytes * i + SL.TU); };
  auto slot_q = [&](int i) { return (void*)(ck + SL.bytes * i + SL.Q); };
  auto slot_tq = [&](int i) { return keep_tq(h) ? (void*)(ck + SL.bytes * i + SL.TQ) : nullptr; };
  S* first = ck ? slot_y(0) : shadow;  // where the rounded (or copied) U_n goes
  dgx::Work w0 = w;
  if (ck) w0.TU = slot_tu(0);
  const void* M = h->fp64 ? (const void*)&h->mesh64 : (const void*)&h->mesh32;
  const dgx::Table* t = h->tab;
  cudaError_t err =
      launch(h, DGX_K_TRACE, st, [&] { return t->trace_from64(M, h->var[DGX_K_TRACE], U64, w0.TU, first, st); });
  if (err != cudaSuccess) return DGX_ECUDA;
  const S* y0 = (h->fp64 && !ck) ? (const S*)U64 : first;
  const int s = h->stages;
  for (int i = 0; i < s; ++i) {
    dgx::Stage<S> sa{};
    for (int j = 0; j < i; ++j) sa.k[j] = (const S*)(base + L.K + state * j);
    sa.i = i;
    sa.last = (i == s - 1);
    if (!sa.last)
      for (int j = 0; j <= i; ++j) sa.ca[j] = (S)h->A[(i + 1) * dgx::MAXSTAGES + j];
    for (int j = 0; j < s; ++j) sa.cb[j] = (S)h->b[j];
    const S dts = (S)dt;  // the kernels form the same S products from a per-element dt
    for (int j = 0; j < s; ++j) {
      sa.caf[j] = dts * sa.ca[j];
      sa.cbf[j] = dts * sa.cb[j];
    }
    sa.dte = dte;
    sa.base = y0;
    sa.Un = U64;
    sa.Y = (ck && !sa.last) ? slot_y(i + 1) : Y;
    sa.Kout = sa.last ? nullptr : (S*)(base + L.K + state * i);
    sa.shadow = shadow;  // FP32: rounded U_{n+1} (unused by the next step, which re-rounds U64)
    dgx::Work wi = w;
    if (ck) {
      wi.TU = slot_tu(i);
      wi.Q = h->viscous ? slot_q(i) : nullptr;
      wi.TQ = slot_tq(i);
    }
    sa.TU = (S*)((ck && !sa.last) ? slot_tu(i + 1) : w.TU);
    const S* Uin = (i == 0) ? y0 : (ck ? slot_y(i) : Y);
    if (h->viscous) err = launch(h, DGX_K_BR1, st, [&] { return t->br1(M, h->var[DGX_K_BR1], h->curv, Uin, wi, st); });
    cudaStream_t st_main = st;
    if (fork && sa.last && err == cudaSuccess) {  // U_{n+1} on the second stream
      err = cudaEventRecord(h->ev_fork, st);
      if (err == cudaSuccess) err = cudaStreamWaitEvent(h->side, h->ev_fork, 0);
      st = h->side;
    }
    if (err == cudaSuccess) err = launch(h, DGX_K_FACE, st, [&] { return t->face(M, h->viscous, h->curv, wi, st); });
    if (err == cudaSuccess)
      err = launch(h, DGX_K_ELEM_STAGE, st, [&] {
        if (h->contraction != DGX_CONTRACT_CUDA_CORE)
          return t->elem_tc(M, h->contraction, h->viscous, h->curv, Uin, wi, nullptr, &sa, st);
        bool used = false;
        if (h->pipeline) {
          const cudaError_t e = t->elem_pipe(M, h->var[DGX_K_ELEM_STAGE], h->viscous, h->curv, Uin, wi, nullptr, &sa,
                                             h->nsm, st, &used);
          if (e != cudaSuccess || used) return e;
        }
        return t->elem_stage(M, h->var[DGX_K_ELEM_STAGE], h->viscous, h->curv, Uin, wi, &sa, st);
      });
    if (st != st_main) {
      if (err == cudaSuccess) err = cudaEventRecord(h->ev_join, st);
      st = st_main;
    }
    if (err != cudaSuccess) return DGX_ECUDA;
  }
  return DGX_OK;
}

template <typename S>
dgx_status ark_adjoint_impl(dgx_handle* h, const void* stages, double* lam64, double dt, void* workspace,
                            cudaStream_t st) {
  const Layout L = layout(h, DGX_OP_ARK_ADJOINT);
  dgx::VjpWork vw = vjp_work_at(h, workspace, L);
  const size_t state_b = (size_t)h->E * h->nf * h->N * h->s;
  const size_t state_a = align256(state_b);
  char* base = (char*)workspace;
  auto NU = [&](int j) { return (S*)(base + L.NU + state_a * j); };
  const Slot SL = slot_layout(h);
  const int s = h->stages;
  for (int i = s - 1; i >= 0; --i) {
    const char* slot = (const char*)stages + SL.bytes * i;
    const void* y = slot + SL.y;
    vw.TU = (void*)(slot + SL.TU);
    vw.Q = h->viscous ? (void*)(slot + SL.Q) : nullptr;
    vw.TQ = keep_tq(h) ? (void*)(slot + SL.TQ) : nullptr;
    dgx::Cot<S> cot{}, fin{};
    if (h->fp64) {
      cot.lam64 = lam64;
    } else if (i == s - 1) {  // first reverse stage: read lambda_{n+1} in FP64, keep an FP32 copy
      cot.lam64 = lam64;
      cot.lam_out = (S*)(base + L.LAM);
    } else {
      cot.lam = (const S*)(base + L.LAM);
    }
    cot.c_lam = (S)(dt * h->b[i]);
    if (i < s - 1) {  // the element kernel finishes nu_{i+1} (its gather) and uses it directly
      cot.nu_prev = NU(i + 1);
      cot.c_prev = (S)(dt * h->A[(i + 1) * dgx::MAXSTAGES + i]);
    }
    for (int j = i + 2; j < s; ++j) {
      const double a = h->A[j * dgx::MAXSTAGES + i];
      if (a != 0.0) {
        cot.nu[cot.n_nu] = NU(j);
        cot.c_nu[cot.n_nu] = (S)(dt * a);
        ++cot.n_nu;
      }
    }
    if (i == 0) {
      fin.lam64_out = lam64;
      for (int j = 1; j < s; ++j) fin.nu_all[fin.n_all++] = NU(j);
    }
    const cudaError_t err = vjp_chain<S>(h, y, cot, fin, NU(i), vw, st, /*have_forward=*/true, /*gather=*/i == 0);
    if (err != cudaSuccess) return DGX_ECUDA;
  }
  return DGX_OK;
}

// ------------------------------------------------------------ DG-IP scheme
// One residual (traces and own-face viscous fluxes, face fluxes, element):
// f to out, or with stage != nullptr the fused ARK stage update.
template <typename S>
cudaError_t dgip_residual(dgx_handle* h, const void* U, const int8_t* mask, const void* Uim, void* out,
                          const dgx::DgipWork& w, const void* stage, cudaStream_t st) {
  const void* M = h->fp64 ? (const void*)&h->mesh64 : (const void*)&h->mesh32;
  const dgx::Dgip<S> dp = dgip_params<S>(h, mask, Uim);
  const dgx::DgipTable* t = h->dtab;
  cudaError_t err = launch(h, DGX_K_DGIP_TRACE, st, [&] { return t->trace(M, &dp, h->viscous, U, w, st); });
  if (err == cudaSuccess) err = launch(h, DGX_K_DGIP_FACE, st, [&] { return t->face(M, &dp, h->viscous, w, st); });
  if (err == cudaSuccess)
    err = launch(h, DGX_K_DGIP_ELEM, st, [&] { return t->elem(M, &dp, h->viscous, U, w, out, stage, st); });
  return err;
}

// g = (df/dU)^T lam: forward traces, then the element, face and gather adjoints.
template <typename S>
cudaError_t dgip_vjp(dgx_handle* h, const void* U, const void* lam, void* g, const dgx::DgipWork& w,
                     cudaStream_t st) {
  const void* M = h->fp64 ? (const void*)&h->mesh64 : (const void*)&h->mesh32;
  const dgx::Dgip<S> dp = dgip_params<S>(h, nullptr, nullptr);
  const dgx::DgipTable* t = h->dtab;
  // the adjoint needs the traces of U alone (its face kernel reads them; the
  // gather recomputes the face gradients it needs): the trace kernel without
  // its viscous part -- unless the stage checkpoint holds them (w.QF set:
  // traces and face gradients of the forward stage, read in place)
  cudaError_t err = cudaSuccess;
  if (!w.QF) err = launch(h, DGX_K_DGIP_VJP_TRACE, st, [&] { return t->trace(M, &dp, false, U, w, st); });
  if (err == cudaSuccess)
    err = launch(h, DGX_K_DGIP_VJP_ELEM, st, [&] { return t->vjp_elem(M, h->viscous, U, lam, w, st); });
  if (err == cudaSuccess)
    err = launch(h, DGX_K_DGIP_VJP_FACE, st, [&] { return t->vjp_face(M, &dp, h->viscous, w, st); });
  if (err == cudaSuccess)
    err = launch(h, DGX_K_DGIP_VJP_GATHER, st, [&] { return t->vjp_gather(M, &dp, h->viscous, U, w, g, st); });
  return err;
}

// One explicit ARK step of the DG-IP scheme (stage states optionally kept as
// checkpoints, as dgx_ark_step_stages describes).
template <typename S>
dgx_status dgip_ark_impl(dgx_handle* h, double* U64, double dt, void* stages, void* workspace, cudaStream_t st) {
  const Layout L = layout(h, DGX_OP_ARK);
  const dgx::DgipWork w = dgip_work_at(h, workspace, L);
  char* base = (char*)workspace;
  S* Y = (S*)(base + L.Y);
  const size_t state = align256((size_t)h->E * h->nf * h->N * h->s);
  S* shadow = h->fp64 ? nullptr : (S*)(base + L.SH);
  const Slot SL = slot_layout(h);
  char* ck = (char*)stages;
  auto slot_y = [&](int i) { return (S*)(ck + SL.bytes * i + SL.y); };
  S* first = ck ? slot_y(0) : shadow;  // the working-precision (or checkpointed) copy of U_n
  const void* M = h->fp64 ? (const void*)&h->mesh64 : (const void*)&h->mesh32;
  cudaError_t err = cudaSuccess;
  if (first)
    err = launch(h, DGX_K_TRACE, st,
                 [&] { return h->tab->trace_from64(M, h->var[DGX_K_TRACE], U64, w.TU, first, st); });
  if (err != cudaSuccess) return DGX_ECUDA;
  const S* y0 = (h->fp64 && !ck) ? (const S*)U64 : first;
  const int s = h->stages;
  for (int i = 0; i < s && err == cudaSuccess; ++i) {
    dgx::Stage<S> sa{};
    for (int j = 0; j < i; ++j) sa.k[j] = (const S*)(base + L.K + state * j);
    sa.i = i;
    sa.last = (i == s - 1);
    if (!sa.last)
      for (int j = 0; j <= i; ++j) sa.ca[j] = (S)h->A[(i + 1) * dgx::MAXSTAGES + j];
    for (int j = 0; j < s; ++j) sa.cb[j] = (S)h->b[j];
    const S dts = (S)dt;
    for (int j = 0; j < s; ++j) {
      sa.caf[j] = dts * sa.ca[j];
      sa.cbf[j] = dts * sa.cb[j];
    }
    sa.base = y0;
    sa.Un = U64;
    sa.Y = (ck && !sa.last) ? slot_y(i + 1) : Y;
    sa.Kout = sa.last ? nullptr : (S*)(base + L.K + state * i);
    sa.shadow = shadow;
    const S* Uin = (i == 0) ? y0 : (ck ? slot_y(i) : Y);
    dgx::DgipWork wi = w;
    if (ck && keep_dgip_faces(h)) {  // the stage's traces and face gradients go to its checkpoint
      wi.TU = ck + SL.bytes * i + SL.TU;
      wi.QF = ck + SL.bytes * i + SL.QF;
    }
    err = dgip_residual<S>(h, Uin, nullptr, nullptr, nullptr, wi, &sa, st);
  }
  return cuda_status(err);
}

// Discrete adjoint of one DG-IP ARK step (the reverse stage recurrence of
// Sec. 4.2 composed from single VJPs): for i = s .. 1,
// mu_i = dt (b_i lam + sum_{j>i} a_ji nu_j) formed in FP64 and rounded to the
// working precision, nu_i = (df/dU)(y_i)^T mu_i; then lam += sum_i nu_i in FP64.
template <typename S>
dgx_status dgip_ark_adjoint_impl(dgx_handle* h, const void* stages, double* lam64, double dt, void* workspace,
                                 cudaStream_t st) {
  const Layout L = layout(h, DGX_OP_ARK_ADJOINT);
  const dgx::DgipWork w = dgip_work_at(h, workspace, L);
  const size_t n = (size_t)h->E * h->nf * h->N;
  const size_t state_a = align256(n * h->s);
  char* base = (char*)workspace;
  auto NU = [&](int j) { return (S*)(base + L.NU + state_a * j); };
  S* mu = (S*)(base + L.LAM);
  const Slot SL = slot_layout(h);
  const int s = h->stages;
  for (int i = s - 1; i >= 0; --i) {
    dgx::LinComb<S> lc{};
    lc.n = n;
    lc.lam = lam64;
    lc.c_lam = dt * h->b[i];
    for (int j = i + 1; j < s; ++j) {
      const double a = h->A[j * dgx::MAXSTAGES + i];
      if (a != 0.0) {
        lc.in[lc.m] = NU(j);
        lc.c[lc.m] = dt * a;
        ++lc.m;
      }
    }
    lc.out = mu;
    cudaError_t err = dgx::lincomb<S>(lc, st);
    const void* y = (const char*)stages + SL.bytes * i + SL.y;
    dgx::DgipWork wi = w;
    if (keep_dgip_faces(h)) {  // the forward stage's traces and face gradients, from its checkpoint
      wi.TU = (char*)stages + SL.bytes * i + SL.TU;
      wi.QF = (char*)stages + SL.bytes * i + SL.QF;
    }
    if (err == cudaSuccess) err = dgip_vjp<S>(h, y, mu, NU(i), wi, st);
    if (err != cudaSuccess) return DGX_ECUDA;
  }
  dgx::LinComb<S> fin{};
  fin.n = n;
  fin.acc64 = lam64;
  for (int j = 0; j < s; ++j) {
    fin.in[fin.m] = NU(j);
    fin.c[fin.m] = 1.0;
    ++fin.m;
  }
  return cuda_status(dgx::lincomb<S>(fin, st));
}

// ------------------------------------------------------------ over-integration
// f = Pi f'(I U) (Sec. 5, the rule of order 3k): the states live on the
// (p+1)^d nodes, h->inner evaluates the collocated DG-IP operator of degree
// M-1 at the M^d points.  Workspace: the interpolated state, the point
// residual (or cotangent), the point gradient, the U_im interpolant of the
// split form, then the ARK / adjoint stage arrays at the nodes, then the
// inner handle's own workspace.
struct OiLayout {
  size_t Uq, Fq, Gq, Xq, Y, K, NU, MU, inner, total;
};

OiLayout layout_oi(const dgx_handle* h, int op) {
  const dgx_handle* q = h->inner;
  const size_t sq = align256((size_t)q->E * q->nf * q->N * q->s);
  const size_t sp = align256((size_t)h->E * h->nf * h->N * h->s);
  const int s = h->stages > 0 ? h->stages : 1;
  OiLayout L{};
  size_t off = 0;
  L.Uq = off;
  off += sq;
  L.Fq = off;
  off += sq;
  if (op == DGX_OP_RHS) {
    L.Xq = off;
    off += sq;
  }
  if (op == DGX_OP_VJP || op == DGX_OP_ARK_ADJOINT) {
    L.Gq = off;
    off += sq;
  }
  if (op == DGX_OP_ARK) {
    L.Y = off;
    off += sp;
    L.K = off;
    off += sp * s;
  }
  if (op == DGX_OP_ARK_ADJOINT) {
    L.NU = off;
    off += sp * s;
    L.MU = off;
    off += sp;
  }
  L.inner = off;
  const int iop = op == DGX_OP_ARK ? DGX_OP_RHS : (op == DGX_OP_ARK_ADJOINT ? DGX_OP_VJP : op);
  off += layout(q, iop).total;
  L.total = off;
  return L;
}

// one transfer: the [no][ni] matrix a along every direction of each element,
// on curved elements optionally scaled by Jacobians at its input and output
// points (pre, post: [E][points], or nullptr)
cudaError_t oi_transfer(dgx_handle* h, int kind, const void* in, void* out, bool to_quad, const double* a,
                        cudaStream_t st, const void* pre = nullptr, const void* post = nullptr) {
  const int ni = to_quad ? h->n : h->Mq, no = to_quad ? h->Mq : h->n;
  return launch(h, kind, st, [&] {
    return dgx::oi_apply(h->d, h->fp64, in, out, h->E, h->nf, ni, no, a, pre, post, h->nsm, st);
  });
}

// f = Pi f'(I U) into out (U_im: the implicit state of the split form, or
// nullptr); on curved elements f = J^-1 Pi (J' f'(I U)), the mass w_q J_q at
// the nodes and J' at the M points (d_oiJq set)
template <typename S>
cudaError_t oi_residual(dgx_handle* h, const void* U, const void* Uim, void* out, char* base, const OiLayout& L,
                        cudaStream_t st) {
  dgx_handle* q = h->inner;
  void* Uq = base + L.Uq;
  void* Fq = base + L.Fq;
  void* Xq = Uim ? base + L.Xq : nullptr;
  cudaError_t err = oi_transfer(h, DGX_K_OI_TO_QUAD, U, Uq, true, h->oiI, st);
  if (err == cudaSuccess && Uim) err = oi_transfer(h, DGX_K_OI_TO_QUAD, Uim, Xq, true, h->oiI, st);
  if (err == cudaSuccess) {
    const dgx::DgipWork w = dgip_work_at(q, base + L.inner, layout(q, DGX_OP_RHS));
    err = dgip_residual<S>(q, Uq, Uim ? h->d_mask : nullptr, Xq, Fq, w, nullptr, st);
  }
  if (err == cudaSuccess)
    err = h->d_oiJq ? oi_transfer(h, DGX_K_OI_TO_NODES, Fq, out, false, h->oiP, st, h->d_oiJq, h->d_iJ)
                    : oi_transfer(h, DGX_K_OI_TO_NODES, Fq, out, false, h->oiP, st);
  return err;
}

// g = I^T (df'/dU')^T (Pi^T lam); curved: Pi^T lam becomes J' Pi^T (J^-1 lam)
template <typename S>
cudaError_t oi_vjp(dgx_handle* h, const void* U, const void* lam, void* g, char* base, const OiLayout& L,
                   cudaStream_t st) {
  dgx_handle* q = h->inner;
  void* Uq = base + L.Uq;
  void* Lq = base + L.Fq;
  void* Gq = base + L.Gq;
  cudaError_t err = oi_transfer(h, DGX_K_OI_TO_QUAD, U, Uq, true, h->oiI, st);
  if (err == cudaSuccess)
    err = h->d_oiJq ? oi_transfer(h, DGX_K_OI_TO_QUAD, lam, Lq, true, h->oiPT, st, h->d_iJ, h->d_oiJq)
                    : oi_transfer(h, DGX_K_OI_TO_QUAD, lam, Lq, true, h->oiPT, st);
  if (err == cudaSuccess) {
    const dgx::DgipWork w = dgip_work_at(q, base + L.inner, layout(q, DGX_OP_VJP));
    err = dgip_vjp<S>(q, Uq, Lq, Gq, w, st);
  }
  if (err == cudaSuccess) err = oi_transfer(h, DGX_K_OI_TO_NODES, Gq, g, false, h->oiIT, st);
  return err;
}

// One explicit ARK step with the over-integrated operator: y_i = U_n +
// dt sum_{j<i} a_ij k_j formed in FP64 and rounded to the working precision
// (kept in the stage slots when given), k_i = f(y_i), then
// U_{n+1} = U_n + dt sum_j b_j k_j accumulated in FP64.
template <typename S>
dgx_status oi_ark_impl(dgx_handle* h, double* U64, double dt, void* stages, void* workspace, cudaStream_t st) {
  const OiLayout L = layout_oi(h, DGX_OP_ARK);
  char* base = (char*)workspace;
  const size_t n = (size_t)h->E * h->nf * h->N;
  const size_t sp = align256(n * h->s);
  auto K = [&](int j) { return (S*)(base + L.K + sp * j); };
  const Slot SL = slot_layout(h);
  const int s = h->stages;
  cudaError_t err = cudaSuccess;
  for (int i = 0; i < s && err == cudaSuccess; ++i) {
    S* y = stages ? (S*)((char*)stages + SL.bytes * i + SL.y) : (S*)(base + L.Y);
    const S* in = y;
    if (i == 0 && h->fp64 && !stages) {
      in = (const S*)U64;
    } else {
      dgx::LinComb<S> lc{};
      lc.n = n;
      lc.lam = U64;
      lc.c_lam = 1.0;
      for (int j = 0; j < i; ++j) {
        const double a = h->A[i * dgx::MAXSTAGES + j];
        if (a != 0.0) {
          lc.in[lc.m] = K(j);
          lc.c[lc.m] = dt * a;
          ++lc.m;
        }
      }
      lc.out = y;
      err = dgx::lincomb<S>(lc, st);
    }
    if (err == cudaSuccess) err = oi_residual<S>(h, in, nullptr, K(i), base, L, st);
  }
  if (err != cudaSuccess) return DGX_ECUDA;
  dgx::LinComb<S> fin{};
  fin.n = n;
  fin.acc64 = U64;
  for (int j = 0; j < s; ++j)
    if (h->b[j] != 0.0) {
      fin.in[fin.m] = K(j);
      fin.c[fin.m] = dt * h->b[j];
      ++fin.m;
    }
  return cuda_status(dgx::lincomb<S>(fin, st));
}

// Its discrete adjoint, the reverse stage recurrence of the DG-IP scheme
// with the over-integrated VJP.
template <typename S>
dgx_status oi_ark_adjoint_impl(dgx_handle* h, const void* stages, double* lam64, double dt, void* workspace,
                               cudaStream_t st) {
  const OiLayout L = layout_oi(h, DGX_OP_ARK_ADJOINT);
  char* base = (char*)workspace;
  const size_t n = (size_t)h->E * h->nf * h->N;
  const size_t sp = align256(n * h->s);
  auto NU = [&](int j) { return (S*)(base + L.NU + sp * j); };
  S* mu = (S*)(base + L.MU);
  const Slot SL = slot_layout(h);
  const int s = h->stages;
  for (int i = s - 1; i >= 0; --i) {
    dgx::LinComb<S> lc{};
    lc.n = n;
    lc.lam = lam64;
    lc.c_lam = dt * h->b[i];
    for (int j = i + 1; j < s; ++j) {
      const double a = h->A[j * dgx::MAXSTAGES + i];
      if (a != 0.0) {
        lc.in[lc.m] = NU(j);
        lc.c[lc.m] = dt * a;
        ++lc.m;
      }
    }
    lc.out = mu;
    cudaError_t err = dgx::lincomb<S>(lc, st);
    const void* y = (const char*)stages + SL.bytes * i + SL.y;
    if (err == cudaSuccess) err = oi_vjp<S>(h, y, mu, NU(i), base, L, st);
    if (err != cudaSuccess) return DGX_ECUDA;
  }
  dgx::LinComb<S> fin{};
  fin.n = n;
  fin.acc64 = lam64;
  for (int j = 0; j < s; ++j) {
    fin.in[fin.m] = NU(j);
    fin.c[fin.m] = 1.0;
    ++fin.m;
  }
  return cuda_status(dgx::lincomb<S>(fin, st));
}

// The 1D transfers of an M-point rule on the degree-p nodes (FP64, from the
// compile-time Gauss rules of basis1d.h): I[m][j] = l_j(z_m),
// Pi[q][m] = omega_m l_q(z_m) / w_q, and their transposes.
void oi_matrices(dgx_handle* h) {
  const dgx::Basis1 b = dgx::make_basis1(h->p), z = dgx::make_basis1(h->Mq - 1);
  const int n = b.n, M = z.n;
  for (int m = 0; m < M; ++m)
    for (int j = 0; j < n; ++j) {
      double l = 1.0;
      for (int k = 0; k < n; ++k)
        if (k != j) l *= (z.x[m] - b.x[k]) / (b.x[j] - b.x[k]);
      h->oiI[m * n + j] = l;
      h->oiIT[j * M + m] = l;
      const double pq = z.w[m] * l / b.w[j];
      h->oiP[j * M + m] = pq;
      h->oiPT[m * n + j] = pq;
    }
}

// ------------------------------------------------------------ work model
struct Pointwise {
  double conv, visc, visc_n, wall_visc, llf_unit, llf_area, conv_vjp, visc_vjp, visc_n_vjp, llf_unit_vjp,
      llf_area_vjp, dgip_face, dgip_face_euler, dgip_face_vjp, dgip_face_euler_vjp, visc_n_axis, visc_n_axis_vjp,
      dgip_face_gen, dgip_face_vjp_gen;  // *_gen: general K-products (FP32 and curved kernels)
};

template <int D>
Pointwise count_pointwise() {
  using C = dgx::Count;
  dgx::Gas<C> g;
  g.gamma = 1.4;
  g.gm1 = 0.4;
  g.mu = 1e-3;
  g.lam = -2e-3 / 3;
  g.kcv = 2e-3;
  C U[D + 2], V[D + 2], Q[D][D + 2], nv[D], F[D][D + 2], G[D + 2], Ub[D + 2], Vb[D + 2], Qb[D][D + 2];
  for (int f = 0; f < D + 2; ++f) {
    U[f] = 1.0 + 0.1 * f;
    V[f] = 1.05 + 0.09 * f;
    G[f] = 0.3 - 0.05 * f;
    Ub[f] = Vb[f] = 0.0;
    for (int a = 0; a < D; ++a) {
      Q[a][f] = 0.2 * (a + 1) - 0.03 * f;
      Qb[a][f] = 0.0;
      F[a][f] = 0.1 * (a - f);
    }
  }
  U[D + 1] = V[D + 1] = 3.0;
  for (int a = 0; a < D; ++a) nv[a] = 0.3 + 0.2 * a;
  Pointwise pc{};
  auto cnt = [](auto&& fn) {
    dgx::Count::ops = 0;
    fn();
    return (double)dgx::Count::ops;
  };
  C Fo[D][D + 2], Go[D + 2];
  pc.conv = cnt([&] { dgx::conv_flux_all<D, C>(U, g, Fo); });
  pc.visc = cnt([&] { dgx::visc_flux_all<D, C>(U, Q, g, Fo); });
  pc.visc_n = cnt([&] { dgx::visc_flux_normal<D, C>(U, Q, nv, g, Go); });
  pc.visc_n_axis = cnt([&] { dgx::visc_flux_axis<D, 0, C>(U, Q, C(1.0), g, Go); });
  pc.wall_visc = cnt([&] { dgx::wall_visc_flux<D, C>(U, Q, nv, g, Go); });
  pc.llf_unit = cnt([&] { dgx::llf_flux<D, C, true>(U, V, nv, g, Go); });
  pc.llf_area = cnt([&] { dgx::llf_flux<D, C, false>(U, V, nv, g, Go); });
  pc.conv_vjp = cnt([&] { dgx::conv_flux_all_vjp<D, C>(U, F, g, Ub); });
  pc.visc_vjp = cnt([&] { dgx::visc_flux_all_vjp<D, C>(U, Q, F, g, Ub, Qb); });
  pc.visc_n_vjp = cnt([&] { dgx::visc_flux_normal_vjp<D, C>(U, Q, nv, G, g, Ub, Qb); });
  pc.visc_n_axis_vjp = cnt([&] { dgx::visc_flux_axis_vjp<D, 0, C>(U, Q, C(1.0), G, g, Ub, Qb); });
  pc.llf_unit_vjp = cnt([&] { dgx::llf_flux_vjp<D, C, true>(U, V, nv, G, g, Ub, Vb); });
  pc.llf_area_vjp = cnt([&] { dgx::llf_flux_vjp<D, C, false>(U, V, nv, G, g, Ub, Vb); });
  {  // DG-IP face function (interior face point), forward and its dual-number adjoint
    C HL[D][D + 2], HR[D][D + 2], Fb[D + 2], Hb[D][D + 2];
    for (int f = 0; f < D + 2; ++f) {
      Fb[f] = 0.1;
      for (int a = 0; a < D; ++a) Hb[a][f] = 0.2;
    }
    const C tau = 10.0;
    pc.dgip_face = cnt([&] { dgx::dgip_face_fn<D, C, C, true, dgx::DGIP_INTERIOR, true>(U, V, nv, g, g, tau, false, false, Go, HL, HR); });
    pc.dgip_face_euler =
        cnt([&] { dgx::dgip_face_fn<D, C, C, false, dgx::DGIP_INTERIOR, true>(U, V, nv, g, g, tau, false, false, Go, HL, HR); });
    pc.dgip_face_vjp = cnt([&] {
      dgx::dgip_face_fn_vjp_host<D, C, true>(U, V, nv, g, tau, Fb, Hb, Hb, Ub, Vb);
    });
    pc.dgip_face_euler_vjp = cnt([&] {
      dgx::dgip_face_fn_vjp_host<D, C, false>(U, V, nv, g, tau, Fb, Hb, Hb, Ub, Vb);
    });
    pc.dgip_face_gen = cnt([&] {
      dgx::dgip_face_fn<D, C, C, true, dgx::DGIP_INTERIOR, true, false>(U, V, nv, g, g, tau, false, false, Go, HL, HR);
    });
    pc.dgip_face_vjp_gen = cnt([&] {
      dgx::dgip_face_fn_vjp_host<D, C, true, false>(U, V, nv, g, tau, Fb, Hb, Hb, Ub, Vb);
    });
  }
  return pc;
}

// Algorithmic flops and bytes of one launch of a kernel kind on this handle.
void kernel_work(const dgx_handle* h, int kind, double& flops, double& bytes) {
  if (h->inner && ((kind >= DGX_K_DGIP_TRACE && kind <= DGX_K_DGIP_VJP_GATHER) || kind == DGX_K_DGIP_VJP_TRACE)) {
    // run at the M points
    kernel_work(h->inner, kind, flops, bytes);
    return;
  }
  if (kind == DGX_K_OI_TO_QUAD || kind == DGX_K_OI_TO_NODES) {  // one transfer: values in and out
    flops = bytes = 0.0;
    if (!h->inner) return;
    const int ni = kind == DGX_K_OI_TO_QUAD ? h->n : h->Mq, no = kind == DGX_K_OI_TO_QUAD ? h->Mq : h->n;
    double macs = 0.0, ext = 1.0;  // pass a: no x (no^a ni^(d-1-a)) outputs of ni terms each
    for (int a = 0; a < h->d; ++a) {
      double pts = 1.0;
      for (int b = 0; b < h->d; ++b) pts *= b <= a ? no : ni;
      macs += pts * ni;
      ext = pts;
    }
    flops = 2.0 * h->E * h->nf * macs;
    bytes = (double)h->E * h->nf * (ext + std::pow((double)ni, h->d)) * h->s;
    return;
  }
  const Pointwise pc = h->d == 2 ? count_pointwise<2>() : count_pointwise<3>();
  const double E = h->E, N = h->N, nf = h->nf, nfp = h->nfp, NF = h->NF, D = h->d, n = h->n, s = (double)h->s;
  const double STATE = nf * N, FACE = NF * nf * nfp, F = h->nFaces;
  const bool v = h->viscous, c = h->curv;
  const double geo_node = c ? (D * D * N + N) * s : D * s;  // per element
  const double geo_face = c ? NF * D * nfp * s : 0.0;
  const int st = h->stages > 0 ? h->stages : 1;
  flops = bytes = 0.0;
  switch (kind) {
    case DGX_K_TRACE:
      flops = E * FACE * 2 * n;
      bytes = E * (STATE + FACE) * s;
      // ARK step: the trace kernel reads the FP64 master state and also writes
      // the working-precision copy of it that the first stage evaluates
      if (h->stages > 0) bytes = E * (STATE * 8.0 + FACE * s + STATE * s);
      break;
    case DGX_K_BR1:
      flops = E * (NF * nfp * nf * 2 + N * D * nf * 2 * n + N * D * nf * (c ? (8 * D + 1) : 5) +
                   NF * nfp * D * nf * 2 * n + NF * nfp * (c ? pc.visc_n : pc.visc_n_axis));
      bytes = E * ((STATE + 2 * FACE + D * STATE + FACE) * s + geo_node + geo_face);
      // FP64 stage checkpoints and VJPs: the traces of Q are also written
      if (keep_tq(h)) bytes += E * D * FACE * s;
      break;
    case DGX_K_FACE:
      flops = F * nfp * ((c ? pc.llf_area : pc.llf_unit) + (v ? 3 * nf : 0));
      bytes = E * FACE * s * (2 + (v ? 1 : 0)) + (c ? F * D * nfp * s : 0.0);
      break;
    case DGX_K_ELEM:
    case DGX_K_ELEM_STAGE: {
      flops = E * N * (pc.conv + (v ? pc.visc + D * nf : 0) + (c ? D * nf * (2 * D - 1) + nf : 0) +
                       D * nf * (2 * n + 6));
      bytes = E * ((STATE + (v ? D * STATE : 0) + FACE + (kind == DGX_K_ELEM ? STATE : 0)) * s + geo_node);
      if (kind == DGX_K_ELEM_STAGE) {  // averaged over the stages of the tableau
        double fl = 0, by = 0;
        for (int i = 0; i < st; ++i) {
          fl += E * STATE * 2 * (i + 1) + E * FACE * 2 * n;
          const bool last = i == st - 1;
          by += E * ((1 + i) * STATE * s + (last ? 16 * STATE : 2 * STATE * s) + FACE * s);
        }
        flops += fl / st;
        bytes += by / st;
      }
      break;
    }
    case DGX_K_VJP_ELEM: {
      flops = E * (FACE * 2 * n + N * D * nf * 2 * n + N * (pc.conv_vjp + (v ? pc.visc_vjp : 0)) +
                   (c ? N * D * D * nf * 2 + STATE : 0));
      bytes = E * ((STATE + (v ? 2 * D * STATE : 0) + FACE + STATE) * s + geo_node);
      // cotangent combination mu = c_lam lambda + sum_j c_j nu_j, averaged over the
      // reverse stages of the ARK adjoint (plain VJP without a tableau: lambda only)
      double fl = 0, by = 0;
      if (h->stages > 0) {
        for (int i = 0; i < st; ++i) {
          const bool first = i == st - 1;  // first reverse stage: no gather to finish
          int nnu = 0;
          for (int j = i + (first ? 1 : 2); j < st; ++j) nnu += h->A[j * dgx::MAXSTAGES + i] != 0.0;
          const double lam_b = h->fp64 ? (h->b[i] != 0.0 ? 8.0 : 0.0) : (first ? 8.0 + 4.0 : (h->b[i] != 0.0 ? 4.0 : 0.0));
          fl += E * STATE * 2 * (1 + nnu + (first ? 0 : 1));
          by += E * STATE * (lam_b + nnu * s);
          if (!first) {  // fused gather of nu_{i+1}: trace cotangents (+ jump cotangents), nu read + written
            fl += E * (STATE * 4 * D + (v ? FACE * 2 : 0));
            by += E * ((FACE * (v ? 2 : 1) + 2 * STATE) * s);
          }
        }
        fl /= st;
        by /= st;
      } else {
        fl = E * STATE * 2;
        by = E * STATE * s;
      }
      flops += fl;
      bytes += by;
      break;
    }
    case DGX_K_VJP_FACE:
      flops = F * nfp * (nf + (c ? pc.llf_area_vjp : pc.llf_unit_vjp));
      bytes = E * FACE * s * 3 + (c ? F * D * nfp * s : 0.0);
      break;
    case DGX_K_VJP_BR1:
      flops = E * (NF * nfp * (D * nf * 2 * n + (c ? pc.visc_n_vjp : pc.visc_n_axis_vjp)) + N * D * nf * 4 * D +
                   N * D * nf * (c ? 2 * D : 1) +
                   N * nf * D * 2 * n + NF * nfp * nf * (c ? D * (2 * n + 2) : 2 * n + 1) + NF * nfp * nf * 4);
      // face arrays: TU, both sides' Fhat_bar, TU_bar read and written, JB written
      bytes = E * ((6 * FACE + 2 * D * STATE + 2 * STATE) * s + geo_node + geo_face);
      if (keep_tq(h)) {  // the stored traces of Q replace Q and its tracing
        flops -= E * NF * nfp * D * nf * 2 * n;
        bytes += E * (D * FACE - D * STATE) * s;
      }
      break;
    case DGX_K_DGIP_VJP_TRACE:  // the traces alone
      flops = E * FACE * 2 * n;
      bytes = E * (STATE + FACE) * s;
      break;
    case DGX_K_DGIP_TRACE:  // traces; face gradients and own-face viscous fluxes
      flops = E * FACE * 2 * n + (v ? E * NF * nfp * (D * nf * 2 * n + (c ? pc.visc_n : pc.visc_n_axis)) : 0.0);
      bytes = E * ((STATE + FACE + (v ? FACE : 0)) * s + D * s);
      break;
    case DGX_K_DGIP_FACE:  // both sides' traces and G read; FF and HA of both sides written
      flops = F * nfp * ((v ? (!c && s == 8 ? pc.dgip_face : pc.dgip_face_gen) : pc.dgip_face_euler) + (v ? 3 * nf : 0));
      bytes = E * FACE * s * (2 + (v ? 1 + D : 0));
      break;
    case DGX_K_DGIP_ELEM:  // U, FF (+ HA) in, f out; gradient lines, flux, tangential terms, divergence + lift
      flops = E * N * (pc.conv + (v ? pc.visc + D * nf * 2 * n + (D - 1) * D * nf * 4 : 0) + D * nf * (2 * n + 6) +
                       (v ? D * nf * 4 : 0));
      bytes = E * ((2 * STATE + FACE + (v ? D * FACE : 0)) * s + D * s);
      break;
    case DGX_K_DGIP_VJP_ELEM:  // U, lambda in; the local part of g, FFb (+ HAb) out
      flops = E * N * (pc.conv_vjp + D * nf * 2 * n + D * nf * 8 + (v ? pc.visc_vjp + 2 * D * nf * 2 * n : 0)) +
              (v ? E * NF * (D - 1) * nf * nfp * 2 * n : 0.0);
      bytes = E * ((3 * STATE + FACE + (v ? D * FACE : 0)) * s + D * s);
      break;
    case DGX_K_DGIP_VJP_FACE:  // traces, FFb (+ HAb) of both sides read; TUb (+ Gb) written
      flops = F * nfp * (v ? (!c && s == 8 ? pc.dgip_face_vjp : pc.dgip_face_vjp_gen) : pc.dgip_face_euler_vjp);
      bytes = E * FACE * s * (3 + (v ? D + 1 : 0));
      break;
    case DGX_K_DGIP_VJP_GATHER:  // U, gpart, TUb (+ Gb) in, g out
      flops = E * (FACE * 2 * n + STATE * 2 * D +
                   (v ? NF * nfp * (D * nf * 2 * n + (c ? pc.visc_n_vjp : pc.visc_n_axis_vjp) + (D - 1) * nf * 2 * n +
                                    2 * n * nf)
                      : 0));
      bytes = E * ((3 * STATE + FACE + (v ? FACE : 0)) * s + D * s);
      break;
    case DGX_K_VJP_GATHER:
      flops = E * ((v ? FACE * 2 : 0) + STATE * 4 * D);
      bytes = E * ((FACE + (v ? FACE : 0) + 2 * STATE) * s);
      if (h->stages > 0) {  // ARK adjoint: the one gather per step also forms lambda_n = lambda_{n+1} + sum_j nu_j
        flops += E * STATE * st;
        bytes += E * STATE * (16.0 + (st - 1) * s);
      }
      break;
    default:
      break;
  }
}

// ------------------------------------------------------------ autotuning
bool is_tile_kind(int k) { return k != DGX_K_FACE && k != DGX_K_VJP_FACE && k < DGX_K_DGIP_TRACE; }

size_t tile_smem(const dgx_handle* h, int kind, int V) {
  const dgx::Table* t = h->tab;
  const dgx::VjpTable* v = (const dgx::VjpTable*)t->vjp;
  switch (kind) {
    case DGX_K_TRACE: return t->smem(0, V);
    case DGX_K_BR1: return t->smem(1, V);
    case DGX_K_ELEM:
    case DGX_K_ELEM_STAGE: return t->smem(2, V);
    case DGX_K_VJP_ELEM: return v ? v->smem(0, V) : 0;
    case DGX_K_VJP_BR1: return v ? v->smem(1, V) : 0;
    case DGX_K_VJP_GATHER: return v ? v->smem(2, V) : 0;
    default: return 0;
  }
}

template <typename T>
struct DevBuf {  // scratch owned by a set-up call
  T* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  bool alloc(size_t bytes) { return cudaMalloc((void**)&p, bytes ? bytes : 1) == cudaSuccess; }
};

}  // namespace

int64_t dgx::Count::ops = 0;

extern "C" {

const char* dgx_kernel_name(int32_t kind) {
  static const char* names[DGX_KERNEL_KINDS] = {"trace",      "br1",           "face",          "elem",
                                                "elem_stage", "vjp_elem",      "vjp_face",      "vjp_br1",
                                                "vjp_gather", "dgip_trace",    "dgip_face",     "dgip_elem",
                                                "dgip_vjp_elem", "dgip_vjp_face", "dgip_vjp_gather",
                                                "oi_to_quad",    "oi_to_nodes",   "dgip_vjp_trace"};
  return (kind >= 0 && kind < DGX_KERNEL_KINDS) ? names[kind] : "unknown";
}

dgx_status dgx_profile_enable(dgx_handle* h, int32_t enable) {
  if (!h) return DGX_EINVAL;
  if (enable && h->ev_pool.empty()) {
    h->ev_pool.resize(8192);
    for (auto& e : h->ev_pool)
      if (cudaEventCreate(&e) != cudaSuccess) return DGX_ECUDA;
  }
  if (!enable && h->prof) profile_collect(h);
  h->prof = enable != 0;
  return h->inner ? dgx_profile_enable(h->inner, enable) : DGX_OK;
}

dgx_status dgx_profile_read(dgx_handle* h, int32_t kind, int64_t* launches, double* ms) {
  if (!h || kind < 0 || kind >= DGX_KERNEL_KINDS) return DGX_EINVAL;
  profile_collect(h);
  int64_t nl = h->prof_launches[kind];
  double t = h->prof_ms[kind];
  if (h->inner) {  // the point operator's kernels
    int64_t il = 0;
    double im = 0.0;
    dgx_profile_read(h->inner, kind, &il, &im);
    nl += il;
    t += im;
  }
  if (launches) *launches = nl;
  if (ms) *ms = t;
  return DGX_OK;
}

dgx_status dgx_kernel_work(const dgx_handle* h, int32_t kind, double* flops, double* bytes) {
  if (!h || kind < 0 || kind >= DGX_KERNEL_KINDS || !h->has_mesh) return DGX_EINVAL;
  double f = 0, b = 0;
  kernel_work(h, kind, f, b);
  if (flops) *flops = f;
  if (bytes) *bytes = b;
  return DGX_OK;
}

dgx_status dgx_profile_reset(dgx_handle* h) {
  if (!h) return DGX_EINVAL;
  profile_collect(h);
  for (int k = 0; k < DGX_KERNEL_KINDS; ++k) {
    h->prof_launches[k] = 0;
    h->prof_ms[k] = 0.0;
  }
  return h->inner ? dgx_profile_reset(h->inner) : DGX_OK;
}

const char* dgx_status_string(dgx_status s) {
  switch (s) {
    case DGX_OK: return "ok";
    case DGX_EINVAL: return "invalid argument";
    case DGX_ENOMEM: return "out of memory";
    case DGX_ECUDA: return "CUDA error";
    case DGX_ENONFINITE: return "non-finite residual";
    case DGX_ETIMEOUT: return "device wait timed out";
    case DGX_EUNSUPPORTED: return "unsupported";
    case DGX_ESTATE: return "call out of order";
  }
  return "unknown status";
}

// Device of a handle, for the allocation-free entry point in noalloc.cu (not part of the C ABI).
__attribute__((visibility("hidden"))) int dgx_internal_handle_device(const dgx_handle* h) {
  return h ? h->dev : -1;
}

// point_op: the degree-(M-1) DG-IP handle of an over-integrated handle, whose
// degree may reach 7 (DG-IP launch table alone above 5).
static dgx_status create_impl(const dgx_problem_desc* desc, dgx_handle** out, bool point_op) {
  if (!out) return DGX_EINVAL;
  *out = nullptr;
  if (!desc) return DGX_EINVAL;
  if (desc->dim != 2 && desc->dim != 3) return DGX_EINVAL;
  if (desc->p < 1 || desc->p > (point_op ? 7 : 5) || desc->n_elem < 1) return DGX_EINVAL;
  if (desc->precision != DGX_FP64 && desc->precision != DGX_FP32) return DGX_EINVAL;
  if (!(desc->gamma > 1.0)) return DGX_EINVAL;
  if (desc->viscous && (!(desc->Re > 0.0) || !(desc->Pr > 0.0))) return DGX_EINVAL;
  if (desc->conv_flux != DGX_FLUX_LLF && desc->conv_flux != DGX_FLUX_VIJAYASUNDARAM) return DGX_EINVAL;
  if (desc->visc_flux != DGX_VISC_BR1 && desc->visc_flux != DGX_VISC_SIPG) return DGX_EINVAL;
  if (!(desc->penalty_alpha >= 0.0) || !std::isfinite(desc->penalty_alpha)) return DGX_EINVAL;
  const bool dgip = desc->conv_flux == DGX_FLUX_VIJAYASUNDARAM;
  // the schemes are LLF + BR1 and Vijayasundaram + SIPG
  if (desc->viscous && (desc->visc_flux == DGX_VISC_SIPG) != dgip) return DGX_EUNSUPPORTED;
  if (desc->quad_points != 0) {  // over-integration: DG-IP, p + 1 <= M <= the kernels' largest n
    if (desc->quad_points < desc->p + 1) return DGX_EINVAL;
    if (!dgip || desc->quad_points > dgx::OI_MAXQ) return DGX_EUNSUPPORTED;
  }
  dgx_handle* h = new (std::nothrow) dgx_handle();
  if (!h) return DGX_ENOMEM;
  h->desc = *desc;
  h->d = desc->dim;
  h->p = desc->p;
  h->n = desc->p + 1;
  h->N = ipow(h->n, h->d);
  h->nf = h->d + 2;
  h->nfp = ipow(h->n, h->d - 1);
  h->NF = 2 * h->d;
  h->E = desc->n_elem;
  h->T = (256 / h->N) > 0 ? 256 / h->N : 1;
  h->viscous = desc->viscous != 0;
  h->fp64 = desc->precision == DGX_FP64;
  h->s = h->fp64 ? 8 : 4;
  h->dgip = dgip;
  h->alpha = desc->penalty_alpha > 0.0 ? desc->penalty_alpha : 1.0;
  if (h->p <= 5) {
    if (h->d == 2) h->tab = h->fp64 ? dgx::table_d2_f64(h->p) : dgx::table_d2_f32(h->p);
    else h->tab = h->fp64 ? dgx::table_d3_f64(h->p) : dgx::table_d3_f32(h->p);
    h->dtab = h->tab ? (const dgx::DgipTable*)h->tab->dgip : nullptr;
  } else if (h->dgip) {  // point operator of degree 6 or 7: DG-IP launches only
    if (h->d == 2) h->dtab = (const dgx::DgipTable*)(h->fp64 ? dgx::dgip_only_d2_f64(h->p) : dgx::dgip_only_d2_f32(h->p));
    else h->dtab = (const dgx::DgipTable*)(h->fp64 ? dgx::dgip_only_d3_f64(h->p) : dgx::dgip_only_d3_f32(h->p));
  }
  if ((!h->tab && h->p <= 5) || (h->dgip && !h->dtab)) {
    delete h;
    return DGX_EUNSUPPORTED;
  }
  dgx_status st = DGX_OK;
  if (h->fp64) {
    std::vector<Tab<double>> t(6);
    for (int p = 1; p <= 5; ++p) fill_tab(p, t[p]);
    st = upload(t, &h->d_tabs);
  } else {
    std::vector<Tab<float>> t(6);
    for (int p = 1; p <= 5; ++p) fill_tab(p, t[p]);
    st = upload(t, &h->d_tabs);
  }
  // default tile variant: about 256 threads, or the largest smaller one whose
  // shared memory fits (small 3D elements in FP64)
  for (int k = 0; k < DGX_KERNEL_KINDS && h->tab; ++k) {
    if (!is_tile_kind(k)) continue;
    int v = 1;
    while (v > 0 && tile_smem(h, k, v) > dgx::SMEM_LIMIT) --v;
    h->var[k] = v;
  }
  {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) {
      h->dev = dev;
      if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0) h->nsm = nsm;
    }
  }
  if (st == DGX_OK && cudaMalloc((void**)&h->d_flags, sizeof(unsigned)) != cudaSuccess) st = DGX_ENOMEM;
  if (st == DGX_OK && cudaMemset(h->d_flags, 0, sizeof(unsigned)) != cudaSuccess) st = DGX_ECUDA;
  if (st == DGX_OK && (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
                       cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                       cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess))
    st = DGX_ECUDA;
  if (st == DGX_OK && desc->quad_points != 0) {  // the degree-(M-1) operator at the M points
    dgx_problem_desc dq = *desc;
    dq.p = desc->quad_points - 1;
    dq.quad_points = 0;
    st = create_impl(&dq, &h->inner, /*point_op=*/true);
    if (st == DGX_OK) {
      h->inner->pen_k = h->p;
      h->Mq = desc->quad_points;
      oi_matrices(h);
    }
  }
  if (st != DGX_OK) {
    dgx_destroy(h);
    return st;
  }
  *out = h;
  return DGX_OK;
}

dgx_status dgx_create(const dgx_problem_desc* desc, dgx_handle** out) { return create_impl(desc, out, false); }

dgx_status dgx_destroy(dgx_handle* h) {
  if (!h) return DGX_EINVAL;
  if (h->inner) dgx_destroy(h->inner);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  free_mesh(h);
  if (h->d_mask) cudaFree(h->d_mask);
  if (h->d_tabs) cudaFree(h->d_tabs);
  if (h->d_flags) cudaFree(h->d_flags);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->side) cudaStreamDestroy(h->side);
  delete h;
  return DGX_OK;
}

dgx_status dgx_query(const dgx_handle* h, int32_t* n_elem, int32_t* nodes, int32_t* fields, int32_t* face_points,
                     int32_t* tile) {
  if (!h) return DGX_EINVAL;
  if (n_elem) *n_elem = h->E;
  if (nodes) *nodes = h->N;
  if (fields) *fields = h->nf;
  if (face_points) *face_points = h->nfp;
  if (tile) *tile = h->T;
  return DGX_OK;
}

dgx_status dgx_set_mesh_boxes(dgx_handle* h, const double* lo, const double* size, const int32_t* neighbor,
                              const int8_t* nbr_face, const int8_t* orient) {
  if (!h || !lo || !size || !neighbor || !nbr_face || !orient) return DGX_EINVAL;
  const int E = h->E, d = h->d;
  for (size_t i = 0; i < (size_t)E * d; ++i)
    if (!(size[i] > 0.0) || !std::isfinite(size[i]) || !std::isfinite(lo[i])) return DGX_EINVAL;
  std::vector<int4> faces;
  dgx_status st = check_connectivity(h, neighbor, nbr_face, orient, faces);
  if (st != DGX_OK) return st;
  free_mesh(h);
  std::vector<double> rh((size_t)E * d);
  for (size_t i = 0; i < rh.size(); ++i) rh[i] = 2.0 / size[i];
  if ((st = upload_connectivity(h, neighbor, nbr_face, orient, faces)) != DGX_OK) return st;
  if ((st = upload_real(h, rh, &h->d_rh)) != DGX_OK) return st;
  {  // 1/l = |dT| / |T| = 2 sum_a 1/h_a for a box (SIPG penalty), FP64 corners and sizes
    std::vector<double> il(E, 0.0);
    for (int e = 0; e < E; ++e)
      for (int a = 0; a < d; ++a) il[e] += 2.0 / size[(size_t)e * d + a];
    std::vector<double> vlo(lo, lo + (size_t)E * d), vsz(size, size + (size_t)E * d);
    if ((st = upload_real(h, il, &h->d_il)) != DGX_OK) return st;
    if ((st = upload(vlo, (void**)&h->d_lo)) != DGX_OK) return st;
    if ((st = upload(vsz, (void**)&h->d_size)) != DGX_OK) return st;
  }
  h->h_lo.assign(lo, lo + (size_t)E * d);
  h->h_size.assign(size, size + (size_t)E * d);
  h->h_xyz.clear();
  h->curv = false;
  h->geo_override = false;
  h->mesh64 = mesh_view<double>(h);
  h->mesh32 = mesh_view<float>(h);
  if (h->inner && (st = dgx_set_mesh_boxes(h->inner, lo, size, neighbor, nbr_face, orient)) != DGX_OK) return st;
  h->has_mesh = true;
  return DGX_OK;
}

namespace {

// Gauss-Lobatto points of n >= 2 per direction on [-1, 1], ascending: the
// end points and the roots of P'_{n-1}, by Newton's method from the
// Chebyshev-Lobatto points (P and P' by the three-term recurrence,
// P'' = (2x P' - p(p+1) P) / (1 - x^2)).
std::vector<double> lobatto_points(int n) {
  const int p = n - 1;
  std::vector<double> x(n);
  x[0] = -1.0;
  x[p] = 1.0;
  for (int j = 1; j < p; ++j) {
    double t = -std::cos(M_PI * j / p);
    for (int it = 0; it < 100; ++it) {
      double P0 = 1.0, P1 = t;
      for (int k = 1; k < p; ++k) {
        const double P2 = ((2 * k + 1) * t * P1 - k * P0) / (k + 1);
        P0 = P1;
        P1 = P2;
      }
      const double dP = p * (P0 - t * P1) / (1.0 - t * t);             // P_p'
      const double d2P = (2.0 * t * dP - p * (p + 1.0) * P1) / (1.0 - t * t);  // P_p''
      const double dt = dP / d2P;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    x[j] = t;
  }
  return x;
}

// L[m][j] = l_j(xe_m), the Lagrange basis through nodes x at the points xe
std::vector<double> lagrange_matrix(const std::vector<double>& x, const std::vector<double>& xe) {
  const int n = (int)x.size(), m = (int)xe.size();
  std::vector<double> L((size_t)m * n, 1.0);
  for (int r = 0; r < m; ++r)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k)
        if (k != j) L[r * n + j] *= (xe[r] - x[k]) / (x[j] - x[k]);
  return L;
}

// D[i][j] = l_j'(x_i) by barycentric weights, rows summing to zero
std::vector<double> derivative_matrix(const std::vector<double>& x) {
  const int n = (int)x.size();
  std::vector<double> b(n, 1.0), D((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) b[j] /= (x[j] - x[k]);
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < n; ++j)
      if (j != i) {
        D[i * n + j] = (b[j] / b[i]) / (x[i] - x[j]);
        s += D[i * n + j];
      }
    D[i * n + i] = -s;
  }
  return D;
}

// Metric terms of the degree-p element maps given by their node coordinates
// (host, FP64): Ja[E][a][c][N] = J dxi_a/dx_c, iJ[E][N] = 1/J and, when
// asked, J[E][N] (J = det dx/dxi at each node).  2D: the cofactors of dx/dxi.
// 3D: the conservative curl form Ja[i][c] = -(D_j (X_l d_k X_m) - D_k (X_l
// d_j X_m)), (c, m, l) and (i, j, k) cyclic, with X_l d X_m taken as its
// degree-p interpolant through the Gauss-Lobatto points (the map evaluated
// there, X_l relative to the element's mean) and carried back to the Gauss
// nodes exactly: Ja is a degree-p polynomial per direction, so the Gauss
// derivative matrices satisfy the metric identities, and its trace on a face
// depends on that face's Lobatto points only, the same from both sides of a
// conforming face (a uniform flow stays at rest).  The mean offset drops out
// exactly (the curl of c grad X_m vanishes) and would only add rounding.
dgx_status nodal_metrics(int d, int p, int E, const double* xyz, std::vector<double>& Ja, std::vector<double>& iJ,
                         std::vector<double>* Jout) {
  const int n = p + 1, N = ipow(n, d);
  const Basis B = make_basis(p);
  // derivative of nodal data along direction a
  auto along = [&](const double* v, int a, double* out) {
    for (int q = 0; q < N; ++q) {
      const int fp = fpoint_of(n, q, a), qa = (q / pw(n, a)) % n;
      double s = 0.0;
      for (int m = 0; m < n; ++m) s += B.D[qa * n + m] * v[node_of(n, m, fp, a)];
      out[q] = s;
    }
  };
  // an n x n matrix along direction a of nodal data
  auto apply = [&](const double* Mat, const double* v, int a, double* out) {
    for (int q = 0; q < N; ++q) {
      const int fp = fpoint_of(n, q, a), qa = (q / pw(n, a)) % n;
      double s = 0.0;
      for (int m = 0; m < n; ++m) s += Mat[qa * n + m] * v[node_of(n, m, fp, a)];
      out[q] = s;
    }
  };
  std::vector<double> G2L, L2G, DL, XL, dXL;
  if (d == 3) {
    const std::vector<double> xl = lobatto_points(n), xg(B.x.begin(), B.x.end());
    G2L = lagrange_matrix(xg, xl);  // Gauss-node values -> the map at the Lobatto points
    L2G = lagrange_matrix(xl, xg);  // Lobatto values -> Gauss nodes
    DL = derivative_matrix(xl);
    XL.resize(3 * N);
    dXL.resize(9 * N);
  }
  Ja.assign((size_t)E * d * d * N, 0.0);
  iJ.assign((size_t)E * N, 0.0);
  if (Jout) Jout->assign((size_t)E * N, 0.0);
  std::vector<double> dX(d * d * N), G(N), tmp(N), tmp2(N);
  for (int e = 0; e < E; ++e) {
    const double* X = xyz + (size_t)e * d * N;
    for (int c = 0; c < d; ++c)
      for (int b = 0; b < d; ++b) along(X + c * N, b, &dX[(c * d + b) * N]);  // dX[c][b] = dx_c/dxi_b
    double* JaE = &Ja[(size_t)e * d * d * N];
    for (int q = 0; q < N; ++q) {
      double J;
      auto m = [&](int c, int b) { return dX[(c * d + b) * N + q]; };
      if (d == 2) {
        J = m(0, 0) * m(1, 1) - m(0, 1) * m(1, 0);
        JaE[(0 * d + 0) * N + q] = m(1, 1);
        JaE[(0 * d + 1) * N + q] = -m(0, 1);
        JaE[(1 * d + 0) * N + q] = -m(1, 0);
        JaE[(1 * d + 1) * N + q] = m(0, 0);
      } else {
        J = m(0, 0) * (m(1, 1) * m(2, 2) - m(1, 2) * m(2, 1)) - m(0, 1) * (m(1, 0) * m(2, 2) - m(1, 2) * m(2, 0)) +
            m(0, 2) * (m(1, 0) * m(2, 1) - m(1, 1) * m(2, 0));
      }
      if (!(J > 0.0)) return DGX_EINVAL;  // inverted or degenerate element
      iJ[(size_t)e * N + q] = 1.0 / J;
      if (Jout) (*Jout)[(size_t)e * N + q] = J;
    }
    if (d == 3) {
      // the map at the Lobatto points, relative to its mean
      for (int c = 0; c < 3; ++c) {
        apply(G2L.data(), X + c * N, 0, tmp.data());
        apply(G2L.data(), tmp.data(), 1, tmp2.data());
        apply(G2L.data(), tmp2.data(), 2, &XL[c * N]);
        double mean = 0.0;
        for (int q = 0; q < N; ++q) mean += XL[c * N + q];
        mean /= N;
        for (int q = 0; q < N; ++q) XL[c * N + q] -= mean;
        for (int b = 0; b < 3; ++b) apply(DL.data(), &XL[c * N], b, &dXL[(c * 3 + b) * N]);
      }
      for (int c = 0; c < 3; ++c) {
        const int mm = (c + 1) % 3, ll = (c + 2) % 3;
        for (int i = 0; i < 3; ++i) {
          const int j = (i + 1) % 3, k = (i + 2) % 3;
          for (int q = 0; q < N; ++q) G[q] = XL[ll * N + q] * dXL[(mm * 3 + k) * N + q];
          apply(DL.data(), G.data(), j, tmp.data());
          for (int q = 0; q < N; ++q) G[q] = XL[ll * N + q] * dXL[(mm * 3 + j) * N + q];
          apply(DL.data(), G.data(), k, tmp2.data());
          for (int q = 0; q < N; ++q) G[q] = -(tmp[q] - tmp2[q]);  // at the Lobatto points
          apply(L2G.data(), G.data(), 0, tmp.data());
          apply(L2G.data(), tmp.data(), 1, tmp2.data());
          apply(L2G.data(), tmp2.data(), 2, &JaE[(i * 3 + c) * N]);
        }
      }
    }
  }
  return DGX_OK;
}

// The node coordinates [E][d][n^d] of the degree-p maps evaluated at the M
// points per direction ([E][d][M^d]): the [M][n] matrix I along each direction.
std::vector<double> interpolate_nodes(int d, int n, int M, int E, const double* xyz, const double* I) {
  const int N = ipow(n, d), NQ = ipow(M, d);
  std::vector<double> out((size_t)E * d * NQ), a(NQ), b(NQ);
  for (size_t r = 0; r < (size_t)E * d; ++r) {
    std::copy(xyz + r * N, xyz + (r + 1) * N, a.begin());
    int lo = 1;  // extent of the directions already at M points
    for (int dir = 0; dir < d; ++dir) {
      const int hi = ipow(n, d - 1 - dir);  // directions still at the nodes
      for (int t = 0; t < hi; ++t)
        for (int m = 0; m < M; ++m)
          for (int l = 0; l < lo; ++l) {
            double s = 0.0;
            for (int j = 0; j < n; ++j) s += I[m * n + j] * a[l + lo * (j + n * t)];
            b[l + lo * (m + M * t)] = s;
          }
      std::swap(a, b);
      lo *= M;
    }
    std::copy(a.begin(), a.begin() + NQ, out.begin() + r * NQ);
  }
  return out;
}

// Curved mesh of handle h; J_out (optional) receives J at the nodes.  An
// over-integrated handle also gives its point operator the element maps at
// the M points and keeps J there for the projection's weights.
dgx_status set_nodes_impl(dgx_handle* h, const double* xyz, const int32_t* neighbor, const int8_t* nbr_face,
                          const int8_t* orient, std::vector<double>* J_out) {
  const int E = h->E, d = h->d, N = h->N;
  for (size_t i = 0; i < (size_t)E * d * N; ++i)
    if (!std::isfinite(xyz[i])) return DGX_EINVAL;
  std::vector<int4> faces;
  dgx_status st = check_connectivity(h, neighbor, nbr_face, orient, faces);
  if (st != DGX_OK) return st;
  std::vector<double> Ja, iJ;
  if ((st = nodal_metrics(d, h->p, E, xyz, Ja, iJ, J_out)) != DGX_OK) return st;
  free_mesh(h);
  if ((st = upload_connectivity(h, neighbor, nbr_face, orient, faces)) != DGX_OK) return st;
  if ((st = upload_metrics(h, Ja, iJ, faces)) != DGX_OK) return st;
  if (h->dgip && (st = upload_dgip_metrics(h, Ja, iJ)) != DGX_OK) return st;
  if (h->inner) {
    const std::vector<double> xq = interpolate_nodes(d, h->n, h->Mq, E, xyz, h->oiI);
    std::vector<double> Jq;
    if ((st = set_nodes_impl(h->inner, xq.data(), neighbor, nbr_face, orient, &Jq)) != DGX_OK ||
        (st = upload_real(h, Jq, &h->d_oiJq)) != DGX_OK) {
      free_mesh(h);
      return st;
    }
  }
  h->h_xyz.assign(xyz, xyz + (size_t)E * d * N);
  h->h_lo.clear();
  h->h_size.clear();
  h->curv = true;
  h->geo_override = false;
  h->has_mesh = true;
  h->mesh64 = mesh_view<double>(h);
  h->mesh32 = mesh_view<float>(h);
  return DGX_OK;
}

}  // namespace

dgx_status dgx_set_mesh_nodes(dgx_handle* h, const double* xyz, const int32_t* neighbor, const int8_t* nbr_face,
                              const int8_t* orient) {
  if (!h || !xyz || !neighbor || !nbr_face || !orient) return DGX_EINVAL;
  return set_nodes_impl(h, xyz, neighbor, nbr_face, orient, nullptr);
}

dgx_status dgx_mesh_metrics(int32_t dim, int32_t p, int32_t n_elem, const double* xyz, double* J, double* metric) {
  if (!xyz || !J || !metric || (dim != 2 && dim != 3) || p < 1 || p > dgx::MAXN - 1 || n_elem < 1)
    return DGX_EINVAL;
  const int N = ipow(p + 1, dim);
  for (size_t i = 0; i < (size_t)n_elem * dim * N; ++i)
    if (!std::isfinite(xyz[i])) return DGX_EINVAL;
  std::vector<double> Ja, iJ, Jv;
  const dgx_status st = nodal_metrics(dim, p, n_elem, xyz, Ja, iJ, &Jv);
  if (st != DGX_OK) return st;
  std::copy(Jv.begin(), Jv.end(), J);
  for (int e = 0; e < n_elem; ++e)
    for (int q = 0; q < N; ++q)
      for (int a = 0; a < dim; ++a)
        for (int c = 0; c < dim; ++c)
          metric[(((size_t)e * N + q) * dim + a) * dim + c] = Ja[(((size_t)e * dim + a) * dim + c) * N + q];
  return DGX_OK;
}

dgx_status dgx_set_geometry(dgx_handle* h, const double* J, const double* metric) {
  if (!h || !J || !metric) return DGX_EINVAL;
  // the point operator of over-integration needs the geometry at the M
  // points, which nodal values of J and the metric do not determine
  if (h->inner) return DGX_EUNSUPPORTED;
  if (!h->has_mesh) return DGX_ESTATE;
  const int E = h->E, d = h->d, N = h->N;
  for (size_t i = 0; i < (size_t)E * N; ++i)
    if (!(J[i] > 0.0) || !std::isfinite(J[i])) return DGX_EINVAL;
  for (size_t i = 0; i < (size_t)E * N * d * d; ++i)
    if (!std::isfinite(metric[i])) return DGX_EINVAL;
  std::vector<double> Ja((size_t)E * d * d * N), iJ((size_t)E * N);
  for (int e = 0; e < E; ++e)
    for (int q = 0; q < N; ++q) {
      iJ[(size_t)e * N + q] = 1.0 / J[(size_t)e * N + q];
      for (int a = 0; a < d; ++a)
        for (int c = 0; c < d; ++c)
          Ja[(((size_t)e * d + a) * d + c) * N + q] = metric[(((size_t)e * N + q) * d + a) * d + c];
    }
  std::vector<int4> faces;
  dgx_status st = check_connectivity(h, h->h_nb.data(), h->h_nbf.data(), h->h_ori.data(), faces);
  if (st != DGX_OK) return st;
  void** geo[] = {&h->d_Ja, &h->d_iJ, &h->d_SnE, &h->d_SnF, &h->d_JaF, &h->d_iJF, &h->d_il};
  for (void** g : geo)
    if (*g) {
      cudaFree(*g);
      *g = nullptr;
    }
  if ((st = upload_metrics(h, Ja, iJ, faces)) != DGX_OK ||
      (h->dgip && (st = upload_dgip_metrics(h, Ja, iJ)) != DGX_OK)) {
    free_mesh(h);
    return st;
  }
  h->curv = true;
  h->geo_override = true;
  h->mesh64 = mesh_view<double>(h);
  h->mesh32 = mesh_view<float>(h);
  return DGX_OK;
}

dgx_status dgx_set_tableau(dgx_handle* h, int32_t stages, const double* A, const double* b, const double* c) {
  if (!h || !A || !b || !c || stages < 1 || stages > dgx::MAXSTAGES) return DGX_EINVAL;
  for (int i = 0; i < stages; ++i)
    for (int j = i; j < stages; ++j)
      if (A[i * stages + j] != 0.0) return DGX_EINVAL;  // explicit only
  h->stages = stages;
  for (int i = 0; i < stages; ++i) {
    for (int j = 0; j < stages; ++j) h->A[i * dgx::MAXSTAGES + j] = A[i * stages + j];
    h->b[i] = b[i];
    h->c[i] = c[i];
  }
  return DGX_OK;
}

size_t dgx_stage_bytes(const dgx_handle* h) {
  if (!h || h->stages == 0) return 0;
  return slot_layout(h).bytes * h->stages;
}

size_t dgx_workspace_bytes(const dgx_handle* h, int32_t op) {
  if (!h) return 0;
  if (op == DGX_OP_ARK && h->stages == 0) return 0;
  if ((op == DGX_OP_ARK_ADJOINT || op == DGX_OP_ARK_STEP_ADJOINT) && h->stages == 0) return 0;
  if (op == DGX_OP_HDG) {
    if (!h->fp64 || h->d != 2) return 0;
    const size_t nu = (size_t)h->nf * h->N;
    return align256((size_t)h->E * nu * nu * sizeof(double));
  }
  if (op < DGX_OP_RHS || op > DGX_OP_ARK_STEP_ADJOINT) return 0;
  if ((op == DGX_OP_VJP || op == DGX_OP_ARK_ADJOINT || op == DGX_OP_ARK_STEP_ADJOINT) && !h->tab->vjp) return 0;
  if (h->inner) {
    if (op == DGX_OP_ARK_STEP_ADJOINT) return layout_oi(h, DGX_OP_ARK).total + layout_oi(h, DGX_OP_ARK_ADJOINT).total;
    return layout_oi(h, op).total;
  }
  if (op == DGX_OP_ARK_STEP_ADJOINT)  // the forward's and the adjoint's workspaces side by side
    return layout(h, DGX_OP_ARK).total + layout(h, DGX_OP_ARK_ADJOINT).total;
  return layout(h, op).total;
}

dgx_status dgx_rhs(dgx_handle* h, const void* U, void* dUdt, void* workspace, void* stream) {
  if (!h || !U || !dUdt || !workspace || U == dUdt) return DGX_EINVAL;
  if (!h->has_mesh) return DGX_ESTATE;
  if (((uintptr_t)workspace & 255) != 0) return DGX_EINVAL;
  if (h->dgip) {
    if (h->has_farfield && !h->has_uinf) return DGX_ESTATE;
    cudaStream_t st = (cudaStream_t)stream;
    if (h->inner) {
      const OiLayout L = layout_oi(h, DGX_OP_RHS);
      return cuda_status(h->fp64 ? oi_residual<double>(h, U, nullptr, dUdt, (char*)workspace, L, st)
                                 : oi_residual<float>(h, U, nullptr, dUdt, (char*)workspace, L, st));
    }
    const dgx::DgipWork w = dgip_work_at(h, workspace, layout(h, DGX_OP_RHS));
    return cuda_status(h->fp64 ? dgip_residual<double>(h, U, nullptr, nullptr, dUdt, w, nullptr, st)
                               : dgip_residual<float>(h, U, nullptr, nullptr, dUdt, w, nullptr, st));
  }
  const Layout L = layout(h, DGX_OP_RHS);
  const dgx::Work w = work_at(h, workspace, L);
  cudaStream_t st = (cudaStream_t)stream;
  const void* M = h->fp64 ? (const void*)&h->mesh64 : (const void*)&h->mesh32;
  const dgx::Table* t = h->tab;
  cudaError_t err = launch(h, DGX_K_TRACE, st, [&] { return t->trace(M, h->var[DGX_K_TRACE], U, w.TU, st); });
  if (err == cudaSuccess && h->viscous)
    err = launch(h, DGX_K_BR1, st, [&] { return t->br1(M, h->var[DGX_K_BR1], h->curv, U, w, st); });
  if (err == cudaSuccess) err = launch(h, DGX_K_FACE, st, [&] { return t->face(M, h->viscous, h->curv, w, st); });
  if (err == cudaSuccess)
    err = launch(h, DGX_K_ELEM, st, [&] {
      if (h->contraction != DGX_CONTRACT_CUDA_CORE)
        return t->elem_tc(M, h->contraction, h->viscous, h->curv, U, w, dUdt, nullptr, st);
      bool used = false;
      if (h->pipeline) {
        const cudaError_t e = t->elem_pipe(M, h->var[DGX_K_ELEM], h->viscous, h->curv, U, w, dUdt, nullptr, h->nsm,
                                           st, &used);
        if (e != cudaSuccess || used) return e;
      }
      return t->elem(M, h->var[DGX_K_ELEM], h->viscous, h->curv, U, w, dUdt, st);
    });
  return cuda_status(err);
}

dgx_status dgx_rhs_vjp(dgx_handle* h, const void* U, const void* lambda, void* gU, void* workspace, void* stream) {
  if (!h || !U || !lambda || !gU || !workspace || gU == U || gU == lambda) return DGX_EINVAL;
  if (!h->has_mesh) return DGX_ESTATE;
  if (!h->tab->vjp) return DGX_EUNSUPPORTED;
  if (((uintptr_t)workspace & 255) != 0) return DGX_EINVAL;
  if (h->dgip) {
    if (h->has_farfield && !h->has_uinf) return DGX_ESTATE;
    cudaStream_t st = (cudaStream_t)stream;
    if (h->inner) {
      const OiLayout L = layout_oi(h, DGX_OP_VJP);
      return cuda_status(h->fp64 ? oi_vjp<double>(h, U, lambda, gU, (char*)workspace, L, st)
                                 : oi_vjp<float>(h, U, lambda, gU, (char*)workspace, L, st));
    }
    const dgx::DgipWork w = dgip_work_at(h, workspace, layout(h, DGX_OP_VJP));
    return cuda_status(h->fp64 ? dgip_vjp<double>(h, U, lambda, gU, w, st) : dgip_vjp<float>(h, U, lambda, gU, w, st));
  }
  const Layout L = layout(h, DGX_OP_VJP);
  const dgx::VjpWork vw = vjp_work_at(h, workspace, L);
  cudaStream_t st = (cudaStream_t)stream;
  if (h->fp64) {
    dgx::Cot<double> cot{}, fin{};
    cot.lam = (const double*)lambda;
    cot.c_lam = 1.0;
    return cuda_status(vjp_chain<double>(h, U, cot, fin, gU, vw, st));
  }
  dgx::Cot<float> cot{}, fin{};
  cot.lam = (const float*)lambda;
  cot.c_lam = 1.0;
  return cuda_status(vjp_chain<float>(h, U, cot, fin, gU, vw, st));
}

dgx_status dgx_ark_step(dgx_handle* h, double* U64, double dt, void* workspace, void* stream) {
  if (!h || !U64 || !workspace || !std::isfinite(dt)) return DGX_EINVAL;
  if (!h->has_mesh || h->stages == 0) return DGX_ESTATE;
  if (((uintptr_t)workspace & 255) != 0) return DGX_EINVAL;
  if (h->dgip) {
    if (h->has_farfield && !h->has_uinf) return DGX_ESTATE;
    if (h->inner)
      return h->fp64 ? oi_ark_impl<double>(h, U64, dt, nullptr, workspace, (cudaStream_t)stream)
                     : oi_ark_impl<float>(h, U64, dt, nullptr, workspace, (cudaStream_t)stream);
    return h->fp64 ? dgip_ark_impl<double>(h, U64, dt, nullptr, workspace, (cudaStream_t)stream)
                   : dgip_ark_impl<float>(h, U64, dt, nullptr, workspace, (cudaStream_t)stream);
  }
  if (h->fp64) return ark_impl<double>(h, U64, dt, nullptr, workspace, (cudaStream_t)stream);
  return ark_impl<float>(h, U64, dt, nullptr, workspace, (cudaStream_t)stream);
}

dgx_status dgx_ark_step_stages(dgx_handle* h, double* U64, double dt, void* stages, void* workspace, void* stream) {
  if (!h || !U64 || !stages || !workspace || !std::isfinite(dt)) return DGX_EINVAL;
  if (((uintptr_t)stages & 255) != 0) return DGX_EINVAL;
  if (!h->has_mesh || h->stages == 0) return DGX_ESTATE;
  if (((uintptr_t)workspace & 255) != 0) return DGX_EINVAL;
  if (h->dgip) {
    if (h->has_farfield && !h->has_uinf) return DGX_ESTATE;
    if (h->inner)
      return h->fp64 ? oi_ark_impl<double>(h, U64, dt, stages, workspace, (cudaStream_t)stream)
                     : oi_ark_impl<float>(h, U64, dt, stages, workspace, (cudaStream_t)stream);
    return h->fp64 ? dgip_ark_impl<double>(h, U64, dt, stages, workspace, (cudaStream_t)stream)
                   : dgip_ark_impl<float>(h, U64, dt, stages, workspace, (cudaStream_t)stream);
  }
  if (h->fp64) return ark_impl<double>(h, U64, dt, stages, workspace, (cudaStream_t)stream);
  return ark_impl<float>(h, U64, dt, stages, workspace, (cudaStream_t)stream);
}

dgx_status dgx_ark_adjoint_step(dgx_handle* h, const void* stages, double* lam64, double dt, void* workspace,
                                void* stream) {
  if (!h || !stages || !lam64 || !workspace || !std::isfinite(dt)) return DGX_EINVAL;
  if (!h->has_mesh || h->stages == 0) return DGX_ESTATE;
  if (!h->tab->vjp) return DGX_EUNSUPPORTED;
  if (((uintptr_t)workspace & 255) != 0) return DGX_EINVAL;
  if (h->dgip && h->has_farfield && !h->has_uinf) return DGX_ESTATE;
  if (h->inner)
    return h->fp64 ? oi_ark_adjoint_impl<double>(h, stages, lam64, dt, workspace, (cudaStream_t)stream)
                   : oi_ark_adjoint_impl<float>(h, stages, lam64, dt, workspace, (cudaStream_t)stream);
  if (h->dgip)
    return h->fp64 ? dgip_ark_adjoint_impl<double>(h, stages, lam64, dt, workspace, (cudaStream_t)stream)
                   : dgip_ark_adjoint_impl<float>(h, stages, lam64, dt, workspace, (cudaStream_t)stream);
  if (h->fp64) return ark_adjoint_impl<double>(h, stages, lam64, dt, workspace, (cudaStream_t)stream);
  return ark_adjoint_impl<float>(h, stages, lam64, dt, workspace, (cudaStream_t)stream);
}

dgx_status dgx_ark_step_adjoint(dgx_handle* h, double* U64, double* lam64, double dt, void* stages, void* workspace,
                                void* stream) {
  if (!h || !U64 || !lam64 || !stages || !workspace || !std::isfinite(dt)) return DGX_EINVAL;
  if (((uintptr_t)stages & 255) != 0 || ((uintptr_t)workspace & 255) != 0) return DGX_EINVAL;
  if (!h->has_mesh || h->stages == 0) return DGX_ESTATE;
  if (!h->tab->vjp) return DGX_EUNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  if (h->dgip && h->has_farfield && !h->has_uinf) return DGX_ESTATE;
  if (h->inner) {  // the step, then its adjoint, on the caller's stream
    char* ws2 = (char*)workspace + layout_oi(h, DGX_OP_ARK).total;
    dgx_status s = h->fp64 ? oi_ark_impl<double>(h, U64, dt, stages, workspace, st)
                           : oi_ark_impl<float>(h, U64, dt, stages, workspace, st);
    if (s == DGX_OK)
      s = h->fp64 ? oi_ark_adjoint_impl<double>(h, stages, lam64, dt, ws2, st)
                  : oi_ark_adjoint_impl<float>(h, stages, lam64, dt, ws2, st);
    return s;
  }
  if (h->dgip) {  // the step, then its adjoint, on the caller's stream
    char* ws2 = (char*)workspace + layout(h, DGX_OP_ARK).total;
    dgx_status s = h->fp64 ? dgip_ark_impl<double>(h, U64, dt, stages, workspace, st)
                           : dgip_ark_impl<float>(h, U64, dt, stages, workspace, st);
    if (s == DGX_OK)
      s = h->fp64 ? dgip_ark_adjoint_impl<double>(h, stages, lam64, dt, ws2, st)
                  : dgip_ark_adjoint_impl<float>(h, stages, lam64, dt, ws2, st);
    return s;
  }
  char* ws_adj = (char*)workspace + layout(h, DGX_OP_ARK).total;  // a multiple of 256 bytes
  dgx_status s = h->fp64 ? ark_impl<double>(h, U64, dt, stages, workspace, st, nullptr, /*fork=*/true)
                         : ark_impl<float>(h, U64, dt, stages, workspace, st, nullptr, /*fork=*/true);
  if (s != DGX_OK) {  // whatever reached the second stream still joins the caller's
    cudaEventRecord(h->ev_join, h->side);
    cudaStreamWaitEvent(st, h->ev_join, 0);
    return s;
  }
  s = h->fp64 ? ark_adjoint_impl<double>(h, stages, lam64, dt, ws_adj, st)
              : ark_adjoint_impl<float>(h, stages, lam64, dt, ws_adj, st);
  if (cudaStreamWaitEvent(st, h->ev_join, 0) != cudaSuccess && s == DGX_OK) s = DGX_ECUDA;
  return s;
}

dgx_status dgx_set_wait_limit(dgx_handle* h, int64_t polls) {
  if (!h) return DGX_EINVAL;
  h->wait_polls = polls < 0 ? (1u << 22) : (uint32_t)std::min<int64_t>(polls, 1u << 22);
  h->mesh64.wait_polls = h->wait_polls;
  h->mesh32.wait_polls = h->wait_polls;
  return h->inner ? dgx_set_wait_limit(h->inner, polls) : DGX_OK;
}

dgx_status dgx_hdg_sizes(const dgx_handle* h, int32_t* nu, int32_t* nh) {
  if (!h) return DGX_EINVAL;
  if (nu) *nu = h->nf * h->N;
  if (nh) *nh = h->NF * h->nf * h->nfp;
  return DGX_OK;
}

dgx_status dgx_hdg_blocks(dgx_handle* h, const double* U, const double* Uhat, double gamma, double* K, double* C,
                          double* D, double* A33, double* R, double* hres, void* stream) {
  if (!h || !U || !Uhat || !K || !C || !D || !A33 || !std::isfinite(gamma) || (!R) != (!hres)) return DGX_EINVAL;
  if (!h->fp64 || h->d != 2 || h->inner) return DGX_EUNSUPPORTED;
  if (!h->has_mesh) return DGX_ESTATE;
  if (h->curv && !h->d_JaF) return DGX_EUNSUPPORTED;  // curved: the DG-IP face metric (DG-IP handles)
  if (h->has_farfield && !h->has_uinf) return DGX_ESTATE;
  dgx::HdgArgs a{};
  a.E = h->E;
  if (h->curv) {
    a.Ja = (const double*)h->d_Ja;
    a.iJ = (const double*)h->d_iJ;
    a.SnE = (const double*)h->d_SnE;
    a.JaF = (const double*)h->d_JaF;
    a.iJF = (const double*)h->d_iJF;
  } else {
    a.rh = (const double*)h->d_rh;
  }
  a.il = (const double*)h->d_il;
  a.nb = h->d_nb;
  a.tk2 = 10.0 * (h->p + 1) * (h->p + 1);
  const dgx::Basis1 b = dgx::make_basis1(h->p);
  for (int i = 0; i < b.n; ++i) a.w[i] = b.w[i];
  for (int f = 0; f < 4; ++f) a.Uinf[f] = h->Uinf[f];
  a.gas = h->mesh64.gas;
  return cuda_status(dgx::hdg_jacobian(h->p, a, U, Uhat, gamma, K, C, D, A33, R, hres, (cudaStream_t)stream));
}

dgx_status dgx_hdg_condense(dgx_handle* h, const double* K, const double* C, const double* D, const double* A33,
                            double* KinvC, double* S, void* workspace, void* stream) {
  if (!h || !K || !C || !D || !A33 || !KinvC || !S || !workspace) return DGX_EINVAL;
  if (((uintptr_t)workspace & 255) != 0) return DGX_EINVAL;
  if (!h->fp64 || h->d != 2 || h->inner) return DGX_EUNSUPPORTED;
  if (!h->has_mesh) return DGX_ESTATE;
  const int nu = h->nf * h->N, nh = h->NF * h->nf * h->nfp;
  return cuda_status(dgx::hdg_condense(h->E, nu, nh, K, C, D, A33, KinvC, S, (double*)workspace,
                                       (cudaStream_t)stream));
}

dgx_status dgx_set_farfield(dgx_handle* h, const double* U_inf) {
  if (!h || !U_inf) return DGX_EINVAL;
  if (!h->dgip) return DGX_EUNSUPPORTED;
  for (int f = 0; f < h->nf; ++f)
    if (!std::isfinite(U_inf[f])) return DGX_EINVAL;
  double m2 = 0.0;
  for (int i = 0; i < h->d; ++i) m2 += U_inf[1 + i] * U_inf[1 + i];
  const double p = (h->desc.gamma - 1.0) * (U_inf[h->d + 1] - 0.5 * m2 / U_inf[0]);
  if (!(U_inf[0] > 0.0) || !(p > 0.0)) return DGX_EINVAL;  // not a physical state
  for (int f = 0; f < 5; ++f) h->Uinf[f] = f < h->nf ? U_inf[f] : 0.0;
  h->has_uinf = true;
  return h->inner ? dgx_set_farfield(h->inner, U_inf) : DGX_OK;
}

dgx_status dgx_set_explicit_mask(dgx_handle* h, const int8_t* mask) {
  if (!h) return DGX_EINVAL;
  if (!h->dgip) return DGX_EUNSUPPORTED;
  if (!mask) {
    if (h->d_mask) cudaFree(h->d_mask);
    h->d_mask = nullptr;
    return DGX_OK;
  }
  std::vector<int8_t> m(mask, mask + h->E);
  for (int8_t& v : m) v = v ? 1 : 0;
  return upload(m, (void**)&h->d_mask);
}

dgx_status dgx_rhs_split(dgx_handle* h, const void* U_ex, const void* U_im, void* dUdt, void* workspace,
                         void* stream) {
  if (!h || !U_ex || !U_im || !dUdt || !workspace || dUdt == U_ex || dUdt == U_im) return DGX_EINVAL;
  if (!h->dgip) return DGX_EUNSUPPORTED;
  if (!h->has_mesh || !h->d_mask) return DGX_ESTATE;
  if (h->has_farfield && !h->has_uinf) return DGX_ESTATE;
  if (((uintptr_t)workspace & 255) != 0) return DGX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (h->inner) {
    const OiLayout L = layout_oi(h, DGX_OP_RHS);
    return cuda_status(h->fp64 ? oi_residual<double>(h, U_ex, U_im, dUdt, (char*)workspace, L, st)
                               : oi_residual<float>(h, U_ex, U_im, dUdt, (char*)workspace, L, st));
  }
  const dgx::DgipWork w = dgip_work_at(h, workspace, layout(h, DGX_OP_RHS));
  return cuda_status(h->fp64 ? dgip_residual<double>(h, U_ex, h->d_mask, U_im, dUdt, w, nullptr, st)
                             : dgip_residual<float>(h, U_ex, h->d_mask, U_im, dUdt, w, nullptr, st));
}

dgx_status dgx_mms_source(dgx_handle* h, double t, double kx, double ky, double omega, void* dUdt, void* stream) {
  if (!h || !dUdt || !std::isfinite(t) || !std::isfinite(kx) || !std::isfinite(ky) || !std::isfinite(omega))
    return DGX_EINVAL;
  if (h->d != 2) return DGX_EUNSUPPORTED;
  if (!h->has_mesh || h->curv || !h->d_lo) return DGX_ESTATE;
  dgx::MmsNodes nodes{};
  const dgx::Basis1 b = dgx::make_basis1(h->p);
  for (int i = 0; i < b.n; ++i) nodes.xi[i] = b.x[i];
  const double mu = h->viscous ? 1.0 / h->desc.Re : 0.0;
  const double kcv = h->viscous ? h->desc.gamma * mu / h->desc.Pr : 0.0;
  const long long total = (long long)h->E * h->N;
  const int blocks = (int)((total + 255) / 256);
  cudaStream_t st = (cudaStream_t)stream;
  if (h->fp64)
    dgx::k_mms_source<double><<<blocks, 256, 0, st>>>(h->E, h->n, nodes, h->d_lo, h->d_size, t, kx, ky, omega,
                                                      h->desc.gamma - 1.0, kcv, (double*)dUdt);
  else
    dgx::k_mms_source<float><<<blocks, 256, 0, st>>>(h->E, h->n, nodes, h->d_lo, h->d_size, t, kx, ky, omega,
                                                     h->desc.gamma - 1.0, kcv, (float*)dUdt);
  return cuda_status(cudaGetLastError());
}

dgx_status dgx_check(dgx_handle* h) {
  if (!h) return DGX_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return DGX_ECUDA;
  unsigned flags = 0;
  if (cudaMemcpy(&flags, h->d_flags, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return DGX_ECUDA;
  if (cudaMemset(h->d_flags, 0, sizeof(unsigned)) != cudaSuccess) return DGX_ECUDA;
  if (h->inner) {  // the point residuals' flags
    const dgx_status si = dgx_check(h->inner);
    if (si == DGX_ECUDA) return si;
    if (si == DGX_ENONFINITE) flags |= 1u;
    if (si == DGX_ETIMEOUT) flags |= 2u;
  }
  if (flags & 1u) return DGX_ENONFINITE;
  if (flags & 2u) return DGX_ETIMEOUT;
  return DGX_OK;
}

static dgx_status autotune_impl(dgx_handle* h, const double* U64, int32_t reps, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const size_t state64 = (size_t)h->E * h->nf * h->N * 8;
  const bool adj = h->tab->vjp != nullptr;
  DevBuf<double> U, lam;
  DevBuf<char> stages, ws_ark, ws_adj;
  if (!U.alloc(state64) || !lam.alloc(state64) || !stages.alloc(dgx_stage_bytes(h) + 256) ||
      !ws_ark.alloc(dgx_workspace_bytes(h, DGX_OP_ARK) + 256) ||
      (adj && !ws_adj.alloc(dgx_workspace_bytes(h, DGX_OP_ARK_ADJOINT) + 256)))
    return DGX_ENOMEM;
  auto al = [](char* p) { return (void*)(((uintptr_t)p + 255) & ~(uintptr_t)255); };
  const bool was_prof = h->prof;
  dgx_status s = dgx_profile_enable(h, 1);
  if (s != DGX_OK) return s;
  const double dt = 1e-12;
  double best[DGX_KERNEL_KINDS];
  int choice[DGX_KERNEL_KINDS];
  for (int k = 0; k < DGX_KERNEL_KINDS; ++k) {
    best[k] = 1e300;
    choice[k] = h->var[k];
  }
  for (int V = 0; V < dgx::NVARIANTS; ++V) {
    bool valid[DGX_KERNEL_KINDS] = {};
    for (int k = 0; k < DGX_KERNEL_KINDS; ++k) {
      if (!is_tile_kind(k)) continue;
      valid[k] = tile_smem(h, k, V) <= dgx::SMEM_LIMIT;
      h->var[k] = valid[k] ? V : choice[k];
    }
    for (int rep = -1; rep < reps; ++rep) {  // rep -1: warm-up
      if (rep == 0) dgx_profile_reset(h);
      if (cudaMemcpyAsync(U.p, U64, state64, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return DGX_ECUDA;
      if (cudaMemsetAsync(lam.p, 0, state64, st) != cudaSuccess) return DGX_ECUDA;
      s = dgx_ark_step_stages(h, U.p, dt, al(stages.p), al(ws_ark.p), stream);
      if (s == DGX_OK && adj) s = dgx_ark_adjoint_step(h, al(stages.p), lam.p, dt, al(ws_adj.p), stream);
      if (s != DGX_OK) {
        dgx_profile_enable(h, was_prof);
        return s;
      }
    }
    for (int k = 0; k < DGX_KERNEL_KINDS; ++k) {
      int64_t n = 0;
      double ms = 0;
      dgx_profile_read(h, k, &n, &ms);
      if (valid[k] && n > 0 && ms / n < best[k]) {
        best[k] = ms / n;
        choice[k] = V;
      }
    }
  }
  for (int k = 0; k < DGX_KERNEL_KINDS; ++k) h->var[k] = choice[k];
  // persistent TMA-fed element kernel or not: keep whichever is faster
  double elem_ms[2] = {1e300, 1e300};
  const bool was_pipe = h->pipeline;
  for (int pipe = 0; pipe < 2; ++pipe) {
    h->pipeline = pipe != 0;
    for (int rep = -1; rep < reps; ++rep) {
      if (rep == 0) dgx_profile_reset(h);
      if (cudaMemcpyAsync(U.p, U64, state64, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return DGX_ECUDA;
      s = dgx_ark_step_stages(h, U.p, dt, al(stages.p), al(ws_ark.p), stream);
      if (s != DGX_OK) {
        h->pipeline = was_pipe;
        dgx_profile_enable(h, was_prof);
        return s;
      }
    }
    int64_t n = 0;
    double ms = 0;
    dgx_profile_read(h, DGX_K_ELEM_STAGE, &n, &ms);
    if (n > 0) elem_ms[pipe] = ms / n;
  }
  h->pipeline = elem_ms[1] < elem_ms[0];
  dgx_profile_reset(h);
  dgx_profile_enable(h, was_prof);
  return cudaStreamSynchronize(st) == cudaSuccess ? DGX_OK : DGX_ECUDA;
}

// On any failure the handle keeps the tile variants, pipeline choice and
// profiler state it had before the call.
dgx_status dgx_autotune(dgx_handle* h, const double* U64, int32_t reps, void* stream) {
  if (!h || !U64 || reps < 1) return DGX_EINVAL;
  if (!h->has_mesh || h->stages == 0) return DGX_ESTATE;
  if (h->dgip) return DGX_OK;  // the DG-IP kernels have one tile shape: nothing to choose
  int saved[DGX_KERNEL_KINDS];
  std::copy(h->var, h->var + DGX_KERNEL_KINDS, saved);
  const bool saved_pipe = h->pipeline, saved_prof = h->prof;
  const dgx_status s = autotune_impl(h, U64, reps, stream);
  if (s != DGX_OK) {
    std::copy(saved, saved + DGX_KERNEL_KINDS, h->var);
    h->pipeline = saved_pipe;
    dgx_profile_enable(h, saved_prof);
  }
  return s;
}

dgx_status dgx_set_pipeline(dgx_handle* h, int32_t enable) {
  if (!h) return DGX_EINVAL;
  h->pipeline = enable != 0;
  return DGX_OK;
}

dgx_status dgx_set_contraction(dgx_handle* h, int32_t mode) {
  if (!h) return DGX_EINVAL;
  if (mode != DGX_CONTRACT_CUDA_CORE && mode != DGX_CONTRACT_TF32 && mode != DGX_CONTRACT_BF16 &&
      mode != DGX_CONTRACT_3XTF32)
    return DGX_EINVAL;
  if (mode != DGX_CONTRACT_CUDA_CORE && (h->fp64 || !h->tab->elem_tc)) return DGX_EUNSUPPORTED;
  h->contraction = mode;
  return DGX_OK;
}

dgx_status dgx_get_contraction(const dgx_handle* h, int32_t* mode) {
  if (!h || !mode) return DGX_EINVAL;
  *mode = h->contraction;
  return DGX_OK;
}

dgx_status dgx_get_variants(const dgx_handle* h, int32_t* variants) {
  if (!h || !variants) return DGX_EINVAL;
  for (int k = 0; k < DGX_KERNEL_KINDS; ++k) variants[k] = h->var[k];
  return DGX_OK;
}

dgx_status dgx_set_variants(dgx_handle* h, const int32_t* variants) {
  if (!h || !variants) return DGX_EINVAL;
  for (int k = 0; k < DGX_KERNEL_KINDS; ++k) {
    if (variants[k] < 0 || variants[k] >= dgx::NVARIANTS) return DGX_EINVAL;
    if (is_tile_kind(k) && h->has_mesh && tile_smem(h, k, variants[k]) > dgx::SMEM_LIMIT) return DGX_EINVAL;
  }
  for (int k = 0; k < DGX_KERNEL_KINDS; ++k) h->var[k] = variants[k];
  return DGX_OK;
}

}  // extern "C"

// ============================================================== batched runtime
struct dgx_batch {
  struct Group {
    dgx_handle* h = nullptr;
    int64_t off = 0;                 // offset (doubles) of the group in the packed state
    std::vector<int> members;        // instance indices
    std::vector<int64_t> elem_off;   // element offset of each member inside the group
    void* d_dte = nullptr;           // per-element time step in the group's precision
    size_t ws_off = 0;               // the group's slice of the batch workspace
    cudaStream_t st = nullptr;       // groups run concurrently, each on its own stream
    cudaEvent_t done = nullptr;      // the group's work is complete (joins the caller's stream)
  };
  int count = 0;
  std::vector<int64_t> offset;       // per instance (doubles), offset[count] = total
  std::vector<Group> groups;
  std::vector<double> dt;
  bool dt_set = false;
  size_t ws_bytes = 0;
  cudaStream_t cap = nullptr;
  cudaEvent_t start = nullptr;       // fork point on the caller's stream
  cudaGraphExec_t exec = nullptr;
  double* g_U = nullptr;
  void* g_ws = nullptr;
  // persistent form: one launch per phase over every group's work items
  bool pers_ok = false;                // 2D boxes, CUDA-core contraction, one precision
  bool persistent = false;
  int nsm = 148;
  dgx::BItem* d_items = nullptr;       // the phases' item lists, concatenated
  int n_items[4] = {}, item_off[4] = {};
  void* d_groups = nullptr;            // BGroup<S>[groups] for the prepared (U64, workspace)
  double* p_U = nullptr;
  void* p_ws = nullptr;
};

namespace {
bool same_group(const dgx_handle* a, const dgx_handle* b) {
  return a->d == b->d && a->p == b->p && a->fp64 == b->fp64 && a->viscous == b->viscous && a->curv == b->curv &&
         a->contraction == b->contraction &&
         a->desc.gamma == b->desc.gamma && (!a->viscous || (a->desc.Re == b->desc.Re && a->desc.Pr == b->desc.Pr));
}

void batch_free(dgx_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_groups) cudaFree(b->d_groups);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->start) cudaEventDestroy(b->start);
  for (auto& g : b->groups) {
    if (g.d_dte) cudaFree(g.d_dte);
    if (g.done) cudaEventDestroy(g.done);
    if (g.st) cudaStreamDestroy(g.st);
    if (g.h) dgx_destroy(g.h);
  }
  delete b;
}

// Persistent form: the per-group inputs of one ARK step (what ark_impl passes
// each group's kernels, with the per-element time step) uploaded once per
// (state, workspace) pair.
template <typename S>
dgx_status batch_prepare_t(dgx_batch* b, double* U64, void* ws) {
  std::vector<dgx::BGroup<S>> G(b->groups.size());
  for (size_t k = 0; k < b->groups.size(); ++k) {
    const auto& g = b->groups[k];
    dgx_handle* h = g.h;
    dgx::BGroup<S>& B = G[k];
    B.M = *(const dgx::Mesh<S>*)(h->fp64 ? (const void*)&h->mesh64 : (const void*)&h->mesh32);
    B.P = h->p;
    B.visc = h->viscous ? 1 : 0;
    char* base = (char*)ws + g.ws_off;
    const Layout L = layout(h, DGX_OP_ARK);
    B.w = work_at(h, base, L);
    double* Ug = U64 + g.off;
    B.U64 = Ug;
    const size_t state = align256((size_t)h->E * h->nf * h->N * h->s);
    S* Y = (S*)(base + L.Y);
    S* shadow = h->fp64 ? nullptr : (S*)(base + L.SH);
    B.first = shadow;
    const S* y0 = h->fp64 ? (const S*)Ug : shadow;
    const int s = h->stages;
    for (int i = 0; i < s; ++i) {
      dgx::Stage<S> sa{};
      for (int j = 0; j < i; ++j) sa.k[j] = (const S*)(base + L.K + state * j);
      sa.i = i;
      sa.last = (i == s - 1);
      if (!sa.last)
        for (int j = 0; j <= i; ++j) sa.ca[j] = (S)h->A[(i + 1) * dgx::MAXSTAGES + j];
      for (int j = 0; j < s; ++j) sa.cb[j] = (S)h->b[j];
      sa.dte = (const S*)g.d_dte;
      sa.base = y0;
      sa.Un = Ug;
      sa.Y = Y;
      sa.Kout = sa.last ? nullptr : (S*)(base + L.K + state * i);
      sa.shadow = shadow;
      sa.TU = (S*)B.w.TU;
      B.st[i] = sa;
      B.Uin[i] = (i == 0) ? y0 : Y;
    }
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return DGX_ECUDA;  // no launch still reads the old table
  if (!b->d_groups && cudaMalloc(&b->d_groups, G.size() * sizeof(dgx::BGroup<S>)) != cudaSuccess) return DGX_ENOMEM;
  if (cudaMemcpy(b->d_groups, G.data(), G.size() * sizeof(dgx::BGroup<S>), cudaMemcpyHostToDevice) != cudaSuccess)
    return DGX_ECUDA;
  b->p_U = U64;
  b->p_ws = ws;
  return DGX_OK;
}

dgx_status batch_prepare(dgx_batch* b, double* U64, void* ws) {
  if (b->p_U == U64 && b->p_ws == ws && b->d_groups) return DGX_OK;
  return b->groups[0].h->fp64 ? batch_prepare_t<double>(b, U64, ws) : batch_prepare_t<float>(b, U64, ws);
}

template <typename S>
dgx_status batch_run_persistent_t(dgx_batch* b, cudaStream_t st) {
  const auto* G = (const dgx::BGroup<S>*)b->d_groups;
  auto phase = [&](int ph, int stage) {
    return dgx::batch_phase<S>(ph, stage, G, b->d_items + b->item_off[ph], b->n_items[ph], b->nsm, st);
  };
  cudaError_t e = phase(0, 0);
  const int s = b->groups[0].h->stages;
  for (int i = 0; i < s && e == cudaSuccess; ++i) {
    if (b->n_items[1] > 0) e = phase(1, i);
    if (e == cudaSuccess) e = phase(2, i);
    if (e == cudaSuccess) e = phase(3, i);
  }
  return cuda_status(e);
}

// Every group's step on its own stream (disjoint state ranges and workspace
// slices), forked from and joined back to st by events, so small groups'
// kernels overlap instead of running one group after another.
dgx_status batch_run(dgx_batch* b, double* U64, void* ws, cudaStream_t st) {
  if (b->persistent) {  // tables prepared for (U64, ws) by the caller, outside any capture
    if (b->p_U != U64 || b->p_ws != ws) return DGX_ESTATE;
    return b->groups[0].h->fp64 ? batch_run_persistent_t<double>(b, st) : batch_run_persistent_t<float>(b, st);
  }
  if (cudaEventRecord(b->start, st) != cudaSuccess) return DGX_ECUDA;
  dgx_status s = DGX_OK;
  for (auto& g : b->groups) {
    dgx_handle* h = g.h;
    void* wg = (char*)ws + g.ws_off;
    if (cudaStreamWaitEvent(g.st, b->start, 0) != cudaSuccess) s = DGX_ECUDA;
    if (s == DGX_OK)
      s = h->fp64 ? ark_impl<double>(h, U64 + g.off, 0.0, nullptr, wg, g.st, (const double*)g.d_dte)
                  : ark_impl<float>(h, U64 + g.off, 0.0, nullptr, wg, g.st, (const float*)g.d_dte);
    // every stream that was forked joins back, also after an error
    if (cudaEventRecord(g.done, g.st) != cudaSuccess && s == DGX_OK) s = DGX_ECUDA;
    if (cudaStreamWaitEvent(st, g.done, 0) != cudaSuccess && s == DGX_OK) s = DGX_ECUDA;
    if (s != DGX_OK) break;
  }
  return s;
}
}  // namespace

extern "C" {

dgx_status dgx_batch_create(dgx_handle* const* inst, int32_t count, dgx_batch** out) {
  if (!out) return DGX_EINVAL;
  *out = nullptr;
  if (!inst || count < 1) return DGX_EINVAL;
  const dgx_handle* h0 = inst[0];
  for (int i = 0; i < count; ++i) {
    const dgx_handle* h = inst[i];
    if (!h) return DGX_EINVAL;
    if (h->dgip) return DGX_EUNSUPPORTED;  // batches run the LLF/BR1 scheme
    if (h->geo_override) return DGX_EUNSUPPORTED;  // the batch rebuilds geometry from the mesh description
    if (!h->has_mesh || h->stages == 0) return DGX_ESTATE;
    if (h->stages != h0->stages) return DGX_EINVAL;
    for (int r = 0; r < dgx::MAXSTAGES * dgx::MAXSTAGES; ++r)
      if (h->A[r] != h0->A[r]) return DGX_EINVAL;
    for (int j = 0; j < h->stages; ++j)
      if (h->b[j] != h0->b[j] || h->c[j] != h0->c[j]) return DGX_EINVAL;
  }
  dgx_batch* b = new (std::nothrow) dgx_batch();
  if (!b) return DGX_ENOMEM;
  b->count = count;
  b->dt.assign(count, 0.0);
  std::vector<int> group_of(count, -1);
  std::vector<const dgx_handle*> rep;
  for (int i = 0; i < count; ++i) {
    int g = -1;
    for (size_t k = 0; k < rep.size(); ++k)
      if (same_group(rep[k], inst[i])) g = (int)k;
    if (g < 0) {
      g = (int)rep.size();
      rep.push_back(inst[i]);
      b->groups.emplace_back();
    }
    group_of[i] = g;
    b->groups[g].members.push_back(i);
  }
  b->offset.assign(count + 1, 0);
  int64_t off = 0;
  dgx_status st = DGX_OK;
  for (auto& g : b->groups) {
    const dgx_handle* r = inst[g.members[0]];
    const int d = r->d, NF = r->NF, N = r->N, nf = r->nf;
    int64_t E = 0;
    for (int i : g.members) {
      g.elem_off.push_back(E);
      E += inst[i]->E;
    }
    dgx_problem_desc desc = r->desc;
    desc.n_elem = (int32_t)E;
    if ((st = dgx_create(&desc, &g.h)) != DGX_OK) break;
    std::vector<int32_t> nb;
    std::vector<int8_t> nbf, ori;
    std::vector<double> lo, size, xyz;
    for (size_t m = 0; m < g.members.size(); ++m) {
      const dgx_handle* h = inst[g.members[m]];
      for (int x : h->h_nb) nb.push_back(x >= 0 ? (int32_t)(x + g.elem_off[m]) : x);
      nbf.insert(nbf.end(), h->h_nbf.begin(), h->h_nbf.end());
      ori.insert(ori.end(), h->h_ori.begin(), h->h_ori.end());
      lo.insert(lo.end(), h->h_lo.begin(), h->h_lo.end());
      size.insert(size.end(), h->h_size.begin(), h->h_size.end());
      xyz.insert(xyz.end(), h->h_xyz.begin(), h->h_xyz.end());
    }
    (void)NF;
    (void)d;
    st = r->curv ? dgx_set_mesh_nodes(g.h, xyz.data(), nb.data(), nbf.data(), ori.data())
                 : dgx_set_mesh_boxes(g.h, lo.data(), size.data(), nb.data(), nbf.data(), ori.data());
    if (st != DGX_OK) break;
    std::vector<double> A(r->stages * r->stages);
    for (int i = 0; i < r->stages; ++i)
      for (int j = 0; j < r->stages; ++j) A[i * r->stages + j] = r->A[i * dgx::MAXSTAGES + j];
    if ((st = dgx_set_tableau(g.h, r->stages, A.data(), r->b, r->c)) != DGX_OK) break;
    for (int k = 0; k < DGX_KERNEL_KINDS; ++k) g.h->var[k] = r->var[k];
    g.h->contraction = r->contraction;
    if (cudaMalloc((void**)&g.d_dte, (size_t)E * g.h->s) != cudaSuccess) {
      st = DGX_ENOMEM;
      break;
    }
    if (cudaMemset(g.d_dte, 0, (size_t)E * g.h->s) != cudaSuccess) {
      st = DGX_ECUDA;
      break;
    }
    if (cudaStreamCreateWithFlags(&g.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming) != cudaSuccess) {
      st = DGX_ECUDA;
      break;
    }
    g.off = off;
    for (size_t m = 0; m < g.members.size(); ++m) b->offset[g.members[m]] = off + g.elem_off[m] * nf * N;
    off += E * nf * N;
    g.ws_off = b->ws_bytes;  // group workspaces side by side (each a multiple of 256 bytes)
    b->ws_bytes += dgx_workspace_bytes(g.h, DGX_OP_ARK);
  }
  b->offset[count] = off;
  if (st == DGX_OK) {  // the persistent form's work items (largest degree first)
    b->pers_ok = true;
    for (const auto& g : b->groups)
      b->pers_ok = b->pers_ok && g.h->d == 2 && !g.h->curv && g.h->contraction == DGX_CONTRACT_CUDA_CORE &&
                   g.h->fp64 == b->groups[0].h->fp64;
    b->nsm = b->groups[0].h->nsm;
    if (b->pers_ok) {
      std::vector<dgx::BItem> all;
      std::vector<int> order(b->groups.size());
      for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
      std::stable_sort(order.begin(), order.end(),
                       [&](int x, int y) { return b->groups[x].h->p > b->groups[y].h->p; });
      for (int ph = 0; ph < 4; ++ph) {
        b->item_off[ph] = (int)all.size();
        for (int k : order) {
          const dgx_handle* h = b->groups[k].h;
          if (ph == 1 && !h->viscous) continue;
          const int units = ph == 2 ? (h->nFaces * h->nfp + 255) / 256
                                    : (h->E + dgx::batch_tile_elems(h->p) - 1) / dgx::batch_tile_elems(h->p);
          for (int u = 0; u < units; ++u) all.push_back(dgx::BItem{k, u});
        }
        b->n_items[ph] = (int)all.size() - b->item_off[ph];
      }
      if (upload(all, (void**)&b->d_items) != DGX_OK) b->pers_ok = false;
    }
  }
  if (st == DGX_OK && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) st = DGX_ECUDA;
  if (st == DGX_OK && cudaEventCreateWithFlags(&b->start, cudaEventDisableTiming) != cudaSuccess) st = DGX_ECUDA;
  if (st != DGX_OK) {
    batch_free(b);
    return st;
  }
  *out = b;
  return DGX_OK;
}

dgx_status dgx_batch_destroy(dgx_batch* b) {
  if (!b) return DGX_EINVAL;
  batch_free(b);
  return DGX_OK;
}

dgx_status dgx_batch_layout(const dgx_batch* b, int64_t* offsets, int32_t* groups) {
  if (!b) return DGX_EINVAL;
  if (offsets)
    for (int i = 0; i <= b->count; ++i) offsets[i] = b->offset[i];
  if (groups) *groups = (int32_t)b->groups.size();
  return DGX_OK;
}

size_t dgx_batch_workspace_bytes(const dgx_batch* b) { return b ? b->ws_bytes : 0; }

dgx_status dgx_batch_set_dt(dgx_batch* b, const double* dt) {
  if (!b || !dt) return DGX_EINVAL;
  for (int i = 0; i < b->count; ++i)
    if (!std::isfinite(dt[i])) return DGX_EINVAL;
  for (auto& g : b->groups) {
    std::vector<double> dte((size_t)g.h->E);
    for (size_t m = 0; m < g.members.size(); ++m) {
      const int64_t e0 = g.elem_off[m];
      const int64_t e1 = (m + 1 < g.members.size()) ? g.elem_off[m + 1] : g.h->E;
      for (int64_t e = e0; e < e1; ++e) dte[e] = dt[g.members[m]];
    }
    cudaError_t err;
    if (g.h->fp64) {
      err = cudaMemcpy(g.d_dte, dte.data(), dte.size() * sizeof(double), cudaMemcpyHostToDevice);
    } else {
      const std::vector<float> dtf(dte.begin(), dte.end());
      err = cudaMemcpy(g.d_dte, dtf.data(), dtf.size() * sizeof(float), cudaMemcpyHostToDevice);
    }
    if (err != cudaSuccess) return DGX_ECUDA;
  }
  for (int i = 0; i < b->count; ++i) b->dt[i] = dt[i];
  b->dt_set = true;
  return DGX_OK;
}

dgx_status dgx_batch_step(dgx_batch* b, double* U64, void* workspace, void* stream) {
  if (!b || !U64 || !workspace || ((uintptr_t)workspace & 255) != 0) return DGX_EINVAL;
  if (!b->dt_set) return DGX_ESTATE;
  if (b->persistent) {
    const dgx_status s = batch_prepare(b, U64, workspace);
    if (s != DGX_OK) return s;
  }
  return batch_run(b, U64, workspace, (cudaStream_t)stream);
}

dgx_status dgx_batch_set_persistent(dgx_batch* b, int32_t enable) {
  if (!b) return DGX_EINVAL;
  if (enable && !b->pers_ok) return DGX_EUNSUPPORTED;
  if (b->persistent != (enable != 0) && b->exec) {  // the captured graph is of the other form
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  b->persistent = enable != 0;
  return DGX_OK;
}

dgx_status dgx_batch_step_graph(dgx_batch* b, double* U64, void* workspace, void* stream) {
  if (!b || !U64 || !workspace || ((uintptr_t)workspace & 255) != 0) return DGX_EINVAL;
  if (!b->dt_set) return DGX_ESTATE;
  if (!b->exec || b->g_U != U64 || b->g_ws != workspace) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    if (b->persistent) {  // the tables must exist before the capture starts
      const dgx_status s = batch_prepare(b, U64, workspace);
      if (s != DGX_OK) return s;
    }
    if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) return DGX_ECUDA;
    const dgx_status s = batch_run(b, U64, workspace, b->cap);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
    if (s != DGX_OK || e != cudaSuccess || !graph) {
      if (graph) cudaGraphDestroy(graph);
      return s != DGX_OK ? s : DGX_ECUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      b->exec = nullptr;
      return DGX_ECUDA;
    }
    b->g_U = U64;
    b->g_ws = workspace;
  }
  return cudaGraphLaunch(b->exec, (cudaStream_t)stream) == cudaSuccess ? DGX_OK : DGX_ECUDA;
}

dgx_status dgx_batch_autotune(dgx_batch* b, const double* U64, int32_t reps, void* stream) {
  if (!b || !U64) return DGX_EINVAL;
  for (auto& g : b->groups) {
    const dgx_status s = dgx_autotune(g.h, U64 + g.off, reps, stream);
    if (s != DGX_OK) return s;
  }
  if (b->exec) {  // variants changed: capture again on the next graph step
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return DGX_OK;
}

}  // extern "C"
