/*
 * dgx -- explicit discontinuous-Galerkin right-hand side for the compressible
 * Euler / Navier-Stokes equations on one NVIDIA B300 (sm_103a).
 *
 * The library evaluates the explicit-region operator of a geometry-split IMEX
 * scheme (the paper's Sec. 3.3 DG weak form with the mass matrix of the
 * semi-discrete system in Sec. 4.2) and advances it with the explicit ARK
 * stage and solution updates of Sec. 4.2 / Algorithm 1.  Readings used where
 * the paper differs or is silent:
 *   - convective numerical flux: local Lax-Friedrichs (Rusanov), wave speed
 *     max over both sides of |u.n| + c (the paper uses the Vijayasundaram flux);
 *   - viscous terms: BR1 (Bassi-Rebay 1) lifted gradient of the conservative
 *     variables and the central viscous flux 1/2 (G^- - G^+), each side's
 *     F^nu(U, Q) dotted with its own outward area normal (the paper uses SIPG);
 *   - collocated nodal basis on (p+1)^d Gauss-Legendre points, diagonal mass;
 *   - adiabatic no-slip walls: LLF against the mirror state, BR1 face value
 *     U_w = (rho, 0, .., rho e_i) (App. B no-slip state) and the wall viscous
 *     flux F^nu(U_w, Q^-).n with zero normal heat flux;
 *   - sign: f(U) = dU/dt = -M^{-1} B(U), B the weak form of Sec. 3.3, so the
 *     ERK update reads y_i = U_n + dt sum_j a_ij f(y_j).
 *
 * Data layout (all device buffers are caller-owned):
 *   state U[E][nf][N], nf = d + 2 fields (rho, rho u, rho v, [rho w], rho E),
 *   N = (p+1)^d nodes, node q = q0 + n q1 (+ n^2 q2), x index fastest;
 *   FP64 handles take double buffers, FP32 handles float buffers (the ARK master
 *   state is always double).
 * Mesh tables (host arrays, copied): neighbor[E][2d] = element across local face
 *   f (faces 2a: xi_a = -1, 2a+1: xi_a = +1) or -(1+tag) on a boundary
 *   (tag 0 = adiabatic no-slip wall, tag 1 = farfield (DG-IP scheme only));
 *   nbr_face[E][2d] = the neighbour's local
 *   face; orient[E][2d] maps the own face point (s, t) -- the two remaining
 *   local indices in increasing axis order, index s + n t -- to the
 *   neighbour's (u, v): bit 2 swaps s and t first, bit 0 reverses u, bit 1
 *   reverses v (2D: only bit 0).
 *
 * Errors: every entry point returns a dgx_status; host-side validation fails
 * synchronously with DGX_EINVAL and leaves the handle unchanged.  Device-side
 * conditions (a non-finite residual) raise a flag that dgx_check() reports.
 * No entry point exits, throws or prints.  All compute calls are asynchronous
 * on the given stream (a cudaStream_t passed as void*; NULL = legacy default
 * stream) and allocate nothing: scratch memory is the caller's workspace.
 */
#ifndef DGX_H
#define DGX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DGX_OK = 0,
  DGX_EINVAL = 1,       /* bad argument, inconsistent mesh table, size mismatch     */
  DGX_ENOMEM = 2,       /* host or device allocation failed (set-up calls only)     */
  DGX_ECUDA = 3,        /* a CUDA runtime call failed                               */
  DGX_ENONFINITE = 4,   /* a kernel produced NaN/Inf (reported by dgx_check)        */
  DGX_ETIMEOUT = 5,     /* a bounded device wait gave up (reported by dgx_check)    */
  DGX_EUNSUPPORTED = 6, /* valid request the library does not implement            */
  DGX_ESTATE = 7        /* call out of order (e.g. compute before a mesh is set)    */
} dgx_status;

typedef enum { DGX_FP64 = 0, DGX_FP32 = 1 } dgx_precision;

/* Workspace kinds for dgx_workspace_bytes. */
typedef enum {
  DGX_OP_RHS = 0,
  DGX_OP_VJP = 1,
  DGX_OP_ARK = 2,
  DGX_OP_ARK_ADJOINT = 3,
  DGX_OP_ARK_STEP_ADJOINT = 4, /* dgx_ark_step_adjoint */
  DGX_OP_HDG = 5               /* dgx_hdg_condense */
} dgx_op;

/* Spatial scheme: convective numerical flux and viscous discretisation.
 *   DGX_FLUX_LLF + DGX_VISC_BR1: local Lax-Friedrichs and BR1 (the default);
 *   DGX_FLUX_VIJAYASUNDARAM + DGX_VISC_SIPG: the paper's DG-IP operator (Sec. 3.3,
 *     Eq. bilinear_form_interior_sdg): the Vijayasundaram flux
 *     A_n^+({U}) U^+ + A_n^-({U}) U^- of the Sec. 3.2 eigen-split and the symmetric
 *     interior penalty (viscous surface term, adjoint-consistency term and penalty
 *     tau = alpha (k+1)^2 / l, l = |T| / |dT|, the face taking the larger 1/l of its
 *     two elements) with the element's own (broken) gradient; adiabatic walls by
 *     App. B.1.2 (K_w: no normal heat flux; the convective flux against the mirror
 *     state), farfield boundaries (tag 1) by App. B.1.1.  Box meshes and curved
 *     meshes (dgx_set_mesh_nodes / dgx_set_geometry: metric terms traced to the
 *     faces, area normals, 1/l from Gauss rules of J and of the face areas),
 *     for every residual, adjoint and ARK entry point (over-integration:
 *     box meshes and dgx_set_mesh_nodes meshes). */
typedef enum { DGX_FLUX_LLF = 0, DGX_FLUX_VIJAYASUNDARAM = 1 } dgx_conv_flux;
typedef enum { DGX_VISC_BR1 = 0, DGX_VISC_SIPG = 1 } dgx_visc_flux;

/* Problem statement (Sec. 2): dimension, polynomial degree k = p, element
 * count, viscous (Navier-Stokes, 1) or inviscid (Euler, 0), arithmetic
 * precision and the nondimensional parameters.  With rho_ref = |u_ref| =
 * L_ref = 1 and theta_inf = 1: R = 1/(gamma Ma^2), mu = 1/Re (constant),
 * kappa = c_p mu / Pr, lambda = -2 mu / 3 (Stokes).  Re, Pr are ignored when
 * viscous = 0; Ma only fixes R, which the operator does not depend on.
 * conv_flux / visc_flux select the scheme (LLF + BR1 or Vijayasundaram +
 * SIPG; other pairs give DGX_EUNSUPPORTED; visc_flux is ignored when
 * viscous = 0); penalty_alpha is the SIPG alpha (0 means the paper's 1).
 *
 * quad_points (DG-IP scheme): 0 = collocated (the volume and face
 * integrals by the (p+1)-point Gauss rule of the nodes); M in [p+1, 8] = the
 * nonlinear terms integrated by the M-point Gauss rule per direction (Sec. 5:
 * a rule of order 3k, M = ceil((3p+1)/2), which is 2, 4, 5, 7, 8 for
 * p = 1 .. 5).  The handle then
 * evaluates f = Pi f'(I U): I interpolates U to the M points, f' is the
 * collocated DG-IP operator of degree M-1 there with the penalty of degree p,
 * tau = alpha (p+1)^2 / l, and Pi[q][m] = omega_m l_q(z_m) / w_q projects back
 * (exact: the degree-p test functions lie in the degree-(M-1) space).  On a
 * curved mesh (dgx_set_mesh_nodes) f' runs on the element maps evaluated at
 * the M points (J', metric terms and normals of the degree-p map there) and,
 * with the nodal mass w_q J_q, f = J^-1 Pi (J' f'(I U)).  States stay on the
 * (p+1)^d nodes; every residual, VJP and ARK entry point applies the rule;
 * dgx_set_geometry, the HDG entry points and the batch runtime return
 * DGX_EUNSUPPORTED for such a handle; dgx_mms_source still samples the source
 * at the nodes.  quad_points is read only by dgx_create. */
typedef struct {
  int32_t dim;        /* 2 or 3                                  */
  int32_t p;          /* 1 .. 5                                  */
  int32_t n_elem;     /* E >= 1                                  */
  int32_t viscous;    /* 0 Euler, 1 Navier-Stokes                */
  int32_t precision;  /* dgx_precision                           */
  double gamma, Re, Pr, Ma;
  int32_t conv_flux;  /* dgx_conv_flux                           */
  int32_t visc_flux;  /* dgx_visc_flux                           */
  double penalty_alpha;
  int32_t quad_points;  /* 0 collocated, else M (over-integration)  */
} dgx_problem_desc;

typedef struct dgx_handle dgx_handle;

/* Create a handle (host + device set-up; allocates the handle's own small
 * tables).  *out is NULL on failure. */
dgx_status dgx_create(const dgx_problem_desc* desc, dgx_handle** out);
dgx_status dgx_destroy(dgx_handle* h);

/* Mesh of axis-aligned boxes (Sec. 3.1 mesh T_h): lower corner lo[E][d] and
 * edge lengths size[E][d] > 0 (host, double).  Geometry is exact:
 * J = prod(h_a/2), J dxi_a/dx_b = delta_ab prod_{c != a} h_c/2, so thin
 * wall layers never go through coordinate differences.  Connectivity as in
 * the header comment.  Replaces any previous mesh. */
dgx_status dgx_set_mesh_boxes(dgx_handle* h, const double* lo, const double* size,
                              const int32_t* neighbor, const int8_t* nbr_face, const int8_t* orient);

/* Curvilinear mesh: node coordinates xyz[E][d][N] at the Gauss nodes (host,
 * double); the element map is their degree-p tensor interpolant.  Metric terms
 * are computed in FP64 on the host: 2D J dxi/dx = [[y_eta, -x_eta], [-y_xi, x_xi]],
 * 3D the conservative curl form (discrete metric identities hold exactly).
 * Interior faces use the averaged area normal (Sn^- - Sn^+)/2 in the
 * convective flux, so the flux is exactly antisymmetric across a face. */
dgx_status dgx_set_mesh_nodes(dgx_handle* h, const double* xyz,
                              const int32_t* neighbor, const int8_t* nbr_face, const int8_t* orient);

/* The metric terms dgx_set_mesh_nodes derives, on the host alone (no handle,
 * no device): for n_elem elements of degree p (1 .. 7) in dim = 2 or 3 with
 * node coordinates xyz[E][d][N] (host, double), J[E][N] = det dx/dxi and
 * metric[E][N][d][d], metric[e][q][a][b] = J dxi_a/dx_b (caller-owned host
 * arrays), in the layout dgx_set_geometry takes.  DGX_EINVAL for bad
 * arguments, non-finite coordinates or an element with J <= 0 at a node. */
dgx_status dgx_mesh_metrics(int32_t dim, int32_t p, int32_t n_elem, const double* xyz, double* J, double* metric);

/* Geometry override (Sec. 3.1 element maps, given rather than derived): the
 * Jacobian J[E][N] > 0 and the metric terms metric[E][N][d][d],
 * metric[e][q][a][b] = J dxi_a/dx_b at the Gauss nodes (host, double,
 * copied), replacing the metrics of the current mesh, whose connectivity
 * stays.  Face normals follow from the metric as for dgx_set_mesh_nodes (each
 * side's J dxi_a/dx traced to its face, averaged across interior faces); the
 * handle then runs the curvilinear kernels.  The caller answers for the
 * metric identities (sum_a d/dxi_a (J dxi_a/dx_b) = 0 discretely, which free
 * stream preservation needs).  DGX_ESTATE without a mesh, DGX_EUNSUPPORTED on
 * over-integrated handles (their point operator needs the geometry at the M
 * points, which nodal values do not fix) and, afterwards, in dgx_batch_create
 * (the batch rebuilds geometry from the mesh description); the next
 * dgx_set_mesh_* call drops the override. */
dgx_status dgx_set_geometry(dgx_handle* h, const double* J, const double* metric);

/* Explicit Butcher tableau of an (s)-stage ERK (Sec. 4.2, padded ERK half of
 * the ARK pair): A[s][s] row-major, strictly lower triangular, b[s], c[s]
 * (host, double, copied).  s <= 8.  Default: none (dgx_ark_step -> DGX_ESTATE). */
dgx_status dgx_set_tableau(dgx_handle* h, int32_t stages, const double* A, const double* b, const double* c);

/* Bytes of caller-allocated device workspace for an operation (0 on error).
 * The workspace must be 256-byte aligned; its contents need not be
 * initialised and are not preserved between calls. */
size_t dgx_workspace_bytes(const dgx_handle* h, int32_t op);

/* f = dU/dt = -M^{-1} B(U) (Sec. 3.3 weak form, Sec. 4.2 semi-discrete system):
 * U, dUdt device [E][nf][N] in the handle's precision (distinct buffers).
 * Covers face traces, BR1 gradient, LLF + BR1 face fluxes, volume fluxes,
 * lifting and the inverse (diagonal) mass matrix. */
dgx_status dgx_rhs(dgx_handle* h, const void* U, void* dUdt, void* workspace, void* stream);

/* Vector-Jacobian product gU = (df/dU)^T lambda of the operator above
 * (hand-written adjoint: transposed contractions, transposed lifts and traces,
 * pointwise flux Jacobians^T).  At exact ties of the LLF wave speed the
 * interior side is differentiated; d|x|/dx at 0 is taken as 0. */
dgx_status dgx_rhs_vjp(dgx_handle* h, const void* U, const void* lambda, void* gU, void* workspace,
                       void* stream);

/* One explicit ARK step (Sec. 4.2 stage update y_i = U_n + dt sum_{j<i} a_ij f(y_j)
 * and solution update U_{n+1} = U_n + dt sum_i b_i f(y_i); Algorithm 1 without
 * the FSAL shortcut).  U64 (device, double [E][nf][N]) is updated in place;
 * the stage residual and update are fused, the stage accumulation is in FP64
 * (FP32 handles evaluate f in FP32 on a rounded copy of the stage state). */
dgx_status dgx_ark_step(dgx_handle* h, double* U64, double dt, void* workspace, void* stream);

/* Bytes of one step's stage-checkpoint buffer (0 before dgx_set_tableau).  The
 * buffer holds s equal slots of dgx_stage_bytes / s bytes; slot i (0-based)
 * begins with the stage state y_{i+1} [E][nf][N] in the handle's precision,
 * followed (LLF/BR1 scheme) by that stage's face traces and (viscous) BR1
 * gradient (FP64: also the gradient's face traces), which the adjoint reuses
 * instead of recomputing them; DG-IP slots hold the stage state (FP64 viscous:
 * also its face traces and face gradients, read by the adjoint). */
size_t dgx_stage_bytes(const dgx_handle* h);

/* The same step, also storing the stage states y_1..y_s it evaluates and their
 * traces / gradients (stage checkpointing for the adjoint) in stages, a device
 * buffer of dgx_stage_bytes(h) bytes, 256-byte aligned (y_1 = U_n, rounded to
 * FP32 on FP32 handles). */
dgx_status dgx_ark_step_stages(dgx_handle* h, double* U64, double dt, void* stages, void* workspace, void* stream);

/* Discrete adjoint of one explicit ARK step (reverse of the Sec. 4.2 stage
 * recurrence): with cotangent lam on U_{n+1},
 *   mu_i = dt (b_i lam + sum_{j>i} a_ji nu_j),  nu_i = (df/dU)(y_i)^T mu_i,
 *   lam_n = lam + sum_i nu_i,   i = s .. 1.
 * stages = the y_i of the step (from dgx_ark_step_stages); lam64 (device,
 * double [E][nf][N]) holds lambda_{n+1} on entry and lambda_n on exit; the
 * accumulation into lam64 is in FP64.  DG-IP scheme: composed from single
 * VJPs (mu_i formed in FP64 and rounded to the working precision). */
dgx_status dgx_ark_adjoint_step(dgx_handle* h, const void* stages, double* lam64, double dt, void* workspace,
                                void* stream);

/* One ARK step and its discrete adjoint in one call: the same results, bit for
 * bit, as dgx_ark_step_stages(h, U64, dt, stages, ...) followed by
 * dgx_ark_adjoint_step(h, stages, lam64, dt, ...) (U64: U_n in, U_{n+1} out;
 * lam64: lambda_{n+1} in, lambda_n out; stages as for those calls).  The
 * reverse stages need only the stage checkpoints, not U_{n+1}, so the last
 * stage's face and element kernels, which form U_{n+1}, run on a second
 * stream owned by the handle while the adjoint runs on `stream`; that stream
 * waits for them before the call's work ends (fork and join by events, so the
 * call can be captured into a CUDA graph).  DG-IP scheme: the step, then its
 * adjoint, both on `stream`.  Workspace:
 * dgx_workspace_bytes(h, DGX_OP_ARK_STEP_ADJOINT), 256-byte aligned. */
dgx_status dgx_ark_step_adjoint(dgx_handle* h, double* U64, double* lam64, double dt, void* stages, void* workspace,
                                void* stream);

/* Residual for callers that cannot allocate device memory (no counterpart in
 * the paper; a deployment convenience).  Same result as dgx_rhs, but the
 * scratch comes from a fixed array inside the library instead of a caller
 * workspace, so the call allocates nothing: for hosts that reserve all device
 * memory up front or plugin hosts that pass only inputs and outputs.
 * Limit: dgx_workspace_bytes(h, DGX_OP_RHS) must not exceed
 * DGX_NOALLOC_SCRATCH_BYTES (64 MiB), else DGX_EINVAL.  The handle's device
 * (the one current at dgx_create) must be current, else DGX_EINVAL.  Under
 * CUDA's default lazy module loading the 64 MiB array is created on a device
 * by the first call there and then held until the process exits; that first
 * call also looks up the array's device address (cached per device and
 * context; a call in a new context, e.g. after cudaDeviceReset, looks it up
 * again).  Make the first call on each device as a warm-up, before reserving
 * the rest of device memory and before any stream capture.  All calls on a
 * device share the array: calls that may overlap on the GPU race and must be
 * serialised. */
#define DGX_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
dgx_status dgx_rhs_noalloc(dgx_handle* h, const void* U, void* dUdt, void* stream);

/* Arithmetic-throughput probe (measurement only; no counterpart in the paper):
 * one launch of threads (a positive multiple of 256) threads, each running
 * eight independent chains of iters fused multiply-adds in the given precision
 * (DGX_FP64 or DGX_FP32) and storing one value to out (device, threads
 * elements of that precision).  *flops = 16 * iters * threads, the launch's
 * exact flop count; the caller times the launch (CUDA events on stream) to
 * obtain the device's measured FMA peak, the denominator of ALU-bound roofline
 * fractions.  DGX_EINVAL for bad sizes or precision. */
dgx_status dgx_probe_fma(int32_t precision, int64_t iters, void* out, int64_t threads, double* flops, void* stream);

/* Bound of the consumer waits of the persistent TMA-fed kernels (polls of
 * mbarrier.try_wait; default 2^22, the largest allowed; polls < 0 restores
 * it).  A wait that runs out makes the CTA raise the timeout flag (dgx_check
 * then returns DGX_ETIMEOUT), wait with the default bound for its own copies
 * still in flight and return; the residual of its remaining tiles is not
 * written.  Meant for exercising the timeout path: with polls = 0 every
 * persistent CTA gives up at its first wait. */
dgx_status dgx_set_wait_limit(dgx_handle* h, int64_t polls);

/* Element-local blocks of the implicit region's Newton system (Sec. 4.3) for
 * the HDG-IP discretisation of Sec. 3.4 (no mixed variables: the element
 * unknowns are U), FP64 handles on 2D meshes (else DGX_EUNSUPPORTED): box
 * meshes, and curved meshes of DG-IP handles (dgx_set_mesh_nodes or
 * dgx_set_geometry: the metric terms at the nodes and traced to the faces,
 * each element's own area normal; other curved handles DGX_EUNSUPPORTED):
 * for every element T, with its nodal state U (device [E][nf][N]) and the
 * facet state Uhat on its faces (device [E][2d][nf][n], the element's own
 * face-point order), the element form R_T (Eq.
 * bilinear_form_interior_hdg_ip_element with the HDG flux of Eq.
 * inviscid_numerical_flux, S_c = A_n^+(Uhat); K_w on adiabatic walls) and the
 * facet form h_T (Eq. bilinear_form_interior_hdg_ip_facet; the farfield and
 * no-slip transmission conditions of App. B.2 on boundary facets), both tested
 * with the nodal / facet basis, and the blocks of an SDIRK stage
 * M y + gamma R(y, yhat) = rhs (gamma = dt a_ii, M = diag(w_q J_q)):
 *   K = M + gamma dR/dU [E][nu][nu],  C = gamma dR/dUhat [E][nu][nh],
 *   D = dh/dU [E][nh][nu],            A33 = dh/dUhat [E][nh][nh]
 * (row-major; nu = nf N element DOFs in U's order, nh = 2d nf n facet DOFs in
 * Uhat's order; see dgx_hdg_sizes), by forward-mode differentiation of the
 * forms (one thread per element and column).  tau = 10 (k+1)^2 / l (the
 * paper's HDG-IP alpha).  R and h (device [E][nu], [E][nh]) receive the forms'
 * values when not NULL.  The global facet assembly and solve are the
 * caller's. */
dgx_status dgx_hdg_sizes(const dgx_handle* h, int32_t* nu, int32_t* nh);
dgx_status dgx_hdg_blocks(dgx_handle* h, const double* U, const double* Uhat, double gamma, double* K, double* C,
                          double* D, double* A33, double* R, double* hres, void* stream);
/* Static condensation of the element blocks (Eq. SchurCompliment,
 * local_solve_static_condensation): KinvC = K^{-1} C [E][nu][nh] (the local
 * recovery operator) and S = A33 - D K^{-1} C [E][nh][nh] (the element's
 * contribution to the Schur complement), by Gauss-Jordan elimination with
 * partial pivoting, one CTA per element.  Workspace: E nu nu doubles
 * (dgx_workspace_bytes(h, DGX_OP_HDG)), 256-byte aligned. */
dgx_status dgx_hdg_condense(dgx_handle* h, const double* K, const double* C, const double* D, const double* A33,
                            double* KinvC, double* S, void* workspace, void* stream);

/* Farfield state U_inf (App. B.1.1, Eq. farfield_state) of the DG-IP scheme:
 * conservative (rho, rho u, .., rho E), nf host doubles, copied.  Required
 * before a residual on a mesh with farfield faces (else DGX_ESTATE). */
dgx_status dgx_set_farfield(dgx_handle* h, const double* U_inf);

/* Geometry split of Sec. 4.1 (Eq. union_mesh) for the DG-IP scheme: mask[E]
 * (host, copied) is 1 for the elements of the explicit region T^ex and 0 for
 * the implicit region T^im; NULL removes the split.  With a split set,
 * dgx_rhs_split evaluates the explicit residual R^DG(U^ex, U^im) of Sec. 4.2.1
 * (Eq. semidiscrete_time_sdg; Algorithm 1 calls it with y_i^ex and y_{i-1}^im):
 * explicit elements read U_ex, implicit ones U_im (both device [E][nf][N] in
 * the handle's precision; only the elements of each region are read); faces
 * between the regions are the DG side of the interface (Sec. 4.1.1, Eq.
 * interface_bilinearform_explicit): treated like interior faces against the
 * implicit element's polynomial (state and gradient), with the averaged
 * diffusion matrix {K} in the adjoint-consistency term, and only the explicit
 * side receives the flux.  dUdt is f on explicit elements and 0 on implicit
 * ones.  Workspace: dgx_workspace_bytes(h, DGX_OP_RHS). */
dgx_status dgx_set_explicit_mask(dgx_handle* h, const int8_t* mask);
dgx_status dgx_rhs_split(dgx_handle* h, const void* U_ex, const void* U_im, void* dUdt, void* workspace,
                         void* stream);

/* Manufactured-solution source of Sec. 5.1.1 (the MMS of Gassner et al.,
 * U_e = (s+4, s+4, s+4, (s+4)^2), s = sin(pi (kx x + ky y) - omega pi t), 2D):
 * dUdt += S(x, t) = dU_e/dt + div(F^c - F^nu)(U_e) at every node, with the
 * handle's gamma, mu = 1/Re, Pr (mu = 0 for Euler).  Box meshes; dUdt device
 * [E][nf][N] in the handle's precision. */
dgx_status dgx_mms_source(dgx_handle* h, double t, double kx, double ky, double omega, void* dUdt, void* stream);

/* Synchronise with the device and report (then clear) device-side flags:
 * DGX_ENONFINITE if any residual value was NaN/Inf since the last check. */
dgx_status dgx_check(dgx_handle* h);

const char* dgx_status_string(dgx_status s);

/* Kernel kinds reported by the profiler. */
typedef enum {
  DGX_K_TRACE = 0,       /* face traces of a state                              */
  DGX_K_BR1 = 1,         /* BR1 lifted gradient + own-face viscous fluxes       */
  DGX_K_FACE = 2,        /* numerical flux at every unique face point           */
  DGX_K_ELEM = 3,        /* volume + lift + inverse mass                        */
  DGX_K_ELEM_STAGE = 4,  /* the same fused with the ARK stage update and traces */
  DGX_K_VJP_ELEM = 5,    /* adjoint of the element kernel                       */
  DGX_K_VJP_FACE = 6,    /* adjoint of the face fluxes                          */
  DGX_K_VJP_BR1 = 7,     /* adjoint of the BR1 gradient and viscous face fluxes */
  DGX_K_VJP_GATHER = 8,  /* adjoint of the traces (gather into the element)     */
  DGX_K_DGIP_TRACE = 9,  /* DG-IP: traces and own-face viscous normal fluxes     */
  DGX_K_DGIP_FACE = 10,  /* DG-IP: numerical flux and adjoint-term vectors       */
  DGX_K_DGIP_ELEM = 11,  /* DG-IP: volume + lift + adjoint term + inverse mass   */
  DGX_K_DGIP_VJP_ELEM = 12,   /* DG-IP adjoint: element part and face cotangents */
  DGX_K_DGIP_VJP_FACE = 13,   /* DG-IP adjoint: face function (dual numbers)     */
  DGX_K_DGIP_VJP_GATHER = 14, /* DG-IP adjoint: traces and face gradients        */
  DGX_K_OI_TO_QUAD = 15,      /* over-integration: nodes -> M points (I, Pi^T)   */
  DGX_K_OI_TO_NODES = 16,     /* over-integration: M points -> nodes (Pi, I^T)   */
  DGX_K_DGIP_VJP_TRACE = 17,  /* DG-IP adjoint: the traces of U alone            */
  DGX_KERNEL_KINDS = 18
} dgx_kernel_kind;

/* Per-kernel device timing (tracing).  While enabled, every kernel the
 * library enqueues is bracketed by two CUDA events on its stream (enabling
 * creates a pool of 8192 events; launches beyond 4096 between two reads are
 * not recorded).  Not meant for use inside a stream capture.
 * dgx_profile_read synchronises on the recorded events and returns, for one
 * kernel kind, the launch count and summed device milliseconds accumulated
 * since the last reset. */
dgx_status dgx_profile_enable(dgx_handle* h, int32_t enable);
dgx_status dgx_profile_read(dgx_handle* h, int32_t kind, int64_t* launches, double* ms);
dgx_status dgx_profile_reset(dgx_handle* h);
const char* dgx_kernel_name(int32_t kind);

/* Algorithmic work of one launch of a kernel kind on this handle's mesh (for
 * roofline reporting): flops counted from the implemented arithmetic (the
 * pointwise physics is counted operation by operation, a fused multiply-add
 * being two flops; contractions from their loop structure) and bytes of the
 * kernel's compulsory traffic (each input read once, each output written once).
 * With a tableau set, the element-stage and VJP-element figures are averages
 * over the (reverse) stages of an ARK step and its adjoint, the gather
 * figure includes the adjoint step's lambda update, and the trace figure is
 * that of the step's first kernel (FP64 state in, traces and the
 * working-precision state out). */
dgx_status dgx_kernel_work(const dgx_handle* h, int32_t kind, double* flops, double* bytes);

/* Tile-size autotuner.  Tile kernels come in 4 variants: 0..2 use one CTA of
 * about 128 / 256 / 512 threads per tile of max(1, threads / N) elements;
 * 3 (elements of at most 32 nodes) uses one warp per element with warp-level
 * synchronisation only.
 * dgx_autotune times every variant of every tile kernel (event profiler, reps
 * timed repetitions of one ARK step and, when built, its adjoint, on a scratch
 * copy of the device state U64) and keeps the fastest per kernel; variants
 * whose shared memory exceeds the 227 KB per-CTA limit are skipped; it also
 * keeps or drops the persistent TMA-fed element kernel (dgx_set_pipeline),
 * whichever runs the stage faster.  It is a
 * set-up call: it allocates and frees its scratch and synchronises the stream.
 * Requires a mesh and a tableau.  variants[] is indexed by dgx_kernel_kind. */
dgx_status dgx_autotune(dgx_handle* h, const double* U64, int32_t reps, void* stream);
dgx_status dgx_get_variants(const dgx_handle* h, int32_t* variants);
/* Persistent, TMA-fed kernels (default on): a grid of (SMs x resident CTAs)
 * CTAs walks the element tiles; each tile's contiguous input blocks arrive by
 * cp.async.bulk into a double buffer while the previous tile is computed.
 * Used where every block is a 16-byte multiple and 16-byte aligned (else the
 * one-CTA-per-tile kernels run).  Same arithmetic either way. */
dgx_status dgx_set_pipeline(dgx_handle* h, int32_t enable);
dgx_status dgx_set_variants(dgx_handle* h, const int32_t* variants);

/* Engine of the 1D differentiation contractions of the forward element kernel
 * (the volume term of the Sec. 3.3 weak form together with the surface lift), an
 * opt-in for FP32 handles:
 *   DGX_CONTRACT_CUDA_CORE  FP32 (or FP64) fused multiply-adds (default);
 *   DGX_CONTRACT_TF32       tcgen05 tensor cores, operands rounded to TF32
 *                           (10-bit mantissa), FP32 accumulation: relative
 *                           error of the residual about 1e-3;
 *   DGX_CONTRACT_BF16       tcgen05 kind::f16, operands rounded to BF16
 *                           (7-bit mantissa), FP32 accumulation: relative
 *                           error of the residual about 1e-2;
 *   DGX_CONTRACT_3XTF32     tcgen05, every operand split into two TF32 parts
 *                           and three products accumulated: close to FP32.
 * Each (direction, element, field, line) is one row of a GEMM against the
 * fixed [Dh | -L(-1) | -L(+1)] operand (n + 2 <= 8 columns, zero-padded to the
 * MMA's K of 8 (TF32) or 16 (BF16); M = 128 rows per MMA, accumulator in
 * tensor memory).  Applies to dgx_rhs and the ARK stage
 * kernels of this handle (and of batches created from it); the adjoint
 * kernels always contract on CUDA cores, so with a tensor-core contraction
 * the adjoint step differentiates the CUDA-core residual at the stage states
 * the tensor-core forward produced.  DGX_EUNSUPPORTED for FP64 handles,
 * DGX_EINVAL for another mode.  The element tile is the 256-thread shape
 * whatever the autotuned variant, and the persistent pipeline is bypassed. */
typedef enum {
  DGX_CONTRACT_CUDA_CORE = 0,
  DGX_CONTRACT_TF32 = 1,
  DGX_CONTRACT_BF16 = 2,
  DGX_CONTRACT_3XTF32 = 3
} dgx_contraction;
dgx_status dgx_set_contraction(dgx_handle* h, int32_t mode);
dgx_status dgx_get_contraction(const dgx_handle* h, int32_t* mode);

/* Batched ensemble: many independent instances (meshes, degrees, physics)
 * advanced together.  Instances are grouped by (dimension, degree, precision,
 * physics, mesh kind, contraction engine); each group's meshes are concatenated into one internal
 * handle, so every kernel launch covers all instances of a group and the
 * tile variant is autotuned per group (per degree).  All instances must share
 * the tableau.  The state of all instances is one packed FP64 buffer:
 * instance i occupies doubles [offsets[i], offsets[i] + E_i nf_i N_i)
 * (dgx_batch_layout, offsets has count + 1 entries).  Each instance has its own
 * time step (dgx_batch_set_dt, host array of count doubles, uploaded once).
 * The groups of a step run concurrently, each on a stream of the batch,
 * forked from and joined back to the caller's stream by events; the workspace
 * holds one slice per group.  The instance handles are only read by
 * dgx_batch_create. */
typedef struct dgx_batch dgx_batch;
dgx_status dgx_batch_create(dgx_handle* const* inst, int32_t count, dgx_batch** out);
dgx_status dgx_batch_destroy(dgx_batch* b);
dgx_status dgx_batch_layout(const dgx_batch* b, int64_t* offsets, int32_t* groups);
size_t dgx_batch_workspace_bytes(const dgx_batch* b);
dgx_status dgx_batch_set_dt(dgx_batch* b, const double* dt);
/* One explicit ARK step of every instance (enqueued kernel by kernel). */
dgx_status dgx_batch_step(dgx_batch* b, double* U64, void* workspace, void* stream);
/* The same step as one CUDA graph: captured (on a private stream) at the first
 * call and whenever U64 or workspace change, then launched on the given
 * stream; later dt changes need no recapture.  Make a dgx_batch_step or
 * dgx_batch_autotune call first so kernel attributes are set outside capture. */
dgx_status dgx_batch_step_graph(dgx_batch* b, double* U64, void* workspace, void* stream);
/* Form of the batched step.  0 (default): each group runs its own kernels on
 * its own stream (a graph of concurrent per-group launches).  1: persistent:
 * one launch per phase of each stage (first traces, BR1 gradient, face
 * fluxes, element + stage update) covers every group -- a grid of SMs x
 * resident CTAs walks a work list of (group, element tile) items ordered by
 * decreasing degree and runs, per item, the group's own tile arithmetic for
 * its degree (256-thread tiles), so a step is 1 + 3 s launches whatever the
 * number of groups, with identical results bit for bit.  The per-group
 * inputs are tabulated in device memory the first time a step sees a (U64,
 * workspace) pair (a synchronising set-up; make that call outside any stream
 * capture: dgx_batch_step_graph does it before capturing).  Requires 2D box
 * meshes, the CUDA-core contraction and one precision for all instances,
 * else DGX_EUNSUPPORTED. */
dgx_status dgx_batch_set_persistent(dgx_batch* b, int32_t enable);
/* Autotune every group on the packed state U64 (see dgx_autotune). */
dgx_status dgx_batch_autotune(dgx_batch* b, const double* U64, int32_t reps, void* stream);

/* Sizes the binding needs: element count, nodes per element, fields, face
 * points per face, the chosen element-tile size. */
dgx_status dgx_query(const dgx_handle* h, int32_t* n_elem, int32_t* nodes, int32_t* fields,
                     int32_t* face_points, int32_t* tile);

#ifdef __cplusplus
}
#endif
#endif
