"""Python binding of libdgx.so (the C ABI in include/dgx.h).

Argument marshalling only: torch supplies device memory and the current CUDA
stream, every step of the computation runs in the library's kernels.  There
is no CPU fallback -- importing works anywhere, but constructing a ``Solver``
raises if the shared library is missing or no CUDA device is present.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdgx.so")

FP64, FP32 = 0, 1
OP_RHS, OP_VJP, OP_ARK, OP_ARK_ADJOINT, OP_ARK_STEP_ADJOINT, OP_HDG = 0, 1, 2, 3, 4, 5
STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error", 4: "non-finite residual",
          5: "device wait timed out", 6: "unsupported", 7: "call out of order"}


class DGXError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"{where}: {STATUS.get(code, code)} (status {code})")
        self.code = code


class _Desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("p", ctypes.c_int32), ("n_elem", ctypes.c_int32),
                ("viscous", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("gamma", ctypes.c_double), ("Re", ctypes.c_double), ("Pr", ctypes.c_double),
                ("Ma", ctypes.c_double), ("conv_flux", ctypes.c_int32), ("visc_flux", ctypes.c_int32),
                ("penalty_alpha", ctypes.c_double), ("quad_points", ctypes.c_int32)]


_lib = None

EXPORTS = ["dgx_create", "dgx_destroy", "dgx_set_mesh_boxes", "dgx_set_mesh_nodes", "dgx_set_tableau",
           "dgx_workspace_bytes", "dgx_rhs", "dgx_rhs_vjp", "dgx_ark_step", "dgx_check",
           "dgx_status_string", "dgx_query", "dgx_profile_enable", "dgx_profile_read", "dgx_profile_reset",
           "dgx_kernel_name", "dgx_ark_step_stages", "dgx_ark_adjoint_step", "dgx_rhs_noalloc",
           "dgx_stage_bytes", "dgx_kernel_work", "dgx_autotune", "dgx_get_variants", "dgx_set_variants",
           "dgx_batch_create", "dgx_batch_destroy", "dgx_batch_layout", "dgx_batch_workspace_bytes",
           "dgx_batch_set_dt", "dgx_batch_step", "dgx_batch_step_graph", "dgx_batch_autotune", "dgx_set_pipeline",
           "dgx_set_contraction", "dgx_get_contraction", "dgx_ark_step_adjoint", "dgx_probe_fma",
           "dgx_set_farfield", "dgx_set_explicit_mask", "dgx_rhs_split", "dgx_mms_source",
           "dgx_set_wait_limit", "dgx_batch_set_persistent", "dgx_hdg_sizes", "dgx_hdg_blocks",
           "dgx_hdg_condense", "dgx_set_geometry", "dgx_mesh_metrics"]
SCHEMES = {"llf-br1": (0, 0), "dgip": (1, 1)}   # (conv_flux, visc_flux)
CONTRACTIONS = {"cuda_core": 0, "tf32": 1, "bf16": 2, "3xtf32": 3}
KERNELS = ["trace", "br1", "face", "elem", "elem_stage", "vjp_elem", "vjp_face", "vjp_br1", "vjp_gather",
           "dgip_trace", "dgip_face", "dgip_elem", "dgip_vjp_elem", "dgip_vjp_face", "dgip_vjp_gather",
           "oi_to_quad", "oi_to_nodes", "dgip_vjp_trace"]


def load_library(path: str = LIB_PATH):
    """Load libdgx.so and declare its signatures (no GPU needed)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    vp, i32, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    lib.dgx_create.argtypes = [ctypes.POINTER(_Desc), ctypes.POINTER(vp)]
    lib.dgx_destroy.argtypes = [vp]
    lib.dgx_set_mesh_boxes.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.dgx_set_mesh_nodes.argtypes = [vp, vp, vp, vp, vp]
    lib.dgx_set_geometry.argtypes = [vp, vp, vp]
    lib.dgx_mesh_metrics.argtypes = [i32, i32, i32, vp, vp, vp]
    lib.dgx_set_tableau.argtypes = [vp, i32, vp, vp, vp]
    lib.dgx_workspace_bytes.argtypes = [vp, i32]
    lib.dgx_workspace_bytes.restype = ctypes.c_size_t
    lib.dgx_rhs.argtypes = [vp, vp, vp, vp, vp]
    lib.dgx_rhs_vjp.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.dgx_ark_step.argtypes = [vp, vp, dbl, vp, vp]
    lib.dgx_ark_step_stages.argtypes = [vp, vp, dbl, vp, vp, vp]
    lib.dgx_ark_adjoint_step.argtypes = [vp, vp, vp, dbl, vp, vp]
    lib.dgx_ark_step_adjoint.argtypes = [vp, vp, vp, dbl, vp, vp, vp]
    lib.dgx_rhs_noalloc.argtypes = [vp, vp, vp, vp]
    lib.dgx_stage_bytes.argtypes = [vp]
    lib.dgx_kernel_work.argtypes = [vp, i32, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
    lib.dgx_autotune.argtypes = [vp, vp, i32, vp]
    lib.dgx_set_pipeline.argtypes = [vp, i32]
    lib.dgx_set_contraction.argtypes = [vp, i32]
    lib.dgx_get_contraction.argtypes = [vp, ctypes.POINTER(i32)]
    lib.dgx_get_variants.argtypes = [vp, ctypes.POINTER(i32)]
    lib.dgx_set_variants.argtypes = [vp, ctypes.POINTER(i32)]
    lib.dgx_batch_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(vp)]
    lib.dgx_batch_destroy.argtypes = [vp]
    lib.dgx_batch_layout.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(i32)]
    lib.dgx_batch_workspace_bytes.argtypes = [vp]
    lib.dgx_batch_set_dt.argtypes = [vp, vp]
    lib.dgx_batch_step.argtypes = [vp, vp, vp, vp]
    lib.dgx_batch_step_graph.argtypes = [vp, vp, vp, vp]
    lib.dgx_batch_autotune.argtypes = [vp, vp, i32, vp]
    lib.dgx_check.argtypes = [vp]
    lib.dgx_status_string.argtypes = [i32]
    lib.dgx_status_string.restype = ctypes.c_char_p
    lib.dgx_query.argtypes = [vp] + [ctypes.POINTER(i32)] * 5
    lib.dgx_profile_enable.argtypes = [vp, i32]
    lib.dgx_profile_read.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(dbl)]
    lib.dgx_profile_reset.argtypes = [vp]
    lib.dgx_kernel_name.argtypes = [i32]
    lib.dgx_kernel_name.restype = ctypes.c_char_p
    lib.dgx_probe_fma.argtypes = [i32, ctypes.c_int64, vp, ctypes.c_int64, ctypes.POINTER(dbl), vp]
    lib.dgx_set_farfield.argtypes = [vp, vp]
    lib.dgx_set_wait_limit.argtypes = [vp, ctypes.c_int64]
    lib.dgx_batch_set_persistent.argtypes = [vp, i32]
    lib.dgx_hdg_sizes.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.dgx_hdg_blocks.argtypes = [vp, vp, vp, dbl, vp, vp, vp, vp, vp, vp, vp]
    lib.dgx_hdg_condense.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.dgx_set_explicit_mask.argtypes = [vp, vp]
    lib.dgx_rhs_split.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.dgx_mms_source.argtypes = [vp, dbl, dbl, dbl, dbl, vp, vp]
    for name in EXPORTS:
        getattr(lib, name).restype = getattr(lib, name).restype or ctypes.c_int
    lib.dgx_workspace_bytes.restype = ctypes.c_size_t
    lib.dgx_status_string.restype = ctypes.c_char_p
    lib.dgx_kernel_name.restype = ctypes.c_char_p
    lib.dgx_stage_bytes.restype = ctypes.c_size_t
    lib.dgx_batch_workspace_bytes.restype = ctypes.c_size_t
    _lib = lib
    return lib


def mesh_metrics(mesh):
    """J[E][N] and metric[E][N][d][d] = J dxi_a/dx_b that the library derives
    from a node-coordinate mesh (dgx_mesh_metrics: host only, no GPU)."""
    lib = load_library()
    E, N, d = mesh.n_elem, mesh.N, mesh.dim
    xyz = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
    J = np.empty((E, N))
    metric = np.empty((E, N, d, d))
    _check(lib.dgx_mesh_metrics(d, mesh.p, E, _ptr(xyz), _ptr(J), _ptr(metric)), "dgx_mesh_metrics")
    return J, metric


def measure_fma_peak(precision: str, reps: int = 5, iters: Optional[int] = None) -> float:
    """Measured FMA throughput (TFLOP/s, best of ``reps``) of the current CUDA
    device in "fp64" or "fp32": dgx_probe_fma launches, each timed with CUDA
    events on the current stream (the denominator of ALU-bound roofline
    fractions)."""
    lib = load_library()
    prec = FP64 if precision == "fp64" else FP32
    iters = iters or (4096 if prec == FP64 else 65536)     # launches of ~10 ms
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    threads = nsm * 2048
    out = torch.empty(threads, dtype=torch.float64 if prec == FP64 else torch.float32, device="cuda")
    flops = ctypes.c_double()
    stream = torch.cuda.current_stream()
    best = 0.0
    for k in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _check(lib.dgx_probe_fma(prec, iters, ctypes.c_void_p(out.data_ptr()), threads, ctypes.byref(flops),
                                 ctypes.c_void_p(stream.cuda_stream)), "dgx_probe_fma")
        e1.record(stream)
        torch.cuda.synchronize()
        if k:   # the first launch is a warm-up
            best = max(best, flops.value / (e0.elapsed_time(e1) / 1e3) / 1e12)
    return best


def _check(code, where):
    if code != 0:
        raise DGXError(code, where)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Solver:
    """Explicit DG right-hand side on one mesh (see include/dgx.h).

    ``mesh`` is a :class:`paper_2607_16044_b300.inputs.Mesh`; ``phys`` an
    :class:`inputs.Physics`.  ``precision`` is "fp64" or "fp32".
    ``quad_points`` (DG-IP scheme, box or curved meshes): None for the collocated
    operator, "3k" for the over-integration rule of order 3k (M = (3p+2)//2
    Gauss points per direction), or an explicit M in [p+1, 8].
    """

    def __init__(self, mesh, phys, precision: str = "fp64", device: Optional[torch.device] = None,
                 scheme: str = "llf-br1", alpha: float = 1.0, U_inf=None, quad_points=None):
        if not torch.cuda.is_available():
            raise RuntimeError("dgx needs a CUDA device; there is no CPU fallback")
        self.lib = load_library()
        self.mesh = mesh
        self.phys = phys
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        conv, visc = SCHEMES[scheme]
        self.scheme = scheme
        if quad_points == "3k":
            quad_points = (3 * mesh.p + 2) // 2
        self.quad_points = int(quad_points or 0)
        desc = _Desc(mesh.dim, mesh.p, mesh.n_elem, int(phys.viscous), FP64 if precision == "fp64" else FP32,
                     phys.gamma, phys.Re if phys.viscous else 0.0, phys.Pr, phys.Ma, conv, visc, float(alpha),
                     self.quad_points)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(self.lib.dgx_create(ctypes.byref(desc), ctypes.byref(h)), "dgx_create")
        self.h = h
        self.shape = (mesh.n_elem, mesh.dim + 2, mesh.N)
        self.set_mesh(mesh)
        self._ws = {}
        self.stages = 0
        if U_inf is not None:
            self.set_farfield(U_inf)

    def set_mesh(self, mesh):
        """Upload a mesh (boxes or node coordinates) of the handle's dimension,
        degree and element count, replacing the current one."""
        if (mesh.dim, mesh.p, mesh.n_elem) != (self.mesh.dim, self.mesh.p, self.mesh.n_elem):
            raise ValueError("the mesh must keep the handle's dimension, degree and element count")
        nb = np.ascontiguousarray(mesh.neighbor, dtype=np.int32)
        nbf = np.ascontiguousarray(mesh.nbr_face, dtype=np.int8)
        ori = np.ascontiguousarray(mesh.orient, dtype=np.int8)
        if mesh.kind == "boxes":
            lo = np.ascontiguousarray(mesh.lo, dtype=np.float64)
            sz = np.ascontiguousarray(mesh.size, dtype=np.float64)
            _check(self.lib.dgx_set_mesh_boxes(self.h, _ptr(lo), _ptr(sz), _ptr(nb), _ptr(nbf), _ptr(ori)),
                   "dgx_set_mesh_boxes")
        else:
            xyz = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
            _check(self.lib.dgx_set_mesh_nodes(self.h, _ptr(xyz), _ptr(nb), _ptr(nbf), _ptr(ori)),
                   "dgx_set_mesh_nodes")
        self.mesh = mesh

    def set_farfield(self, U_inf):
        """Free-stream state (conservative) of the farfield boundaries (DG-IP scheme)."""
        u = np.ascontiguousarray(U_inf, dtype=np.float64)
        _check(self.lib.dgx_set_farfield(self.h, _ptr(u)), "dgx_set_farfield")

    def set_geometry(self, J, metric):
        """Replace the mesh's metrics by J[E][N] and metric[E][N][d][d] = J dxi_a/dx_b
        (host arrays; the connectivity stays)."""
        Jh = np.ascontiguousarray(J, dtype=np.float64)
        Mh = np.ascontiguousarray(metric, dtype=np.float64)
        E, N, d = self.mesh.n_elem, self.mesh.N, self.mesh.dim
        if Jh.shape != (E, N) or Mh.shape != (E, N, d, d):
            raise ValueError("J must be [E][N] and metric [E][N][d][d]")
        _check(self.lib.dgx_set_geometry(self.h, _ptr(Jh), _ptr(Mh)), "dgx_set_geometry")

    def set_explicit_mask(self, mask):
        """Explicit-region element mask of the geometry split (None removes it)."""
        if mask is None:
            _check(self.lib.dgx_set_explicit_mask(self.h, None), "dgx_set_explicit_mask")
            return
        m = np.ascontiguousarray(np.asarray(mask, dtype=bool), dtype=np.int8)
        _check(self.lib.dgx_set_explicit_mask(self.h, _ptr(m)), "dgx_set_explicit_mask")

    def close(self):
        if getattr(self, "h", None):
            self.lib.dgx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ helpers
    def workspace(self, op: int) -> torch.Tensor:
        nbytes = int(self.lib.dgx_workspace_bytes(self.h, op))
        if nbytes == 0:
            raise DGXError(7, "dgx_workspace_bytes")
        ws = self._ws.get(op)
        if ws is None or ws.numel() < nbytes:
            ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            self._ws[op] = ws
        return ws

    @staticmethod
    def _aligned(ws: torch.Tensor):
        p = ws.data_ptr()
        return ctypes.c_void_p((p + 255) & ~255)

    def _state(self, U, name="U", dtype=None):
        dtype = dtype or self.dtype
        if not (isinstance(U, torch.Tensor) and U.is_cuda and U.dtype == dtype and U.is_contiguous()
                and tuple(U.shape) == self.shape):
            raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor of shape {self.shape}")
        return ctypes.c_void_p(U.data_ptr())

    def empty_state(self, dtype=None):
        return torch.empty(self.shape, dtype=dtype or self.dtype, device=self.device)

    def set_tableau(self, A, b, c):
        """Explicit tableau (e.g. ``tableaux.ars343_explicit()``)."""
        A = np.ascontiguousarray(A, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        c = np.ascontiguousarray(c, dtype=np.float64)
        _check(self.lib.dgx_set_tableau(self.h, len(b), _ptr(A), _ptr(b), _ptr(c)), "dgx_set_tableau")
        self.stages = len(b)
        self._ws.pop(OP_ARK, None)
        self._ws.pop(OP_ARK_ADJOINT, None)
        self._ws.pop(OP_ARK_STEP_ADJOINT, None)

    # ------------------------------------------------------------------ compute
    def rhs(self, U: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        out = self.empty_state() if out is None else out
        ws = self.workspace(OP_RHS)
        _check(self.lib.dgx_rhs(self.h, self._state(U), self._state(out, "out"), self._aligned(ws),
                                _stream_ptr(stream)), "dgx_rhs")
        return out

    def rhs_split(self, U_ex: torch.Tensor, U_im: torch.Tensor, out: Optional[torch.Tensor] = None,
                  stream=None) -> torch.Tensor:
        """R^DG(U_ex, U_im) of the geometry split (explicit elements read U_ex,
        implicit ones U_im; f = 0 on implicit elements)."""
        out = self.empty_state() if out is None else out
        ws = self.workspace(OP_RHS)
        _check(self.lib.dgx_rhs_split(self.h, self._state(U_ex, "U_ex"), self._state(U_im, "U_im"),
                                      self._state(out, "out"), self._aligned(ws), _stream_ptr(stream)),
               "dgx_rhs_split")
        return out

    def mms_source(self, t: float, out: torch.Tensor, kx=2.0, ky=2.0, omega=200.0, stream=None) -> torch.Tensor:
        """out += the manufactured-solution source S(x, t) (2D, box meshes)."""
        _check(self.lib.dgx_mms_source(self.h, float(t), float(kx), float(ky), float(omega),
                                       self._state(out, "out"), _stream_ptr(stream)), "dgx_mms_source")
        return out

    def hdg_blocks(self, U: torch.Tensor, Uhat: torch.Tensor, gamma: float, forms: bool = False, stream=None):
        """Element-local HDG-IP Newton blocks (K, C, D, A33[, R, h]) of an SDIRK
        stage with gamma = dt a_ii (FP64, 2D; box meshes, or curved meshes of a DG-IP
        handle); Uhat is [E][2d][nf][n]."""
        nu, nh = ctypes.c_int32(), ctypes.c_int32()
        _check(self.lib.dgx_hdg_sizes(self.h, ctypes.byref(nu), ctypes.byref(nh)), "dgx_hdg_sizes")
        E = self.shape[0]
        dev = self.device
        K = torch.empty((E, nu.value, nu.value), dtype=torch.float64, device=dev)
        C = torch.empty((E, nu.value, nh.value), dtype=torch.float64, device=dev)
        D = torch.empty((E, nh.value, nu.value), dtype=torch.float64, device=dev)
        A = torch.empty((E, nh.value, nh.value), dtype=torch.float64, device=dev)
        R = torch.empty((E, nu.value), dtype=torch.float64, device=dev) if forms else None
        h = torch.empty((E, nh.value), dtype=torch.float64, device=dev) if forms else None
        if not (U.is_cuda and U.dtype == torch.float64 and U.is_contiguous() and Uhat.is_cuda
                and Uhat.dtype == torch.float64 and Uhat.is_contiguous() and Uhat.numel() == E * nh.value):
            raise ValueError("U and Uhat must be contiguous CUDA float64 tensors")
        p = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        _check(self.lib.dgx_hdg_blocks(self.h, p(U), p(Uhat), float(gamma), p(K), p(C), p(D), p(A), p(R), p(h),
                                       _stream_ptr(stream)), "dgx_hdg_blocks")
        return (K, C, D, A, R, h) if forms else (K, C, D, A)

    def hdg_condense(self, K, C, D, A33, stream=None):
        """(K^{-1} C, A33 - D K^{-1} C) per element."""
        KinvC = torch.empty_like(C)
        S = torch.empty_like(A33)
        ws = self.workspace(OP_HDG)
        p = lambda t: ctypes.c_void_p(t.data_ptr())
        _check(self.lib.dgx_hdg_condense(self.h, p(K), p(C), p(D), p(A33), p(KinvC), p(S), self._aligned(ws),
                                         _stream_ptr(stream)), "dgx_hdg_condense")
        return KinvC, S

    def rhs_noalloc(self, U: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
        """f = dU/dt without a workspace: for callers that may not allocate
        device memory (the scratch is the library's fixed 64 MiB array, shared
        by every call on the device; overlapping calls race)."""
        _check(self.lib.dgx_rhs_noalloc(self.h, self._state(U), self._state(out, "out"), _stream_ptr(stream)),
               "dgx_rhs_noalloc")
        return out

    def rhs_vjp(self, U: torch.Tensor, lam: torch.Tensor, out: Optional[torch.Tensor] = None,
                stream=None) -> torch.Tensor:
        out = self.empty_state() if out is None else out
        ws = self.workspace(OP_VJP)
        _check(self.lib.dgx_rhs_vjp(self.h, self._state(U), self._state(lam, "lambda"), self._state(out, "out"),
                                    self._aligned(ws), _stream_ptr(stream)), "dgx_rhs_vjp")
        return out

    def ark_step(self, U64: torch.Tensor, dt: float, stream=None) -> torch.Tensor:
        ws = self.workspace(OP_ARK)
        _check(self.lib.dgx_ark_step(self.h, self._state(U64, "U64", torch.float64), float(dt), self._aligned(ws),
                                     _stream_ptr(stream)), "dgx_ark_step")
        return U64

    def stage_buffer(self) -> torch.Tensor:
        """Device buffer for one step's stage checkpoints (dgx_stage_bytes)."""
        nbytes = int(self.lib.dgx_stage_bytes(self.h))
        if not nbytes:
            raise DGXError(7, "stage_buffer (no tableau)")
        raw = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        off = (-raw.data_ptr()) % 256
        return raw[off:off + nbytes]

    def stage_state(self, stages: torch.Tensor, i: int) -> torch.Tensor:
        """View of the stage state y_{i+1} stored in a stage buffer."""
        slot = stages.numel() // self.stages
        nbytes = int(np.prod(self.shape)) * (8 if self.dtype == torch.float64 else 4)
        return stages[slot * i: slot * i + nbytes].view(self.dtype).view(self.shape)

    def _stages_ptr(self, stages):
        if not (stages.is_cuda and stages.dtype == torch.uint8 and stages.is_contiguous()
                and stages.numel() == int(self.lib.dgx_stage_bytes(self.h)) and stages.data_ptr() % 256 == 0):
            raise ValueError("stages must come from stage_buffer()")
        return ctypes.c_void_p(stages.data_ptr())

    def ark_step_stages(self, U64: torch.Tensor, dt: float, stages: torch.Tensor, stream=None) -> torch.Tensor:
        ws = self.workspace(OP_ARK)
        _check(self.lib.dgx_ark_step_stages(self.h, self._state(U64, "U64", torch.float64), float(dt),
                                            self._stages_ptr(stages), self._aligned(ws), _stream_ptr(stream)),
               "dgx_ark_step_stages")
        return U64

    def ark_adjoint_step(self, stages: torch.Tensor, lam64: torch.Tensor, dt: float, stream=None) -> torch.Tensor:
        """lam64: cotangent of U_{n+1} on entry, of U_n on exit (FP64, in place)."""
        ws = self.workspace(OP_ARK_ADJOINT)
        _check(self.lib.dgx_ark_adjoint_step(self.h, self._stages_ptr(stages),
                                             self._state(lam64, "lam64", torch.float64), float(dt),
                                             self._aligned(ws), _stream_ptr(stream)), "dgx_ark_adjoint_step")
        return lam64

    def ark_step_adjoint(self, U64: torch.Tensor, lam64: torch.Tensor, dt: float, stages: torch.Tensor,
                         stream=None):
        """One ARK step (U64: U_n -> U_{n+1}, stage checkpoints in stages) and
        its discrete adjoint (lam64: lambda_{n+1} -> lambda_n) in one call; the
        kernels that form U_{n+1} overlap the adjoint on a second stream."""
        ws = self.workspace(OP_ARK_STEP_ADJOINT)
        _check(self.lib.dgx_ark_step_adjoint(self.h, self._state(U64, "U64", torch.float64),
                                             self._state(lam64, "lam64", torch.float64), float(dt),
                                             self._stages_ptr(stages), self._aligned(ws), _stream_ptr(stream)),
               "dgx_ark_step_adjoint")
        return U64, lam64

    def capture(self, fn, warmup: int = 2):
        """Capture fn() -- any sequence of this library's calls on the current
        stream, with fixed buffers and arguments -- into a CUDA graph.  The
        workspaces must already exist (warm-up calls create them) and the
        profiler must be off.  Returns a torch.cuda.CUDAGraph; replay() it."""
        side = torch.cuda.Stream(device=self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(side):
            for _ in range(warmup):
                fn()
        torch.cuda.current_stream(self.device).wait_stream(side)
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        return g

    def check(self):
        _check(self.lib.dgx_check(self.h), "dgx_check")

    def supports_adjoint(self) -> bool:
        return int(self.lib.dgx_workspace_bytes(self.h, OP_VJP)) > 0

    # ------------------------------------------------------------------ tracing
    def profile(self, enable: bool = True):
        _check(self.lib.dgx_profile_enable(self.h, int(enable)), "dgx_profile_enable")

    def profile_reset(self):
        _check(self.lib.dgx_profile_reset(self.h), "dgx_profile_reset")

    def autotune(self, U64: torch.Tensor, reps: int = 3, stream=None):
        """Pick the fastest tile variant per kernel on this state (set-up call)."""
        _check(self.lib.dgx_autotune(self.h, self._state(U64, "U64", torch.float64), int(reps),
                                     _stream_ptr(stream)), "dgx_autotune")
        return self.variants()

    def set_pipeline(self, enable: bool):
        """Select the persistent TMA-fed kernels (default) or the one-CTA-per-tile ones."""
        _check(self.lib.dgx_set_pipeline(self.h, int(enable)), "dgx_set_pipeline")

    def set_contraction(self, mode: str):
        """Contraction engine of the forward element kernel: "cuda_core" (default),
        "tf32", "bf16" or "3xtf32" (tcgen05 tensor cores, FP32 handles only)."""
        if mode not in CONTRACTIONS:
            raise ValueError(f"contraction must be one of {sorted(CONTRACTIONS)}")
        _check(self.lib.dgx_set_contraction(self.h, CONTRACTIONS[mode]), "dgx_set_contraction")

    @property
    def contraction(self) -> str:
        v = ctypes.c_int32()
        _check(self.lib.dgx_get_contraction(self.h, ctypes.byref(v)), "dgx_get_contraction")
        return {c: k for k, c in CONTRACTIONS.items()}[v.value]

    def variants(self) -> dict:
        v = (ctypes.c_int32 * len(KERNELS))()
        _check(self.lib.dgx_get_variants(self.h, v), "dgx_get_variants")
        return {k: v[i] for i, k in enumerate(KERNELS)}

    def set_variants(self, variants: dict):
        cur = self.variants()
        cur.update(variants)
        v = (ctypes.c_int32 * len(KERNELS))(*[cur[k] for k in KERNELS])
        _check(self.lib.dgx_set_variants(self.h, v), "dgx_set_variants")

    def kernel_work(self, name: str):
        """(algorithmic flops, algorithmic bytes) of one launch of a kernel kind."""
        fl, by = ctypes.c_double(), ctypes.c_double()
        _check(self.lib.dgx_kernel_work(self.h, KERNELS.index(name), ctypes.byref(fl), ctypes.byref(by)),
               "dgx_kernel_work")
        return fl.value, by.value

    def profile_read(self) -> dict:
        """{kernel name: (launches, total device ms)} since the last reset."""
        out = {}
        for k, name in enumerate(KERNELS):
            n, ms = ctypes.c_int64(), ctypes.c_double()
            _check(self.lib.dgx_profile_read(self.h, k, ctypes.byref(n), ctypes.byref(ms)), "dgx_profile_read")
            if n.value:
                out[name] = (n.value, ms.value)
        return out


class Residual(torch.autograd.Function):
    """f = dU/dt as a differentiable torch op; backward is the hand-written
    adjoint kernel chain (dgx_rhs_vjp), not autograd of anything."""

    @staticmethod
    def forward(ctx, U, solver):
        ctx.solver = solver
        ctx.save_for_backward(U)
        return solver.rhs(U.contiguous())

    @staticmethod
    def backward(ctx, grad_out):
        (U,) = ctx.saved_tensors
        return ctx.solver.rhs_vjp(U.contiguous(), grad_out.contiguous()), None


def residual(U: torch.Tensor, solver: Solver) -> torch.Tensor:
    return Residual.apply(U, solver)


def adjoint_trajectory(solver: Solver, U0: torch.Tensor, dt: float, nsteps: int, lam_final: torch.Tensor,
                       checkpoints: Optional[list] = None):
    """Gradient of <lam_final, U_N> w.r.t. U_0 through N explicit ARK steps.

    Forward: store U_n (FP64) before every step (one checkpoint per step).
    Reverse: for n = N-1 .. 0 recompute the step's stage states from U_n and
    apply the step's adjoint, both by dgx_ark_step_adjoint (the recomputed
    U_{n+1} is not needed and overlaps the adjoint).  Returns (U_N, lam_0).
    """
    U = U0.clone()
    ckpt = checkpoints if checkpoints is not None else []
    ckpt.clear()
    for _ in range(nsteps):
        ckpt.append(U.clone())
        solver.ark_step(U, dt)
    lam = lam_final.clone()
    stages = solver.stage_buffer()
    work = torch.empty_like(U)
    for n in reversed(range(nsteps)):
        work.copy_(ckpt[n])
        solver.ark_step_adjoint(work, lam, dt, stages)
    return U, lam


class Batch:
    """Many independent instances advanced together (see dgx_batch_* in dgx.h).

    ``solvers``: Solver objects with mesh and tableau set (the same tableau);
    ``dt``: one time step per instance.  States live in one packed FP64 buffer
    (``pack`` / ``unpack``)."""

    def __init__(self, solvers, dt):
        self.lib = load_library()
        self.solvers = list(solvers)
        n = len(self.solvers)
        handles = (ctypes.c_void_p * n)(*[s.h.value for s in self.solvers])
        b = ctypes.c_void_p()
        _check(self.lib.dgx_batch_create(handles, n, ctypes.byref(b)), "dgx_batch_create")
        self.b = b
        offs = (ctypes.c_int64 * (n + 1))()
        ng = ctypes.c_int32()
        _check(self.lib.dgx_batch_layout(b, offs, ctypes.byref(ng)), "dgx_batch_layout")
        self.offsets = [offs[i] for i in range(n + 1)]
        self.groups = ng.value
        self.device = self.solvers[0].device
        self.set_dt(dt)
        nbytes = int(self.lib.dgx_batch_workspace_bytes(b))
        raw = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        off = (-raw.data_ptr()) % 256
        self._ws_raw = raw
        self.ws = ctypes.c_void_p(raw.data_ptr() + off)

    def set_dt(self, dt):
        arr = np.ascontiguousarray(dt, dtype=np.float64)
        if arr.shape != (len(self.solvers),):
            raise ValueError("one dt per instance")
        _check(self.lib.dgx_batch_set_dt(self.b, _ptr(arr)), "dgx_batch_set_dt")
        self.dt = arr

    def empty(self):
        return torch.empty(self.offsets[-1], dtype=torch.float64, device=self.device)

    def _range(self, i):
        n = int(np.prod(self.solvers[i].shape))
        return self.offsets[i], self.offsets[i] + n

    def pack(self, states):
        """Packed FP64 state (instances are stored group by group, see dgx_batch_layout)."""
        out = self.empty()
        for i, U in enumerate(states):
            a, b = self._range(i)
            out[a:b] = torch.as_tensor(U, dtype=torch.float64).reshape(-1)
        return out

    def unpack(self, packed):
        return [packed[slice(*self._range(i))].view(s.shape) for i, s in enumerate(self.solvers)]

    def _packed(self, U):
        if not (U.is_cuda and U.dtype == torch.float64 and U.is_contiguous() and U.numel() == self.offsets[-1]):
            raise ValueError("packed state must come from Batch.empty()/pack()")
        return ctypes.c_void_p(U.data_ptr())

    def step(self, U, graph: bool = False, stream=None):
        fn = self.lib.dgx_batch_step_graph if graph else self.lib.dgx_batch_step
        _check(fn(self.b, self._packed(U), self.ws, _stream_ptr(stream)), "dgx_batch_step")
        return U

    def set_persistent(self, enable: bool = True):
        """One persistent launch per phase over all groups (True) or the graph
        of concurrent per-group launches (False)."""
        _check(self.lib.dgx_batch_set_persistent(self.b, int(bool(enable))), "dgx_batch_set_persistent")

    def autotune(self, U, reps: int = 3, stream=None):
        _check(self.lib.dgx_batch_autotune(self.b, self._packed(U), int(reps), _stream_ptr(stream)),
               "dgx_batch_autotune")

    def close(self):
        if getattr(self, "b", None):
            self.lib.dgx_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
