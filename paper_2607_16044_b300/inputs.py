"""Seeded synthetic inputs: meshes, connectivity and initial states.

This module generates *inputs* only -- element geometry, face connectivity
tables and closed-form / seeded initial states.  It contains none of the DG
method's arithmetic (no basis, metric, flux or residual code); node positions
use numpy's own Gauss-Legendre routine.  Both the CUDA path and the CPU oracle
consume what it produces, so it is the one module the two sides share.

Conventions (the same as the C ABI):

* ``d`` = 2 or 3, ``n = p + 1`` nodes per direction, ``N = n**d`` per element,
  ``nf = d + 2`` conserved fields ordered (rho, rho*u, rho*v[, rho*w], rho*E).
* A state is an array ``U[E][nf][N]``; node ``q = q0 + n*q1 (+ n*n*q2)``
  (x index fastest).
* Local faces ``2a`` (xi_a = -1) and ``2a+1`` (xi_a = +1), a = 0..d-1.
* ``neighbor[e][f]`` = element across face f, or ``-(1 + tag)`` on a physical
  boundary (tag 0 = adiabatic no-slip wall).  ``nbr_face[e][f]`` = the
  neighbour's local face index.  ``orient[e][f]`` maps the own face point
  (s, t) -- the two remaining local indices in increasing axis order, index
  ``s + n*t`` -- to the neighbour's face point (u, v): bit 2 swaps (s, t)
  first, then bit 0 reverses u and bit 1 reverses v.  In 2D only bit 0 is used.
"""
from __future__ import annotations

import dataclasses
import json
from typing import Optional, Sequence

import numpy as np

WALL = 0


def gauss_points(p: int) -> np.ndarray:
    """Gauss-Legendre abscissae on [-1, 1] (numpy's routine), ascending."""
    x, _ = np.polynomial.legendre.leggauss(p + 1)
    return x


@dataclasses.dataclass
class Mesh:
    dim: int
    p: int
    n_elem: int
    kind: str                          # "boxes" (axis-aligned) or "nodes" (curvilinear)
    xyz: np.ndarray                    # [E][d][N] physical coordinates of the nodes
    neighbor: np.ndarray               # int32 [E][2d]
    nbr_face: np.ndarray               # int8  [E][2d]
    orient: np.ndarray                 # int8  [E][2d]
    lo: Optional[np.ndarray] = None    # [E][d]  lower corner  (boxes only)
    size: Optional[np.ndarray] = None  # [E][d]  edge lengths  (boxes only)
    shape: Optional[tuple] = None      # structured element counts (for convenience)

    @property
    def n(self):
        return self.p + 1

    @property
    def N(self):
        return self.n ** self.dim

    @property
    def nf(self):
        return self.dim + 2

    def as_nodes(self) -> "Mesh":
        """Same mesh described by node coordinates instead of boxes."""
        return dataclasses.replace(self, kind="nodes", lo=None, size=None)


def _node_multi_index(dim, n):
    """q -> (q0, q1[, q2]) with q0 fastest."""
    q = np.arange(n ** dim)
    return [(q // n ** a) % n for a in range(dim)]


def structured_box_mesh(p: int, edges: Sequence[np.ndarray], periodic: Sequence[bool],
                        wall_tag: int = WALL) -> Mesh:
    """Tensor-product mesh of axis-aligned boxes.

    ``edges[a]`` are the vertex coordinates along axis a (length n_a + 1).
    Element index ``e = i0 + n0*(i1 + n1*i2)``.  Non-periodic ends are walls.
    """
    dim = len(edges)
    counts = [len(ed) - 1 for ed in edges]
    E = int(np.prod(counts))
    n = p + 1
    N = n ** dim
    xi = gauss_points(p)
    idx = np.arange(E)
    ii = [(idx // int(np.prod(counts[:a]))) % counts[a] for a in range(dim)]
    lo = np.stack([np.asarray(edges[a], dtype=np.float64)[ii[a]] for a in range(dim)], axis=1)
    hi = np.stack([np.asarray(edges[a], dtype=np.float64)[ii[a] + 1] for a in range(dim)], axis=1)
    size = hi - lo
    qi = _node_multi_index(dim, n)
    xyz = np.empty((E, dim, N))
    for a in range(dim):
        xyz[:, a, :] = lo[:, a:a + 1] + 0.5 * (1.0 + xi[qi[a]])[None, :] * size[:, a:a + 1]
    neighbor = np.empty((E, 2 * dim), dtype=np.int32)
    nbr_face = np.empty((E, 2 * dim), dtype=np.int8)
    orient = np.zeros((E, 2 * dim), dtype=np.int8)
    stride = [int(np.prod(counts[:a])) for a in range(dim)]
    for a in range(dim):
        for side in (0, 1):
            f = 2 * a + side
            step = -1 if side == 0 else 1
            j = ii[a] + step
            inside = (j >= 0) & (j < counts[a])
            wrapped = j % counts[a]
            nb = idx + (wrapped - ii[a]) * stride[a]
            if periodic[a]:
                neighbor[:, f] = nb
                nbr_face[:, f] = f ^ 1
            else:
                neighbor[:, f] = np.where(inside, nb, -(1 + wall_tag))
                nbr_face[:, f] = np.where(inside, f ^ 1, -1)
    return Mesh(dim, p, E, "boxes", xyz, neighbor, nbr_face, orient, lo, size, tuple(counts))


def uniform_edges(a: float, b: float, n: int) -> np.ndarray:
    return np.linspace(a, b, n + 1)


def wall_stretched_edges(n_half: int, ratio: float, y0: float = -1.0, y1: float = 1.0) -> np.ndarray:
    """Edges on [y0, y1] with ``n_half`` layers growing geometrically from each wall."""
    half = 0.5 * (y1 - y0)
    h = ratio ** np.arange(n_half)
    h = h / h.sum() * half
    lower = y0 + np.concatenate([[0.0], np.cumsum(h)])
    lower[-1] = y0 + half
    upper = (y1 - (lower - y0))[::-1]
    return np.concatenate([lower, upper[1:]])


# ---------------------------------------------------------------------------
# Curvilinear meshes.  The geometry of each element is the degree-p polynomial
# map that interpolates a smooth global map at the element's Gauss-Lobatto
# points, so neighbouring elements share their faces exactly; the C ABI then
# receives that map sampled at the Gauss nodes.
# ---------------------------------------------------------------------------

def _lobatto_points(p):
    inner = np.polynomial.legendre.Legendre.basis(p).deriv().roots() if p > 1 else np.array([])
    return np.concatenate([[-1.0], np.sort(np.real(inner)), [1.0]])


def _lagrange_matrix(nodes, at):
    L = np.ones((len(at), len(nodes)))
    for j in range(len(nodes)):
        for k in range(len(nodes)):
            if k != j:
                L[:, j] *= (at - nodes[k]) / (nodes[j] - nodes[k])
    return L


def warped_mesh(p: int, counts: Sequence[int], length: Sequence[float], amp: float,
                periodic: Optional[Sequence[bool]] = None, mixed: bool = False) -> Mesh:
    """Smoothly warped tensor mesh of [0, L_0] x ... with a periodic sine warp.

    x_a' = x_a + amp * L_a * prod_b sin(2 pi k_a x_b / L_b)  (vanishes on the
    box boundary, so periodic wrap and walls stay planar), k_a = 1; with
    ``mixed`` k_a = a + 1, so the displacement gradient is no longer rank one
    and J is not a degree-p polynomial in each direction.
    """
    dim = len(counts)
    periodic = periodic if periodic is not None else [True] * dim
    edges = [uniform_edges(0.0, length[a], counts[a]) for a in range(dim)]
    base = structured_box_mesh(p, edges, periodic)
    n = p + 1
    gl = _lobatto_points(p)
    xg = gauss_points(p)
    L1 = _lagrange_matrix(gl, xg)            # Lobatto values -> Gauss values (1D)
    qi = _node_multi_index(dim, n)
    # physical Lobatto points of each element
    xl = np.empty((base.n_elem, dim, n ** dim))
    for a in range(dim):
        xl[:, a, :] = base.lo[:, a:a + 1] + 0.5 * (1.0 + gl[qi[a]])[None, :] * base.size[:, a:a + 1]
    warped = np.empty_like(xl)
    for a in range(dim):
        k = a + 1 if mixed else 1
        prod = np.ones((base.n_elem, n ** dim))
        for b in range(dim):
            prod = prod * np.sin(2.0 * np.pi * k * xl[:, b, :] / length[b])
        warped[:, a, :] = xl[:, a, :] + amp * length[a] * prod
    # tensor-product interpolation Lobatto -> Gauss
    xyz = np.empty_like(warped)
    for a in range(dim):
        v = warped[:, a, :].reshape((base.n_elem,) + (n,) * dim)   # axes (q_{d-1}, ..., q0)
        for ax in range(dim):
            v = np.moveaxis(np.tensordot(v, L1, axes=([1 + ax], [1])), -1, 1 + ax)
        xyz[:, a, :] = v.reshape(base.n_elem, -1)
    return Mesh(dim, p, base.n_elem, "nodes", xyz, base.neighbor, base.nbr_face, base.orient,
                shape=base.shape)


def rotate_elements(mesh: Mesh, seed: int) -> Mesh:
    """Give every element a random local frame (a signed axis permutation).

    Node order, face numbering, ``nbr_face`` and ``orient`` are rewritten so
    the mesh is geometrically the same but no longer has aligned local frames.
    The result is always a "nodes" mesh.
    """
    rng = np.random.default_rng(seed)
    dim, n, E = mesh.dim, mesh.n, mesh.n_elem
    perms, signs = [], []
    for _ in range(E):
        perm = rng.permutation(dim)
        sign = rng.choice([-1, 1], size=dim)
        # keep right-handed frames (positive Jacobian)
        if np.linalg.det(np.eye(dim)[perm] * sign[:, None]) < 0:
            sign[0] = -sign[0]
        perms.append(perm)
        signs.append(sign)
    qi_local = _node_multi_index(dim, n)

    def global_multi(e, loc):          # local multi-index -> global (structured) multi-index
        g = [0] * dim
        for a in range(dim):
            g[perms[e][a]] = loc[a] if signs[e][a] > 0 else n - 1 - loc[a]
        return g

    xyz = np.empty_like(mesh.xyz)
    for e in range(E):
        gq = np.zeros(n ** dim, dtype=np.int64)
        for a in range(dim):
            ga = qi_local[a] if signs[e][a] > 0 else n - 1 - qi_local[a]
            gq += ga * n ** perms[e][a]
        xyz[e] = mesh.xyz[e][:, gq]

    def local_face_of(e, gface):
        A, S = gface // 2, gface % 2
        for a in range(dim):
            if perms[e][a] == A:
                s_local = S if signs[e][a] > 0 else 1 - S
                return 2 * a + s_local
        raise AssertionError

    def face_points(e, f):             # local face -> list of global multi-indices of its points
        a = f // 2
        rest = [b for b in range(dim) if b != a]
        pts = []
        for t in range(n if dim == 3 else 1):
            for s in range(n):
                loc = [0] * dim
                loc[a] = 0 if f % 2 == 0 else n - 1
                loc[rest[0]] = s
                if dim == 3:
                    loc[rest[1]] = t
                pts.append(global_multi(e, loc))
        return pts

    neighbor = np.empty_like(mesh.neighbor)
    nbr_face = np.empty_like(mesh.nbr_face)
    orient = np.zeros_like(mesh.orient)
    for e in range(E):
        for f in range(2 * dim):
            a = f // 2
            S_local = f % 2
            A = perms[e][a]
            S = S_local if signs[e][a] > 0 else 1 - S_local
            gface = 2 * A + S
            nb = mesh.neighbor[e, gface]
            neighbor[e, f] = nb
            if nb < 0:
                nbr_face[e, f] = -1
                continue
            gnf = mesh.nbr_face[e, gface]
            lnf = local_face_of(nb, gnf)
            nbr_face[e, f] = lnf
            own = face_points(e, f)
            oth = face_points(nb, lnf)
            # match by position along the face (drop the normal-axis index)
            key = lambda g: tuple(g[b] for b in range(dim) if b != A)
            oth_index = {key(g): i for i, g in enumerate(oth)}
            mapping = [oth_index[key(g)] for g in own]
            orient[e, f] = _encode_orient(mapping, n, dim)
    return Mesh(dim, mesh.p, E, "nodes", xyz, neighbor, nbr_face, orient, shape=mesh.shape)


def orient_map(code: int, n: int, dim: int) -> np.ndarray:
    """Own face-point index -> neighbour face-point index for an orientation code."""
    if dim == 2:
        s = np.arange(n)
        return n - 1 - s if code & 1 else s
    s = np.tile(np.arange(n), n)
    t = np.repeat(np.arange(n), n)
    if code & 4:
        s, t = t, s
    u = n - 1 - s if code & 1 else s
    v = n - 1 - t if code & 2 else t
    return u + n * v


def _encode_orient(mapping, n, dim):
    mapping = np.asarray(mapping)
    for code in range(2 if dim == 2 else 8):
        if np.array_equal(orient_map(code, n, dim), mapping):
            return code
    raise AssertionError("face mapping is not a valid orientation")


# ---------------------------------------------------------------------------
# Physical parameters and initial states
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Physics:
    gamma: float = 1.4
    Re: float = 0.0          # 0 / inf -> inviscid (Euler)
    Pr: float = 0.72
    Ma: float = 1.0
    viscous: bool = False


def primitive_to_conservative(rho, vel, p, gamma):
    """(rho, velocity list, p) -> U = (rho, rho*u..., rho*E) with ideal-gas E."""
    d = len(vel)
    ke = 0.5 * sum(v * v for v in vel)
    U = [rho] + [rho * v for v in vel] + [p / (gamma - 1.0) + rho * ke]
    return np.stack(U, axis=-2) if np.ndim(rho) > 1 else np.stack(U)


def _stack_state(rho, vel, p, gamma):
    ke = 0.5 * sum(v * v for v in vel)
    comps = [rho] + [rho * v for v in vel] + [p / (gamma - 1.0) + rho * ke]
    return np.stack(comps, axis=1)          # [E][nf][N]


def isentropic_vortex(mesh: Mesh, t: float = 0.0, gamma: float = 1.4, eps: float = 5.0,
                      box=(-5.0, 5.0), uinf=(1.0, 1.0)) -> np.ndarray:
    """Shu-type isentropic vortex of strength ``eps`` in free stream (1, u_inf, 1).

    At time t the exact solution is the initial vortex translated by u_inf*t
    and wrapped periodically into ``box`` (nearest image).
    """
    x, y = mesh.xyz[:, 0, :], mesh.xyz[:, 1, :]
    L = box[1] - box[0]
    xc = box[0] + 0.5 * L + uinf[0] * t
    yc = box[0] + 0.5 * L + uinf[1] * t
    dx = (x - xc + 0.5 * L) % L - 0.5 * L
    dy = (y - yc + 0.5 * L) % L - 0.5 * L
    r2 = dx * dx + dy * dy
    g = np.exp(0.5 * (1.0 - r2))
    du = -eps / (2 * np.pi) * g * dy
    dv = eps / (2 * np.pi) * g * dx
    dT = -(gamma - 1.0) * eps ** 2 / (8.0 * gamma * np.pi ** 2) * g * g
    rho = (1.0 + dT) ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    return _stack_state(rho, [uinf[0] + du, uinf[1] + dv], p, gamma)


def channel_state(mesh: Mesh, phys: Physics, seed: int, amp: float = 1e-3) -> np.ndarray:
    """Poiseuille profile u = 1 - s^2 (s = wall-normal coordinate in [-1, 1]),
    rho = 1, p = 1/(gamma Ma^2), each conserved field times (1 + amp*xi),
    xi ~ U(-1, 1) i.i.d. per node from ``numpy.random.default_rng(seed)``."""
    d = mesh.dim
    s = mesh.xyz[:, d - 1, :]
    rho = np.ones_like(s)
    vel = [1.0 - s * s] + [np.zeros_like(s)] * (d - 1)
    p = np.full_like(s, 1.0 / (phys.gamma * phys.Ma ** 2))
    U = _stack_state(rho, vel, p, phys.gamma)
    rng = np.random.default_rng(seed)
    return U * (1.0 + amp * rng.uniform(-1.0, 1.0, size=U.shape))


def taylor_green(mesh: Mesh, phys: Physics) -> np.ndarray:
    """Taylor-Green vortex on [0, 2 pi)^3, isothermal (theta = 1), p_inf = 1/(gamma Ma^2)."""
    x, y, z = mesh.xyz[:, 0, :], mesh.xyz[:, 1, :], mesh.xyz[:, 2, :]
    u = np.sin(x) * np.cos(y) * np.cos(z)
    v = -np.cos(x) * np.sin(y) * np.cos(z)
    w = np.zeros_like(x)
    pinf = 1.0 / (phys.gamma * phys.Ma ** 2)
    p = pinf + (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0) / 16.0
    R = 1.0 / (phys.gamma * phys.Ma ** 2)
    rho = p / R
    return _stack_state(rho, [u, v, w], p, phys.gamma)


def random_state(mesh: Mesh, seed: int, gamma: float = 1.4, amp: float = 0.1) -> np.ndarray:
    """Random nodal state, i.i.d. per node, whose face traces stay physical.

    Gauss-node extrapolation to a face amplifies nodal noise by at most
    sum_j |l_j(+-1)| (< 3.75 for p <= 5), so amp = 0.1 keeps the traced density
    and pressure positive."""
    rng = np.random.default_rng(seed)
    E, N, d = mesh.n_elem, mesh.N, mesh.dim
    rho = 1.0 + amp * rng.uniform(-1, 1, size=(E, N))
    vel = [0.5 + amp * rng.uniform(-1, 1, size=(E, N)) for _ in range(d)]
    p = 1.0 + amp * rng.uniform(-1, 1, size=(E, N))
    return _stack_state(rho, vel, p, gamma)


def gaussian_cotangent(shape, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(shape)


# ---------------------------------------------------------------------------
# The five benchmark workloads
# ---------------------------------------------------------------------------

def vortex_workload(p=3, cells=16):
    """2D Euler isentropic vortex, periodic [-5,5]^2, cells x cells quads."""
    mesh = structured_box_mesh(p, [uniform_edges(-5, 5, cells)] * 2, [True, True])
    phys = Physics(gamma=1.4, viscous=False)
    return mesh, phys, isentropic_vortex(mesh, 0.0, phys.gamma)


def channel2d_workload(p=4, nx=256, n_half=64, ratio=1.15, seed=2):
    """2D NS channel: x in [0,5) periodic, y in [-1,1] wall-stretched, walls at y=+-1."""
    mesh = structured_box_mesh(p, [uniform_edges(0.0, 5.0, nx), wall_stretched_edges(n_half, ratio)],
                               [True, False])
    phys = Physics(gamma=1.4, Re=1000.0, Pr=0.72, Ma=0.3, viscous=True)
    return mesh, phys, channel_state(mesh, phys, seed)


def tgv_workload(p=3, cells=32):
    mesh = structured_box_mesh(p, [uniform_edges(0.0, 2 * np.pi, cells)] * 3, [True] * 3)
    phys = Physics(gamma=1.4, Re=1600.0, Pr=0.71, Ma=0.1, viscous=True)
    return mesh, phys, taylor_green(mesh, phys)


def channel3d_workload(p=5, nxy=48, n_half=24, ratio=1.1, seed=5):
    ex = uniform_edges(0.0, 2 * np.pi, nxy)
    mesh = structured_box_mesh(p, [ex, ex, wall_stretched_edges(n_half, ratio)], [True, True, False])
    phys = Physics(gamma=1.4, Re=1000.0, Pr=0.72, Ma=0.3, viscous=True)
    return mesh, phys, channel_state(mesh, phys, seed)


def ensemble_manifest(count=64, seed=4):
    """(cells, p, viscous, dt) per instance, drawn from ``default_rng(seed)``."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        cells = int(rng.integers(8, 97))
        p = int(rng.integers(2, 6))
        viscous = bool(i % 2 == 1)
        h = 10.0 / cells
        dt = 0.1 * h / (2.6 * (2 * p + 1))
        out.append({"cells": cells, "p": p, "viscous": viscous, "dt": dt})
    return out


def ensemble_instance(spec):
    mesh = structured_box_mesh(spec["p"], [uniform_edges(-5, 5, spec["cells"])] * 2, [True, True])
    if spec["viscous"]:
        phys = Physics(gamma=1.4, Re=1000.0, Pr=0.72, Ma=1.0 / np.sqrt(1.4), viscous=True)
    else:
        phys = Physics(gamma=1.4, viscous=False)
    return mesh, phys, isentropic_vortex(mesh, 0.0, phys.gamma)


def manifest_json(count=64, seed=4):
    return json.dumps(ensemble_manifest(count, seed), indent=1)
