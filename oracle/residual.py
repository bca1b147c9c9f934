"""The explicit DG right-hand side f(U) = dU/dt = -M^{-1} B(U) (oracle).

Test infrastructure only.  Follows Sec. 3.3 of the paper (weak form of DG-IP:
volume term (F^nu - F^c) : grad V, numerical-flux surface term, mass matrix),
with the convective numerical flux read as local Lax-Friedrichs and the
viscous terms as BR1 (Bassi-Rebay 1) instead of SIPG, on collocated
Gauss-Legendre nodes.  With B the form that the paper's weak form puts on the
left-hand side (Eq. of the DG-IP weak form), the ODE is M dU/dt = -B(U); the
ERK update (Sec. 4.2) then reads y_i = U_n + dt sum_j a_ij f(y_j).

For every node q of an element (w_q = product of 1D weights, J_q = Jacobian):

  B_q = sum_r w_r (F^nu - F^c)(r) : grad l_q(x_r) + sum_faces w_f s_J l_q(x_f) Fstar_n,
  f_q = -B_q / (w_q J_q).

With Ftilde_a = sum_c Ja[a][c] F_c (contravariant flux) and
Dhat[i][m] = w_m D[m][i] / w_i this is, per node,

  f_q = (1/J_q) sum_a sum_m Dhat[q_a][m] (F^c - F^nu)~_a(.., m, ..)
        - sum_faces l_{q_a}(+-1) / (w_{q_a} J_q) * Fhat(face point of q),

where Fhat = s_J Fstar_n is the area-weighted outward numerical flux:

  Fhat = LLF(U^-, U^+; Sn_bar) - Fhat^nu,  Sn_bar = (Sn^- - Sn^+)/2 inside
         (the two sides' outward area normals averaged; equal to Sn^- on
         watertight faces), Sn^- on walls,
  Fhat^nu = 1/2 (G^- - G^+) on interior faces, G = F^nu(U_f, Q_f) . Sn_own
            (each side's viscous flux with its own outward normal),
  Fhat^nu = F^{nu,w}(U_w, Q^-) . Sn on adiabatic walls (q.n = 0).

BR1 gradient (conservative variables), per node:

  Q_a(q) = (1/J_q) sum_b Ja[b][a] (D_b U)(q)
           + sum_faces l_{q_b}(+-1) / (w_{q_b} J_q) (Uhat - U^-) Sn_a,
  Uhat = (U^- + U^+)/2 inside, U_w = (rho, 0, .., rho e_i) on walls.

Convective wall flux: LLF against the mirror state (rho, m - 2(m.n)n, rho E),
which makes the wall mass flux exactly zero.

The same code evaluates the full mesh or, for sampled parity at large sizes,
only a subset of elements (it then works on the 1- or 2-ring around them).
"""
import numpy as np
import torch

from . import physics as ph
from .basis import Basis1D
from .geometry import Geometry, along, trace


def orient_index(code, n, d):
    """Own face-point index -> neighbour face-point index (mesh convention)."""
    if d == 2:
        s = np.arange(n)
        return n - 1 - s if code & 1 else s
    s = np.tile(np.arange(n), n)
    t = np.repeat(np.arange(n), n)
    if code & 4:
        s, t = t, s
    u = n - 1 - s if code & 1 else s
    v = n - 1 - t if code & 2 else t
    return u + n * v


class DGOperator:
    def __init__(self, mesh, gas: ph.Gas):
        self.mesh = mesh
        self.gas = gas
        self.d = d = mesh.dim
        self.n = n = mesh.p + 1
        self.E = mesh.n_elem
        self.nf = d + 2
        self.nfp = n ** (d - 1)
        self.basis = Basis1D(mesh.p)
        self.geo = Geometry(mesh, self.basis)
        self.nb = torch.as_tensor(np.asarray(mesh.neighbor, dtype=np.int64))
        self.nbf = torch.as_tensor(np.asarray(mesh.nbr_face, dtype=np.int64))
        ori = np.asarray(mesh.orient, dtype=np.int64)
        maps = np.stack([orient_index(c, n, d) for c in range(8 if d == 3 else 2)])
        self.omap = torch.as_tensor(maps[ori])                     # [E][2d][nfp]
        b = self.basis
        self.D = torch.as_tensor(b.D)
        w = torch.as_tensor(b.w)
        self.Dhat = (w[None, :] * self.D.T) / w[:, None]          # Dhat[i][m] = w_m D[m][i] / w_i
        self.lift_vec = [torch.as_tensor(b.lm) / w, torch.as_tensor(b.lp) / w]

    # ------------------------------------------------------------------ helpers
    def nodes(self, V):
        """[k][c][N] -> [k][c][n]..[n] (direction a on axis -1-a)."""
        return V.reshape(V.shape[:2] + (self.n,) * self.d)

    def ring(self, S):
        nb = self.nb[S].reshape(-1)
        return torch.unique(torch.cat([S, nb[nb >= 0]]))

    def element_traces(self, Vn):
        """Vn[k][c][n..n] -> T[k][2d][c][nfp]."""
        k, c = Vn.shape[:2]
        out = []
        for a in range(self.d):
            for side in (0, 1):
                out.append(trace(Vn, a, side, self.d, self.basis).reshape(k, c, self.nfp))
        return torch.stack(out, 1)

    def gather_neighbor(self, Tfull, S):
        """Neighbour's trace of each face of the elements S, in own face-point order.

        Boundary faces get zeros (callers substitute boundary states)."""
        nb = self.nb[S].clamp(min=0)                               # [k][2d]
        nbf = self.nbf[S].clamp(min=0)
        T = Tfull[nb, nbf]                                          # [k][2d][c][nfp]
        idx = self.omap[S].unsqueeze(2).expand(-1, -1, T.shape[2], -1)
        return torch.gather(T, 3, idx)

    def lift(self, Fface, J, sign=1.0):
        """sum_faces sign * l_{q_a}(+-1)/(w_{q_a} J_q) Fface(face point of q)."""
        k, _, c, _ = Fface.shape
        d, n = self.d, self.n
        out = 0
        for a in range(d):
            for side in (0, 1):
                Ff = Fface[:, 2 * a + side].reshape((k, c) + (n,) * (d - 1))
                ax = 1 + d - a
                vec = self.lift_vec[side].to(Fface.dtype)
                shape = [1] * (2 + d)
                shape[ax] = n
                out = out + Ff.unsqueeze(ax) * vec.reshape(shape)
        return sign * out / J.unsqueeze(1)

    def _faces_flat(self, X):
        """[k][2d][c][nfp] -> [k*2d*nfp][c] style views for pointwise physics."""
        k, f, c, p = X.shape
        return X.permute(0, 1, 3, 2).reshape(k * f * p, c)

    def _unflat(self, Y, k):
        c = Y.shape[1]
        return Y.reshape(k, 2 * self.d, self.nfp, c).permute(0, 1, 3, 2)

    # ------------------------------------------------------------------ pieces
    def br1_gradient(self, Un_S, TU_S, TUn_S, S):
        """Q[k][a][field][n..n] for the elements S (BR1 lifted gradient)."""
        d = self.d
        J = self.geo.J[S].to(Un_S.dtype)
        Ja = self.geo.Ja[S].to(Un_S.dtype)
        dU = [along(Un_S, b, d, self.D) for b in range(d)]           # D_b U
        wall = (self.nb[S] < 0)
        # Uhat - U^- per face point
        k = len(S)
        Uw = self._unflat(ph.wall_state(self._faces_flat(TU_S), d), k)
        jump = torch.where(wall[:, :, None, None], Uw - TU_S, 0.5 * (TUn_S - TU_S))
        Sn = self.geo.Sn[S].to(Un_S.dtype)
        Q = []
        for a in range(d):
            vol = sum(Ja[:, b, a].unsqueeze(1) * dU[b] for b in range(d)) / J.unsqueeze(1)
            surf = self.lift(jump * Sn[:, :, a].unsqueeze(2), J)
            Q.append(vol + surf)
        return torch.stack(Q, 1)

    def viscous_face_flux(self, TU_S, TQ_S, S):
        """TQ_S[k][2d][a][nf][nfp] -> G[k][2d][nf][nfp] = each side's F^nu(U_f, Q_f) . Sn_own  (wall: F^{nu,w})."""
        d, k = self.d, len(S)
        Sn = self.geo.Sn[S].to(TU_S.dtype)
        Uf = self._faces_flat(TU_S)
        Qf = TQ_S.permute(0, 1, 4, 2, 3).reshape(k * 2 * d * self.nfp, d, self.nf)
        Snf = Sn.permute(0, 1, 3, 2).reshape(-1, d)
        G_int = ph.normal_viscous_flux(Uf, Qf, Snf, self.gas, d)
        G_wall = ph.adiabatic_wall_viscous_flux(Uf, Qf, Snf, self.gas, d)
        wall = (self.nb[S] < 0)[:, :, None, None]
        return torch.where(wall, self._unflat(G_wall, k), self._unflat(G_int, k))

    def convective_face_flux(self, TU_S, TUn_S, S):
        d, k = self.d, len(S)
        # interior faces: averaged area normal (Sn^- - Sn^+)/2, so the flux is
        # exactly antisymmetric across the face (equal to Sn^- on watertight
        # faces up to rounding); walls: own normal
        Sn_own = self.geo.Sn[S]
        Sn_nb = self.gather_neighbor(self.geo.Sn, S)
        wall_f = (self.nb[S] < 0)[:, :, None, None]
        Sn = torch.where(wall_f, Sn_own, 0.5 * (Sn_own - Sn_nb)).to(TU_S.dtype)
        UL = self._faces_flat(TU_S)
        Snf = Sn.permute(0, 1, 3, 2).reshape(-1, d)
        UR_int = self._faces_flat(TUn_S)
        UR_wall = ph.mirror_state(UL, Snf, d)
        wall = (self.nb[S] < 0)[:, :, None, None].reshape(k, 2 * d, 1, 1)
        wall_flat = wall.expand(k, 2 * d, self.nfp, 1).reshape(-1, 1)
        UR = torch.where(wall_flat, UR_wall, UR_int)
        return self._unflat(ph.llf_flux(UL, UR, Snf, self.gas, d), k)

    # ------------------------------------------------------------------ operator
    def residual(self, U, elems=None, return_parts=False):
        """f(U) = dU/dt for all elements (U[E][nf][N]) or for the listed ones."""
        d, nf, E = self.d, self.nf, self.E
        viscous = self.gas.viscous
        S0 = torch.arange(E) if elems is None else torch.as_tensor(elems, dtype=torch.long)
        S1 = self.ring(S0) if (elems is not None) else S0
        S2 = (self.ring(S1) if viscous else S1) if (elems is not None) else S0
        Un = self.nodes(U)
        dtype = U.dtype
        TU = torch.zeros((E, 2 * d, nf, self.nfp), dtype=dtype)
        TU = TU.index_put((S2,), self.element_traces(Un[S2]))
        parts = {}
        if viscous:
            TUn_1 = self.gather_neighbor(TU, S1)
            Q1 = self.br1_gradient(Un[S1], TU[S1], TUn_1, S1)          # [k1][a][nf][n..]
            k1 = len(S1)
            TQ1 = torch.stack([self.element_traces(Q1[:, a]) for a in range(d)], 2)  # [k1][2d][a][nf][nfp]
            G1 = self.viscous_face_flux(TU[S1], TQ1, S1)
            Gfull = torch.zeros((E, 2 * d, nf, self.nfp), dtype=dtype).index_put((S1,), G1)
            pos = torch.full((E,), -1, dtype=torch.long)
            pos[S1] = torch.arange(k1)
            Q0 = Q1[pos[S0]]
            Gn0 = self.gather_neighbor(Gfull, S0)
            wall0 = (self.nb[S0] < 0)[:, :, None, None]
            Fv_face = torch.where(wall0, Gfull[S0], 0.5 * (Gfull[S0] - Gn0))
            parts["Q"] = Q0
        TUn_0 = self.gather_neighbor(TU, S0)
        Fc_face = self.convective_face_flux(TU[S0], TUn_0, S0)
        Fface = Fc_face - Fv_face if viscous else Fc_face
        # volume term
        k0 = len(S0)
        U0 = Un[S0]
        flatU = U0.permute(0, *range(2, 2 + d), 1).reshape(-1, nf)
        F = ph.convective_flux(flatU, self.gas, d)                   # [m][i][nf]
        if viscous:
            Qflat = parts["Q"].permute(0, *range(3, 3 + d), 1, 2).reshape(-1, d, nf)
            F = F - ph.viscous_flux(flatU, Qflat, self.gas, d)
        F = F.reshape((k0,) + (self.n,) * d + (d, nf)).permute(0, 1 + d, 2 + d, *range(1, 1 + d))
        J = self.geo.J[S0].to(dtype)
        Ja = self.geo.Ja[S0].to(dtype)
        vol = 0
        for a in range(d):
            Ft = sum(Ja[:, a, c].unsqueeze(1) * F[:, c] for c in range(d))
            vol = vol + along(Ft, a, d, self.Dhat)
        f = vol / J.unsqueeze(1) + self.lift(Fface, J, sign=-1.0)
        f = f.reshape(k0, nf, -1)
        if return_parts:
            parts.update(TU=TU[S0], Fface=Fface)
            return f, parts
        return f


def term_scale(op, U, elems=None):
    """Per-node magnitude of the terms the residual sums (test infrastructure).

    The same weak form as ``residual`` with every flux and every matrix entry
    replaced by its absolute value: (1/J) sum_a sum_m |Dhat| (|F^c~| + |F^nu~|)
    + sum_faces |l/w| (|Fhat^c| + |Fhat^nu|) / J.  Two FP64 evaluations of f that
    differ only in rounding order agree to a small multiple of eps times this
    scale, however much the terms cancel (low-Mach or near-uniform states).
    """
    d, nf = op.d, op.nf
    S0 = torch.arange(op.E) if elems is None else torch.as_tensor(elems, dtype=torch.long)
    f, parts = op.residual(U, elems, return_parts=True)
    Un = op.nodes(U)[S0]
    flatU = Un.permute(0, *range(2, 2 + d), 1).reshape(-1, nf)
    F = ph.convective_flux(flatU, op.gas, d).abs()
    if op.gas.viscous:
        Qflat = parts["Q"].permute(0, *range(3, 3 + d), 1, 2).reshape(-1, d, nf)
        F = F + ph.viscous_flux(flatU, Qflat, op.gas, d).abs()
    k0 = len(S0)
    F = F.reshape((k0,) + (op.n,) * d + (d, nf)).permute(0, 1 + d, 2 + d, *range(1, 1 + d))
    J = op.geo.J[S0]
    Ja = op.geo.Ja[S0].abs()
    vol = 0
    for a in range(d):
        Ft = sum(Ja[:, a, c].unsqueeze(1) * F[:, c] for c in range(d))
        vol = vol + along(Ft, a, d, op.Dhat.abs())
    saved = op.lift_vec
    op.lift_vec = [v.abs() for v in saved]
    try:
        surf = op.lift(parts["Fface"].abs(), J)
    finally:
        op.lift_vec = saved
    return (vol / J.unsqueeze(1) + surf).reshape(k0, nf, -1)


def residual(mesh, gas, U, elems=None):
    """Convenience: f(U) for a mesh (numpy or torch U[E][nf][N])."""
    op = DGOperator(mesh, gas)
    Ut = torch.as_tensor(U)
    return op.residual(Ut, elems)


def submesh_around(mesh, elems, rings):
    """The elements within ``rings`` neighbour steps of ``elems`` as a mesh of
    their own (test infrastructure for sampled parity on very large meshes).

    Returns (submesh, global ids of its elements, local ids of ``elems``).
    Neighbours outside the kept set are replaced by the element itself; only
    elements at the outermost ring see such faces, and their residuals and
    gradients are never used by the sampled rows.
    """
    import dataclasses
    keep = np.unique(np.asarray(elems, dtype=np.int64))
    for _ in range(rings):
        nb = mesh.neighbor[keep].reshape(-1)
        keep = np.unique(np.concatenate([keep, nb[nb >= 0]]))
    pos = np.full(mesh.n_elem, -1, dtype=np.int64)
    pos[keep] = np.arange(len(keep))
    nb = mesh.neighbor[keep].astype(np.int64)
    inside = nb >= 0
    mapped = np.where(inside, pos[np.where(inside, nb, 0)], nb)
    outside = inside & (mapped < 0)
    self_ids = np.repeat(np.arange(len(keep))[:, None], nb.shape[1], axis=1)
    nbf = mesh.nbr_face[keep].copy()
    ori = mesh.orient[keep].copy()
    faces = np.tile(np.arange(nb.shape[1]), (len(keep), 1))
    mapped = np.where(outside, self_ids, mapped)
    nbf = np.where(outside, faces ^ 1, nbf)
    ori = np.where(outside, 0, ori)
    sub = dataclasses.replace(
        mesh, n_elem=len(keep), xyz=mesh.xyz[keep], neighbor=mapped.astype(np.int32),
        nbr_face=nbf.astype(np.int8), orient=ori.astype(np.int8),
        lo=None if mesh.lo is None else mesh.lo[keep], size=None if mesh.size is None else mesh.size[keep])
    return sub, keep, pos[np.asarray(elems, dtype=np.int64)]
