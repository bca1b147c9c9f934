"""DG-IP operator of the paper: Vijayasundaram flux + symmetric interior
penalty (oracle; test infrastructure only).

Follows Sec. 3.3 of the paper, the DG-IP weak form (Eq. weak_form_sdg_ip with
B_I of Eq. bilinear_form_interior_sdg):

  B_I(U; V) = sum_T int_T (F^nu(U, grad U) - F^c(U)) : grad V
            + int_{dT} F^{c,*}_n(U, U^-) . V
            - sum_F int_F {K grad U} : [V]          (viscous surface term)
            - sum_F int_F {K^T grad V} : [U]        (adjoint consistency)
            + sum_F int_F tau {K} [U] : [V]         (penalty),

with [psi] = psi^+ (x) n^+ + psi^- (x) n^-, {psi} = (psi^+ + psi^-)/2, the
Vijayasundaram flux F^{c,*}_n = A_n^+(Ubar) U + A_n^-(Ubar) U^-, Ubar = {U}
(Eq. upwinding_Vijayasundaram_sdg, eigen-split of Sec. 3.2) and the penalty
tau = alpha (k+1)^2 / l, alpha = 1, l = |T| / |dT| (Eq. penalty_coefficient_ip).
Boundary forms (App. B.1): farfield (Eq. bilinear_form_sdg_exterior_farfield,
boundary state U_Gamma of the characteristic decomposition) and adiabatic wall
(Eq. bilinear_form_sdg_exterior_adiabaticwall, K_w with q.n = 0).  The DG side
of the geometry-split interface (Sec. 4.1.1, Eq. interface_bilinearform_explicit)
treats a face to an implicit element like an interior face against U^im, with
the averaged K in the adjoint-consistency term and only the explicit side
receiving the contribution.

Discretisation: the collocated nodal basis on Gauss-Legendre points of the
LLF/BR1 oracle (``residual``), so f = dU/dt = -M^{-1} B(U) with the diagonal
mass matrix.  Because F^nu is linear in its gradient argument, every K-product
is the viscous flux evaluated with a substituted gradient: K(U)(delta (x) n) =
F^nu(U, grad U := delta (x) n), and K^T(U) grad V : (delta (x) n) =
grad V . F^nu(U, delta (x) n).  Per own face point, with the area normal Sn
(s_J n) and quadrature weight w_f:

  Fhat = F^{c,*}_n s_J - 1/2 (G^+ - G^-) + (tau / s_J) {F^nu}(delta (x) Sn) . Sn,
  G = F^nu(U_f, grad U_f) . Sn_own (each side its own outward normal),
  H = c F^nu(U_f; delta (x) Sn)       (c = 1/2 inside, own K),
  f_q = (1/J_q)[volume] - sum_faces l_q(x_f)/(w_q J_q) w_f Fhat
        + (1/(w_q J_q)) sum_faces w_f grad l_q(x_f) . H,

delta = U^+ - U^- (own minus neighbour); on interior faces Sn is the average
(Sn^+ - Sn^-)/2 of the two sides' area normals (as in ``residual``).  Walls:
Vijayasundaram flux against the mirror state (rho, m - 2(m.n)n, rho E) --
zero mass flux, the reading the LLF path uses --, G = F^{nu,w}(U, grad U).Sn,
delta = U - U_w, H = F^{nu,w}(U; delta (x) Sn) (weight 1).  Farfield:
F^c(U_Gamma).Sn, G = F^nu(U_inf, grad U).Sn, delta = U - U_inf,
H = F^nu(U_inf; delta (x) Sn).  Interface (own explicit, neighbour implicit):
as inside but H = {F^nu}(delta (x) Sn) (weight 1, averaged K).

grad U is the broken gradient of the element's own polynomial (no lifting).
At face points it is the exact gradient of the polynomial: the traces of the
nodal reference derivatives D_b U mapped by the traced metric terms
Ja_f / J_f (exact on affine elements; on curved elements the traces of the
nodal interpolants of Ja and J).  grad l_q(x_f) is formed the same way.
Readings (where the paper is silent or its print is garbled): the face
penalty is tau_F = alpha (k+1)^2 max(1/l^+, 1/l^-); the wall form, printed
without tau in its penalty term, takes tau; {K_w(U_h)} on a wall is K_w at the
interior trace; at lambda_k = 0 the farfield state takes the interior value.
"""
import numpy as np
import torch

from . import physics as ph
from .geometry import along, trace
from .residual import DGOperator

WALL, FARFIELD = 0, 1


class SIPGOperator(DGOperator):
    def __init__(self, mesh, gas, alpha=1.0, U_inf=None, explicit=None, k_penalty=None):
        super().__init__(mesh, gas)
        d, n, E = self.d, self.n, self.E
        self.alpha = float(alpha)
        self.U_inf = None if U_inf is None else torch.as_tensor(np.asarray(U_inf, dtype=np.float64))
        # element mask of the explicit region (None: every element explicit)
        self.explicit = None if explicit is None else torch.as_tensor(np.asarray(explicit, dtype=bool))
        geo = self.geo
        b = self.basis
        # face traces of the metric terms and of J: [E][2d][d][d][nfp], [E][2d][nfp]
        JaF = torch.zeros((E, 2 * d, d, d, self.nfp), dtype=torch.float64)
        JF = torch.zeros((E, 2 * d, self.nfp), dtype=torch.float64)
        for a0 in range(d):
            for side in (0, 1):
                JF[:, 2 * a0 + side] = trace(geo.J, a0, side, d, b).reshape(E, -1)
                for a in range(d):
                    for c in range(d):
                        JaF[:, 2 * a0 + side, a, c] = trace(geo.Ja[:, a, c], a0, side, d, b).reshape(E, -1)
        self.JaF, self.JF = JaF, JF
        # characteristic length l = |T| / |dT| and the face penalty
        w = torch.as_tensor(b.w)
        Wn = self._node_weights(w)
        vol = (geo.J * Wn).reshape(E, -1).sum(1)
        area = 0
        for a0 in range(d):
            wf = self._face_weights(w, a0).reshape(-1)
            for side in (0, 1):
                sJ = torch.sqrt((geo.Sn[:, 2 * a0 + side] ** 2).sum(1))       # [E][nfp]
                area = area + (sJ * wf).sum(1)
        self.inv_l = area / vol                                               # [E]
        k = mesh.p if k_penalty is None else k_penalty      # the solution degree of tau = alpha (k+1)^2 / l
        inv_l_nb = self.inv_l[self.nb.clamp(min=0)]
        face_inv_l = torch.where(self.nb >= 0, torch.maximum(self.inv_l[:, None], inv_l_nb),
                                 self.inv_l[:, None].expand(-1, 2 * d))
        self.tau = self.alpha * (k + 1) ** 2 * face_inv_l                    # [E][2d]

    # -------------------------------------------------------------- weights
    def _node_weights(self, w):
        d, n = self.d, self.n
        W = torch.ones((n,) * d, dtype=torch.float64)
        for a in range(d):
            shape = [1] * d
            shape[d - 1 - a] = n
            W = W * w.reshape(shape)
        return W

    def _face_weights(self, w, a0):
        """Tangential weights of the faces normal to a0 as a face-point array [nfp]
        (remaining directions in increasing order, the first fastest)."""
        d, n = self.d, self.n
        W = torch.ones((n,) * d, dtype=torch.float64)
        for a in range(d):
            if a == a0:
                continue
            shape = [1] * d
            shape[d - 1 - a] = n
            W = W * w.reshape(shape)
        idx = [slice(None)] * d
        idx[d - 1 - a0] = 0
        return W[tuple(idx)].reshape(-1)

    # -------------------------------------------------------------- pieces
    def _states(self, U, U_im):
        if self.explicit is None or U_im is None:
            return U
        m = self.explicit.reshape((-1,) + (1,) * (U.dim() - 1))
        return torch.where(m, U, torch.as_tensor(U_im, dtype=U.dtype))

    def gradients(self, Un):
        """Broken gradient of each element's polynomial: at the nodes
        Q[k][c][nf][n..] and at the face points TQ[k][2d][c][nf][nfp]."""
        d, E = self.d, Un.shape[0]
        J, Ja = self.geo.J.to(Un.dtype), self.geo.Ja.to(Un.dtype)
        dU = [along(Un, b, d, self.D) for b in range(d)]                 # reference derivatives
        Q = torch.stack([sum(Ja[:, b, c].unsqueeze(1) * dU[b] for b in range(d)) / J.unsqueeze(1)
                         for c in range(d)], 1)
        TdU = [self.element_traces(dU[b]) for b in range(d)]              # [k][2d][nf][nfp]
        JaF, JF = self.JaF.to(Un.dtype), self.JF.to(Un.dtype)
        TQ = torch.stack([sum(JaF[:, :, b, c].unsqueeze(2) * TdU[b] for b in range(d)) / JF.unsqueeze(2)
                          for c in range(d)], 2)                          # [k][2d][c][nf][nfp]
        return Q, TQ

    def _flatQ(self, TQ):
        k = TQ.shape[0]
        return TQ.permute(0, 1, 4, 2, 3).reshape(k * 2 * self.d * self.nfp, self.d, self.nf)

    def _flatS(self, Sn):
        return Sn.permute(0, 1, 3, 2).reshape(-1, self.d)

    def _unflatH(self, H, k):
        """[k*2d*nfp][c][nf] -> [k][2d][c][nf][nfp]."""
        return H.reshape(k, 2 * self.d, self.nfp, self.d, self.nf).permute(0, 1, 3, 4, 2)

    def face_terms(self, TU, TQ):
        """Fhat[E][2d][nf][nfp] (area-weighted numerical flux of every own face
        point) and H[E][2d][c][nf][nfp] (the adjoint-consistency vectors)."""
        d, E, nf = self.d, self.E, self.nf
        gas = self.gas
        nb = self.nb
        S = torch.arange(E)
        TUn = self.gather_neighbor(TU, S)
        TQn = torch.stack([self.gather_neighbor(TQ[:, :, c], S) for c in range(d)], 2)
        Sn_own = self.geo.Sn.to(TU.dtype)
        Sn_nb = self.gather_neighbor(self.geo.Sn, S).to(TU.dtype)
        inner = (nb >= 0)[:, :, None, None]
        Sbar = torch.where(inner, 0.5 * (Sn_own - Sn_nb), Sn_own)
        UL = self._faces_flat(TU)
        UR = self._faces_flat(TUn)
        QL, QR = self._flatQ(TQ), self._flatQ(TQn)
        SL, SR, SB = self._flatS(Sn_own), self._flatS(Sn_nb), self._flatS(Sbar)
        tau = self.tau.to(TU.dtype)[:, :, None].expand(E, 2 * d, self.nfp).reshape(-1)
        sJ = torch.sqrt((SB * SB).sum(1))
        kind = nb[:, :, None].expand(E, 2 * d, self.nfp).reshape(-1)
        is_int = kind >= 0
        is_wall = kind == -(1 + WALL)
        is_far = kind == -(1 + FARFIELD)
        iface = torch.zeros_like(is_int)
        if self.explicit is not None:
            ex_own = self.explicit[:, None].expand(E, 2 * d)
            ex_nb = self.explicit[nb.clamp(min=0)]
            iface = ((nb >= 0) & ex_own & ~ex_nb)[:, :, None].expand(E, 2 * d, self.nfp).reshape(-1)

        def visc(U, Q, Sn=None, wall=False):
            return ph.adiabatic_viscous_flux(U, Q, Sn, gas, d) if wall else ph.viscous_flux(U, Q, gas, d)

        def ndot(F, Sn):                      # F[k][i][nf] . Sn[k][i]
            return (F * Sn.unsqueeze(2)).sum(1)

        def outer(delta, Sn):                 # gradient argument delta (x) Sn: [k][i][nf]
            return Sn.unsqueeze(2) * delta.unsqueeze(1)

        # interior and interface faces
        dlt = UL - UR
        F_int = ph.vijayasundaram_flux(UL, UR, SB, gas, d)
        G_own = ndot(visc(UL, QL), SL)
        G_nb = ndot(visc(UR, QR), SR)
        KL = visc(UL, outer(dlt, SB))
        KR = visc(UR, outer(dlt, SB))
        F_int = F_int - 0.5 * (G_own - G_nb) + (tau / sJ).unsqueeze(1) * 0.5 * ndot(KL + KR, SB)
        H_int = torch.where(iface[:, None, None], 0.5 * (KL + KR), 0.5 * KL)
        # walls
        Um = ph.mirror_state(UL, SL, d)
        Uw = ph.wall_state(UL, d)
        dw = UL - Uw
        Kw = visc(UL, outer(dw, SL), SL, wall=True)
        sJL = torch.sqrt((SL * SL).sum(1))
        F_wall = ph.vijayasundaram_flux(UL, Um, SL, gas, d) - ndot(visc(UL, QL, SL, wall=True), SL) \
            + (tau / sJL).unsqueeze(1) * ndot(Kw, SL)
        Fhat = torch.where(is_int[:, None], F_int, F_wall)
        H = torch.where(is_int[:, None, None], H_int, Kw)
        # farfield
        if self.U_inf is not None:
            Ui = self.U_inf.to(TU.dtype).expand_as(UL)
            UG = ph.farfield_boundary_state(UL, Ui, SL, gas, d)
            di = UL - Ui
            Ki = visc(Ui, outer(di, SL))
            F_far = ph.normal_convective_flux(UG, SL, gas, d) - ndot(visc(Ui, QL), SL) \
                + (tau / sJL).unsqueeze(1) * ndot(Ki, SL)
            Fhat = torch.where(is_far[:, None], F_far, Fhat)
            H = torch.where(is_far[:, None, None], Ki, H)
        elif bool(is_far.any()):
            raise ValueError("farfield faces need U_inf")
        return self._unflat(Fhat, E), self._unflatH(H, E)

    def adjoint_term(self, H):
        """(1/(w_q J_q)) sum_faces sum_f w_f grad l_q(x_f) . H(f) at every node
        ([E][nf][n..]), with grad l_q(x_f) = sum_a (Ja_f[a][c] / J_f) d l_q / d xi_a."""
        d, n, E, nf = self.d, self.n, self.E, self.nf
        b = self.basis
        w = torch.as_tensor(b.w)
        dl = [b.dlm, b.dlp]                                                 # l_j'(-1), l_j'(+1)
        out = torch.zeros((E, nf) + (n,) * d, dtype=H.dtype)
        JaF, JF = self.JaF.to(H.dtype), self.JF.to(H.dtype)
        D = torch.as_tensor(b.D)
        for a0 in range(d):
            wf = self._face_weights(w, a0)
            for side in (0, 1):
                fidx = 2 * a0 + side
                Hf = H[:, fidx]                                              # [E][c][nf][nfp]
                ax = 2 + d - 1 - a0                                          # node axis of a0
                lvec = torch.as_tensor(b.lp if side else b.lm, dtype=H.dtype)
                dvec = torch.as_tensor(dl[side], dtype=H.dtype)
                shape = [1] * (2 + d)
                shape[ax] = n
                for a in range(d):
                    Ht = sum(JaF[:, fidx, a, c].unsqueeze(1) * Hf[:, c] for c in range(d)) / JF[:, fidx].unsqueeze(1)
                    X = (Ht * wf).reshape((E, nf) + (n,) * (d - 1)).unsqueeze(ax)     # size 1 along a0
                    if a == a0:
                        out = out + X * dvec.reshape(shape)
                    else:
                        Y = along(X, a, d, D.T)                            # sum_m D[m][q_a] X(m)
                        out = out + Y * lvec.reshape(shape)
        Wn = self._node_weights(w)
        return out / (Wn * self.geo.J.to(H.dtype)).unsqueeze(1)

    # -------------------------------------------------------------- operator
    def residual(self, U, U_im=None, return_parts=False):
        """f(U) = dU/dt on every element; with an explicit-element mask, the
        explicit elements read U, the implicit ones U_im, and f is returned on
        the explicit elements (zero on the implicit ones)."""
        d, nf, E = self.d, self.nf, self.E
        Ue = self._states(U, U_im)
        Un = self.nodes(Ue)
        Q, TQ = self.gradients(Un)
        TU = self.element_traces(Un)
        Fhat, H = self.face_terms(TU, TQ)
        flatU = Un.permute(0, *range(2, 2 + d), 1).reshape(-1, nf)
        F = ph.convective_flux(flatU, self.gas, d)
        if self.gas.viscous:
            Qflat = Q.permute(0, *range(3, 3 + d), 1, 2).reshape(-1, d, nf)
            F = F - ph.viscous_flux(flatU, Qflat, self.gas, d)
        F = F.reshape((E,) + (self.n,) * d + (d, nf)).permute(0, 1 + d, 2 + d, *range(1, 1 + d))
        J = self.geo.J.to(Ue.dtype)
        Ja = self.geo.Ja.to(Ue.dtype)
        vol = 0
        for a in range(d):
            Ft = sum(Ja[:, a, c].unsqueeze(1) * F[:, c] for c in range(d))
            vol = vol + along(Ft, a, d, self.Dhat)
        f = vol / J.unsqueeze(1) + self.lift(Fhat, J, sign=-1.0)
        if self.gas.viscous:
            f = f + self.adjoint_term(H)
        f = f.reshape(E, nf, -1)
        if self.explicit is not None:
            f = torch.where(self.explicit[:, None, None], f, torch.zeros_like(f))
        if return_parts:
            return f, {"Fhat": Fhat, "H": H, "Q": Q, "TU": TU}
        return f



def over_integration_points(p):
    """M = ceil((3k + 1) / 2) Gauss points per direction: exact for degree 3k (Sec. 5)."""
    return (3 * p + 2) // 2


class OverIntegratedSIPG:
    """The DG-IP operator with its volume and face integrals taken by the
    M-point Gauss rule per direction (Sec. 5: the nonlinear terms are
    integrated by a rule of order 3k, M = ceil((3k+1)/2) by default) on the
    degree-k solution space; the mass matrix is the Gauss-node one (exact on
    boxes, the collocated w_q J_q on curved elements, as in the collocated
    operator).

    Written through an identity.  Every degree-k test function l_q lies in
    the degree-(M-1) Lagrange space of the M Gauss points,
    l_q = sum_r l_q(z_r) L_r, and the weak form is linear in the test
    function, so the over-integrated form tested with l_q is
    sum_r l_q(z_r) B'_r, where B'_r is the collocated degree-(M-1) form of
    the same polynomial state tested with L_r: collocation at the M points
    is exactly the M-point rule, and the state's values, traces and
    gradients there are those of the degree-k polynomial.  The element map
    is the degree-k interpolant of the node coordinates; at the M points it
    is represented exactly by the interpolated coordinates, from which the
    degree-(M-1) operator takes J', its metric terms and normals.  With
    B'_r = -omega_r J'_r f'_r and the collocated mass w_q J_q this gives

        f = J^-1 Pi (J' f'(I U)),

    I interpolating U to the M points (I[m][j] = l_j(z_m)), f' the
    collocated DG-IP operator there with the penalty of the true degree,
    tau = alpha (k+1)^2 / l, and Pi[q][m] = omega_m l_q(z_m) / w_q
    projecting back; on boxes J' = J and f = Pi f'(I U).  Pinned by
    ``brute.BruteSIPG.residual_sipg_oi`` (affine elements: every integrand
    evaluated pointwise at the M-point rule instead), and on curved
    elements by conservation (sum_q w_q J_q f_q = 0 on a periodic mesh),
    free-stream preservation and the manufactured-solution rate.
    """

    def __init__(self, mesh, gas, alpha=1.0, U_inf=None, explicit=None, M=None):
        import dataclasses
        from .basis import Basis1D, gauss_legendre, lagrange_eval
        from .geometry import Geometry
        self.mesh, self.gas, self.p = mesh, gas, mesh.p
        self.d = d = mesh.dim
        self.n = n = mesh.p + 1
        self.M = M = over_integration_points(mesh.p) if M is None else int(M)
        if M < n:
            raise ValueError("the rule needs at least p + 1 points")
        x, w = (np.asarray(v) for v in gauss_legendre(n))
        z, om = (np.asarray(v) for v in gauss_legendre(M))
        self.I = torch.as_tensor(lagrange_eval(x, z))                           # [M][n]
        self.Pi = torch.as_tensor(om[None, :] * lagrange_eval(x, z).T / w[:, None])  # [n][M]
        if mesh.kind == "boxes":
            qi = [(np.arange(M ** d) // M ** a) % M for a in range(d)]         # direction a: stride M^a
            xyz = np.empty((mesh.n_elem, d, M ** d))
            for a in range(d):
                xyz[:, a, :] = mesh.lo[:, a:a + 1] + 0.5 * (1.0 + z[qi[a]])[None, :] * mesh.size[:, a:a + 1]
        else:   # the degree-k element map at the M points
            xyz = self._apply(torch.as_tensor(mesh.xyz, dtype=torch.float64), self.I, n, M).numpy()
        self.mesh_q = dataclasses.replace(mesh, p=M - 1, xyz=xyz)
        self.inner = SIPGOperator(self.mesh_q, gas, alpha=alpha, U_inf=U_inf, explicit=explicit,
                                  k_penalty=mesh.p)
        E = mesh.n_elem
        self.J = self.Jq = None                                                # boxes: J' = J cancels
        if mesh.kind != "boxes":
            self.J = Geometry(mesh, Basis1D(mesh.p)).J.reshape(E, 1, -1)       # at the nodes
            self.Jq = self.inner.geo.J.reshape(E, 1, -1)                       # at the M points

    def _apply(self, V, Mat, m_in, m_out):
        """Mat ([m_out][m_in]) applied along every reference direction."""
        d = self.d
        k, c = V.shape[:2]
        X = V.reshape((k, c) + (m_in,) * d)
        for a in range(d):
            X = along(X, a, d, Mat.to(V.dtype))
        return X.reshape(k, c, m_out ** d)

    def interpolate(self, U):
        return self._apply(torch.as_tensor(U), self.I, self.n, self.M)

    def project(self, F):
        return self._apply(torch.as_tensor(F), self.Pi, self.M, self.n)

    def residual(self, U, U_im=None):
        Uq = self.interpolate(U)
        Uimq = None if U_im is None else self.interpolate(U_im)
        Fq = self.inner.residual(Uq, Uimq)
        if self.J is None:
            return self.project(Fq)
        return self.project(self.Jq * Fq) / self.J
