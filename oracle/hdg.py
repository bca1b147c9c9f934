"""Element-local HDG-IP forms and their static-condensation blocks (oracle;
test infrastructure only).

Follows Sec. 3.4 of the paper (HDG-IP: element form of Eq.
bilinear_form_interior_hdg_ip_element, facet transmission form of Eq.
bilinear_form_interior_hdg_ip_facet, HDG numerical flux of Eq.
inviscid_numerical_flux with S_c = A_n^+(Uhat), i.e.
Fhat*_n = A_n^+(Uhat) U + A_n^-(Uhat) Uhat), its boundary forms (App. B.2:
farfield transmission through the flux-vector split, adiabatic walls with K_w
in the element form and the Dirichlet condition Uhat = U_w on the facet), and
the Newton system of an SDIRK stage and its static condensation (Sec. 4.3,
Eq. implicit_system, statically_condensed_system, SchurCompliment,
local_solve_static_condensation) for HDG-IP (no mixed variables: Z = U).

Per element T, with U its nodal state, Uhat the facet state on its faces (in
the element's own face-point order) and the collocated Gauss rules:

  R_T(U, Uhat)[q] = B_I tested with l_q  (volume (F^nu - F^c) : grad l_q,
                     + Fhat*_n . l_q - K(Uhat) grad U : (l_q (x) n)
                     - K^T(Uhat) grad l_q : ((U - Uhat) (x) n)
                     + tau K(Uhat)((U - Uhat) (x) n) : (l_q (x) n) on every face;
                     K_w (no normal heat flux) on wall faces),
  h_T(U, Uhat)[j]  = the facet form tested with the facet basis at face point j:
                     interior:  -Fhat*_n + (K(Uhat) grad U - tau K(Uhat)((U - Uhat) (x) n)) n
                     farfield:  A_n^+(Uhat)(Uhat - U) - A_n^-(Uhat)(Uhat - U_inf)
                     wall:      Uhat - U_w(U)        (U_w the no-slip state of the trace)
  (each times the face quadrature weight and the area factor),

tau = alpha (k+1)^2 / l with alpha = 10 for HDG-IP and l = |T|/|dT| of the
element.  With these element residuals the stage equation of an SDIRK stage
reads M y + gamma R_T(y, yhat) = rhs (gamma = dt a_ii, M = diag(w_q J_q)), and
the element blocks of its Newton matrix are

  K = M + gamma dR/dU,  C = gamma dR/dUhat,  D = dh/dU,  A33_T = dh/dUhat,

the element's Schur contribution S_T = A33_T - D K^{-1} C and the local
recovery operator K^{-1} C.  The element residual is written with the DG-IP
operator's machinery (``sipg``): its face flux and adjoint-consistency
vector are the HDG ones, built from Uhat in place of the neighbour.
Readings: U_w on a wall facet is the no-slip state of the interior trace;
at lambda_k = 0 the flux split is that of ``physics.split_jacobian``.
"""
import numpy as np
import torch

from . import physics as ph
from .geometry import along
from .sipg import FARFIELD, WALL, SIPGOperator


class HDGIPLocal(SIPGOperator):
    def __init__(self, mesh, gas, alpha=10.0, U_inf=None):
        super().__init__(mesh, gas, alpha=alpha, U_inf=U_inf)
        # HDG: the penalty of a face is its own element's (no neighbour in the form)
        k = mesh.p
        self.tau = self.alpha * (k + 1) ** 2 * self.inv_l[:, None].expand(-1, 2 * self.d).clone()

    def hdg_flux(self, U, Uh, Sn):
        """Fhat*_n = A_n^+(Uhat) U + A_n^-(Uhat) Uhat through the area normal Sn."""
        Ap, Am = ph.split_jacobian(Uh, Sn, self.gas, self.d)
        return (Ap @ U.unsqueeze(2)).squeeze(2) + (Am @ Uh.unsqueeze(2)).squeeze(2)

    def forms(self, U, Uhat):
        """(R [E][nf][N], h [E][2d][nf][nfp]) for nodal states U and facet states Uhat."""
        d, nf, E = self.d, self.nf, self.E
        gas = self.gas
        Un = self.nodes(U)
        Q, TQ = self.gradients(Un)
        TU = self.element_traces(Un)
        Sn = self.geo.Sn.to(U.dtype)
        UL = self._faces_flat(TU)
        UH = self._faces_flat(Uhat)
        QL = self._flatQ(TQ)
        SL = self._flatS(Sn)
        sJ = torch.sqrt((SL * SL).sum(1))
        tau = self.tau.to(U.dtype)[:, :, None].expand(E, 2 * d, self.nfp).reshape(-1)
        kind = self.nb[:, :, None].expand(E, 2 * d, self.nfp).reshape(-1)
        wall = (kind == -(1 + WALL))[:, None]
        gw = ph.Gas(gas.gamma, Re=1.0 / gas.mu if gas.mu > 0 else 0.0, Pr=gas.Pr, viscous=gas.viscous)
        gw.k_over_cv = 0.0                                     # K_w: no normal heat flux (see sipg R17)

        def visc(Us, G, g):
            return ph.viscous_flux(Us, G, g, d)

        def ndot(F, S):
            return (F * S.unsqueeze(2)).sum(1)

        dl = UL - UH
        G = SL.unsqueeze(2) * dl.unsqueeze(1)                   # delta (x) Sn
        K_i, K_w = visc(UH, G, gas), visc(UH, G, gw)
        Kd = torch.where(wall[:, :, None], K_w, K_i)            # K(Uhat)(delta (x) Sn)
        V_i, V_w = visc(UH, QL, gas), visc(UH, QL, gw)
        Kg = torch.where(wall[:, :, None], V_w, V_i)            # K(Uhat) grad U
        Fs = self.hdg_flux(UL, UH, SL)
        Fhat = Fs - ndot(Kg, SL) + (tau / sJ).unsqueeze(1) * ndot(Kd, SL)
        H = Kd
        # facet residuals (times the face weight, applied below)
        h_int = -Fhat
        Uw = ph.wall_state(UL, d)
        h_wall = sJ.unsqueeze(1) * (UH - Uw)
        h = torch.where(wall, h_wall, h_int)
        if self.U_inf is not None:
            Ui = self.U_inf.to(U.dtype).expand_as(UL)
            Ap, Am = ph.split_jacobian(UH, SL, gas, d)
            h_far = (Ap @ (UH - UL).unsqueeze(2)).squeeze(2) - (Am @ (UH - Ui).unsqueeze(2)).squeeze(2)
            far = (kind == -(1 + FARFIELD))[:, None]
            h = torch.where(far, h_far, h)
        Fhat = self._unflat(Fhat, E)
        H = self._unflatH(H, E)
        h = self._unflat(h, E)
        w = torch.as_tensor(self.basis.w)
        for a0 in range(d):
            wf = self._face_weights(w, a0).to(U.dtype)
            h[:, 2 * a0:2 * a0 + 2] = h[:, 2 * a0:2 * a0 + 2] * wf
        # element residual: f as in the DG-IP operator, then R = -M f
        flatU = Un.permute(0, *range(2, 2 + d), 1).reshape(-1, nf)
        F = ph.convective_flux(flatU, gas, d)
        if gas.viscous:
            Qflat = Q.permute(0, *range(3, 3 + d), 1, 2).reshape(-1, d, nf)
            F = F - ph.viscous_flux(flatU, Qflat, gas, d)
        F = F.reshape((E,) + (self.n,) * d + (d, nf)).permute(0, 1 + d, 2 + d, *range(1, 1 + d))
        J = self.geo.J.to(U.dtype)
        Ja = self.geo.Ja.to(U.dtype)
        vol = 0
        for a in range(d):
            Ft = sum(Ja[:, a, c].unsqueeze(1) * F[:, c] for c in range(d))
            vol = vol + along(Ft, a, d, self.Dhat)
        f = vol / J.unsqueeze(1) + self.lift(Fhat, J, sign=-1.0)
        if gas.viscous:
            f = f + self.adjoint_term(H)
        Wn = self._node_weights(w).to(U.dtype)
        R = -(f * (Wn * J).unsqueeze(1)).reshape(E, nf, -1)
        return R, h

    def mass(self):
        """Diagonal of M per element: w_q J_q for every field, [E][nf][N]."""
        w = torch.as_tensor(self.basis.w)
        Wn = self._node_weights(w)
        MJ = (Wn * self.geo.J).reshape(self.E, 1, -1)
        return MJ.expand(self.E, self.nf, -1)

    def blocks(self, U, Uhat, gamma):
        """K, C, D, A33_T per element ([E][nu][nu], [E][nu][nh], [E][nh][nu],
        [E][nh][nh]; element DOFs in U's field-major order, facet DOFs in
        Uhat's [face][field][point] order), by differentiating ``forms``."""
        E = self.E
        nu = self.nf * self.n ** self.d
        nh = 2 * self.d * self.nf * self.nfp
        U = torch.as_tensor(U, dtype=torch.float64)
        Uhat = torch.as_tensor(Uhat, dtype=torch.float64)

        def fn(u, uh):
            R, h = self.forms(u.reshape(U.shape), uh.reshape(Uhat.shape))
            return R.reshape(E, nu), h.reshape(E, nh)

        JR_u = torch.autograd.functional.jacobian(lambda u: fn(u, Uhat.reshape(-1))[0], U.reshape(-1), vectorize=True)
        JR_h = torch.autograd.functional.jacobian(lambda uh: fn(U.reshape(-1), uh)[0], Uhat.reshape(-1), vectorize=True)
        Jh_u = torch.autograd.functional.jacobian(lambda u: fn(u, Uhat.reshape(-1))[1], U.reshape(-1), vectorize=True)
        Jh_h = torch.autograd.functional.jacobian(lambda uh: fn(U.reshape(-1), uh)[1], Uhat.reshape(-1), vectorize=True)
        # element-diagonal blocks: rows of element e against its own columns
        ar = torch.arange(E)
        JR_u = JR_u.reshape(E, nu, E, nu)[ar, :, ar]
        JR_h = JR_h.reshape(E, nu, E, nh)[ar, :, ar]
        Jh_u = Jh_u.reshape(E, nh, E, nu)[ar, :, ar]
        Jh_h = Jh_h.reshape(E, nh, E, nh)[ar, :, ar]
        M = torch.diag_embed(self.mass().reshape(E, nu))
        return M + gamma * JR_u, gamma * JR_h, Jh_u, Jh_h

    def schur(self, U, Uhat, gamma):
        """(K^{-1} C, S_T = A33_T - D K^{-1} C) per element."""
        K, C, D, A33 = self.blocks(U, Uhat, gamma)
        KinvC = torch.linalg.solve(K, C)
        return KinvC, A33 - D @ KinvC
