"""Dense brute-force evaluation of the DG weak form on tiny affine meshes.

Test infrastructure only; its sole job is to pin ``residual``.  It shares the
pointwise physics (``physics``: fluxes, LLF, wall states, which the tests pin
separately against closed forms) but none of the discretisation code: it
builds its own Lagrange polynomials (numpy.polynomial, nodes from numpy's
Gauss-Legendre routine), fits each element's affine map from its node
coordinates, integrates every term of the weak form (Sec. 3.3: volume term
(F^nu - F^c) : grad V, surface numerical flux, BR1 lifting, mass matrix) with
an independent higher-order Gauss rule, finds the neighbour's value at each
face point by locating that physical point inside the neighbour (ignoring the
nbr_face / orient tables), and solves with the dense mass matrix.

On affine elements every integrand is a polynomial the higher-order rule
integrates exactly, and the collocated scheme's Gauss-node quadrature is exact
for the same integrands, so the two must agree to rounding.
"""
import itertools

import numpy as np
import torch
from numpy.polynomial import Polynomial

from . import physics as ph


class _Lagrange:
    def __init__(self, n):
        self.x, _ = np.polynomial.legendre.leggauss(n)
        self.l = []
        for j in range(n):
            others = [self.x[k] for k in range(n) if k != j]
            poly = Polynomial.fromroots(others)
            self.l.append(poly / poly(self.x[j]))
        self.dl = [lj.deriv() for lj in self.l]

    def val(self, t):
        return np.array([lj(t) for lj in self.l])

    def der(self, t):
        return np.array([lj(t) for lj in self.dl])


def _t(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float64))


class BruteDG:
    def __init__(self, mesh, gas, period=None):
        self.mesh, self.gas = mesh, gas
        self.d = d = mesh.dim
        self.n = n = mesh.p + 1
        self.N = n ** d
        self.nf = d + 2
        self.L = _Lagrange(n)
        self.xq, self.wq = np.polynomial.legendre.leggauss(n + 3)
        self.multi = [tuple((q // n ** a) % n for a in range(d)) for q in range(self.N)]
        self.period = period
        # affine maps x = x0 + A xi fitted from the node coordinates
        self.x0, self.A = [], []
        xi = self.L.x
        design = np.array([[1.0] + [xi[m[a]] for a in range(d)] for m in self.multi])
        for e in range(mesh.n_elem):
            coef, *_ = np.linalg.lstsq(design, mesh.xyz[e].T, rcond=None)
            self.x0.append(coef[0])
            self.A.append(coef[1:].T)          # A[c][a] = dx_c / dxi_a

    # ---- polynomial evaluation of nodal data of element e at a reference point
    def basis_at(self, xi):
        vals = [self.L.val(xi[a]) for a in range(self.d)]
        ders = [self.L.der(xi[a]) for a in range(self.d)]
        phi = np.array([np.prod([vals[a][m[a]] for a in range(self.d)]) for m in self.multi])
        grad = np.array([[np.prod([(ders if b == a else vals)[b][m[b]] for b in range(self.d)])
                          for a in range(self.d)] for m in self.multi])      # [N][a] d/dxi_a
        return phi, grad

    def locate(self, e, x):
        """Reference coordinates of physical point x in element e (with periodic images)."""
        Ainv = np.linalg.inv(self.A[e])
        shifts = [np.zeros(self.d)]
        if self.period is not None:
            shifts = [np.array(s) * np.array(self.period)
                      for s in itertools.product([-1, 0, 1], repeat=self.d)]
        best = None
        for s in shifts:
            xi = Ainv @ (x + s - self.x0[e])
            err = np.max(np.abs(xi)) - 1.0
            if best is None or err < best[0]:
                best = (err, xi)
        assert best[0] < 1e-9, "face point not found in neighbour"
        return best[1]

    def face_points(self, a, side):
        rest = [b for b in range(self.d) if b != a]
        pts = []
        for idx in itertools.product(range(self.n), repeat=self.d - 1):
            xi = np.zeros(self.d)
            xi[a] = -1.0 if side == 0 else 1.0
            for k, b in enumerate(rest):
                xi[b] = self.L.x[idx[k]]
            pts.append((xi, idx))
        return pts, rest

    def normal(self, e, a, side):
        J = np.linalg.det(self.A[e])
        Ainv = np.linalg.inv(self.A[e])
        v = J * Ainv[a, :]                    # J grad xi_a
        return v if side == 1 else -v

    # ---- the operator
    def residual(self, U):
        d, n, N, nf = self.d, self.n, self.N, self.nf
        mesh, gas = self.mesh, self.gas
        E = mesh.n_elem
        U = np.asarray(U, dtype=np.float64)
        quad = list(itertools.product(range(len(self.xq)), repeat=d))
        qpts = [(np.array([self.xq[i[a]] for a in range(d)]), np.prod([self.wq[i[a]] for a in range(d)]))
                for i in quad]
        # mass matrices (dense, exact) and basis tables at quadrature points
        tab = [self.basis_at(x) for x, _ in qpts]
        mass, Ainvs, Js = [], [], []
        for e in range(E):
            J = abs(np.linalg.det(self.A[e]))
            Ainv = np.linalg.inv(self.A[e])
            M = sum(w * np.outer(phi, phi) for (x, w), (phi, _) in zip(qpts, tab)) * J
            mass.append(M)
            Ainvs.append(Ainv)
            Js.append(J)

        def eval_at(e, V, xi):                  # V[c][N] nodal data of element e
            phi, _ = self.basis_at(xi)
            return V @ phi

        def face_rhs(e, a, side, values):       # sum over face points of values * l_q * face weight
            pts, rest = self.face_points(a, side)
            # integrate the face interpolant of ``values`` against l_q with the high rule
            out = np.zeros((values.shape[1], N))
            for iq in itertools.product(range(len(self.xq)), repeat=d - 1):
                xi = np.zeros(d)
                xi[a] = -1.0 if side == 0 else 1.0
                wt = 1.0
                face_phi = np.ones(len(pts))
                for k, b in enumerate(rest):
                    xi[b] = self.xq[iq[k]]
                    wt *= self.wq[iq[k]]
                for m, (_, idx) in enumerate(pts):
                    face_phi[m] = np.prod([self.L.val(xi[b])[idx[k]] for k, b in enumerate(rest)])
                phi, _ = self.basis_at(xi)
                val = values.T @ face_phi         # [c]
                out += wt * np.outer(val, phi)
            return out

        def neighbour_value(e, a, side, xi, V):
            f = 2 * a + side
            nb = mesh.neighbor[e, f]
            x = self.x0[e] + self.A[e] @ xi
            xin = self.locate(nb, x)
            return nb, xin, eval_at(nb, V[nb], xin)

        def wall(e, f):
            return mesh.neighbor[e, f] < 0

        # BR1 gradient, by projection
        Q = np.zeros((E, d, nf, N))
        if gas.viscous:
            for e in range(E):
                rhs = np.zeros((d, nf, N))
                for (x, w), (phi, gref) in zip(qpts, tab):
                    gx = gref @ self.Ainv_T(Ainvs[e])       # [N][c] d l_r / d x_c
                    gradU = U[e] @ gx                       # [nf][c]
                    for c in range(d):
                        rhs[c] += w * Js[e] * np.outer(gradU[:, c], phi)
                for a in range(d):
                    for side in (0, 1):
                        pts, _ = self.face_points(a, side)
                        Sn = self.normal(e, a, side)
                        jump = np.zeros((len(pts), nf))
                        for m, (xi, _) in enumerate(pts):
                            Um = eval_at(e, U[e], xi)
                            if wall(e, 2 * a + side):
                                Uhat = ph.wall_state(_t(Um[None]), d).numpy()[0]
                            else:
                                _, _, Up = neighbour_value(e, a, side, xi, U)
                                Uhat = 0.5 * (Um + Up)
                            jump[m] = Uhat - Um
                        for c in range(d):
                            rhs[c] += face_rhs(e, a, side, jump * Sn[c])
                for c in range(d):
                    Q[e, c] = np.linalg.solve(mass[e], rhs[c].T).T

        def visc_G(e, xi, Sn, at_wall):
            Uf = eval_at(e, U[e], xi)
            Qf = np.stack([eval_at(e, Q[e, c], xi) for c in range(d)])
            if at_wall:
                return ph.adiabatic_wall_viscous_flux(_t(Uf[None]), _t(Qf[None]), _t(Sn[None]), gas, d).numpy()[0]
            return ph.normal_viscous_flux(_t(Uf[None]), _t(Qf[None]), _t(Sn[None]), gas, d).numpy()[0]

        f_out = np.zeros((E, nf, N))
        for e in range(E):
            B = np.zeros((nf, N))
            # volume: - int (F^c - F^nu) : grad l_q
            for (x, w), (phi, gref) in zip(qpts, tab):
                gx = gref @ self.Ainv_T(Ainvs[e])           # [N][c]
                Un = U[e] @ phi                               # interpolated nodal flux below
                # interpolant of the nodal flux (collocation), evaluated at x
                Fn = ph.convective_flux(_t(U[e].T), gas, d).numpy()       # [N][i][nf]
                if gas.viscous:
                    Fn = Fn - ph.viscous_flux(_t(U[e].T), _t(Q[e].transpose(2, 0, 1)), gas, d).numpy()
                Fx = np.einsum("r,rif->if", phi, Fn)
                B -= w * Js[e] * np.einsum("if,qi->fq", Fx, gx)
            # surface
            for a in range(d):
                for side in (0, 1):
                    f_id = 2 * a + side
                    pts, _ = self.face_points(a, side)
                    Sn = self.normal(e, a, side)
                    vals = np.zeros((len(pts), nf))
                    for m, (xi, _) in enumerate(pts):
                        Um = eval_at(e, U[e], xi)
                        if wall(e, f_id):
                            Up = ph.mirror_state(_t(Um[None]), _t(Sn[None]), d).numpy()[0]
                        else:
                            nb, xin, Up = neighbour_value(e, a, side, xi, U)
                        Fc = ph.llf_flux(_t(Um[None]), _t(Up[None]), _t(Sn[None]), gas, d).numpy()[0]
                        Fv = 0.0
                        if gas.viscous:
                            if wall(e, f_id):
                                Fv = visc_G(e, xi, Sn, True)
                            else:
                                # neighbour's own outward normal at the shared face
                                an = int(np.argmax(np.abs(xin)))
                                sn = 1 if xin[an] > 0 else 0
                                Snb = self.normal(nb, an, sn)
                                Gm = visc_G(e, xi, Sn, False)
                                Gp = visc_G(nb, xin, Snb, False)
                                Fv = 0.5 * (Gm - Gp)
                        vals[m] = Fc - Fv
                    B += face_rhs(e, a, side, vals)
            f_out[e] = -np.linalg.solve(mass[e], B.T).T
        return f_out

    @staticmethod
    def Ainv_T(Ainv):
        # d l / d x_c = sum_a d l / d xi_a * d xi_a / d x_c = gref @ Ainv
        return Ainv


class BruteSIPG(BruteDG):
    """Dense brute-force evaluation of the DG-IP weak form of Sec. 3.3 (the
    Vijayasundaram flux + symmetric interior penalty, with the farfield and
    adiabatic-wall forms of App. B.1 and the explicit side of the interface
    form of Sec. 4.1.1) on tiny affine meshes; pins ``sipg``.

    Independent of ``sipg``'s discretisation code: its own Lagrange
    polynomials, the gradient of each element's polynomial evaluated from
    them at any point (no traces of metric terms), the characteristic length
    from the affine map (|T| = |det A| 2^d, |dT| = sum |Sn| 2^(d-1)), the
    neighbour's value found by locating the physical point, every face term
    -- including the adjoint-consistency term int grad l_q . H ds -- integrated
    against the basis (and its gradient) with a higher-order rule, and the
    dense mass matrix.  Pointwise quantities are collocated at the Gauss
    nodes (volume) and the face Gauss points (faces) and interpolated, as in
    the collocated scheme; shared with ``sipg``: only the pointwise physics.
    """

    def residual_sipg(self, U, alpha=1.0, U_inf=None, explicit=None, U_im=None):
        d, n, N, nf = self.d, self.n, self.N, self.nf
        mesh, gas = self.mesh, self.gas
        E = mesh.n_elem
        U = np.asarray(U, dtype=np.float64)
        if explicit is not None:
            U = np.where(np.asarray(explicit, dtype=bool)[:, None, None], U, np.asarray(U_im, dtype=np.float64))
        quad = list(itertools.product(range(len(self.xq)), repeat=d))
        qpts = [(np.array([self.xq[i[a]] for a in range(d)]), np.prod([self.wq[i[a]] for a in range(d)]))
                for i in quad]
        tab = [self.basis_at(x) for x, _ in qpts]
        Ainvs = [np.linalg.inv(self.A[e]) for e in range(E)]
        Js = [abs(np.linalg.det(self.A[e])) for e in range(E)]
        mass = [sum(w * np.outer(phi, phi) for (x, w), (phi, _) in zip(qpts, tab)) * Js[e] for e in range(E)]
        nodes_ref = [np.array([self.L.x[m[a]] for a in range(d)]) for m in self.multi]

        def value(e, xi):
            phi, _ = self.basis_at(xi)
            return U[e] @ phi

        def grad(e, xi):                          # [nf][c] gradient of the element's polynomial
            _, gref = self.basis_at(xi)
            return U[e] @ (gref @ Ainvs[e])

        # characteristic lengths from the affine maps
        inv_l = np.zeros(E)
        for e in range(E):
            area = sum(np.linalg.norm(self.normal(e, a, s)) * 2.0 ** (d - 1) for a in range(d) for s in (0, 1))
            inv_l[e] = area / (Js[e] * 2.0 ** d)
        ex = np.ones(E, dtype=bool) if explicit is None else np.asarray(explicit, dtype=bool)

        def T(x):
            return _t(np.asarray(x)[None])

        def visc(Uf, G, Sn=None, wall=False):
            if wall:
                return ph.adiabatic_viscous_flux(T(Uf), T(G), T(Sn), gas, d).numpy()[0]
            return ph.viscous_flux(T(Uf), T(G), gas, d).numpy()[0]      # [i][nf]

        def outer(delta, Sn):
            return np.outer(Sn, delta)                                    # [i][nf]

        f_out = np.zeros((E, nf, N))
        for e in range(E):
            if not ex[e]:
                continue
            B = np.zeros((nf, N))
            # volume: - int (F^c - F^nu(U, grad U)) : grad l_q, nodal fluxes interpolated
            Fn = np.zeros((N, d, nf))
            for r in range(N):
                Ur = U[e][:, r]
                Fr = ph.convective_flux(T(Ur), gas, d).numpy()[0]
                if gas.viscous:
                    Fr = Fr - visc(Ur, grad(e, nodes_ref[r]).T)
                Fn[r] = Fr
            for (x, w), (phi, gref) in zip(qpts, tab):
                gx = gref @ Ainvs[e]
                Fx = np.einsum("r,rif->if", phi, Fn)
                B -= w * Js[e] * np.einsum("if,qi->fq", Fx, gx)
            for a in range(d):
                for side in (0, 1):
                    fid = 2 * a + side
                    pts, rest = self.face_points(a, side)
                    Sn = self.normal(e, a, side)
                    nbe = mesh.neighbor[e, fid]
                    vals = np.zeros((len(pts), nf))
                    hv = np.zeros((len(pts), d, nf))
                    for m, (xi, _) in enumerate(pts):
                        Um = value(e, xi)
                        Gm = grad(e, xi).T                                   # [c][nf]
                        if nbe >= 0:
                            nb, xin, Up = neighbour_value(self, e, a, side, xi, U, value)
                            Gp = grad(nb, xin).T
                            an = int(np.argmax(np.abs(xin)))
                            Snb = self.normal(nb, an, 1 if xin[an] > 0 else 0)
                            Sb = 0.5 * (Sn - Snb)
                            sJ = np.linalg.norm(Sb)
                            tau = alpha * (mesh.p + 1) ** 2 * max(inv_l[e], inv_l[nb])
                            F = ph.vijayasundaram_flux(T(Um), T(Up), T(Sb), gas, d).numpy()[0]
                            dl = Um - Up
                            KL, KR = visc(Um, outer(dl, Sb)), visc(Up, outer(dl, Sb))
                            F = F - 0.5 * (visc(Um, Gm).T @ Sn - visc(Up, Gp).T @ Snb) \
                                + tau / sJ * 0.5 * (KL + KR).T @ Sb
                            hv[m] = 0.5 * (KL + KR) if not ex[nb] else 0.5 * KL
                        elif nbe == -1:                                       # adiabatic wall
                            tau = alpha * (mesh.p + 1) ** 2 * inv_l[e]
                            sJ = np.linalg.norm(Sn)
                            Ur = ph.mirror_state(T(Um), T(Sn), d).numpy()[0]
                            Uw = ph.wall_state(T(Um), d).numpy()[0]
                            Kw = visc(Um, outer(Um - Uw, Sn), Sn, True)
                            F = ph.vijayasundaram_flux(T(Um), T(Ur), T(Sn), gas, d).numpy()[0] \
                                - visc(Um, Gm, Sn, True).T @ Sn + tau / sJ * Kw.T @ Sn
                            hv[m] = Kw
                        else:                                                 # farfield
                            tau = alpha * (mesh.p + 1) ** 2 * inv_l[e]
                            sJ = np.linalg.norm(Sn)
                            Ui = np.asarray(U_inf, dtype=np.float64)
                            UG = ph.farfield_boundary_state(T(Um), T(Ui), T(Sn), gas, d).numpy()[0]
                            Ki = visc(Ui, outer(Um - Ui, Sn))
                            F = ph.normal_convective_flux(T(UG), T(Sn), gas, d).numpy()[0] \
                                - visc(Ui, Gm).T @ Sn + tau / sJ * Ki.T @ Sn
                            hv[m] = Ki
                        vals[m] = F
                    B += self._face_integral(e, a, side, pts, rest, vals, None)
                    if gas.viscous:
                        B -= self._face_integral(e, a, side, pts, rest, None, hv, Ainvs[e])
            f_out[e] = -np.linalg.solve(mass[e], B.T).T
        return f_out

    def residual_sipg_oi(self, U, M, alpha=1.0, U_inf=None, explicit=None, U_im=None):
        """The DG-IP weak form with every volume and face integrand evaluated
        pointwise (the degree-k state, its gradient and the fluxes at each
        point of the rule) and integrated by the M-point Gauss rule per
        direction (Sec. 5: the rule of order 3k); exact dense mass matrix.
        Pins ``sipg.OverIntegratedSIPG`` (which goes through collocation at
        the M points instead)."""
        d, N, nf = self.d, self.N, self.nf
        mesh, gas = self.mesh, self.gas
        E = mesh.n_elem
        U = np.asarray(U, dtype=np.float64)
        if explicit is not None:
            U = np.where(np.asarray(explicit, dtype=bool)[:, None, None], U, np.asarray(U_im, dtype=np.float64))
        ex = np.ones(E, dtype=bool) if explicit is None else np.asarray(explicit, dtype=bool)
        z, wz = np.polynomial.legendre.leggauss(M)
        vol = [(np.array([z[i[a]] for a in range(d)]), np.prod([wz[i[a]] for a in range(d)]))
               for i in itertools.product(range(M), repeat=d)]
        exact = list(itertools.product(range(len(self.xq)), repeat=d))
        Ainvs = [np.linalg.inv(self.A[e]) for e in range(E)]
        Js = [abs(np.linalg.det(self.A[e])) for e in range(E)]
        mass = []
        for e in range(E):
            Mm = np.zeros((N, N))
            for i in exact:
                phi, _ = self.basis_at(np.array([self.xq[i[a]] for a in range(d)]))
                Mm += np.prod([self.wq[i[a]] for a in range(d)]) * np.outer(phi, phi)
            mass.append(Mm * Js[e])
        inv_l = np.zeros(E)
        for e in range(E):
            area = sum(np.linalg.norm(self.normal(e, a, s)) * 2.0 ** (d - 1) for a in range(d) for s in (0, 1))
            inv_l[e] = area / (Js[e] * 2.0 ** d)

        def value(e, xi):
            phi, _ = self.basis_at(xi)
            return U[e] @ phi

        def grad(e, xi):                                  # [c][nf]
            _, gref = self.basis_at(xi)
            return (U[e] @ (gref @ Ainvs[e])).T

        def T(x):
            return _t(np.asarray(x)[None])

        def visc(Uf, G, Sn=None, wall=False):
            if wall:
                return ph.adiabatic_viscous_flux(T(Uf), T(G), T(Sn), gas, d).numpy()[0]
            return ph.viscous_flux(T(Uf), T(G), gas, d).numpy()[0]

        tk2 = alpha * (mesh.p + 1) ** 2
        f_out = np.zeros((E, nf, N))
        for e in range(E):
            if not ex[e]:
                continue
            B = np.zeros((nf, N))
            for x, w in vol:                              # - int (F^c - F^nu) : grad l_q
                phi, gref = self.basis_at(x)
                Ux = U[e] @ phi
                Fx = ph.convective_flux(T(Ux), gas, d).numpy()[0]
                if gas.viscous:
                    Fx = Fx - visc(Ux, grad(e, x))
                B -= w * Js[e] * np.einsum("if,qi->fq", Fx, gref @ Ainvs[e])
            for a in range(d):
                rest = [b for b in range(d) if b != a]
                for side in (0, 1):
                    Sn = self.normal(e, a, side)
                    nbe = mesh.neighbor[e, 2 * a + side]
                    for iq in itertools.product(range(M), repeat=d - 1):
                        xi = np.zeros(d)
                        xi[a] = 1.0 if side else -1.0
                        wt = 1.0
                        for k, b in enumerate(rest):
                            xi[b] = z[iq[k]]
                            wt *= wz[iq[k]]
                        Um, Gm = value(e, xi), grad(e, xi)
                        if nbe >= 0:
                            nb, xin, Up = neighbour_value(self, e, a, side, xi, U, value)
                            Gp = grad(nb, xin)
                            an = int(np.argmax(np.abs(xin)))
                            Snb = self.normal(nb, an, 1 if xin[an] > 0 else 0)
                            Sb = 0.5 * (Sn - Snb)
                            tau = tk2 * max(inv_l[e], inv_l[nb])
                            F = ph.vijayasundaram_flux(T(Um), T(Up), T(Sb), gas, d).numpy()[0]
                            if gas.viscous:
                                dl = np.outer(Sb, Um - Up)
                                KL, KR = visc(Um, dl), visc(Up, dl)
                                F = F - 0.5 * (visc(Um, Gm).T @ Sn - visc(Up, Gp).T @ Snb) \
                                    + tau / np.linalg.norm(Sb) * 0.5 * (KL + KR).T @ Sb
                                H = 0.5 * KL if ex[nb] else 0.5 * (KL + KR)
                        elif nbe == -1:                   # adiabatic wall
                            Ur = ph.mirror_state(T(Um), T(Sn), d).numpy()[0]
                            F = ph.vijayasundaram_flux(T(Um), T(Ur), T(Sn), gas, d).numpy()[0]
                            if gas.viscous:
                                tau = tk2 * inv_l[e]
                                Uw = ph.wall_state(T(Um), d).numpy()[0]
                                H = visc(Um, np.outer(Sn, Um - Uw), Sn, True)
                                F = F - visc(Um, Gm, Sn, True).T @ Sn + tau / np.linalg.norm(Sn) * H.T @ Sn
                        else:                             # farfield
                            Ui = np.asarray(U_inf, dtype=np.float64)
                            UG = ph.farfield_boundary_state(T(Um), T(Ui), T(Sn), gas, d).numpy()[0]
                            F = ph.normal_convective_flux(T(UG), T(Sn), gas, d).numpy()[0]
                            if gas.viscous:
                                tau = tk2 * inv_l[e]
                                H = visc(Ui, np.outer(Sn, Um - Ui))
                                F = F - visc(Ui, Gm).T @ Sn + tau / np.linalg.norm(Sn) * H.T @ Sn
                        phi, gref = self.basis_at(xi)
                        B += wt * np.outer(F, phi)
                        if gas.viscous:                   # - int grad l_q . H
                            B -= wt * np.einsum("cf,qc->fq", H, gref @ Ainvs[e])
            f_out[e] = -np.linalg.solve(mass[e], B.T).T
        return f_out

    def _face_integral(self, e, a, side, pts, rest, vals, hv, Ainv=None):
        """int_F (face interpolant of vals) l_q ds, or int_F grad l_q . (face
        interpolant of hv) ds, with the higher rule on the reference face (the
        area factor is inside vals / hv, which carry the area normal)."""
        d, N = self.d, self.N
        nf = self.nf
        out = np.zeros((nf, N))
        for iq in itertools.product(range(len(self.xq)), repeat=d - 1):
            xi = np.zeros(d)
            xi[a] = -1.0 if side == 0 else 1.0
            wt = 1.0
            for k, b in enumerate(rest):
                xi[b] = self.xq[iq[k]]
                wt *= self.wq[iq[k]]
            face_phi = np.array([np.prod([self.L.val(xi[b])[idx[k]] for k, b in enumerate(rest)])
                                 for (_, idx) in pts])
            phi, gref = self.basis_at(xi)
            if vals is not None:
                out += wt * np.outer(vals.T @ face_phi, phi)
            else:
                Hx = np.einsum("m,mcf->cf", face_phi, hv)            # [c][nf]
                gx = gref @ Ainv                                     # [N][c]
                out += wt * np.einsum("cf,qc->fq", Hx, gx)
        return out


def neighbour_value(brute, e, a, side, xi, U, value):
    nb = brute.mesh.neighbor[e, 2 * a + side]
    x = brute.x0[e] + brute.A[e] @ xi
    xin = brute.locate(nb, x)
    return nb, xin, value(nb, xin)


class BruteHDG(BruteSIPG):
    """Dense brute-force evaluation of the HDG-IP element and facet forms of
    Sec. 3.4 (App. B.2 on boundaries) on tiny affine meshes; pins ``hdg``.
    Independent of ``hdg``/``sipg``: its own Lagrange polynomials and
    quadrature (as ``BruteSIPG``), and the flux split A_n^{+-}(Uhat) from a
    numerical eigen-decomposition of the Jacobian obtained by differentiating
    the normal flux (not from the closed-form eigenvectors).  Returns the
    element residual (the form tested with each nodal basis function, before
    any mass inverse) and the facet residual (tested with each face-point
    basis function), in ``hdg``'s layouts.  |A| is the principal square root
    of A^2 (Schur-based ``scipy.linalg.sqrtm``; A has real eigenvalues and is
    diagonalisable), A^{+-} = (A +- |A|)/2."""

    def _split(self, Uh, Sn):
        import scipy.linalg
        d = self.d
        f = lambda u: ph.normal_convective_flux(u[None], _t(Sn[None]), self.gas, d)[0]
        A = torch.autograd.functional.jacobian(f, _t(Uh)).numpy()
        absA = np.real(scipy.linalg.sqrtm(A @ A))
        return 0.5 * (A + absA), 0.5 * (A - absA)

    def residual_hdg(self, U, Uhat, alpha=10.0, U_inf=None):
        d, n, N, nf = self.d, self.n, self.N, self.nf
        mesh, gas = self.mesh, self.gas
        E = mesh.n_elem
        nfp = n ** (d - 1)
        U = np.asarray(U, dtype=np.float64)
        Uhat = np.asarray(Uhat, dtype=np.float64)
        quad = list(itertools.product(range(len(self.xq)), repeat=d))
        qpts = [(np.array([self.xq[i[a]] for a in range(d)]), np.prod([self.wq[i[a]] for a in range(d)]))
                for i in quad]
        tab = [self.basis_at(x) for x, _ in qpts]
        Ainvs = [np.linalg.inv(self.A[e]) for e in range(E)]
        Js = [abs(np.linalg.det(self.A[e])) for e in range(E)]
        nodes_ref = [np.array([self.L.x[m[a]] for a in range(d)]) for m in self.multi]
        _, wg = np.polynomial.legendre.leggauss(n)
        gw = ph.Gas(gas.gamma, Re=1.0 / gas.mu if gas.mu > 0 else 0.0, Pr=gas.Pr, viscous=gas.viscous)
        gw.k_over_cv = 0.0

        def T(x):
            return _t(np.asarray(x)[None])

        def visc(Uf, G, g):
            return ph.viscous_flux(T(Uf), T(G), g, d).numpy()[0]

        R = np.zeros((E, nf, N))
        H = np.zeros((E, 2 * d, nf, nfp))
        for e in range(E):
            B = np.zeros((nf, N))
            Fn = np.zeros((N, d, nf))
            for r in range(N):
                Ur = U[e][:, r]
                _, gref = self.basis_at(nodes_ref[r])
                Fr = ph.convective_flux(T(Ur), gas, d).numpy()[0]
                if gas.viscous:
                    Fr = Fr - visc(Ur, (U[e] @ (gref @ Ainvs[e])).T, gas)
                Fn[r] = Fr
            for (x, w), (phi, gref) in zip(qpts, tab):
                gx = gref @ Ainvs[e]
                B -= w * Js[e] * np.einsum("if,qi->fq", np.einsum("r,rif->if", phi, Fn), gx)
            area = sum(np.linalg.norm(self.normal(e, a, s)) * 2.0 ** (d - 1) for a in range(d) for s in (0, 1))
            tau = alpha * (mesh.p + 1) ** 2 * area / (Js[e] * 2.0 ** d)
            for a in range(d):
                for side in (0, 1):
                    fid = 2 * a + side
                    pts, rest = self.face_points(a, side)
                    Sn = self.normal(e, a, side)
                    sJ = np.linalg.norm(Sn)
                    kind = mesh.neighbor[e, fid]
                    g = gw if kind == -1 else gas
                    vals = np.zeros((len(pts), nf))
                    hv = np.zeros((len(pts), d, nf))
                    for m, (xi, idx) in enumerate(pts):
                        # hdg's face-point index: the first remaining direction fastest
                        fp = sum(idx[k] * n ** k for k in range(d - 1))
                        Uh = Uhat[e, fid, :, fp]
                        phi, gref = self.basis_at(xi)
                        Um = U[e] @ phi
                        Gm = (U[e] @ (gref @ Ainvs[e])).T
                        Ap, Am = self._split(Uh, Sn)
                        dl = Um - Uh
                        Kd = visc(Uh, outer_(dl, Sn), g)
                        vals[m] = Ap @ Um + Am @ Uh - visc(Uh, Gm, g).T @ Sn + tau / sJ * Kd.T @ Sn
                        hv[m] = Kd
                        wf = np.prod([wg[i] for i in idx]) if d > 1 else 1.0
                        if kind == -1:
                            H[e, fid, :, fp] = wf * sJ * (Uh - ph.wall_state(T(Um), d).numpy()[0])
                        elif kind == -2:
                            Ui = np.asarray(U_inf, dtype=np.float64)
                            H[e, fid, :, fp] = wf * (Ap @ (Uh - Um) - Am @ (Uh - Ui))
                        else:
                            H[e, fid, :, fp] = -wf * vals[m]
                    B += self._face_integral(e, a, side, pts, rest, vals, None)
                    if gas.viscous:
                        B -= self._face_integral(e, a, side, pts, rest, None, hv, Ainvs[e])
            R[e] = B
        return R, H


def outer_(delta, Sn):
    return np.outer(Sn, delta)
