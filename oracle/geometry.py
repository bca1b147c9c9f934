"""Element geometry for the oracle (test infrastructure only).

Sec. 3.1 of the paper asks for shape-regular quadrilateral elements; the
collocated reading maps each element from [-1,1]^d by the degree-p
tensor-product interpolant x(xi) of its node coordinates.  Quantities:

* ``J``   -- det(dx/dxi) at every node.
* ``Ja``  -- Ja[b][c] = J * d(xi_b)/d(x_c) at every node (contravariant metric
             scaled by J).  2D: Ja_0 = (y_eta, -x_eta), Ja_1 = (-y_xi, x_xi).
             3D: the conservative curl form of Kopriva (2006),
             J a^i_n = -e_i . curl_xi( X_l grad_xi X_m ), (n, m, l) cyclic,
             with X_l grad_xi X_m replaced by its degree-p interpolant through
             the (p+1)^3 Gauss-Lobatto points (the map evaluated there) and the
             curl taken exactly; Ja is then a degree-p polynomial per
             direction, carried to the Gauss nodes exactly.  So the Gauss
             derivative matrices satisfy the metric identities
             sum_i D_i Ja_i = 0, and the trace of Ja_a on a face depends on the
             map's values at that face's Lobatto points only: both elements of
             a conforming face see the same area normal, and a uniform flow
             stays at rest on any curved mesh.  (Interpolating at the Gauss
             nodes instead also satisfies the identities, but its face traces
             extrapolate interior values and differ from side to side.)  X_l
             enters relative to the element's mean: the curl of c grad X_m
             vanishes identically (derivatives along different directions
             commute), and the offset only adds rounding.
* ``Sn``  -- area-weighted outward normal at every face point: +-Ja_a traced
             to the face xi_a = +-1 (s_J * n in the paper's notation).

Axis-aligned boxes (lower corner + edge lengths per element) take the exact
closed forms J = prod(h_a / 2) and Ja_a = e_a * prod_{b != a}(h_b / 2), so the
wall-adjacent 2e-5-thin layers never go through coordinate differences.

Array layout: node tensors carry the element axis first and the reference
directions reversed (``[..., i_{d-1}, ..., i_0]``), matching node index
q = i0 + n*i1 (+ n*n*i2).
"""
import numpy as np
import torch

from .basis import Basis1D, derivative_matrix, gauss_lobatto_points, lagrange_eval


def along(V, a, dim, M):
    """Apply the n x n matrix M along reference direction a of node tensor V.

    V has node axes as its last ``dim`` axes; direction a is axis -1-a.
    Returns W with W[.., i_a, ..] = sum_j M[i_a, j] V[.., j, ..].
    """
    ax = V.dim() - 1 - a
    Vt = torch.movedim(V, ax, -1)
    W = Vt @ M.T.to(V.dtype)
    return torch.movedim(W, -1, ax)


def trace(V, a, side, dim, basis):
    """Interpolate V along direction a to xi_a = -1 (side 0) or +1 (side 1).

    The result keeps the remaining node axes in their original order, so
    flattening them gives the face-point index s + n*t.
    """
    vec = torch.as_tensor(basis.lp if side else basis.lm, dtype=torch.float64).to(V.dtype)
    ax = V.dim() - 1 - a
    return torch.tensordot(V, vec, dims=([ax], [0]))


class Geometry:
    def __init__(self, mesh, basis: Basis1D):
        self.dim = d = mesh.dim
        self.n = n = basis.n
        self.E = E = mesh.n_elem
        self.basis = basis
        node_shape = (E,) + (n,) * d
        if mesh.kind == "boxes":
            h = torch.as_tensor(mesh.size, dtype=torch.float64)               # [E][d]
            half = 0.5 * h
            Jel = torch.prod(half, dim=1)                                      # [E]
            self.J = Jel.reshape((E,) + (1,) * d).expand(node_shape).clone()
            Ja = torch.zeros((E, d, d) + (n,) * d, dtype=torch.float64)
            for b in range(d):
                val = torch.ones(E, dtype=torch.float64)
                for c in range(d):
                    if c != b:
                        val = val * half[:, c]
                Ja[:, b, b] = val.reshape((E,) + (1,) * d)
            self.Ja = Ja
        else:
            X = torch.as_tensor(mesh.xyz, dtype=torch.float64).reshape((E, d) + (n,) * d)
            D = torch.as_tensor(basis.D)
            # dX[c][b] = d x_c / d xi_b
            dX = torch.stack([torch.stack([along(X[:, c], b, d, D) for b in range(d)], 1)
                              for c in range(d)], 1)                          # [E, c, b, ...]
            if d == 2:
                self.J = dX[:, 0, 0] * dX[:, 1, 1] - dX[:, 0, 1] * dX[:, 1, 0]
                Ja = torch.zeros((E, 2, 2) + (n,) * 2, dtype=torch.float64)
                Ja[:, 0, 0] = dX[:, 1, 1]      # y_eta
                Ja[:, 0, 1] = -dX[:, 0, 1]     # -x_eta
                Ja[:, 1, 0] = -dX[:, 1, 0]     # -y_xi
                Ja[:, 1, 1] = dX[:, 0, 0]      # x_xi
                self.Ja = Ja
            else:
                m = dX
                self.J = (m[:, 0, 0] * (m[:, 1, 1] * m[:, 2, 2] - m[:, 1, 2] * m[:, 2, 1])
                          - m[:, 0, 1] * (m[:, 1, 0] * m[:, 2, 2] - m[:, 1, 2] * m[:, 2, 0])
                          + m[:, 0, 2] * (m[:, 1, 0] * m[:, 2, 1] - m[:, 1, 1] * m[:, 2, 0]))
                # the map at the Lobatto points, relative to the element mean
                xl = gauss_lobatto_points(n)
                G2L = torch.as_tensor(lagrange_eval(basis.x, xl))              # Gauss values -> Lobatto
                L2G = torch.as_tensor(lagrange_eval(xl, basis.x))              # Lobatto values -> Gauss
                DL = torch.as_tensor(derivative_matrix(xl))
                XL = X
                for a in range(3):
                    XL = along(XL, a, 4, G2L)
                XL = XL - XL.mean(dim=(2, 3, 4), keepdim=True)
                dXL = torch.stack([torch.stack([along(XL[:, c], b, 3, DL) for b in range(3)], 1)
                                   for c in range(3)], 1)                      # [E, c, b, ...]
                Ja = torch.zeros((E, 3, 3) + (n,) * 3, dtype=torch.float64)
                for nn in range(3):
                    mm, ll = (nn + 1) % 3, (nn + 2) % 3
                    # G_b = X_l * d X_m / d xi_b at the Lobatto points = its Lobatto interpolant
                    G = [XL[:, ll] * dXL[:, mm, b] for b in range(3)]
                    for i in range(3):
                        j, k = (i + 1) % 3, (i + 2) % 3
                        curl_i = along(G[k], j, 3, DL) - along(G[j], k, 3, DL)
                        for a in range(3):
                            curl_i = along(curl_i, a, 3, L2G)
                        Ja[:, i, nn] = -curl_i
                self.Ja = Ja
        # face area-normals Sn[E][2d][d][nfp]
        nfp = n ** (d - 1)
        Sn = torch.zeros((E, 2 * d, d, nfp), dtype=torch.float64)
        for a in range(d):
            for side in (0, 1):
                for c in range(d):
                    tr = trace(self.Ja[:, a, c], a, side, d, basis).reshape(E, nfp)
                    Sn[:, 2 * a + side, c] = tr if side else -tr
        self.Sn = Sn
