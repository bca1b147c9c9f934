"""Pins of the oracle's 1D basis and element geometry against closed forms."""
import math

import numpy as np
import pytest
import torch

from oracle.basis import Basis1D
from oracle.geometry import Geometry, along
from paper_2607_16044_b300 import inputs as I


def test_gauss_closed_forms():
    b = Basis1D(1)
    assert np.allclose(b.x, [-1 / math.sqrt(3), 1 / math.sqrt(3)], atol=1e-15)
    assert np.allclose(b.w, [1, 1], atol=1e-15)
    b = Basis1D(2)
    assert np.allclose(b.x, [-math.sqrt(0.6), 0, math.sqrt(0.6)], atol=1e-15)
    assert np.allclose(b.w, [5 / 9, 8 / 9, 5 / 9], atol=1e-15)


@pytest.mark.parametrize("p", range(1, 8))
def test_gauss_matches_library_and_exactness(p):
    b = Basis1D(p)
    x, w = np.polynomial.legendre.leggauss(p + 1)
    assert np.allclose(b.x, x, atol=2e-15) and np.allclose(b.w, w, atol=2e-15)
    assert abs(b.w.sum() - 2) < 1e-14
    for k in range(2 * p + 2):            # exact for degree <= 2n - 1
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(b.w, b.x ** k) - exact) < 1e-13


@pytest.mark.parametrize("p", range(1, 8))
def test_derivative_matrix(p):
    b = Basis1D(p)
    assert np.max(np.abs(b.D.sum(1))) < 1e-12           # rows annihilate constants
    for k in range(p + 1):                               # exact on P^p
        dk = k * b.x ** (k - 1) if k else np.zeros_like(b.x)
        assert np.max(np.abs(b.D @ b.x ** k - dk)) < 1e-11
    for k in range(p + 1):                               # boundary interpolation exact on P^p
        assert abs(b.lp @ b.x ** k - 1.0) < 1e-13
        assert abs(b.lm @ b.x ** k - (-1.0) ** k) < 1e-13
    # SBP property of the Gauss collocation: W D + (W D)^T = l(1) l(1)^T - l(-1) l(-1)^T
    Q = np.diag(b.w) @ b.D
    B = np.outer(b.lp, b.lp) - np.outer(b.lm, b.lm)
    assert np.max(np.abs(Q + Q.T - B)) < 1e-12




def test_geometry_boxes_and_warped_2d():
    m = I.warped_mesh(4, [3, 4], [2.0, 1.0], 0.04)
    b = Basis1D(4)
    g = Geometry(m, b)
    assert torch.all(g.J > 0)
    w2 = torch.as_tensor(np.outer(b.w, b.w))              # [i1][i0]
    area = (g.J * w2).sum()
    assert abs(area.item() - 2.0) < 1e-12                  # warp keeps the box boundary
    # discrete metric identity sum_a D_a (Ja_a)_c = 0
    D = torch.as_tensor(b.D)
    for c in range(2):
        ident = sum(along(g.Ja[:, a, c], a, 2, D) for a in range(2))
        assert ident.abs().max() < 1e-13
    # boxes: exact J and Ja
    mb = I.structured_box_mesh(3, [I.uniform_edges(0, 2, 2), I.wall_stretched_edges(4, 1.5)], [True, False])
    gb = Geometry(mb, Basis1D(3))
    h = torch.as_tensor(mb.size)
    assert torch.allclose(gb.J[:, 0, 0], h[:, 0] * h[:, 1] / 4, rtol=0, atol=1e-16)
    assert torch.allclose(gb.Ja[:, 0, 0, 0, 0], h[:, 1] / 2) and torch.all(gb.Ja[:, 0, 1] == 0)


def test_geometry_warped_3d_metric_identities():
    m = I.warped_mesh(3, [2, 2, 2], [1.0, 1.5, 2.0], 0.03)
    b = Basis1D(3)
    g = Geometry(m, b)
    assert torch.all(g.J > 0)
    w3 = torch.as_tensor(np.einsum("i,j,k->ijk", b.w, b.w, b.w))
    assert abs((g.J * w3).sum().item() - 3.0) < 1e-11
    D = torch.as_tensor(b.D)
    for c in range(3):
        ident = sum(along(g.Ja[:, a, c], a, 3, D) for a in range(3))
        assert ident.abs().max() < 1e-12
    # the curl form agrees with the cross-product form up to discretisation
    # error; on an affine (unwarped) mesh it is exact
    ma = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 2)] * 3, [True] * 3).as_nodes()
    ga = Geometry(ma, b)
    gb = Geometry(I.structured_box_mesh(3, [I.uniform_edges(0, 1, 2)] * 3, [True] * 3), b)
    assert torch.allclose(ga.Ja, gb.Ja, atol=1e-14) and torch.allclose(ga.J, gb.J, atol=1e-15)


def test_face_normals_opposite():
    m = I.rotate_elements(I.warped_mesh(3, [3, 3], [1.0, 1.0], 0.05), 2)
    g = Geometry(m, Basis1D(3))
    from oracle.residual import orient_index
    for e in range(m.n_elem):
        for f in range(4):
            nb, nf, o = m.neighbor[e, f], m.nbr_face[e, f], m.orient[e, f]
            mine = g.Sn[e, f]
            theirs = g.Sn[nb, nf][:, orient_index(o, 4, 2)]
            assert torch.allclose(mine, -theirs, atol=1e-13)


def test_gauss_lobatto_closed_forms():
    from oracle.basis import gauss_lobatto_points
    r = math.sqrt
    want = {2: [-1, 1], 3: [-1, 0, 1], 4: [-1, -1 / r(5), 1 / r(5), 1], 5: [-1, -r(3 / 7), 0, r(3 / 7), 1],
            6: [-1, -r(1 / 3 + 2 * r(7) / 21), -r(1 / 3 - 2 * r(7) / 21), r(1 / 3 - 2 * r(7) / 21),
                r(1 / 3 + 2 * r(7) / 21), 1]}
    for n, x in want.items():
        assert np.allclose(gauss_lobatto_points(n), x, atol=1e-15, rtol=0)


def _mixed_warp_3d(p=3, rotate=None):
    m = I.warped_mesh(p, [3, 3, 2], [1.0, 1.2, 1.0], 0.02, mixed=True)
    return I.rotate_elements(m, rotate) if rotate is not None else m


def test_face_normals_opposite_3d_curved():
    """A warp whose displacement gradient is not rank one and rotated local
    frames: each face's area normal, traced from either element, is the
    same up to sign (the curl form through the Lobatto interpolant depends
    on the face's own points only)."""
    m = _mixed_warp_3d(3, rotate=4)
    g = Geometry(m, Basis1D(3))
    from oracle.residual import orient_index
    scale = g.Sn.abs().max()
    for e in range(m.n_elem):
        for f in range(6):
            nb, nf, o = m.neighbor[e, f], m.nbr_face[e, f], m.orient[e, f]
            mine = g.Sn[e, f]
            theirs = g.Sn[nb, nf][:, orient_index(o, 4, 3)]
            assert (mine + theirs).abs().max() < 1e-13 * scale


@pytest.mark.parametrize("p", [2, 3, 4])
def test_geometry_curved_3d_identities_and_volume(p):
    m = _mixed_warp_3d(p, rotate=5)
    b = Basis1D(p)
    g = Geometry(m, b)
    assert torch.all(g.J > 0)
    w3 = torch.as_tensor(np.einsum("i,j,k->ijk", b.w, b.w, b.w))
    assert abs((g.J * w3).sum().item() - 1.2) < 1e-6       # quadrature of the exact volume
    D = torch.as_tensor(b.D)
    for c in range(3):
        ident = sum(along(g.Ja[:, a, c], a, 3, D) for a in range(3))
        assert ident.abs().max() < 1e-13 * g.Ja.abs().max() * (p + 1) ** 2


@pytest.mark.parametrize("op", ["llf-br1", "dgip"])
def test_free_stream_3d_curved(op):
    """A uniform flow stays at rest on a curved 3D mesh with rotated frames."""
    from oracle import physics as ph
    from oracle.residual import DGOperator
    from oracle.sipg import SIPGOperator
    m = _mixed_warp_3d(3, rotate=6)
    gas = ph.Gas(1.4, Re=80.0, Pr=0.72, viscous=True)
    U = np.zeros((m.n_elem, 5, m.N))
    U[:, 0], U[:, 1], U[:, 2], U[:, 3], U[:, 4] = 1.2, 0.3, -0.2, 0.1, 3.0
    cls = DGOperator if op == "llf-br1" else SIPGOperator
    f = cls(m, gas).residual(torch.as_tensor(U))
    assert f.abs().max() < 1e-13 * 4.0 / 0.1
