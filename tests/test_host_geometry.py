"""Host logic of the library's geometry (no GPU): the metric terms that
dgx_set_mesh_nodes derives (exported as dgx_mesh_metrics) against the
oracle's Geometry, whose 3D curl form is pinned on its own (metric
identities, face normals equal across faces, free-stream preservation)."""
import numpy as np
import pytest
import torch

from oracle.basis import Basis1D
from oracle.geometry import Geometry
from paper_2607_16044_b300 import inputs as I
from paper_2607_16044_b300.dgx import mesh_metrics


def _cases():
    yield "warped2d", I.rotate_elements(I.warped_mesh(3, [3, 4], [1.0, 1.3], 0.03, mixed=True), 1)
    yield "sheared2d", I.rotate_elements(I.structured_box_mesh(2, [I.uniform_edges(0, 1, 3),
                                                                   I.wall_stretched_edges(2, 1.4)], [True, False]), 2)
    for p in (1, 2, 3, 5, 7):
        yield f"warped3d-p{p}", I.rotate_elements(I.warped_mesh(p, [3, 3, 2], [1.0, 1.2, 1.0], 0.02, mixed=True), 3)


@pytest.mark.parametrize("name,mesh", list(_cases()), ids=[c[0] for c in _cases()])
def test_library_metrics_match_the_oracle(name, mesh):
    J, metric = mesh_metrics(mesh)
    g = Geometry(mesh, Basis1D(mesh.p))
    E, N, d = mesh.n_elem, mesh.N, mesh.dim
    Jo = g.J.reshape(E, N).numpy()
    Mo = g.Ja.reshape(E, d, d, N).permute(0, 3, 1, 2).numpy()
    # rounding of the two evaluation orders, amplified by the derivative
    # matrices (norm ~ (p+1)^2)
    tol = 1e-14 * (mesh.p + 1) ** 2
    assert np.abs(J - Jo).max() < tol * np.abs(Jo).max()
    assert np.abs(metric - Mo).max() < tol * np.abs(Mo).max()


def test_library_metrics_reject_inverted_elements():
    from paper_2607_16044_b300.dgx import DGXError
    m = I.warped_mesh(2, [2, 2], [1.0, 1.0], 0.0)
    xyz = m.xyz.copy()
    xyz[0, 0] = -xyz[0, 0]                  # mirror one element: J < 0
    bad = I.Mesh(2, m.p, m.n_elem, "nodes", xyz, m.neighbor, m.nbr_face, m.orient)
    with pytest.raises(DGXError):
        mesh_metrics(bad)
