"""The geometry override (dgx_set_geometry): metric terms handed to the
library instead of derived from node coordinates.  Parity against the oracle
with the oracle's own metrics, the exact box metrics through the curvilinear
kernels against the box kernels, and the override's bookkeeping."""
import numpy as np
import pytest
import torch

from oracle.residual import DGOperator
from paper_2607_16044_b300 import inputs as I
from tests.parity_util import TOL, gas_of, oracle_rhs, quantize32, record, rel_err

pytestmark = pytest.mark.gpu


def _ns():
    return I.Physics(gamma=1.4, Re=300.0, Pr=0.72, Ma=0.3, viscous=True)


def _metrics(mesh):
    """J[E][N] and J dxi_a/dx_b as [E][N][d][d] from the oracle's geometry."""
    op = DGOperator(mesh, gas_of(_ns()))
    E, d, N = mesh.n_elem, mesh.dim, mesh.N
    J = op.geo.J.reshape(E, N).numpy()
    M = op.geo.Ja.reshape(E, d, d, N).permute(0, 3, 1, 2).numpy()
    return J, M


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dim", [2, 3])
def test_override_with_the_oracle_metrics_matches_the_oracle(dim, prec):
    from paper_2607_16044_b300.dgx import Solver
    if dim == 2:
        mesh = I.rotate_elements(I.warped_mesh(3, [5, 4], [1.0, 1.2], 0.04, periodic=[True, False]), 7)
    else:
        mesh = I.warped_mesh(2, [2, 3, 2], [1.0, 1.0, 1.0], 0.03, periodic=[True, True, False])
    U = I.random_state(mesh, 800 + dim)
    s = Solver(mesh, _ns(), prec)
    s.set_geometry(*_metrics(mesh))
    dt = torch.float64 if prec == "fp64" else torch.float32
    f = s.rhs(torch.as_tensor(U).to("cuda", dt).contiguous()).double().cpu().numpy()
    s.check()
    ref = oracle_rhs(mesh, _ns(), U if prec == "fp64" else quantize32(U))
    err = rel_err(f, ref)
    record(f"geometry-override-{dim}d-{prec}", rel=err)
    assert err < TOL[prec], err


def test_exact_box_metrics_through_the_curvilinear_kernels():
    """A stretched box mesh: the box kernels, and the same connectivity with
    the boxes' exact metrics (J = prod h/2, J dxi_a/dx_a = prod_{c != a} h_c/2)
    handed over, which runs the curvilinear kernels; both equal the oracle."""
    from paper_2607_16044_b300.dgx import Solver
    mesh = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 5), I.wall_stretched_edges(2, 1.3)], [True, False])
    U = torch.as_tensor(I.random_state(mesh, 810)).cuda()
    s0 = Solver(mesh, _ns(), "fp64")
    s1 = Solver(mesh, _ns(), "fp64")
    E, N = mesh.n_elem, mesh.N
    half = 0.5 * mesh.size
    J = np.repeat(np.prod(half, 1)[:, None], N, 1)
    M = np.zeros((E, N, 2, 2))
    M[:, :, 0, 0] = half[:, 1:2]
    M[:, :, 1, 1] = half[:, 0:1]
    s1.set_geometry(J, M)
    f0, f1 = s0.rhs(U).cpu().numpy(), s1.rhs(U).cpu().numpy()
    s0.check()
    s1.check()
    ref = oracle_rhs(mesh, _ns(), U.cpu().numpy())
    assert rel_err(f0, ref) < TOL["fp64"]
    assert rel_err(f1, ref) < TOL["fp64"]
    assert rel_err(f1, f0) < 1e-13


def test_override_bookkeeping():
    """Invalid metrics are refused, the batch runtime refuses an overridden
    handle, and the overridden handle still matches the oracle."""
    from paper_2607_16044_b300.dgx import Batch, DGXError, Solver
    from paper_2607_16044_b300.tableaux import ars343_explicit
    mesh = I.warped_mesh(2, [3, 3], [1.0, 1.0], 0.04)
    J, M = _metrics(mesh)
    s = Solver(mesh, _ns(), "fp64")
    s.set_tableau(*ars343_explicit())
    bad = J.copy()
    bad[1, 2] = -1.0
    with pytest.raises(DGXError) as err:
        s.set_geometry(bad, M)
    assert err.value.code == 1
    s.set_geometry(J, M)
    with pytest.raises(DGXError) as err:
        Batch([s], [1e-3])
    assert err.value.code == 6
    U = torch.as_tensor(I.random_state(mesh, 820)).cuda()
    f_override = s.rhs(U).cpu().numpy()
    s.check()
    ref = oracle_rhs(mesh, _ns(), U.cpu().numpy())
    assert rel_err(f_override, ref) < TOL["fp64"]


@pytest.mark.parametrize("scheme,M", [("llf-br1", None), ("dgip", None), ("dgip", "3k")])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_free_stream_on_a_curved_3d_mesh(scheme, M, prec):
    """A uniform flow on a rotated 3D warp whose displacement gradient is not
    rank one: every operator keeps it at rest (the face normals of the two
    sides of a face agree, the metric identities hold).  The FP64 oracle
    leaves 1.5e-12 (collocated) to 4.1e-12 (over-integrated) here, about
    2e4 eps; the bound is ten times that at the kernel's precision (the
    Gauss-node curl form left 4.8 on this mesh, where a random state's
    residual is about 110)."""
    from paper_2607_16044_b300.dgx import Solver
    mesh = I.rotate_elements(I.warped_mesh(3, [4, 4, 3], [1.0, 1.2, 1.0], 0.02, mixed=True), 9)
    U = np.zeros((mesh.n_elem, 5, mesh.N))
    U[:, 0], U[:, 1], U[:, 2], U[:, 3], U[:, 4] = 1.2, 0.3, -0.2, 0.1, 3.0
    dt = torch.float64 if prec == "fp64" else torch.float32
    s = Solver(mesh, _ns(), prec, scheme=scheme, quad_points=M)
    f = s.rhs(torch.as_tensor(U).to("cuda", dt).contiguous()).double().abs().max().item()
    s.check()
    eps = 2.2e-16 if prec == "fp64" else 1.2e-7
    record(f"free-stream-3d-{scheme}-{M}-{prec}", abs=f)
    assert f < 10 * 2e4 * eps
