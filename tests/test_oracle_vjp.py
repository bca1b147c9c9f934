"""Pins of the oracle's vector-Jacobian product (complex step, FD, adjoint identity)."""
import numpy as np
import pytest
import torch

from oracle.physics import Gas
from oracle.residual import DGOperator
from oracle.vjp import jacobian_cs, jvp_cs, vjp
from paper_2607_16044_b300 import inputs as I


def _mesh(kind, p):
    if kind == "periodic":
        return I.structured_box_mesh(p, [I.uniform_edges(0, 1, 2), I.uniform_edges(0, 1.5, 2)], [True, True])
    if kind == "wall":
        return I.structured_box_mesh(p, [I.uniform_edges(0, 1, 2), I.wall_stretched_edges(1, 1.0)], [True, False])
    return I.rotate_elements(I.warped_mesh(p, [2, 2], [1.0, 1.0], 0.04), 3)


@pytest.mark.parametrize("kind", ["periodic", "wall", "warped"])
@pytest.mark.parametrize("viscous", [False, True])
def test_vjp_equals_complex_step_jacobian_transpose(kind, viscous):
    m = _mesh(kind, 2)
    op = DGOperator(m, Gas(1.4, Re=30.0, viscous=viscous))
    U = torch.as_tensor(I.random_state(m, 4))
    lam = torch.as_tensor(I.gaussian_cotangent(U.shape, 5))
    Jm = jacobian_cs(op, U)
    ref = (Jm.T @ lam.reshape(-1)).reshape(U.shape)
    g = vjp(op, U, lam)
    assert (g - ref).abs().max() <= 1e-13 * ref.abs().max()


@pytest.mark.parametrize("viscous", [False, True])
def test_vjp_central_differences(viscous):
    m = _mesh("wall", 3)
    op = DGOperator(m, Gas(1.4, Re=30.0, viscous=viscous))
    U = torch.as_tensor(I.random_state(m, 6))
    lam = torch.as_tensor(I.gaussian_cotangent(U.shape, 7))
    g = vjp(op, U, lam)
    rng = np.random.default_rng(8)
    for _ in range(3):
        v = torch.as_tensor(rng.standard_normal(U.shape))
        eps = 1e-6 * U.abs().max().item()
        fd = ((op.residual(U + eps * v) - op.residual(U - eps * v)) * lam).sum() / (2 * eps)
        ad = (g * v).sum()
        assert abs(fd - ad) <= 1e-6 * abs(ad)


def test_adjoint_identity_larger_mesh():
    m = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 5), I.wall_stretched_edges(3, 1.3)], [True, False])
    op = DGOperator(m, Gas(1.4, Re=100.0, viscous=True))
    U = torch.as_tensor(I.random_state(m, 9))
    lam = torch.as_tensor(I.gaussian_cotangent(U.shape, 10))
    v = torch.as_tensor(I.gaussian_cotangent(U.shape, 11))
    lhs = (lam * jvp_cs(op, U, v)).sum()
    rhs = (vjp(op, U, lam) * v).sum()
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_subset_vjp_matches_full():
    m = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 6), I.wall_stretched_edges(2, 1.3)], [True, False])
    op = DGOperator(m, Gas(1.4, Re=100.0, viscous=True))
    U = torch.as_tensor(I.random_state(m, 9))
    lam = torch.as_tensor(I.gaussian_cotangent(U.shape, 10))
    g = vjp(op, U, lam)
    from oracle.vjp import vjp_rows
    rows = [0, 9, 17]
    assert torch.allclose(vjp_rows(op, U, lam, rows), g[rows], rtol=1e-13, atol=1e-13 * g.abs().max())
