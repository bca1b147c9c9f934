"""Pins of the explicit ARK stage/solution updates and of their adjoint."""
import numpy as np
import pytest
import torch

from oracle import ark
from oracle.physics import Gas
from oracle.residual import DGOperator
from oracle.vjp import vjp
from paper_2607_16044_b300 import inputs as I
from tests import mms_sympy


def test_ars343_order_conditions():
    A, b, c = ark.ars343()
    assert np.allclose(A.sum(1), c, atol=2e-10)
    assert abs(b.sum() - 1) < 1e-9
    assert abs(b @ c - 0.5) < 1e-9
    assert abs(b @ c ** 2 - 1 / 3) < 1e-9
    assert abs(b @ A @ c - 1 / 6) < 1e-9
    g = ark.ARS343_GAMMA                      # root of 6 g^3 - 18 g^2 + 9 g - 1 in (0, 1)
    assert abs(6 * g ** 3 - 18 * g ** 2 + 9 * g - 1) < 1e-9
    assert np.all(np.triu(A) == 0)           # explicit
    assert not np.allclose(A[-1], b)         # not FSAL: final update needed (Algorithm 1)


@pytest.mark.parametrize("scheme,order", [(ark.forward_euler, 1), (ark.heun2, 2), (ark.ars343, 3)])
def test_temporal_order_nonlinear_system(scheme, order):
    """Nonlinear ODE against a tight DOP853 solution.  (On linear problems the
    explicit ARS(3,4,3) half is one order better: b.A.A.c = 1/24.)"""
    from scipy.integrate import solve_ivp

    def rhs_np(t, y):
        return np.array([-y[0] * y[1] + 0.3 * y[2], y[0] ** 2 - 0.5 * y[1], -np.sin(y[0]) * y[2]])
    y0 = np.array([1.0, 0.5, -0.7])
    ref = solve_ivp(rhs_np, (0, 1), y0, method="DOP853", rtol=1e-13, atol=1e-14).y[:, -1]
    A, b, c = scheme()
    errs = []
    for nsteps in (20, 40, 80):
        y = torch.as_tensor(y0)
        for _ in range(nsteps):
            y = ark.erk_step(lambda v: torch.as_tensor(rhs_np(0, v.numpy())), y, 1.0 / nsteps, A, b)
        errs.append(np.linalg.norm(y.numpy() - ref))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - order) < 0.2), rates


@pytest.mark.slow
def test_mms_temporal_order_explicit_dg():
    """The paper's MMS (Sec. 5.1.1: [0,1]^2 periodic, kx = ky = 2, omega = 200,
    mu = 0.01, one period t = 0.01): the explicit DG with RK1/RK2/ARS(3,4,3)
    converges in time at orders 1/2/3 (Fig. of the MMS errors)."""
    mu = 0.01
    fns = mms_sympy.build(2, 1.4, mu, 0.72)
    mesh = I.structured_box_mesh(4, [I.uniform_edges(0, 1, 8)] * 2, [True, True])
    op = DGOperator(mesh, Gas(1.4, Re=1 / mu, Pr=0.72, viscous=True))

    def source(t):
        Ut = mms_sympy.evaluate(fns["Ut"], mesh.xyz, t)
        div = mms_sympy.evaluate(fns["divFc"], mesh.xyz, t) - mms_sympy.evaluate(fns["divFv"], mesh.xyz, t)
        return torch.as_tensor(Ut + div)

    rhs = lambda y, t: op.residual(y) + source(t)
    U0 = torch.as_tensor(mms_sympy.evaluate(fns["U"], mesh.xyz, 0.0))
    Ue = mms_sympy.evaluate(fns["U"], mesh.xyz, 0.01)
    for scheme, order, steps in ((ark.forward_euler, 1, (200, 400)), (ark.heun2, 2, (25, 50)),
                                 (ark.ars343, 3, (10, 20))):
        A, b, c = scheme()
        errs = []
        for n in steps:
            y, dt = U0.clone(), 0.01 / n
            for k in range(n):
                y = ark.erk_step(rhs, y, dt, A, b, t0=k * dt, c=c)
            errs.append(np.sqrt(np.mean((y.numpy() - Ue) ** 2)))
        rate = np.log2(errs[0] / errs[1])
        assert abs(rate - order) < 0.35, (scheme.__name__, errs, rate)


def test_vortex_spatial_convergence():
    """Exact advection of the isentropic vortex: observed order near p + 1 = 4."""
    A, b, c = ark.ars343()
    errs = []
    for cells in (4, 8, 16):
        m, phys, U0 = I.vortex_workload(p=3, cells=cells)
        op = DGOperator(m, Gas(1.4))
        U, dt = torch.as_tensor(U0), 0.16 / cells
        n = int(round(0.5 / dt))
        for _ in range(n):
            U = ark.erk_step(op.residual, U, dt, A, b)
        ex = I.isentropic_vortex(m, n * dt, 1.4)
        errs.append(np.sqrt(np.mean((U.numpy()[:, 0] - ex[:, 0]) ** 2)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 3.3), (errs, rates)


def test_adjoint_recurrence_matches_autograd():
    A, b, c = ark.ars343()
    m = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 3), I.wall_stretched_edges(1, 1.0)], [True, False])
    op = DGOperator(m, Gas(1.4, Re=20.0, viscous=True))
    U = torch.as_tensor(I.random_state(m, 1))
    lam = torch.as_tensor(I.gaussian_cotangent(U.shape, 2))
    dt = 1e-3
    _, ys, _ = ark.erk_step(op.residual, U, dt, A, b, return_stages=True)
    lam_n = ark.erk_adjoint_step(lambda y, mu: vjp(op, y, mu), ys, lam, dt, A, b)
    Ut = U.clone().requires_grad_(True)
    out = ark.erk_step(op.residual, Ut, dt, A, b)
    (ref,) = torch.autograd.grad(out, Ut, lam)
    assert torch.allclose(lam_n, ref, rtol=1e-12, atol=1e-12 * ref.abs().max())


def test_package_tableau_matches_oracle_tableau():
    """The product's copy of the published coefficients equals the oracle's."""
    from paper_2607_16044_b300.tableaux import ars343_explicit
    A, b, c = ars343_explicit()
    A2, b2, c2 = ark.ars343()
    assert np.array_equal(A, A2) and np.array_equal(b, b2) and np.array_equal(c, c2)


def test_ars343_explicit_stability_radius():
    """|R(z)| <= 1 along the imaginary axis up to about 2.8 for the explicit
    ARS(3,4,3) half; together with the vortex operator's spectral radius (~154
    on the 16x16 p = 3 mesh) this bounds its stable dt near 0.018."""
    A, b, c = ark.ars343()

    def R(z):
        return 1 + z * b @ np.linalg.solve(np.eye(4) - z * A, np.ones(4))
    assert abs(R(2.7j)) <= 1.0 + 1e-12
    assert abs(R(3.0j)) > 1.0
