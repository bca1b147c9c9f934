"""Pins of the oracle residual: brute force, invariants, manufactured solution."""
import numpy as np
import pytest
import torch

from oracle.brute import BruteDG
from oracle.physics import Gas
from oracle.residual import DGOperator
from paper_2607_16044_b300 import inputs as I
from tests import mms_sympy


def _mass_weights(op):
    w = op.basis.w
    W = w
    for _ in range(op.d - 1):
        W = np.multiply.outer(w, W)
    return torch.as_tensor(W.reshape(-1)) * op.geo.J.reshape(op.E, -1)


@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_brute_force_2d_rotated_with_walls(p, viscous):
    m = I.rotate_elements(I.structured_box_mesh(p, [I.uniform_edges(0, 1, 3), I.uniform_edges(0, 1.5, 2)],
                                                [True, False]), 11 + p)
    gas = Gas(1.4, Re=50.0, Pr=0.72, viscous=viscous)
    U = I.random_state(m, 7)
    f1 = DGOperator(m, gas).residual(torch.as_tensor(U)).numpy()
    f2 = BruteDG(m, gas, period=[1, 1.5]).residual(U)
    assert np.abs(f1 - f2).max() / np.abs(f1).max() < 1e-12


@pytest.mark.parametrize("viscous", [False, True])
def test_brute_force_3d_rotated(viscous):
    m = I.rotate_elements(I.structured_box_mesh(2, [I.uniform_edges(0, 1, 2), I.uniform_edges(0, 1.5, 2),
                                                    I.uniform_edges(0, 2, 2)], [True, True, False]), 5)
    gas = Gas(1.4, Re=50.0, Pr=0.72, viscous=viscous)
    U = I.random_state(m, 8)
    f1 = DGOperator(m, gas).residual(torch.as_tensor(U)).numpy()
    f2 = BruteDG(m, gas, period=[1, 1.5, 2]).residual(U)
    assert np.abs(f1 - f2).max() / np.abs(f1).max() < 1e-12


def _free_stream(mesh, gamma=1.4):
    d = mesh.dim
    one = np.ones((mesh.n_elem, mesh.N))
    vel = [0.7 * one, -0.4 * one, 0.3 * one][:d]
    return I._stack_state(one, vel, 2.0 * one, gamma)


@pytest.mark.parametrize("case", ["box2", "stretched2", "warped2", "warped3", "rot3"])
@pytest.mark.parametrize("viscous", [False, True])
def test_free_stream_preservation(case, viscous):
    if case == "box2":
        m = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 4)] * 2, [True, True])
    elif case == "stretched2":
        m = I.structured_box_mesh(4, [I.uniform_edges(0, 5, 4), I.wall_stretched_edges(6, 1.15)], [True, True])
    elif case == "warped2":
        m = I.rotate_elements(I.warped_mesh(4, [4, 3], [1.0, 1.0], 0.05), 3)
    elif case == "warped3":
        m = I.warped_mesh(3, [2, 2, 2], [1.0, 1.0, 1.0], 0.03)
    else:
        m = I.rotate_elements(I.warped_mesh(2, [2, 2, 2], [1.0, 1.0, 1.0], 0.03), 9)
    gas = Gas(1.4, Re=100.0, viscous=viscous)
    f = DGOperator(m, gas).residual(torch.as_tensor(_free_stream(m))).numpy()
    # scale: |F^c| / h_min
    hmin = 1e-2 if case != "stretched2" else 1e-4
    assert np.abs(f).max() < 1e-12 * 4.0 / hmin


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("viscous", [False, True])
def test_conservation_periodic(d, viscous):
    if d == 2:
        m = I.rotate_elements(I.warped_mesh(3, [3, 4], [1.0, 1.3], 0.05), 4)
    else:
        m = I.rotate_elements(I.structured_box_mesh(2, [I.uniform_edges(0, 1, 2), I.uniform_edges(0, 1, 3),
                                                        I.uniform_edges(0, 2, 2)], [True] * 3), 6)
    gas = Gas(1.4, Re=50.0, viscous=viscous)
    op = DGOperator(m, gas)
    U = I.random_state(m, 21)
    f = op.residual(torch.as_tensor(U))
    wJ = _mass_weights(op)
    total = (f * wJ[:, None, :]).sum((0, 2))
    scale = (f.abs() * wJ[:, None, :]).sum((0, 2))
    assert torch.all(total.abs() < 1e-13 * scale)


def test_wall_conservation_of_mass():
    """With walls only the mass integral is conserved (no mass flux through walls)."""
    m = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 3), I.wall_stretched_edges(2, 1.3)], [True, False])
    gas = Gas(1.4, Re=50.0, viscous=True)
    op = DGOperator(m, gas)
    f = op.residual(torch.as_tensor(I.random_state(m, 5)))
    wJ = _mass_weights(op)
    total = (f[:, 0] * wJ).sum()
    assert abs(total) < 1e-13 * (f[:, 0].abs() * wJ).sum()


@pytest.mark.parametrize("viscous", [False, True])
def test_xy_swap_symmetry(viscous):
    p, nc = 3, 3
    m = I.structured_box_mesh(p, [I.uniform_edges(0, 1, nc)] * 2, [True, True])
    gas = Gas(1.4, Re=50.0, viscous=viscous)
    op = DGOperator(m, gas)
    U = I.random_state(m, 13)
    n = p + 1

    def swap(V):
        # element (i, j) <-> (j, i); node (q0, q1) <-> (q1, q0); rho u <-> rho v
        V = V.reshape(nc, nc, 4, n, n)
        V = V.transpose(1, 0, 2, 4, 3)[:, :, [0, 2, 1, 3]]
        return V.reshape(nc * nc, 4, n * n)
    f = op.residual(torch.as_tensor(U)).numpy()
    fs = op.residual(torch.as_tensor(swap(U))).numpy()
    assert np.abs(swap(f) - fs).max() < 1e-13 * np.abs(f).max()


def test_translation_equivariance():
    nc, p = 4, 2
    m = I.structured_box_mesh(p, [I.uniform_edges(0, 1, nc)] * 2, [True, True])
    gas = Gas(1.4, Re=80.0, viscous=True)
    op = DGOperator(m, gas)
    U = I.random_state(m, 17)
    shift = lambda V: np.roll(V.reshape(nc, nc, 4, -1), 1, axis=1).reshape(nc * nc, 4, -1)
    f = op.residual(torch.as_tensor(U)).numpy()
    assert np.abs(shift(f) - op.residual(torch.as_tensor(shift(U))).numpy()).max() < 1e-13 * np.abs(f).max()


def test_one_dimensional_profile():
    """A state depending on x only gives x-only rates and a zero rho*v rate."""
    nc, p = 3, 3
    m = I.structured_box_mesh(p, [I.uniform_edges(0, 1, nc)] * 2, [True, True])
    x = m.xyz[:, 0, :]
    rho = 1 + 0.2 * np.sin(2 * np.pi * x)
    U = I._stack_state(rho, [0.5 + 0.1 * np.cos(2 * np.pi * x), 0 * x], 1 + 0.1 * np.sin(4 * np.pi * x), 1.4)
    f = DGOperator(m, Gas(1.4, Re=30.0, viscous=True)).residual(torch.as_tensor(U)).numpy()
    assert np.abs(f[:, 2]).max() < 1e-13
    fr = f.reshape(nc, nc, 4, p + 1, p + 1)                    # [j][i][field][q1][q0]
    assert np.abs(fr - fr[:1, :, :, :1, :]).max() < 1e-12 * np.abs(f).max()


@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("p", [2, 3])
def test_manufactured_solution_truncation_order(p, viscous):
    """f(U_e) -> -div(F^c - F^nu)(U_e) at the rate of the scheme's truncation error
    (Sec. 5.1.1 manufactured solution, derived symbolically from Sec. 2)."""
    mu = 0.01
    fns = mms_sympy.build(2, 1.4, mu if viscous else 0.0, 0.72)
    gas = Gas(1.4, Re=1 / mu if viscous else 0.0, Pr=0.72, viscous=viscous)
    errs = []
    for nc in (8, 16):
        m = I.structured_box_mesh(p, [I.uniform_edges(0, 1, nc)] * 2, [True, True])
        U = mms_sympy.evaluate(fns["U"], m.xyz, 0.0)
        exact = -(mms_sympy.evaluate(fns["divFc"], m.xyz, 0.0) - mms_sympy.evaluate(fns["divFv"], m.xyz, 0.0))
        f = DGOperator(m, gas).residual(torch.as_tensor(U)).numpy()
        errs.append(np.sqrt(np.mean((f - exact) ** 2)) / np.sqrt(np.mean(exact ** 2)))
    rate = np.log2(errs[0] / errs[1])
    bound = {2: 1.2e-2, 3: 5e-4}[p]
    assert errs[1] < bound and rate > p - 0.4, (errs, rate)


def test_manufactured_solution_3d():
    mu = 0.01
    fns = mms_sympy.build(3, 1.4, mu, 0.72, 1, 1, 1, 200)
    gas = Gas(1.4, Re=1 / mu, Pr=0.72, viscous=True)
    errs = []
    for nc in (3, 6):
        m = I.structured_box_mesh(2, [I.uniform_edges(0, 2, nc)] * 3, [True] * 3)
        U = mms_sympy.evaluate(fns["U"], m.xyz, 0.0)
        exact = -(mms_sympy.evaluate(fns["divFc"], m.xyz, 0.0) - mms_sympy.evaluate(fns["divFv"], m.xyz, 0.0))
        f = DGOperator(m, gas).residual(torch.as_tensor(U)).numpy()
        errs.append(np.sqrt(np.mean((f - exact) ** 2)) / np.sqrt(np.mean(exact ** 2)))
    assert errs[1] < errs[0] / 2.5, errs


def test_subset_evaluation_matches_full():
    m = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 5), I.wall_stretched_edges(2, 1.2)], [True, False])
    gas = Gas(1.4, Re=50.0, viscous=True)
    op = DGOperator(m, gas)
    U = torch.as_tensor(I.random_state(m, 3))
    full = op.residual(U)
    elems = [0, 7, 13, 19]
    sub = op.residual(U, elems)
    assert torch.allclose(sub, full[elems], atol=0, rtol=1e-15)
