"""Pins of the element-local HDG-IP oracle (Sec. 3.4 forms, Sec. 4.3 blocks):
the dense brute-force forms, exact rates and facet balance on a continuous
polynomial state with the exact trace as facet state, the mass block, and
the static-condensation identity against a dense solve of the local system."""
import numpy as np
import pytest
import torch

from oracle import physics as ph
from oracle.brute import BruteHDG
from oracle.hdg import HDGIPLocal
from paper_2607_16044_b300 import inputs as I

UINF = np.array([1.1, 0.4, -0.3, 2.0 / 0.4 + 0.5 * (0.4 ** 2 + 0.3 ** 2) / 1.1])


def _perturbed_traces(op, U, seed, amp=0.05):
    T = op.element_traces(op.nodes(torch.as_tensor(U)))
    return T * (1 + amp * torch.as_tensor(np.random.default_rng(seed).standard_normal(tuple(T.shape))))


@pytest.mark.parametrize("case", ["walls-p1", "walls-p2", "walls-p3", "farfield-p2", "euler-p3", "rotated-p2"])
def test_hdg_forms_match_brute_force(case):
    kind, p = case.split("-p")
    p = int(p)
    tag = 1 if kind == "farfield" else 0
    mesh = I.structured_box_mesh(p, [I.uniform_edges(0, 1, 3), I.wall_stretched_edges(1, 1.0)], [True, False],
                                 wall_tag=tag)
    if kind == "rotated":
        mesh = I.rotate_elements(mesh, 3)
    gas = ph.Gas(1.4, Re=100.0, Pr=0.72, viscous=kind != "euler")
    op = HDGIPLocal(mesh, gas, U_inf=UINF if tag else None)
    U = I.random_state(mesh, 4)
    Uh = _perturbed_traces(op, U, 5)
    R, h = op.forms(torch.as_tensor(U), Uh)
    Rb, hb = BruteHDG(mesh, gas, period=[1.0, 100.0]).residual_hdg(U, Uh.numpy(), U_inf=UINF)
    assert np.abs(R.numpy() - Rb).max() < 1e-12 * np.abs(Rb).max()
    assert np.abs(h.numpy() - hb).max() < 1e-12 * np.abs(hb).max()


def test_hdg_poiseuille_exact_trace():
    """rho = 1, u = 1 - y^2, v = 0, p const between adiabatic walls, facet state
    = the exact (continuous) trace: the penalty and adjoint-consistency terms
    vanish, the flux split reduces to F_n(Uhat), so R = -M (exact rates); the
    wall facets hold Uhat = U_w and every interior facet's two contributions
    cancel (continuous normal flux)."""
    p = 4
    mesh = I.structured_box_mesh(p, [I.uniform_edges(0, 0.5, 3), I.wall_stretched_edges(2, 1.4)], [True, False])
    gas = ph.Gas(1.4, Re=100.0, Pr=0.72, viscous=True)
    op = HDGIPLocal(mesh, gas)
    y = mesh.xyz[:, 1, :]
    U = torch.as_tensor(I._stack_state(np.ones_like(y), [1 - y * y, 0 * y], np.full_like(y, 3.0), 1.4))
    Uh = op.element_traces(op.nodes(U))
    R, h = op.forms(U, Uh)
    mu = gas.mu
    exact = torch.as_tensor(np.stack([0 * y, -2 * mu + 0 * y, 0 * y, mu * (6 * y * y - 2)], 1))
    assert (R + op.mass() * exact).abs().max() < 1e-11
    wall = torch.as_tensor(mesh.neighbor < 0)
    assert h[wall].abs().max() < 1e-12
    pair = op.gather_neighbor(h, torch.arange(mesh.n_elem))      # the neighbour's contribution at the same points
    assert (h + pair)[~wall].abs().max() < 1e-11 * h.abs().max()


def test_hdg_blocks_mass_and_static_condensation():
    """K - gamma dR/dU is the diagonal mass matrix; the condensed system
    S uhat = h - D K^{-1} w with S = A33 - D K^{-1} C reproduces the dense
    solve of [[K, C], [D, A33]] [z; uhat] = [w; h] for one element."""
    mesh = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 2), I.wall_stretched_edges(1, 1.0)], [True, False])
    gas = ph.Gas(1.4, Re=50.0, Pr=0.72, viscous=True)
    op = HDGIPLocal(mesh, gas)
    U = I.random_state(mesh, 6)
    Uh = _perturbed_traces(op, U, 7)
    gamma = 0.013
    K, C, D, A33 = op.blocks(U, Uh, gamma)
    K0, _, _, _ = op.blocks(U, Uh, 0.0)
    assert torch.allclose(K0, torch.diag_embed(op.mass().reshape(mesh.n_elem, -1)), rtol=0, atol=0)
    KinvC, S = op.schur(U, Uh, gamma)
    rng = np.random.default_rng(8)
    for e in range(mesh.n_elem):
        full = torch.cat([torch.cat([K[e], C[e]], 1), torch.cat([D[e], A33[e]], 1)], 0)
        w = torch.as_tensor(rng.standard_normal(K.shape[1]))
        hh = torch.as_tensor(rng.standard_normal(A33.shape[1]))
        sol = torch.linalg.solve(full, torch.cat([w, hh]))
        uh = torch.linalg.solve(S[e], hh - D[e] @ torch.linalg.solve(K[e], w))
        z = torch.linalg.solve(K[e], w) - KinvC[e] @ uh
        assert torch.allclose(torch.cat([z, uh]), sol, rtol=1e-10, atol=1e-10)


def test_hdg_penalty_uses_alpha_10_and_own_length():
    hx, hy = 0.3, 0.05
    mesh = I.structured_box_mesh(3, [np.array([0, hx, 2 * hx]), np.array([0, hy, 2 * hy])], [True, False])
    op = HDGIPLocal(mesh, ph.Gas(1.4, Re=50.0, viscous=True))
    want = 10.0 * 16 * 2 * (hx + hy) / (hx * hy)
    assert torch.allclose(op.tau, torch.full_like(op.tau, want), rtol=1e-14)
