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


# ------------------------------------------------------------ curved elements
# The forms take the element geometry of the DG-IP operator (metric terms at
# the nodes and traced to the faces, each element's own area normal), so the
# paper's curved implicit region (walls of bodies) is covered.

def test_hdg_forms_match_brute_force_sheared_affine():
    """Non-rectangular affine elements: the traced metric, the tangential
    part of grad l_q on faces and the area normals all enter."""
    mesh = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 3), I.wall_stretched_edges(1, 1.0)], [True, False])
    xyz = mesh.xyz.copy()
    xyz[:, 0, :] += 0.3 * xyz[:, 1, :]
    mesh = I.Mesh(2, mesh.p, mesh.n_elem, "nodes", xyz, mesh.neighbor, mesh.nbr_face, mesh.orient)
    gas = ph.Gas(1.4, Re=100.0, Pr=0.72, viscous=True)
    op = HDGIPLocal(mesh, gas)
    U = I.random_state(mesh, 4)
    Uh = _perturbed_traces(op, U, 5)
    R, h = op.forms(torch.as_tensor(U), Uh)
    Rb, hb = BruteHDG(mesh, gas, period=[1.0, 100.0]).residual_hdg(U, Uh.numpy())
    assert np.abs(R.numpy() - Rb).max() < 1e-12 * np.abs(Rb).max()
    assert np.abs(h.numpy() - hb).max() < 1e-12 * np.abs(hb).max()


def test_hdg_free_stream_on_curved_elements():
    """A uniform state with its own trace as facet state: every element
    residual vanishes (metric identities) and the two contributions to each
    interior facet cancel (opposite area normals)."""
    mesh = I.rotate_elements(I.warped_mesh(3, [3, 4], [1.0, 1.3], 0.03, mixed=True), 7)
    op = HDGIPLocal(mesh, ph.Gas(1.4, Re=100.0, Pr=0.72, viscous=True))
    U = np.zeros((mesh.n_elem, 4, mesh.N))
    U[:, 0], U[:, 1], U[:, 2], U[:, 3] = 1.2, 0.3, -0.2, 3.0
    U = torch.as_tensor(U)
    R, h = op.forms(U, op.element_traces(op.nodes(U)))
    assert R.abs().max() < 1e-14
    pair = op.gather_neighbor(h, torch.arange(mesh.n_elem))
    assert (h + pair).abs().max() < 1e-13 * h.abs().max()


@pytest.mark.parametrize("viscous", [False, True])
def test_hdg_manufactured_solution_order_on_curved_elements(viscous):
    """The exact solution and its exact facet values on warped elements: the
    element residual approaches -M times the exact rate at the scheme's
    truncation order (p - 1 with the interior penalty, p inviscid); a wrong
    metric term, normal or lift weight leaves an O(1) error."""
    from tests import mms_sympy
    p, mu = 2, 0.01
    fns = mms_sympy.build(2, 1.4, mu if viscous else 0.0, 0.72)
    gas = ph.Gas(1.4, Re=1 / mu if viscous else 0.0, Pr=0.72, viscous=viscous)
    errs = []
    for nc in (8, 16):
        mesh = I.warped_mesh(p, [nc, nc], [1.0, 1.0], 0.02, mixed=True)
        op = HDGIPLocal(mesh, gas)
        U = mms_sympy.evaluate(fns["U"], mesh.xyz, 0.0)
        Xf = op.element_traces(op.nodes(torch.as_tensor(mesh.xyz)))              # [E][2d][d][nfp]
        E, nfp = mesh.n_elem, Xf.shape[-1]
        Uh = mms_sympy.evaluate(fns["U"], Xf.reshape(E * 4, 2, nfp).numpy(), 0.0).reshape(E, 4, 4, nfp)
        exact = -(mms_sympy.evaluate(fns["divFc"], mesh.xyz, 0.0) - mms_sympy.evaluate(fns["divFv"], mesh.xyz, 0.0))
        R, _ = op.forms(torch.as_tensor(U), torch.as_tensor(Uh))
        f = (-R / op.mass()).numpy()
        errs.append(np.sqrt(np.mean((f - exact) ** 2)) / np.sqrt(np.mean(exact ** 2)))
    rate = np.log2(errs[0] / errs[1])
    assert rate > (p - 1 if viscous else p) - 0.4, (errs, rate)
