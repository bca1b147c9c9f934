"""Pins of the DG-IP oracle (Vijayasundaram flux + symmetric interior penalty,
farfield and adiabatic-wall forms, geometry-split interface): the
characteristic splitting against the Jacobian obtained by differentiating the
flux, hand-computed flux values, the dense brute-force weak form, free-stream
preservation, conservation, exact Poiseuille rates and the manufactured
solution's truncation order."""
import numpy as np
import pytest
import torch

from oracle import physics as ph
from oracle.brute import BruteSIPG
from oracle.sipg import OverIntegratedSIPG, SIPGOperator, over_integration_points
from paper_2607_16044_b300 import inputs as I
from tests import mms_sympy


def _states(d, k, seed):
    rng = np.random.default_rng(seed)
    g = 1.4
    rho = rng.uniform(0.5, 2.0, k)
    vel = rng.uniform(-1.5, 1.5, (k, d))
    p = rng.uniform(0.3, 3.0, k)
    U = np.concatenate([rho[:, None], rho[:, None] * vel, (p / (g - 1) + 0.5 * rho * (vel ** 2).sum(1))[:, None]], 1)
    Sn = rng.standard_normal((k, d)) * rng.uniform(0.2, 3.0, (k, 1))
    return torch.as_tensor(U), torch.as_tensor(Sn)


def _flux_jacobian(U, Sn, gas, d):
    """dF_n/dU by differentiating the normal convective flux (autograd)."""
    rows = []
    for k in range(U.shape[0]):
        f = lambda u: ph.normal_convective_flux(u[None], Sn[k:k + 1], gas, d)[0]
        rows.append(torch.autograd.functional.jacobian(f, U[k]))
    return torch.stack(rows)


@pytest.mark.parametrize("d", [2, 3])
def test_split_jacobian_reconstructs_the_flux_jacobian(d):
    """Sec. 3.2: A_n^+ + A_n^- = A_n = dF_n/dU, and A_n^+ (A_n^-) has the
    positive (negative) parts of u.n - c|n|, u.n (d-fold), u.n + c|n| as its
    eigenvalues."""
    gas = ph.Gas(1.4)
    U, Sn = _states(d, 12, 1 + d)
    Ap, Am = ph.split_jacobian(U, Sn, gas, d)
    A = _flux_jacobian(U, Sn, gas, d)
    assert torch.allclose(Ap + Am, A, rtol=1e-12, atol=1e-12)
    rho, u, p, _ = ph.primitives(U, gas, d)
    c = torch.sqrt(1.4 * p / rho)
    sJ = Sn.norm(dim=1)
    un = (u * Sn).sum(1) / sJ
    for k in range(U.shape[0]):
        lam = np.sort(np.array([un[k] - c[k]] + [un[k]] * d + [un[k] + c[k]]) * sJ[k].item())
        ev_p = np.sort(np.linalg.eigvals(Ap[k].numpy()).real)
        ev_m = np.sort(np.linalg.eigvals(Am[k].numpy()).real)
        assert np.allclose(ev_p, np.sort(np.maximum(lam, 0)), atol=1e-10)
        assert np.allclose(ev_m, np.sort(np.minimum(lam, 0)), atol=1e-10)


def test_vijayasundaram_worked_example():
    """Hand-computed: left (rho, u, p) = (1, 0, 1), right (0.125, 0, 0.1),
    gamma 1.4, unit normal (1, 0).  The average state is rho = 0.5625, m = 0,
    rho E = 1.375, so p = 0.55, c^2 = 1.4 p / rho, H = (1.375 + p) / rho and
    u.n = 0.  Then A^+ U_L + A^- U_R = F_n(Ubar) + |A|(U_L - U_R)/2, and with
    u.n = 0 only the two acoustic waves (speed c) carry the jump
    (d rho, d rho E) = (0.875, 2.25): linearised dp = 0.4 * 2.25 = 0.9, wave
    strengths 0.9/(2c^2) each, so |A| dU = (0.9/c, 0, 0, 0.9 H/c) and
    F* = (0.45/c, 0.55, 0, 0.45 H/c)."""
    gas = ph.Gas(1.4)
    UL = torch.tensor([[1.0, 0.0, 0.0, 2.5]], dtype=torch.float64)
    UR = torch.tensor([[0.125, 0.0, 0.0, 0.25]], dtype=torch.float64)
    F = ph.vijayasundaram_flux(UL, UR, torch.tensor([[1.0, 0.0]], dtype=torch.float64), gas, 2)[0].numpy()
    c = np.sqrt(1.4 * 0.55 / 0.5625)
    H = (1.375 + 0.55) / 0.5625
    assert np.allclose(F, [0.45 / c, 0.55, 0.0, 0.45 * H / c], rtol=1e-14, atol=1e-15), F


@pytest.mark.parametrize("d", [2, 3])
def test_vijayasundaram_consistency_conservation_upwinding(d):
    gas = ph.Gas(1.4)
    U, Sn = _states(d, 16, 10 + d)
    V, _ = _states(d, 16, 20 + d)
    # consistency F*(U, U) = F_n(U) (homogeneity of the Euler flux: A_n(U) U = F_n(U))
    assert torch.allclose(ph.vijayasundaram_flux(U, U, Sn, gas, d), ph.normal_convective_flux(U, Sn, gas, d),
                          rtol=1e-13, atol=1e-13)
    # conservation F*(U, V; n) = -F*(V, U; -n)
    assert torch.allclose(ph.vijayasundaram_flux(U, V, Sn, gas, d), -ph.vijayasundaram_flux(V, U, -Sn, gas, d),
                          rtol=1e-13, atol=1e-13)
    # supersonic along n (all eigenvalues of A_n(Ubar) positive): F* = A_n(Ubar) U_own
    rho = torch.ones(16, dtype=torch.float64)
    nh = Sn / Sn.norm(dim=1, keepdim=True)
    Uf = torch.cat([rho[:, None], 3.0 * nh, torch.full((16, 1), 4.5 + 1.0 / 0.4, dtype=torch.float64)], 1)
    Ug = Uf * 1.05
    Ubar = 0.5 * (Uf + Ug)
    A = _flux_jacobian(Ubar, Sn, gas, d)
    want = (A @ Uf.unsqueeze(2)).squeeze(2)
    assert torch.allclose(ph.vijayasundaram_flux(Uf, Ug, Sn, gas, d), want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("d", [2, 3])
def test_farfield_state_solves_its_defining_equation(d):
    """App. B.1.1: A_n(U) U_Gamma = A_n^+(U) U + A_n^-(U) U_inf (A_n from the
    flux derivative); supersonic outflow takes U, supersonic inflow U_inf."""
    gas = ph.Gas(1.4)
    U, Sn = _states(d, 16, 30 + d)
    Ui, _ = _states(d, 16, 40 + d)
    UG = ph.farfield_boundary_state(U, Ui, Sn, gas, d)
    A = _flux_jacobian(U, Sn, gas, d)
    Ap, Am = ph.split_jacobian(U, Sn, gas, d)
    lhs = (A @ UG.unsqueeze(2)).squeeze(2)
    rhs = (Ap @ U.unsqueeze(2)).squeeze(2) + (Am @ Ui.unsqueeze(2)).squeeze(2)
    assert torch.allclose(lhs, rhs, rtol=1e-11, atol=1e-11)
    nh = Sn / Sn.norm(dim=1, keepdim=True)
    for sgn in (1.0, -1.0):
        Us = torch.cat([torch.ones(16, 1, dtype=torch.float64), sgn * 3.0 * nh,
                        torch.full((16, 1), 4.5 + 1.0 / 0.4, dtype=torch.float64)], 1)
        UG = ph.farfield_boundary_state(Us, Ui, Sn, gas, d)
        assert torch.allclose(UG, Us if sgn > 0 else Ui, rtol=1e-13, atol=1e-13)


def test_adiabatic_viscous_flux_has_no_normal_heat_flux():
    d = 2
    gas = ph.Gas(1.4, Re=100.0, Pr=0.72, viscous=True)
    U, Sn = _states(d, 8, 50)
    Q = torch.as_tensor(np.random.default_rng(51).standard_normal((8, d, d + 2)))
    Fw = ph.adiabatic_viscous_flux(U, Q, Sn, gas, d)
    F = ph.viscous_flux(U, Q, gas, d)
    u, gu, ge = ph.velocity_temperature_gradients(U, Q, gas, d)
    # momentum rows unchanged; energy: the normal heat flux removed, the tangential one kept
    assert torch.allclose(Fw[:, :, :d + 1], F[:, :, :d + 1], rtol=1e-15, atol=1e-15)
    work = (Fw[:, :, 1:d + 1] * u.unsqueeze(1)).sum(2)              # tau . u per direction
    heat_w = Fw[:, :, d + 1] - work
    assert torch.allclose((heat_w * Sn).sum(1), torch.zeros(8, dtype=torch.float64), atol=1e-13)
    t = torch.stack([-Sn[:, 1], Sn[:, 0]], 1)
    heat = F[:, :, d + 1] - work
    assert torch.allclose((heat_w * t).sum(1), (heat * t).sum(1), rtol=1e-12, atol=1e-13)


def _gas(viscous=True, Re=50.0):
    return ph.Gas(1.4, Re=Re, Pr=0.72, viscous=viscous)


@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_brute_force_2d_rotated_walls(p, viscous):
    m = I.rotate_elements(I.structured_box_mesh(p, [I.uniform_edges(0, 1, 3), I.wall_stretched_edges(1, 1.0)],
                                                [True, False]), 11 + p)
    U = I.random_state(m, 7)
    f1 = SIPGOperator(m, _gas(viscous)).residual(torch.as_tensor(U)).numpy()
    f2 = BruteSIPG(m, _gas(viscous), period=[1.0, 100.0]).residual_sipg(U)
    assert np.abs(f1 - f2).max() / np.abs(f1).max() < 1e-12


def test_brute_force_2d_sheared_affine():
    """Non-rectangular affine elements (a sheared periodic mesh): the face
    metric traces, the tangential part of grad l_q on faces and the averaged
    area normal all enter."""
    m = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 3), I.uniform_edges(0, 1, 2)], [True, True])
    xyz = m.xyz.copy()
    xyz[:, 0, :] += 0.3 * xyz[:, 1, :]
    m = I.Mesh(2, m.p, m.n_elem, "nodes", xyz, m.neighbor, m.nbr_face, m.orient)
    U = I.random_state(m, 9)
    f1 = SIPGOperator(m, _gas()).residual(torch.as_tensor(U)).numpy()
    brute = BruteSIPG(m, _gas(), period=[1.0, 1.0])
    brute.locate = _sheared_locate(brute, 0.3)
    f2 = brute.residual_sipg(U)
    assert np.abs(f1 - f2).max() / np.abs(f1).max() < 1e-12


def _sheared_locate(brute, s):
    """Periodic images of the sheared unit square are shifted by (1, 0) and (s, 1)."""
    import itertools

    def locate(e, x):
        Ainv = np.linalg.inv(brute.A[e])
        best = None
        for i, j in itertools.product([-1, 0, 1], repeat=2):
            xi = Ainv @ (x + np.array([i + s * j, j]) - brute.x0[e])
            err = np.max(np.abs(xi)) - 1.0
            if best is None or err < best[0]:
                best = (err, xi)
        assert best[0] < 1e-9
        return best[1]
    return locate


@pytest.mark.parametrize("viscous", [False, True])
def test_brute_force_3d_rotated_walls(viscous):
    m = I.rotate_elements(I.structured_box_mesh(2, [I.uniform_edges(0, 1, 2), I.uniform_edges(0, 1.5, 2),
                                                    I.wall_stretched_edges(1, 1.0)], [True, True, False]), 5)
    U = I.random_state(m, 8)
    f1 = SIPGOperator(m, _gas(viscous)).residual(torch.as_tensor(U)).numpy()
    f2 = BruteSIPG(m, _gas(viscous), period=[1.0, 1.5, 100.0]).residual_sipg(U)
    assert np.abs(f1 - f2).max() / np.abs(f1).max() < 1e-12


@pytest.mark.parametrize("viscous", [False, True])
def test_brute_force_farfield(viscous):
    """Farfield boundaries (tag 1) on both ends of y, free stream at an angle."""
    m = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 3), I.uniform_edges(0, 1, 2)], [True, False], wall_tag=1)
    Uinf = np.array([1.1, 0.4, -0.3, 2.0 / 0.4 + 0.5 * (0.4 ** 2 + 0.3 ** 2) / 1.1])
    U = I.random_state(m, 10)
    f1 = SIPGOperator(m, _gas(viscous), U_inf=Uinf).residual(torch.as_tensor(U)).numpy()
    f2 = BruteSIPG(m, _gas(viscous), period=[1.0, 100.0]).residual_sipg(U, U_inf=Uinf)
    assert np.abs(f1 - f2).max() / np.abs(f1).max() < 1e-12


def test_brute_force_interface():
    """Geometry split: the middle column of elements implicit (state U_im), the
    rest explicit; interface faces use the averaged K in the adjoint term and
    feed only the explicit side; implicit elements get f = 0."""
    m = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 4), I.wall_stretched_edges(1, 1.0)], [True, False])
    ix = np.arange(m.n_elem) % 4
    explicit = ix != 2
    U = I.random_state(m, 11)
    Uim = I.random_state(m, 12)
    f1 = SIPGOperator(m, _gas(), explicit=explicit).residual(torch.as_tensor(U), torch.as_tensor(Uim)).numpy()
    f2 = BruteSIPG(m, _gas(), period=[1.0, 100.0]).residual_sipg(U, explicit=explicit, U_im=Uim)
    assert np.abs(f1 - f2).max() / np.abs(f1).max() < 1e-12
    assert np.all(f1[~explicit] == 0)
    # only the interface faces see U_im: elements away from column 2 are unchanged
    far = (ix == 0)
    f_all = SIPGOperator(m, _gas()).residual(torch.as_tensor(U)).numpy()
    assert np.abs(f1[far] - f_all[far]).max() < 1e-13 * np.abs(f_all).max()


@pytest.mark.parametrize("case", ["box", "stretched", "warped2", "warped3"])
def test_free_stream_preservation(case):
    if case == "box":
        m = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 4)] * 2, [True, True])
    elif case == "stretched":
        m = I.structured_box_mesh(4, [I.uniform_edges(0, 1, 3), I.wall_stretched_edges(3, 1.6, 0.0, 1.0)],
                                  [True, True])
    elif case == "warped2":
        m = I.rotate_elements(I.warped_mesh(3, [3, 4], [1.0, 1.3], 0.05), 2)
    else:
        m = I.warped_mesh(2, [2, 2, 2], [1.0, 1.0, 1.0], 0.04)
    d = m.dim
    U = np.zeros((m.n_elem, d + 2, m.N))
    U[:, 0] = 1.2
    U[:, 1] = 0.3
    U[:, 2] = -0.2
    if d == 3:
        U[:, 3] = 0.1
    U[:, d + 1] = 3.0
    f = SIPGOperator(m, _gas()).residual(torch.as_tensor(U)).numpy()
    # scale |F^c| (~4) over the smallest element size (the penalty adds (k+1)^2 / l)
    hmin = 1e-2 if case != "stretched" else 5e-3
    assert np.abs(f).max() < 1e-13 * 4.0 / hmin


@pytest.mark.parametrize("viscous", [False, True])
def test_conservation_periodic(viscous):
    m = I.rotate_elements(I.warped_mesh(3, [3, 4], [1.0, 1.3], 0.05), 4)
    op = SIPGOperator(m, _gas(viscous))
    U = torch.as_tensor(I.random_state(m, 5))
    f = op.residual(U)
    w = op.basis.w
    W = torch.as_tensor(np.multiply.outer(w, w).reshape(-1)) * op.geo.J.reshape(op.E, -1)
    tot = (f * W.unsqueeze(1)).sum((0, 2))
    scale = (f.abs() * W.unsqueeze(1)).sum((0, 2))
    assert (tot.abs() / scale).max() < 1e-13


def test_penalty_and_length_closed_form():
    """tau = alpha (k+1)^2 / l, l = |T| / |dT|: for an h_x x h_y box
    1/l = 2 (h_x + h_y) / (h_x h_y); on a face the larger of the two sides'."""
    hx = np.array([0.1, 0.3, 0.2])
    hy = np.array([0.05, 0.4])
    ex = np.concatenate([[0.0], np.cumsum(hx)])
    ey = np.concatenate([[0.0], np.cumsum(hy)])
    m = I.structured_box_mesh(3, [ex, ey], [True, False])
    op = SIPGOperator(m, _gas(), alpha=1.0)
    i, j = np.arange(m.n_elem) % 3, np.arange(m.n_elem) // 3
    want = 2 * (hx[i] + hy[j]) / (hx[i] * hy[j])
    assert np.allclose(op.inv_l.numpy(), want, rtol=1e-14)
    for e in range(m.n_elem):
        for f in range(4):
            nb = m.neighbor[e, f]
            ref = want[e] if nb < 0 else max(want[e], want[nb])
            assert abs(op.tau[e, f].item() - 16.0 * ref) < 1e-12 * 16 * ref


@pytest.mark.parametrize("p", [4, 5])
def test_poiseuille_exact_rates_with_walls(p):
    """rho = 1, u = 1 - y^2, v = 0, p const between adiabatic walls: the state is
    continuous and equals the no-slip wall state at the walls, so the penalty
    and adjoint-consistency terms vanish and the operator reproduces the
    exact rates d(rho u)/dt = -2 mu, d(rho E)/dt = mu (6 y^2 - 2)."""
    mesh = I.structured_box_mesh(p, [I.uniform_edges(0, 0.5, 3), I.wall_stretched_edges(4, 1.4)], [True, False])
    gas = ph.Gas(1.4, Re=100.0, Pr=0.72, viscous=True)
    y = mesh.xyz[:, 1, :]
    U = I._stack_state(np.ones_like(y), [1 - y * y, 0 * y], np.full_like(y, 3.0), 1.4)
    f = SIPGOperator(mesh, gas).residual(torch.as_tensor(U)).numpy()
    mu = gas.mu
    exact = np.stack([0 * y, -2 * mu + 0 * y, 0 * y, mu * (6 * y * y - 2)], 1)
    assert np.max(np.abs(f - exact)) < 2e-11


@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("p", [2, 3])
def test_manufactured_solution_truncation_order(p, viscous):
    """f(U_e) -> -div(F^c - F^nu)(U_e) at the scheme's truncation-error rate
    (Sec. 5.1.1 manufactured solution, derived symbolically from Sec. 2): the
    nodal truncation error is O(h^p) for the convective part and O(h^(p-1))
    for interior-penalty viscous terms (penalty ~ 1/h on O(h^(p+1)) jumps over
    the O(h) mass); a wrong viscous average, lift or metric term is O(1)."""
    mu = 0.01
    fns = mms_sympy.build(2, 1.4, mu if viscous else 0.0, 0.72)
    gas = ph.Gas(1.4, Re=1 / mu if viscous else 0.0, Pr=0.72, viscous=viscous)
    errs = []
    for nc in (8, 16):
        m = I.structured_box_mesh(p, [I.uniform_edges(0, 1, nc)] * 2, [True, True])
        U = mms_sympy.evaluate(fns["U"], m.xyz, 0.0)
        exact = -(mms_sympy.evaluate(fns["divFc"], m.xyz, 0.0) - mms_sympy.evaluate(fns["divFv"], m.xyz, 0.0))
        f = SIPGOperator(m, gas).residual(torch.as_tensor(U)).numpy()
        errs.append(np.sqrt(np.mean((f - exact) ** 2)) / np.sqrt(np.mean(exact ** 2)))
    rate = np.log2(errs[0] / errs[1])
    assert rate > (p - 1 if viscous else p) - 0.4, (errs, rate)


# ---------------------------------------------------------------- over-integration
# The order-3k rule of Sec. 5 on the degree-k space: the oracle goes through
# collocation at the M points; the brute force integrates every volume and face
# integrand pointwise at the M-point rule, with its own basis and mass matrix.

def test_over_integration_points_are_order_3k():
    for p in range(1, 6):
        M = over_integration_points(p)
        assert 2 * M - 1 >= 3 * p and 2 * (M - 1) - 1 < 3 * p


@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("p,M", [(1, 3), (2, 3), (2, 4), (3, 5)])
def test_over_integration_brute_force_2d_walls(p, M, viscous):
    m = I.structured_box_mesh(p, [I.uniform_edges(0, 1, 3), I.wall_stretched_edges(2, 1.0)], [True, False])
    U = I.random_state(m, 20 + p)
    f1 = OverIntegratedSIPG(m, _gas(viscous), M=M).residual(torch.as_tensor(U)).numpy()
    f2 = BruteSIPG(m, _gas(viscous), period=[1.0, 100.0]).residual_sipg_oi(U, M)
    assert np.abs(f1 - f2).max() / np.abs(f1).max() < 1e-12


def test_over_integration_brute_force_3d():
    m = I.structured_box_mesh(1, [I.uniform_edges(0, 1, 2), I.uniform_edges(0, 1.5, 2),
                                  I.wall_stretched_edges(1, 1.0)], [True, True, False])
    U = I.random_state(m, 23)
    f1 = OverIntegratedSIPG(m, _gas(True), M=3).residual(torch.as_tensor(U)).numpy()
    f2 = BruteSIPG(m, _gas(True), period=[1.0, 1.5, 100.0]).residual_sipg_oi(U, 3)
    assert np.abs(f1 - f2).max() / np.abs(f1).max() < 1e-12


@pytest.mark.parametrize("viscous", [False, True])
def test_over_integration_brute_force_farfield(viscous):
    m = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 3), I.uniform_edges(0, 1, 2)], [True, False], wall_tag=1)
    Uinf = np.array([1.1, 0.4, -0.3, 2.0 / 0.4 + 0.5 * (0.4 ** 2 + 0.3 ** 2) / 1.1])
    U = I.random_state(m, 24)
    f1 = OverIntegratedSIPG(m, _gas(viscous), U_inf=Uinf).residual(torch.as_tensor(U)).numpy()
    f2 = BruteSIPG(m, _gas(viscous), period=[1.0, 100.0]).residual_sipg_oi(U, 4, U_inf=Uinf)
    assert np.abs(f1 - f2).max() / np.abs(f1).max() < 1e-12


def test_over_integration_brute_force_interface():
    m = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 4), I.wall_stretched_edges(1, 1.0)], [True, False])
    explicit = (np.arange(m.n_elem) % 4) != 2
    U, Uim = I.random_state(m, 25), I.random_state(m, 26)
    f1 = OverIntegratedSIPG(m, _gas(), explicit=explicit).residual(torch.as_tensor(U), torch.as_tensor(Uim)).numpy()
    f2 = BruteSIPG(m, _gas(), period=[1.0, 100.0]).residual_sipg_oi(U, 4, explicit=explicit, U_im=Uim)
    assert np.abs(f1 - f2).max() / np.abs(f1).max() < 1e-12
    assert np.all(f1[~explicit] == 0)


@pytest.mark.parametrize("viscous", [False, True])
def test_over_integration_with_p_plus_1_points_is_the_collocated_operator(viscous):
    """M = k + 1: the M points are the solution nodes, interpolation and
    projection are identities, and the operator is the collocated one."""
    m = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 3), I.wall_stretched_edges(2, 1.0)], [True, False])
    U = torch.as_tensor(I.random_state(m, 27))
    f1 = OverIntegratedSIPG(m, _gas(viscous), M=4).residual(U)
    f0 = SIPGOperator(m, _gas(viscous)).residual(U)
    assert torch.equal(f1, f0)


def test_over_integration_free_stream_and_conservation():
    m = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 3), I.wall_stretched_edges(3, 1.6, 0.0, 1.0)],
                              [True, True])
    op = OverIntegratedSIPG(m, _gas(True))
    U = np.zeros((m.n_elem, 4, m.N))
    U[:, 0], U[:, 1], U[:, 2], U[:, 3] = 1.2, 0.3, -0.2, 3.0
    assert op.residual(torch.as_tensor(U)).abs().max() < 1e-13 * 4.0 / 5e-3
    f = op.residual(torch.as_tensor(I.random_state(m, 28)))
    _, w = np.polynomial.legendre.leggauss(3)
    W = torch.as_tensor(np.multiply.outer(w, w).reshape(-1) * np.prod(m.size, 1)[:, None] / 4.0)
    tot = (f * W.unsqueeze(1)).sum((0, 2))
    scale = (f.abs() * W.unsqueeze(1)).sum((0, 2))
    assert (tot.abs() / scale).max() < 1e-13


def test_over_integration_changes_the_aliased_operator():
    """The rule matters: for a rough state the M-point operator differs from
    the collocated one (aliasing of the nonlinear fluxes), and raising M
    further changes it less and less (convergence to the exact integrals)."""
    m = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 3), I.uniform_edges(0, 1, 2)], [True, True])
    U = torch.as_tensor(I.random_state(m, 29))
    f = {M: OverIntegratedSIPG(m, _gas(True), M=M).residual(U) for M in (3, 4, 6, 8, 10)}
    d = [float((f[M] - f[10]).abs().max() / f[10].abs().max()) for M in (3, 4, 6, 8)]
    assert d[0] > 1e-4
    assert d[0] > d[1] > d[2] > d[3]


def test_vijayasundaram_derivative_at_a_zero_eigenvalue_is_the_mean_of_the_one_sided_ones():
    """A_n^+(Ubar) U+ + A_n^-(Ubar) U- is not differentiable where an
    eigenvalue of A_n(Ubar) vanishes (here u.n = 0 exactly: no normal
    velocity on either side).  The oracle's derivative there is the mean of
    the derivatives from both sides, measured by one-sided differences."""
    gas = ph.Gas(1.4)
    d = 2
    UL = torch.tensor([[1.1, 0.4, 0.0, 2.7]], dtype=torch.float64)
    UR = torch.tensor([[0.9, -0.3, 0.0, 2.4]], dtype=torch.float64)
    Sn = torch.tensor([[0.0, 1.3]], dtype=torch.float64)      # normal along y: u.n = v = 0
    w = torch.tensor([[0.2, -0.4, 1.0, 0.3]], dtype=torch.float64)  # moves v through 0
    lam = torch.tensor([[0.7, -0.2, 0.5, 1.1]], dtype=torch.float64)

    def F(t):
        return (ph.vijayasundaram_flux(UL + t * w, UR + t * w, Sn, gas, d) * lam).sum()

    h = 1e-7
    right = (F(h) - F(0.0)) / h
    left = (F(0.0) - F(-h)) / h
    assert abs(right - left) > 1e-3 * abs(right)               # a genuine kink
    UL_ = UL.clone().requires_grad_(True)
    UR_ = UR.clone().requires_grad_(True)
    f = (ph.vijayasundaram_flux(UL_, UR_, Sn, gas, d) * lam).sum()
    gL, gR = torch.autograd.grad(f, (UL_, UR_))
    deriv = float(((gL + gR) * w).sum())
    assert abs(deriv - 0.5 * float(left + right)) < 1e-6 * abs(float(right))


# ------------------------------------------- over-integration on curved elements
# f = J^-1 Pi (J' f'(I U)): the element map is the degree-k interpolant of the
# node coordinates, evaluated at the M points for the point operator.  Affine
# non-box elements go against the pointwise brute force; curved elements
# against conservation, free stream and the manufactured-solution rate.

@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("p,M", [(1, 3), (2, 4)])
def test_over_integration_brute_force_2d_rotated(p, M, viscous):
    m = I.rotate_elements(I.structured_box_mesh(p, [I.uniform_edges(0, 1, 3), I.wall_stretched_edges(1, 1.0)],
                                                [True, False]), 31 + p)
    U = I.random_state(m, 32)
    f1 = OverIntegratedSIPG(m, _gas(viscous), M=M).residual(torch.as_tensor(U)).numpy()
    f2 = BruteSIPG(m, _gas(viscous), period=[1.0, 100.0]).residual_sipg_oi(U, M)
    assert np.abs(f1 - f2).max() / np.abs(f1).max() < 1e-12


def test_over_integration_brute_force_2d_sheared_affine():
    m = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 3), I.uniform_edges(0, 1, 2)], [True, True])
    xyz = m.xyz.copy()
    xyz[:, 0, :] += 0.3 * xyz[:, 1, :]
    m = I.Mesh(2, m.p, m.n_elem, "nodes", xyz, m.neighbor, m.nbr_face, m.orient)
    U = I.random_state(m, 33)
    f1 = OverIntegratedSIPG(m, _gas()).residual(torch.as_tensor(U)).numpy()
    brute = BruteSIPG(m, _gas(), period=[1.0, 1.0])
    brute.locate = _sheared_locate(brute, 0.3)
    f2 = brute.residual_sipg_oi(U, 4)
    assert np.abs(f1 - f2).max() / np.abs(f1).max() < 1e-12


def test_over_integration_brute_force_3d_rotated():
    m = I.rotate_elements(I.structured_box_mesh(1, [I.uniform_edges(0, 1, 2), I.uniform_edges(0, 1.5, 2),
                                                    I.wall_stretched_edges(1, 1.0)], [True, True, False]), 34)
    U = I.random_state(m, 35)
    f1 = OverIntegratedSIPG(m, _gas(True), M=3).residual(torch.as_tensor(U)).numpy()
    f2 = BruteSIPG(m, _gas(True), period=[1.0, 1.5, 100.0]).residual_sipg_oi(U, 3)
    assert np.abs(f1 - f2).max() / np.abs(f1).max() < 1e-12


def _warped(d):
    """Warps whose J is no degree-p polynomial (J' at the M points differs
    from the interpolant of the nodal J)."""
    if d == 2:
        return I.rotate_elements(I.warped_mesh(3, [3, 4], [1.0, 1.3], 0.03, mixed=True), 36)
    return I.warped_mesh(3, [3, 3, 2], [1.0, 1.0, 1.0], 0.02, mixed=True)


@pytest.mark.parametrize("d", [2, 3])
def test_over_integration_curved_conservation(d):
    """sum_q w_q J_q f_q = sum_m omega_m J'_m f'_m: the point operator's
    total, which the interior faces cancel on a periodic mesh.  Dropping the
    J'/J weights (f = Pi f') breaks it by the O(h) variation of J."""
    m = _warped(d)
    op = OverIntegratedSIPG(m, _gas(True))
    f = op.residual(torch.as_tensor(I.random_state(m, 37)))
    w = np.polynomial.legendre.leggauss(m.p + 1)[1]
    Wq = w
    for _ in range(d - 1):
        Wq = np.multiply.outer(w, Wq)
    W = torch.as_tensor(Wq.reshape(-1))[None, None, :] * op.J
    tot = (f * W).sum((0, 2))
    scale = (f.abs() * W).sum((0, 2))
    assert (tot.abs() / scale).max() < 1e-13
    unweighted = (op.project(op.inner.residual(op.interpolate(torch.as_tensor(I.random_state(m, 37))))) * W).sum((0, 2))
    assert (unweighted.abs() / scale).max() > 1e-6


@pytest.mark.parametrize("d", [2, 3])
def test_over_integration_curved_free_stream(d):
    """A uniform state stays at rest: the point operator's element maps at
    the M points keep their face normals equal across faces (the 3D curl
    form through the Lobatto interpolant) and the metric identities."""
    m = _warped(d)
    U = np.zeros((m.n_elem, d + 2, m.N))
    U[:, 0], U[:, 1], U[:, 2], U[:, d + 1] = 1.2, 0.3, -0.2, 3.0
    if d == 3:
        U[:, 3] = 0.1
    f = OverIntegratedSIPG(m, _gas(True)).residual(torch.as_tensor(U))
    assert f.abs().max() < 1e-13 * 4.0 / 1e-2


def test_over_integration_curved_with_p_plus_1_points_is_the_collocated_operator():
    m = _warped(2)
    U = torch.as_tensor(I.random_state(m, 38))
    f1 = OverIntegratedSIPG(m, _gas(True), M=m.p + 1).residual(U)
    f0 = SIPGOperator(m, _gas(True)).residual(U)
    assert (f1 - f0).abs().max() < 1e-13 * f0.abs().max()


@pytest.mark.parametrize("viscous", [False, True])
def test_over_integration_curved_manufactured_solution_order(viscous):
    """The manufactured solution on warped elements: the truncation error
    falls at the scheme's rate (as on boxes); a wrong metric or J weighting
    at the M points leaves an O(1) error."""
    p = 2
    mu = 0.01
    fns = mms_sympy.build(2, 1.4, mu if viscous else 0.0, 0.72)
    gas = ph.Gas(1.4, Re=1 / mu if viscous else 0.0, Pr=0.72, viscous=viscous)
    errs = []
    for nc in (8, 16):
        m = I.warped_mesh(p, [nc, nc], [1.0, 1.0], 0.02, mixed=True)
        U = mms_sympy.evaluate(fns["U"], m.xyz, 0.0)
        exact = -(mms_sympy.evaluate(fns["divFc"], m.xyz, 0.0) - mms_sympy.evaluate(fns["divFv"], m.xyz, 0.0))
        f = OverIntegratedSIPG(m, gas).residual(torch.as_tensor(U)).numpy()
        errs.append(np.sqrt(np.mean((f - exact) ** 2)) / np.sqrt(np.mean(exact ** 2)))
    rate = np.log2(errs[0] / errs[1])
    assert rate > (p - 1 if viscous else p) - 0.4, (errs, rate)
