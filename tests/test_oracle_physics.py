"""Pins of the oracle's pointwise physics and of the operator on closed-form states."""
import os

import numpy as np
import pytest
import torch

from oracle import physics as ph
from oracle.residual import DGOperator
from paper_2607_16044_b300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = {}
    for line in open(os.path.join(GOLDEN, name)):
        if line.startswith("#") or not line.strip():
            continue
        k, lo, hi, dec = line.split()
        rows[k] = (float(lo), float(hi), int(dec))
    return rows


def test_mms_local_mach_and_reynolds_ranges_printed_in_paper():
    """Sec. 5.1.1 prints Ma in [0.95, 1.34] and Re in [424.26, 707.11] for the MMS state."""
    g = _golden("mms_local_numbers.txt")
    s = np.linspace(-1.0, 1.0, 20001)
    rho = s + 4
    U = torch.as_tensor(np.stack([rho, rho, rho, rho ** 2], 1))
    gas = ph.Gas(1.4)
    r, u, p, _ = ph.primitives(U, gas, 2)
    c = ph.sound_speed(U, gas, 2)
    speed = torch.sqrt((u * u).sum(1))
    Ma = (speed / c).numpy()
    Re = (r * speed / 0.01).numpy()                    # rho |u| L / mu, L = 1
    for name, vals in (("Ma", Ma), ("Re", Re)):
        lo, hi, dec = g[name]
        # "approximately": within one unit of the last printed decimal
        tol = 10.0 ** (-dec) * 1.0001
        assert abs(vals.min() - lo) <= tol and abs(vals.max() - hi) <= tol, (name, vals.min(), vals.max())


def test_llf_consistency_and_symmetry():
    rng = np.random.default_rng(0)
    m = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 3)] * 2, [True, True])
    U = torch.as_tensor(I.random_state(m, 1)[:, :, 0])
    V = torch.as_tensor(I.random_state(m, 2)[:, :, 0])
    Sn = torch.as_tensor(rng.standard_normal((U.shape[0], 2)))
    gas = ph.Gas(1.4)
    # consistency: F*(U, U) = F(U).Sn
    assert torch.allclose(ph.llf_flux(U, U, Sn, gas, 2), ph.normal_convective_flux(U, Sn, gas, 2), atol=1e-14)
    # conservation: F*(U, V; n) = -F*(V, U; -n)
    assert torch.allclose(ph.llf_flux(U, V, Sn, gas, 2), -ph.llf_flux(V, U, -Sn, gas, 2), atol=1e-13)


def _rusanov_by_hand(UL, UR, Sn, gamma, d):
    """Local Lax-Friedrichs flux written out from rho, u, p, c for one pair of
    states: 1/2 (F(UL) + F(UR)).Sn - 1/2 lam (UR - UL) with
    lam = max(|u_L.Sn| + c_L |Sn|, |u_R.Sn| + c_R |Sn|), c = sqrt(gamma p / rho)."""
    def parts(U):
        rho = U[0]
        u = U[1:1 + d] / rho
        p = (gamma - 1.0) * (U[d + 1] - 0.5 * rho * float(u @ u))
        c = np.sqrt(gamma * p / rho)
        un = float(u @ Sn)
        F = np.concatenate([[rho * un], rho * u * un + p * Sn, [(U[d + 1] + p) * un]])
        return F, abs(un) + c * np.sqrt(float(Sn @ Sn))
    FL, sL = parts(UL)
    FR, sR = parts(UR)
    lam = max(sL, sR)
    return 0.5 * (FL + FR) - 0.5 * lam * (UR - UL), lam


@pytest.mark.parametrize("d", [2, 3])
def test_llf_wave_speed_closed_form(d):
    """The dissipation of the LLF flux (the convective face flux of the LLF/BR1
    scheme's reading of Sec. 3.3) is -lam/2 (UR - UL) with lam the larger of the two
    sides' |u.Sn| + c|Sn|, written out here from rho, u, p and gamma.  Fails
    for any other wave speed (e.g. lam scaled by a constant or taken from
    one side only)."""
    rng = np.random.default_rng(40 + d)
    gamma = 1.4
    gas = ph.Gas(gamma)
    for _ in range(20):
        rho = rng.uniform(0.5, 2.0, 2)
        vel = rng.uniform(-1.5, 1.5, (2, d))
        p = rng.uniform(0.3, 3.0, 2)
        U = [np.concatenate([[rho[k]], rho[k] * vel[k], [p[k] / (gamma - 1) + 0.5 * rho[k] * vel[k] @ vel[k]]])
             for k in range(2)]
        Sn = rng.standard_normal(d) * rng.uniform(0.1, 3.0)
        want, lam = _rusanov_by_hand(U[0], U[1], Sn, gamma, d)
        got = ph.llf_flux(torch.as_tensor(U[0])[None], torch.as_tensor(U[1])[None],
                          torch.as_tensor(Sn)[None], gas, d)[0].numpy()
        assert np.allclose(got, want, rtol=1e-14, atol=1e-14), (got, want)
        # the dissipation alone: F* - (F_L + F_R)/2 = -lam/2 (U_R - U_L)
        FL = ph.normal_convective_flux(torch.as_tensor(U[0])[None], torch.as_tensor(Sn)[None], gas, d)[0].numpy()
        FR = ph.normal_convective_flux(torch.as_tensor(U[1])[None], torch.as_tensor(Sn)[None], gas, d)[0].numpy()
        diss = got - 0.5 * (FL + FR)
        assert np.allclose(diss, -0.5 * lam * (U[1] - U[0]), rtol=1e-13, atol=1e-14)


def test_llf_worked_example():
    """A hand-computed 1D Riemann pair through the unit normal (1, 0):
    left (rho, u, p) = (1, 0, 1), right (0.125, 0, 0.1), gamma = 1.4 (the
    classical shock-tube data).  c_L = sqrt(1.4), c_R = sqrt(1.12), so
    lam = sqrt(1.4) (both states at rest); the mass flux is then
    -lam/2 (0.125 - 1) = 0.4375 sqrt(1.4), the momentum flux (1 + 0.1)/2 = 0.55
    and the energy flux -lam/2 (0.25 - 2.5) = 1.125 sqrt(1.4)."""
    gas = ph.Gas(1.4)
    UL = torch.tensor([[1.0, 0.0, 0.0, 2.5]], dtype=torch.float64)
    UR = torch.tensor([[0.125, 0.0, 0.0, 0.25]], dtype=torch.float64)
    F = ph.llf_flux(UL, UR, torch.tensor([[1.0, 0.0]], dtype=torch.float64), gas, 2)[0].numpy()
    s = np.sqrt(1.4)
    assert np.allclose(F, [0.4375 * s, 0.55, 0.0, 1.125 * s], rtol=1e-15, atol=1e-15), F


def test_wall_states_and_zero_mass_flux():
    m = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 3)] * 2, [True, True])
    U = torch.as_tensor(I.random_state(m, 3)[:, :, 0])
    Sn = torch.as_tensor(np.random.default_rng(1).standard_normal((U.shape[0], 2)))
    gas = ph.Gas(1.4)
    Um = ph.mirror_state(U, Sn, 2)
    _, u, p, _ = ph.primitives(U, gas, 2)
    _, um, pm, _ = ph.primitives(Um, gas, 2)
    assert torch.allclose(p, pm, rtol=1e-13)                        # same pressure
    assert torch.allclose((u * Sn).sum(1), -(um * Sn).sum(1), atol=1e-13)
    F = ph.llf_flux(U, Um, Sn, gas, 2)
    assert F[:, 0].abs().max() < 1e-14                              # no mass through the wall
    Uw = ph.wall_state(U, 2)
    _, uw, pw, _ = ph.primitives(Uw, gas, 2)
    assert uw.abs().max() == 0 and torch.allclose(pw, p, rtol=1e-13)  # rho e_i kept


@pytest.mark.parametrize("p", [4, 5])
def test_poiseuille_exact_rates_with_walls(p):
    """rho = 1, u = 1 - y^2, v = 0, p const between adiabatic walls y = +-1.

    Continuous rates: d(rho u)/dt = mu u_yy = -2 mu, d(rho E)/dt = mu (u_y^2 + u u_yy)
    = mu (6 y^2 - 2), others zero.  The state is polynomial of degree <= 4, so
    for p >= 4 the discrete operator reproduces these to rounding, even on
    the wall-stretched mesh."""
    mesh = I.structured_box_mesh(p, [I.uniform_edges(0, 0.5, 3), I.wall_stretched_edges(4, 1.4)], [True, False])
    gas = ph.Gas(1.4, Re=100.0, Pr=0.72, viscous=True)
    y = mesh.xyz[:, 1, :]
    rho = np.ones_like(y)
    U = I._stack_state(rho, [1 - y * y, 0 * y], np.full_like(y, 3.0), 1.4)
    f = DGOperator(mesh, gas).residual(torch.as_tensor(U)).numpy()
    mu = gas.mu
    exact = np.stack([0 * y, -2 * mu + 0 * y, 0 * y, mu * (6 * y * y - 2)], 1)
    assert np.max(np.abs(f - exact)) < 2e-11
