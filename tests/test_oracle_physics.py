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
