"""GPU parity of the forward residual (dgx_rhs) against the FP64 oracle."""
import numpy as np
import pytest
import torch

from paper_2607_16044_b300 import inputs as I
from tests.parity_util import TOL, noise_floor, oracle_rhs_and_scale, quantize32, record, rel_err, scaled_err

pytestmark = pytest.mark.gpu


def _solver(mesh, phys, prec):
    from paper_2607_16044_b300.dgx import Solver
    return Solver(mesh, phys, prec)


def _run(mesh, phys, U, prec):
    s = _solver(mesh, phys, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    Ud = torch.as_tensor(U).to("cuda", dt).contiguous()
    f = s.rhs(Ud)
    s.check()
    return f.double().cpu().numpy()


def _euler():
    return I.Physics(gamma=1.4, viscous=False)


def _ns(Re=200.0):
    return I.Physics(gamma=1.4, Re=Re, Pr=0.72, Ma=0.3, viscous=True)


def _check(mesh, phys, U, prec, name=None, plain=True):
    """Parity: ||f_gpu - f_oracle||_inf per field against the oracle's term scale
    (always) and against ||f_oracle||_inf (``plain``: well-conditioned states).
    FP32 runs compare with the oracle on the FP32-rounded input."""
    got = _run(mesh, phys, U, prec)
    Uref = U if prec == "fp64" else quantize32(U)
    ref, T = oracle_rhs_and_scale(mesh, phys, Uref)
    err, serr = rel_err(got, ref), scaled_err(got, ref, T)
    record(name or f"{mesh.dim}d-p{mesh.p}-{'ns' if phys.viscous else 'euler'}-{mesh.kind}-{prec}",
           rel=err, scaled=serr, E=mesh.n_elem)
    assert serr < TOL[prec], serr
    if plain:
        assert err < TOL[prec], err
    return err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_2d_euler_periodic_boxes(p, prec):
    mesh = I.structured_box_mesh(p, [I.uniform_edges(-1, 1, 9), I.uniform_edges(0, 1.3, 7)], [True, True])
    _check(mesh, _euler(), I.random_state(mesh, 100 + p), prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_2d_ns_channel_walls_stretched(p, prec):
    mesh = I.structured_box_mesh(p, [I.uniform_edges(0, 1, 9), I.wall_stretched_edges(4, 1.5)], [True, False])
    _check(mesh, _ns(), I.random_state(mesh, 200 + p), prec)


@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("p", [2, 4])
def test_2d_curvilinear_rotated(p, viscous):
    mesh = I.rotate_elements(I.warped_mesh(p, [5, 4], [1.0, 1.2], 0.04, periodic=[True, False]), 31 + p)
    _check(mesh, _ns() if viscous else _euler(), I.random_state(mesh, 300 + p), "fp64")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("viscous", [False, True])
def test_3d_boxes(p, viscous, prec):
    cells = {1: 4, 2: 3, 3: 3, 4: 2, 5: 2}[p]
    mesh = I.structured_box_mesh(p, [I.uniform_edges(0, 1, cells), I.uniform_edges(0, 1.2, cells + 1),
                                     I.wall_stretched_edges(1, 1.0)], [True, True, False])
    _check(mesh, _ns() if viscous else _euler(), I.random_state(mesh, 400 + p), prec)


@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("p", [2, 3])
def test_3d_curvilinear_rotated(p, viscous):
    mesh = I.rotate_elements(I.warped_mesh(p, [2, 3, 2], [1.0, 1.0, 1.0], 0.03, periodic=[True, True, False]),
                             41 + p)
    _check(mesh, _ns() if viscous else _euler(), I.random_state(mesh, 500 + p), "fp64")


@pytest.mark.parametrize("viscous", [False, True])
def test_single_element_self_periodic(viscous):
    """E = 1: the element is its own neighbour across every face."""
    mesh = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 1), I.uniform_edges(0, 2, 1)], [True, True])
    _check(mesh, _ns() if viscous else _euler(), I.random_state(mesh, 7), "fp64")


def test_one_element_thick_channel():
    mesh = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 5), I.uniform_edges(-1, 1, 1)], [True, False])
    _check(mesh, _ns(), I.random_state(mesh, 8), "fp64")


def test_vortex_config_full_size():
    """16 x 16 vortex, p = 3: FP64 plain relative error; FP32 against the term
    scale (the state's own FP32 rounding sensitivity is 2.5e-5 in the plain norm)."""
    mesh, phys, U = I.vortex_workload()
    _check(mesh, phys, U, "fp64", "vortex-fp64")
    _check(mesh, phys, U, "fp32", "vortex-fp32", plain=False)


def _sampled(mesh, phys, U, prec, n_sample, seed, name):
    got = _run(mesh, phys, U, prec)
    rng = np.random.default_rng(seed)
    elems = np.unique(np.concatenate([rng.choice(mesh.n_elem, n_sample, replace=False),
                                      [0, mesh.n_elem - 1]]))
    Uref = U if prec == "fp64" else quantize32(U)
    ref, T = oracle_rhs_and_scale(mesh, phys, Uref, elems)
    err, serr = rel_err(got[elems], ref), scaled_err(got[elems], ref, T)
    record(name, rel=err, scaled=serr, E=mesh.n_elem, sampled=len(elems))
    return err, serr


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_channel2d_config_full_size_sampled(prec):
    """256 x 128 wall-stretched channel, p = 4, Re 1000: sampled elements incl. both walls."""
    mesh, phys, U = I.channel2d_workload()
    err, serr = _sampled(mesh, phys, U, prec, 48, 1, f"channel2d-{prec}")
    if prec == "fp64":
        assert serr < TOL[prec] and err < TOL[prec], (err, serr)
    else:
        # The BR1 gradient across the 2e-5-thin wall layers differentiates data
        # with 1e-3 node-to-node noise: FP32 rounding of the state alone moves
        # f by ~5e-5 of its term scale.  Bound FP32 by that floor.
        rng = np.random.default_rng(1)
        elems = np.unique(np.concatenate([rng.choice(mesh.n_elem, 48, replace=False), [0, mesh.n_elem - 1]]))
        floor = noise_floor(mesh, phys, quantize32(U), 2.0 ** -24, elems)
        record("channel2d-fp32-floor", scaled=floor)
        assert serr < max(TOL[prec], 4.0 * floor), (serr, floor)


def test_channel2d_full_size_perturbed_fp32():
    """256 x 128 wall-stretched channel, p = 4, FP32, on a well-conditioned
    state (the Poiseuille profile with 10 % seeded perturbations instead of
    1e-3): sampled elements incl. both walls at the plain FP32 target."""
    mesh, phys, _ = I.channel2d_workload()
    U = I.channel_state(mesh, phys, 2, amp=0.1)
    err, serr = _sampled(mesh, phys, U, "fp32", 48, 1, "channel2d-perturbed-fp32")
    assert err < TOL["fp32"] and serr < TOL["fp32"], (err, serr)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tgv_config_full_size_sampled(prec):
    """32^3 Taylor-Green vortex at Ma 0.1 (p_inf = 71): ill-conditioned in the
    plain norm (FP64 noise floor 3.7e-11), so only the term-scaled error is bounded."""
    mesh, phys, U = I.tgv_workload()
    err, serr = _sampled(mesh, phys, U, prec, 24, 2, f"tgv-{prec}")
    assert serr < TOL[prec], serr


def test_nonfinite_flag_and_invalid_arguments():
    from paper_2607_16044_b300.dgx import DGXError, Solver
    mesh = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 3)] * 2, [True, True])
    s = Solver(mesh, _euler(), "fp64")
    U = torch.as_tensor(I.random_state(mesh, 1)).cuda()
    U[1, 0, 3] = float("nan")
    s.rhs(U)
    with pytest.raises(DGXError) as ei:
        s.check()
    assert ei.value.code == 4
    s.check()                                             # flag cleared
    with pytest.raises(ValueError):
        s.rhs(U.float())                                  # wrong dtype rejected by the binding
    bad = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 3)] * 2, [True, True])
    bad.neighbor[0, 1] = 5                                # not reciprocal
    with pytest.raises(DGXError) as ei:
        Solver(bad, _euler(), "fp64")
    assert ei.value.code == 1


@pytest.mark.parametrize("case", ["2d-ns-walls", "2d-euler-curv", "3d-ns", "3d-euler-p3"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_pipelined_kernels_bit_identical(case, prec):
    """The persistent TMA-fed element kernel and the one-CTA-per-tile kernel
    compute the same arithmetic: residual and ARK step agree bit for bit."""
    from paper_2607_16044_b300.tableaux import ars343_explicit
    if case == "2d-ns-walls":
        mesh = I.structured_box_mesh(4, [I.uniform_edges(0, 1, 13), I.wall_stretched_edges(5, 1.3)], [True, False])
        phys = _ns()
    elif case == "2d-euler-curv":
        mesh = I.rotate_elements(I.warped_mesh(3, [6, 5], [1.0, 1.0], 0.04), 5)
        phys = _euler()
    elif case == "3d-ns":
        mesh = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 4)] * 2 + [I.wall_stretched_edges(2, 1.2)],
                                     [True, True, False])
        phys = _ns()
    else:
        mesh = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 5)] * 3, [True] * 3)
        phys = _euler()
    U0 = I.random_state(mesh, 77)
    dt = torch.float64 if prec == "fp64" else torch.float32
    res = []
    for pipe in (True, False):
        s = _solver(mesh, phys, prec)
        s.set_pipeline(pipe)
        s.set_tableau(*ars343_explicit())
        f = s.rhs(torch.as_tensor(U0).to("cuda", dt).contiguous())
        U = torch.as_tensor(U0).cuda()
        s.ark_step(U, 1e-4)
        s.check()
        res.append((f, U))
    assert torch.equal(res[0][0], res[1][0])
    assert torch.equal(res[0][1], res[1][1])
