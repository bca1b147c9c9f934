"""GPU parity of the hand-written adjoint (dgx_rhs_vjp, ARK adjoint) against the oracle."""
import numpy as np
import pytest
import torch

from oracle import ark
from oracle.residual import DGOperator
from oracle.vjp import vjp, vjp_rows
from paper_2607_16044_b300 import inputs as I
from tests.parity_util import TOL, gas_of, quantize32, record, rel_err

pytestmark = pytest.mark.gpu


def _gpu_vjp(mesh, phys, U, lam, prec):
    from paper_2607_16044_b300.dgx import Solver
    s = Solver(mesh, phys, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    g = s.rhs_vjp(torch.as_tensor(U).to("cuda", dt).contiguous(), torch.as_tensor(lam).to("cuda", dt).contiguous())
    s.check()
    return g.double().cpu().numpy()


def _oracle_vjp(mesh, phys, U, lam, elems=None):
    op = DGOperator(mesh, gas_of(phys))
    if elems is None:
        return vjp(op, torch.as_tensor(U), torch.as_tensor(lam)).numpy()
    return vjp_rows(op, torch.as_tensor(U), torch.as_tensor(lam), elems).numpy()


def _check(mesh, phys, U, lam, prec, name):
    got = _gpu_vjp(mesh, phys, U, lam, prec)
    if prec == "fp32":
        U, lam = quantize32(U), quantize32(lam)
    ref = _oracle_vjp(mesh, phys, U, lam)
    err = rel_err(got, ref)
    record(name, rel=err, E=mesh.n_elem)
    assert err < TOL[prec], err


def _euler():
    return I.Physics(gamma=1.4, viscous=False)


def _ns(Re=200.0):
    return I.Physics(gamma=1.4, Re=Re, Pr=0.72, Ma=0.3, viscous=True)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_vjp_2d_boxes_walls(p, viscous, prec):
    mesh = I.structured_box_mesh(p, [I.uniform_edges(0, 1, 7), I.wall_stretched_edges(3, 1.4)], [True, False])
    U = I.random_state(mesh, 600 + p)
    lam = I.gaussian_cotangent(U.shape, 700 + p)
    _check(mesh, _ns() if viscous else _euler(), U, lam, prec, f"vjp-2d-p{p}-{'ns' if viscous else 'euler'}-{prec}")


@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("p", [2, 4])
def test_vjp_2d_curvilinear_rotated(p, viscous):
    mesh = I.rotate_elements(I.warped_mesh(p, [5, 4], [1.0, 1.2], 0.04, periodic=[True, False]), 61 + p)
    U = I.random_state(mesh, 800 + p)
    lam = I.gaussian_cotangent(U.shape, 900 + p)
    _check(mesh, _ns() if viscous else _euler(), U, lam, "fp64", f"vjp-2d-curv-p{p}-{'ns' if viscous else 'euler'}")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("p", [1, 3, 5])
def test_vjp_3d_boxes(p, viscous, prec):
    cells = {1: 3, 3: 2, 5: 2}[p]
    mesh = I.structured_box_mesh(p, [I.uniform_edges(0, 1, cells), I.uniform_edges(0, 1.2, cells + 1),
                                     I.wall_stretched_edges(1, 1.0)], [True, True, False])
    U = I.random_state(mesh, 1000 + p)
    lam = I.gaussian_cotangent(U.shape, 1100 + p)
    _check(mesh, _ns() if viscous else _euler(), U, lam, prec, f"vjp-3d-p{p}-{'ns' if viscous else 'euler'}-{prec}")


@pytest.mark.parametrize("viscous", [False, True])
def test_vjp_3d_curvilinear_rotated(viscous):
    mesh = I.rotate_elements(I.warped_mesh(2, [2, 3, 2], [1.0, 1.0, 1.0], 0.03, periodic=[True, True, False]), 71)
    U = I.random_state(mesh, 1200)
    lam = I.gaussian_cotangent(U.shape, 1300)
    _check(mesh, _ns() if viscous else _euler(), U, lam, "fp64", f"vjp-3d-curv-{'ns' if viscous else 'euler'}")


def test_vjp_single_element_self_periodic():
    mesh = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 1), I.uniform_edges(0, 2, 1)], [True, True])
    U = I.random_state(mesh, 3)
    _check(mesh, _ns(), U, I.gaussian_cotangent(U.shape, 4), "fp64", "vjp-single-element")


def test_vjp_channel2d_full_size_sampled():
    """Full 256 x 128 p = 4 channel, seeded Gaussian cotangent: sampled rows vs the oracle."""
    mesh, phys, U = I.channel2d_workload()
    lam = I.gaussian_cotangent(U.shape, 102)
    got = _gpu_vjp(mesh, phys, U, lam, "fp64")
    rng = np.random.default_rng(5)
    rows = np.unique(np.concatenate([rng.choice(mesh.n_elem, 12, replace=False), [0, mesh.n_elem - 1]]))
    ref = _oracle_vjp(mesh, phys, U, lam, rows)
    err = rel_err(got[rows], ref)
    record("vjp-channel2d-fp64", rel=err, sampled=len(rows))
    assert err < 1e-12, err


def test_autograd_function_and_adjoint_identity():
    """torch.autograd.Function backward = dgx_rhs_vjp; <lam, J v> = <J^T lam, v> with J v by central FD."""
    from paper_2607_16044_b300.dgx import Solver, residual
    mesh = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 6), I.wall_stretched_edges(2, 1.3)], [True, False])
    phys = _ns()
    s = Solver(mesh, phys, "fp64")
    U = torch.as_tensor(I.random_state(mesh, 7)).cuda().requires_grad_(True)
    lam = torch.as_tensor(I.gaussian_cotangent(U.shape, 8)).cuda()
    f = residual(U, s)
    (g,) = torch.autograd.grad(f, U, lam)
    v = torch.as_tensor(I.gaussian_cotangent(U.shape, 9)).cuda()
    eps = 1e-6 * U.detach().abs().max().item()
    with torch.no_grad():
        jv = (s.rhs(U + eps * v) - s.rhs(U - eps * v)) / (2 * eps)
    lhs = (lam * jv).sum().item()
    rhs = (g * v).sum().item()
    assert abs(lhs - rhs) <= 1e-6 * abs(rhs), (lhs, rhs)


def test_ark_adjoint_step_matches_oracle():
    """One ARS(3,4,3) step's adjoint (stage checkpoints + reverse recurrence) vs the oracle's."""
    from paper_2607_16044_b300.dgx import Solver
    from paper_2607_16044_b300.tableaux import ars343_explicit
    mesh = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 6), I.wall_stretched_edges(2, 1.3)], [True, False])
    phys = _ns()
    U0 = I.random_state(mesh, 11)
    lam0 = I.gaussian_cotangent(U0.shape, 12)
    dt = 2e-5
    s = Solver(mesh, phys, "fp64")
    s.set_tableau(*ars343_explicit())
    U = torch.as_tensor(U0).cuda()
    stages = s.stage_buffer()
    s.ark_step_stages(U, dt, stages)
    lam = torch.as_tensor(lam0).cuda()
    s.ark_adjoint_step(stages, lam, dt)
    s.check()
    op = DGOperator(mesh, gas_of(phys))
    A, b, c = ark.ars343()
    Uref, ys, _ = ark.erk_step(op.residual, torch.as_tensor(U0), dt, A, b, return_stages=True)
    assert rel_err(U.cpu().numpy(), Uref.numpy()) < 1e-13
    got_ys = np.concatenate([s.stage_state(stages, i).cpu().numpy() for i in range(4)])
    assert rel_err(got_ys, torch.stack(ys).numpy().reshape(-1, *U0.shape[1:])) < 1e-13
    ref = ark.erk_adjoint_step(lambda y, mu: vjp(op, y, mu), ys, torch.as_tensor(lam0), dt, A, b).numpy()
    got = lam.cpu().numpy()
    err = rel_err(got - lam0, ref - lam0)
    record("ark-adjoint-fp64", rel=err)
    assert err < TOL["fp64"], err


def test_multi_step_adjoint_checkpointing():
    """Gradient through 5 ARK steps (checkpoint U_n, recompute stages) vs the oracle's
    reverse recurrence.  The vortex is shifted off the element faces: centred on
    a face (or on the periodic seam) it is mirror-symmetric there, |u.n| + c
    ties exactly on both sides, and the LLF flux has a kink whose one-sided
    derivative depends on rounding -- neither side is "the" gradient there."""
    from paper_2607_16044_b300.dgx import Solver, adjoint_trajectory
    from paper_2607_16044_b300.tableaux import ars343_explicit
    mesh, phys, _ = I.vortex_workload(p=2, cells=6)
    U0 = I.isentropic_vortex(mesh, t=0.37, gamma=phys.gamma)
    lamN = I.gaussian_cotangent(U0.shape, 13)
    dt, nsteps = 0.05, 5
    s = Solver(mesh, phys, "fp64")
    s.set_tableau(*ars343_explicit())
    UN, lam0 = adjoint_trajectory(s, torch.as_tensor(U0).cuda(), dt, nsteps, torch.as_tensor(lamN).cuda())
    s.check()
    op = DGOperator(mesh, gas_of(phys))
    A, b, c = ark.ars343()
    Us, ysall = [torch.as_tensor(U0)], []
    for _ in range(nsteps):
        Un, ys, _ = ark.erk_step(op.residual, Us[-1], dt, A, b, return_stages=True)
        Us.append(Un)
        ysall.append(ys)
    lam = torch.as_tensor(lamN)
    for n in reversed(range(nsteps)):
        lam = ark.erk_adjoint_step(lambda y, mu: vjp(op, y, mu), ysall[n], lam, dt, A, b)
    err = rel_err(lam0.cpu().numpy() - lamN, lam.numpy() - lamN)
    record("multistep-adjoint-fp64", rel=err)
    assert err < TOL["fp64"], err


def test_ark_adjoint_step_euler_periodic_fp32():
    """FP32 adjoint step (FP64 lambda accumulation) on a fully periodic Euler mesh."""
    from paper_2607_16044_b300.dgx import Solver
    from paper_2607_16044_b300.tableaux import ars343_explicit
    mesh = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 5), I.uniform_edges(0, 1, 4)], [True, True])
    phys = _euler()
    U0 = I.random_state(mesh, 21)
    lam0 = I.gaussian_cotangent(U0.shape, 22)
    dt = 1e-3
    s = Solver(mesh, phys, "fp32")
    s.set_tableau(*ars343_explicit())
    U = torch.as_tensor(U0).cuda()
    stages = s.stage_buffer()
    s.ark_step_stages(U, dt, stages)
    lam = torch.as_tensor(lam0).cuda()
    s.ark_adjoint_step(stages, lam, dt)
    s.check()
    op = DGOperator(mesh, gas_of(phys))
    A, b, c = ark.ars343()
    ys = [torch.as_tensor(s.stage_state(stages, i).double().cpu().numpy()) for i in range(4)]  # FP32 stage states
    ref = ark.erk_adjoint_step(lambda y, mu: vjp(op, y, mu), ys, torch.as_tensor(lam0), dt, A, b).numpy()
    err = rel_err(lam.cpu().numpy() - lam0, ref - lam0)
    record("ark-adjoint-fp32", rel=err)
    assert err < 1e-5, err


@pytest.mark.parametrize("case", ["2d-p2-euler", "2d-p3-ns", "2d-p4-ns-walls", "2d-p4-ns-curv", "3d-p1-ns", "3d-p2-ns"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_warp_variant_bit_identical(case, prec):
    """Every tile kernel run one warp per element (variant 3) equals the
    CTA-tile variant bit for bit: residual, VJP, ARK step and its adjoint."""
    from paper_2607_16044_b300.dgx import KERNELS, Solver
    from paper_2607_16044_b300.tableaux import ars343_explicit
    if case == "2d-p2-euler":
        mesh, phys = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 9)] * 2, [True, True]), _euler()
    elif case == "2d-p3-ns":
        mesh, phys = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 7), I.uniform_edges(0, 1, 5)], [True, True]), _ns()
    elif case == "2d-p4-ns-walls":
        mesh = I.structured_box_mesh(4, [I.uniform_edges(0, 1, 11), I.wall_stretched_edges(3, 1.3)], [True, False])
        phys = _ns()
    elif case == "2d-p4-ns-curv":
        mesh, phys = I.rotate_elements(I.warped_mesh(4, [5, 4], [1.0, 1.0], 0.04, periodic=[True, False]), 8), _ns()
    elif case == "3d-p1-ns":
        mesh = I.structured_box_mesh(1, [I.uniform_edges(0, 1, 5)] * 2 + [I.wall_stretched_edges(2, 1.2)],
                                     [True, True, False])
        phys = _ns()
    else:
        mesh = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 3)] * 2 + [I.wall_stretched_edges(1, 1.0)],
                                     [True, True, False])
        phys = _ns()
    U0 = I.random_state(mesh, 88)
    lam0 = I.gaussian_cotangent(U0.shape, 89)
    dt = torch.float64 if prec == "fp64" else torch.float32
    outs = []
    for var in (None, 3):                   # the handle's default CTA variants, then warp per element
        s = Solver(mesh, phys, prec)
        s.set_tableau(*ars343_explicit())
        if var is not None:
            tile_kinds = [k for k in KERNELS if k not in ("face", "vjp_face")]
            s.set_variants({k: var for k in tile_kinds})
        Ud = torch.as_tensor(U0).to("cuda", dt).contiguous()
        f = s.rhs(Ud)
        g = s.rhs_vjp(Ud, torch.as_tensor(lam0).to("cuda", dt).contiguous())
        U = torch.as_tensor(U0).cuda()
        stages = s.stage_buffer()
        s.ark_step_stages(U, 1e-4, stages)
        lam = torch.as_tensor(lam0).cuda()
        s.ark_adjoint_step(stages, lam, 1e-4)
        s.check()
        outs.append((f, g, U, lam))
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a, b)


def test_channel3d_config_full_size_sampled_fp32():
    """48^3 p = 5 wall-stretched 3D channel (24M nodes), FP32: sampled residual
    rows and VJP rows against the oracle evaluated on the rings around them."""
    from oracle.residual import DGOperator, submesh_around, term_scale
    from oracle.vjp import vjp_rows
    from paper_2607_16044_b300.dgx import Solver
    from tests.parity_util import noise_floor, scaled_err
    mesh, phys, U0 = I.channel3d_workload()
    lam0 = I.gaussian_cotangent(U0.shape, 105)
    s = Solver(mesh, phys, "fp32")
    U32 = torch.as_tensor(U0).cuda().float()
    f = s.rhs(U32).double().cpu().numpy()
    g = s.rhs_vjp(U32, torch.as_tensor(lam0).cuda().float()).double().cpu().numpy()
    s.check()
    rng = np.random.default_rng(7)
    rows = np.unique(np.concatenate([rng.choice(mesh.n_elem, 6, replace=False), [0, mesh.n_elem - 1]]))
    Uq, lq = quantize32(U0), quantize32(lam0)
    gas = gas_of(phys)
    # forward rows: residuals need the 2-ring (BR1)
    sub, keep, loc = submesh_around(mesh, rows, 3)
    op = DGOperator(sub, gas)
    Ut = torch.as_tensor(Uq[keep])
    ref = op.residual(Ut, loc).numpy()
    T = term_scale(op, Ut, loc).numpy()
    ferr = scaled_err(f[rows], ref, T)
    # VJP rows: g_e collects the residuals of the 2-ring of e, each depending on its own 2-ring
    sub4, keep4, loc4 = submesh_around(mesh, rows, 5)
    op4 = DGOperator(sub4, gas)
    gref = vjp_rows(op4, torch.as_tensor(Uq[keep4]), torch.as_tensor(lq[keep4]), loc4).numpy()
    gerr = rel_err(g[rows], gref)
    record("channel3d-fp32", scaled=ferr, vjp_rel=gerr, sampled=len(rows))
    assert ferr < 1e-5, ferr
    assert gerr < TOL["fp32"], gerr


def _ark_adjoint_vs_oracle(mesh, phys, prec, dt, seed, ys_from_gpu=False, ys_rounded=False):
    """One ARS(3,4,3) step with stage checkpoints, then its adjoint, against the
    oracle's reverse recurrence, linearised at the oracle's own stage states
    (``ys_rounded``: each rounded to FP32, the precision the FP32 kernels
    evaluate in) or at the GPU's stage states (``ys_from_gpu``)."""
    from paper_2607_16044_b300.dgx import Solver
    from paper_2607_16044_b300.tableaux import ars343_explicit
    U0 = I.random_state(mesh, seed)
    lam0 = I.gaussian_cotangent(U0.shape, seed + 1)
    s = Solver(mesh, phys, prec)
    s.set_tableau(*ars343_explicit())
    U = torch.as_tensor(U0).cuda()
    stages = s.stage_buffer()
    s.ark_step_stages(U, dt, stages)
    lam = torch.as_tensor(lam0).cuda()
    s.ark_adjoint_step(stages, lam, dt)
    s.check()
    op = DGOperator(mesh, gas_of(phys))
    A, b, c = ark.ars343()
    if ys_from_gpu:
        ys = [torch.as_tensor(s.stage_state(stages, i).double().cpu().numpy()) for i in range(4)]
    else:
        _, ys, _ = ark.erk_step(op.residual, torch.as_tensor(U0), dt, A, b, return_stages=True)
        if ys_rounded:
            ys = [torch.as_tensor(quantize32(y.numpy())) for y in ys]
    ref = ark.erk_adjoint_step(lambda y, mu: vjp(op, y, mu), ys, torch.as_tensor(lam0), dt, A, b).numpy()
    return rel_err(lam.cpu().numpy() - lam0, ref - lam0)


def test_ark_adjoint_3d_curvilinear_rotated_ns_fp64():
    """Reverse stages with the fused gather on a rotated curved 3D mesh (every
    face-orientation code, scattered jump cotangents, metric terms)."""
    mesh = I.rotate_elements(I.warped_mesh(2, [2, 3, 2], [1.0, 1.0, 1.0], 0.03, periodic=[True, True, False]), 73)
    err = _ark_adjoint_vs_oracle(mesh, _ns(), "fp64", 1e-4, 31)
    record("ark-adjoint-3d-curv-fp64", rel=err)
    assert err < TOL["fp64"], err


def test_ark_adjoint_ns_walls_fp32():
    """FP32 viscous adjoint step on a wall-bounded box mesh (box line-assembly of
    P_b, FP32 stage coefficients, FP64 lambda update)."""
    mesh = I.structured_box_mesh(4, [I.uniform_edges(0, 1, 7), I.wall_stretched_edges(3, 1.3)], [True, False])
    err = _ark_adjoint_vs_oracle(mesh, _ns(), "fp32", 2e-5, 41, ys_from_gpu=True)
    record("ark-adjoint-ns-walls-fp32", rel=err)
    assert err < 1e-5, err


def test_ark_adjoint_self_periodic_ns_fp64():
    """One element across a periodic direction: the element is its own neighbour
    there, so jump cotangents are scattered into its own opposite face."""
    mesh = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 1), I.wall_stretched_edges(2, 1.2)], [True, False])
    err = _ark_adjoint_vs_oracle(mesh, _ns(), "fp64", 1e-4, 51)
    record("ark-adjoint-self-periodic-fp64", rel=err)
    assert err < TOL["fp64"], err


def test_ark_adjoint_ns_walls_fp32_at_oracle_stages():
    """The same FP32 adjoint step, the oracle now linearised at its own FP64
    stage states rounded to FP32 (not at the GPU's): checks the forward FP32
    stage states and the adjoint together."""
    mesh = I.structured_box_mesh(4, [I.uniform_edges(0, 1, 7), I.wall_stretched_edges(3, 1.3)], [True, False])
    err = _ark_adjoint_vs_oracle(mesh, _ns(), "fp32", 2e-5, 41, ys_rounded=True)
    record("ark-adjoint-ns-walls-fp32-oracle-stages", rel=err)
    assert err < TOL["fp32"], err


def test_vjp_channel2d_full_size_perturbed_fp32():
    """256 x 128 wall-stretched channel, p = 4, FP32, on a well-conditioned
    state (the Poiseuille profile with 10 % seeded perturbations): sampled VJP
    rows, including both walls, at the plain FP32 target."""
    mesh, phys, _ = I.channel2d_workload()
    U = I.channel_state(mesh, phys, 2, amp=0.1)
    lam = I.gaussian_cotangent(U.shape, 102)
    got = _gpu_vjp(mesh, phys, U, lam, "fp32")
    rng = np.random.default_rng(3)
    rows = np.unique(np.concatenate([rng.choice(mesh.n_elem, 24, replace=False), [0, mesh.n_elem - 1]]))
    ref = _oracle_vjp(mesh, phys, quantize32(U), quantize32(lam), rows)
    err = rel_err(got[rows], ref)
    record("vjp-channel2d-perturbed-fp32", rel=err, sampled=len(rows))
    assert err < TOL["fp32"], err
