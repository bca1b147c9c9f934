"""GPU parity of the paper's DG-IP operator (Vijayasundaram flux + symmetric
interior penalty; farfield and adiabatic-wall forms; geometry-split interface;
manufactured-solution source; ARK step) against the FP64 oracle (oracle.sipg)."""
import numpy as np
import pytest
import torch

from oracle import ark
from oracle.residual import submesh_around
from oracle.sipg import SIPGOperator
from paper_2607_16044_b300 import inputs as I
from tests import mms_sympy
from tests.parity_util import TOL, gas_of, quantize32, record, rel_err

pytestmark = pytest.mark.gpu

UINF2 = np.array([1.1, 0.4, -0.3, 2.0 / 0.4 + 0.5 * (0.4 ** 2 + 0.3 ** 2) / 1.1])


def _solver(mesh, phys, prec, **kw):
    from paper_2607_16044_b300.dgx import Solver
    return Solver(mesh, phys, prec, scheme="dgip", **kw)


def _euler():
    return I.Physics(gamma=1.4, viscous=False)


def _ns(Re=200.0):
    return I.Physics(gamma=1.4, Re=Re, Pr=0.72, Ma=0.3, viscous=True)


def _dt(prec):
    return torch.float64 if prec == "fp64" else torch.float32


def _oracle(mesh, phys, U, U_inf=None, explicit=None, U_im=None):
    op = SIPGOperator(mesh, gas_of(phys), U_inf=U_inf, explicit=explicit)
    return op.residual(torch.as_tensor(U), None if U_im is None else torch.as_tensor(U_im)).numpy()


def _check(mesh, phys, U, prec, name, U_inf=None):
    s = _solver(mesh, phys, prec, U_inf=U_inf)
    f = s.rhs(torch.as_tensor(U).to("cuda", _dt(prec)).contiguous())
    s.check()
    Uref = U if prec == "fp64" else quantize32(U)
    ref = _oracle(mesh, phys, Uref, U_inf)
    err = rel_err(f.double().cpu().numpy(), ref)
    record(name, rel=err, E=mesh.n_elem)
    assert err < TOL[prec], err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_dgip_2d_euler_periodic(p, prec):
    mesh = I.structured_box_mesh(p, [I.uniform_edges(-1, 1, 7), I.uniform_edges(0, 1.3, 5)], [True, True])
    _check(mesh, _euler(), I.random_state(mesh, 600 + p), prec, f"dgip-2d-euler-p{p}-{prec}")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_dgip_2d_ns_walls_stretched(p, prec):
    mesh = I.structured_box_mesh(p, [I.uniform_edges(0, 1, 7), I.wall_stretched_edges(3, 1.5)], [True, False])
    _check(mesh, _ns(), I.random_state(mesh, 610 + p), prec, f"dgip-2d-ns-walls-p{p}-{prec}")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("viscous", [False, True])
def test_dgip_3d_boxes_walls(p, viscous, prec):
    cells = {1: 3, 2: 3, 3: 2, 4: 2, 5: 2}[p]
    mesh = I.structured_box_mesh(p, [I.uniform_edges(0, 1, cells), I.uniform_edges(0, 1.2, cells + 1),
                                     I.wall_stretched_edges(1, 1.0)], [True, True, False])
    _check(mesh, _ns() if viscous else _euler(), I.random_state(mesh, 620 + p), prec,
           f"dgip-3d-{'ns' if viscous else 'euler'}-p{p}-{prec}")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("viscous", [False, True])
def test_dgip_farfield(viscous, prec):
    """Farfield boundaries (tag 1, App. B.1.1) on both ends of y."""
    mesh = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 6), I.uniform_edges(0, 1, 4)], [True, False], wall_tag=1)
    _check(mesh, _ns() if viscous else _euler(), I.random_state(mesh, 630), prec,
           f"dgip-farfield-{'ns' if viscous else 'euler'}-{prec}", U_inf=UINF2)


def test_dgip_single_element_self_periodic():
    mesh = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 1), I.uniform_edges(0, 2, 1)], [True, True])
    _check(mesh, _ns(), I.random_state(mesh, 7), "fp64", "dgip-self-periodic")


def _vjp_check(mesh, phys, prec, name, U_inf=None, seed=640):
    from oracle.vjp import vjp
    U = I.random_state(mesh, seed)
    lam = I.gaussian_cotangent(U.shape, seed + 1)
    s = _solver(mesh, phys, prec, U_inf=U_inf)
    g = s.rhs_vjp(torch.as_tensor(U).to("cuda", _dt(prec)).contiguous(),
                  torch.as_tensor(lam).to("cuda", _dt(prec)).contiguous())
    s.check()
    if prec == "fp32":
        U, lam = quantize32(U), quantize32(lam)
    op = SIPGOperator(mesh, gas_of(phys), U_inf=U_inf)
    ref = vjp(op, torch.as_tensor(U), torch.as_tensor(lam)).numpy()
    err = rel_err(g.double().cpu().numpy(), ref)
    record(name, rel=err, E=mesh.n_elem)
    assert err < TOL[prec], err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("viscous", [False, True])
def test_dgip_vjp_2d_walls(p, viscous, prec):
    mesh = I.structured_box_mesh(p, [I.uniform_edges(0, 1, 5), I.wall_stretched_edges(2, 1.4)], [True, False])
    _vjp_check(mesh, _ns() if viscous else _euler(), prec, f"dgip-vjp-2d-{viscous}-p{p}-{prec}")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_dgip_vjp_3d_walls(p, prec):
    mesh = I.structured_box_mesh(p, [I.uniform_edges(0, 1, 2), I.uniform_edges(0, 1.2, 3),
                                     I.wall_stretched_edges(1, 1.0)], [True, True, False])
    _vjp_check(mesh, _ns(), prec, f"dgip-vjp-3d-p{p}-{prec}")


@pytest.mark.parametrize("viscous", [False, True])
def test_dgip_vjp_farfield(viscous):
    mesh = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 4), I.uniform_edges(0, 1, 3)], [True, False], wall_tag=1)
    _vjp_check(mesh, _ns() if viscous else _euler(), "fp64", f"dgip-vjp-farfield-{viscous}", U_inf=UINF2)


def test_dgip_vjp_adjoint_identity_central_differences():
    """<lambda, J v> by central differences of the GPU residual (step 1e-6 of
    the state scale) against <J^T lambda, v> from the GPU adjoint."""
    mesh = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 4), I.wall_stretched_edges(2, 1.3)], [True, False])
    U = I.random_state(mesh, 650)
    lam = I.gaussian_cotangent(U.shape, 651)
    v = I.gaussian_cotangent(U.shape, 652) * np.abs(U)
    s = _solver(mesh, _ns(), "fp64")
    Ud = torch.as_tensor(U).cuda()
    g = s.rhs_vjp(Ud, torch.as_tensor(lam).cuda()).cpu().numpy()
    eps = 1e-6
    fp = s.rhs(torch.as_tensor(U + eps * v).cuda()).cpu().numpy()
    fm = s.rhs(torch.as_tensor(U - eps * v).cuda()).cpu().numpy()
    s.check()
    jv = (fp - fm) / (2 * eps)
    lhs, rhs = float((lam * jv).sum()), float((g * v).sum())
    record("dgip-adjoint-fd", rel=abs(lhs - rhs) / abs(rhs))
    assert abs(lhs - rhs) < 1e-6 * abs(rhs), (lhs, rhs)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dim", [2, 3])
def test_dgip_geometry_split_interface(dim, prec):
    """R^DG(U^ex, U^im) with an implicit strip (Sec. 4.1): explicit elements
    read U_ex, implicit ones U_im; interface faces against the implicit side."""
    if dim == 2:
        mesh = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 6), I.wall_stretched_edges(2, 1.3)], [True, False])
        col = np.arange(mesh.n_elem) % 6
        explicit = (col != 2) & (col != 3)
    else:
        mesh = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 4), I.uniform_edges(0, 1, 2),
                                         I.wall_stretched_edges(1, 1.0)], [True, True, False])
        col = np.arange(mesh.n_elem) % 4
        explicit = col != 1
    phys = _ns()
    Uex = I.random_state(mesh, 660)
    Uim = I.random_state(mesh, 661)
    s = _solver(mesh, phys, prec)
    s.set_explicit_mask(explicit)
    f = s.rhs_split(torch.as_tensor(Uex).to("cuda", _dt(prec)).contiguous(),
                    torch.as_tensor(Uim).to("cuda", _dt(prec)).contiguous())
    s.check()
    if prec == "fp32":
        Uex, Uim = quantize32(Uex), quantize32(Uim)
    ref = _oracle(mesh, phys, Uex, explicit=explicit, U_im=Uim)
    got = f.double().cpu().numpy()
    assert np.all(got[~explicit] == 0)
    err = rel_err(got[explicit], ref[explicit])
    record(f"dgip-split-{dim}d-{prec}", rel=err)
    assert err < TOL[prec], err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("viscous", [False, True])
def test_mms_source_matches_symbolic(viscous, prec):
    """The device source of Sec. 5.1.1 against dU_e/dt + div(F^c - F^nu)(U_e)
    differentiated symbolically (sympy) from the fluxes of Sec. 2."""
    mu = 0.01
    phys = I.Physics(gamma=1.4, Re=1 / mu, Pr=0.72, Ma=0.3, viscous=viscous)
    mesh = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 8)] * 2, [True, True])
    fns = mms_sympy.build(2, 1.4, mu if viscous else 0.0, 0.72)
    t = 0.0037
    want = mms_sympy.evaluate(fns["Ut"], mesh.xyz, t) + mms_sympy.evaluate(fns["divFc"], mesh.xyz, t) \
        - mms_sympy.evaluate(fns["divFv"], mesh.xyz, t)
    for scheme in ("dgip", "llf-br1"):
        from paper_2607_16044_b300.dgx import Solver
        s = Solver(mesh, phys, prec, scheme=scheme)
        out = torch.zeros(s.shape, dtype=_dt(prec), device="cuda")
        s.mms_source(t, out)
        s.check()
        err = rel_err(out.double().cpu().numpy(), want)
        assert err < (1e-13 if prec == "fp64" else 1e-6), (scheme, err)


def test_dgip_ark_step_matches_oracle():
    """One ARS(3,4,3) step of the DG-IP operator (fused stage updates, FP64
    accumulation) against the oracle's ERK step."""
    from paper_2607_16044_b300.tableaux import ars343_explicit
    mesh = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 5), I.wall_stretched_edges(2, 1.3)], [True, False])
    phys = _ns()
    U0 = I.random_state(mesh, 670)
    dt = 2e-5
    for prec in ("fp64", "fp32"):
        s = _solver(mesh, phys, prec)
        s.set_tableau(*ars343_explicit())
        U = torch.as_tensor(U0).cuda()
        s.ark_step(U, dt)
        s.check()
        op = SIPGOperator(mesh, gas_of(phys))
        A, b, c = ark.ars343()
        Uref = ark.erk_step(op.residual, torch.as_tensor(U0), dt, A, b).numpy()
        err = rel_err(U.cpu().numpy() - U0, Uref - U0)
        record(f"dgip-ark-{prec}", rel=err)
        assert err < TOL[prec], (prec, err)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_dgip_channel2d_full_size_sampled(prec):
    """256 x 128 wall-stretched channel, p = 4 (the 2D NS configuration), DG-IP:
    sampled elements incl. both walls against the oracle on their 2-ring
    sub-mesh; FP32 on the 10 %-perturbed state (well conditioned)."""
    mesh, phys, _ = I.channel2d_workload()
    U = I.channel_state(mesh, phys, 2, amp=0.1 if prec == "fp32" else 1e-3)
    s = _solver(mesh, phys, prec)
    f = s.rhs(torch.as_tensor(U).to("cuda", _dt(prec)).contiguous()).double().cpu().numpy()
    s.check()
    rng = np.random.default_rng(9)
    rows = np.unique(np.concatenate([rng.choice(mesh.n_elem, 24, replace=False), [0, mesh.n_elem - 1]]))
    Uref = U if prec == "fp64" else quantize32(U)
    sub, keep, loc = submesh_around(mesh, rows, 2)
    ref = SIPGOperator(sub, gas_of(phys)).residual(torch.as_tensor(Uref[keep])).numpy()[loc]
    err = rel_err(f[rows], ref)
    record(f"dgip-channel2d-{prec}", rel=err, sampled=len(rows))
    assert err < TOL[prec], err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_dgip_ark_adjoint_matches_oracle(prec):
    """Discrete adjoint of one DG-IP ARS(3,4,3) step (reverse stage recurrence
    composed from single VJPs) against the oracle's recurrence, linearised at
    the oracle's stage states (FP32: rounded to FP32); the one-call step +
    adjoint equals the separate calls bit for bit."""
    from oracle.vjp import vjp
    from paper_2607_16044_b300.tableaux import ars343_explicit
    mesh = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 5), I.wall_stretched_edges(2, 1.3)], [True, False])
    phys = _ns()
    U0 = I.random_state(mesh, 680)
    lam0 = I.gaussian_cotangent(U0.shape, 681)
    dt = 2e-5
    s = _solver(mesh, phys, prec)
    s.set_tableau(*ars343_explicit())
    U = torch.as_tensor(U0).cuda()
    stages = s.stage_buffer()
    s.ark_step_stages(U, dt, stages)
    lam = torch.as_tensor(lam0).cuda()
    s.ark_adjoint_step(stages, lam, dt)
    U2 = torch.as_tensor(U0).cuda()
    lam2 = torch.as_tensor(lam0).cuda()
    s.ark_step_adjoint(U2, lam2, dt, s.stage_buffer())
    s.check()
    assert torch.equal(U, U2) and torch.equal(lam, lam2)
    op = SIPGOperator(mesh, gas_of(phys))
    A, b, c = ark.ars343()
    _, ys, _ = ark.erk_step(op.residual, torch.as_tensor(U0), dt, A, b, return_stages=True)
    if prec == "fp32":
        ys = [torch.as_tensor(quantize32(y.numpy())) for y in ys]
    ref = ark.erk_adjoint_step(lambda y, mu: vjp(op, y, mu), ys, torch.as_tensor(lam0), dt, A, b).numpy()
    err = rel_err(lam.cpu().numpy() - lam0, ref - lam0)
    record(f"dgip-ark-adjoint-{prec}", rel=err)
    assert err < TOL[prec], err


def _sampled_rows_and_vjp(op_factory, mesh, U, lam, rows):
    """Oracle residual rows and VJP rows of the DG-IP operator for a few
    elements of a large mesh: the residual of an element reads its face
    neighbours (their traces and own gradients), so rows + 2 rings of
    elements hold every residual that the rows' residuals and VJP rows need;
    the VJP rows come from autograd of the sub-mesh residual with the
    cotangent kept on the rows' 1-ring."""
    sub, keep, loc = submesh_around(mesh, rows, 2)
    op = op_factory(sub)
    Ut = torch.as_tensor(U[keep]).clone().requires_grad_(True)
    f = op.residual(Ut)
    ring = set(int(x) for x in loc)
    for r in loc:
        ring.update(int(x) for x in sub.neighbor[r] if x >= 0)
    lt = torch.zeros_like(Ut)
    idx = torch.as_tensor(sorted(ring))
    lt[idx] = torch.as_tensor(lam[keep])[idx]
    (g,) = torch.autograd.grad(f, Ut, grad_outputs=lt)
    return f.detach().numpy()[loc], g.numpy()[loc]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_dgip_channel3d_full_size_sampled(prec):
    """The 48^3 p = 5 wall-stretched 3D channel (the bench's DG-IP leg):
    residual and VJP rows of sampled elements, both walls included, against
    the oracle on the rings around them; FP32 on the 10 %-perturbed state."""
    mesh, phys, _ = I.channel3d_workload()
    U = I.channel_state(mesh, phys, 5, amp=0.1 if prec == "fp32" else 1e-3)
    lam = I.gaussian_cotangent(U.shape, 105)
    s = _solver(mesh, phys, prec)
    Ud = torch.as_tensor(U).to("cuda", _dt(prec)).contiguous()
    f = s.rhs(Ud).double().cpu().numpy()
    g = s.rhs_vjp(Ud, torch.as_tensor(lam).to("cuda", _dt(prec)).contiguous()).double().cpu().numpy()
    s.check()
    del s, Ud
    torch.cuda.empty_cache()
    rng = np.random.default_rng(11)
    rows = np.unique(np.concatenate([rng.choice(mesh.n_elem, 6, replace=False), [0, mesh.n_elem - 1]]))
    Uref, lref = (U, lam) if prec == "fp64" else (quantize32(U), quantize32(lam))
    fref, gref = _sampled_rows_and_vjp(lambda m: SIPGOperator(m, gas_of(phys)), mesh, Uref, lref, rows)
    ferr, gerr = rel_err(f[rows], fref), rel_err(g[rows], gref)
    record(f"dgip-channel3d-{prec}", rel=ferr, vjp_rel=gerr, sampled=len(rows))
    assert ferr < TOL[prec], ferr
    assert gerr < TOL[prec], gerr


# ---------------------------------------------------------------- curvilinear
def _curved(case):
    if case == "warped2d-walls":
        return I.warped_mesh(3, [5, 4], [1.0, 1.2], 0.04, periodic=[True, False])
    if case == "rotated2d":
        return I.rotate_elements(I.warped_mesh(3, [4, 4], [1.0, 1.3], 0.05), 3)
    if case == "rotated2d-walls-p5":
        return I.rotate_elements(I.warped_mesh(5, [3, 3], [1.0, 1.0], 0.04, periodic=[True, False]), 4)
    return I.warped_mesh(2, [2, 3, 2], [1.0, 1.0, 1.0], 0.03, periodic=[True, True, False])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("case", ["warped2d-walls", "rotated2d", "rotated2d-walls-p5", "warped3d-walls"])
def test_dgip_curvilinear(case, viscous, prec):
    """The paper's operator on curved elements (metric terms traced to the
    faces, area normals, contravariant adjoint-consistency vectors, 1/l from
    the geometry): parity with the oracle on warped and rotated meshes."""
    mesh = _curved(case)
    _check(mesh, _ns() if viscous else _euler(), I.random_state(mesh, 690), prec,
           f"dgip-curv-{case}-{viscous}-{prec}")


def test_dgip_curvilinear_split_and_ark():
    """Curved elements: the geometry-split residual and one ARS(3,4,3) step
    against the oracle."""
    from paper_2607_16044_b300.tableaux import ars343_explicit
    mesh = _curved("warped2d-walls")
    phys = _ns()
    col = np.arange(mesh.n_elem) % 5
    explicit = col != 2
    Uex, Uim = I.random_state(mesh, 691), I.random_state(mesh, 692)
    s = _solver(mesh, phys, "fp64")
    s.set_explicit_mask(explicit)
    f = s.rhs_split(torch.as_tensor(Uex).cuda(), torch.as_tensor(Uim).cuda()).cpu().numpy()
    ref = _oracle(mesh, phys, Uex, explicit=explicit, U_im=Uim)
    assert np.all(f[~explicit] == 0)
    err = rel_err(f[explicit], ref[explicit])
    record("dgip-curv-split", rel=err)
    assert err < TOL["fp64"], err
    s.set_explicit_mask(None)
    s.set_tableau(*ars343_explicit())
    U0 = I.random_state(mesh, 693)
    U = torch.as_tensor(U0).cuda()
    dt = 2e-5
    s.ark_step(U, dt)
    s.check()
    op = SIPGOperator(mesh, gas_of(phys))
    A, b, c = ark.ars343()
    Uref = ark.erk_step(op.residual, torch.as_tensor(U0), dt, A, b).numpy()
    err = rel_err(U.cpu().numpy() - U0, Uref - U0)
    record("dgip-curv-ark", rel=err)
    assert err < TOL["fp64"], err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("case", ["warped2d-walls", "rotated2d", "rotated2d-walls-p5", "warped3d-walls"])
def test_dgip_vjp_curvilinear(case, viscous, prec):
    """The DG-IP adjoint on curved elements against the oracle's autograd."""
    _vjp_check(_curved(case), _ns() if viscous else _euler(), prec, f"dgip-vjp-curv-{case}-{viscous}-{prec}",
               seed=695)


def test_dgip_ark_adjoint_curvilinear():
    """One DG-IP ARS(3,4,3) step and its discrete adjoint on a warped mesh
    against the oracle's recurrences."""
    from oracle.vjp import vjp
    from paper_2607_16044_b300.tableaux import ars343_explicit
    mesh = _curved("warped2d-walls")
    phys = _ns()
    U0 = I.random_state(mesh, 696)
    lam0 = I.gaussian_cotangent(U0.shape, 697)
    dt = 2e-5
    s = _solver(mesh, phys, "fp64")
    s.set_tableau(*ars343_explicit())
    U, lam = torch.as_tensor(U0).cuda(), torch.as_tensor(lam0).cuda()
    s.ark_step_adjoint(U, lam, dt, s.stage_buffer())
    s.check()
    op = SIPGOperator(mesh, gas_of(phys))
    A, b, c = ark.ars343()
    _, ys, _ = ark.erk_step(op.residual, torch.as_tensor(U0), dt, A, b, return_stages=True)
    ref = ark.erk_adjoint_step(lambda y, mu: vjp(op, y, mu), ys, torch.as_tensor(lam0), dt, A, b).numpy()
    err = rel_err(lam.cpu().numpy() - lam0, ref - lam0)
    record("dgip-ark-adjoint-curv", rel=err)
    assert err < TOL["fp64"], err


def test_dgip_geometry_override_on_boxes():
    """A DG-IP box handle given the boxes' exact metrics runs the curvilinear
    kernels and still equals the oracle (and the box kernels)."""
    mesh = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 5), I.wall_stretched_edges(2, 1.3)], [True, False])
    U = torch.as_tensor(I.random_state(mesh, 694)).cuda()
    s0, s1 = _solver(mesh, _ns(), "fp64"), _solver(mesh, _ns(), "fp64")
    E, N = mesh.n_elem, mesh.N
    half = 0.5 * mesh.size
    J = np.repeat(np.prod(half, 1)[:, None], N, 1)
    M = np.zeros((E, N, 2, 2))
    M[:, :, 0, 0] = half[:, 1:2]
    M[:, :, 1, 1] = half[:, 0:1]
    s1.set_geometry(J, M)
    f0, f1 = s0.rhs(U).cpu().numpy(), s1.rhs(U).cpu().numpy()
    s0.check()
    s1.check()
    ref = _oracle(mesh, _ns(), U.cpu().numpy())
    assert rel_err(f1, ref) < TOL["fp64"]
    assert rel_err(f1, f0) < 1e-13
