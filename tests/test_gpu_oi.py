"""GPU parity of the over-integrated DG-IP operator (the nonlinear terms by the
M-point Gauss rule of order 3k, Sec. 5) against the FP64 oracle
(oracle.sipg.OverIntegratedSIPG): residual, VJP, geometry-split form, ARK step
and its adjoint, and the M = p+1 case, which is the collocated operator bit
for bit."""
import numpy as np
import pytest
import torch

from oracle import ark
from oracle.residual import submesh_around
from oracle.sipg import OverIntegratedSIPG, SIPGOperator
from oracle.vjp import vjp
from paper_2607_16044_b300 import inputs as I
from tests.parity_util import TOL, gas_of, quantize32, record, rel_err

pytestmark = pytest.mark.gpu

UINF2 = np.array([1.1, 0.4, -0.3, 2.0 / 0.4 + 0.5 * (0.4 ** 2 + 0.3 ** 2) / 1.1])


def _solver(mesh, phys, prec, M="3k", **kw):
    from paper_2607_16044_b300.dgx import Solver
    return Solver(mesh, phys, prec, scheme="dgip", quad_points=M, **kw)


def _euler():
    return I.Physics(gamma=1.4, viscous=False)


def _ns(Re=200.0):
    return I.Physics(gamma=1.4, Re=Re, Pr=0.72, Ma=0.3, viscous=True)


def _dt(prec):
    return torch.float64 if prec == "fp64" else torch.float32


def _oracle(mesh, phys, M=None, **kw):
    return OverIntegratedSIPG(mesh, gas_of(phys), M=M, **kw)


def _rhs_check(mesh, phys, prec, name, M="3k", seed=700, U_inf=None):
    U = I.random_state(mesh, seed)
    s = _solver(mesh, phys, prec, M, U_inf=U_inf)
    f = s.rhs(torch.as_tensor(U).to("cuda", _dt(prec)).contiguous())
    s.check()
    Uref = U if prec == "fp64" else quantize32(U)
    ref = _oracle(mesh, phys, None if M == "3k" else M, U_inf=U_inf).residual(torch.as_tensor(Uref)).numpy()
    err = rel_err(f.double().cpu().numpy(), ref)
    record(name, rel=err, E=mesh.n_elem, M=s.quad_points)
    assert err < TOL[prec], err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("viscous", [False, True])
def test_oi_2d_walls_stretched(p, viscous, prec):
    mesh = I.structured_box_mesh(p, [I.uniform_edges(0, 1, 7), I.wall_stretched_edges(3, 1.5)], [True, False])
    _rhs_check(mesh, _ns() if viscous else _euler(), prec, f"oi-2d-{viscous}-p{p}-{prec}", seed=700 + p)


@pytest.mark.parametrize("p,M", [(1, 3), (1, 6), (2, 3), (2, 5), (2, 6), (4, 6), (3, 8), (5, 7)])
def test_oi_2d_other_rules(p, M):
    mesh = I.structured_box_mesh(p, [I.uniform_edges(0, 1, 5), I.wall_stretched_edges(2, 1.4)], [True, False])
    _rhs_check(mesh, _ns(), "fp64", f"oi-2d-p{p}-M{M}", M=M, seed=710 + M)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_oi_3d_walls(p, prec):
    cells = {1: 3, 2: 2, 3: 2, 4: 1, 5: 1}[p]
    mesh = I.structured_box_mesh(p, [I.uniform_edges(0, 1, cells), I.uniform_edges(0, 1.2, cells + 1),
                                     I.wall_stretched_edges(1, 1.0)], [True, True, False])
    _rhs_check(mesh, _ns(), prec, f"oi-3d-p{p}-{prec}", seed=720 + p)


@pytest.mark.parametrize("viscous", [False, True])
def test_oi_farfield(viscous):
    mesh = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 5), I.uniform_edges(0, 1, 4)], [True, False], wall_tag=1)
    _rhs_check(mesh, _ns() if viscous else _euler(), "fp64", f"oi-farfield-{viscous}", seed=730, U_inf=UINF2)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dim", [2, 3])
def test_oi_with_p_plus_1_points_is_the_collocated_operator(dim, prec):
    """M = p+1: the transfers are identities (exactly: l_j at the nodes is 0 or
    1, omega_m / w_q = 1), so residual and VJP equal the collocated handle's
    bit for bit."""
    if dim == 2:
        mesh = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 5), I.wall_stretched_edges(2, 1.4)], [True, False])
    else:
        mesh = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 2), I.uniform_edges(0, 1, 3),
                                         I.wall_stretched_edges(1, 1.0)], [True, True, False])
    U = torch.as_tensor(I.random_state(mesh, 740)).to("cuda", _dt(prec)).contiguous()
    lam = torch.as_tensor(I.gaussian_cotangent(U.shape, 741)).to("cuda", _dt(prec)).contiguous()
    s0 = _solver(mesh, _ns(), prec, None)
    s1 = _solver(mesh, _ns(), prec, mesh.p + 1)
    assert torch.equal(s0.rhs(U), s1.rhs(U))
    assert torch.equal(s0.rhs_vjp(U, lam), s1.rhs_vjp(U, lam))
    s0.check()
    s1.check()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,p", [(2, 2), (2, 3), (2, 5), (3, 2), (3, 4)])
def test_oi_vjp(dim, p, prec):
    if dim == 2:
        mesh = I.structured_box_mesh(p, [I.uniform_edges(0, 1, 5), I.wall_stretched_edges(2, 1.4)], [True, False])
    else:
        mesh = I.structured_box_mesh(p, [I.uniform_edges(0, 1, 2), I.uniform_edges(0, 1.2, 3),
                                         I.wall_stretched_edges(1, 1.0)], [True, True, False])
    U = I.random_state(mesh, 750 + p)
    lam = I.gaussian_cotangent(U.shape, 751 + p)
    s = _solver(mesh, _ns(), prec)
    g = s.rhs_vjp(torch.as_tensor(U).to("cuda", _dt(prec)).contiguous(),
                  torch.as_tensor(lam).to("cuda", _dt(prec)).contiguous())
    s.check()
    if prec == "fp32":
        U, lam = quantize32(U), quantize32(lam)
    ref = vjp(_oracle(mesh, _ns()), torch.as_tensor(U), torch.as_tensor(lam)).numpy()
    err = rel_err(g.double().cpu().numpy(), ref)
    record(f"oi-vjp-{dim}d-p{p}-{prec}", rel=err)
    assert err < TOL[prec], err


def test_oi_geometry_split_interface():
    mesh = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 6), I.wall_stretched_edges(2, 1.3)], [True, False])
    col = np.arange(mesh.n_elem) % 6
    explicit = (col != 2) & (col != 3)
    Uex, Uim = I.random_state(mesh, 760), I.random_state(mesh, 761)
    s = _solver(mesh, _ns(), "fp64")
    s.set_explicit_mask(explicit)
    f = s.rhs_split(torch.as_tensor(Uex).cuda(), torch.as_tensor(Uim).cuda()).cpu().numpy()
    s.check()
    ref = _oracle(mesh, _ns(), explicit=explicit).residual(torch.as_tensor(Uex), torch.as_tensor(Uim)).numpy()
    assert np.all(f[~explicit] == 0)
    err = rel_err(f[explicit], ref[explicit])
    record("oi-split-2d", rel=err)
    assert err < TOL["fp64"], err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_oi_ark_step_and_adjoint(prec):
    """One ARS(3,4,3) step with the over-integrated operator and its discrete
    adjoint against the oracle's recurrences; the one-call step + adjoint
    equals the separate calls bit for bit."""
    from paper_2607_16044_b300.tableaux import ars343_explicit
    mesh = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 5), I.wall_stretched_edges(2, 1.3)], [True, False])
    phys = _ns()
    U0 = I.random_state(mesh, 770)
    lam0 = I.gaussian_cotangent(U0.shape, 771)
    dt = 2e-5
    s = _solver(mesh, phys, prec)
    s.set_tableau(*ars343_explicit())
    U = torch.as_tensor(U0).cuda()
    s.ark_step(U, dt)
    Us = torch.as_tensor(U0).cuda()
    stages = s.stage_buffer()
    s.ark_step_stages(Us, dt, stages)
    lam = torch.as_tensor(lam0).cuda()
    s.ark_adjoint_step(stages, lam, dt)
    U2, lam2 = torch.as_tensor(U0).cuda(), torch.as_tensor(lam0).cuda()
    s.ark_step_adjoint(U2, lam2, dt, s.stage_buffer())
    s.check()
    assert torch.equal(Us, U2) and torch.equal(lam, lam2)
    op = _oracle(mesh, phys)
    A, b, c = ark.ars343()
    Uref, ys, _ = ark.erk_step(op.residual, torch.as_tensor(U0), dt, A, b, return_stages=True)
    err = rel_err(U.cpu().numpy() - U0, Uref.numpy() - U0)
    record(f"oi-ark-{prec}", rel=err)
    assert err < TOL[prec], err
    assert rel_err(Us.cpu().numpy() - U0, Uref.numpy() - U0) < TOL[prec]
    if prec == "fp32":
        ys = [torch.as_tensor(quantize32(y.numpy())) for y in ys]
    ref = ark.erk_adjoint_step(lambda y, mu: vjp(op, y, mu), ys, torch.as_tensor(lam0), dt, A, b).numpy()
    err = rel_err(lam.cpu().numpy() - lam0, ref - lam0)
    record(f"oi-ark-adjoint-{prec}", rel=err)
    assert err < TOL[prec], err


def test_oi_differs_from_collocated_where_it_should():
    """On a rough state the order-3k rule changes the residual (aliasing);
    on a uniform flow both vanish."""
    mesh = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 5), I.uniform_edges(0, 1, 4)], [True, True])
    U = torch.as_tensor(I.random_state(mesh, 780)).cuda()
    f0 = _solver(mesh, _ns(), "fp64", None).rhs(U)
    f1 = _solver(mesh, _ns(), "fp64").rhs(U)
    assert float((f1 - f0).abs().max() / f0.abs().max()) > 1e-4
    Uc = torch.zeros_like(U)
    Uc[:, 0], Uc[:, 1], Uc[:, 2], Uc[:, 3] = 1.2, 0.3, -0.2, 3.0
    assert float(_solver(mesh, _ns(), "fp64").rhs(Uc).abs().max()) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_oi_channel2d_p3_full_size_sampled(prec):
    """The 256 x 128 wall-stretched 2D channel at p = 3 with the order-3k rule
    (M = 5): sampled elements including both walls against the oracle on
    their 2-ring sub-mesh; FP32 on the 10 %-perturbed state."""
    mesh, phys, _ = I.channel2d_workload(p=3)
    U = I.channel_state(mesh, phys, 2, amp=0.1 if prec == "fp32" else 1e-3)
    s = _solver(mesh, phys, prec)
    f = s.rhs(torch.as_tensor(U).to("cuda", _dt(prec)).contiguous()).double().cpu().numpy()
    s.check()
    rng = np.random.default_rng(19)
    rows = np.unique(np.concatenate([rng.choice(mesh.n_elem, 16, replace=False), [0, mesh.n_elem - 1]]))
    Uref = U if prec == "fp64" else quantize32(U)
    sub, keep, loc = submesh_around(mesh, rows, 2)
    ref = _oracle(sub, phys).residual(torch.as_tensor(Uref[keep])).numpy()[loc]
    err = rel_err(f[rows], ref)
    record(f"oi-channel2d-p3-{prec}", rel=err, sampled=len(rows))
    assert err < TOL[prec], err


def test_oi_handle_bookkeeping():
    """An over-integrated handle: the event profiler reports the two transfers
    and the point operator's three DG-IP kernels per residual; a non-finite
    state is flagged through the point operator's kernels; the calls it does
    not support answer DGX_EUNSUPPORTED; the allocation-free entry point gives
    the workspace-based residual."""
    import ctypes
    from paper_2607_16044_b300.dgx import DGXError
    mesh = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 4), I.wall_stretched_edges(2, 1.3)], [True, False])
    s = _solver(mesh, _ns(), "fp64")
    U = torch.as_tensor(I.random_state(mesh, 790)).cuda()
    f = s.rhs(U)
    s.profile(True)
    s.profile_reset()
    for _ in range(3):
        s.rhs(U, out=f)
    torch.cuda.synchronize()
    prof = s.profile_read()
    s.profile(False)
    assert {k: v[0] for k, v in prof.items()} == {"oi_to_quad": 3, "oi_to_nodes": 3, "dgip_trace": 3,
                                                   "dgip_face": 3, "dgip_elem": 3}
    for k in prof:
        fl, by = s.kernel_work(k)
        assert fl > 0 and by > 0
    out = torch.full_like(U, float("nan"))
    assert s.lib.dgx_rhs_noalloc(s.h, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    torch.cuda.synchronize()
    assert torch.equal(out, f)
    s.check()
    Ubad = U.clone()
    Ubad[3, 0, 2] = float("nan")
    s.rhs(Ubad)
    with pytest.raises(DGXError) as err:
        s.check()
    assert err.value.code == 4  # DGX_ENONFINITE
    s.check()  # the flag was cleared
    Uh = torch.zeros((mesh.n_elem, 4, 4, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(DGXError) as err:
        s.hdg_blocks(U, Uh, 0.1)
    assert err.value.code == 6  # DGX_EUNSUPPORTED


def test_oi_channel3d_p5_full_size_sampled():
    """The 48^3 p = 5 channel with the order-3k rule (8 points per direction,
    the bench's over-integration leg), FP64: residual and VJP rows of sampled
    elements against the oracle on the rings around them, on the 10 %-perturbed
    state (on the 1e-3-perturbed one the residual is a small difference of
    large terms across the 2e-5-thin wall cells, and its rounding floor sits
    at the 1e-12 bar)."""
    from tests.test_gpu_dgip import _sampled_rows_and_vjp
    mesh, phys, _ = I.channel3d_workload()
    U = I.channel_state(mesh, phys, 5, amp=0.1)
    lam = I.gaussian_cotangent(U.shape, 107)
    s = _solver(mesh, phys, "fp64")
    assert s.quad_points == 8
    Ud = torch.as_tensor(U).cuda()
    f = s.rhs(Ud).cpu().numpy()
    g = s.rhs_vjp(Ud, torch.as_tensor(lam).cuda()).cpu().numpy()
    s.check()
    del s, Ud
    torch.cuda.empty_cache()
    rng = np.random.default_rng(13)
    rows = np.unique(np.concatenate([rng.choice(mesh.n_elem, 4, replace=False), [0, mesh.n_elem - 1]]))
    fref, gref = _sampled_rows_and_vjp(lambda m: OverIntegratedSIPG(m, gas_of(phys)), mesh, U, lam, rows)
    ferr, gerr = rel_err(f[rows], fref), rel_err(g[rows], gref)
    record("oi-channel3d-p5-fp64", rel=ferr, vjp_rel=gerr, sampled=len(rows))
    assert ferr < TOL["fp64"], ferr
    assert gerr < TOL["fp64"], gerr


# ---------------------------------------------------------------- curved elements
# f = J^-1 Pi (J' f'(I U)): the point operator runs on the element maps
# evaluated at the M points; the projection carries the Jacobians.

def _curved(dim, p, kind="warped"):
    if dim == 2 and kind == "warped":   # J is no degree-p polynomial (mixed warp)
        return I.rotate_elements(I.warped_mesh(p, [5, 4], [1.0, 1.3], 0.03, mixed=True), 40 + p)
    if dim == 2:                        # rotated local frames, wall-stretched layers, adiabatic walls
        return I.rotate_elements(I.structured_box_mesh(p, [I.uniform_edges(0, 1, 5), I.wall_stretched_edges(2, 1.4)],
                                                       [True, False]), 41 + p)
    if kind == "warped":
        return I.warped_mesh(p, [3, 3, 2], [1.0, 1.0, 1.0], 0.02, mixed=True)
    return I.rotate_elements(I.structured_box_mesh(p, [I.uniform_edges(0, 1, 2), I.uniform_edges(0, 1.2, 2),
                                                       I.wall_stretched_edges(1, 1.0)], [True, True, False]), 42 + p)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("dim", [2, 3])
def test_oi_curved_rhs(dim, p, prec):
    _rhs_check(_curved(dim, p), _ns(), prec, f"oi-curved-{dim}d-p{p}-{prec}", seed=800 + p)


@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("dim,p", [(2, 2), (2, 4), (3, 2), (3, 3)])
def test_oi_curved_walls_rotated(dim, p, viscous):
    _rhs_check(_curved(dim, p, "rotated"), _ns() if viscous else _euler(), "fp64",
               f"oi-rotated-{dim}d-p{p}-{viscous}", seed=810 + p)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,p", [(2, 2), (2, 3), (2, 5), (3, 2), (3, 4)])
def test_oi_curved_vjp(dim, p, prec):
    mesh = _curved(dim, p)
    U = I.random_state(mesh, 820 + p)
    lam = I.gaussian_cotangent(U.shape, 821 + p)
    s = _solver(mesh, _ns(), prec)
    g = s.rhs_vjp(torch.as_tensor(U).to("cuda", _dt(prec)).contiguous(),
                  torch.as_tensor(lam).to("cuda", _dt(prec)).contiguous())
    s.check()
    if prec == "fp32":
        U, lam = quantize32(U), quantize32(lam)
    ref = vjp(_oracle(mesh, _ns()), torch.as_tensor(U), torch.as_tensor(lam)).numpy()
    err = rel_err(g.double().cpu().numpy(), ref)
    record(f"oi-curved-vjp-{dim}d-p{p}-{prec}", rel=err)
    assert err < TOL[prec], err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_oi_curved_ark_step_and_adjoint(prec):
    from paper_2607_16044_b300.tableaux import ars343_explicit
    mesh = _curved(2, 3)
    phys = _ns()
    U0 = I.random_state(mesh, 830)
    lam0 = I.gaussian_cotangent(U0.shape, 831)
    dt = 2e-5
    s = _solver(mesh, phys, prec)
    s.set_tableau(*ars343_explicit())
    U = torch.as_tensor(U0).cuda()
    stages = s.stage_buffer()
    s.ark_step_stages(U, dt, stages)
    lam = torch.as_tensor(lam0).cuda()
    s.ark_adjoint_step(stages, lam, dt)
    s.check()
    op = _oracle(mesh, phys)
    A, b, c = ark.ars343()
    Uref, ys, _ = ark.erk_step(op.residual, torch.as_tensor(U0), dt, A, b, return_stages=True)
    err = rel_err(U.cpu().numpy() - U0, Uref.numpy() - U0)
    record(f"oi-curved-ark-{prec}", rel=err)
    assert err < TOL[prec], err
    if prec == "fp32":
        ys = [torch.as_tensor(quantize32(y.numpy())) for y in ys]
    ref = ark.erk_adjoint_step(lambda y, mu: vjp(op, y, mu), ys, torch.as_tensor(lam0), dt, A, b).numpy()
    err = rel_err(lam.cpu().numpy() - lam0, ref - lam0)
    record(f"oi-curved-ark-adjoint-{prec}", rel=err)
    assert err < TOL[prec], err


def test_oi_curved_geometry_split_interface():
    mesh = _curved(2, 3)
    col = np.arange(mesh.n_elem) % 5
    explicit = col != 2
    Uex, Uim = I.random_state(mesh, 840), I.random_state(mesh, 841)
    s = _solver(mesh, _ns(), "fp64")
    s.set_explicit_mask(explicit)
    f = s.rhs_split(torch.as_tensor(Uex).cuda(), torch.as_tensor(Uim).cuda()).cpu().numpy()
    s.check()
    ref = _oracle(mesh, _ns(), explicit=explicit).residual(torch.as_tensor(Uex), torch.as_tensor(Uim)).numpy()
    assert np.all(f[~explicit] == 0)
    err = rel_err(f[explicit], ref[explicit])
    record("oi-curved-split-2d", rel=err)
    assert err < TOL["fp64"], err


def test_oi_curved_mesh_changes_and_geometry_override():
    """Replacing a curved mesh by boxes drops the Jacobian weights (the box
    result equals a fresh box handle's bit for bit) and a new curved mesh
    brings them back; M = p+1 on a curved mesh is the collocated operator up
    to the rounding of the weights; the nodal geometry override is refused."""
    from paper_2607_16044_b300.dgx import DGXError
    curved = _curved(2, 3)
    boxes = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 5), I.uniform_edges(0, 1.3, 4)], [True, True])
    U = torch.as_tensor(I.random_state(curved, 850)).cuda()
    s = _solver(curved, _ns(), "fp64")
    f_curved = s.rhs(U).clone()
    s.set_mesh(boxes)
    assert torch.equal(s.rhs(U), _solver(boxes, _ns(), "fp64").rhs(U))
    s.set_mesh(curved)
    assert torch.equal(s.rhs(U), f_curved)
    f0 = _solver(curved, _ns(), "fp64", None).rhs(U)
    f1 = _solver(curved, _ns(), "fp64", curved.p + 1).rhs(U)
    assert float((f1 - f0).abs().max() / f0.abs().max()) < 1e-14
    J = np.ones((curved.n_elem, curved.N))
    metric = np.zeros((curved.n_elem, curved.N, 2, 2))
    metric[..., 0, 0] = metric[..., 1, 1] = 1.0
    with pytest.raises(DGXError) as err:
        s.set_geometry(J, metric)
    assert err.value.code == 6  # DGX_EUNSUPPORTED
    s.check()
