"""dgx_ark_step_adjoint: one ARK step and its adjoint in one call, the kernels
that form U_{n+1} overlapping the adjoint on the handle's second stream.  The
same kernels run on the same inputs as the two separate calls, so U_{n+1},
lambda_n and the stage checkpoints must agree bit for bit; the separate calls
are themselves held to the oracle by test_gpu_vjp and test_gpu_ark."""
import pytest
import torch

from paper_2607_16044_b300 import inputs as I
from paper_2607_16044_b300.tableaux import ars343_explicit

pytestmark = pytest.mark.gpu


def _ns():
    return I.Physics(gamma=1.4, Re=200.0, Pr=0.72, Ma=0.3, viscous=True)


def _euler():
    return I.Physics(gamma=1.4, viscous=False)


CASES = {
    "ns-channel-p4": lambda: I.structured_box_mesh(4, [I.uniform_edges(0, 1, 9), I.wall_stretched_edges(3, 1.3)],
                                                   [True, False]),
    "ns-curved-p3": lambda: I.rotate_elements(I.warped_mesh(3, [5, 4], [1.0, 1.2], 0.04, periodic=[True, False]), 5),
    "euler-3d-p2": lambda: I.structured_box_mesh(2, [I.uniform_edges(0, 1, 3), I.uniform_edges(0, 1, 3),
                                                     I.uniform_edges(0, 1, 4)], [True, True, True]),
}


def _pair(name, prec, seed):
    from paper_2607_16044_b300.dgx import Solver
    mesh = CASES[name]()
    phys = _euler() if name.startswith("euler") else _ns()
    U0 = torch.as_tensor(I.random_state(mesh, seed)).cuda()
    lam0 = torch.as_tensor(I.gaussian_cotangent(tuple(U0.shape), seed + 1)).cuda()
    s = Solver(mesh, phys, prec)
    s.set_tableau(*ars343_explicit())
    return s, U0, lam0


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_step_adjoint_matches_separate_calls(name, prec):
    s, U0, lam0 = _pair(name, prec, 31)
    dt = 1e-4
    U_a, lam_a, st_a = U0.clone(), lam0.clone(), s.stage_buffer()
    s.ark_step_stages(U_a, dt, st_a)
    s.ark_adjoint_step(st_a, lam_a, dt)
    U_b, lam_b, st_b = U0.clone(), lam0.clone(), s.stage_buffer()
    s.ark_step_adjoint(U_b, lam_b, dt, st_b)
    s.check()
    assert torch.equal(U_a, U_b)
    assert torch.equal(lam_a, lam_b)
    for i in range(s.stages):
        assert torch.equal(s.stage_state(st_a, i), s.stage_state(st_b, i))


def test_step_adjoint_graph_replay():
    """Captured into a CUDA graph (fork and join across the handle's streams)
    and replayed: the same bits as the eager call, step after step."""
    s, U0, lam0 = _pair("ns-channel-p4", "fp32", 41)
    dt = 1e-4
    U_e, lam_e, st_e = U0.clone(), lam0.clone(), s.stage_buffer()
    U_g, lam_g, st_g = U0.clone(), lam0.clone(), s.stage_buffer()
    s.ark_step_adjoint(U_g, lam_g, dt, st_g)       # creates the workspace before capture
    s.check()
    g = s.capture(lambda: s.ark_step_adjoint(U_g, lam_g, dt, st_g), warmup=0)
    for _ in range(3):
        U_g.copy_(U0)
        lam_g.copy_(lam0)
        g.replay()
        torch.cuda.synchronize()
        U_e.copy_(U0)
        lam_e.copy_(lam0)
        s.ark_step_adjoint(U_e, lam_e, dt, st_e)
        s.check()
        assert torch.equal(U_e, U_g)
        assert torch.equal(lam_e, lam_g)


def test_step_adjoint_workspace_and_validation():
    from paper_2607_16044_b300.dgx import (DGXError, OP_ARK, OP_ARK_ADJOINT, OP_ARK_STEP_ADJOINT, Solver)
    s, U0, lam0 = _pair("ns-channel-p4", "fp32", 51)
    lib, h = s.lib, s.h
    assert lib.dgx_workspace_bytes(h, OP_ARK_STEP_ADJOINT) == (lib.dgx_workspace_bytes(h, OP_ARK)
                                                               + lib.dgx_workspace_bytes(h, OP_ARK_ADJOINT))
    with pytest.raises(DGXError):   # no tableau: call out of order
        t = Solver(CASES["ns-channel-p4"](), _ns(), "fp32")
        t.ark_step_adjoint(U0.clone(), lam0.clone(), 1e-4, s.stage_buffer())
    ws = s.workspace(OP_ARK_STEP_ADJOINT)
    stages = s.stage_buffer()
    assert lib.dgx_ark_step_adjoint(h, U0.data_ptr(), lam0.data_ptr(), float("nan"), stages.data_ptr(),
                                    s._aligned(ws), None) == 1
    assert lib.dgx_ark_step_adjoint(h, U0.data_ptr(), lam0.data_ptr(), 1e-4, stages.data_ptr() + 8,
                                    s._aligned(ws), None) == 1
