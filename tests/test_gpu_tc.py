"""Tensor-core (tcgen05) contraction engine of the FP32 element kernel.

TF32 rounds every operand of the 1D differentiation / lift contraction to a
10-bit mantissa (unit roundoff 2^-11), so each contracted term carries a
relative error of up to about 2^-10; the residual then deviates from the
oracle by a few 1e-4 of the magnitude of the terms it sums.  BF16 keeps a
7-bit mantissa (unit roundoff 2^-8): eight times coarser, a few 1e-3.  3xTF32
splits each operand into two TF32 parts and keeps three of the four products,
which leaves a 2^-22 relative term: it must meet the FP32 bar of the CUDA-core
path.
"""
import numpy as np
import pytest
import torch

from paper_2607_16044_b300 import inputs as I
from paper_2607_16044_b300.tableaux import ars343_explicit
from tests.parity_util import TOL, oracle_rhs_and_scale, quantize32, record, rel_err, scaled_err
from tests.test_gpu_ark import increment_err

pytestmark = pytest.mark.gpu

TOL_TC = {"tf32": 3e-3, "bf16": 2.4e-2, "3xtf32": TOL["fp32"]}
MODES = ["tf32", "bf16", "3xtf32"]


def _solver(mesh, phys, mode):
    from paper_2607_16044_b300.dgx import Solver
    s = Solver(mesh, phys, "fp32")
    s.set_contraction(mode)
    assert s.contraction == mode
    return s


def _rhs(mesh, phys, U, mode):
    s = _solver(mesh, phys, mode)
    f = s.rhs(torch.as_tensor(U).to("cuda", torch.float32).contiguous())
    s.check()
    return f.double().cpu().numpy()


def _euler():
    return I.Physics(gamma=1.4, viscous=False)


def _ns(Re=200.0):
    return I.Physics(gamma=1.4, Re=Re, Pr=0.72, Ma=0.3, viscous=True)


def _mesh(dim, p, ragged=False):
    if dim == 2:
        nx, ny = (9, 7) if ragged else (8, 6)
        return I.structured_box_mesh(p, [I.uniform_edges(-1, 1, nx), I.wall_stretched_edges(ny // 2, 1.3)],
                                     [True, False])
    cells = {1: 4, 2: 3, 3: 3, 4: 2, 5: 2}[p]
    return I.structured_box_mesh(p, [I.uniform_edges(0, 1, cells), I.uniform_edges(0, 1.2, cells + 1),
                                     I.wall_stretched_edges(1, 1.0)], [True, True, False])


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("dim", [2, 3])
def test_tc_rhs_vs_oracle(dim, p, viscous, mode):
    mesh = _mesh(dim, p, ragged=True)
    phys = _ns() if viscous else _euler()
    U = I.random_state(mesh, 700 + 10 * dim + p)
    got = _rhs(mesh, phys, U, mode)
    ref, T = oracle_rhs_and_scale(mesh, phys, quantize32(U))
    serr, err = scaled_err(got, ref, T), rel_err(got, ref)
    record(f"tc-{mode}-{dim}d-p{p}-{'ns' if viscous else 'euler'}", rel=err, scaled=serr, E=mesh.n_elem)
    assert serr < TOL_TC[mode], serr
    if mode == "3xtf32":
        assert err < TOL["fp32"], err


@pytest.mark.parametrize("mode", MODES)
def test_tc_tgv_periodic_p3(mode):
    """3D Taylor-Green vortex (periodic cube, p = 3) on a 4^3 mesh: the shape of
    the tensor-core comparison workload at a size the oracle evaluates whole."""
    mesh, phys, U = I.tgv_workload(p=3, cells=4)
    got = _rhs(mesh, phys, U, mode)
    ref, T = oracle_rhs_and_scale(mesh, phys, quantize32(U))
    serr = scaled_err(got, ref, T)
    record(f"tc-{mode}-tgv-4^3", scaled=serr, rel=rel_err(got, ref), E=mesh.n_elem)
    assert serr < TOL_TC[mode], serr


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("p", [2, 4])
def test_tc_curvilinear_matches_cuda_core(p, mode):
    """Curvilinear elements (metric terms in the flux): the tensor-core result
    against the CUDA-core FP32 result on the same input, relative to the
    residual's term scale."""
    mesh = I.rotate_elements(I.warped_mesh(p, [5, 4], [1.0, 1.2], 0.04, periodic=[True, False]), 31 + p)
    phys = _ns()
    U = I.random_state(mesh, 900 + p)
    got = _rhs(mesh, phys, U, mode)
    base = _rhs(mesh, phys, U, "cuda_core")
    _, T = oracle_rhs_and_scale(mesh, phys, quantize32(U))
    d = scaled_err(got, base, T)
    record(f"tc-{mode}-curv-p{p}-vs-cuda-core", scaled=d, E=mesh.n_elem)
    assert d < TOL_TC[mode], d


@pytest.mark.parametrize("mode", MODES)
def test_tc_ark_step_matches_cuda_core(mode):
    """Stage-update form of the kernel: three ARS(3,4,3) steps of the NS channel
    with the tensor-core engine against the CUDA-core FP32 steps."""
    from paper_2607_16044_b300.dgx import Solver
    mesh = I.structured_box_mesh(4, [I.uniform_edges(0, 1, 9), I.wall_stretched_edges(3, 1.3)], [True, False])
    phys = _ns()
    U0 = I.random_state(mesh, 77)
    out = {}
    for m in ("cuda_core", mode):
        s = Solver(mesh, phys, "fp32")
        s.set_contraction(m)
        s.set_tableau(*ars343_explicit())
        U = torch.as_tensor(U0).cuda().contiguous()
        for _ in range(3):
            s.ark_step(U, 2e-4)
        s.check()
        out[m] = U.cpu().numpy()
    err = increment_err(out[mode], out["cuda_core"], U0, {"tf32": 3e-3, "bf16": 2.4e-2, "3xtf32": 3e-5}[mode])
    record(f"tc-{mode}-ark-vs-cuda-core", worst=err)
    assert err < 1.0, err


def test_tc_mode_validation():
    from paper_2607_16044_b300.dgx import DGXError, Solver
    mesh = _mesh(2, 3)
    s64 = Solver(mesh, _euler(), "fp64")
    with pytest.raises(DGXError):
        s64.set_contraction("tf32")
    s64.set_contraction("cuda_core")
    s32 = Solver(mesh, _euler(), "fp32")
    with pytest.raises(ValueError):
        s32.set_contraction("fp8")
    s32.set_contraction("bf16")
    assert s32.contraction == "bf16"
    s32.set_contraction("3xtf32")
    assert s32.contraction == "3xtf32"
    s32.set_contraction("cuda_core")
    assert s32.contraction == "cuda_core"


def test_tc_batch_matches_single():
    """A batch built from tensor-core instances steps each one as its own solver does."""
    from paper_2607_16044_b300.dgx import Batch, Solver
    phys = _euler()
    meshes = [I.vortex_workload(p=3, cells=c)[0] for c in (6, 8)]
    solvers, states = [], []
    for k, m in enumerate(meshes):
        s = Solver(m, phys, "fp32")
        s.set_contraction("tf32")
        s.set_tableau(*ars343_explicit())
        solvers.append(s)
        states.append(I.vortex_workload(p=3, cells=(6, 8)[k])[2])
    b = Batch(solvers, [0.01, 0.01])
    U = b.pack([torch.as_tensor(x).cuda() for x in states])
    b.step(U)
    got = b.unpack(U)
    for s, x, g in zip(solvers, states, got):
        ref = torch.as_tensor(x).cuda().contiguous()
        s.ark_step(ref, 0.01)
        s.check()
        assert torch.equal(g.reshape(ref.shape), ref)
