"""The allocation-free residual entry point (dgx_rhs_noalloc) against dgx_rhs.

Some callers cannot allocate device memory while they run (hosts that reserve
all device memory at start-up, plugin hosts that pass only inputs and
outputs); dgx_rhs_noalloc serves them from a fixed scratch array inside the
library.  These tests call it through the C ABI and compare with the
workspace-based dgx_rhs on two consecutive calls (the scratch keeps the first
call's contents, which must not leak into the second; the device's free
memory must not change across the second call), and check that a mesh too
large for the fixed scratch is rejected.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2607_16044_b300 import inputs as I
from tests.parity_util import TOL, rel_err

pytestmark = pytest.mark.gpu


def _solver(mesh, phys, prec="fp64"):
    from paper_2607_16044_b300.dgx import Solver
    return Solver(mesh, phys, prec)


def _noalloc(s, U, out):
    lib = s.lib
    code = lib.dgx_rhs_noalloc(s.h, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return code


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_matches_rhs_on_two_calls(prec):
    mesh = I.structured_box_mesh(3, [I.uniform_edges(0, 1, 9), I.wall_stretched_edges(3, 1.3)], [True, False])
    phys = I.Physics(gamma=1.4, Re=300.0, Pr=0.72, Ma=0.3, viscous=True)
    s = _solver(mesh, phys, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    # every tensor the test needs exists before the first call, so nothing
    # else allocates device memory between the two calls
    Us = [torch.as_tensor(I.random_state(mesh, seed)).to("cuda", dt).contiguous() for seed in (1, 2)]
    refs = [s.rhs(U).double().cpu().numpy() for U in Us]
    outs = [torch.full_like(U, float("nan")) for U in Us]
    torch.cuda.synchronize()
    # first call: the warm-up that creates the fixed array under lazy loading
    assert _noalloc(s, Us[0], outs[0]) == 0
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    # second call in a row, on another state: must allocate nothing
    assert _noalloc(s, Us[1], outs[1]) == 0
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before, (free_before, free_after)
    s.check()
    for out, ref in zip(outs, refs):
        got = out.double().cpu().numpy()
        assert rel_err(got, ref) < TOL[prec]


def test_noalloc_rejects_meshes_beyond_the_fixed_scratch():
    # 3D, p = 5, FP64, NS: about 52 KB of scratch per element -> 1400 elements > 64 MiB
    mesh = I.structured_box_mesh(5, [I.uniform_edges(0, 1, 14), I.uniform_edges(0, 1, 10),
                                     I.uniform_edges(0, 1, 10)], [True, True, True])
    phys = I.Physics(gamma=1.4, Re=300.0, Pr=0.72, Ma=0.3, viscous=True)
    s = _solver(mesh, phys, "fp64")
    assert s.lib.dgx_workspace_bytes(s.h, 0) > 64 * 1024 * 1024
    U = torch.as_tensor(I.random_state(mesh, 3)).cuda()
    out = torch.empty_like(U)
    assert _noalloc(s, U, out) == 1          # DGX_EINVAL, nothing launched
