"""GPU parity of the element-local HDG-IP Newton blocks (dgx_hdg_blocks) and
their static condensation (dgx_hdg_condense) against the oracle (oracle.hdg):
the forms' values, K, C, D, A33, K^{-1} C and the element Schur contribution."""
import numpy as np
import pytest
import torch

from oracle import physics as ph
from oracle.hdg import HDGIPLocal
from paper_2607_16044_b300 import inputs as I
from tests.parity_util import gas_of, record

pytestmark = pytest.mark.gpu

UINF = np.array([1.1, 0.4, -0.3, 2.0 / 0.4 + 0.5 * (0.4 ** 2 + 0.3 ** 2) / 1.1])


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _check_blocks(mesh, phys, tag, scheme, case, p):
    from paper_2607_16044_b300.dgx import Solver
    U0 = I.random_state(mesh, 20 + p)
    op = HDGIPLocal(mesh, gas_of(phys), U_inf=UINF if tag else None)
    T = op.element_traces(op.nodes(torch.as_tensor(U0)))
    Uh0 = (T * (1 + 0.05 * torch.as_tensor(np.random.default_rng(30 + p).standard_normal(tuple(T.shape))))).numpy()
    gamma = 0.0137
    s = Solver(mesh, phys, "fp64", scheme=scheme, U_inf=UINF if tag else None)
    K, C, D, A, R, h = s.hdg_blocks(torch.as_tensor(U0).cuda(), torch.as_tensor(Uh0).cuda().contiguous(), gamma,
                                   forms=True)
    KinvC, S = s.hdg_condense(K, C, D, A)
    s.check()
    Rr, hr = op.forms(torch.as_tensor(U0), torch.as_tensor(Uh0))
    Kr, Cr, Dr, Ar = op.blocks(U0, Uh0, gamma)
    KCr, Sr = op.schur(U0, Uh0, gamma)
    errs = {"R": _rel(R.cpu(), Rr.reshape(mesh.n_elem, -1)), "h": _rel(h.cpu(), hr.reshape(mesh.n_elem, -1)),
            "K": _rel(K.cpu(), Kr), "C": _rel(C.cpu(), Cr), "D": _rel(D.cpu(), Dr), "A33": _rel(A.cpu(), Ar),
            "KinvC": _rel(KinvC.cpu(), KCr), "S": _rel(S.cpu(), Sr)}
    record(f"hdg-{case}", **errs)
    for k, v in errs.items():
        assert v < 1e-12, (k, v)


@pytest.mark.parametrize("case", ["walls-p1", "walls-p2", "walls-p3", "walls-p4", "walls-p5", "farfield-p2",
                                  "euler-p3"])
def test_hdg_blocks_and_condensation_match_oracle(case):
    kind, p = case.split("-p")
    p = int(p)
    tag = 1 if kind == "farfield" else 0
    cols = 2 if p <= 3 else 1
    mesh = I.structured_box_mesh(p, [I.uniform_edges(0, 1, cols), I.wall_stretched_edges(1, 1.0)], [True, False],
                                 wall_tag=tag)
    phys = I.Physics(gamma=1.4, Re=100.0, Pr=0.72, Ma=0.3, viscous=kind != "euler")
    _check_blocks(mesh, phys, tag, "dgip" if tag else "llf-br1", case, p)


@pytest.mark.parametrize("case", ["warped-p2", "warped-p3", "warped-p5", "rotated-walls-p3", "warped-farfield-p2",
                                  "warped-euler-p4"])
def test_hdg_blocks_on_curved_elements_match_oracle(case):
    """Curved elements (the paper's implicit region lies on curved walls):
    warps whose J is no degree-p polynomial, rotated wall elements, farfield
    faces on a warped mesh; the blocks from the metric terms at the nodes and
    traced to the faces (a DG-IP handle's curved geometry)."""
    kind, p = case.rsplit("-p", 1)
    p = int(p)
    tag = 1 if "farfield" in kind else 0
    if kind == "rotated-walls":
        mesh = I.rotate_elements(I.structured_box_mesh(p, [I.uniform_edges(0, 1, 2), I.wall_stretched_edges(1, 1.0)],
                                                       [True, False]), 50 + p)
    else:
        periodic = [True, not tag]
        mesh = I.rotate_elements(I.warped_mesh(p, [3, 2], [1.0, 1.3], 0.03, periodic=periodic, mixed=True), 51 + p)
        if tag:
            nb = mesh.neighbor.copy()
            nb[nb == -1] = -2                      # the box walls become farfield faces
            mesh = I.Mesh(2, mesh.p, mesh.n_elem, "nodes", mesh.xyz, nb, mesh.nbr_face, mesh.orient)
    phys = I.Physics(gamma=1.4, Re=100.0, Pr=0.72, Ma=0.3, viscous="euler" not in kind)
    _check_blocks(mesh, phys, tag, "dgip", f"curved-{case}", p)
