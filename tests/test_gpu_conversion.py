"""FP64 -> FP32 conversion of the ARK step's state: the rounded stage state
y_1 = fl32(U_n) that the first kernel of an FP32 ARK step stores must equal
IEEE round-to-nearest-even bit for bit,
here against numpy's float64 -> float32 cast, on doubles chosen to exercise
the rounding: exact ties of both parities, values just above and below a
tie, the ends of the binary32 normal range (including rounding up to
infinity), binary32 subnormal results, zeros and random magnitudes.  The state
is not physical, so the residual kernels that follow flag non-finite values;
only the stored conversion is compared."""
import numpy as np
import pytest
import torch

from paper_2607_16044_b300 import inputs as I
from paper_2607_16044_b300.tableaux import ars343_explicit

pytestmark = pytest.mark.gpu


def _doubles(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        m = int(rng.integers(0, 1 << 23))
        ex = int(rng.integers(897, 1151))  # binary32 normal range
        sign = int(rng.integers(0, 2)) << 63
        for low in (0x10000000, 0x0FFFFFFF, 0x10000001, 0, 0x1FFFFFFF, int(rng.integers(0, 1 << 29))):
            out.append(np.uint64(sign | (ex << 52) | (m << 29) | low).view(np.float64))
    out = np.array(out[:count], dtype=np.float64)
    special = np.array([3.4028234663852886e38, 3.4028235677973366e38, -3.4028235677973366e38,
                        1.1754943508222875e-38, 1.1754942e-38, 7e-39, 1.401298464324817e-45, 7e-46,
                        0.0, -0.0, 1.0, -2.5, 1e-300, 1e39])
    mags = rng.standard_normal(count // 4) * 10.0 ** rng.integers(-44, 39, count // 4)
    return np.concatenate([special, mags, out])


def test_state_rounding_bitwise():
    from paper_2607_16044_b300.dgx import DGXError, Solver
    mesh = I.structured_box_mesh(2, [I.uniform_edges(0, 1, 16), I.uniform_edges(0, 1, 16)], [True, True])
    phys = I.Physics(gamma=1.4, Re=100.0, Pr=0.72, Ma=0.3, viscous=True)
    s = Solver(mesh, phys, "fp32")
    s.set_tableau(*ars343_explicit())
    shape = (mesh.n_elem, mesh.dim + 2, mesh.N)
    vals = _doubles(int(np.prod(shape)), 3)[: int(np.prod(shape))]
    U = torch.as_tensor(vals.reshape(shape)).cuda()
    stages = s.stage_buffer()
    s.ark_step_stages(U, 0.0, stages)
    torch.cuda.synchronize()
    y1 = s.stage_state(stages, 0).cpu().numpy()
    with np.errstate(over="ignore"):
        ref = vals.reshape(shape).astype(np.float32)
    try:
        s.check()
    except DGXError as e:   # non-physical state: the residual kernels flag it
        assert e.code == 4, e
    assert np.array_equal(y1.view(np.uint32), ref.view(np.uint32))
