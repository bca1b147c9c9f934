"""The C-ABI library loads and exports every entry point that include/dgx.h declares (CPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dgx.h")
LIB = os.path.join(ROOT, "paper_2607_16044_b300", "libdgx.so")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dgx_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_entry_points():
    names = declared()
    for required in ("dgx_create", "dgx_rhs", "dgx_rhs_vjp", "dgx_ark_step", "dgx_check", "dgx_destroy"):
        assert required in names


@pytest.mark.skipif(not os.path.exists(LIB), reason="library not built")
def test_library_exports_every_declared_symbol():
    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True, check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing


@pytest.mark.skipif(not os.path.exists(LIB), reason="library not built")
def test_library_loads_without_gpu():
    from paper_2607_16044_b300 import dgx
    lib = dgx.load_library()
    assert lib.dgx_status_string(0) == b"ok"
    assert lib.dgx_workspace_bytes(None, 0) == 0
    for name in declared():
        assert hasattr(lib, name)


@pytest.mark.skipif(not os.path.exists(LIB), reason="library not built")
def test_host_validation_without_gpu():
    """Host-side argument checks answer before any device work."""
    from paper_2607_16044_b300 import dgx
    lib = dgx.load_library()
    assert lib.dgx_ark_step_adjoint(None, None, None, 1e-3, None, None, None) == 1
    assert lib.dgx_set_wait_limit(None, 0) == 1
    assert lib.dgx_rhs_split(None, None, None, None, None, None) == 1
    assert lib.dgx_set_farfield(None, None) == 1
    assert lib.dgx_ark_step_stages(None, None, 1e-3, None, None, None) == 1
    assert lib.dgx_ark_adjoint_step(None, None, None, 1e-3, None, None) == 1
    assert lib.dgx_workspace_bytes(None, dgx.OP_ARK_STEP_ADJOINT) == 0


def _enum_values(prefix):
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(" + prefix + r"[A-Z0-9_]+)\s*=\s*(\d+)", text)}


def test_binding_constants_match_header():
    """The Python binding's operation, contraction and kernel-kind numbers are
    the ones include/dgx.h declares."""
    from paper_2607_16044_b300 import dgx
    ops = _enum_values("DGX_OP_")
    assert (dgx.OP_RHS, dgx.OP_VJP, dgx.OP_ARK, dgx.OP_ARK_ADJOINT, dgx.OP_ARK_STEP_ADJOINT) == (
        ops["DGX_OP_RHS"], ops["DGX_OP_VJP"], ops["DGX_OP_ARK"], ops["DGX_OP_ARK_ADJOINT"],
        ops["DGX_OP_ARK_STEP_ADJOINT"])
    con = _enum_values("DGX_CONTRACT_")
    assert dgx.CONTRACTIONS == {"cuda_core": con["DGX_CONTRACT_CUDA_CORE"], "tf32": con["DGX_CONTRACT_TF32"],
                                "bf16": con["DGX_CONTRACT_BF16"], "3xtf32": con["DGX_CONTRACT_3XTF32"]}
    kinds = _enum_values("DGX_K")
    assert len(dgx.KERNELS) == kinds["DGX_KERNEL_KINDS"]
    for i, name in enumerate(dgx.KERNELS):
        assert kinds["DGX_K_" + name.upper()] == i


def test_problem_desc_layout_matches_header(tmp_path):
    """The binding's dgx_problem_desc has the header's fields at the header's
    offsets (compiled with the host C compiler)."""
    import ctypes
    from paper_2607_16044_b300 import dgx
    names = [n for n, _ in dgx._Desc._fields_]
    src = tmp_path / "desc.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "dgx.h"\nint main(void) {\n'
                   + "".join(f'  printf("%zu\\n", offsetof(dgx_problem_desc, {n}));\n' for n in names)
                   + '  printf("%zu\\n", sizeof(dgx_problem_desc));\n  return 0;\n}\n')
    exe = tmp_path / "desc"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [getattr(dgx._Desc, n).offset for n in names] + [ctypes.sizeof(dgx._Desc)]
    assert got == want


@pytest.mark.skipif(not os.path.exists(LIB), reason="library not built")
def test_over_integration_descriptor_checks_without_gpu():
    """quad_points below p + 1 is invalid; above 8 points (the largest rule), or
    with the LLF scheme, unsupported (answered before any device work)."""
    import ctypes
    from paper_2607_16044_b300 import dgx
    lib = dgx.load_library()

    def create(p, M, scheme="dgip"):
        conv, visc = dgx.SCHEMES[scheme]
        d = dgx._Desc(2, p, 4, 1, dgx.FP64, 1.4, 100.0, 0.72, 0.3, conv, visc, 1.0, M)
        h = ctypes.c_void_p()
        return lib.dgx_create(ctypes.byref(d), ctypes.byref(h))

    status = _enum_values("DGX_E")
    assert create(3, 3) == status["DGX_EINVAL"]
    assert create(5, 9) == status["DGX_EUNSUPPORTED"]
    assert create(2, 4, "llf-br1") == status["DGX_EUNSUPPORTED"]
