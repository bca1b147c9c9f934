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
    assert lib.dgx_ark_step_stages(None, None, 1e-3, None, None, None) == 1
    assert lib.dgx_ark_adjoint_step(None, None, None, 1e-3, None, None) == 1
    assert lib.dgx_workspace_bytes(None, dgx.OP_ARK_STEP_ADJOINT) == 0
