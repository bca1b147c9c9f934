"""Host-side checks of the kernels' pointwise physics (compiled for the CPU
with nvcc, no GPU): the axis-normal viscous flux that box faces use, and its
hand-derived adjoint, against the full-tensor flux through the same normal."""
import os
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2607_16044_b300", "csrc")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


@pytest.mark.skipif(not os.path.exists(NVCC), reason="nvcc not available")
def test_axis_viscous_flux_matches_the_full_flux():
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "axis_flux_check")
        cmd = [NVCC, "-std=c++17", "--expt-relaxed-constexpr", "-x", "cu", "-I", CSRC,
               os.path.join(HERE, "axis_flux_check.cu"), "-o", exe]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        out = subprocess.run([exe], capture_output=True, text=True)
        assert out.returncode == 0, out.stdout + out.stderr
        assert "OK" in out.stdout


@pytest.mark.skipif(not os.path.exists(NVCC), reason="nvcc not available")
def test_dgip_box_face_function_matches_the_general_form():
    """The DG-IP face function with an axis normal (rank-one axis K-products,
    no |n|) against the general form: values, dual-number tangents and the
    hand-derived interior adjoint, every axis and orientation, 2D and 3D."""
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "dgip_axis_check")
        cmd = [NVCC, "-std=c++17", "--expt-relaxed-constexpr", "-x", "cu", "-I", CSRC,
               os.path.join(HERE, "dgip_axis_check.cu"), "-o", exe]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        out = subprocess.run([exe], capture_output=True, text=True)
        assert out.returncode == 0, out.stdout + out.stderr
        assert "OK" in out.stdout
