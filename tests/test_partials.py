"""Vertex partials (heget.cuh): each amplitude vertex -- vvvxxx, ggggxx,
iovxx0 of arXiv:0909.5257 Sec. 4 -- equals the contraction of any one of its
wavefunctions with the partial vertex of the others.  The generator uses this
to share the partial between diagrams; the check compiles the device library
for the host and compares both forms on random complex inputs."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_0909_5257_gb300", "csrc")


def test_partial_contractions_equal_the_vertex_functions(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "partials_check")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, "-o", exe,
                    os.path.join(HERE, "native", "partials_check.cpp")], check=True)
    worst = float(subprocess.run([exe], check=True, capture_output=True, text=True).stdout)
    assert worst < 1e-14
