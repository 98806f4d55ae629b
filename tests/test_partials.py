"""Vertex partials (heget.cuh): each amplitude vertex -- vvvxxx, ggggxx,
iovxx0 of arXiv:0909.5257 Sec. 4 -- equals the contraction of any one of its
wavefunctions with the partial vertex of the others.  The generator uses this
to share the partial between diagrams.  The checks compile the device library
(and the generator) for the host: both forms of each vertex on random complex
inputs, and whole programs built with and without partials."""
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


def test_schedules_compute_the_same_colour_amplitudes(tmp_path):
    """The generator's program with shared vertex partials (either schedule
    order) and the one with a vertex call per diagram give the same colour
    amplitudes on random inputs and share one mask table (the straight-line
    kernels of every variant read the runtime program's table)."""
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "program_variants_check")
    subprocess.run([cxx, "-O1", "-std=c++17", "-fopenmp", "-I", CSRC, "-o", exe,
                    os.path.join(HERE, "native", "program_variants_check.cpp"),
                    os.path.join(CSRC, "generator.cpp")], check=True)
    procs = ["21,21,21,21,21", "2,-2,21,21,21", "2,2,2,2,21", "21,21,21,21,21,21",
             "2,-2,21,21,21,21", "2,2,2,2,21,21", "2,2,2,2,21,21,21", "2,21,2,21,21", "2,-2,1,-1,21",
             "2,-2,21,21,21,21,21", "21,21,21,21,21,21,21"]
    r = subprocess.run([exe] + procs, capture_output=True, text=True)
    assert r.returncode == 0, "mask tables differ between build options"
    lines = r.stdout.split()
    for k in range(len(procs)):
        name, worst, n_part = lines[3 * k], float(lines[3 * k + 1]), int(lines[3 * k + 2])
        assert worst < 1e-13, (name, worst)
    assert int(lines[3 * 3 + 2]) > 0  # gg > gggg shares partials
    assert int(lines[3 * 10 + 2]) == 81 + 225  # gg > ggggg: vvv and gggg groups
