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


def test_helicity_shared_layout_gives_the_per_lane_amplitudes(tmp_path):
    """The helicity-shared layout (helshare.h: every produced wavefunction once
    per helicity pattern of its own legs, in an arena of variant blocks
    released after their last reader) and the split layout (the wavefunctions
    of up to n_ext - 3 legs shared that way in a prologue, level by level, the
    rest per combination with one transient current) give every diagram
    amplitude of every summed helicity combination bit for bit as the
    per-combination evaluation through the program's slots (host, FP64, random
    inputs); every block lies in its arena and no op's output block overlaps
    its inputs.  So does the per-combination evaluation with register
    forwarding, its skipped stores leaving their slots NaN."""
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "helshare_check")
    subprocess.run([cxx, "-O1", "-std=c++17", "-fopenmp", "-I", CSRC, "-o", exe,
                    os.path.join(HERE, "native", "helshare_check.cpp"),
                    os.path.join(CSRC, "generator.cpp"), os.path.join(CSRC, "helshare.cpp")], check=True)
    procs = ["21,21,21,21", "2,-2,21,21", "21,21,21,21,21", "2,2,2,2,21", "21,21,21,21,21,21",
             "2,-2,21,21,21,21", "2,2,2,2,21,21", "2,2,2,2,21,21,21", "2,-2,21,21,21,21,21",
             "21,21,21,21,21,21,21", "2,21,2,21,21", "2,-2,1,-1,21",
             # crossings and other flavours
             "2,1,2,1,21", "2,-2,2,-2,21", "-1,-1,-1,-1,21", "21,2,2,21,21", "2,21,2,21",
             "2,21,2,21,21,21", "2,1,2,1,21,21", "2,-2,1,-1,21,21"]
    r = subprocess.run([exe] + procs, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    rows = [line.split() for line in r.stdout.splitlines()]
    assert [row[0] for row in rows] == procs
    for name, compared, mismatched, arena, s_compared, s_mismatched, s_area, f_compared, f_mismatched in rows:
        assert int(compared) > 0 and int(mismatched) == 0, name
        assert int(f_compared) == int(compared) and int(f_mismatched) == 0, name
        if len(name.split(",")) >= 5:
            assert int(s_compared) == int(compared) and int(s_mismatched) == 0, name
    # g g -> 5g: 112 combinations x 7245 diagrams compared; prologue area of
    # the wavefunctions of up to 4 legs
    assert int(rows[9][1]) == 112 * 7245 and int(rows[9][6]) == 16180
    # the full helicity sum: every one of the 2^n combinations, the vanishing ones included
    full = ["21,21,21,21,21,21", "2,-2,21,21,21,21,21", "21,21,21,21,21,21,21", "2,2,2,2,21,21,21"]
    r = subprocess.run([exe, "--all"] + full, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    for line, name in zip(r.stdout.splitlines(), full):
        f = line.split()
        n_ext = len(name.split(","))
        assert f[0] == name and int(f[1]) % (1 << n_ext) == 0
        assert int(f[2]) == int(f[5]) == int(f[8]) == 0 and int(f[1]) == int(f[4]) == int(f[7]), line
