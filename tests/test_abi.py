"""The C ABI library builds, loads and exports every symbol include/mea.h
declares; host-side generator checks that need no GPU."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mea.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mea_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_0909_5257_gb300 import mea
    lib = mea.load()
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_generator_table1_and_table5_counts():
    """Table 1 (diagrams, colours) and Table 5 (distinct colour-matrix values) of
    the product generator for all twelve processes."""
    from paper_0909_5257_gb300 import mea
    g = os.path.join(ROOT, "tests", "golden")
    t5 = {}
    for line in open(os.path.join(g, "table5_unique.txt")):
        line = line.split("#")[0].split()
        if line:
            t5[int(line[0])] = [int(x) for x in line[1:]]
    for line in open(os.path.join(g, "table1_counts.txt")):
        f = line.split("#")[0].split()
        if not f:
            continue
        pdg = [int(x) for x in f[1:-2]]
        P = mea.Process(pdg, host_only=True)
        assert P.info["n_diagrams"] == int(f[-2]), f[0]
        assert P.info["n_colour"] == int(f[-1]), f[0]
        num, den = P.colour_matrix_exact()
        m = num.shape[0]
        uniq = len(set(num[np.triu_indices(m)].tolist()) - {0})
        fam = 0 if pdg[0] == 21 else (1 if pdg[1] < 0 else 2)
        assert uniq == t5[len(pdg) - 2][fam], f[0]


@pytest.mark.parametrize("pdg", [[21] * 4, [21] * 5, [21] * 6, [2, -2, 21, 21], [2, -2, 21, 21, 21],
                                 [2, -2, 21, 21, 21, 21]])
def test_generator_colour_matrix_equals_oracle(pdg):
    """Same basis elements (gluon traces, single-line strings), independent
    algorithms: exact colour matrices must coincide element by element."""
    import oracle
    from paper_0909_5257_gb300 import mea
    P = mea.Process(pdg, host_only=True)
    O = oracle.OracleProcess(pdg)
    num, den = P.colour_matrix_exact()
    N = num / den
    # product basis: gluons -> trace starting with the last leg; one line -> string
    m = P.n_colour
    assert m == O.n_colour
    okey = {}
    for a in range(m):
        (closed, row, col, gl), = O.basis(a)
        if closed:
            r = gl.index(len(pdg) - 1)
            gl = gl[r:] + gl[:r]
        okey[tuple(gl)] = a
    import itertools
    gl_legs = [l for l in range(len(pdg)) if pdg[l] == 21]
    if pdg[0] == 21:
        words = [tuple([len(pdg) - 1] + list(w)) for w in itertools.permutations(sorted(gl_legs[:-1]))]
    else:
        words = [tuple(w) for w in itertools.permutations(sorted(gl_legs))]
    perm = [okey[w] for w in words]
    Oc = O.colour_matrix()[np.ix_(perm, perm)]
    assert np.allclose(N, Oc, rtol=1e-14, atol=1e-15)


def test_generator_helicity_counts():
    from paper_0909_5257_gb300 import mea
    want = {(21,) * 4: 6, (21,) * 5: 20, (21,) * 6: 50, (21,) * 7: 112, (2, -2, 21, 21): 4,
            (2, -2, 21, 21, 21): 12, (2, -2, 21, 21, 21, 21): 28, (2, -2) + (21,) * 5: 60,
            (2, 2, 2, 2, 21): 12, (2, 2, 2, 2, 21, 21, 21): 48}
    for pdg, h in want.items():
        assert mea.Process(list(pdg), host_only=True).info["n_hel_nonzero"] == h


def test_host_only_handle_refuses_evaluation():
    from paper_0909_5257_gb300 import mea
    P = mea.Process([21] * 4, host_only=True)
    with pytest.raises(mea.MeaError) as e:
        P.evaluate(0, 0, n_events=1)
    assert e.value.status == -2


def test_kernel_variant_out_of_range_is_an_argument_error():
    """mea_options.kernel_variant is checked before any device work."""
    from paper_0909_5257_gb300 import mea
    for v in (-1, 7):
        with pytest.raises(mea.MeaError) as e:
            mea.Process([21] * 5, kernel_variant=v)
        assert e.value.status == -1


def test_helicity_sharing_option_out_of_range_is_an_argument_error():
    """mea_options.helicity_sharing is checked before any device work."""
    from paper_0909_5257_gb300 import mea
    for v in (-1, 5):
        with pytest.raises(mea.MeaError) as e:
            mea.Process([21] * 6, helicity_sharing=v)
        assert e.value.status == -1


def test_helicity_shared_evaluation_counts():
    """Per event the helicity-shared evaluation makes each wavefunction once
    per helicity pattern of its legs: g g -> 5g 114 098 variants against
    112 x 4183 per-lane copies, 2.2x fewer FLOPs than the per-lane program
    (colour entries excluded), in a work space of 7716 32-byte variants."""
    from paper_0909_5257_gb300 import mea
    info = mea.Process([21] * 7, host_only=True).info
    per_lane = info["n_hel_nonzero"] * (info["flops_per_hel"] - 4 * info["n_colour_entries"])
    assert info["hs_variants"] == 114098 and info["hs_arena_variants"] == 7716
    assert 2.1 < per_lane / info["hs_flops_per_event"] < 2.4
    small = mea.Process([2, 2, 2, 2, 21, 21, 21], host_only=True).info
    assert 0 < small["hs_variants"] < small["n_hel_nonzero"] * small["n_ops"]
    # split evaluation: the wavefunctions of up to 4 legs in a prologue area of
    # 16 180 variants per event, the rest per lane
    assert info["hsp_area_variants"] == 16180
    assert info["hs_flops_per_event"] < info["hsp_flops_per_event"] < per_lane


def test_vertex_partials_reduce_the_flop_count():
    """The program shares vertex partials (fewer FLOPs than one vertex call
    per diagram) where diagrams share all amplitude-vertex inputs but one; the
    2 -> 2 processes have no such groups.  Counts from the op costs of
    heget.cuh: gg>ggg 12 702 -> 9 742, gg>gggg 144 232 -> 86 272 per helicity."""
    from paper_0909_5257_gb300 import mea
    for pdg, plain, part in (([21] * 5, 12702, 9742), ([21] * 6, 144232, 86272)):
        info = mea.Process(pdg, host_only=True).info
        assert info["flops_per_hel_plain"] == plain
        assert info["flops_per_hel"] == part
    info = mea.Process([21] * 4, host_only=True).info
    assert info["flops_per_hel"] == info["flops_per_hel_plain"]


def test_binding_rejects_tensors_the_kernels_would_misread():
    """The Python binding checks dtype, contiguity, device and size of torch
    arguments before handing their addresses to the library (MEA_E_ARG)."""
    torch = pytest.importorskip("torch")
    from paper_0909_5257_gb300 import mea
    P = mea.Process([21] * 5, host_only=True)
    n = 8
    cases = [
        (torch.zeros((n, 5, 4), dtype=torch.float32), torch.zeros(n, dtype=torch.float64), "float64"),
        (torch.zeros((n, 5, 4), dtype=torch.float64), torch.zeros(n, dtype=torch.float64), "CUDA"),
        (torch.zeros((n, 4, 5), dtype=torch.float64).transpose(1, 2), torch.zeros(n, dtype=torch.float64),
         "contiguous"),
    ]
    for mom, me2, word in cases:
        for call in (P.evaluate, P.evaluate_noalloc, P.autotune):
            with pytest.raises(mea.MeaError) as e:
                call(mom, me2)
            assert e.value.status == -1 and word in str(e.value)
    # mistyped outputs of the allocation-free entry point (the other arguments
    # given as raw addresses, which pass to the library unchecked; the check
    # raises before the call)
    for me2, flags, word in ((torch.zeros(n, dtype=torch.float32), None, "float64"),
                             (0, torch.zeros(n, dtype=torch.int32), "uint8")):
        with pytest.raises(mea.MeaError) as e:
            P.evaluate_noalloc(0, me2, n_events=n, flags=flags)
        assert e.value.status == -1 and word in str(e.value)
