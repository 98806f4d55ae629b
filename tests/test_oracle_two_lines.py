"""Independent pin of the oracle's two-quark-line processes: q Q -> q Q g
evaluated diagram by diagram with explicit colour indices (SU(3) generators
as matrices) from the textbook Feynman-gauge rules, with spinors, gamma
matrices and polarisation vectors of the tests' own (tests/physics_ref.py).
For identical quarks the amplitude with the final quarks exchanged enters
with the Fermi sign.  Checks the colour- and helicity-summed |M|^2 (averaged
1/4 * 1/9) of u d -> u d g and u u -> u u g against the oracle, and the Ward
identity of the independent evaluation itself."""
import numpy as np
import pytest

import oracle
from paper_0909_5257_gb300 import phasespace as ps
from tests import physics_ref as ref

C = ref.quark_quark_gluon_colours()
G_COL = np.einsum("dxzwva,exzwva->de", C.conj(), C)


def _helicities():
    for h in range(32):
        yield [1 if (h >> (4 - i)) & 1 else -1 for i in range(5)]


def _me2_distinct(m, g):
    tot = 0.0
    for lam in _helicities():
        L = ref.quark_quark_gluon_diagrams(m, lam, g)
        tot += float(np.real(L.conj() @ G_COL @ L))
    return tot / 36.0


def _me2_identical(m, g):
    tot = 0.0
    for lam in _helicities():
        direct = np.einsum("d,dxzwva->xzwva", ref.quark_quark_gluon_diagrams(m, lam, g), C)
        mx = m[[0, 1, 3, 2, 4]]
        lx = [lam[0], lam[1], lam[3], lam[2], lam[4]]
        exch = np.einsum("d,dxzwva->xzwva", ref.quark_quark_gluon_diagrams(mx, lx, g), C)
        exch = np.transpose(exch, (2, 1, 0, 3, 4))  # outgoing colours follow their momenta
        tot += float(np.sum(np.abs(direct - exch) ** 2))
    return tot / 36.0


def _events(n):
    return ps.generate(ps.PhaseSpaceConfig(3, rs_lo=200.0, rs_hi=2000.0, seed=ps.SEED_BASE + 41), n)


@pytest.mark.parametrize("pdg,fn", [([2, 1, 2, 1, 21], _me2_distinct), ([2, 2, 2, 2, 21], _me2_identical)])
def test_two_quark_lines_against_explicit_diagrams(pdg, fn):
    mom = _events(6)
    g = ref.g_s()
    want = oracle.OracleProcess(pdg).me2(mom)
    for m, w in zip(mom, want):
        assert abs(fn(m, g) / w - 1.0) < 1e-12


def test_explicit_diagrams_satisfy_the_ward_identity():
    """Replacing the gluon's polarisation by its momentum cancels the colour
    sum of the five diagrams (relative vertex signs of the evaluation)."""
    g = ref.g_s()
    for m in _events(3):
        for lam in _helicities():
            L = ref.quark_quark_gluon_diagrams(m, lam, g)
            W = ref.quark_quark_gluon_diagrams(m, lam, g, ward=True)
            norm = float(np.real(L.conj() @ G_COL @ L))
            if norm > 0:
                assert float(np.real(W.conj() @ G_COL @ W)) < 1e-8 * norm * np.max(m[:, 0]) ** 2
