"""The pins catch plausible mistakes: each test builds a copy of the oracle
with one deliberate mistake planted (OQ_MUTATION in qcd_oracle.cpp) and checks
that the battery of pins -- closed forms, Parke-Taylor (gluons and one quark line),
Ward identities, Bose symmetry, the collinear limit of u u -> u u g g --
rejects it, while the unmutated copy passes the same battery.

Mutations: 1 a dropped term of the ggg vertex, 2 a flipped sign of one gggg
colour structure, 3 the metric dropped from the gluon propagator (index slip),
4 the wrong momentum direction in the antiquark propagator, 5 the colour
average of two gluons (1/64) applied to every initial state, 6 a flipped sign of the qqg vertex
in the gluon current, 7 the crossing sign of outgoing legs forgotten in the
propagator momenta.
"""
import os

import numpy as np
import pytest

import oracle
from paper_0909_5257_gb300 import phasespace as ps
from tests import physics_ref as ref
from tests import test_oracle_collinear as coll


def _events(n_final, n, lo=300.0, hi=3000.0):
    return ps.generate(ps.PhaseSpaceConfig(n_final, rs_lo=lo, rs_hi=hi, seed=ps.SEED_BASE + 17), n)


def _battery(lib):
    """Names of the pins this oracle library fails."""
    failed = []
    mom2 = _events(2, 16)
    for name, pdg, fn in (("gg>gg closed form", [21] * 4, ref.me2_gg_gg),
                          ("uu~>gg closed form", [2, -2, 21, 21], ref.me2_uubar_gg),
                          ("uu>uu closed form", [2, 2, 2, 2], ref.me2_uu_uu)):
        got = oracle.OracleProcess(pdg, lib=lib).me2(mom2)
        if not np.all(np.abs(got / fn(mom2) - 1.0) < 1e-12):
            failed.append(name)
    mom3 = _events(3, 4)
    got = oracle.OracleProcess([21] * 5, lib=lib).me2(mom3)
    want = np.array([ref.gluon_me2_leading_colour_exact(m) for m in mom3])
    if not np.all(np.abs(got / want - 1.0) < 1e-11):
        failed.append("Parke-Taylor gg>ggg")
    for pdg in ([21] * 5, [2, -2, 21, 21, 21]):
        P = oracle.OracleProcess(pdg, lib=lib)
        N = P.colour_matrix()
        n = len(pdg)
        m = _events(n - 2, 1)[0]
        hels = list(range(0, 1 << n, 5))
        norm = max(float(np.sum(np.abs(P.jamp(m, h)) ** 2)) for h in hels)
        bad = False
        for leg in [i for i in range(n) if pdg[i] == 21]:
            for h in hels:
                W = P.jamp(m, h, ward_leg=leg)
                if not np.sum(np.abs(W) ** 2) < 1e-20 * norm:
                    bad = True
        if bad:
            failed.append(f"Ward identity {pdg}")
    P = oracle.OracleProcess([2, -2, 21, 21, 21], lib=lib)
    g = ref.g_s()
    orders = [P.basis(a)[0][3] for a in range(P.n_colour)]
    k = ref.all_outgoing(mom3[0])
    bad = False
    for hel in range(32):
        ho = ref.outgoing_helicities(hel, 5)
        neg = [i for i in range(5) if ho[i] < 0]
        if len(neg) != 2 or ho[0] == ho[1]:
            continue
        qm = 0 if ho[0] < 0 else 1
        gm = [i for i in neg if i >= 2][0]
        J = P.jamp(mom3[0], hel)
        for a, gl in enumerate(orders):
            a2 = ref.quark_line_mhv_sq(k, [0, 1] + gl, qm, 1 - qm, gm)
            if not abs(abs(J[a]) ** 2 / (g ** 6 * 8 * a2) - 1.0) < 1e-10:
                bad = True
    if bad:
        failed.append("quark-line MHV uu~>ggg")
    P = oracle.OracleProcess([21] * 5, lib=lib)
    base = P.me2(mom3)
    if not np.allclose(P.me2(mom3[:, [0, 1, 4, 2, 3]]), base, rtol=1e-12, atol=0):
        failed.append("Bose symmetry gg>ggg")
    small, big, leg, kernel, n_phi, z = coll.CASES[0]
    ev = coll._events(small, 2, ps.SEED_BASE + 63)
    r = coll._ratio(small, big, ev, leg, z, 1e-5, kernel, n_phi, lib=lib)
    if not np.all(np.abs(r - 1.0) < 5e-4):
        failed.append("collinear limit uu>uugg")
    return failed


@pytest.fixture(scope="module")
def variants(tmp_path_factory):
    d = tmp_path_factory.mktemp("oracle_variants")
    cache = {}

    def get(k):
        if k not in cache:
            path = os.path.join(str(d), f"liboracle_m{k}.so")
            cache[k] = oracle.load_variant(oracle.build_variant(path, k))
        return cache[k]
    return get


def test_unmutated_copy_passes_the_battery(variants):
    assert _battery(variants(0)) == []


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7])
def test_planted_mistake_is_caught(variants, k):
    failed = _battery(variants(k))
    assert failed, f"mutation {k} passed every pin"
