"""Second, independent pin of the oracle's amplitudes: the Berends-Giele
recursion with colour-ordered Feynman rules (tests/physics_ref.py), for pure
gluon processes and for one quark line (u u~ -> n g).

In the trace basis with Tr(t^a t^b) = delta/2 the oracle's colour amplitude of
ordering alpha is J_alpha = g^{n-2} 2^{n/2} A(alpha) up to a phase, so
|J_alpha|^2 / (g^{2n-4} 2^n |A_BG(alpha)|^2) = 1 for every ordering and every
helicity combination, MHV or not.  The polarisation vectors on the BG side are
built in a different gauge from the oracle's.
"""
import numpy as np
import pytest

import oracle
from paper_0909_5257_gb300 import phasespace as ps
from tests import physics_ref as ref

_cache = {}


def proc(n):
    if n not in _cache:
        _cache[n] = oracle.OracleProcess([21] * n)
    return _cache[n]


def _check(n, n_events, hel_stride, max_orders=None):
    P = proc(n)
    g = ref.g_s()
    mom = ps.generate(ps.PhaseSpaceConfig(n - 2, rs_lo=300.0, rs_hi=3000.0, seed=ps.SEED_BASE + 17), n_events)
    orders = [tuple(P.basis(a)[0][3]) for a in range(P.n_colour)]
    checked = 0
    for m in mom:
        k = ref.all_outgoing(m)
        hels = list(range(0, 1 << n, hel_stride))
        Js = {hel: P.jamp(m, hel) for hel in hels}
        scale = max(np.max(np.abs(J)) ** 2 for J in Js.values())  # event scale
        for hel in hels:
            lam = ref.helicities(hel, n)
            eps = np.array([ref.polarisation(m[i], lam[i], outgoing=i >= 2) for i in range(n)])
            J = Js[hel]
            for a, order in enumerate(orders[:max_orders]):
                A = ref.bg_amplitude(k, eps, order)
                want = g ** (2 * n - 4) * 2 ** n * abs(A) ** 2
                got = abs(J[a]) ** 2
                assert abs(got - want) <= 1e-10 * want + 1e-20 * scale
                checked += 1
    assert checked > 0


@pytest.mark.parametrize("n", [4, 5])
def test_bg_all_helicities(n):
    _check(n, 2, 1)


def test_bg_six_gluons():
    _check(6, 1, 5)


@pytest.mark.slow
def test_bg_seven_gluons():
    _check(7, 1, 37, max_orders=120)


def _check_quark_line(n, n_events, hel_stride, max_orders=None):
    """u u~ -> (n-2) g: in the string basis (T^{a_s1}...T^{a_sk})_{i j} the
    oracle's colour amplitude is J_alpha = g^{n-2} 2^{(n-2)/2} A(alpha) up to a
    phase, A the colour-ordered quark-line amplitude with the generators read
    from the antiquark end: every ordering, every helicity combination."""
    pdg = [2, -2] + [21] * (n - 2)
    P = oracle.OracleProcess(pdg)
    g = ref.g_s()
    mom = ps.generate(ps.PhaseSpaceConfig(n - 2, rs_lo=300.0, rs_hi=3000.0, seed=ps.SEED_BASE + 23), n_events)
    orders = [tuple(P.basis(a)[0][3]) for a in range(P.n_colour)]
    checked = 0
    for m in mom:
        hels = list(range(0, 1 << n, hel_stride))
        Js = {hel: P.jamp(m, hel) for hel in hels}
        scale = max(np.max(np.abs(J)) ** 2 for J in Js.values())
        for hel in hels:
            lam = ref.helicities(hel, n)
            eps = {i: ref.polarisation(m[i], lam[i], outgoing=True) for i in range(2, n)}
            right = ref.u_spinor(m[0], lam[0])
            left = ref.vbar_spinor(m[1], lam[1])
            J = Js[hel]
            for a, order in enumerate(orders[:max_orders]):
                A = ref.bg_quark_line_amplitude(m, eps, order, left, right)
                want = g ** (2 * n - 4) * 2 ** (n - 2) * abs(A) ** 2
                got = abs(J[a]) ** 2
                assert abs(got - want) <= 1e-10 * want + 1e-20 * scale
                checked += 1
    assert checked > 0


@pytest.mark.parametrize("n", [4, 5, 6])
def test_bg_quark_line_all_helicities(n):
    _check_quark_line(n, 2, 1)


def test_bg_quark_line_seven_partons():
    _check_quark_line(7, 1, 7, max_orders=30)
