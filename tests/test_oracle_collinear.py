"""Oracle pin for the two-quark-line processes with several gluons: the
collinear factorisation of tree-level QCD amplitudes.

When an outgoing parton P splits into two collinear massless partons with
light-cone momentum fractions z and 1 - z and invariant s = (p1 + p2)^2 -> 0,
the colour- and helicity-summed squared matrix element factorises,
    |M_{n+1}|^2  ->  (2 g^2 / s) P(z) |M_n|^2 ,
with the unregularised Altarelli-Parisi kernels
    q -> q(z) g(1-z):  P_qq(z) = C_F (1 + z^2) / (1 - z),          C_F = 4/3,
    g -> g(z) g(1-z):  <P_gg(z)> = 2 C_A [z/(1-z) + (1-z)/z + z(1-z)], C_A = 3,
the latter after averaging the gluon's azimuthal (spin) correlation over two
azimuths 90 degrees apart.  The initial-state averages (1/4, 1/(n_a n_b))
are the same on both sides, and no identical-particle factor enters |M|^2.

This ties u u -> u u + 3g (786 diagrams, 240 colours) to u u -> u u + 2g and
that to u u -> u u g, which is pinned diagram by diagram with explicit colour
indices (test_oracle_two_lines.py).  The limit is approached linearly in the
relative transverse momentum, so the ratio is checked at two values of it
(1e-4 and 1e-5 of the parton's energy): the deviation must shrink about
tenfold between them and be below 5e-4 at the smaller.  A dropped diagram,
a wrong relative sign between the quark and gluon vertices, or a wrong
colour factor moves the ratio by O(1).
"""
import numpy as np
import pytest

import oracle
from paper_0909_5257_gb300 import phasespace as ps

G2 = 4.0 * np.pi * 0.118
CF, CA = 4.0 / 3.0, 3.0


def _mdot(a, b):
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]


def _boost_to_rest(p, Q):
    """Lorentz boost of the 4-vector p into the rest frame of Q."""
    M = np.sqrt(_mdot(Q, Q))
    b = -Q[1:] / Q[0]
    b2 = b @ b
    gam = Q[0] / M
    bp = b @ p[1:]
    e = gam * (p[0] + bp)
    sp = p[1:] + ((gam - 1.0) * bp / b2 + gam * p[0]) * b
    return np.concatenate([[e], sp])


def split(event, leg, z, rel_kt, phi):
    """The (n+1)-parton event in which outgoing parton `leg` of `event` splits
    into two massless partons with light-cone fractions z (kept at `leg`) and
    1 - z (appended last), relative transverse momentum rel_kt * E_leg at
    azimuth phi; the final state is then boosted to its rest frame and
    rescaled so that momentum is conserved exactly with the same incoming
    pair.  Returns the event and s = (p_leg + p_new)^2."""
    P = event[leg]
    E = P[0]
    u = P[1:] / E
    n = np.concatenate([[1.0], -u])  # light-like, n.P = 2E
    a = np.cross(u, [0.0, 0.0, 1.0] if abs(u[2]) < 0.9 else [1.0, 0.0, 0.0])
    a /= np.linalg.norm(a)
    b = np.cross(u, a)
    e = np.cos(phi) * a + np.sin(phi) * b
    kt = rel_kt * E
    kperp = np.concatenate([[0.0], kt * e])
    pn = 2.0 * E
    p1 = z * P + kperp + kt ** 2 / (2.0 * z * pn) * n
    p2 = (1.0 - z) * P - kperp + kt ** 2 / (2.0 * (1.0 - z) * pn) * n
    fin = [event[i] for i in range(2, event.shape[0])]
    fin[leg - 2] = p1
    fin.append(p2)
    Q = np.sum(fin, axis=0)
    rs = event[0, 0] + event[1, 0]
    M = np.sqrt(_mdot(Q, Q))
    fin = [_boost_to_rest(p, Q) * (rs / M) for p in fin]
    for p in fin:  # exactly massless after the floating-point boost
        p[0] = np.linalg.norm(p[1:])
    out = np.array([event[0], event[1]] + fin)
    s = _mdot(out[leg] + out[-1], out[leg] + out[-1])
    return out, s


def _ratio(pdg_small, pdg_big, events, leg, z, rel_kt, kernel, n_phi, lib=None):
    small = oracle.OracleProcess(pdg_small, lib=lib).me2(events)
    rows, splits = [], []
    for ev in events:
        for k in range(n_phi):
            big_ev, s = split(ev, leg, z, rel_kt, 0.3 + k * np.pi / 2.0)
            rows.append(big_ev)
            splits.append(s)
    big = oracle.OracleProcess(pdg_big, lib=lib).me2(np.array(rows)).reshape(len(events), n_phi)
    s = np.array(splits).reshape(len(events), n_phi)
    lim = (2.0 * G2 / s) * kernel(z) * small[:, None]
    return (big / lim).mean(axis=1)


def _events(pdg, n, seed):
    return ps.generate(ps.PhaseSpaceConfig(len(pdg) - 2, rs_lo=500.0, rs_hi=5000.0, seed=seed), n)


def p_qq(z):
    return CF * (1.0 + z * z) / (1.0 - z)


def p_gg(z):
    return 2.0 * CA * (z / (1.0 - z) + (1.0 - z) / z + z * (1.0 - z))


CASES = [
    # (reduced process, split process, leg that splits, kernel, azimuths, z)
    ([2, 2, 2, 2, 21], [2, 2, 2, 2, 21, 21], 2, p_qq, 1, 0.37),
    ([2, 2, 2, 2, 21, 21], [2, 2, 2, 2, 21, 21, 21], 2, p_qq, 1, 0.37),
    ([2, 2, 2, 2, 21, 21], [2, 2, 2, 2, 21, 21, 21], 3, p_qq, 1, 0.62),
    ([2, 2, 2, 2, 21, 21], [2, 2, 2, 2, 21, 21, 21], 5, p_gg, 2, 0.41),
]


@pytest.mark.parametrize("small,big,leg,kernel,n_phi,z", CASES)
def test_collinear_limit_factorises(small, big, leg, kernel, n_phi, z):
    events = _events(small, 3, ps.SEED_BASE + 61 + leg)
    r1 = _ratio(small, big, events, leg, z, 1e-4, kernel, n_phi)
    r2 = _ratio(small, big, events, leg, z, 1e-5, kernel, n_phi)
    d1, d2 = np.abs(r1 - 1.0), np.abs(r2 - 1.0)
    assert np.all(d2 < 5e-4), (r1, r2)
    assert np.all((d2 < 0.2 * d1) | (d2 < 2e-5)), (r1, r2)


def test_split_event_is_physical():
    ev = _events([2, 2, 2, 2, 21, 21], 1, ps.SEED_BASE + 5)[0]
    big, s = split(ev, 2, 0.37, 1e-3, 0.3)
    tot = big[0] + big[1] - big[2:].sum(axis=0)
    rs = ev[0, 0] + ev[1, 0]
    assert np.abs(tot).max() < 1e-12 * rs
    for p in big:
        assert abs(_mdot(p, p)) < 1e-9 * rs ** 2
    assert s > 0 and s < 1e-5 * rs ** 2
