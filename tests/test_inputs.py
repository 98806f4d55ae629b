"""The seeded synthetic input generator (Philox4x32-10 + RAMBO + jet cuts)."""
import os

import numpy as np
import pytest

from paper_0909_5257_gb300 import phasespace as ps
from tests import physics_ref as ref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        vals = [int(x, 16) for x in r]
        assert ps.philox4x32_10(vals[0:4], vals[4:6]) == vals[6:10]


@pytest.mark.parametrize("n_final", [2, 3, 4, 5])
def test_rambo_events_physical(n_final):
    cfg = ps.PhaseSpaceConfig(n_final, rs_lo=300.0, rs_hi=3000.0)
    mom, att = ps.generate(cfg, 4000, return_attempts=True)
    assert (att >= 0).all()
    rs = mom[:, 0, 0] + mom[:, 1, 0]
    assert (rs >= 300.0 * (1 - 1e-12)).all() and (rs <= 3000.0 * (1 + 1e-12)).all()
    tot = mom[:, 0] + mom[:, 1] - mom[:, 2:].sum(1)
    assert np.abs(tot).max() < 1e-10 * rs.max()
    m2 = ref.mdot(mom[:, 2:], mom[:, 2:])
    assert np.abs(m2).max() < 1e-9 * rs.max() ** 2
    fin = mom[:, 2:]
    pt = np.hypot(fin[..., 1], fin[..., 2])
    eta = np.arcsinh(fin[..., 3] / pt)
    phi = np.arctan2(fin[..., 2], fin[..., 1])
    assert (pt > 20.0).all() and (np.abs(eta) < 2.5).all()
    for i in range(n_final):
        for j in range(i + 1, n_final):
            dphi = np.angle(np.exp(1j * (phi[:, i] - phi[:, j])))
            assert (np.hypot(eta[:, i] - eta[:, j], dphi) > 0.4).all()


def test_generator_is_deterministic_and_sliceable():
    cfg = ps.PhaseSpaceConfig(4)
    a = ps.generate(cfg, 100)
    b = ps.generate(cfg, 60, first_event=40)
    assert np.array_equal(a[40:], b)
    c = ps.generate(ps.PhaseSpaceConfig(4, seed=cfg.seed + 1), 100)
    assert not np.array_equal(a, c)


def test_sqrt_s_log_uniform():
    cfg = ps.PhaseSpaceConfig(2, rs_lo=200.0, rs_hi=2000.0)
    mom, att = ps.generate(cfg, 20000, return_attempts=True)
    # events accepted at the first attempt follow the log-uniform draw exactly
    u = np.log((mom[att == 0, 0, 0] * 2) / 200.0) / np.log(10.0)
    hist, _ = np.histogram(u, bins=10, range=(0, 1))
    assert hist.min() > 0.85 * hist.mean()


@pytest.mark.parametrize("n_final", [3, 4])
def test_relative_pt_cut(n_final):
    """The paper's Eq. (cuts-ptjj): with ptij_min every accepted event has
    min(pT_i, pT_j) Delta R_ij > ptij_min for every pair; events whose first
    draw already passes both cut sets are the same draw with and without it;
    the cut removes points (more redraws)."""
    base = ps.PhaseSpaceConfig(n_final, rs_lo=100.0, rs_hi=1000.0, dr_min=0.0)
    cut = ps.PhaseSpaceConfig(n_final, rs_lo=100.0, rs_hi=1000.0, dr_min=0.0, ptij_min=20.0)
    a, att_a = ps.generate(base, 4000, return_attempts=True)
    b, att_b = ps.generate(cut, 4000, return_attempts=True)
    assert (att_b >= 0).all()
    fin = b[:, 2:]
    pt = np.hypot(fin[..., 1], fin[..., 2])
    eta = np.arcsinh(fin[..., 3] / pt)
    phi = np.arctan2(fin[..., 2], fin[..., 1])
    for i in range(n_final):
        for j in range(i + 1, n_final):
            dphi = np.angle(np.exp(1j * (phi[:, i] - phi[:, j])))
            ptij = np.minimum(pt[:, i], pt[:, j]) * np.hypot(eta[:, i] - eta[:, j], dphi)
            assert (ptij > 20.0).all()
    both0 = (att_a == 0) & (att_b == 0)
    assert both0.any() and np.array_equal(a[both0], b[both0])
    assert att_b.sum() > att_a.sum()
    # ptij_min <= 0 is no cut: the stream equals the default one
    off = ps.generate(ps.PhaseSpaceConfig(n_final, rs_lo=100.0, rs_hi=1000.0, dr_min=0.0, ptij_min=0.0), 4000)
    assert np.array_equal(off, a)
