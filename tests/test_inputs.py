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


def _uncut(n_final, rs=1000.0):
    """The generator with every cut open (pT > 0, |eta| < 1e9, no Delta R):
    RAMBO's flat massless n-body phase space at fixed sqrt(s)."""
    return ps.PhaseSpaceConfig(n_final, rs_lo=rs, rs_hi=rs, pt_min=0.0, eta_max=1e9, dr_min=0.0,
                               seed=ps.SEED_BASE + 71)


@pytest.mark.parametrize("n_final", [3, 4, 5])
def test_rambo_is_flat_single_parton_energy(n_final):
    """Flatness of Eq. (phase-space) for n >= 3, pinned by a closed form: in
    flat massless n-body phase space the energy fraction x = 2E/sqrt(s) of
    any one parton has the density (n-1)(n-2) x (1-x)^(n-3) on [0, 1]
    (integrate the other n-1 momenta out: Phi_{n-1} of the recoil system of
    squared mass s(1-x) grows as (1-x)^(n-3), times x from d^3p/E), i.e.
    Beta(2, n-2).  Kolmogorov-Smirnov on 60 000 events per parton; a RAMBO
    map with a wrong Jacobian or conformal boost fails it by orders of
    magnitude."""
    stats = pytest.importorskip("scipy.stats")
    rs = 1000.0
    mom = ps.generate(_uncut(n_final, rs), 60000)
    x = 2.0 * mom[:, 2:, 0] / rs
    for i in range(n_final):
        p = stats.kstest(x[:, i], stats.beta(2, n_final - 2).cdf).pvalue
        assert p > 1e-4, (i, p)
    # the first and second moments of Beta(2, n-2)
    assert abs(x.mean() - 2.0 / n_final) < 3e-3
    assert abs((x ** 2).mean() - 6.0 / (n_final * (n_final + 1))) < 3e-3


def test_rambo_three_body_dalitz_plot_is_uniform():
    """n = 3: the Dalitz variables (x1, x2) are uniform over the triangle
    x1 + x2 > 1, x1 < 1, x2 < 1 (constant matrix element of flat phase
    space); chi-square over a 10 x 10 grid of the unit square restricted to
    the triangle (cells cut by the diagonal carry their area fraction)."""
    stats = pytest.importorskip("scipy.stats")
    rs = 1000.0
    n = 200000
    mom = ps.generate(_uncut(3, rs), n)
    x1 = 2.0 * mom[:, 2, 0] / rs
    x2 = 2.0 * mom[:, 3, 0] / rs
    assert np.all(x1 + x2 >= 1.0 - 1e-12)
    k = 10
    h, _, _ = np.histogram2d(x1, x2, bins=k, range=[[0, 1], [0, 1]])
    # area of each cell inside the triangle (exact: the diagonal crosses cells (i, k-1-i))
    area = np.zeros((k, k))
    for i in range(k):
        for j in range(k):
            if i + j >= k:
                area[i, j] = 1.0
            elif i + j == k - 1:
                area[i, j] = 0.5
    expect = n * area / area.sum()
    m = expect > 0
    chi2 = float((((h - expect) ** 2)[m] / expect[m]).sum())
    dof = int(m.sum()) - 1
    assert stats.chi2.sf(chi2, dof) > 1e-4, (chi2, dof)
    assert h[~m].sum() == 0


@pytest.mark.parametrize("n_final", [3, 5])
def test_rambo_is_isotropic(n_final):
    """Flat phase space has no preferred direction: cos(theta) of every
    parton is uniform on [-1, 1] and phi uniform on (-pi, pi]."""
    stats = pytest.importorskip("scipy.stats")
    mom = ps.generate(_uncut(n_final), 40000)
    fin = mom[:, 2:]
    cth = fin[..., 3] / np.linalg.norm(fin[..., 1:], axis=-1)
    phi = np.arctan2(fin[..., 2], fin[..., 1])
    for i in range(n_final):
        assert stats.kstest(cth[:, i], stats.uniform(-1, 2).cdf).pvalue > 1e-4
        assert stats.kstest(phi[:, i], stats.uniform(-np.pi, 2 * np.pi).cdf).pvalue > 1e-4
