"""Partonic cross section at fixed sqrt(s_hat): the estimator (flux, phase-space
volume, symmetry factor, acceptance from the redraw count, units) pinned to
an independent integral of the 2 -> 2 closed forms over the cut region, and
the GPU entry point mea_partonic_cross_section checked against the same
estimator built from the oracle on the identical generator events.

sigma_hat = 1/(2 s) * S * integral_cuts dPhi_n |M|^2; for two massless partons
dPhi_2 = dcos(theta) dphi / (32 pi^2), and the cuts pT > pt_min, |eta| < eta_max
(the two partons are back to back, Delta R = pi) become
|cos(theta)| < min(tanh(eta_max), sqrt(1 - (2 pt_min / sqrt(s))^2)).
"""
import math

import numpy as np
import pytest

import oracle
from paper_0909_5257_gb300 import phasespace as ps
from tests import physics_ref as ref

GEV2_PB = 0.3893794e9
SEED = ps.SEED_BASE + 515


def _phi(nf, s):
    return (2 * math.pi) ** (4 - 3 * nf) * (math.pi / 2) ** (nf - 1) * s ** (nf - 2) / (
        math.factorial(nf - 1) * math.factorial(nf - 2))


def _symmetry(pdg):
    out = 1.0
    for p in set(pdg[2:]):
        out /= math.factorial(pdg[2:].count(p))
    return out


def closed_form_sigma(fn, pdg, rs, pt_min=20.0, eta_max=2.5):
    """Gauss-Legendre integral of a 2 -> 2 closed form over the cut region (pb)."""
    s = rs * rs
    cmax = min(math.tanh(eta_max), math.sqrt(1.0 - (2.0 * pt_min / rs) ** 2))
    x, w = np.polynomial.legendre.leggauss(400)
    c = cmax * x
    sn = np.sqrt(1.0 - c * c)
    e = rs / 2
    mom = np.zeros((len(c), 4, 4))
    mom[:, 0] = [e, 0, 0, e]
    mom[:, 1] = [e, 0, 0, -e]
    mom[:, 2, 0] = e
    mom[:, 2, 1] = e * sn
    mom[:, 2, 3] = e * c
    mom[:, 3, 0] = e
    mom[:, 3, 1] = -e * sn
    mom[:, 3, 3] = -e * c
    integral = cmax * np.sum(w * fn(mom))  # integral over cos(theta); phi gives 2 pi
    return _symmetry(pdg) / (2 * s) * integral * 2 * math.pi / (32 * math.pi ** 2) * GEV2_PB


def oracle_sigma(pdg, rs, n, first=0, pt_min=20.0, eta_max=2.5, dr_min=0.4, ptij_min=0.0):
    """The estimator on the host generator's events with the oracle's |M|^2."""
    nf = len(pdg) - 2
    cfg = ps.PhaseSpaceConfig(nf, rs_lo=rs, rs_hi=rs, seed=SEED, pt_min=pt_min, eta_max=eta_max, dr_min=dr_min,
                              ptij_min=ptij_min)
    mom, att = ps.generate(cfg, n, first_event=first, return_attempts=True)
    me2 = oracle.OracleProcess(pdg).me2(mom)
    ok = att >= 0
    f = np.where(ok, me2, 0.0)
    drawn = np.sum(np.where(ok, att + 1, 4096))
    pre = _symmetry(pdg) * _phi(nf, rs * rs) / (2 * rs * rs) * GEV2_PB
    mean = f.sum() / drawn
    var = max(0.0, (f * f).sum() / drawn - mean * mean)
    return pre * mean, pre * math.sqrt(var / drawn), int(ok.sum()), int(drawn)


def test_phase_space_volume_closed_forms():
    s = 1.7e5
    assert abs(_phi(2, s) * 8 * math.pi - 1.0) < 1e-14
    assert abs(_phi(3, s) * 256 * math.pi ** 3 / s - 1.0) < 1e-14


@pytest.mark.parametrize("pdg,fn", [([21] * 4, ref.me2_gg_gg), ([2, -2, 21, 21], ref.me2_uubar_gg)])
def test_estimator_matches_closed_form_integral(pdg, fn):
    rs = 500.0
    want = closed_form_sigma(fn, pdg, rs)
    got, err, acc, drawn = oracle_sigma(pdg, rs, 200000)
    assert acc == 200000 and drawn > acc
    assert abs(got - want) < 4 * err, (got, want, err)
    assert err < 0.015 * want


@pytest.mark.gpu
@pytest.mark.parametrize("pdg,n", [([21] * 4, 1 << 15), ([2, -2, 21, 21], 1 << 15), ([21] * 5, 1 << 12)])
def test_gpu_cross_section_equals_oracle_estimator(pdg, n):
    torch = pytest.importorskip("torch")  # noqa: F841
    from paper_0909_5257_gb300 import mea
    rs = 500.0
    P = mea.Process(pdg)
    r = P.partonic_cross_section(rs, n, seed=SEED, precision=mea.PREC_FP64)
    want, err, acc, drawn = oracle_sigma(pdg, rs, n)
    assert r["n_accepted"] == acc and r["n_drawn"] == drawn
    assert abs(r["phase_space"] / _phi(len(pdg) - 2, rs * rs) - 1.0) < 1e-14
    assert r["symmetry"] == _symmetry(pdg)
    assert abs(r["sigma_pb"] / want - 1.0) < 1e-10
    assert abs(r["error_pb"] / err - 1.0) < 1e-6
    rm = P.partonic_cross_section(rs, n, seed=SEED, precision=mea.PREC_MIXED)
    assert abs(rm["sigma_pb"] / want - 1.0) < 1e-5


@pytest.mark.gpu
def test_gpu_cross_section_converges_to_closed_form():
    from paper_0909_5257_gb300 import mea
    rs = 800.0
    P = mea.Process([21] * 4)
    r = P.partonic_cross_section(rs, 1 << 21, seed=SEED, precision=mea.PREC_MIXED)
    want = closed_form_sigma(ref.me2_gg_gg, [21] * 4, rs)
    assert abs(r["sigma_pb"] - want) < 5 * r["error_pb"]
    assert r["error_pb"] < 5e-3 * want


@pytest.mark.gpu
def test_gpu_cross_section_with_the_papers_relative_pt_cut():
    """Eq. (cuts) as printed: pT > 20 GeV, |eta| < 2.5 and the relative
    transverse momentum min(pT_i, pT_j) Delta R_ij > 20 GeV (no Delta R cut)."""
    from paper_0909_5257_gb300 import mea
    pdg, rs, n = [21] * 5, 500.0, 1 << 12
    P = mea.Process(pdg)
    r = P.partonic_cross_section(rs, n, seed=SEED, precision=mea.PREC_FP64, dr_min=0.0, ptij_min=20.0)
    want, err, acc, drawn = oracle_sigma(pdg, rs, n, dr_min=0.0, ptij_min=20.0)
    assert r["n_accepted"] == acc and r["n_drawn"] == drawn
    assert abs(r["sigma_pb"] / want - 1.0) < 1e-10
    loose = P.partonic_cross_section(rs, n, seed=SEED, precision=mea.PREC_FP64, dr_min=0.0)
    assert loose["n_drawn"] < r["n_drawn"]  # the cut removes points
