"""The shared and forwarding amplitude kernels (amp_hs_kernel.cu, amp_kernel.cu) on the GPU.

On the tensor-core path (mixed precision, processes without a straight-line
kernel) the amplitude stage can run as the per-lane interpreter (one lane per
event and helicity combination), as the helicity-shared kernel (one warp per
event, every wavefunction evaluated once per helicity pattern of its own
legs) or as the split kernel (the wavefunctions of up to n_ext - 3 legs
shared that way in a prologue, the rest per lane with one transient current
in registers); the per-lane interpreter also with each op's output forwarded
to the next op in registers (mode 4).  All apply the same HELAS operations to the same inputs, so
every diagram amplitude, and with it |M|^2 and the flags, is the same bit for
bit:
checked here for the serving processes and g g -> 4g, for the non-zero and
the full helicity sums, across several chunks with a ragged tail and after
autotuning.  Parity with the oracle of the tuned default path is in
test_gpu_parity.py and test_gpu_5jet_golden.py.
"""
import numpy as np
import pytest

from paper_0909_5257_gb300 import phasespace as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# name, pdg, sqrt(s) range, events, chunk (0: automatic)
CASES = [
    ("gg>gggg", [21] * 6, (300.0, 3000.0), 1037, 0),
    ("uu~>gggg", [2, -2] + [21] * 4, (300.0, 3000.0), 1037, 300),
    ("uu>uuggg", [2, 2, 2, 2, 21, 21, 21], (500.0, 5000.0), 517, 128),
    ("uu~>ggggg", [2, -2] + [21] * 5, (500.0, 5000.0), 301, 0),
    ("gg>ggggg", [21] * 7, (500.0, 5000.0), 97, 40),
]


def _mea():
    from paper_0909_5257_gb300 import mea
    return mea


def _events(pdg, rs, n, seed):
    d = torch.empty((n, len(pdg), 4), dtype=torch.float64, device="cuda")
    _mea().generate_phase_space(len(pdg) - 2, n, d, seed=seed, rs_lo=rs[0], rs_hi=rs[1])
    return d


def _run(P, mom, hel_mode=0):
    mea = _mea()
    n = mom.shape[0]
    out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    fl = torch.full((n,), 0xFF, dtype=torch.uint8, device="cuda")
    P.evaluate(mom, out, precision=mea.PREC_MIXED, flags=fl, hel_mode=hel_mode)
    P.check_status()
    return out, fl


@pytest.mark.parametrize("name,pdg,rs,n,chunk", CASES)
def test_helicity_shared_equals_per_lane_bit_for_bit(name, pdg, rs, n, chunk):
    mea = _mea()
    mom = _events(pdg, rs, n, ps.SEED_BASE + 611)
    lane = mea.Process(pdg, helicity_sharing=1, auto_tune=False, chunk_events=chunk)
    a, fa = _run(lane, mom)
    assert torch.isfinite(a).all()
    for mode in (2, 3, 4):
        other = mea.Process(pdg, helicity_sharing=mode, auto_tune=False, chunk_events=chunk)
        b, fb = _run(other, mom)
        assert torch.equal(a, b), (name, mode, float(((a - b).abs() / a.abs()).max()))
        assert torch.equal(fa, fb), (name, mode)


@pytest.mark.parametrize("name,pdg,rs,n,chunk", CASES[:3])
def test_split_kernel_every_candidate_shape(name, pdg, rs, n, chunk):
    """Tuned split kernel (shared-memory and global prologue areas, several
    tile shapes timed): its choice equals the per-lane kernel bit for bit."""
    mea = _mea()
    mom = _events(pdg, rs, n, ps.SEED_BASE + 614)
    lane = mea.Process(pdg, helicity_sharing=1, auto_tune=False, chunk_events=chunk)
    a, _ = _run(lane, mom)
    P = mea.Process(pdg, helicity_sharing=3, auto_tune=False, chunk_events=chunk)
    scratch = torch.empty(n, dtype=torch.float64, device="cuda")
    r = P.autotune(mom, scratch, precision=mea.PREC_MIXED)
    assert r["helicity_shared"] == 2 and r["candidates"] >= 2
    b, _ = _run(P, mom)
    assert torch.equal(a, b), r


def test_helicity_shared_full_helicity_sum():
    """All 2^n combinations (the vanishing ones included): 64 helicity lanes."""
    mea = _mea()
    pdg = [21] * 6
    mom = _events(pdg, (300.0, 3000.0), 333, ps.SEED_BASE + 612)
    lane = mea.Process(pdg, helicity_sharing=1, auto_tune=False)
    a, _ = _run(lane, mom, hel_mode=mea.HEL_SUM_ALL)
    for mode in (2, 3, 4):
        shared = mea.Process(pdg, helicity_sharing=mode, auto_tune=False)
        b, _ = _run(shared, mom, hel_mode=mea.HEL_SUM_ALL)
        assert torch.equal(a, b), mode
        c, _ = _run(shared, mom)
        assert torch.allclose(b, c, rtol=1e-6, atol=0)


@pytest.mark.parametrize("pdg,rs", [([21] * 6, (300.0, 3000.0)), ([2, -2] + [21] * 5, (500.0, 5000.0))])
def test_autotune_chooses_among_both_kernels_without_changing_a_bit(pdg, rs):
    mea = _mea()
    mom = _events(pdg, rs, 2048 if len(pdg) == 6 else 512, ps.SEED_BASE + 613)
    ref = mea.Process(pdg, helicity_sharing=1, auto_tune=False)
    P = mea.Process(pdg, auto_tune=False)
    a, _ = _run(ref, mom)
    scratch = torch.empty(mom.shape[0], dtype=torch.float64, device="cuda")
    r = P.autotune(mom, scratch, precision=mea.PREC_MIXED)
    assert r["candidates"] >= 2 and r["best_ms"] > 0
    b, _ = _run(P, mom)
    assert torch.equal(a, b), r
