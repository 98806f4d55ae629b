"""GPU parity at the serving workload's 2 -> 5 subprocesses, every event of a
1024-event sample against stored oracle values.

tests/golden/golden_5jet_*.txt hold |M|^2 of the FP64 oracle for events
0..1023 of the seeded host input generator (sqrt(s) log-uniform in
[500 GeV, 5 TeV], jet cuts), written by tests/golden/make_5jet_golden.py,
which calls nothing but the oracle and the generator.  The same host-generated
momenta are evaluated here through the C ABI:
  * FP64 path: every event within 1e-12 relative;
  * mixed path (FP32 amplitudes, tensor-core colour-amplitude and colour-sum
    stages, flagged events re-evaluated in FP64): median <= 1e-6 and max
    <= 1e-4 relative, re-evaluated events within 1e-12;
both with the automatic chunking (one chunk here) and with chunks of 300
events (three full chunks and a ragged one of 124), so that the multi-CTA,
multi-chunk and ragged-tail paths of the tensor-core stages meet the oracle.
"""
import os
import sys

import numpy as np
import pytest

from paper_0909_5257_gb300 import phasespace as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_5jet_golden as golden  # noqa: E402

_cache = {}


def _data(name, pdg, nf):
    if name not in _cache:
        idx, val = golden.read(name)
        assert idx == list(range(len(idx)))
        mom = ps.generate(golden.config(nf), len(idx))
        _cache[name] = (mom, np.array(val))
    return _cache[name]


def _mea():
    from paper_0909_5257_gb300 import mea
    return mea


@pytest.mark.parametrize("name,pdg,nf", golden.SUBPROCESSES)
@pytest.mark.parametrize("chunk", [0, 300])
def test_5jet_every_event_against_stored_oracle_values(name, pdg, nf, chunk):
    mea = _mea()
    mom, ref = _data(name, pdg, nf)
    n = mom.shape[0]
    P = mea.Process(pdg, chunk_events=chunk, auto_tune=False)
    d_mom = torch.from_numpy(mom).cuda()
    out = {}
    for prec in (mea.PREC_FP64, mea.PREC_MIXED):
        o = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        f = torch.full((n,), 0xFF, dtype=torch.uint8, device="cuda")
        P.evaluate(d_mom, o, precision=prec, flags=f)
        P.check_status()
        out[prec] = (o.cpu().numpy(), f.cpu().numpy())
    g64, f64 = out[mea.PREC_FP64]
    rel64 = np.abs(g64 / ref - 1.0)
    assert np.all(np.isfinite(g64))
    assert rel64.max() <= 1e-12, f"{name}: FP64 max rel {rel64.max():.3e} at {int(rel64.argmax())}"
    assert not np.any(f64 & 0x1E)
    g32, f32 = out[mea.PREC_MIXED]
    rel32 = np.abs(g32 / ref - 1.0)
    assert np.all(np.isfinite(g32))
    assert np.median(rel32) <= 1e-6, f"{name}: mixed median {np.median(rel32):.3e}"
    assert rel32.max() <= 1e-4, f"{name}: mixed max {rel32.max():.3e}"
    re = (f32 & mea.FLAG_REEVALUATED) != 0
    if re.any():
        assert rel32[re].max() <= 1e-12
