"""mea_evaluate_noalloc: evaluation for callers that cannot let the library
allocate device memory (applications whose device memory belongs to their
own pool allocator, latency-critical loops that cannot take cudaMalloc's
implicit device synchronisation).  Its scratch is a fixed device array inside
the library, so it is checked here against mea_evaluate on the same inputs,
for two calls in a row (the array keeps the previous call's contents), and
for the clean rejection of a request larger than that array.  The file is
named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [([21, 21, 21, 21, 21], 3, 3001), ([2, -2, 21, 21, 21], 3, 2049), ([2, 2, 2, 2, 21], 3, 777)]


def _lib():
    from paper_0909_5257_gb300 import mea
    return mea, mea.load()


@pytest.mark.parametrize("pdg,nf,n", CASES)
@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_evaluate_two_calls(pdg, nf, n, prec):
    mea, lib = _lib()
    P = mea.Process(pdg)
    mom = torch.empty((n, nf + 2, 4), dtype=torch.float64, device="cuda")
    mea.generate_phase_space(nf, n, mom, seed=0x09095257 + 11)
    ref = torch.empty(n, dtype=torch.float64, device="cuda")
    ref_flags = torch.empty(n, dtype=torch.uint8, device="cuda")
    P.evaluate(mom, ref, precision=prec, flags=ref_flags)
    for call in range(2):
        out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        flags = torch.full((n,), 0xFF, dtype=torch.uint8, device="cuda")
        rc = lib.mea_evaluate_noalloc(P._h, ctypes.c_void_p(mom.data_ptr()), n, prec,
                                      ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(flags.data_ptr()), None)
        assert rc == 0, lib.mea_last_error().decode()
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a)), f"call {call}"
        assert np.max(np.abs(a / b - 1.0)) <= 1e-12, f"call {call}"
        assert torch.equal(flags, ref_flags), f"call {call}"


def test_noalloc_rejects_requests_beyond_its_array():
    mea, lib = _lib()
    P = mea.Process([21, 21, 21, 21, 21])
    small = torch.zeros((4, 5, 4), dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    n_too_big = 1 << 24  # the flagged-event list alone needs 64 MiB
    rc = lib.mea_evaluate_noalloc(P._h, ctypes.c_void_p(small.data_ptr()), n_too_big, 1,
                                  ctypes.c_void_p(out.data_ptr()), None, None)
    assert rc == -1
    assert b"bytes of scratch" in lib.mea_last_error()
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0
