"""mea_evaluate_noalloc: evaluation for callers that cannot let the library
allocate device memory (applications whose device memory belongs to their
own pool allocator, latency-critical loops that cannot take cudaMalloc's
implicit device synchronisation).  Its scratch is a fixed device array inside
the library, so it is checked here against mea_evaluate on the same inputs,
for two calls in a row (the array keeps the previous call's contents):
straight-line kernels (3-jet), the table-driven kernel with its wavefunction
and colour-amplitude work space placed in the array (gg -> gggg), every event
flagged and re-evaluated in FP64 through the flagged-event list in the array,
and a process tuned by mea_autotune beforehand; plus the clean rejection of a
request larger than the array.  The file is named so that pytest collects it
last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEED = 0x09095257 + 11
# pdg, n_final, events, sqrt(s) range
CASES = [([21, 21, 21, 21, 21], 3, 3001, (200.0, 2000.0)), ([2, -2, 21, 21, 21], 3, 2049, (200.0, 2000.0)),
         ([2, 2, 2, 2, 21], 3, 777, (200.0, 2000.0)), ([21] * 6, 4, 37, (300.0, 3000.0))]


def _lib():
    from paper_0909_5257_gb300 import mea
    return mea, mea.load()


def _events(mea, nf, n, lo, hi):
    mom = torch.empty((n, nf + 2, 4), dtype=torch.float64, device="cuda")
    mea.generate_phase_space(nf, n, mom, seed=SEED, rs_lo=lo, rs_hi=hi)
    return mom


def _noalloc(lib, P, mom, prec):
    """One call through the C ABI into fresh (poisoned) output buffers."""
    n = mom.shape[0]
    out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    flags = torch.full((n,), 0xFF, dtype=torch.uint8, device="cuda")
    rc = lib.mea_evaluate_noalloc(P._h, ctypes.c_void_p(mom.data_ptr()), n, prec,
                                  ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(flags.data_ptr()), None)
    assert rc == 0, lib.mea_last_error().decode()
    torch.cuda.synchronize()
    return out, flags


@pytest.mark.parametrize("pdg,nf,n,rs", CASES)
@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_evaluate_two_calls(pdg, nf, n, rs, prec):
    mea, lib = _lib()
    P = mea.Process(pdg)
    mom = _events(mea, nf, n, *rs)
    ref = torch.empty(n, dtype=torch.float64, device="cuda")
    ref_flags = torch.empty(n, dtype=torch.uint8, device="cuda")
    P.evaluate(mom, ref, precision=prec, flags=ref_flags)
    tensor_colour = prec == 1 and len(pdg) >= 6  # mea_evaluate's colour stages run on tcgen05 here
    for call in range(2):
        out, flags = _noalloc(lib, P, mom, prec)
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a)), f"call {call}"
        rel = np.abs(a / b - 1.0)
        if tensor_colour:
            # CUDA-core colour sum against the tensor-core one: the mixed tolerance
            assert np.median(rel) <= 1e-6 and rel.max() <= 1e-4, f"call {call}: {np.median(rel)} {rel.max()}"
        else:
            assert np.array_equal(a, b), f"call {call}: max rel {rel.max():.3e}"
            assert torch.equal(flags, ref_flags), f"call {call}"


@pytest.mark.parametrize("pdg,nf,n,rs", [CASES[0], CASES[3]])
def test_noalloc_reevaluates_every_flagged_event_in_fp64(pdg, nf, n, rs):
    """With a flag threshold no event can meet (1e-30) every event of the
    mixed path is flagged, listed in the array and re-evaluated in FP64: the
    results equal the FP64 path to 1e-12 and carry the re-evaluated and
    cancellation bits, on two calls in a row."""
    mea, lib = _lib()
    P = mea.Process(pdg, flag_threshold=1e-30)
    mom = _events(mea, nf, n, *rs)
    ref = torch.empty(n, dtype=torch.float64, device="cuda")
    P.evaluate(mom, ref, precision=mea.PREC_FP64)
    for call in range(2):
        out, flags = _noalloc(lib, P, mom, mea.PREC_MIXED)
        rel = np.abs(out.cpu().numpy() / ref.cpu().numpy() - 1.0)
        assert rel.max() <= 1e-12, f"call {call}: {rel.max():.3e}"
        f = flags.cpu().numpy()
        assert np.all(f & mea.FLAG_REEVALUATED) and np.all(f & mea.FLAG_CANCEL), f"call {call}"


def test_noalloc_uses_the_tuned_configuration():
    """After mea_autotune has picked a launch configuration (possibly another
    straight-line kernel variant, i.e. another FP32 rounding order), the
    allocation-free entry point runs the same one: bitwise equal results."""
    mea, lib = _lib()
    pdg, nf, n, rs = CASES[0]
    P = mea.Process(pdg)
    mom = _events(mea, nf, 1 << 14, *rs)
    scratch = torch.empty(1 << 14, dtype=torch.float64, device="cuda")
    P.autotune(mom, scratch, precision=mea.PREC_MIXED)
    ref = torch.empty(n, dtype=torch.float64, device="cuda")
    P.evaluate(mom[:n], ref, precision=mea.PREC_MIXED)
    out, _ = _noalloc(lib, P, mom[:n].contiguous(), mea.PREC_MIXED)
    assert torch.equal(out, ref)


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
    # the binding refuses a too-small output tensor before calling the library
    with pytest.raises(mea.MeaError) as e:
        P.evaluate_noalloc(small, out[:2], n_events=4)
    assert e.value.status == -1
