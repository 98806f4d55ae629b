"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

FP64 path: every event within 1e-12 relative (the bar stated for the FP64
path).  Mixed path (FP32 amplitudes, compensated colour amplitudes, flagged
events re-evaluated in FP64): median relative error <= 1e-6 and maximum
<= 1e-4.  Event counts span several CTA tiles and end in a ragged tail.
"""
import numpy as np
import pytest

import oracle
from paper_0909_5257_gb300 import phasespace as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# name, pdg, sqrt(s) range, events (several tiles + ragged tail; oracle-affordable)
CASES = [
    ("gg>gg", [21] * 4, (200.0, 2000.0), 4099),
    ("uu~>gg", [2, -2, 21, 21], (200.0, 2000.0), 4099),
    ("uu>uu", [2, 2, 2, 2], (200.0, 2000.0), 2051),
    ("gg>ggg", [21] * 5, (200.0, 2000.0), 1037),
    ("uu~>ggg", [2, -2, 21, 21, 21], (200.0, 2000.0), 1037),
    ("uu>uug", [2, 2, 2, 2, 21], (200.0, 2000.0), 1037),
    ("gg>gggg", [21] * 6, (300.0, 3000.0), 131),
    ("uu~>gggg", [2, -2] + [21] * 4, (300.0, 3000.0), 203),
    ("uu>uugg", [2, 2, 2, 2, 21, 21], (300.0, 3000.0), 257),
    ("uu>uuggg", [2, 2, 2, 2, 21, 21, 21], (500.0, 5000.0), 37),
    ("uu~>ggggg", [2, -2] + [21] * 5, (500.0, 5000.0), 23),
    ("gg>ggggg", [21] * 7, (500.0, 5000.0), 5),
    # crossings and other flavours through the same generator (no emitted
    # kernels: these run the interpreter / tensor-core path)
    ("ug>ug", [2, 21, 2, 21], (200.0, 2000.0), 2051),
    ("gu>ugg", [21, 2, 2, 21, 21], (200.0, 2000.0), 1037),
    ("ud>udg", [2, 1, 2, 1, 21], (200.0, 2000.0), 1037),
    ("uu~>dd~g", [2, -2, 1, -1, 21], (200.0, 2000.0), 1037),
    ("uu~>uu~g", [2, -2, 2, -2, 21], (200.0, 2000.0), 1037),
    ("d~d~>d~d~g", [-1, -1, -1, -1, 21], (200.0, 2000.0), 1037),
]

_ref_cache = {}
_proc_cache = {}


def _mea():
    from paper_0909_5257_gb300 import mea
    return mea


def _case(name):
    for c in CASES:
        if c[0] == name:
            return c
    raise KeyError(name)


def _data(name):
    if name not in _ref_cache:
        _, pdg, (lo, hi), n = _case(name)
        mom = ps.generate(ps.PhaseSpaceConfig(len(pdg) - 2, rs_lo=lo, rs_hi=hi,
                                              seed=ps.SEED_BASE + 101), n)
        ref = oracle.OracleProcess(pdg).me2(mom)
        _ref_cache[name] = (mom, ref)
    return _ref_cache[name]


def _proc(pdg, **kw):
    key = (tuple(pdg), tuple(sorted(kw.items())))
    if key not in _proc_cache:
        _proc_cache[key] = _mea().Process(pdg, **kw)
    return _proc_cache[key]


def _run(pdg, mom, precision, hel_mode=0, hel=None, **kw):
    mea = _mea()
    P = _proc(pdg, **kw)
    d_mom = torch.from_numpy(mom).cuda()
    out = torch.full((mom.shape[0],), float("nan"), dtype=torch.float64, device="cuda")
    flags = torch.zeros(mom.shape[0], dtype=torch.uint8, device="cuda")
    d_hel = torch.from_numpy(hel).cuda() if hel is not None else None
    P.evaluate(d_mom, out, hel_mode=hel_mode, hel=d_hel, precision=precision, flags=flags)
    torch.cuda.synchronize()
    return out.cpu().numpy(), flags.cpu().numpy()


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_fp64_path_matches_oracle(name):
    _, pdg, _, _ = _case(name)
    mom, ref = _data(name)
    got, flags = _run(pdg, mom, _mea().PREC_FP64)
    rel = np.abs(got / ref - 1.0)
    assert np.all(np.isfinite(got))
    assert rel.max() <= 1e-12, f"{name}: max rel {rel.max():.3e} at {int(rel.argmax())}"
    assert not np.any(flags)


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_mixed_path_matches_oracle(name):
    _, pdg, _, _ = _case(name)
    mom, ref = _data(name)
    got, flags = _run(pdg, mom, _mea().PREC_MIXED)
    rel = np.abs(got / ref - 1.0)
    assert np.all(np.isfinite(got))
    assert np.median(rel) <= 1e-6, f"{name}: median rel {np.median(rel):.3e}"
    assert rel.max() <= 1e-4, f"{name}: max rel {rel.max():.3e}"
    # re-evaluated events carry the FP64 result
    re = (flags & _mea().FLAG_REEVALUATED) != 0
    if re.any():
        assert rel[re].max() <= 1e-12


@pytest.mark.parametrize("name", ["gg>gg", "uu~>gg", "uu>uu", "gg>ggg", "uu~>ggg", "uu>uug"])
def test_every_straight_line_variant_matches_oracle(name):
    """Each emitted FP32 kernel variant (kernel_variant 1..6: body with shared
    vertex partials or one vertex call per diagram, at 128, 85 or 168
    registers) meets the mixed-path bar on its own; the register cap changes
    no bit."""
    _, pdg, _, _ = _case(name)
    mom, ref = _data(name)
    outs = []
    for v in (1, 2, 3, 4, 5, 6):
        got, _ = _run(pdg, mom, _mea().PREC_MIXED, kernel_variant=v)
        rel = np.abs(got / ref - 1.0)
        assert np.all(np.isfinite(got))
        assert np.median(rel) <= 1e-6, f"{name} variant {v}: median rel {np.median(rel):.3e}"
        assert rel.max() <= 1e-4, f"{name} variant {v}: max rel {rel.max():.3e}"
        outs.append(got)
    for k in (2, 4):  # same body at another register cap
        assert np.array_equal(outs[0], outs[k]) and np.array_equal(outs[1], outs[k + 1])


@pytest.mark.parametrize("name", ["gg>ggg", "uu~>ggg", "uu>uug", "gg>gggg"])
def test_per_helicity_given_mode(name):
    """MEA_HEL_GIVEN: one helicity combination per event, equal to the oracle's
    colour-summed value of that combination (times 1/4)."""
    _, pdg, _, _ = _case(name)
    mom, _ = _data(name)
    mom = mom[:37]
    n = len(pdg)
    _, hel_ref = oracle.OracleProcess(pdg).me2(mom, per_helicity=True)
    rng = np.random.default_rng(5)
    hidx = rng.integers(0, 1 << n, size=mom.shape[0])
    hel = np.array([[1 if (h >> (n - 1 - l)) & 1 else -1 for l in range(n)] for h in hidx], dtype=np.int8)
    got, _ = _run(pdg, mom, _mea().PREC_FP64, hel_mode=_mea().HEL_GIVEN, hel=hel)
    want = 0.25 * hel_ref[np.arange(mom.shape[0]), hidx]
    scale = 0.25 * hel_ref.max(axis=1)
    assert np.all(np.abs(got - want) <= 1e-12 * np.abs(want) + 1e-24 * scale)


@pytest.mark.parametrize("name", ["gg>gg", "uu~>ggg", "uu>uug", "gg>gggg"])
def test_sum_all_equals_sum_nonzero(name):
    _, pdg, _, _ = _case(name)
    mom, ref = _data(name)
    got, _ = _run(pdg, mom, _mea().PREC_FP64, hel_mode=_mea().HEL_SUM_ALL)
    assert np.max(np.abs(got / ref - 1.0)) <= 1e-12


def test_deterministic_and_batch_independent():
    """Same inputs give bitwise-identical output, alone or inside a larger batch."""
    pdg = [21] * 5
    mom, _ = _data("gg>ggg")
    a, _ = _run(pdg, mom, _mea().PREC_MIXED)
    b, _ = _run(pdg, mom, _mea().PREC_MIXED)
    c, _ = _run(pdg, mom[100:357], _mea().PREC_MIXED)
    assert np.array_equal(a, b)
    assert np.array_equal(a[100:357], c)
    d, _ = _run(pdg, mom, _mea().PREC_FP64)
    e, _ = _run(pdg, mom[5:6], _mea().PREC_FP64)
    assert d[5] == e[0]


@pytest.mark.parametrize("name", ["gg>ggg", "uu>uug", "uu~>ggg"])
def test_exact_power_scaling_fp64(name):
    _, pdg, _, _ = _case(name)
    mom, _ = _data(name)
    a, _ = _run(pdg, mom, _mea().PREC_FP64)
    b, _ = _run(pdg, 4.0 * mom, _mea().PREC_FP64)
    n = len(pdg)
    assert np.array_equal(b, a * 4.0 ** (8 - 2 * n))


def test_empty_and_single_event():
    pdg = [2, -2, 21, 21, 21]
    mom, ref = _data("uu~>ggg")
    mea = _mea()
    P = _proc(pdg)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    P.evaluate(torch.from_numpy(mom[:1]).cuda(), out, n_events=0, precision=mea.PREC_FP64)
    torch.cuda.synchronize()
    assert out.item() == 0.0
    got, _ = _run(pdg, mom[:1], mea.PREC_FP64)
    assert abs(got[0] / ref[0] - 1.0) <= 1e-12


def test_device_generator_matches_host_generator():
    mea = _mea()
    for nf, (lo, hi), dr, ptij in [(2, (200.0, 2000.0), 0.4, 0.0), (3, (200.0, 2000.0), 0.4, 0.0),
                                   (5, (500.0, 5000.0), 0.4, 0.0), (4, (100.0, 1000.0), 0.0, 20.0)]:
        n = 4096
        cfg = ps.PhaseSpaceConfig(nf, rs_lo=lo, rs_hi=hi, seed=ps.SEED_BASE + 3, dr_min=dr, ptij_min=ptij)
        host, att_h = ps.generate(cfg, n, first_event=1000, return_attempts=True)
        dev = torch.empty((n, nf + 2, 4), dtype=torch.float64, device="cuda")
        att = torch.empty(n, dtype=torch.int32, device="cuda")
        mea.generate_phase_space(nf, n, dev, first_event=1000, seed=cfg.seed, rs_lo=lo, rs_hi=hi,
                                 dr_min=dr, ptij_min=ptij, attempts=att)
        torch.cuda.synchronize()
        d = dev.cpu().numpy()
        same = att.cpu().numpy() == att_h
        assert same.mean() > 0.999
        scale = host[same][:, :, 0].max()
        assert np.abs(d[same] - host[same]).max() <= 1e-12 * scale


def test_host_buffer_entry_point():
    pdg = [21] * 5
    mom, ref = _data("gg>ggg")
    mea = _mea()
    P = _proc(pdg)
    got, flags = P.evaluate_host(mom, precision=mea.PREC_FP64, with_flags=True)
    assert np.max(np.abs(got / ref - 1.0)) <= 1e-12
    dev, _ = _run(pdg, mom, mea.PREC_FP64)
    assert np.array_equal(got, dev)


def test_argument_errors():
    mea = _mea()
    with pytest.raises(mea.MeaError) as e:
        mea.Process([21, 21, 11, 21])
    assert e.value.status == -2
    P = _proc([21] * 4)
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(mea.MeaError) as e:
        P.evaluate(None, out, n_events=4)
    assert e.value.status == -1
    with pytest.raises(mea.MeaError) as e:
        P.evaluate(out, out, n_events=4, hel_mode=mea.HEL_GIVEN, hel=None)
    assert e.value.status == -1


@pytest.mark.parametrize("name,nf,lo,hi", [("gg>ggg", 3, 200.0, 2000.0), ("uu~>ggg", 3, 200.0, 2000.0),
                                           ("uu>uug", 3, 200.0, 2000.0)])
def test_full_size_sampled(name, nf, lo, hi):
    """2^20 events generated on the device and evaluated in the benchmark's
    launch configuration; a random sample is checked against the oracle."""
    mea = _mea()
    _, pdg, _, _ = _case(name)
    n = 1 << 20
    mom = torch.empty((n, nf + 2, 4), dtype=torch.float64, device="cuda")
    mea.generate_phase_space(nf, n, mom, seed=ps.SEED_BASE + 1, rs_lo=lo, rs_hi=hi)
    out32 = torch.empty(n, dtype=torch.float64, device="cuda")
    out64 = torch.empty(n, dtype=torch.float64, device="cuda")
    P = _proc(pdg)
    P.evaluate(mom, out32, precision=mea.PREC_MIXED)
    P.evaluate(mom, out64, precision=mea.PREC_FP64)
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(3).choice(n, 96, replace=False))
    sample = mom[torch.from_numpy(idx).cuda()].cpu().numpy()
    ref = oracle.OracleProcess(pdg).me2(sample)
    g32 = out32.cpu().numpy()
    g64 = out64.cpu().numpy()
    assert np.all(np.isfinite(g32)) and np.all(np.isfinite(g64))
    assert np.max(np.abs(g64[idx] / ref - 1.0)) <= 1e-12
    r32 = np.abs(g32[idx] / ref - 1.0)
    assert np.median(r32) <= 1e-6 and r32.max() <= 1e-4
    # every event: mixed within 1e-4 of the FP64 GPU path
    assert np.max(np.abs(g32 / g64 - 1.0)) <= 1e-4


@pytest.mark.parametrize("name", ["gg>gg", "uu~>gg", "gg>ggg", "uu~>ggg", "uu>uug", "uu>uugg", "uu~>gggg"])
def test_tensor_core_colour_stage_forced(name):
    """Mixed path with the colour contraction forced onto the tcgen05 GEMM
    (colour_mode 2) for small colour bases, against the oracle."""
    _, pdg, _, _ = _case(name)
    mom, ref = _data(name)
    got, flags = _run(pdg, mom, _mea().PREC_MIXED, colour_mode=2)
    _proc(pdg, colour_mode=2).check_status()
    rel = np.abs(got / ref - 1.0)
    assert np.all(np.isfinite(got))
    assert np.median(rel) <= 1e-6, f"{name}: median rel {np.median(rel):.3e}"
    assert rel.max() <= 1e-4, f"{name}: max rel {rel.max():.3e}"


@pytest.mark.parametrize("name", ["gg>gggg", "uu~>gggg", "uu>uuggg", "uu~>ggggg", "gg>ggggg"])
def test_tensor_core_colour_stage_default_for_large_bases(name):
    """Processes without a straight-line kernel take the tensor-core stages by
    default (diagram amplitudes out, colour amplitudes and colour sum on
    tcgen05); the CUDA-core stage (colour_mode 1, two-sum colour amplitudes)
    on the same inputs agrees within the mixed tolerance."""
    _, pdg, _, _ = _case(name)
    mom, ref = _data(name)
    tc, _ = _run(pdg, mom, _mea().PREC_MIXED)
    _proc(pdg).check_status()
    cc, _ = _run(pdg, mom, _mea().PREC_MIXED, colour_mode=1)
    assert np.max(np.abs(tc / ref - 1.0)) <= 1e-4
    assert np.max(np.abs(cc / ref - 1.0)) <= 1e-4
    assert np.max(np.abs(tc / cc - 1.0)) <= 1e-4


@pytest.mark.parametrize("pdg,nf,lo,hi,n,chunk", [([21] * 7, 5, 500.0, 5000.0, 1001, 400),
                                                  ([2, -2, 21, 21, 21, 21, 21], 5, 500.0, 5000.0, 4999, 2000),
                                                  ([21] * 6, 4, 300.0, 3000.0, 20011, 0)])
def test_tensor_path_several_chunks_against_fp64(pdg, nf, lo, hi, n, chunk):
    """The tensor-core path splits large requests into event chunks that bound
    its scratch: gg>5g at 1001 events in chunks of 400 and uu~>5g at 4999 in
    chunks of 2000 (ragged last chunks), gg>4g at 20011 events with the
    automatic chunk size.  Every event agrees with the GPU FP64 path (itself
    pinned to the oracle at 1e-12)."""
    mea = _mea()
    P = _proc(pdg, chunk_events=chunk)
    d_mom = torch.empty((n, nf + 2, 4), dtype=torch.float64, device="cuda")
    mea.generate_phase_space(nf, n, d_mom, seed=ps.SEED_BASE + 211, rs_lo=lo, rs_hi=hi)
    mixed = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    fp64 = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    P.evaluate(d_mom, mixed, precision=mea.PREC_MIXED)
    P.evaluate(d_mom, fp64, precision=mea.PREC_FP64)
    P.check_status()
    rel = (mixed / fp64 - 1.0).abs().cpu().numpy()
    assert np.all(np.isfinite(rel))
    assert np.median(rel) <= 1e-6, np.median(rel)
    assert rel.max() <= 1e-4, rel.max()


def _collinear_event(n_final, delta, rs_scale=1000.0):
    """A massless event with final partons 0 and 1 at an angle delta (their
    invariant ~ a b delta^2), the others spread out, the last one balancing
    the spatial momentum; the incoming pair along z carries the total energy."""
    rng = np.random.default_rng(5)
    fin = []
    a, b = 0.3 * rs_scale, 0.2 * rs_scale
    n1 = np.array([np.sin(0.7), 0.0, np.cos(0.7)])
    n2 = np.array([np.sin(0.7 + delta), 0.0, np.cos(0.7 + delta)])
    fin.append(np.concatenate([[a], a * n1]))
    fin.append(np.concatenate([[b], b * n2]))
    for k in range(n_final - 3):
        th, ph = rng.uniform(1.0, 2.0), rng.uniform(0, 2 * np.pi)
        e = rs_scale * rng.uniform(0.1, 0.3)
        fin.append(np.array([e, e * np.sin(th) * np.cos(ph), e * np.sin(th) * np.sin(ph), e * np.cos(th)]))
    tot = np.sum(fin, axis=0)
    last = -tot[1:]
    fin.append(np.concatenate([[np.linalg.norm(last)], last]))
    rs = sum(f[0] for f in fin)
    pin = [np.array([rs / 2, 0, 0, rs / 2]), np.array([rs / 2, 0, 0, -rs / 2])]
    return np.array(pin + fin)


@pytest.mark.parametrize("pdg", [[21] * 5, [21] * 6])
def test_input_check_flags(pdg):
    """MEA_FLAG_MOMENTUM marks an event whose momenta do not balance (1e-6
    sqrt(s) added to one component); MEA_FLAG_QGUARD marks an event with two
    final partons 1e-7 rad apart (invariant ~1e-15 of the energy squared):
    on the mixed path it is re-evaluated in FP64 and agrees with the FP64 path;
    ordinary events carry neither bit.  Straight-line kernel (gg>ggg) and
    tensor-core path (gg>gggg)."""
    mea = _mea()
    nf = len(pdg) - 2
    good = ps.generate(ps.PhaseSpaceConfig(nf, rs_lo=300.0, rs_hi=3000.0, seed=ps.SEED_BASE + 307), 64)
    mom = good.copy()
    rs = np.sqrt((mom[5, 0, 0] + mom[5, 1, 0]) ** 2 - (mom[5, 0, 3] + mom[5, 1, 3]) ** 2)
    mom[5, 2, 1] += 1e-6 * rs
    mom[9] = _collinear_event(nf, 1e-7)
    out = {}
    for prec in (mea.PREC_MIXED, mea.PREC_FP64):
        got, fl = _run(pdg, mom, prec)
        out[prec] = (got, fl)
        assert fl[5] & 0x10 and not fl[5] & 0x08
        assert fl[9] & 0x08 and not fl[9] & 0x10
        others = np.delete(fl, [5, 9])
        assert not np.any(others & 0x18)
    gm, fm = out[mea.PREC_MIXED]
    g64, _ = out[mea.PREC_FP64]
    assert fm[9] & 0x01  # re-evaluated in FP64
    assert np.isfinite(g64[9]) and g64[9] > 0
    assert gm[9] == g64[9]


def test_bounded_wait_timeout_is_reported_and_the_context_survives():
    """A bounded mbarrier wait that expires (mea_probe_bounded_wait: nothing
    arrives) is reported by check_status as MEA_E_TIMEOUT, the indicator then
    resets, and the same context still evaluates correctly on the tensor-core
    path -- no hang, no fault."""
    mea = _mea()
    pdg = [21] * 6
    P = _proc(pdg)
    P.check_status()
    P.probe_bounded_wait(1000)
    with pytest.raises(mea.MeaError) as e:
        P.check_status()
    assert e.value.status == -5
    P.check_status()
    with pytest.raises(mea.MeaError):
        P.probe_bounded_wait(0)
    mom, ref = _data("gg>gggg")
    got, _ = _run(pdg, mom, mea.PREC_MIXED)
    P.check_status()
    assert np.median(np.abs(got / ref - 1.0)) <= 1e-6


@pytest.mark.parametrize("pdg,nf", [([2, 2, 2, 2, 21], 3), ([21] * 6, 4)])
def test_host_pipeline_across_chunks_equals_device_path(pdg, nf):
    """mea_evaluate_host works in chunks of 2^18 events on two streams, staging
    pageable buffers and copying page-locked ones directly; across several chunks (and a ragged last one) and a second
    call that reuses the buffers, every result and flag equals the
    device-resident evaluation bit for bit (straight-line and tensor-core
    paths)."""
    mea = _mea()
    n = (1 << 18) * 2 + 12345 if nf == 3 else 3001
    P = _proc(pdg)
    d_mom = torch.empty((n, nf + 2, 4), dtype=torch.float64, device="cuda")
    mea.generate_phase_space(nf, n, d_mom, seed=ps.SEED_BASE + 401, rs_lo=300.0, rs_hi=3000.0)
    ref = torch.empty(n, dtype=torch.float64, device="cuda")
    rfl = torch.empty(n, dtype=torch.uint8, device="cuda")
    P.evaluate(d_mom, ref, precision=mea.PREC_MIXED, flags=rfl)
    h = d_mom.cpu().numpy()
    for _ in range(2):
        got, fl = P.evaluate_host(h, precision=mea.PREC_MIXED, with_flags=True)
        assert np.array_equal(got, ref.cpu().numpy())
        assert np.array_equal(fl, rfl.cpu().numpy())
    # page-locked input and outputs: copied by the DMA engines without staging
    hp = d_mom.cpu().pin_memory().numpy()
    out = torch.full((n,), -1.0, dtype=torch.float64).pin_memory().numpy()
    fl = torch.full((n,), 0xEE, dtype=torch.uint8).pin_memory().numpy()
    got, fl2 = P.evaluate_host(hp, precision=mea.PREC_MIXED, out=out, flags=fl)
    assert got is out and fl2 is fl
    assert np.array_equal(out, ref.cpu().numpy())
    assert np.array_equal(fl, rfl.cpu().numpy())
    # pinned momenta, pageable results (mixed placement)
    got = P.evaluate_host(hp, precision=mea.PREC_MIXED)
    assert np.array_equal(got, ref.cpu().numpy())
