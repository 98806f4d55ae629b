"""Benchmark: helicity-summed |M|^2 events/s per subprocess, mixed vs FP64 path; p50/p99.

Default workload "serve" -- the serving configuration: requests over
g g -> 5g (7245 diagrams, 720 colours), u u~ -> 5g (1890 diagrams, 120 colours)
and u u -> u u + 3g (786 diagrams, 240 colours), process mix 40/40/20 % by
request, request sizes log-uniform in [2^10, 2^18] events, sqrt(s_hat)
log-uniform in [500 GeV, 5 TeV] (RAMBO flat massless phase space in the
partonic centre-of-mass frame, cuts pT > 20 GeV, |eta| < 2.5, Delta R > 0.4,
alpha_s = 0.118).  Synthetic, seeded data; momenta generated on the device
before timing.  Inputs are larger than L2 (one request of 2^18 events holds
59 MB of momenta plus GBs of tensor-path scratch), so no explicit flush.

One step = REQS_PER_STEP requests.  After W warm-up steps, the K timed steps'
requests are all submitted to the continuous-batching server (mea_server_*)
at once and the timed region ends when the last completes: `value` is the
whole job's events/s at saturation (capacity), `ms_per_step` the timed
region / K.  Then, with the same requests:
  * latency: Poisson arrivals at 0.8 x the measured capacity, `p50_ms` and
    `p99_ms` of submit-to-completion latency (mixed path);
  * e2e: every request's momenta copied from pinned host memory to the
    device, submitted, and its |M|^2 copied back, inside the timed region;
  * per subprocess: device-timed (CUDA events) mixed events/s on 2^16-2^17
    events, FP64 events/s on a subsample of the same inputs, the mixed-vs-FP64
    relative error (median / p99 / max) and the flagged fraction;
  * roofline of the dominant kernel (the stage with the largest share of the
    mix's device time, timed per stage with CUDA events on its stream), the
    tensor-core stages' useful and executed rates against the sustained BF16
    peak, measured FP32 / FP64 pipe peaks (FMA-chain kernel, this GPU);
  * cpu_baseline: the FP64 oracle on the host cores on a bounded sample of the
    mix, and the FP64 GPU path's largest relative error against it there.
Other workloads (also reported as extra keys unless --no-extra): "3jet"
(gg>ggg, uu~>ggg, uu>uug, 2^20 each), "4jet" (gg>gggg, uu~>gggg), "batch"
(one CUDA graph over four uneven subprocesses), "2jet"; "single" evaluates one
subprocess (--process, --events) inside an NVTX range "eval" for profilers.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload serve|3jet|4jet|2jet|batch|single]
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "helicity-summed |M|^2 events/s per subprocess, mixed vs FP64 path; p50/p99"
SEED_BASE = 0x09095257
FP32_LANES_PER_SM = 128
MAX_SM_MHZ = 2070.0

# ---- serving workload ------------------------------------------------------
SERVE_MIX = [("gg>ggggg", [21] * 7, 5, 0.4), ("uu~>ggggg", [2, -2, 21, 21, 21, 21, 21], 5, 0.4),
             ("uu>uuggg", [2, 2, 2, 2, 21, 21, 21], 5, 0.2)]
SERVE_RS = (500.0, 5000.0)
SERVE_SIZES = (1 << 10, 1 << 18)
REQS_PER_STEP = 3
SERVE_SLOTS = 4
SERVE_CHUNK = 1 << 12
SERVE_LOAD = 0.8
# per-subprocess device-timed pass: events (mixed), FP64 subsample, oracle sample
SUB_EVENTS = {"gg>ggggg": 1 << 16, "uu~>ggggg": 1 << 17, "uu>uuggg": 1 << 17}
FP64_EVENTS = {"gg>ggggg": 2048, "uu~>ggggg": 8192, "uu>uuggg": 16384}
CPU_SAMPLE = {"gg>ggggg": 16, "uu~>ggggg": 16, "uu>uuggg": 8}
REF_PER_STEP = {"gg>ggggg": 4, "uu~>ggggg": 4, "uu>uuggg": 2}
# ncu (dram__bytes_read.sum + dram__bytes_write.sum) per event of the dominant
# kernel, from the full-size one-pass ncu capture summarised under profiles/,
# keyed by (subprocess, stage, amplitude kernel 0 per-lane / 1 helicity-shared
# / 2 split, threads, events per CTA, grid): a launch in another configuration
# reports null
TRAFFIC_BYTES_PER_EVENT = {("gg>ggggg", "amplitudes", 0, 128, 1, 1368): (41.71e9 + 35.25e9) / 2731,
                           ("gg>ggggg", "amplitudes", 0, 224, 2, 760): (42.30e9 + 35.25e9) / 2731,
                           ("gg>ggggg", "amplitudes", 1, 128, 4, 456): (3.19e9 + 18.99e9) / 2731,
                           ("gg>ggggg", "amplitudes", 2, 448, 4, 304): (5.52e9 + 19.09e9) / 2731}

# ---- device-resident workloads (extra keys) ------------------------------------
WORKLOADS = {
    # name: (subprocesses, events per subprocess per GPU, seed offset)
    "3jet": ([("gg>ggg", [21, 21, 21, 21, 21], 3, 200.0, 2000.0),
              ("uu~>ggg", [2, -2, 21, 21, 21], 3, 200.0, 2000.0),
              ("uu>uug", [2, 2, 2, 2, 21], 3, 200.0, 2000.0)], 1 << 20, 1),
    "2jet": ([("gg>gg", [21, 21, 21, 21], 2, 200.0, 2000.0),
              ("uu~>gg", [2, -2, 21, 21], 2, 200.0, 2000.0)], 1 << 14, 0),
    "4jet": ([("gg>gggg", [21] * 6, 4, 300.0, 3000.0),
              ("uu~>gggg", [2, -2, 21, 21, 21, 21], 4, 300.0, 3000.0)], 1 << 20, 2),
}
WORKLOAD_TEXT = {
    "3jet": "gg>ggg + uu~>ggg + uu>uug, 2^20 events each per GPU, sqrt(s) in [200 GeV, 2 TeV]",
    "2jet": "gg>gg + uu~>gg, 2^14 events each per GPU, sqrt(s) in [200 GeV, 2 TeV]",
    "4jet": "gg>gggg + uu~>gggg, 2^20 events each per GPU, sqrt(s) in [300 GeV, 3 TeV]",
}
SINGLE = {
    "gg3g": ([21] * 5, 200.0, 2000.0), "uu3g": ([2, -2, 21, 21, 21], 200.0, 2000.0),
    "uuuug": ([2, 2, 2, 2, 21], 200.0, 2000.0), "gg4g": ([21] * 6, 300.0, 3000.0),
    "uu4g": ([2, -2, 21, 21, 21, 21], 300.0, 3000.0), "uuuu3g": ([2, 2, 2, 2, 21, 21, 21], 500.0, 5000.0),
    "uu5g": ([2, -2] + [21] * 5, 500.0, 5000.0), "gg5g": ([21] * 7, 500.0, 5000.0),
}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # nvidia-smi takes a moment to start: wait (up to 3 s) for its first
        # sample so that the timed region that follows is covered
        t_end = time.time() + 3.0
        while time.time() < t_end and self.proc.poll() is None:
            try:
                if os.path.getsize(self.file.name) > 0:
                    break
            except OSError:
                break
            time.sleep(0.02)

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        self.file.close()
        os.unlink(self.file.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def shard_first_event(rank: int, n_per_rank: int) -> int:
    """Weak scaling: rank r evaluates events [r*n, (r+1)*n) of the seeded stream."""
    return rank * n_per_rank


def max_over_ranks_value(x: float, dist=None, device=None) -> float:
    """Max of a host scalar over all ranks (timing only; no data-path collective)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def serve_requests(rank: int, n_req: int, seed: int = SEED_BASE + 4):
    """The serving workload's request stream: request k = (subprocess index,
    events, first event of its momenta in that subprocess's generator
    stream), drawn from its own seeded generator, so the stream does not
    depend on how much of it is taken.  Rank r takes requests
    [r*n_req, (r+1)*n_req): the ranks' requests are disjoint (weak scaling)."""
    p = [w for *_, w in SERVE_MIX]
    lo, hi = np.log(SERVE_SIZES[0]), np.log(SERVE_SIZES[1])
    out, nxt = [], [0] * len(SERVE_MIX)
    for k in range((rank + 1) * n_req):
        rng = np.random.default_rng([seed, k])
        kind = int(rng.choice(len(SERVE_MIX), p=p))
        size = min(SERVE_SIZES[1], max(SERVE_SIZES[0], int(round(np.exp(rng.uniform(lo, hi))))))
        if k >= rank * n_req:
            out.append((kind, size, nxt[kind]))
        nxt[kind] += size
    return out


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---- the oracle (reference arm and cpu_baseline) --------------------------------
def run_reference(args):
    """The oracle (FP64 CPU, all host cores), as it stands, on a bounded sample
    of the same workload; rank 0 only."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from paper_0909_5257_gb300 import phasespace as ps
    if args.workload == "serve":
        subs = [(name, pdg, nf, SERVE_RS[0], SERVE_RS[1]) for name, pdg, nf, _ in SERVE_MIX]
        per_step = dict(REF_PER_STEP)
        seed = SEED_BASE + 4
        text = serve_workload_text()
    else:
        subs, _, seed_off = WORKLOADS[args.workload]
        per_step = {s[0]: args.ref_events for s in subs}
        seed = SEED_BASE + seed_off
        text = WORKLOAD_TEXT[args.workload]
    procs, moms = [], []
    total_steps = args.warmup + args.steps
    for name, pdg, nf, lo, hi in subs:
        procs.append(oracle.OracleProcess(pdg))
        moms.append(ps.generate(ps.PhaseSpaceConfig(nf, rs_lo=lo, rs_hi=hi, seed=seed),
                                per_step[name] * total_steps))
    for s in range(args.warmup):
        for (name, *_), P, m in zip(subs, procs, moms):
            k = per_step[name]
            P.me2(m[s * k:(s + 1) * k])
    t0 = time.perf_counter()
    for s in range(args.warmup, total_steps):
        for (name, *_), P, m in zip(subs, procs, moms):
            k = per_step[name]
            P.me2(m[s * k:(s + 1) * k])
    dt = time.perf_counter() - t0
    ev = args.steps * sum(per_step.values())
    value = ev / dt
    cores = oracle.max_threads()
    sample = ", ".join(f"{per_step[s[0]]} {s[0]}" for s in subs)
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": text, "sample_per_step": sample},
        "cpu_baseline": {"value": value, "unit": "events/s", "cores": cores, "kind": "oracle",
                         "sample": f"{sample} events per step (distinct events every step), {args.steps} steps"},
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def serve_workload_text():
    return ("serving: continuous batching over gg>ggggg / uu~>ggggg / uu>uuggg, mix 40/40/20 % by request, "
            "request sizes log-uniform in [2^10, 2^18] events, sqrt(s) in [500 GeV, 5 TeV]")


def cpu_baseline(subs, seed_off, budget_s=12.0, single_budget_s=3.0):
    """Oracle on the host cores over a bounded sample of a device-resident
    workload, and on one core over a smaller one (the paper compares with
    one CPU core)."""
    import oracle
    from paper_0909_5257_gb300 import phasespace as ps
    cores = oracle.max_threads()
    tot_ev, tot_t, parts = 0, 0.0, []
    one_ev, one_t = 0, 0.0
    for name, pdg, nf, lo, hi in subs:
        P = oracle.OracleProcess(pdg)
        probe = ps.generate(ps.PhaseSpaceConfig(nf, rs_lo=lo, rs_hi=hi, seed=SEED_BASE + seed_off), 256)
        t0 = time.perf_counter()
        P.me2(probe)
        rate = 256 / max(time.perf_counter() - t0, 1e-6)
        n = int(min(max(rate * budget_s / len(subs), 256), 1 << 16))
        mom = ps.generate(ps.PhaseSpaceConfig(nf, rs_lo=lo, rs_hi=hi, seed=SEED_BASE + seed_off), n)
        t0 = time.perf_counter()
        P.me2(mom)
        dt = time.perf_counter() - t0
        tot_ev += n
        tot_t += dt
        parts.append(f"{name}: {n} events in {dt:.1f} s")
        k = int(min(max(n / dt / max(cores, 1) * single_budget_s / len(subs), 16), n))
        t0 = time.perf_counter()
        P.me2(mom[:k], threads=1)
        one_t += time.perf_counter() - t0
        one_ev += k
        P.me2(mom[:1], threads=cores)  # the thread count is library state: restore it
    return {"value": tot_ev / tot_t, "unit": "events/s", "cores": cores, "kind": "oracle",
            "sample": "; ".join(parts),
            "single_core_value": one_ev / one_t, "single_core_sample": f"{one_ev} events in {one_t:.1f} s"}


def serve_cpu_baseline(procs):
    """The oracle on the host cores over a bounded sample of the serving mix
    (CPU_SAMPLE events per subprocess, host generator), and the FP64 GPU
    path's relative error against it on those very events."""
    import torch

    import oracle
    from paper_0909_5257_gb300 import mea
    from paper_0909_5257_gb300 import phasespace as ps
    cores = oracle.max_threads()
    tot_ev, tot_t, parts, errs = 0, 0.0, [], {}
    for name, pdg, nf, _ in SERVE_MIX:
        n = CPU_SAMPLE[name]
        mom = ps.generate(ps.PhaseSpaceConfig(nf, rs_lo=SERVE_RS[0], rs_hi=SERVE_RS[1], seed=SEED_BASE + 24), n)
        P = oracle.OracleProcess(pdg)
        t0 = time.perf_counter()
        ref = P.me2(mom)
        dt = time.perf_counter() - t0
        tot_ev += n
        tot_t += dt
        parts.append(f"{name}: {n} events in {dt:.1f} s")
        d = torch.from_numpy(mom).cuda()
        o = torch.empty(n, dtype=torch.float64, device="cuda")
        procs[name].evaluate(d, o, precision=mea.PREC_FP64)
        o2 = torch.empty(n, dtype=torch.float64, device="cuda")
        procs[name].evaluate(d, o2, precision=mea.PREC_MIXED)
        torch.cuda.synchronize()
        r64 = np.abs(o.cpu().numpy() / ref - 1.0)
        r32 = np.abs(o2.cpu().numpy() / ref - 1.0)
        errs[name] = {"events": n, "fp64_max_rel_err": float(r64.max()),
                      "mixed_median_rel_err": float(np.median(r32)), "mixed_max_rel_err": float(r32.max())}
    return ({"value": tot_ev / tot_t, "unit": "events/s", "cores": cores, "kind": "oracle",
             "sample": "; ".join(parts) + " (host generator, sqrt(s) in [500 GeV, 5 TeV])"}, errs)


# ---- device-resident workloads ---------------------------------------------------
def device_workload(name, steps, warmup, rank=0, ws=1, dist=None, autotune=True, sampled=True, fp64_events=None):
    """Evaluate every subprocess of a device-resident workload `steps` times
    (after `warmup`), mixed and FP64 (on the first fp64_events events, all by
    default); per-subprocess rates, errors, the timing of each evaluation
    (CUDA events on the launching stream)."""
    import torch
    from paper_0909_5257_gb300 import mea

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    subs, n, seed_off = WORKLOADS[name]
    stream = torch.cuda.current_stream()
    procs, moms, outs, flags = [], [], [], []
    for sname, pdg, nf, lo, hi in subs:
        P = mea.Process(pdg)
        m = torch.empty((n, nf + 2, 4), dtype=torch.float64, device="cuda")
        mea.generate_phase_space(nf, n, m, first_event=shard_first_event(rank, n), seed=SEED_BASE + seed_off,
                                 rs_lo=lo, rs_hi=hi)
        procs.append(P)
        moms.append(m)
        outs.append(torch.empty(n, dtype=torch.float64, device="cuda"))
        flags.append(torch.empty(n, dtype=torch.uint8, device="cuda"))
    torch.cuda.synchronize()
    tuned = {}
    if autotune:
        for (sname, *_), P, m, o in zip(subs, procs, moms, outs):
            k = n if P.n_ext <= 5 else min(n, 1 << 16)
            k64 = k if fp64_events is None else min(k, fp64_events)
            tuned[sname] = {pn: P.autotune(m[:kk], o[:kk], precision=pr)
                            for pr, pn, kk in ((mea.PREC_MIXED, "mixed", k), (mea.PREC_FP64, "fp64", k64))}
        torch.cuda.synchronize()

    n64 = n if fp64_events is None else min(n, fp64_events)

    def step(prec, ev_pairs=None):
        ne = n if prec == mea.PREC_MIXED else n64
        for i, P in enumerate(procs):
            if ev_pairs is not None:
                ev_pairs[i][0].record(stream)
            P.evaluate(moms[i][:ne], outs[i][:ne], precision=prec, flags=flags[i][:ne], stream=stream)
            if ev_pairs is not None:
                ev_pairs[i][1].record(stream)

    def timed(prec, k):
        for _ in range(warmup if prec == mea.PREC_MIXED else min(warmup, 1)):
            step(prec)
        barrier()
        pairs = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in procs] for _ in range(k)]
        l0 = mea.kernel_launch_count()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for s in range(k):
            step(prec, pairs[s])
        t1.record(stream)
        torch.cuda.synchronize()
        barrier()
        per = [[pairs[s][i][0].elapsed_time(pairs[s][i][1]) for s in range(k)] for i in range(len(procs))]
        ms = max_over_ranks_value(t0.elapsed_time(t1), dist, "cuda")
        return ms / k, per, mea.kernel_launch_count() - l0

    ms_mixed, per_mixed, launches = timed(mea.PREC_MIXED, steps)
    mixed_out = [o.clone() for o in outs]
    mixed_flags = [f.clone() for f in flags]
    torch.cuda.synchronize()
    ms64, per64, _ = timed(mea.PREC_FP64, max(1, min(steps, 3)))
    fp64_out = [o.clone() for o in outs]
    torch.cuda.synchronize()
    per_sub = {}
    for i, (sname, pdg, nf, lo, hi) in enumerate(subs):
        info = procs[i].info
        rel = (mixed_out[i][:n64] / fp64_out[i][:n64] - 1.0).abs()
        d = {"mixed_events_per_s": n / (statistics.median(per_mixed[i]) * 1e-3),
             "fp64_events_per_s": n64 / (statistics.median(per64[i]) * 1e-3), "fp64_events": n64,
             "diagrams": info["n_diagrams"], "colours": info["n_colour"], "helicities": info["n_hel_nonzero"],
             "flagged_fraction": float((mixed_flags[i] != 0).float().mean().item()),
             "mixed_vs_fp64_rel_err_median": float(rel.median().item()),
             "mixed_vs_fp64_rel_err_p99": float(torch.quantile(rel.float(), 0.99).item()),
             "mixed_vs_fp64_rel_err_max": float(rel.max().item())}
        if sampled:
            P = procs[i]
            hels = torch.from_numpy(P.helicities()).to("cuda")
            g = torch.Generator(device="cuda").manual_seed(SEED_BASE + 11 + i)
            pick = torch.randint(0, hels.shape[0], (n,), device="cuda", generator=g)
            hsel = hels[pick].contiguous()
            so = torch.empty(n, dtype=torch.float64, device="cuda")
            P.evaluate(moms[i], so, hel_mode=mea.HEL_GIVEN, hel=hsel, precision=mea.PREC_MIXED, stream=stream)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for _ in range(3):
                P.evaluate(moms[i], so, hel_mode=mea.HEL_GIVEN, hel=hsel, precision=mea.PREC_MIXED, stream=stream)
            ev1.record(stream)
            torch.cuda.synchronize()
            d["sampled_helicity_events_per_s"] = n / (ev0.elapsed_time(ev1) / 3 * 1e-3)
        per_sub[sname] = d
    return {"subs": subs, "n": n, "n64": n64, "procs": procs, "moms": moms, "per_sub": per_sub, "tuned": tuned,
            "ms_mixed": ms_mixed, "ms_fp64": ms64, "per_mixed": per_mixed, "launches": launches}


BATCH_SPEC = [  # (name, pdg, n_final, sqrt(s) range, configured events)
    ("gg>ggg", [21, 21, 21, 21, 21], 3, 200.0, 2000.0, 1 << 18),
    ("uu~>gggg", [2, -2, 21, 21, 21, 21], 4, 300.0, 3000.0, 1 << 20),
    ("uu>uuggg", [2, 2, 2, 2, 21, 21, 21], 5, 300.0, 3000.0, 1 << 19),
    ("gg>gggg", [21] * 6, 4, 300.0, 3000.0, 1 << 17),
]


def batch_workload(steps, warmup, scale=1.0, with_fp64=True):
    """Batched mixed launch: four subprocesses of very uneven cost, counts
    perturbed by a seeded draw, autotuned per process, evaluated by one
    CUDA-graph launch per step (mea_batch_*); mixed vs FP64 graph."""
    import torch
    from paper_0909_5257_gb300 import mea
    rng = np.random.default_rng(SEED_BASE + 3)
    procs, moms, n_ev = [], [], []
    for name, pdg, nf, lo, hi, n in BATCH_SPEC:
        n = max(64, int(n * scale * rng.uniform(0.75, 1.25)))
        P = mea.Process(pdg)
        m = torch.empty((n, nf + 2, 4), dtype=torch.float64, device="cuda")
        mea.generate_phase_space(nf, n, m, seed=SEED_BASE + 3, rs_lo=lo, rs_hi=hi)
        procs.append(P)
        moms.append(m)
        n_ev.append(n)
    tune = {}
    for (name, *_), P, m in zip(BATCH_SPEC, procs, moms):
        k = min(m.shape[0], 1 << 14)
        scratch = torch.empty(k, dtype=torch.float64, device="cuda")
        tune[name] = P.autotune(m[:k], scratch, precision=mea.PREC_MIXED)
    res = {}
    precs = ((mea.PREC_MIXED, "mixed"), (mea.PREC_FP64, "fp64")) if with_fp64 else ((mea.PREC_MIXED, "mixed"),)
    for prec, pname in precs:
        outs = [torch.empty(n, dtype=torch.float64, device="cuda") for n in n_ev]
        flags = [torch.empty(n, dtype=torch.uint8, device="cuda") for n in n_ev]
        B = mea.Batch(list(zip(procs, moms, outs, flags)), precision=prec)
        k = steps if pname == "mixed" else max(1, min(steps, 2))
        for _ in range(max(1, warmup if pname == "mixed" else 1)):
            B.launch()
        torch.cuda.synchronize()
        l0 = mea.kernel_launch_count()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(k):
            B.launch()
        t1.record()
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / k
        res[pname] = {"events_per_s": sum(n_ev) / (ms * 1e-3), "ms_per_launch": ms, "steps": k,
                      "graph_kernel_nodes": B.kernel_nodes, "kernels_launched": mea.kernel_launch_count() - l0}
        res[pname + "_out"] = [o.clone() for o in outs]
        B.close()
    errs = {}
    for i, (name, *_) in enumerate(BATCH_SPEC):
        errs[name] = {"events": n_ev[i],
                      "autotune": {k: tune[name][k] for k in ("threads", "events_per_cta", "register_cap",
                                                                "helicity_shared")}}
        if with_fp64:
            rel = (res["mixed_out"][i] / res["fp64_out"][i] - 1.0).abs()
            errs[name]["mixed_vs_fp64_rel_err_median"] = float(rel.median())
            errs[name]["mixed_vs_fp64_rel_err_max"] = float(rel.max())
    return {"workload": "batched mixed launch (one CUDA graph): " +
                        ", ".join(f"{b[0]} {n}" for b, n in zip(BATCH_SPEC, n_ev)),
            "mixed": res["mixed"], "fp64": res.get("fp64"), "per_subprocess": errs}


# ---- serving headline ---------------------------------------------------------------
def _stage_flops(info, H):
    """Algorithmic work per (event, helicity) pair of each stage of the
    tensor-core path: FP32 FLOPs of the amplitude program without the
    colour-amplitude accumulation (done by the tensor cores there), the
    useful tensor FLOPs of the colour amplitudes (2 FLOP per non-zero
    coefficient for each of Re, Im) and of the colour sum (4 m^2)."""
    nnz = info["n_colour_entries"]
    m = info["n_colour_amplitudes"]
    return {"amplitudes": info["flops_per_hel"] - 4.0 * nnz, "colour_amplitudes": 4.0 * nnz,
            "colour_sum": 4.0 * m * m}


def _cdiv(a, b):
    return -(-a // b)


def _amp_kernel_kind(tune_result):
    """Which amplitude kernel the tensor-core path of a process runs: the
    tuner's choice (0 per-lane interpreter, 1 helicity-shared, 2 split), else
    the untuned default, the per-lane interpreter."""
    return int(tune_result.get("helicity_shared", 0)) if tune_result else 0


AMP_KERNEL_NAMES = {0: "per-lane", 1: "helicity-shared", 2: "split"}


def _jamp_executed_flops(info):
    """Tensor FLOPs the colour-amplitude GEMM executes per (event, helicity)
    pair: Re and Im rows x 2 FLOP x padded diagrams x padded colour columns
    x 3 digit planes (tiles of 64 diagrams, column splits of at most 128)."""
    m, kd = info["n_colour_amplitudes"], info["n_diagrams"]
    nc = min(128, _cdiv(m, 16) * 16)
    splits = _cdiv(m, nc)
    nc = min(nc, _cdiv(_cdiv(m, splits), 16) * 16)
    return 2 * 2 * (_cdiv(kd, 64) * 64) * (splits * nc) * 3


def _colour_sum_executed_flops(info):
    """Tensor FLOPs the colour-sum GEMM executes per pair: 2 rows x 2 FLOP x
    padded K x padded N x MMAs per K step (3 for the 3-way split of J when the
    integer colour matrix is exact in FP16, else 5)."""
    m = info["n_colour_amplitudes"]
    nb = _cdiv(m, 256)
    nc = _cdiv(_cdiv(m, nb), 32) * 32
    n_mma = 3 if info["cf_max_abs_numerator"] <= 2048 else 5
    return 2 * 2 * (_cdiv(m, 64) * 64) * (nb * nc) * n_mma


def run_serve(args):
    import torch
    from paper_0909_5257_gb300 import mea
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    names = [s[0] for s in SERVE_MIX]
    procs = {name: mea.Process(pdg, auto_tune=not args.no_autotune) for name, pdg, _, _ in SERVE_MIX}
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count

    # measured ALU peaks of this GPU (FMA chains), with the SM clock they ran at
    sampler = ClockSampler(local)
    sampler.start()
    fp32_peak, _ = mea.measure_alu_peak(False, 0.3)
    fp64_peak, _ = mea.measure_alu_peak(True, 0.3)
    peak_clocks = sampler.stop()

    phase = {}
    t_phase = time.perf_counter()

    def lap(name):
        nonlocal t_phase
        now = time.perf_counter()
        phase[name] = round(now - t_phase, 1)
        t_phase = now

    # ---- per subprocess: device-timed mixed (stage timing) and FP64 on the same inputs
    per_sub, stage_ms_ev, tune = {}, {}, {}
    reps = max(1, min(args.steps, 3))
    for i, (name, pdg, nf, _) in enumerate(SERVE_MIX):
        P = procs[name]
        n = SUB_EVENTS[name]
        mom = torch.empty((n, nf + 2, 4), dtype=torch.float64, device="cuda")
        mea.generate_phase_space(nf, n, mom, first_event=shard_first_event(rank, n), seed=SEED_BASE + 14,
                                 rs_lo=SERVE_RS[0], rs_hi=SERVE_RS[1])
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        fl = torch.empty(n, dtype=torch.uint8, device="cuda")
        k = min(n, 1 << 16)
        if not args.no_autotune:
            tune[name] = P.autotune(mom[:k], out[:k], precision=mea.PREC_MIXED)
        P.evaluate(mom, out, precision=mea.PREC_MIXED, flags=fl, stream=stream)
        torch.cuda.synchronize()
        P.set_stage_timing(True)
        P.stage_times()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            P.evaluate(mom, out, precision=mea.PREC_MIXED, flags=fl, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        st = P.stage_times()
        P.set_stage_timing(False)
        ms = e0.elapsed_time(e1) / reps
        stage_ms_ev[name] = {k2: (v[0] / reps / n, v[1] / reps) for k2, v in st.items() if v[1] > 0}
        n64 = FP64_EVENTS[name]
        o64 = torch.empty(n64, dtype=torch.float64, device="cuda")
        P.evaluate(mom[:64], o64[:64], precision=mea.PREC_FP64, stream=stream)
        e0.record(stream)
        P.evaluate(mom[:n64], o64, precision=mea.PREC_FP64, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        rel = (out[:n64] / o64 - 1.0).abs()
        info = P.info
        per_sub[name] = {
            "mixed_events_per_s": n / (ms * 1e-3), "mixed_events": n,
            "fp64_events_per_s": n64 / (ms64 * 1e-3), "fp64_events": n64,
            "mixed_vs_fp64_rel_err_median": float(rel.median()), "mixed_vs_fp64_rel_err_p99":
                float(torch.quantile(rel.float(), 0.99)), "mixed_vs_fp64_rel_err_max": float(rel.max()),
            "flagged_fraction": float((fl != 0).float().mean()),
            "diagrams": info["n_diagrams"], "colours": info["n_colour"], "helicities": info["n_hel_nonzero"],
            "stage_ms_per_event": {k2: v[0] for k2, v in stage_ms_ev[name].items()},
            "amplitude_kernel": AMP_KERNEL_NAMES[_amp_kernel_kind(tune.get(name))] +
                                (", forwarding" if (tune.get(name) or {}).get("forwarding") else ""),
        }
        del mom, out, fl, o64
        torch.cuda.empty_cache()

    # ---- the dominant kernel: largest share of the mix's device time per event
    mix_w = {name: w for name, _, _, w in SERVE_MIX}
    share = {(nm, stg): mix_w[nm] * v[0] for nm in names for stg, v in stage_ms_ev[nm].items()}
    dom_nm, dom_stage = max(share, key=share.get)
    tot_share = sum(share.values())
    info = procs[dom_nm].info
    H = info["n_hel_nonzero"]
    fl_stage = _stage_flops(info, H)
    peaks, peak_src = _peaks()
    bf16_sus = peaks.get("bf16_tflops_sustained", 1700.0)
    ms_per_launch = stage_ms_ev[dom_nm][dom_stage][0] * SUB_EVENTS[dom_nm] / max(
        stage_ms_ev[dom_nm][dom_stage][1], 1)
    events_per_launch = SUB_EVENTS[dom_nm] / max(stage_ms_ev[dom_nm][dom_stage][1], 1)
    if dom_stage == "amplitudes":
        tc = tune.get(dom_nm) or {}
        kind = _amp_kernel_kind(tc)
        # algorithmic FLOPs of the kernel that ran: the helicity-shared and the
        # split kernels evaluate (some) wavefunctions once per helicity pattern
        # of their legs
        per_event = {1: info["hs_flops_per_event"], 2: info["hsp_flops_per_event"]}.get(
            kind, H * fl_stage["amplitudes"])
        flop = events_per_launch * per_event
        achieved = flop / (ms_per_launch * 1e-3) / 1e12
        tpe = None if tc.get("forwarding") else TRAFFIC_BYTES_PER_EVENT.get(
            (dom_nm, dom_stage, kind, tc.get("threads"), tc.get("events_per_cta"), tc.get("grid")))
        kname = {1: "amp_hs_kernel<float> (helicity-shared)", 2: "amp_hsp_kernel<float> (split)"}.get(
            kind, "amp_kernel<float> amplitude output" + (" with forwarding" if tc.get("forwarding") else ""))
        roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": achieved / fp32_peak, "traffic": None if tpe is None else tpe * events_per_launch,
                    "kernel": f"{kname} ({dom_nm}), {events_per_launch:.0f} events "
                              "per launch, CUDA events per launch on its stream",
                    "flops_per_event": per_event,
                    "peak_note": "measured on this GPU: FMA-chain kernel (mea_measure_alu_peak), "
                                 f"SM clock median {peak_clocks.get('sm_mhz')} MHz",
                    "share_of_mix_device_time": share[(dom_nm, dom_stage)] / tot_share}
    else:
        flop = events_per_launch * H * fl_stage.get(dom_stage, 0.0)
        achieved = flop / (ms_per_launch * 1e-3) / 1e12
        roofline = {"bound": "tensor", "achieved": achieved, "peak": bf16_sus, "unit": "TFLOP/s",
                    "frac": achieved / bf16_sus, "traffic": None,
                    "kernel": f"{dom_stage} ({dom_nm})", "peak_note": f"bf16 sustained, {peak_src}",
                    "share_of_mix_device_time": share[(dom_nm, dom_stage)] / tot_share}
    # tensor-core stages of every subprocess: useful (algorithmic) and executed rates
    tensor = {}
    for nm in names:
        inf = procs[nm].info
        h = inf["n_hel_nonzero"]
        f = _stage_flops(inf, h)
        for stg, exec_flop in (("colour_amplitudes", _jamp_executed_flops(inf)),
                               ("colour_sum", _colour_sum_executed_flops(inf))):
            if stg in stage_ms_ev[nm]:
                sec = stage_ms_ev[nm][stg][0] * 1e-3  # per event
                useful = h * f[stg] / sec / 1e12
                executed = h * exec_flop / sec / 1e12
                tensor[f"{nm} {stg}"] = {"useful_tflops": useful, "executed_tflops": executed,
                                         "useful_frac": useful / bf16_sus, "executed_frac": executed / bf16_sus}

    lap("per_subprocess_and_roofline")
    # ---- serving: capacity (timed steps), latency under Poisson load, e2e
    n_req = args.steps * REQS_PER_STEP
    reqs = serve_requests(rank, n_req)
    warm = serve_requests(rank + 7, max(1, args.warmup) * REQS_PER_STEP)  # a different slice for warm-up
    datas = []
    for kind, n, first in reqs + warm:
        name, pdg, nf, _ = SERVE_MIX[kind]
        m = torch.empty((n, nf + 2, 4), dtype=torch.float64, device="cuda")
        mea.generate_phase_space(nf, n, m, first_event=first, seed=SEED_BASE + 4 + kind,
                                 rs_lo=SERVE_RS[0], rs_hi=SERVE_RS[1])
        datas.append((name, m, n))
    torch.cuda.synchronize()
    timed_reqs, warm_reqs = datas[:n_req], datas[n_req:]
    outs = [torch.empty(n, dtype=torch.float64, device="cuda") for _, _, n in timed_reqs]
    flags = [torch.empty(n, dtype=torch.uint8, device="cuda") for _, _, n in timed_reqs]
    total = sum(n for _, _, n in timed_reqs)
    budget = 200 << 30

    def serve_all(srv, items, gaps=None, out_list=None, flag_list=None):
        ids = []
        t_next = time.perf_counter()
        for j, (nm, m, n) in enumerate(items):
            if gaps is not None:
                t_next += gaps[j]
                while time.perf_counter() < t_next:
                    time.sleep(min(0.001, max(0.0, t_next - time.perf_counter())))
            o = out_list[j] if out_list is not None else torch.empty(n, dtype=torch.float64, device="cuda")
            f = flag_list[j] if flag_list is not None else None
            ids.append(srv.submit(procs[nm], m, o, flags=f, precision=mea.PREC_MIXED))
        try:
            return [srv.wait(i, timeout_ms=900000) for i in ids]
        except mea.MeaError as err:
            free, tot = torch.cuda.mem_get_info()
            raise RuntimeError(f"serving failed ({err}); device memory free {free / 2**30:.1f} of "
                               f"{tot / 2**30:.1f} GiB") from err

    srv = mea.Server(mem_budget_bytes=budget, n_slots=SERVE_SLOTS, chunk_events=SERVE_CHUNK)
    serve_all(srv, warm_reqs)  # warm-up steps: scratch sized, modules loaded
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    l0 = mea.kernel_launch_count()
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    t0 = time.perf_counter()
    # the timed region as the profiler's collection range (cudaProfilerStart/Stop:
    # process-wide, so the server's worker-thread launches are inside it; no-ops
    # without a profiler)
    torch.cuda.profiler.start()
    serve_all(srv, timed_reqs, out_list=outs, flag_list=flags)
    c1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    wall = time.perf_counter() - t0
    barrier()
    clocks = sampler.stop()
    launches = mea.kernel_launch_count() - l0
    dev_ms = max_over_ranks_value(c0.elapsed_time(c1), dist, "cuda")
    srv_stats = srv.stats()
    srv.close()
    capacity = ws * total / (dev_ms * 1e-3)
    flagged = float(sum(int((f != 0).sum()) for f in flags)) / total

    lap("serving_capacity")
    # latency under Poisson arrivals at SERVE_LOAD x capacity (this rank's share)
    rng = np.random.default_rng(SEED_BASE + 5 + rank)
    mean_gap = (total / len(timed_reqs)) / (SERVE_LOAD * capacity / ws)
    gaps = rng.exponential(mean_gap, size=len(timed_reqs))
    srv = mea.Server(mem_budget_bytes=budget, n_slots=SERVE_SLOTS, chunk_events=SERVE_CHUNK)
    serve_all(srv, warm_reqs[:1])
    t0 = time.perf_counter()
    lat = serve_all(srv, timed_reqs, gaps=gaps, out_list=outs)
    load_wall = time.perf_counter() - t0
    srv.close()
    lat_sorted = sorted(lat)

    def q(f):
        return lat_sorted[min(len(lat_sorted) - 1, int(round(f * (len(lat_sorted) - 1))))]

    by_proc = {}
    for (nm, _, n), l in zip(timed_reqs, lat):
        by_proc.setdefault(nm, []).append(l)

    lap("serving_latency")
    # e2e: momenta from pinned host memory, results back to pinned host memory
    host = [m.cpu().pin_memory() for _, m, _ in timed_reqs]
    host_out = [torch.empty(n, dtype=torch.float64).pin_memory() for _, _, n in timed_reqs]
    dev_in = [torch.empty_like(m) for _, m, _ in timed_reqs]
    copy_stream = torch.cuda.Stream()
    srv = mea.Server(mem_budget_bytes=budget, n_slots=SERVE_SLOTS, chunk_events=SERVE_CHUNK)
    serve_all(srv, warm_reqs[:1])
    barrier()
    t0 = time.perf_counter()
    ids = []
    for j, (nm, _, n) in enumerate(timed_reqs):
        with torch.cuda.stream(copy_stream):
            dev_in[j].copy_(host[j], non_blocking=True)
        copy_stream.synchronize()
        ids.append(srv.submit(procs[nm], dev_in[j], outs[j], precision=mea.PREC_MIXED))
    for j, i in enumerate(ids):
        srv.wait(i, timeout_ms=900000)
        with torch.cuda.stream(copy_stream):
            host_out[j].copy_(outs[j], non_blocking=True)
    copy_stream.synchronize()
    e2e_wall = max_over_ranks_value(time.perf_counter() - t0, dist, "cuda")
    srv.close()
    e2e = {"value": ws * total / e2e_wall, "unit": "events/s",
           "h2d_bytes_per_step": int(sum(h.numel() * 8 for h in host) / args.steps),
           "d2h_bytes_per_step": int(sum(n * 8 for _, _, n in timed_reqs) / args.steps),
           "how": "per request: pinned host momenta -> device (copy stream), mea_server_submit; |M|^2 "
                  "device -> pinned host after completion; wall clock over all requests"}
    del host, host_out, dev_in
    lap("serving_e2e")

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # the capacity the per-subprocess device rates predict for these very
    # requests (their own mix of sizes): the server's efficiency is value / this
    expect_s = sum(n / per_sub[nm]["mixed_events_per_s"] for nm, _, n in timed_reqs)
    expected_capacity = ws * total / expect_s
    # FP64 serving capacity of the same mix, from the per-subprocess FP64 rates
    fp64_cap = 1.0 / sum(mix_w[nm] / per_sub[nm]["fp64_events_per_s"] for nm in names)
    mixed_cap_dev = 1.0 / sum(mix_w[nm] / per_sub[nm]["mixed_events_per_s"] for nm in names)
    out = {
        "metric": METRIC, "value": capacity, "unit": "events/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 amplitudes + tcgen05 f16-digit colour stages (f32 accumulate); f64 prep/re-evaluation",
        "data": "synthetic",
        "config": {"workload": serve_workload_text(), "requests_per_step": REQS_PER_STEP,
                   "requests": len(timed_reqs), "events": int(total), "server_slots": SERVE_SLOTS,
                   "server_chunk_events": SERVE_CHUNK, "alpha_s": 0.118,
                   "l2": "inputs larger than L2 (no flush)",
                   "timed_region": "all K x requests_per_step requests submitted at once; CUDA events on the "
                                   "submitting stream around submission and observed completion"},
        "p50_ms": q(0.50), "p99_ms": q(0.99),
        "serving": {"capacity_events_per_s": capacity, "host_wall_s": wall, "device_ms": dev_ms,
                    "capacity_from_device_rates_for_these_requests": expected_capacity,
                    "server_efficiency": capacity / expected_capacity,
                    "events_by_subprocess": {nm: int(sum(n for x, _, n in timed_reqs if x == nm)) for nm in names},
                    "flagged_fraction": flagged, "server_busy_s": srv_stats["busy_seconds"],
                    "latency": {"offered_load": SERVE_LOAD, "arrivals": "Poisson", "p50_ms": q(0.50),
                                "p99_ms": q(0.99), "max_ms": lat_sorted[-1], "wall_s": load_wall,
                                "served_events_per_s": total / load_wall,
                                "p50_ms_by_subprocess": {k: float(np.median(v)) for k, v in by_proc.items()}},
                    "mixed_capacity_from_device_rates": mixed_cap_dev,
                    "fp64_capacity_from_device_rates": fp64_cap},
        "per_subprocess": per_sub,
        "fp64": {"value": fp64_cap, "unit": "events/s",
                 "note": "mix-weighted from the per-subprocess FP64 device rates (FP64 serving of full-size "
                         "requests would take minutes)"},
        "roofline": roofline,
        "tensor_stages": tensor,
        "alu_peaks": {"fp32_tflops": fp32_peak, "fp64_tflops": fp64_peak, "clocks": peak_clocks,
                      "how": "mea_measure_alu_peak: FMA chains, 8 per thread, 4 x 512 threads per SM, CUDA events"},
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "peaks_source": peak_src,
        "autotuned": {k: {kk: v[kk] for kk in ("threads", "events_per_cta", "grid", "slots_in_shared")}
                      for k, v in tune.items()},
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"], out["fp64_vs_oracle"] = serve_cpu_baseline(procs)
        lap("cpu_baseline")
    if not args.no_extra:
        extra = {}
        # bounded: FP64 on a subsample (2^18 / 2^16 events), the batch's FP64 graph left out
        for wl, n64 in (("3jet", 1 << 18), ("4jet", 1 << 16)):
            t_wl = time.perf_counter()
            r = device_workload(wl, 3, 2, sampled=(wl == "3jet"), fp64_events=n64)
            extra[wl] = {"workload": WORKLOAD_TEXT[wl],
                         "mixed_events_per_s": len(r["subs"]) * r["n"] / (r["ms_mixed"] * 1e-3),
                         "fp64_events_per_s": len(r["subs"]) * r["n64"] / (r["ms_fp64"] * 1e-3),
                         "fp64_events_per_subprocess": r["n64"], "per_subprocess": r["per_sub"],
                         "wall_s": time.perf_counter() - t_wl}
            del r
            torch.cuda.empty_cache()
        t_wl = time.perf_counter()
        extra["batch"] = batch_workload(3, 2, with_fp64=False)
        extra["batch"]["wall_s"] = time.perf_counter() - t_wl
        out["other_workloads"] = extra
        lap("other_workloads")
    out["phase_wall_s"] = phase
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_device(args):
    """A device-resident workload (3jet, 4jet, 2jet) as the headline line."""
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_0909_5257_gb300 import mea
    sampler = ClockSampler(local)
    sampler.start()
    r = device_workload(args.workload, args.steps, args.warmup, rank, ws, dist, autotune=not args.no_autotune,
                        sampled=not args.no_sampled)
    clocks = sampler.stop()
    subs, n, procs = r["subs"], r["n"], r["procs"]
    # roofline of the dominant kernel: the fused straight-line kernel (or the
    # amplitude kernel) of the most expensive subprocess, FP32 pipe
    fp32_peak, _ = mea.measure_alu_peak(False, 0.3)

    def body_flops(i):
        name = subs[i][0]
        plain = name in r["tuned"] and not r["tuned"][name]["mixed"].get("vertex_partials", 1)
        return procs[i].info["flops_per_hel_plain" if plain else "flops_per_hel"]
    cost = [procs[i].info["n_hel_nonzero"] * (body_flops(i) + procs[i].info["colour_flops_per_hel"])
            for i in range(len(procs))]
    per = r["per_mixed"]
    dom = int(np.argmax([c * statistics.median(per[i]) for i, c in enumerate(cost)]))
    achieved = n * cost[dom] / (statistics.mean(per[dom]) * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": None,
                "kernel": f"straight-line / amplitude kernel of {subs[dom][0]}, per-launch CUDA events",
                "peak_note": "measured FMA-chain kernel (mea_measure_alu_peak)"}
    e2e = None
    if rank == 0:
        host = [m.cpu().pin_memory().numpy() for m in r["moms"]]
        outs = [torch.empty(h.shape[0], dtype=torch.float64).pin_memory().numpy() for h in host]
        fls = [torch.empty(h.shape[0], dtype=torch.uint8).pin_memory().numpy() for h in host]
        for P, h, o, f in zip(procs, host, outs, fls):
            P.evaluate_host(h, precision=mea.PREC_MIXED, out=o, flags=f)
        t0 = time.perf_counter()
        k = max(1, min(args.steps, 3))
        for _ in range(k):
            for P, h, o, f in zip(procs, host, outs, fls):
                P.evaluate_host(h, precision=mea.PREC_MIXED, out=o, flags=f)
        dt = time.perf_counter() - t0
        e2e = {"value": n * len(procs) * k / dt, "unit": "events/s",
               "h2d_bytes_per_step": int(sum(h.nbytes for h in host)),
               "d2h_bytes_per_step": int(sum(h.shape[0] * 9 for h in host)), "steps": k}
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    peaks, peak_src = _peaks()
    out = {"metric": METRIC, "value": ws * n * len(procs) / (r["ms_mixed"] * 1e-3), "unit": "events/s",
           "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_mixed"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 amplitudes + f64 prep/re-evaluation", "data": "synthetic",
           "config": {"workload": WORKLOAD_TEXT[args.workload], "events_per_subprocess_per_gpu": n,
                      "l2": "inputs larger than L2 (no flush)", "alpha_s": 0.118},
           "per_subprocess": r["per_sub"],
           "fp64": {"value": ws * n * len(procs) / (r["ms_fp64"] * 1e-3), "unit": "events/s"},
           "roofline": roofline, "e2e": e2e, "gpu_launches": r["launches"], "clocks": clocks,
           "peaks_source": peak_src}
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(subs, WORKLOADS[args.workload][2])
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_single(args):
    """One subprocess, --events events generated on the device, evaluated
    once (tuning on first use; below 2^16 events tuned beforehand on 2^16
    events, as the serving workload's per-subprocess pass is; neither with
    --no-autotune), then again inside an NVTX range "eval" (the range a
    profiler restricts itself to); prints timing and the tuned configuration."""
    import torch
    from paper_0909_5257_gb300 import mea
    pdg, lo, hi = SINGLE[args.process]
    torch.cuda.set_device(0)
    prec = mea.PREC_FP64 if args.precision == "fp64" else mea.PREC_MIXED
    P = mea.Process(pdg, auto_tune=not args.no_autotune, helicity_sharing=args.helicity_sharing)
    n = args.events
    # below 2^16 events the evaluation would not tune itself: tune on 2^16
    # events of the same generator, as the serving workload does
    tune_here = n < (1 << 16) and not args.no_autotune
    n_gen = max(n, 1 << 16) if tune_here else n
    mom = torch.empty((n_gen, len(pdg), 4), dtype=torch.float64, device="cuda")
    mea.generate_phase_space(len(pdg) - 2, n_gen, mom, rs_lo=lo, rs_hi=hi)
    out = torch.empty(n_gen, dtype=torch.float64, device="cuda")
    tuned = None
    if tune_here:
        r = P.autotune(mom[:1 << 16], out[:1 << 16], precision=prec)
        tuned = {k: r[k] for k in ("threads", "events_per_cta", "grid", "slots_in_shared", "helicity_shared",
                                   "register_cap")}
    mom, out = mom[:n], out[:n]
    P.evaluate(mom, out, precision=prec)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("eval")
    e0.record()
    P.evaluate(mom, out, precision=prec)
    e1.record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    P.check_status()
    ms = e0.elapsed_time(e1)
    print(json.dumps({"process": args.process, "events": n, "precision": args.precision, "ms": ms,
                      "events_per_s": n / (ms * 1e-3), "mean_me2": float(out.mean()),
                      "config": tuned}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="serve", choices=["serve", "batch", "single"] + sorted(WORKLOADS))
    ap.add_argument("--process", default="gg5g", choices=sorted(SINGLE), help="single: the subprocess")
    ap.add_argument("--events", type=int, default=4096, help="single: events")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"], help="single: precision")
    ap.add_argument("--helicity-sharing", type=int, default=0, choices=[0, 1, 2, 3],
                    help="single: amplitude kernel of the tensor-core path (0 tuned, 1 per-lane, 2 helicity-shared, "
                         "3 split)")
    ap.add_argument("--scale", type=float, default=1.0, help="batch: multiply the configured event counts")
    ap.add_argument("--ref-events", type=int, default=4096)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="serve: skip the other workloads' extra keys")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-sampled", action="store_true",
                    help="skip the sampled-helicity (one helicity per event) throughput")
    args = ap.parse_args()

    if args.impl == "reference":
        if args.workload in ("batch", "single"):
            print(json.dumps({"impl": "reference", "unavailable": "the oracle arm covers serve/2jet/3jet/4jet"}))
            return
        run_reference(args)
        return
    if args.workload == "serve":
        run_serve(args)
    elif args.workload == "single":
        run_single(args)
    elif args.workload == "batch":
        import torch
        torch.cuda.set_device(0)
        r = batch_workload(args.steps, args.warmup, args.scale)
        out = {"metric": METRIC, "value": r["mixed"]["events_per_s"], "unit": "events/s", "n_gpus": 1,
               "steps": r["mixed"]["steps"], "warmup": args.warmup, "ms_per_step": r["mixed"]["ms_per_launch"],
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f32 amplitudes + tcgen05 f16-digit colour stages; f64 re-evaluation", "data": "synthetic",
               "config": {"workload": r["workload"], "scale": args.scale}, "mixed": r["mixed"], "fp64": r["fp64"],
               "per_subprocess": r["per_subprocess"], "gpu_launches": r["mixed"]["kernels_launched"]}
        print(json.dumps(out), flush=True)
    else:
        run_device(args)


if __name__ == "__main__":
    main()
