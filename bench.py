"""Benchmark: helicity-summed |M|^2 events/s per subprocess, mixed vs FP64 path.

Workload (default "3jet"): g g -> g g g, u u~ -> g g g and u u -> u u g, 2^20
synthetic events each per GPU (RAMBO flat massless phase space in the partonic
centre-of-mass frame, sqrt(s_hat) log-uniform in [200 GeV, 2 TeV], cuts
pT > 20 GeV, |eta| < 2.5, Delta R > 0.4, alpha_s = 0.118).  One step evaluates
every subprocess once.  Momenta are generated on the device before timing and
stay resident (2^20 x 5 x 32 B = 168 MB per subprocess, larger than L2, so no
explicit L2 flush is needed between steps).

Before timing, every subprocess is autotuned once per precision
(mea_autotune on the full launch for the straight-line kernels of the
processes with up to five partons, else on 2^16 events).  The line reports per subprocess the mixed and
FP64 rates, their relative difference (median / p99 / max), the flagged
fraction and the rate of the paper's sampled-helicity mode (one helicity per
event); the roofline of the dominant kernel; e2e through host buffers; clocks;
the oracle on the host cores as cpu_baseline.  Other workloads: --workload
2jet | 4jet | batch (one CUDA graph over four uneven subprocesses) | serve
(Poisson arrivals through the server, p50/p99).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload 3jet|2jet|4jet|batch|serve]
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
# ncu (dram__bytes_read.sum + dram__bytes_write.sum), one 2^20-event launch of
# the mixed-path kernel each subprocess runs: gg>ggg the per-diagram body at
# 128 registers, uu~>ggg the vertex-partial body at 128, uu>uug the per-diagram
# body at 85
TRAFFIC_BYTES_PER_EVENT = {"gg>ggg": (206848000 + 7545397760) / 2 ** 20,
                           "uu~>ggg": (168618752 + 7403264) / 2 ** 20,
                           "uu>uug": (168189952 + 21019136) / 2 ** 20}
SEED_BASE = 0x09095257
FP32_LANES_PER_SM = 128
MAX_SM_MHZ = 2070.0

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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        self.file.close()
        os.unlink(self.file.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
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


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    """The oracle (FP64 CPU, all host cores), as it stands, on a bounded sample
    of the same workload: each step evaluates `ref_events` events of every
    subprocess."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from paper_0909_5257_gb300 import phasespace as ps
    subs, n_full, seed_off = WORKLOADS[args.workload]
    n = args.ref_events
    procs, moms = [], []
    for name, pdg, nf, lo, hi in subs:
        procs.append(oracle.OracleProcess(pdg))
        moms.append(ps.generate(ps.PhaseSpaceConfig(nf, rs_lo=lo, rs_hi=hi, seed=SEED_BASE + seed_off), n))
    for _ in range(args.warmup):
        for P, m in zip(procs, moms):
            P.me2(m[: max(1, n // 16)])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for P, m in zip(procs, moms):
            P.me2(m)
    dt = time.perf_counter() - t0
    ev = args.steps * n * len(subs)
    value = ev / dt
    cores = oracle.max_threads()
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[args.workload], "sample_events_per_subprocess_per_step": n},
        "cpu_baseline": {"value": value, "unit": "events/s", "cores": cores, "kind": "oracle",
                         "sample": f"{n} events of each subprocess per step, {args.steps} steps"},
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def cpu_baseline(subs, seed_off, budget_s=12.0, single_budget_s=3.0):
    """Oracle on the host cores over a bounded sample of the workload, and on
    one core over a smaller one (the paper compares with one CPU core)."""
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


BATCH_SPEC = [  # (name, pdg, n_final, sqrt(s) range, configured events)
    ("gg>ggg", [21, 21, 21, 21, 21], 3, 200.0, 2000.0, 1 << 18),
    ("uu~>gggg", [2, -2, 21, 21, 21, 21], 4, 300.0, 3000.0, 1 << 20),
    ("uu>uuggg", [2, 2, 2, 2, 21, 21, 21], 5, 300.0, 3000.0, 1 << 19),
    ("gg>gggg", [21] * 6, 4, 300.0, 3000.0, 1 << 17),
]


def run_batch(args):
    """Batched mixed launch: four subprocesses of very uneven cost, counts
    perturbed by a seeded draw, autotuned per process, evaluated by one
    CUDA-graph launch per step (mea_batch_*); mixed vs FP64 graph."""
    import torch
    from paper_0909_5257_gb300 import mea
    torch.cuda.set_device(0)
    rng = np.random.default_rng(SEED_BASE + 3)
    procs, moms, n_ev = [], [], []
    for name, pdg, nf, lo, hi, n in BATCH_SPEC:
        n = max(64, int(n * args.scale * rng.uniform(0.75, 1.25)))
        P = mea.Process(pdg)
        m = torch.empty((n, nf + 2, 4), dtype=torch.float64, device="cuda")
        mea.generate_phase_space(nf, n, m, seed=SEED_BASE + 3, rs_lo=lo, rs_hi=hi)
        procs.append(P); moms.append(m); n_ev.append(n)
    tune = {}
    for (name, *_), P, m in zip(BATCH_SPEC, procs, moms):
        k = min(m.shape[0], 1 << 14)
        scratch = torch.empty(k, dtype=torch.float64, device="cuda")
        tune[name] = P.autotune(m[:k], scratch, precision=mea.PREC_MIXED)
    res = {}
    for prec, pname in ((mea.PREC_MIXED, "mixed"), (mea.PREC_FP64, "fp64")):
        outs = [torch.empty(n, dtype=torch.float64, device="cuda") for n in n_ev]
        flags = [torch.empty(n, dtype=torch.uint8, device="cuda") for n in n_ev]
        B = mea.Batch(list(zip(procs, moms, outs, flags)), precision=prec)
        steps = args.steps if pname == "mixed" else max(1, min(args.steps, 2))
        for _ in range(max(1, args.warmup if pname == "mixed" else 1)):
            B.launch()
        torch.cuda.synchronize()
        l0 = mea.kernel_launch_count()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(steps):
            B.launch()
        t1.record()
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / steps
        res[pname] = {"events_per_s": sum(n_ev) / (ms * 1e-3), "ms_per_launch": ms, "steps": steps,
                      "graph_kernel_nodes": B.kernel_nodes, "kernels_launched": mea.kernel_launch_count() - l0}
        res[pname + "_out"] = [o.clone() for o in outs]
        B.close()
    errs = {}
    for i, (name, *_) in enumerate(BATCH_SPEC):
        rel = (res["mixed_out"][i] / res["fp64_out"][i] - 1.0).abs()
        errs[name] = {"events": n_ev[i], "mixed_vs_fp64_rel_err_median": float(rel.median()),
                      "mixed_vs_fp64_rel_err_max": float(rel.max()), "autotune": tune[name]}
    out = {"metric": METRIC, "value": res["mixed"]["events_per_s"], "unit": "events/s", "n_gpus": 1,
           "steps": res["mixed"]["steps"], "warmup": args.warmup, "ms_per_step": res["mixed"]["ms_per_launch"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 amplitudes + tcgen05 f16-split colour sum; f64 re-evaluation", "data": "synthetic",
           "config": {"workload": "batched mixed launch (one CUDA graph): " +
                      ", ".join(f"{b[0]} {n}" for b, n in zip(BATCH_SPEC, n_ev)),
                      "scale": args.scale},
           "fp64": {k: v for k, v in res["fp64"].items()}, "mixed": {k: v for k, v in res["mixed"].items()},
           "per_subprocess": errs, "gpu_launches": res["mixed"]["kernels_launched"]}
    print(json.dumps(out), flush=True)


SERVE_MIX = [("gg>ggggg", [21] * 7, 5, 0.4), ("uu~>ggggg", [2, -2, 21, 21, 21, 21, 21], 5, 0.4),
             ("uu>uuggg", [2, 2, 2, 2, 21, 21, 21], 5, 0.2)]


def run_serve(args):
    """Serving: Poisson arrivals, request sizes log-uniform in
    [2^10, 2^18] x scale events, mix 40/40/20 % of gg>ggggg, uu~>ggggg,
    uu>uuggg, sqrt(s) in [500 GeV, 5 TeV]; offered load a fraction of the
    measured capacity; p50/p99 latency and throughput for the mixed and the
    FP64 path."""
    import torch
    from paper_0909_5257_gb300 import mea
    torch.cuda.set_device(0)
    rng = np.random.default_rng(SEED_BASE + 4)
    procs = {name: mea.Process(pdg) for name, pdg, _, _ in SERVE_MIX}
    n_req = max(8, args.steps * 4)
    lo_n, hi_n = (1 << 10) * args.scale, (1 << 18) * args.scale
    reqs = []
    first = 0
    for k in range(n_req):
        name, pdg, nf, _ = SERVE_MIX[int(rng.choice(3, p=[w for *_, w in SERVE_MIX]))]
        n = max(16, int(np.exp(rng.uniform(np.log(lo_n), np.log(hi_n)))))
        m = torch.empty((n, nf + 2, 4), dtype=torch.float64, device="cuda")
        mea.generate_phase_space(nf, n, m, first_event=first, seed=SEED_BASE + 4, rs_lo=500.0, rs_hi=5000.0)
        first += n
        reqs.append((name, m, n))
    torch.cuda.synchronize()
    results = {}
    for prec, pname in ((mea.PREC_MIXED, "mixed"), (mea.PREC_FP64, "fp64")):
        # capacity: back-to-back submission
        srv = mea.Server(mem_budget_bytes=160 << 30, n_slots=4, chunk_events=1 << 12)
        outs = [torch.empty(n, dtype=torch.float64, device="cuda") for _, _, n in reqs]
        t0 = time.perf_counter()
        ids = [srv.submit(procs[nm], m, o, precision=prec) for (nm, m, n), o in zip(reqs, outs)]
        for i in ids:
            srv.wait(i, timeout_ms=600000)
        cap_s = time.perf_counter() - t0
        total = sum(n for _, _, n in reqs)
        srv.close()
        capacity = total / cap_s
        # Poisson arrivals at 0.8 x capacity
        mean_gap = (total / len(reqs)) / (0.8 * capacity)
        gaps = rng.exponential(mean_gap, size=len(reqs))
        srv = mea.Server(mem_budget_bytes=160 << 30, n_slots=4, chunk_events=1 << 12)
        t0 = time.perf_counter()
        ids = []
        tnext = t0
        for (nm, m, n), o, g in zip(reqs, outs, gaps):
            tnext += g
            while time.perf_counter() < tnext:
                time.sleep(min(0.001, max(0.0, tnext - time.perf_counter())))
            ids.append(srv.submit(procs[nm], m, o, precision=prec))
        for i in ids:
            srv.wait(i, timeout_ms=600000)
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        results[pname] = {"capacity_events_per_s": capacity, "offered_load": 0.8, "events_per_s": total / wall,
                          "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
                          "requests": len(reqs), "events": total}
    out = {"metric": METRIC, "value": results["mixed"]["events_per_s"], "unit": "events/s", "n_gpus": 1,
           "steps": n_req, "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32 amplitudes + tcgen05 f16-split colour sum; f64 re-evaluation",
           "data": "synthetic",
           "config": {"workload": "serving: Poisson arrivals at 0.8 x capacity, sizes log-uniform "
                                  f"[{int(lo_n)}, {int(hi_n)}], mix 40/40/20 gg>ggggg/uu~>ggggg/uu>uuggg",
                      "scale": args.scale, "slots": 4, "chunk_events": 4096},
           "p50_ms": results["mixed"]["p50_ms"], "p99_ms": results["mixed"]["p99_ms"],
           "mixed": results["mixed"], "fp64": results["fp64"]}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="3jet", choices=sorted(WORKLOADS) + ["batch", "serve"])
    ap.add_argument("--scale", type=float, default=1.0,
                    help="batch/serve: multiply the configured event counts (bounded runs)")
    ap.add_argument("--ref-events", type=int, default=4096)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-sampled", action="store_true",
                    help="skip the sampled-helicity (one helicity per event) throughput")
    args = ap.parse_args()

    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batch":
        run_batch(args)
        return
    if args.workload == "serve":
        run_serve(args)
        return

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

    def max_over_ranks(x):
        return max_over_ranks_value(x, dist, "cuda")

    subs, n, seed_off = WORKLOADS[args.workload]
    stream = torch.cuda.current_stream()
    procs, moms, outs, flags = [], [], [], []
    for name, pdg, nf, lo, hi in subs:
        P = mea.Process(pdg)
        m = torch.empty((n, nf + 2, 4), dtype=torch.float64, device="cuda")
        # weak scaling: every rank evaluates its own slice of the event stream
        mea.generate_phase_space(nf, n, m, first_event=shard_first_event(rank, n), seed=SEED_BASE + seed_off,
                                 rs_lo=lo, rs_hi=hi)
        procs.append(P)
        moms.append(m)
        outs.append(torch.empty(n, dtype=torch.float64, device="cuda"))
        flags.append(torch.empty(n, dtype=torch.uint8, device="cuda"))
    torch.cuda.synchronize()
    # one-time tile / register-variant / body choice per subprocess and
    # precision, outside the timed region: the straight-line kernels are tuned
    # on the full launch (their spill footprint competes with the streamed
    # inputs for L2 only at that size), the others on a 2^16-event sample
    tuned = {}
    if not args.no_autotune:
        for (name, *_), P, m, o in zip(subs, procs, moms, outs):
            k = n if P.n_ext <= 5 else min(n, 1 << 16)
            tuned[name] = {pn: P.autotune(m[:k], o[:k], precision=pr)
                           for pr, pn in ((mea.PREC_MIXED, "mixed"), (mea.PREC_FP64, "fp64"))}
        torch.cuda.synchronize()

    def step(prec, ev_pairs=None):
        for i, P in enumerate(procs):
            if ev_pairs is not None:
                ev_pairs[i][0].record(stream)
            P.evaluate(moms[i], outs[i], precision=prec, flags=flags[i], stream=stream)
            if ev_pairs is not None:
                ev_pairs[i][1].record(stream)

    def timed(prec, steps):
        for _ in range(args.warmup):
            step(prec)
        barrier()
        per = [[] for _ in procs]
        pairs = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in procs] for _ in range(steps)]
        l0 = mea.kernel_launch_count()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for s in range(steps):
            step(prec, pairs[s])
        t1.record(stream)
        torch.cuda.synchronize()
        barrier()
        launches = mea.kernel_launch_count() - l0
        ms = t0.elapsed_time(t1)
        for s in range(steps):
            for i in range(len(procs)):
                per[i].append(pairs[s][i][0].elapsed_time(pairs[s][i][1]))
        return max_over_ranks(ms) / steps, per, launches

    sampler = ClockSampler(local)
    sampler.start()
    ms_mixed, per_mixed, launches = timed(mea.PREC_MIXED, args.steps)
    clocks = sampler.stop()
    # the clones run on torch's stream: finish them before the FP64 pass
    # overwrites the outputs on the evaluation stream
    mixed_out = [o.clone() for o in outs]
    mixed_flags = [f.clone() for f in flags]
    torch.cuda.synchronize()

    fp64 = None
    if not args.no_fp64:
        ms64, per64, _ = timed(mea.PREC_FP64, args.steps)
        fp64 = {"value": ws * n * len(procs) / (ms64 * 1e-3), "unit": "events/s", "ms_per_step": ms64}
    fp64_out = [o.clone() for o in outs]
    torch.cuda.synchronize()

    per_sub = {}
    for i, (name, pdg, nf, lo, hi) in enumerate(subs):
        info = procs[i].info
        ms_i = statistics.median(per_mixed[i])
        d = {"mixed_events_per_s": n / (ms_i * 1e-3), "diagrams": info["n_diagrams"], "colours": info["n_colour"],
             "helicities": info["n_hel_nonzero"],
             "flagged_fraction": float((mixed_flags[i] != 0).float().mean().item())}
        if fp64 is not None:
            d["fp64_events_per_s"] = n / (statistics.median(per64[i]) * 1e-3)
            rel = (mixed_out[i] / fp64_out[i] - 1.0).abs()
            d["mixed_vs_fp64_rel_err_median"] = float(rel.median().item())
            d["mixed_vs_fp64_rel_err_max"] = float(rel.max().item())
            d["mixed_vs_fp64_rel_err_p99"] = float(torch.quantile(rel.float(), 0.99).item())
        if not args.no_sampled:
            # the paper's mode (one helicity per event, drawn from the
            # non-vanishing set): throughput only, for comparison with its
            # per-event timings (one sampled helicity = 1/H of a summed event)
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
        per_sub[name] = d

    # roofline of the dominant kernel: the fused amplitude + colour kernel of the
    # most expensive subprocess, FP32 pipe (ALU-bound), algorithmic FLOPs per launch
    # FLOPs of the straight-line body the tuner chose: with the shared vertex
    # partials, or one vertex call per diagram (flops_per_hel_plain)
    def body_flops(i):
        name = subs[i][0]
        plain = name in tuned and not tuned[name]["mixed"].get("vertex_partials", 1)
        return procs[i].info["flops_per_hel_plain" if plain else "flops_per_hel"]
    cost = [procs[i].info["n_hel_nonzero"] * (body_flops(i) + procs[i].info["colour_flops_per_hel"])
            for i in range(len(procs))]
    dom = int(np.argmax([c * statistics.median(per_mixed[i]) for i, c in enumerate(cost)]))
    ms_dom = statistics.mean(per_mixed[dom])
    flops_launch = n * cost[dom]
    achieved = flops_launch / (ms_dom * 1e-3) / 1e12
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak = n_sms * FP32_LANES_PER_SM * 2 * MAX_SM_MHZ * 1e6 / 1e12
    # DRAM bytes per event of each kernel from one ncu capture of the current
    # kernels (dram__bytes_read.sum + dram__bytes_write.sum of one 2^20-event
    # launch, divided by the events), scaled to this launch's events.  Mostly
    # spill write-back for gg>ggg.
    traffic_per_event = TRAFFIC_BYTES_PER_EVENT.get(subs[dom][0])
    traffic = None if traffic_per_event is None else traffic_per_event * n
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic,
                "kernel": (f"gen_kernel<float> straight-line body ({subs[dom][0]})" if len(subs[dom][1]) <= 5
                           else f"amp_kernel<float> + jamp/colour GEMMs ({subs[dom][0]})") +
                          ", per-launch CUDA events incl. the FP64 re-evaluation launch",
                "peak_note": f"derived: {n_sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 FLOP x {MAX_SM_MHZ:.0f} MHz"}

    # end to end through the host-buffer entry point
    e2e = None
    if rank == 0 or ws > 1:
        # inputs and results in pinned host memory: the library's copy engines
        # read and write them directly (pageable arrays would be staged)
        host = [m.cpu().pin_memory().numpy() for m in moms]
        outs = [torch.empty(h.shape[0], dtype=torch.float64).pin_memory().numpy() for h in host]
        fls = [torch.empty(h.shape[0], dtype=torch.uint8).pin_memory().numpy() for h in host]
        for P, h, o, f in zip(procs, host, outs, fls):  # warm-up at full size
            P.evaluate_host(h, precision=mea.PREC_MIXED, out=o, flags=f)
        barrier()
        t0 = time.perf_counter()
        e2e_steps = max(1, min(args.steps, 3))
        for _ in range(e2e_steps):
            for P, h, o, f in zip(procs, host, outs, fls):
                P.evaluate_host(h, precision=mea.PREC_MIXED, out=o, flags=f)
        dt = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": ws * n * len(procs) * e2e_steps / dt, "unit": "events/s",
               "h2d_bytes_per_step": int(sum(h.nbytes for h in host)),
               "d2h_bytes_per_step": int(sum(h.shape[0] * 9 for h in host)), "steps": e2e_steps}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    peaks, peak_src = _peaks()
    out = {
        "metric": METRIC,
        "value": ws * n * len(procs) / (ms_mixed * 1e-3),
        "unit": "events/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_mixed,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 amplitudes (two-sum colour amplitudes) + f64 prep/re-evaluation",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[args.workload], "events_per_subprocess_per_gpu": n,
                   "l2": "inputs larger than L2 (no flush)", "alpha_s": 0.118,
                   "autotuned": {k: {pn: {kk: v[pn][kk] for kk in ("threads", "events_per_cta", "register_cap", "vertex_partials")}
                                     for pn in v} for k, v in tuned.items()}},
        "per_subprocess": per_sub,
        "fp64": fp64,
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "peaks_source": peak_src,
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(subs, seed_off)
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
