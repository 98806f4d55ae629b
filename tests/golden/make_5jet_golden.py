"""Write the stored |M|^2 values of the 5-jet parity tests.

Runs the FP64 oracle (and nothing else of the engine) on events of the seeded
host input generator -- the serving workload's 2 -> 5 subprocesses
g g -> 5g, u u~ -> 5g and u u -> u u + 3g at sqrt(s_hat) log-uniform in
[500 GeV, 5 TeV] with the jet cuts pT > 20 GeV, |eta| < 2.5, Delta R > 0.4 --
and writes one text file per subprocess into this directory:

    golden_5jet_<name>.txt: header lines (# ...) with the generator settings,
    then one line per event: event index and |M|^2 (GeV^-6, 17 significant
    digits), initial helicities and colours averaged (Sec. 2.1,
    Eq. (color-averaged-amplitude) with the 1/4 and 1/(n_a n_b) averages).

The values are the oracle's; the oracle is pinned by the CPU tests
(closed forms, Parke-Taylor, Berends-Giele, Ward identities, collinear
factorisation).  Usage (takes about 15 minutes on 8 host cores):

    python tests/golden/make_5jet_golden.py [n_events]
"""
from __future__ import annotations

import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_0909_5257_gb300 import phasespace as ps  # noqa: E402

# (file name, PDG codes, n_final); the serving workload's generator settings
SUBPROCESSES = [
    ("gg_5g", [21] * 7, 5),
    ("uux_5g", [2, -2, 21, 21, 21, 21, 21], 5),
    ("uu_uu3g", [2, 2, 2, 2, 21, 21, 21], 5),
]
SEED = ps.SEED_BASE + 4
RS_LO, RS_HI = 500.0, 5000.0


def config(n_final: int) -> ps.PhaseSpaceConfig:
    return ps.PhaseSpaceConfig(n_final, rs_lo=RS_LO, rs_hi=RS_HI, seed=SEED)


def path(name: str) -> str:
    return os.path.join(HERE, f"golden_5jet_{name}.txt")


def write(name: str, pdg, n_final: int, n: int) -> None:
    mom = ps.generate(config(n_final), n)
    t0 = time.time()
    me2 = oracle.OracleProcess(pdg).me2(mom)
    dt = time.time() - t0
    with open(path(name), "w") as f:
        f.write(f"# |M|^2 from the FP64 oracle, {name}, pdg {','.join(map(str, pdg))}\n")
        f.write(f"# host generator: seed {SEED:#x}, n_final {n_final}, sqrt(s) log-uniform [{RS_LO}, {RS_HI}] GeV,"
                " pT > 20, |eta| < 2.5, dR > 0.4, first event 0\n")
        f.write(f"# events {n}; alpha_s 0.118\n")
        for i, v in enumerate(me2):
            f.write(f"{i} {v:.17e}\n")
    print(f"{name}: {n} events in {dt:.0f} s", flush=True)


def read(name: str):
    """(event indices, |M|^2) as lists."""
    idx, val = [], []
    with open(path(name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            a, b = line.split()
            idx.append(int(a))
            val.append(float(b))
    return idx, val


if __name__ == "__main__":
    n_events = int(sys.argv[1]) if len(sys.argv) > 1 else 1024
    for nm, p, nf in SUBPROCESSES:
        write(nm, p, nf, n_events)
