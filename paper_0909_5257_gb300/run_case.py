"""Evaluate one subprocess on synthetic events, for profiling.

    python -m paper_0909_5257_gb300.run_case PROCESS N [mixed|fp64]

PROCESS is one of the names below (the workloads' subprocesses); N events are
generated on the device (RAMBO with the workload's sqrt(s) range and cuts),
evaluated once (tuning on first use when N >= 2^16), then evaluated again
inside an NVTX range "eval" -- the range a profiler restricts itself to
(ncu --nvtx --nvtx-include "eval/").  Prints the process name, N and the mean
|M|^2.
"""
import sys

import torch

from . import mea

PROCESSES = {
    "gg3g": ([21] * 5, 200.0, 2000.0),
    "uu3g": ([2, -2, 21, 21, 21], 200.0, 2000.0),
    "uuuug": ([2, 2, 2, 2, 21], 200.0, 2000.0),
    "gg4g": ([21] * 6, 300.0, 3000.0),
    "uu4g": ([2, -2, 21, 21, 21, 21], 300.0, 3000.0),
    "uuuu3g": ([2, 2, 2, 2, 21, 21, 21], 500.0, 5000.0),
    "uu5g": ([2, -2] + [21] * 5, 500.0, 5000.0),
    "gg5g": ([21] * 7, 500.0, 5000.0),
}


def main(argv):
    if len(argv) < 3 or argv[1] not in PROCESSES:
        print(__doc__)
        print("processes:", " ".join(PROCESSES))
        return 2
    name, n = argv[1], int(argv[2])
    prec = mea.PREC_FP64 if len(argv) > 3 and argv[3] == "fp64" else mea.PREC_MIXED
    pdg, lo, hi = PROCESSES[name]
    torch.cuda.set_device(0)
    P = mea.Process(pdg)
    mom = torch.empty((n, len(pdg), 4), dtype=torch.float64, device="cuda")
    mea.generate_phase_space(len(pdg) - 2, n, mom, rs_lo=lo, rs_hi=hi)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    P.evaluate(mom, out, precision=prec)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("eval")
    P.evaluate(mom, out, precision=prec)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    P.check_status()
    print(name, n, float(out.mean()))
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
