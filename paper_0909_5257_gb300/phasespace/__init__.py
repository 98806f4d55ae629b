"""Seeded synthetic phase-space generator (input generator only).

Host side of ``phasespace.h``: Philox4x32-10 counters -> sqrt(s_hat)
log-uniform -> RAMBO flat massless n-body momenta in the partonic
centre-of-mass frame -> jet cuts (pT, |eta|, Delta R), redrawing a rejected
point with the next attempt counter.  The CUDA path compiles the same header
into its device generator, so both sides draw identical integer streams.
This module holds no matrix-element arithmetic.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "phasespace_host.c")
_HDR = os.path.join(_HERE, "phasespace.h")
_LIB_PATH = os.path.join(_HERE, "libphasespace.so")
_lock = threading.Lock()
_lib = None

# Seed base of the synthetic workloads; workload k uses SEED_BASE + k.
SEED_BASE = 0x09095257


class _Cfg(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("n_final", ctypes.c_int),
                ("rs_lo", ctypes.c_double), ("rs_hi", ctypes.c_double),
                ("pt_min", ctypes.c_double), ("eta_max", ctypes.c_double),
                ("dr_min", ctypes.c_double), ("ptij_min", ctypes.c_double)]


@dataclass(frozen=True)
class PhaseSpaceConfig:
    """Synthetic partonic workload: n_final massless partons, sqrt(s_hat) in
    [rs_lo, rs_hi] GeV log-uniform, cuts pT > pt_min, |eta| < eta_max,
    Delta R > dr_min and, if ptij_min > 0, min(pT_i, pT_j) Delta R_ij > ptij_min."""
    n_final: int
    rs_lo: float = 200.0
    rs_hi: float = 2000.0
    seed: int = SEED_BASE
    pt_min: float = 20.0
    eta_max: float = 2.5
    dr_min: float = 0.4
    ptij_min: float = 0.0

    def as_c(self) -> _Cfg:
        return _Cfg(self.seed, self.n_final, self.rs_lo, self.rs_hi,
                    self.pt_min, self.eta_max, self.dr_min, self.ptij_min)


def build(force: bool = False) -> str:
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.ps_generate_host.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_uint64,
                                             ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
            lib.ps_generate_host.restype = ctypes.c_int
            lib.ps_philox_host.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.ps_vegas_host.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64,
                                          ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.ps_vegas_host.restype = ctypes.c_int
            _lib = lib
    return _lib


def generate(cfg: PhaseSpaceConfig, n_events: int, first_event: int = 0,
             return_attempts: bool = False):
    """Momenta [n_events, 2 + n_final, 4] float64 (E, px, py, pz) in GeV."""
    lib = _load()
    out = np.zeros((n_events, 2 + cfg.n_final, 4), dtype=np.float64)
    att = np.zeros(n_events, dtype=np.int32)
    c = cfg.as_c()
    rc = lib.ps_generate_host(ctypes.byref(c), first_event, n_events,
                              out.ctypes.data, att.ctypes.data)
    if rc != 0:
        raise ValueError("phase-space generator rejected its configuration")
    return (out, att) if return_attempts else out


def vegas_points(cfg: PhaseSpaceConfig, edges: np.ndarray, first_event: int, n_events: int):
    """VEGAS points at sqrt(s_hat) = cfg.rs_lo (ps_vegas_event): momenta
    [n, 2 + n_final, 4], weights [n] (0 where the cuts reject), bins
    [n, dims] uint8.  edges: [dims, nb + 1] float64."""
    lib = _load()
    e = np.ascontiguousarray(edges, dtype=np.float64)
    nb = e.shape[1] - 1
    out = np.zeros((n_events, 2 + cfg.n_final, 4), dtype=np.float64)
    w = np.zeros(n_events, dtype=np.float64)
    b = np.zeros((n_events, e.shape[0]), dtype=np.uint8)
    c = cfg.as_c()
    rc = lib.ps_vegas_host(ctypes.byref(c), e.ctypes.data, nb, ctypes.c_uint64(first_event), ctypes.c_int64(n_events),
                           out.ctypes.data, w.ctypes.data, b.ctypes.data)
    if rc != 0:
        raise ValueError("VEGAS point generator rejected its configuration")
    return out, w, b


def rambo_dims(n_final: int) -> int:
    return 2 if n_final == 2 else 4 * n_final


def philox4x32_10(ctr, key):
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib.ps_philox_host(c, k, o)
    return [int(x) for x in o]
