"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Python handle on ``qcd_oracle.cpp``: helicity-summed, colour-summed tree-level
|M|^2 for massless QCD evaluated diagram by diagram from the Feynman rules of
Hagiwara et al. (arXiv:0909.5257), Sec. 2.1 and Sec. 4.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package; the product path never does.  It shares no code with the CUDA
path.

Parity status of each function is pinned by the CPU tests in
``tests/test_oracle_*.py`` (closed forms, Parke-Taylor, Berends-Giele, Ward
identities, helicity zeros, Lorentz invariance, exact scaling, Table 1 and
Table 5 counts, a Gell-Mann brute force of the colour matrix).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qcd_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain g++, OpenMP, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB_PATH) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared",
               "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _configure(lib):
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p
    lib.oq_create.restype = vp
    lib.oq_create.argtypes = [ctypes.POINTER(ctypes.c_int), i32, ctypes.c_double]
    lib.oq_destroy.argtypes = [vp]
    lib.oq_last_error.restype = ctypes.c_char_p
    lib.oq_info.argtypes = [vp, dp, dp, dp]
    lib.oq_me2.argtypes = [vp, dp, i64, dp, dp, i32]
    lib.oq_jamp.argtypes = [vp, dp, i32, i32, dp]
    lib.oq_colour_matrix.argtypes = [vp, dp]
    lib.oq_colour_matrix_exact.argtypes = [vp, dp, dp, dp, dp]
    lib.oq_basis.argtypes = [vp, i32, dp, i32]
    lib.oq_diagram_colour.argtypes = [vp, i32, dp, dp, dp, i32]
    lib.oq_max_threads.restype = i32
    return lib


def build_variant(path: str, mutation: int) -> str:
    """Compile a copy of the oracle with test mutation `mutation` planted
    (OQ_MUTATION, see qcd_oracle.cpp) into `path`; tests only."""
    cmd = ["g++", "-O1", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", f"-DOQ_MUTATION={int(mutation)}", "-o", path, _SRC]
    subprocess.check_call(cmd)
    return path


def load_variant(path: str):
    """ctypes handle of a library built by build_variant, for OracleProcess(lib=...)."""
    return _configure(ctypes.CDLL(path))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            _configure(lib)
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().oq_max_threads())


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


class OracleProcess:
    """One partonic process, e.g. ``OracleProcess([21, 21, 21, 21])`` for gg -> gg.

    ``pdg``: PDG codes, two incoming then the outgoing partons
    (21 gluon, 2 u, -2 u-bar).
    """

    def __init__(self, pdg, alpha_s: float = 0.118, lib=None):
        lib = lib if lib is not None else _load()
        self._lib = lib
        self.pdg = list(pdg)
        self.n_ext = len(self.pdg)
        self.alpha_s = alpha_s
        arr = (ctypes.c_int * self.n_ext)(*self.pdg)
        h = lib.oq_create(arr, self.n_ext, alpha_s)
        if not h:
            raise RuntimeError("oracle: " + lib.oq_last_error().decode())
        self._h = ctypes.c_void_p(h)
        nd, nc, nt = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        lib.oq_info(self._h, ctypes.byref(nd), ctypes.byref(nc), ctypes.byref(nt))
        self.n_diagrams, self.n_colour, self.n_topologies = nd.value, nc.value, nt.value

    def __del__(self):
        try:
            if getattr(self, "_h", None):
                self._lib.oq_destroy(self._h)
        except Exception:
            pass

    def me2(self, momenta, per_helicity: bool = False, threads: int = 0):
        """|M|^2 averaged over initial helicities and colours, summed over the rest.

        momenta: [N, n_ext, 4] float64 (E, px, py, pz).  With per_helicity, also
        returns [N, 2**n_ext] colour-summed-and-averaged values per helicity
        combination (before the 1/4), indexed as in the module docstring of
        qcd_oracle.cpp.
        """
        mom = np.ascontiguousarray(momenta, dtype=np.float64)
        assert mom.ndim == 3 and mom.shape[1] == self.n_ext and mom.shape[2] == 4
        n = mom.shape[0]
        out = np.zeros(n, dtype=np.float64)
        hel = np.zeros((n, 1 << self.n_ext), dtype=np.float64) if per_helicity else None
        rc = self._lib.oq_me2(self._h, _ptr(mom), n, _ptr(out),
                            _ptr(hel) if hel is not None else None, threads)
        if rc != 0:
            raise RuntimeError("oracle: " + self._lib.oq_last_error().decode())
        return (out, hel) if per_helicity else out

    def jamp(self, momenta_one, hel: int, ward_leg: int = -1) -> np.ndarray:
        """Colour amplitudes J_alpha (complex [n_colour]) for one event and helicity."""
        mom = np.ascontiguousarray(momenta_one, dtype=np.float64).reshape(self.n_ext, 4)
        out = np.zeros(2 * self.n_colour, dtype=np.float64)
        rc = self._lib.oq_jamp(self._h, _ptr(mom), hel, ward_leg, _ptr(out))
        if rc != 0:
            raise RuntimeError("oracle: " + self._lib.oq_last_error().decode())
        return out[0::2] + 1j * out[1::2]

    def colour_matrix(self) -> np.ndarray:
        m = self.n_colour
        out = np.zeros((m, m), dtype=np.float64)
        self._lib.oq_colour_matrix(self._h, _ptr(out))
        return out

    def colour_matrix_exact(self):
        """Exact colour matrix as a list of lists of fractions.Fraction (real parts)
        plus the imaginary parts, which must vanish."""
        from fractions import Fraction
        m = self.n_colour
        arrs = [np.zeros((m, m), dtype=np.int64) for _ in range(4)]
        self._lib.oq_colour_matrix_exact(self._h, *[_ptr(a) for a in arrs])
        re = [[Fraction(int(arrs[0][i, j]), int(arrs[1][i, j])) for j in range(m)] for i in range(m)]
        im = [[Fraction(int(arrs[2][i, j]), int(arrs[3][i, j])) for j in range(m)] for i in range(m)]
        return re, im

    def basis(self, alpha: int):
        """Basis element alpha: list of (closed, row, col, gluon_legs)."""
        buf = np.zeros(256, dtype=np.int32)
        n = self._lib.oq_basis(self._h, alpha, _ptr(buf), 256)
        if n < 0:
            raise IndexError(alpha)
        out, i = [], 0
        while i < n:
            ln = int(buf[i]); i += 1
            closed, row, col = bool(buf[i] == 1), int(buf[i + 1]), int(buf[i + 2])
            gl = [int(x) for x in buf[i + 3:i + ln]]
            out.append((closed, row, col, gl))
            i += ln
        return out

    def diagram_colour(self, d: int):
        cap = 4096
        a = np.zeros(cap, dtype=np.int32)
        re = np.zeros(cap)
        im = np.zeros(cap)
        n = self._lib.oq_diagram_colour(self._h, d, _ptr(a), _ptr(re), _ptr(im), cap)
        n = min(n, cap)
        return [(int(a[i]), complex(re[i], im[i])) for i in range(n)]
