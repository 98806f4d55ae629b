"""Thin ctypes binding of libmea.so (C ABI in include/mea.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of the library.  Device buffers are passed as raw pointers (torch
tensors are accepted and unwrapped with ``data_ptr()``); PyTorch is used only
for device memory and streams.  There is no CPU fallback: if the library is
missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmea.so")
_lock = threading.Lock()
_lib = None

MEA_OK = 0
HEL_SUM_NONZERO, HEL_SUM_ALL, HEL_GIVEN = 0, 1, 2
PREC_FP64, PREC_MIXED = 0, 1
FLAG_REEVALUATED, FLAG_NONFINITE, FLAG_CANCEL = 0x01, 0x02, 0x04

_STATUS = {0: "MEA_OK", -1: "MEA_E_ARG", -2: "MEA_E_UNSUPPORTED", -3: "MEA_E_NOMEM",
           -4: "MEA_E_CUDA", -5: "MEA_E_TIMEOUT", -6: "MEA_E_REJECTED"}


class MeaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("alpha_s", ctypes.c_double), ("flag_threshold", ctypes.c_double),
                ("reeval_fp64", ctypes.c_int), ("colour_mode", ctypes.c_int), ("chunk_events", ctypes.c_int64),
                ("auto_tune", ctypes.c_int), ("kernel_variant", ctypes.c_int), ("helicity_sharing", ctypes.c_int)]


class ProcessInfo(ctypes.Structure):
    _fields_ = [("n_ext", ctypes.c_int), ("n_diagrams", ctypes.c_int), ("n_colour", ctypes.c_int),
                ("n_hel_nonzero", ctypes.c_int), ("n_currents", ctypes.c_int), ("n_ops", ctypes.c_int),
                ("n_slots", ctypes.c_int), ("n_colour_amplitudes", ctypes.c_int),
                ("cf_denominator", ctypes.c_int64), ("cf_max_abs_numerator", ctypes.c_int64),
                ("flops_per_hel", ctypes.c_double), ("colour_flops_per_hel", ctypes.c_double),
                ("flops_per_hel_plain", ctypes.c_double), ("n_colour_entries", ctypes.c_int64),
                ("hs_variants", ctypes.c_int64), ("hs_arena_variants", ctypes.c_int),
                ("hs_flops_per_event", ctypes.c_double), ("hsp_area_variants", ctypes.c_int),
                ("hsp_flops_per_event", ctypes.c_double)]


class TuneResult(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int), ("events_per_cta", ctypes.c_int), ("grid", ctypes.c_int),
                ("colour_amps_in_shared", ctypes.c_int), ("slots_in_shared", ctypes.c_int),
                ("candidates", ctypes.c_int), ("best_ms", ctypes.c_double), ("default_ms", ctypes.c_double),
                ("register_cap", ctypes.c_int), ("vertex_partials", ctypes.c_int), ("helicity_shared", ctypes.c_int),
                ("forwarding", ctypes.c_int)]


class BatchItem(ctypes.Structure):
    _fields_ = [("proc", ctypes.c_void_p), ("momenta_dev", ctypes.c_void_p), ("n_events", ctypes.c_int64),
                ("me2_dev", ctypes.c_void_p), ("flags_dev", ctypes.c_void_p)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("events_completed", ctypes.c_uint64), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("busy_seconds", ctypes.c_double), ("reserved_bytes", ctypes.c_size_t)]


STAGES = ("amplitudes", "colour_amplitudes", "colour_sum", "finish", "reevaluation")


class StageTimes(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 5), ("launches", ctypes.c_int64 * 5)]


class PsConfig(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("n_final", ctypes.c_int), ("rs_lo", ctypes.c_double),
                ("rs_hi", ctypes.c_double), ("pt_min", ctypes.c_double), ("eta_max", ctypes.c_double),
                ("dr_min", ctypes.c_double), ("ptij_min", ctypes.c_double)]


def load(path: str | None = None):
    """Load libmea.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            from . import build as _build
            if path is None:
                path = _build.build()
            if not os.path.exists(path):
                raise MeaError(-2, f"CUDA library not found at {path}")
            lib = ctypes.CDLL(path)
            vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
            lib.mea_create_process.argtypes = [vp, i32, vp, vp]
            lib.mea_create_process_host_only.argtypes = [vp, i32, vp, vp]
            lib.mea_process_info.argtypes = [vp, vp]
            lib.mea_colour_matrix.argtypes = [vp, vp, vp]
            lib.mea_helicities.argtypes = [vp, vp, i32, vp]
            lib.mea_destroy_process.argtypes = [vp]
            lib.mea_check_status.argtypes = [vp, vp]
            lib.mea_probe_bounded_wait.argtypes = [vp, ctypes.c_uint32, vp]
            lib.mea_set_stage_timing.argtypes = [vp, i32]
            lib.mea_measure_alu_peak.argtypes = [i32, ctypes.c_double, vp, vp]
            lib.mea_get_stage_times.argtypes = [vp, vp]
            lib.mea_evaluate.argtypes = [vp, vp, i64, i32, vp, i32, vp, vp, vp]
            lib.mea_evaluate_host.argtypes = [vp, vp, i64, i32, vp, vp]
            lib.mea_evaluate_noalloc.argtypes = [vp, vp, i64, i32, vp, vp, vp]
            lib.mea_generate_phase_space.argtypes = [vp, ctypes.c_uint64, i64, vp, vp, vp]
            lib.mea_partonic_cross_section.argtypes = [vp, ctypes.c_double, vp, ctypes.c_uint64, i64, i32, vp]
            lib.mea_partonic_cross_section_vegas.argtypes = [vp, ctypes.c_double, vp, ctypes.c_uint64, vp, i32, vp]
            lib.mea_autotune.argtypes = [vp, vp, i64, i32, vp, vp]
            lib.mea_batch_create.argtypes = [vp, i32, i32, vp]
            lib.mea_batch_launch.argtypes = [vp, vp]
            lib.mea_batch_info.argtypes = [vp, vp]
            lib.mea_batch_destroy.argtypes = [vp]
            lib.mea_server_create.argtypes = [ctypes.c_size_t, i32, i64, vp]
            lib.mea_server_submit.argtypes = [vp, vp, vp, i64, i32, vp, vp, vp]
            lib.mea_server_wait.argtypes = [vp, ctypes.c_uint64, i32, vp]
            lib.mea_server_stats.argtypes = [vp, vp]
            lib.mea_server_destroy.argtypes = [vp]
            lib.mea_last_error.restype = ctypes.c_char_p
            lib.mea_kernel_launch_count.restype = ctypes.c_uint64
            for name in ("mea_create_process", "mea_create_process_host_only", "mea_process_info",
                         "mea_colour_matrix", "mea_helicities", "mea_destroy_process", "mea_evaluate",
                         "mea_evaluate_host", "mea_evaluate_noalloc", "mea_generate_phase_space",
                         "mea_check_status", "mea_autotune", "mea_batch_create", "mea_batch_launch",
                         "mea_batch_info", "mea_batch_destroy", "mea_server_create", "mea_server_submit",
                         "mea_server_wait", "mea_server_stats", "mea_server_destroy", "mea_set_stage_timing",
                         "mea_get_stage_times", "mea_probe_bounded_wait", "mea_measure_alu_peak", "mea_partonic_cross_section",
                         "mea_partonic_cross_section_vegas"):
                getattr(lib, name).restype = ctypes.c_int
            _lib = lib
    return _lib


def _check(rc):
    if rc != MEA_OK:
        raise MeaError(rc, load().mea_last_error().decode(errors="replace"))


def _ptr(x):
    """Raw address of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    raise TypeError(f"cannot take the address of {type(x)}")


def _check_device_tensor(t, name, dtype, min_numel, device_only=True):
    """Reject (MeaError MEA_E_ARG), before any device access, a torch tensor
    the kernels would misread: wrong dtype, strided, on the host, or too
    small.  Raw addresses (ints) and None pass to the library unchecked."""
    if t is None or isinstance(t, int) or not hasattr(t, "data_ptr"):
        return
    if t.dtype != dtype:
        raise MeaError(-1, f"{name}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise MeaError(-1, f"{name}: must be contiguous")
    if device_only and t.device.type != "cuda":
        raise MeaError(-1, f"{name}: must be a CUDA tensor")
    if t.numel() < min_numel:
        raise MeaError(-1, f"{name}: {t.numel()} elements, need at least {min_numel}")


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return ctypes.c_void_p(s.cuda_stream)
    return ctypes.c_void_p(int(s))


def kernel_launch_count() -> int:
    return int(load().mea_kernel_launch_count())


def measure_alu_peak(fp64=False, seconds=0.2):
    """(TFLOP/s, ms) of an FMA-chain kernel on the current device
    (mea_measure_alu_peak): the measured FP32 or FP64 pipe peak."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(load().mea_measure_alu_peak(1 if fp64 else 0, ctypes.c_double(seconds), ctypes.byref(tf), ctypes.byref(ms)))
    return tf.value, ms.value


class Process:
    """A partonic process on the current CUDA device, e.g. ``Process([21]*5)``.

    pdg: PDG codes (two incoming, then outgoing): 21 gluon, 1..5 quarks,
    negative for antiquarks.  host_only builds the tables without a GPU.
    """

    def __init__(self, pdg, alpha_s=0.118, flag_threshold=1e-5, reeval_fp64=True,
                 colour_mode=0, host_only=False, chunk_events=0, auto_tune=True, kernel_variant=0,
                 helicity_sharing=0):
        lib = load()
        self.pdg = list(pdg)
        self.n_ext = len(self.pdg)
        arr = (ctypes.c_int * self.n_ext)(*self.pdg)
        opts = Options(alpha_s, flag_threshold, 1 if reeval_fp64 else 0, colour_mode, chunk_events,
                       1 if auto_tune else 0, kernel_variant, helicity_sharing)
        h = ctypes.c_void_p()
        fn = lib.mea_create_process_host_only if host_only else lib.mea_create_process
        _check(fn(arr, self.n_ext, ctypes.byref(opts), ctypes.byref(h)))
        self._h = h
        info = ProcessInfo()
        _check(lib.mea_process_info(self._h, ctypes.byref(info)))
        self.info = {k: getattr(info, k) for k, _ in ProcessInfo._fields_}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().mea_destroy_process(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_colour(self):
        return self.info["n_colour"]

    def colour_matrix_exact(self):
        m = self.n_colour
        num = np.zeros((m, m), dtype=np.int64)
        den = ctypes.c_int64()
        _check(load().mea_colour_matrix(self._h, _ptr(num), ctypes.byref(den)))
        return num, int(den.value)

    def helicities(self):
        n = ctypes.c_int()
        _check(load().mea_helicities(self._h, None, 0, ctypes.byref(n)))
        out = np.zeros((n.value, self.n_ext), dtype=np.int8)
        _check(load().mea_helicities(self._h, _ptr(out), n.value, ctypes.byref(n)))
        return out

    def evaluate(self, momenta, me2, n_events=None, hel_mode=HEL_SUM_NONZERO, hel=None,
                 precision=PREC_MIXED, flags=None, stream=None):
        """Enqueue |M|^2 of device momenta [N, n_ext, 4] (float64) into device me2 [N]."""
        if n_events is None:
            n_events = int(momenta.shape[0])
        self._check_args(momenta, me2, n_events, flags, hel if hel_mode == HEL_GIVEN else None)
        _check(load().mea_evaluate(self._h, _ptr(momenta), n_events, hel_mode, _ptr(hel), precision,
                                   _ptr(me2), _ptr(flags), _stream(stream)))

    def _check_args(self, momenta, me2, n_events, flags=None, hel=None):
        import torch
        _check_device_tensor(momenta, "momenta", torch.float64, n_events * self.n_ext * 4)
        _check_device_tensor(me2, "me2", torch.float64, n_events)
        _check_device_tensor(flags, "flags", torch.uint8, n_events)
        _check_device_tensor(hel, "hel", torch.int8, n_events * self.n_ext)

    def autotune(self, momenta, scratch_me2, n_sample=None, precision=PREC_MIXED):
        """Time the candidate tile shapes on a device sample and keep the fastest."""
        if n_sample is None:
            n_sample = int(momenta.shape[0])
        self._check_args(momenta, scratch_me2, n_sample)
        r = TuneResult()
        _check(load().mea_autotune(self._h, _ptr(momenta), n_sample, precision, _ptr(scratch_me2),
                                   ctypes.byref(r)))
        return {k: getattr(r, k) for k, _ in TuneResult._fields_}

    def probe_bounded_wait(self, spin_limit=1000, stream=None):
        """Enqueue the timeout probe (mea_probe_bounded_wait): the next
        check_status raises MeaError(MEA_E_TIMEOUT)."""
        _check(load().mea_probe_bounded_wait(self._h, ctypes.c_uint32(spin_limit), _stream(stream)))

    def set_stage_timing(self, enable=True):
        """Record CUDA events around every stage's kernel launches (mea_set_stage_timing)."""
        _check(load().mea_set_stage_timing(self._h, 1 if enable else 0))

    def stage_times(self):
        """{stage: (milliseconds, launches)} since the previous call (synchronises)."""
        st = StageTimes()
        _check(load().mea_get_stage_times(self._h, ctypes.byref(st)))
        return {name: (st.ms[i], st.launches[i]) for i, name in enumerate(STAGES)}

    def check_status(self, stream=None):
        """Synchronise and raise MeaError(MEA_E_TIMEOUT) if a bounded device wait expired."""
        _check(load().mea_check_status(self._h, _stream(stream)))

    def evaluate_noalloc(self, momenta, me2, n_events=None, precision=PREC_MIXED, flags=None, stream=None):
        """mea_evaluate_noalloc: same result as evaluate() with the helicity sum,
        using only the library's fixed device scratch array (no allocation)."""
        if n_events is None:
            n_events = int(momenta.shape[0])
        self._check_args(momenta, me2, n_events, flags)
        _check(load().mea_evaluate_noalloc(self._h, _ptr(momenta), n_events, precision, _ptr(me2),
                                           _ptr(flags), _stream(stream)))

    def partonic_cross_section(self, sqrt_s, n_events, seed=0x09095257, first_event=0, pt_min=20.0,
                               eta_max=2.5, dr_min=0.4, precision=PREC_FP64, ptij_min=0.0):
        """sigma_hat at fixed sqrt(s_hat) in pb with its statistical error
        (mea_partonic_cross_section): generator events first_event .. + n_events.
        ptij_min > 0 adds the paper's relative-pT cut min(pT_i, pT_j) Delta R_ij."""
        cfg = PsConfig(seed, self.n_ext - 2, sqrt_s, sqrt_s, pt_min, eta_max, dr_min, ptij_min)
        r = XsecResult()
        _check(load().mea_partonic_cross_section(self._h, ctypes.c_double(sqrt_s), ctypes.byref(cfg),
                                                 ctypes.c_uint64(first_event), n_events, precision,
                                                 ctypes.byref(r)))
        return {k: getattr(r, k) for k, _ in XsecResult._fields_}

    def partonic_cross_section_vegas(self, sqrt_s, iterations, points_per_iteration, bins=32, alpha=1.5,
                                     seed=0x09095257, first_event=0, pt_min=20.0, eta_max=2.5, dr_min=0.4,
                                     ptij_min=0.0, precision=PREC_FP64):
        """sigma_hat at fixed sqrt(s_hat) in pb by VEGAS over RAMBO's uniforms
        (mea_partonic_cross_section_vegas)."""
        cfg = PsConfig(seed, self.n_ext - 2, sqrt_s, sqrt_s, pt_min, eta_max, dr_min, ptij_min)
        vc = VegasConfig(iterations, points_per_iteration, bins, alpha)
        r = VegasResult()
        _check(load().mea_partonic_cross_section_vegas(self._h, ctypes.c_double(sqrt_s), ctypes.byref(cfg),
                                                       ctypes.c_uint64(first_event), ctypes.byref(vc), precision,
                                                       ctypes.byref(r)))
        return {k: getattr(r, k) for k, _ in VegasResult._fields_}

    def evaluate_host(self, momenta: np.ndarray, precision=PREC_MIXED, with_flags=False, out=None, flags=None):
        """|M|^2 of host momenta through the library's pipelined copies.

        out / flags: optional host arrays (float64[n] / uint8[n]) to fill; page-locked
        arrays (e.g. from a pinned torch tensor) are copied to and from the device
        directly, pageable ones through the library's staging buffers."""
        mom = np.ascontiguousarray(momenta, dtype=np.float64)
        n = mom.shape[0]
        if out is None:
            out = np.zeros(n, dtype=np.float64)
        if out.dtype != np.float64 or out.shape != (n,) or not out.flags.c_contiguous:
            raise ValueError("out must be a contiguous float64 array of n_events")
        fl = flags
        if fl is None and with_flags:
            fl = np.zeros(n, dtype=np.uint8)
        if fl is not None and (fl.dtype != np.uint8 or fl.shape != (n,) or not fl.flags.c_contiguous):
            raise ValueError("flags must be a contiguous uint8 array of n_events")
        with_flags = with_flags or flags is not None
        _check(load().mea_evaluate_host(self._h, _ptr(mom), n, precision, _ptr(out), _ptr(fl)))
        return (out, fl) if with_flags else out


def generate_phase_space(n_final, n, momenta, first_event=0, seed=0x09095257, rs_lo=200.0,
                         rs_hi=2000.0, pt_min=20.0, eta_max=2.5, dr_min=0.4, attempts=None,
                         stream=None, ptij_min=0.0):
    cfg = PsConfig(seed, n_final, rs_lo, rs_hi, pt_min, eta_max, dr_min, ptij_min)
    _check(load().mea_generate_phase_space(ctypes.byref(cfg), first_event, n, _ptr(momenta),
                                           _ptr(attempts), _stream(stream)))


class VegasConfig(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("points_per_iteration", ctypes.c_int64), ("bins", ctypes.c_int),
                ("alpha", ctypes.c_double)]


class VegasResult(ctypes.Structure):
    _fields_ = [("sigma_pb", ctypes.c_double), ("error_pb", ctypes.c_double), ("chi2_per_dof", ctypes.c_double),
                ("last_sigma_pb", ctypes.c_double), ("last_error_pb", ctypes.c_double),
                ("n_points", ctypes.c_int64), ("n_accepted", ctypes.c_int64)]


class XsecResult(ctypes.Structure):
    _fields_ = [("sigma_pb", ctypes.c_double), ("error_pb", ctypes.c_double), ("n_accepted", ctypes.c_int64),
                ("n_drawn", ctypes.c_int64), ("phase_space", ctypes.c_double), ("symmetry", ctypes.c_double)]


class Batch:
    """Several subprocesses evaluated by one CUDA-graph launch.

    items: list of (Process, momenta_dev, me2_dev, flags_dev or None) with
    device tensors; the graph is captured at construction and replayed by
    launch()."""

    def __init__(self, items, precision=PREC_MIXED):
        lib = load()
        self._keep = items
        arr = (BatchItem * len(items))()
        for i, (proc, mom, me2, flags) in enumerate(items):
            arr[i] = BatchItem(proc._h.value, _ptr(mom).value, int(mom.shape[0]), _ptr(me2).value,
                               _ptr(flags).value if flags is not None else None)
        h = ctypes.c_void_p()
        _check(lib.mea_batch_create(arr, len(items), precision, ctypes.byref(h)))
        self._h = h
        n = ctypes.c_int()
        _check(lib.mea_batch_info(self._h, ctypes.byref(n)))
        self.kernel_nodes = n.value

    def launch(self, stream=None):
        _check(load().mea_batch_launch(self._h, _stream(stream)))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().mea_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop (mea_server_*): requests of any
    process are split into chunks of similar device cost, dispatched to
    n_slots streams shortest remaining work first (with aging), admitted by
    a scratch-memory budget committed per process."""

    def __init__(self, mem_budget_bytes=4 << 30, n_slots=4, chunk_events=1 << 14):
        h = ctypes.c_void_p()
        _check(load().mea_server_create(mem_budget_bytes, n_slots, chunk_events, ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def submit(self, proc, momenta, me2, flags=None, precision=PREC_MIXED, n_events=None):
        if n_events is None:
            n_events = int(momenta.shape[0])
        rid = ctypes.c_uint64()
        _check(load().mea_server_submit(self._h, proc._h, _ptr(momenta), n_events, precision, _ptr(me2),
                                        _ptr(flags), ctypes.byref(rid)))
        self._keep[rid.value] = (proc, momenta, me2, flags)
        return rid.value

    def wait(self, req_id, timeout_ms=-1):
        """Returns the request latency in ms; raises MeaError (e.g. MEA_E_TIMEOUT)."""
        lat = ctypes.c_double()
        rc = load().mea_server_wait(self._h, req_id, timeout_ms, ctypes.byref(lat))
        if rc != -5:
            self._keep.pop(req_id, None)
        _check(rc)
        return lat.value

    def stats(self):
        st = ServerStats()
        _check(load().mea_server_stats(self._h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().mea_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
