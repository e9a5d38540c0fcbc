"""Thin Python binding of the C ABI in include/ht.h (argument marshalling only).

Every step of the Hough Transform runs in the CUDA library libht_gb300.so;
this module only converts numpy arrays / torch tensors into pointers and
sizes.  It raises if the library has not been built: there is no CPU
fallback.  Names follow the C ABI (ht_create -> Context, ht_fill -> fill,
ht_find_maxima -> find_maxima, ...).
"""
from __future__ import annotations

import ctypes
import json
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libht_gb300.so")

HT_OK, HT_PENDING, HT_TRUNCATED = 0, 1, 2
HT_E_INVAL, HT_E_NOMEM, HT_E_CUDA, HT_E_BUSY, HT_E_TIMEOUT, HT_E_STATE = -1, -2, -3, -4, -5, -6
HT_MEM_HOST, HT_MEM_DEVICE, HT_ACCUMULATE, HT_FILL_NAIVE, HT_PEAKS_ONLY, HT_MAXIMA_4D = 0, 1, 2, 4, 8, 16
STATUS_NAMES = {0: "HT_OK", 1: "HT_PENDING", 2: "HT_TRUNCATED", -1: "HT_E_INVAL", -2: "HT_E_NOMEM",
                -3: "HT_E_CUDA", -4: "HT_E_BUSY", -5: "HT_E_TIMEOUT", -6: "HT_E_STATE"}


class HTError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class c_binning(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in ("n_theta", "n_phi", "n_a", "n_b", "win_theta", "win_phi")]


class c_ranges(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in ("theta_min", "theta_max", "phi_min", "phi_max",
                                              "a_min", "a_max", "b_min", "b_max")]


TUNING_FIELDS = ("fill_rows", "fill_threads", "fill_hits_staged", "fill_blocks_per_sm",
                 "scan_kind", "scan_stage_bytes", "scan_slots", "scan_blocks_per_sm", "fill_fused_scan",
                 "fill_vote_agg", "bin_cluster")
HT_SCAN_AUTO, HT_SCAN_BULK, HT_SCAN_STREAM, HT_SCAN_DIRECT = 0, 1, 2, 3


class c_tuning(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in TUNING_FIELDS]


class c_server_cfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("n_streams", ctypes.c_uint32),
                ("max_batch", ctypes.c_uint32), ("max_hits_per_event", ctypes.c_uint32),
                ("queue_depth", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("fill_blocks_per_sm", ctypes.c_uint32)]


class c_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("waiting", ctypes.c_uint64),
                ("in_flight", ctypes.c_uint64), ("micro_batches", ctypes.c_uint64), ("mean_batch", ctypes.c_double),
                ("lanes", ctypes.c_uint32), ("lane_bytes", ctypes.c_uint64), ("p50_us", ctypes.c_double),
                ("p99_us", ctypes.c_double), ("mean_us", ctypes.c_double), ("max_us", ctypes.c_double)]


class c_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double)]


PEAK_DTYPE = np.dtype([("itheta", np.uint32), ("iphi", np.uint32), ("ia", np.uint32),
                       ("ib", np.uint32), ("votes", np.uint32), ("a_c", np.float32),
                       ("b_c", np.float32), ("event", np.uint32)])
assert PEAK_DTYPE.itemsize == 32

TRACK_DTYPE = np.dtype([("a", np.float64), ("b", np.float64), ("rho", np.float64), ("varphi", np.float64),
                        ("pt", np.float64), ("theta", np.float64), ("eta", np.float64), ("phi_c", np.float64),
                        ("votes", np.uint32), ("event", np.uint32)])
assert TRACK_DTYPE.itemsize == 72


@dataclass(frozen=True)
class Binning:
    n_theta: int
    n_phi: int
    n_a: int
    n_b: int
    win_theta: int = 0
    win_phi: int = 0

    @property
    def n_slices(self) -> int:
        return self.n_theta * self.n_phi

    @property
    def n_cells(self) -> int:
        return self.n_theta * self.n_phi * self.n_a * self.n_b

    def shape(self):
        return (self.n_theta, self.n_phi, self.n_a, self.n_b)

    def c(self) -> c_binning:
        return c_binning(self.n_theta, self.n_phi, self.n_a, self.n_b, self.win_theta, self.win_phi)


@dataclass(frozen=True)
class Ranges:
    theta_min: float = 0.0
    theta_max: float = float(np.float32(np.pi))
    phi_min: float = float(np.float32(-np.pi))
    phi_max: float = float(np.float32(np.pi))
    a_min: float = -2000.0
    a_max: float = 2000.0
    b_min: float = -2000.0
    b_max: float = 2000.0

    def c(self) -> c_ranges:
        return c_ranges(self.theta_min, self.theta_max, self.phi_min, self.phi_max,
                        self.a_min, self.a_max, self.b_min, self.b_max)


_lib = None


def lib():
    """Load libht_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    P, U32, U64, I = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    sig = {
        "ht_last_error": ([], ctypes.c_char_p),
        "ht_create": ([ctypes.POINTER(c_binning), ctypes.POINTER(c_ranges), U32, U32, P], I),
        "ht_destroy": ([P], I),
        "ht_fill": ([P, P, P, P, U32, U32, P], I),
        "ht_find_maxima": ([P, P, U32, P, U32, P], I),
        "ht_sync": ([P, P], I),
        "ht_check_wait_timeout": ([P, U32], I),
        "ht_last_admitted": ([P, ctypes.POINTER(ctypes.c_uint64)], I),
        "ht_measure_atomics": ([U64, U32, ctypes.POINTER(ctypes.c_double)], I),
        "ht_copy_matrix": ([P, P, U64, U32, P], I),
        "ht_get_edges": ([P, P, P], I),
        "ht_launch_count": ([P], U64),
        "ht_set_matrix": ([P, P, U64, U32, P], I),
        "ht_validate": ([ctypes.POINTER(c_binning), ctypes.POINTER(c_ranges), U32], I),
        "ht_compute_edges": ([ctypes.POINTER(c_binning), ctypes.POINTER(c_ranges), P, P], I),
        "ht_profile": ([P, I], I),
        "ht_profile_read": ([P, P, U32, P], I),
        "ht_compute_b_thresholds": ([ctypes.POINTER(c_binning), ctypes.POINTER(c_ranges), P], I),
        "ht_set_tuning": ([P, ctypes.POINTER(c_tuning)], I),
        "ht_autotune": ([P, U32, ctypes.POINTER(c_tuning), ctypes.POINTER(ctypes.c_double)], I),
        "ht_get_tuning": ([P, ctypes.POINTER(c_tuning)], I),
        "ht_find_maxima_noalloc": ([ctypes.POINTER(c_binning), ctypes.POINTER(c_ranges), U32, P, U32, P, U32, P, P],
                                   I),
        "ht_batch_create": ([ctypes.POINTER(c_binning), ctypes.POINTER(c_ranges), U32, U32, U32, U32, P], I),
        "ht_batch_destroy": ([P], I),
        "ht_batch_run": ([P, P, P, P, P, U32, U32, P, P, U32, P], I),
        "ht_batch_sync": ([P, P], I),
        "ht_batch_copy_matrix": ([P, U32, P, U64], I),
        "ht_batch_set_tuning": ([P, ctypes.POINTER(c_tuning)], I),
        "ht_batch_get_tuning": ([P, ctypes.POINTER(c_tuning)], I),
        "ht_batch_autotune": ([P, U32, ctypes.POINTER(c_tuning), ctypes.POINTER(ctypes.c_double)], I),
        "ht_batch_profile": ([P, I], I),
        "ht_batch_profile_read": ([P, P, U32, P], I),
        "ht_server_create": ([ctypes.POINTER(c_server_cfg), P], I),
        "ht_server_destroy": ([P], I),
        "ht_submit": ([P, ctypes.POINTER(c_binning), ctypes.POINTER(c_ranges), U32, P, P, P, U32,
                       ctypes.POINTER(ctypes.c_uint64)], I),
        "ht_poll": ([P, ctypes.c_uint64, P, U32, P, U32], I),
        "ht_server_get_stats": ([P, ctypes.POINTER(c_server_stats), I], I),
        "ht_track_params": ([ctypes.POINTER(c_binning), ctypes.POINTER(c_ranges), P, U32, ctypes.c_double, P], I),
        "ht_sectors_create": ([ctypes.POINTER(c_binning), ctypes.POINTER(c_ranges), U32, U32, U32, P], I),
        "ht_sectors_destroy": ([P], I),
        "ht_sectors_fill": ([P, P, P, P, U32, U32, P], I),
        "ht_sectors_find_maxima": ([P, P, U32, P, U32, P], I),
        "ht_sectors_copy_matrix": ([P, U32, P, U64], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes, f.restype = args, res
    _lib = L
    return L


def exported_symbols():
    """Names of the C ABI functions declared in include/ht.h that the library exports."""
    L = lib()
    return [n for n in dir(L) if n.startswith("ht_")]


def validate(binning: Binning, ranges: Ranges = Ranges(), threshold: int = 10) -> int:
    """ht_validate: HT_OK or HT_E_INVAL (host only)."""
    b, r = binning.c(), ranges.c()
    return int(lib().ht_validate(ctypes.byref(b), ctypes.byref(r), threshold))


def compute_edges(binning: Binning, ranges: Ranges = Ranges()):
    """ht_compute_edges: the FP32 pseudo-angle edge tables (host only)."""
    et = np.zeros(binning.n_theta + 1, np.float32)
    ep = np.zeros(binning.n_phi + 1, np.float32)
    b, r = binning.c(), ranges.c()
    check(lib().ht_compute_edges(ctypes.byref(b), ctypes.byref(r), et.ctypes.data_as(ctypes.c_void_p),
                                 ep.ctypes.data_as(ctypes.c_void_p)))
    return et, ep


def compute_b_thresholds(binning: Binning, ranges: Ranges = Ranges()):
    """ht_compute_b_thresholds: the n_b + 1 B-bin thresholds (host only)."""
    beta = np.zeros(binning.n_b + 1, np.float32)
    b, r = binning.c(), ranges.c()
    check(lib().ht_compute_b_thresholds(ctypes.byref(b), ctypes.byref(r), beta.ctypes.data_as(ctypes.c_void_p)))
    return beta


def measure_atomics(footprint_bytes: int, updates_per_thread: int = 64) -> float:
    """ht_measure_atomics: L2 atomic increments per second at random words of
    a footprint_bytes device buffer."""
    r = ctypes.c_double()
    check(lib().ht_measure_atomics(int(footprint_bytes), int(updates_per_thread), ctypes.byref(r)))
    return float(r.value)


def track_params(binning: Binning, ranges: Ranges, peaks, b_field_t: float = 2.0):
    """ht_track_params: rho, varphi, p_T, theta, eta of each peak in FP64
    (host only).  ``peaks`` is an array of PEAK_DTYPE; returns TRACK_DTYPE."""
    pk = np.ascontiguousarray(peaks, dtype=PEAK_DTYPE)
    out = np.zeros(pk.size, TRACK_DTYPE)
    b, r = binning.c(), ranges.c()
    check(lib().ht_track_params(ctypes.byref(b), ctypes.byref(r), pk.ctypes.data_as(ctypes.c_void_p), pk.size,
                                float(b_field_t), out.ctypes.data_as(ctypes.c_void_p)))
    return out


def find_maxima_noalloc(binning: Binning, ranges: Ranges, threshold: int, M, n_events: int, out, capacity: int,
                        counts, stream=None):
    """ht_find_maxima_noalloc: Step 2 on n_events device matrices ``M`` (CUDA
    tensor) into the CUDA tensors ``out`` (>= n_events*capacity*32 bytes) and
    ``counts`` (>= n_events int32), with the library's static scratch."""
    if out.numel() * out.element_size() < n_events * capacity * 32:
        raise ValueError("out is smaller than n_events * capacity * 32 bytes")
    if counts.numel() * counts.element_size() < n_events * 4:
        raise ValueError("counts is smaller than n_events * 4 bytes")
    if M.numel() * M.element_size() < n_events * binning.n_cells * 4:
        raise ValueError("M is smaller than n_events matrices")
    b, r = binning.c(), ranges.c()
    check(lib().ht_find_maxima_noalloc(ctypes.byref(b), ctypes.byref(r), threshold, ctypes.c_void_p(M.data_ptr()),
                                       n_events, ctypes.c_void_p(out.data_ptr()), capacity,
                                       ctypes.c_void_p(counts.data_ptr()), _stream_ptr(stream)))


def last_error() -> str:
    return lib().ht_last_error().decode()


def check(status: int, ok=(HT_OK,)) -> int:
    if status not in ok:
        raise HTError(status, last_error())
    return status


# ---------------------------------------------------------------------------
# Pointer marshalling
# ---------------------------------------------------------------------------

def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


_NP_DTYPES = {np.float32: np.dtype(np.float32), np.uint32: np.dtype(np.uint32), np.int32: np.dtype(np.int32)}
_TORCH_DTYPES = None   # numpy dtype -> the tensor dtypes accepted for it (set on first use)


def _np_address(arr) -> int:
    """Address of a C-contiguous numpy array's data (from its buffer when it
    is writable, the cheap route; else through arr.ctypes)."""
    try:
        return ctypes.addressof(ctypes.c_char.from_buffer(arr)) if arr.size else arr.ctypes.data
    except (TypeError, ValueError):
        return arr.ctypes.data


def _ptr_and_mem(a, dtype):
    """(pointer, HT_MEM_* flag, keepalive) for a numpy array or a torch tensor."""
    if type(a) is np.ndarray and a.dtype == _NP_DTYPES[dtype] and a.flags.c_contiguous:
        return ctypes.c_void_p(_np_address(a)), HT_MEM_HOST, a
    if _is_torch(a):
        global _TORCH_DTYPES
        if _TORCH_DTYPES is None:
            import torch
            _TORCH_DTYPES = {np.float32: (torch.float32,), np.uint32: (torch.int32, torch.uint8),
                             np.int32: (torch.int32,)}
        if a.dtype not in _TORCH_DTYPES[dtype]:
            raise TypeError(f"tensor dtype {a.dtype} does not match {dtype}")
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), (HT_MEM_DEVICE if a.is_cuda else HT_MEM_HOST), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(ctypes.c_void_p), HT_MEM_HOST, arr


def _gpu_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name(torch.cuda.current_device())
    except Exception:
        return "unknown"


_BUILD_ID = None


def _kernel_build_id() -> str:
    """Hash of the library's CUDA and C++ sources: a cached launch shape is
    only reused by the kernels it was timed with."""
    global _BUILD_ID
    if _BUILD_ID is None:
        import hashlib
        h = hashlib.sha256()
        csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc")
        for f in sorted(os.listdir(csrc)):
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(f.encode() + b"\0" + fh.read())
        _BUILD_ID = h.hexdigest()[:12]
    return _BUILD_ID


def _tuning_key(kind: str, binning: Binning, ranges: Ranges, threshold: int, sizes: str) -> str:
    """Key of a cached launch-shape choice: GPU name, kernel sources, object
    kind, binning, ranges, threshold and sizes."""
    b, r = binning, ranges
    return (f"{_gpu_name()}|k{_kernel_build_id()}|{kind}|{b.n_theta}x{b.n_phi}x{b.n_a}x{b.n_b}+{b.win_theta},{b.win_phi}|"
            f"{r.theta_min},{r.theta_max},{r.phi_min},{r.phi_max},{r.a_min},{r.a_max},{r.b_min},{r.b_max}|"
            f"T{threshold}|{sizes}")


def _load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def _cached_autotune(path, key: str, run, apply):
    """Launch shapes from the JSON cache at `path` (None: $HT_TUNING_CACHE,
    unset: no cache).  A hit applies the stored shapes without timing; a miss
    times them (run() -> (tuning, us)) and stores the choice.  A stored shape
    the library refuses (apply raises HTError) counts as a miss."""
    path = path if path is not None else os.environ.get("HT_TUNING_CACHE")
    if path:
        hit = _load_cache(path).get(key)
        if isinstance(hit, dict) and isinstance(hit.get("tuning"), dict) and set(hit["tuning"]) <= set(TUNING_FIELDS):
            tun = {n: int(v) for n, v in hit["tuning"].items()}
            try:
                apply(tun)
                return tun, float(hit.get("us_per_event", 0.0))
            except HTError:
                pass
    tun, us = run()
    if path:
        d = _load_cache(path)
        d[key] = {"tuning": tun, "us_per_event": us}
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    return tun, us


class Context:
    """One event at a time (ht_create / ht_fill / ht_find_maxima).  A context
    owns its stream, staging, M_H and counters, so several contexts fed
    round-robin, each on its own stream, keep several events in flight."""

    def __init__(self, binning: Binning, ranges: Ranges = Ranges(), threshold: int = 10,
                 max_hits: int = 65536):
        self.binning, self.ranges, self.threshold, self.max_hits = binning, ranges, threshold, max_hits
        self._h = ctypes.c_void_p()
        b, r = binning.c(), ranges.c()
        check(lib().ht_create(ctypes.byref(b), ctypes.byref(r), threshold, max_hits, ctypes.byref(self._h)))

    def close(self):
        if self._h:
            lib().ht_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def launches(self) -> int:
        return int(lib().ht_launch_count(self._h))

    def set_tuning(self, **kw):
        """ht_set_tuning: launch-shape knobs (see ht_tuning); unspecified = automatic."""
        t = c_tuning(*[int(kw.pop(n, 0)) for n in TUNING_FIELDS])
        if kw:
            raise TypeError(f"unknown tuning fields {sorted(kw)}")
        check(lib().ht_set_tuning(self._h, ctypes.byref(t)))

    def autotune(self, reps: int = 5, cache: str | None = None):
        """ht_autotune: time launch shapes on the last fill's hits and keep the
        fastest.  Returns (chosen tuning dict, microseconds per event).
        cache: a JSON file of earlier choices keyed by (GPU name, binning,
        ranges, threshold, max_hits) -- a hit applies the stored shapes
        without timing (default $HT_TUNING_CACHE; unset: no cache)."""
        def run():
            t, us = c_tuning(), ctypes.c_double()
            check(lib().ht_autotune(self._h, reps, ctypes.byref(t), ctypes.byref(us)))
            return {n: int(getattr(t, n)) for n in TUNING_FIELDS}, float(us.value)
        key = _tuning_key("context", self.binning, self.ranges, self.threshold, f"H{self.max_hits}")
        return _cached_autotune(cache, key, run, lambda t: self.set_tuning(**t))

    def get_tuning(self) -> dict:
        t = c_tuning()
        check(lib().ht_get_tuning(self._h, ctypes.byref(t)))
        return {n: int(getattr(t, n)) for n in TUNING_FIELDS}

    def profile(self, enable: bool = True):
        """ht_profile: start (resetting totals) or stop per-kernel event timing."""
        check(lib().ht_profile(self._h, 1 if enable else 0))

    def profile_read(self) -> dict:
        """ht_profile_read: {kernel: (launches, total_ms)} (synchronises)."""
        arr = (c_kernel_time * 16)()
        n = ctypes.c_uint32()
        check(lib().ht_profile_read(self._h, ctypes.cast(arr, ctypes.c_void_p), 16, ctypes.byref(n)))
        return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms))
                for i in range(min(n.value, 16))}

    def fill(self, x, y, z, accumulate: bool = False, naive: bool = False, peaks_only: bool = False, stream=None):
        n = int(x.numel() if _is_torch(x) else np.asarray(x).size)
        px, mx, kx = _ptr_and_mem(x, np.float32)
        py, my, ky = _ptr_and_mem(y, np.float32)
        pz, mz, kz = _ptr_and_mem(z, np.float32)
        if not (mx == my == mz):
            raise ValueError("x, y, z must all be host or all be device arrays")
        flags = (mx | (HT_ACCUMULATE if accumulate else 0) | (HT_FILL_NAIVE if naive else 0) |
                 (HT_PEAKS_ONLY if peaks_only else 0))
        check(lib().ht_fill(self._h, px, py, pz, n, flags, _stream_ptr(stream)))
        self._keep = (kx, ky, kz)

    def find_maxima(self, capacity: int = 1 << 16, out=None, count=None, stream=None, four_d: bool = False):
        """Host mode (out is None): returns (peaks structured array, total).
        Device mode: ``out`` is a CUDA tensor of >= capacity*32 bytes and
        ``count`` a CUDA int32 tensor; the call only enqueues.  four_d: the
        80-neighbour rule (HT_MAXIMA_4D)."""
        L = lib()
        f4 = HT_MAXIMA_4D if four_d else 0
        if out is not None:
            if out.numel() * out.element_size() < capacity * 32:
                raise ValueError("out is smaller than capacity * 32 bytes")
            check(L.ht_find_maxima(self._h, ctypes.c_void_p(out.data_ptr()), capacity,
                                   ctypes.c_void_p(count.data_ptr()), HT_MEM_DEVICE | f4, _stream_ptr(stream)))
            return None
        buf = np.empty(max(capacity, 1), PEAK_DTYPE)   # the call writes the first min(total, capacity)
        n = ctypes.c_uint32()
        check(L.ht_find_maxima(self._h, buf.ctypes.data_as(ctypes.c_void_p), capacity, ctypes.byref(n),
                               HT_MEM_HOST | f4, _stream_ptr(stream)), ok=(HT_OK, HT_TRUNCATED))
        return buf[: min(n.value, capacity)].copy(), int(n.value)

    def sync(self, stream=None):
        check(lib().ht_sync(self._h, _stream_ptr(stream)))

    def last_admitted(self) -> int:
        """ht_last_admitted: admitted (hit, slice) records of the last fill."""
        n = ctypes.c_uint64()
        check(lib().ht_last_admitted(self._h, ctypes.byref(n)))
        return int(n.value)

    def check_wait_timeout(self, limit_ms: int = 50) -> int:
        """ht_check_wait_timeout: run one bounded device wait that nothing
        ends; returns its status (HT_E_TIMEOUT expected)."""
        return int(lib().ht_check_wait_timeout(self._h, limit_ms))

    def matrix(self) -> np.ndarray:
        M = np.zeros(self.binning.shape(), np.uint32)
        check(lib().ht_copy_matrix(self._h, M.ctypes.data_as(ctypes.c_void_p), M.size, HT_MEM_HOST, None))
        return M

    def matrix_into(self, dst, stream=None):
        check(lib().ht_copy_matrix(self._h, ctypes.c_void_p(dst.data_ptr()), self.binning.n_cells,
                                   HT_MEM_DEVICE, _stream_ptr(stream)))

    def set_matrix(self, M, stream=None):
        """Overwrite M_H (numpy uint32 array, or CUDA tensor of n_cells int32)."""
        if _is_torch(M):
            check(lib().ht_set_matrix(self._h, ctypes.c_void_p(M.data_ptr()), self.binning.n_cells,
                                      HT_MEM_DEVICE if M.is_cuda else HT_MEM_HOST, _stream_ptr(stream)))
            return
        A = np.ascontiguousarray(M, dtype=np.uint32)
        assert A.size == self.binning.n_cells
        check(lib().ht_set_matrix(self._h, A.ctypes.data_as(ctypes.c_void_p), A.size, HT_MEM_HOST, None))

    def edges(self):
        et = np.zeros(self.binning.n_theta + 1, np.float32)
        ep = np.zeros(self.binning.n_phi + 1, np.float32)
        check(lib().ht_get_edges(self._h, et.ctypes.data_as(ctypes.c_void_p), ep.ctypes.data_as(ctypes.c_void_p)))
        return et, ep


class Sectors:
    """Phi sectors (ht_sectors_*): one context per sector, forked and joined
    on the device, peaks merged into the unsplit numbering and order."""

    def __init__(self, binning: Binning, ranges: Ranges = Ranges(), threshold: int = 10, n_sectors: int = 4,
                 max_hits: int = 65536):
        self.binning, self.ranges, self.n_sectors = binning, ranges, n_sectors
        self._h = ctypes.c_void_p()
        b, r = binning.c(), ranges.c()
        check(lib().ht_sectors_create(ctypes.byref(b), ctypes.byref(r), threshold, n_sectors, max_hits,
                                      ctypes.byref(self._h)))

    def close(self):
        if self._h:
            lib().ht_sectors_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def fill(self, x, y, z, accumulate: bool = False, naive: bool = False, peaks_only: bool = False, stream=None):
        n = int(x.numel() if _is_torch(x) else np.asarray(x).size)
        px, mx, kx = _ptr_and_mem(x, np.float32)
        py, my, ky = _ptr_and_mem(y, np.float32)
        pz, mz, kz = _ptr_and_mem(z, np.float32)
        if not (mx == my == mz):
            raise ValueError("x, y, z must all be host or all be device arrays")
        flags = (mx | (HT_ACCUMULATE if accumulate else 0) | (HT_FILL_NAIVE if naive else 0) |
                 (HT_PEAKS_ONLY if peaks_only else 0))
        check(lib().ht_sectors_fill(self._h, px, py, pz, n, flags, _stream_ptr(stream)))
        self._keep = (kx, ky, kz)

    def find_maxima(self, capacity: int = 1 << 16, out=None, count=None, stream=None):
        """As Context.find_maxima, over all sectors (merged)."""
        L = lib()
        if out is not None:
            if out.numel() * out.element_size() < capacity * 32:
                raise ValueError("out is smaller than capacity * 32 bytes")
            check(L.ht_sectors_find_maxima(self._h, ctypes.c_void_p(out.data_ptr()), capacity,
                                           ctypes.c_void_p(count.data_ptr()), HT_MEM_DEVICE, _stream_ptr(stream)))
            return None
        buf = np.empty(max(capacity, 1), PEAK_DTYPE)   # the call writes the first min(total, capacity)
        n = ctypes.c_uint32()
        check(L.ht_sectors_find_maxima(self._h, buf.ctypes.data_as(ctypes.c_void_p), capacity, ctypes.byref(n),
                                       HT_MEM_HOST, _stream_ptr(stream)), ok=(HT_OK, HT_TRUNCATED))
        return buf[: min(n.value, capacity)], int(n.value)

    def matrix(self, sector: int) -> np.ndarray:
        """Sector k's M_H: (n_theta, n_phi / n_sectors, n_a, n_b) uint32."""
        b = self.binning
        M = np.zeros((b.n_theta, b.n_phi // self.n_sectors, b.n_a, b.n_b), np.uint32)
        check(lib().ht_sectors_copy_matrix(self._h, sector, M.ctypes.data_as(ctypes.c_void_p), M.size))
        return M


class Batch:
    """Many events per launch sequence (ht_batch_*)."""

    def __init__(self, binning: Binning, ranges: Ranges = Ranges(), threshold: int = 10, max_events: int = 128,
                 max_hits: int = 1 << 20, capacity: int = 1 << 18):
        self.binning, self.ranges, self.threshold = binning, ranges, threshold
        self.max_events, self.max_hits, self.capacity = max_events, max_hits, capacity
        self._h = ctypes.c_void_p()
        b, r = binning.c(), ranges.c()
        check(lib().ht_batch_create(ctypes.byref(b), ctypes.byref(r), threshold, max_events, max_hits, capacity,
                                    ctypes.byref(self._h)))

    def close(self):
        if self._h:
            lib().ht_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @staticmethod
    def concat(events):
        """(x, y, z, hit_off) of a list of (x, y, z) host arrays."""
        n = [len(e[0]) for e in events]
        off = np.zeros(len(events) + 1, np.uint32)
        off[1:] = np.cumsum(n)
        cat = [np.ascontiguousarray(np.concatenate([e[k] for e in events]) if events else np.zeros(0),
                                    dtype=np.float32) for k in range(3)]
        return cat[0], cat[1], cat[2], off

    def run(self, x, y, z, hit_off, peaks_only: bool = False, naive: bool = False):
        """Host mode: returns (peaks of all events ordered by (event, linear
        index), counts per event); the peaks stop at capacity.  peaks_only:
        HT_PEAKS_ONLY (the matrices are not written); naive: HT_FILL_NAIVE."""
        pk, counts, status = self.run_raw(x, y, z, hit_off, peaks_only, naive)
        return pk, counts

    def run_raw(self, x, y, z, hit_off, peaks_only: bool = False, naive: bool = False):
        """Host mode: (peaks, counts, status) with HT_TRUNCATED allowed."""
        off = np.ascontiguousarray(hit_off, dtype=np.uint32)
        n_events = off.size - 1
        xa, ya, za = (np.ascontiguousarray(a, dtype=np.float32) for a in (x, y, z))
        out = np.empty(self.capacity, PEAK_DTYPE)   # the call writes the first min(total, capacity)
        counts = np.zeros(max(n_events, 1), np.uint32)
        s = check(lib().ht_batch_run(self._h, xa.ctypes.data_as(ctypes.c_void_p), ya.ctypes.data_as(ctypes.c_void_p),
                                     za.ctypes.data_as(ctypes.c_void_p), off.ctypes.data_as(ctypes.c_void_p),
                                     n_events, int(off[-1]), out.ctypes.data_as(ctypes.c_void_p),
                                     counts.ctypes.data_as(ctypes.c_void_p),
                                     HT_MEM_HOST | (HT_PEAKS_ONLY if peaks_only else 0) |
                                     (HT_FILL_NAIVE if naive else 0), None),
                  ok=(HT_OK, HT_TRUNCATED))
        total = int(counts[:n_events].sum())
        return out[: min(total, self.capacity)].copy(), counts[:n_events].copy(), s

    def run_device(self, x, y, z, hit_off, n_hits: int, out, counts, stream=None, peaks_only: bool = False,
                   naive: bool = False):
        """Device mode: CUDA tensors (x, y, z float32; hit_off, counts int32;
        out >= capacity * 32 bytes); only enqueues."""
        n_events = hit_off.numel() - 1
        if out.numel() * out.element_size() < self.capacity * 32:
            raise ValueError("out is smaller than capacity * 32 bytes")
        p = [ctypes.c_void_p(t.data_ptr()) for t in (x, y, z, hit_off, out, counts)]
        check(lib().ht_batch_run(self._h, p[0], p[1], p[2], p[3], n_events, n_hits, p[4], p[5],
                                 HT_MEM_DEVICE | (HT_PEAKS_ONLY if peaks_only else 0) |
                                 (HT_FILL_NAIVE if naive else 0), _stream_ptr(stream)))

    def sync(self, stream=None):
        check(lib().ht_batch_sync(self._h, _stream_ptr(stream)))

    def matrix(self, event: int) -> np.ndarray:
        M = np.zeros(self.binning.shape(), np.uint32)
        check(lib().ht_batch_copy_matrix(self._h, event, M.ctypes.data_as(ctypes.c_void_p), M.size))
        return M

    def set_tuning(self, **kw):
        t = c_tuning(*[int(kw.pop(n, 0)) for n in TUNING_FIELDS])
        if kw:
            raise TypeError(f"unknown tuning fields {sorted(kw)}")
        check(lib().ht_batch_set_tuning(self._h, ctypes.byref(t)))

    def get_tuning(self) -> dict:
        t = c_tuning()
        check(lib().ht_batch_get_tuning(self._h, ctypes.byref(t)))
        return {n: int(getattr(t, n)) for n in TUNING_FIELDS}

    def autotune(self, reps: int = 3, cache: str | None = None):
        """ht_batch_autotune on the last run's events; cache as Context.autotune
        (keyed by GPU name, binning, ranges, threshold, max_events, max_hits)."""
        def run():
            t, us = c_tuning(), ctypes.c_double()
            check(lib().ht_batch_autotune(self._h, reps, ctypes.byref(t), ctypes.byref(us)))
            return {n: int(getattr(t, n)) for n in TUNING_FIELDS}, float(us.value)
        key = _tuning_key("batch", self.binning, self.ranges, self.threshold, f"E{self.max_events}H{self.max_hits}")
        return _cached_autotune(cache, key, run, lambda t: self.set_tuning(**t))

    def profile(self, enable: bool = True):
        check(lib().ht_batch_profile(self._h, 1 if enable else 0))

    def profile_read(self) -> dict:
        arr = (c_kernel_time * 16)()
        n = ctypes.c_uint32()
        check(lib().ht_batch_profile_read(self._h, ctypes.cast(arr, ctypes.c_void_p), 16, ctypes.byref(n)))
        return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms))
                for i in range(min(n.value, 16))}


class Server:
    """Request loop with continuous batching (ht_server_*, ht_submit, ht_poll).
    The arguments are ht_server_cfg's fields (0 = default); peaks_only sets
    HT_PEAKS_ONLY lanes, fill_blocks_per_sm = 1 lets the fills of micro-batches
    in flight on several lanes share every SM."""

    def __init__(self, hbm_budget_bytes: int = 0, n_streams: int = 0, max_batch: int = 0,
                 max_hits_per_event: int = 0, queue_depth: int = 0, peaks_only: bool = False,
                 fill_blocks_per_sm: int = 0):
        cfg = c_server_cfg(hbm_budget_bytes, n_streams, max_batch, max_hits_per_event, queue_depth,
                           HT_PEAKS_ONLY if peaks_only else 0, fill_blocks_per_sm)
        self._h = ctypes.c_void_p()
        check(lib().ht_server_create(ctypes.byref(cfg), ctypes.byref(self._h)))

    def close(self):
        if self._h:
            lib().ht_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, binning: Binning, ranges: Ranges, threshold: int, x, y, z) -> int:
        xa, ya, za = (np.ascontiguousarray(a, dtype=np.float32) for a in (x, y, z))
        b, r, t = binning.c(), ranges.c(), ctypes.c_uint64()
        check(lib().ht_submit(self._h, ctypes.byref(b), ctypes.byref(r), threshold,
                              xa.ctypes.data_as(ctypes.c_void_p), ya.ctypes.data_as(ctypes.c_void_p),
                              za.ctypes.data_as(ctypes.c_void_p), xa.size, ctypes.byref(t)))
        return int(t.value)

    def poll(self, ticket: int, capacity: int = 1 << 14, timeout_us: int = 0):
        """None while pending, else (status, peaks, total); raises on an error status."""
        buf = np.empty(max(capacity, 1), PEAK_DTYPE)   # the call writes the first min(total, capacity)
        n = ctypes.c_uint32()
        s = check(lib().ht_poll(self._h, ticket, buf.ctypes.data_as(ctypes.c_void_p), capacity, ctypes.byref(n),
                                timeout_us), ok=(HT_OK, HT_TRUNCATED, HT_PENDING))
        if s == HT_PENDING:
            return None
        return s, buf[: min(n.value, capacity)].copy(), int(n.value)

    def stats(self, reset: bool = False) -> dict:
        st = c_server_stats()
        check(lib().ht_server_get_stats(self._h, ctypes.byref(st), 1 if reset else 0))
        return {n: getattr(st, n) for n, _ in c_server_stats._fields_}
