"""ctypes binding of libms.so (include/ms.h): argument marshalling only.

The functions named like the C entry points (``ms_multisplit_keys`` ...) take
raw device pointers (ints), sizes and a stream handle exactly like the C ABI.
The helpers below them (``multisplit_keys`` ...) take torch CUDA tensors,
allocate the outputs with torch and call the C entry point on the current
torch stream.  Every step of the computation runs in libms.so's CUDA kernels;
there is no CPU path.  A missing or unloadable library raises ``MsError``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libms.so")

MS_OK, MS_ERR_INVALID_ARG, MS_ERR_UNSUPPORTED, MS_ERR_OUT_OF_MEMORY, MS_ERR_CUDA, MS_ERR_TIMEOUT = range(6)
RANGE_U32, DELTA_F32, RADIX, MOD = 0, 1, 2, 3
MAX_M = 256          # histogram, batched plans, the no-allocation entry point
MAX_M_WIDE = 65536   # ms_multisplit_keys / ms_multisplit_pairs (two digit passes above MAX_M)


class MsError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        name = _STATUS_NAMES.get(status, f"status {status}")
        super().__init__(f"{what}: {name}" if what else name)


_STATUS_NAMES = {0: "MS_OK", 1: "MS_ERR_INVALID_ARG", 2: "MS_ERR_UNSUPPORTED", 3: "MS_ERR_OUT_OF_MEMORY",
                 4: "MS_ERR_CUDA", 5: "MS_ERR_TIMEOUT"}


class _Segment(ctypes.Structure):
    """ms_segment."""

    _fields_ = [
        ("keys_in", ctypes.c_void_p),
        ("vals_in", ctypes.c_void_p),
        ("keys_out", ctypes.c_void_p),
        ("vals_out", ctypes.c_void_p),
        ("offsets", ctypes.c_void_p),
        ("n", ctypes.c_size_t),
    ]


class _Spec(ctypes.Structure):
    """ms_bucket_spec."""

    _fields_ = [
        ("kind", ctypes.c_int32),
        ("m", ctypes.c_uint32),
        ("splitters", ctypes.c_void_p),
        ("x0", ctypes.c_float),
        ("delta", ctypes.c_float),
        ("shift", ctypes.c_uint32),
        ("bits", ctypes.c_uint32),
    ]


_lib = None


def lib() -> ctypes.CDLL:
    """Loads libms.so (built by ``paper_1701_01189_gb300.build``); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise MsError(MS_ERR_UNSUPPORTED, f"{LIB_PATH} is missing; run paper_1701_01189_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, S, I = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
        SP = ctypes.POINTER(_Spec)
        L.ms_multisplit_keys.argtypes = [P, S, SP, P, P, P]
        L.ms_multisplit_pairs.argtypes = [P, P, S, SP, P, P, P, P]
        L.ms_multisplit_keys_noalloc.argtypes = [P, S, SP, P, P, P]
        L.ms_radix_sort.argtypes = [P, P, S, I, I, P, P, P]
        L.ms_radix_sort_r.argtypes = [P, P, S, I, I, I, P, P, P]
        L.ms_histogram.argtypes = [P, S, SP, P, P]
        L.ms_device_status.argtypes = [P]
        L.ms_status_string.argtypes = [I]
        L.ms_status_string.restype = ctypes.c_char_p
        L.ms_version.argtypes = []
        L.ms_version.restype = ctypes.c_char_p
        L.ms_tune_size_class.argtypes = [S]
        L.ms_tune_size_class.restype = ctypes.c_int
        L.ms_tune_set.argtypes = [I, I, I, I, I, I, I]
        L.ms_tune_get.argtypes = [I, I, I, I, P, P, P]
        L.ms_tune_reset.argtypes = []
        L.ms_tune_set_sort.argtypes = [I, I, I]
        L.ms_tune_get_sort.argtypes = [I, I, P]
        L.ms_tune_set_batch.argtypes = [I, I, I, I, I, I]
        L.ms_tune_get_batch.argtypes = [I, I, I, I, P, P]
        for f in ("ms_tune_set", "ms_tune_get", "ms_tune_reset", "ms_tune_set_sort", "ms_tune_get_sort",
                  "ms_tune_set_batch", "ms_tune_get_batch"):
            getattr(L, f).restype = ctypes.c_int
        L.ms_batch_plan_create.argtypes = [ctypes.POINTER(_Segment), ctypes.c_uint32, SP, ctypes.POINTER(P)]
        L.ms_batch_plan_create_dynamic.argtypes = [ctypes.c_uint32, ctypes.c_uint64, I, SP, ctypes.POINTER(P)]
        L.ms_batch_plan_set_segments.argtypes = [P, ctypes.POINTER(_Segment), ctypes.c_uint32, P]
        L.ms_batch_plan_create_dynamic.restype = ctypes.c_int
        L.ms_batch_plan_set_segments.restype = ctypes.c_int
        L.ms_batch_run.argtypes = [P, P]
        L.ms_batch_run_graph.argtypes = [P, P]
        L.ms_batch_plan_destroy.argtypes = [P]
        for f in ("ms_batch_plan_create", "ms_batch_run", "ms_batch_run_graph", "ms_batch_plan_destroy"):
            getattr(L, f).restype = ctypes.c_int
        L.ms_test_expire_lookback.argtypes = [P]
        L.ms_test_expire_lookback.restype = ctypes.c_int
        L.ms_test_expire_lookback_noalloc.argtypes = [P]
        L.ms_noalloc_status.argtypes = [P]
        L.ms_shutdown.argtypes = []
        L.ms_multisplit_pairs_batched.argtypes = [P, ctypes.c_uint32, SP, P, P]
        for f in ("ms_test_expire_lookback_noalloc", "ms_noalloc_status", "ms_shutdown",
                  "ms_multisplit_pairs_batched"):
            getattr(L, f).restype = ctypes.c_int
        L.ms_stage_timing.argtypes = [I]
        L.ms_stage_times.argtypes = [P, P, P, P]
        for f in ("ms_multisplit_keys", "ms_multisplit_pairs", "ms_multisplit_keys_noalloc", "ms_radix_sort",
                  "ms_radix_sort_r", "ms_histogram", "ms_device_status",
                  "ms_stage_timing", "ms_stage_times"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


# ----------------------------------------------------------------- raw C entry points
def ms_multisplit_keys(keys_in: int, n: int, spec: "_Spec", keys_out: int, offsets: int, stream: int) -> int:
    return lib().ms_multisplit_keys(keys_in, n, ctypes.byref(spec), keys_out, offsets, stream)


def ms_multisplit_pairs(keys_in: int, vals_in: int, n: int, spec: "_Spec", keys_out: int, vals_out: int,
                        offsets: int, stream: int) -> int:
    return lib().ms_multisplit_pairs(keys_in, vals_in, n, ctypes.byref(spec), keys_out, vals_out, offsets, stream)


def ms_multisplit_keys_noalloc(keys_in: int, n: int, spec: "_Spec", keys_out: int, offsets: int,
                               stream: int) -> int:
    return lib().ms_multisplit_keys_noalloc(keys_in, n, ctypes.byref(spec), keys_out, offsets, stream)


def ms_radix_sort(keys_in: int, vals_in: int, n: int, begin_bit: int, end_bit: int, keys_out: int,
                  vals_out: int, stream: int) -> int:
    return lib().ms_radix_sort(keys_in, vals_in, n, begin_bit, end_bit, keys_out, vals_out, stream)


def ms_radix_sort_r(keys_in: int, vals_in: int, n: int, begin_bit: int, end_bit: int, r: int, keys_out: int,
                    vals_out: int, stream: int) -> int:
    return lib().ms_radix_sort_r(keys_in, vals_in, n, begin_bit, end_bit, r, keys_out, vals_out, stream)


def ms_histogram(keys: int, n: int, spec: "_Spec", counts: int, stream: int) -> int:
    return lib().ms_histogram(keys, n, ctypes.byref(spec), counts, stream)


def ms_device_status(stream: int) -> int:
    return lib().ms_device_status(stream)


def ms_test_expire_lookback(stream: int) -> int:
    return lib().ms_test_expire_lookback(stream)


def ms_test_expire_lookback_noalloc(stream: int) -> int:
    return lib().ms_test_expire_lookback_noalloc(stream)


def ms_noalloc_status(stream: int) -> int:
    return lib().ms_noalloc_status(stream)


def ms_shutdown() -> int:
    return lib().ms_shutdown()


def ms_multisplit_pairs_batched(segs_dev: int, num_segments: int, spec: "_Spec", offsets: int, stream: int) -> int:
    """segs_dev: device address of num_segments ms_segment records (see segment_records)."""
    return lib().ms_multisplit_pairs_batched(segs_dev, num_segments, ctypes.byref(spec), offsets, stream)


def segment_records(segs) -> bytes:
    """The bytes of an ms_segment array for (keys_in, vals_in, keys_out, vals_out, offsets, n) tuples,
    to be copied to the device for ms_multisplit_pairs_batched."""
    arr = (_Segment * max(1, len(segs)))()
    for i, s in enumerate(segs):
        arr[i] = _Segment(*s)
    return bytes(arr)[:ctypes.sizeof(_Segment) * len(segs)]


def ms_stage_timing(enable: int) -> int:
    return lib().ms_stage_timing(int(enable))


def ms_stage_times():
    """(prescan_ms, scan_ms, postscan_ms, multisplits) recorded since ms_stage_timing(1)."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    k = ctypes.c_uint64()
    _check(lib().ms_stage_times(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(k)),
           "ms_stage_times")
    return a.value, b.value, c.value, k.value


def ms_tune_size_class(n: int) -> int:
    return lib().ms_tune_size_class(n)


def ms_tune_set(kind: int, pairs: int, log2m: int, size_class: int, shape: int, rank: int, reorder: int) -> int:
    return lib().ms_tune_set(kind, pairs, log2m, size_class, shape, rank, reorder)


def ms_tune_get(kind: int, pairs: int, log2m: int, size_class: int):
    """(shape, rank, reorder) used for that key."""
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().ms_tune_get(kind, pairs, log2m, size_class, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "ms_tune_get")
    return a.value, b.value, c.value


def ms_tune_reset() -> int:
    return lib().ms_tune_reset()


def ms_tune_set_sort(pairs: int, size_class: int, method: int) -> int:
    return lib().ms_tune_set_sort(pairs, size_class, method)


def ms_tune_get_sort(pairs: int, size_class: int) -> int:
    """0: one-sweep passes, 1: three-stage multisplit passes."""
    v = ctypes.c_int()
    _check(lib().ms_tune_get_sort(pairs, size_class, ctypes.byref(v)), "ms_tune_get_sort")
    return v.value


def ms_tune_set_batch(kind: int, pairs: int, log2m: int, size_class: int, shape: int, rank: int) -> int:
    return lib().ms_tune_set_batch(kind, pairs, log2m, size_class, shape, rank)


def ms_tune_get_batch(kind: int, pairs: int, log2m: int, size_class: int):
    """(status, shape, rank) of the batched variant table entry."""
    sh, rk = ctypes.c_int(), ctypes.c_int()
    st = lib().ms_tune_get_batch(kind, pairs, log2m, size_class, ctypes.byref(sh), ctypes.byref(rk))
    return st, sh.value, rk.value


def ms_status_string(status: int) -> str:
    return lib().ms_status_string(status).decode()


def ms_version() -> str:
    return lib().ms_version().decode()


def ms_batch_plan_create(segs, spec: "_Spec"):
    """segs: list of (keys_in, vals_in, keys_out, vals_out, offsets, n) pointers/sizes.
    Returns (status, plan handle)."""
    arr = (_Segment * max(1, len(segs)))()
    for i, s in enumerate(segs):
        arr[i] = _Segment(*s)
    h = ctypes.c_void_p()
    st = lib().ms_batch_plan_create(arr, len(segs), ctypes.byref(spec), ctypes.byref(h))
    return st, h


def ms_batch_plan_create_dynamic(max_segments: int, max_elements: int, pairs: bool, spec: "_Spec"):
    h = ctypes.c_void_p()
    st = lib().ms_batch_plan_create_dynamic(max_segments, max_elements, int(bool(pairs)), ctypes.byref(spec),
                                            ctypes.byref(h))
    return st, h


def ms_batch_plan_set_segments(plan, segs, stream: int) -> int:
    arr = (_Segment * max(1, len(segs)))()
    for i, s in enumerate(segs):
        arr[i] = _Segment(*s)
    return lib().ms_batch_plan_set_segments(plan, arr, len(segs), stream)


def ms_batch_run(plan, stream: int) -> int:
    return lib().ms_batch_run(plan, stream)


def ms_batch_run_graph(plan, stream: int) -> int:
    return lib().ms_batch_run_graph(plan, stream)


def ms_batch_plan_destroy(plan) -> int:
    return lib().ms_batch_plan_destroy(plan)


# ----------------------------------------------------------------- torch-tensor helpers
@dataclass
class BucketSpec:
    """A bucket identifier (Section 6, 7.1, 7.3); mirrors ms_bucket_spec.

    For RANGE_U32, ``splitters`` is a torch uint32/int32 CUDA tensor of m-1
    nondecreasing values (kept alive by this object).
    """

    kind: int
    m: int
    splitters: Optional[object] = None
    x0: float = 0.0
    delta: float = 1.0
    shift: int = 0
    bits: int = 0

    def c(self) -> _Spec:
        ptr = None
        if self.splitters is not None:
            ptr = self.splitters.data_ptr()
        return _Spec(self.kind, self.m, ptr, self.x0, self.delta, self.shift, self.bits)

    @staticmethod
    def range_u32(splitters) -> "BucketSpec":
        return BucketSpec(RANGE_U32, int(splitters.numel()) + 1, splitters=splitters)

    @staticmethod
    def delta_f32(m: int, delta: float, x0: float = 0.0) -> "BucketSpec":
        return BucketSpec(DELTA_F32, m, x0=x0, delta=delta)

    @staticmethod
    def radix(shift: int, bits: int) -> "BucketSpec":
        return BucketSpec(RADIX, 1 << bits, shift=shift, bits=bits)

    @staticmethod
    def mod(m: int) -> "BucketSpec":
        return BucketSpec(MOD, m)


def _check(status: int, what: str):
    if status != MS_OK:
        raise MsError(status, what)


def _stream(stream) -> int:
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _u32_view(t):
    import torch

    if not t.is_cuda:
        raise MsError(MS_ERR_INVALID_ARG, "tensor must live on a CUDA device")
    if t.dtype not in (torch.int32, torch.uint32, torch.float32):
        raise MsError(MS_ERR_INVALID_ARG, "tensor must hold 32-bit elements")
    if not t.is_contiguous():
        raise MsError(MS_ERR_INVALID_ARG, "tensor must be contiguous")
    return t


def multisplit_keys(keys, spec: BucketSpec, keys_out=None, offsets=None, stream=None):
    """Stable multisplit of a 1-D CUDA tensor of 32-bit keys.  Returns (keys_out, offsets[m+1])."""
    import torch

    keys = _u32_view(keys)
    n = keys.numel()
    if keys_out is None:
        keys_out = torch.empty_like(keys)
    if offsets is None:
        offsets = torch.empty(spec.m + 1, dtype=torch.int32, device=keys.device)
    cs = spec.c()
    _check(ms_multisplit_keys(keys.data_ptr(), n, cs, keys_out.data_ptr(), offsets.data_ptr(), _stream(stream)),
           "ms_multisplit_keys")
    return keys_out, offsets


def histogram(keys, spec: BucketSpec, counts=None, stream=None):
    """Device histogram (Section 7.3) of a 1-D CUDA tensor of 32-bit keys: counts[m]."""
    import torch

    keys = _u32_view(keys)
    if counts is None:
        counts = torch.empty(spec.m, dtype=torch.int32, device=keys.device)
    _check(ms_histogram(keys.data_ptr(), keys.numel(), spec.c(), counts.data_ptr(), _stream(stream)), "ms_histogram")
    return counts


def multisplit_pairs(keys, vals, spec: BucketSpec, keys_out=None, vals_out=None, offsets=None, stream=None):
    """Stable multisplit of (key, value) pairs.  Returns (keys_out, vals_out, offsets[m+1])."""
    import torch

    keys, vals = _u32_view(keys), _u32_view(vals)
    n = keys.numel()
    if vals.numel() != n:
        raise MsError(MS_ERR_INVALID_ARG, "keys and values differ in length")
    keys_out = torch.empty_like(keys) if keys_out is None else keys_out
    vals_out = torch.empty_like(vals) if vals_out is None else vals_out
    if offsets is None:
        offsets = torch.empty(spec.m + 1, dtype=torch.int32, device=keys.device)
    cs = spec.c()
    _check(ms_multisplit_pairs(keys.data_ptr(), vals.data_ptr(), n, cs, keys_out.data_ptr(), vals_out.data_ptr(),
                               offsets.data_ptr(), _stream(stream)), "ms_multisplit_pairs")
    return keys_out, vals_out, offsets


def radix_sort(keys, vals=None, begin_bit: int = 0, end_bit: int = 32, keys_out=None, vals_out=None,
               stream=None, r: Optional[int] = None):
    """LSD multisplit radix sort (Section 7.1).  Returns (keys_out, vals_out or None).

    ``r`` (1..8) sorts in r-bit digits (ms_radix_sort_r); None takes the tuned
    method with 8-bit digits (ms_radix_sort)."""
    import torch

    keys = _u32_view(keys)
    n = keys.numel()
    keys_out = torch.empty_like(keys) if keys_out is None else keys_out
    vptr = voptr = None
    if vals is not None:
        vals = _u32_view(vals)
        vals_out = torch.empty_like(vals) if vals_out is None else vals_out
        vptr, voptr = vals.data_ptr(), vals_out.data_ptr()
    if r is None:
        _check(ms_radix_sort(keys.data_ptr(), vptr, n, begin_bit, end_bit, keys_out.data_ptr(), voptr,
                             _stream(stream)), "ms_radix_sort")
    else:
        _check(ms_radix_sort_r(keys.data_ptr(), vptr, n, begin_bit, end_bit, int(r), keys_out.data_ptr(), voptr,
                               _stream(stream)), "ms_radix_sort_r")
    return keys_out, (vals_out if vals is not None else None)


class BatchPlan:
    """A batched multisplit over many CUDA tensors (torch) with one bucket spec.

    ``keys`` / ``vals`` are lists of 1-D 32-bit CUDA tensors (vals may be None);
    outputs and offsets are allocated here.  ``run()`` enqueues one persistent
    launch; ``run(graph=True)`` replays it from a CUDA graph.
    """

    def __init__(self, keys, vals, spec: BucketSpec):
        import torch

        self.spec = spec
        self.keys = [_u32_view(k) for k in keys]
        self.vals = None if vals is None else [_u32_view(v) for v in vals]
        self.keys_out = [torch.empty_like(k) for k in self.keys]
        self.vals_out = None if vals is None else [torch.empty_like(v) for v in self.vals]
        dev = self.keys[0].device if self.keys else torch.device("cuda")
        self.offsets = [torch.empty(spec.m + 1, dtype=torch.int32, device=dev) for _ in self.keys]
        segs = []
        for i, k in enumerate(self.keys):
            segs.append((k.data_ptr(), None if vals is None else self.vals[i].data_ptr(),
                         self.keys_out[i].data_ptr(), None if vals is None else self.vals_out[i].data_ptr(),
                         self.offsets[i].data_ptr(), k.numel()))
        self._cspec = spec.c()
        st, self.handle = ms_batch_plan_create(segs, self._cspec)
        _check(st, "ms_batch_plan_create")

    def run(self, graph: bool = False, stream=None):
        f = ms_batch_run_graph if graph else ms_batch_run
        _check(f(self.handle, _stream(stream)), "ms_batch_run")

    def close(self):
        if self.handle is not None and self.handle.value:
            ms_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def device_status(stream=None) -> int:
    """MS_OK, or MS_ERR_TIMEOUT if a device-side bounded wait expired (clears it)."""
    return ms_device_status(_stream(stream))
