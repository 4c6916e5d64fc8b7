"""CPU oracle for stable multisplit and the multisplit radix sort.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` leg may import this
package.  It shares no code with the CUDA library in
``paper_1701_01189_gb300`` and never imports it.

* ``multisplit``  -- Eq. 1 of Section 4.2 evaluated literally, in plain C
  (``ms_oracle.c``): histogram, exclusive prefix sum (global offsets), then an
  ascending pass with a running count per bucket (local offsets).
* ``bucket_ids`` / ``histogram`` -- the bucket identifiers of Section 6
  ("Bucket identification"), Section 7.1 (radix digit) and Section 7.3
  (histogram), same C file.
* ``radix_sort`` -- the result a radix sort must reach (Section 7.1): a
  stable sort of the elements by the key bits [begin_bit, end_bit).  The
  library routine ``numpy.argsort(kind="stable")`` is the step; it is a
  different algorithm from the LSD multisplit passes it checks.

Parity pins for each function live in ``tests/test_oracle_pins.py``.

``multisplit_parallel`` is not part of the oracle: it is the all-core CPU
baseline the benchmark times (``ms_cpu_parallel.c``: chunk histograms, a
bucket-major scan, a stable scatter per chunk, on POSIX threads), checked bit
for bit against ``multisplit`` in ``tests/test_cpu_parallel.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ms_oracle.c")
_PAR_SRC = os.path.join(_HERE, "ms_cpu_parallel.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict = {}

RANGE_U32, DELTA_F32, RADIX, MOD = 0, 1, 2, 3


@dataclass
class Spec:
    """Bucket identifier of the oracle (its own type; not the library's)."""

    kind: int
    m: int
    splitters: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint32))
    x0: float = 0.0
    delta: float = 1.0
    shift: int = 0
    bits: int = 0


class _CSpec(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("m", ctypes.c_uint32),
        ("splitters", ctypes.c_void_p),
        ("x0", ctypes.c_float),
        ("delta", ctypes.c_float),
        ("shift", ctypes.c_uint32),
        ("bits", ctypes.c_uint32),
    ]


def build(mutant: int = 0) -> str:
    """Compile ms_oracle.c with gcc (mutant > 0 plants test mistake #mutant)."""
    os.makedirs(_BUILD, exist_ok=True)
    name = "libms_oracle.so" if mutant == 0 else f"libms_oracle_mut{mutant}.so"
    out = os.path.join(_BUILD, name)
    if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared",
               "-fPIC", f"-DORACLE_MUTANT={int(mutant)}", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def build_parallel() -> str:
    """Compile the all-core CPU baseline (ms_cpu_parallel.c)."""
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, "libms_cpu_parallel.so")
    if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_PAR_SRC):
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O3", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-pthread", "-shared", "-fPIC",
               "-o", tmp, _PAR_SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


_PAR = None


def _par_lib():
    global _PAR
    with _LOCK:
        if _PAR is None:
            lib = ctypes.CDLL(build_parallel())
            P = ctypes.c_void_p
            lib.par_multisplit.argtypes = [P, P, ctypes.c_size_t, P, P, P, P, ctypes.c_int]
            lib.par_multisplit.restype = ctypes.c_int
            _PAR = lib
        return _PAR


def host_threads() -> int:
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def multisplit_parallel(keys, vals, spec: Spec, threads: int | None = None):
    """The all-core CPU baseline (not the oracle): same result as multisplit, m <= 256."""
    keys = _u32(keys)
    n = len(keys)
    ko = np.empty(n, np.uint32)
    vo = None
    vptr = None
    if vals is not None:
        vals = _u32(vals)
        vo = np.empty(n, np.uint32)
        vptr = vals.ctypes.data
    off = np.empty(spec.m + 1, np.uint64)
    cs, _keep = _cspec(spec)
    rc = _par_lib().par_multisplit(keys.ctypes.data, vptr, n, ctypes.byref(cs), ko.ctypes.data,
                                   vo.ctypes.data if vo is not None else None, off.ctypes.data,
                                   int(threads or host_threads()))
    if rc != 0:
        raise RuntimeError(f"par_multisplit failed ({rc})")
    return ko, vo, off


def _lib(mutant: int = 0):
    with _LOCK:
        lib = _LIBS.get(mutant)
        if lib is None:
            lib = ctypes.CDLL(build(mutant))
            P = ctypes.c_void_p
            lib.oracle_bucket_ids.argtypes = [P, ctypes.c_size_t, P, P]
            lib.oracle_bucket_ids.restype = None
            lib.oracle_histogram.argtypes = [P, ctypes.c_size_t, P, P]
            lib.oracle_histogram.restype = None
            lib.oracle_multisplit.argtypes = [P, P, ctypes.c_size_t, P, P, P, P]
            lib.oracle_multisplit.restype = ctypes.c_int
            lib.oracle_position.argtypes = [P, ctypes.c_size_t, P, P, ctypes.c_size_t]
            lib.oracle_position.restype = ctypes.c_uint64
            _LIBS[mutant] = lib
        return lib


def _cspec(spec: Spec):
    spl = np.ascontiguousarray(spec.splitters, dtype=np.uint32)
    if spec.kind == RANGE_U32 and len(spl) != spec.m - 1:
        raise ValueError("range spec needs m-1 splitters")
    cs = _CSpec(spec.kind, spec.m, spl.ctypes.data if len(spl) else None,
                float(np.float32(spec.x0)), float(np.float32(spec.delta)), spec.shift, spec.bits)
    return cs, spl  # keep spl alive with the struct


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


def bucket_ids(keys, spec: Spec, mutant: int = 0) -> np.ndarray:
    keys = _u32(keys)
    ids = np.empty(len(keys), np.uint32)
    cs, _keep = _cspec(spec)
    _lib(mutant).oracle_bucket_ids(keys.ctypes.data, len(keys), ctypes.byref(cs), ids.ctypes.data)
    return ids


def histogram(keys, spec: Spec, mutant: int = 0) -> np.ndarray:
    keys = _u32(keys)
    h = np.empty(spec.m, np.uint64)
    cs, _keep = _cspec(spec)
    _lib(mutant).oracle_histogram(keys.ctypes.data, len(keys), ctypes.byref(cs), h.ctypes.data)
    return h


def multisplit(keys, vals, spec: Spec, mutant: int = 0):
    """Stable multisplit (Eq. 1).  Returns (keys_out, vals_out or None, offsets[m+1])."""
    keys = _u32(keys)
    n = len(keys)
    ko = np.empty(n, np.uint32)
    vo = None
    vptr = None
    if vals is not None:
        vals = _u32(vals)
        if len(vals) != n:
            raise ValueError("keys and values differ in length")
        vo = np.empty(n, np.uint32)
        vptr = vals.ctypes.data
    off = np.empty(spec.m + 1, np.uint64)
    cs, _keep = _cspec(spec)
    rc = _lib(mutant).oracle_multisplit(keys.ctypes.data, vptr, n, ctypes.byref(cs), ko.ctypes.data,
                                        vo.ctypes.data if vo is not None else None, off.ctypes.data)
    if rc != 0:
        raise MemoryError("oracle scratch allocation failed")
    return ko, vo, off


def position(keys, spec: Spec, i: int, hist=None) -> int:
    """p(i) of Eq. 1 for one element (O(i) work)."""
    keys = _u32(keys)
    if hist is None:
        hist = histogram(keys, spec)
    hist = np.ascontiguousarray(hist, dtype=np.uint64)
    cs, _keep = _cspec(spec)
    return int(_lib().oracle_position(keys.ctypes.data, len(keys), ctypes.byref(cs),
                                      hist.ctypes.data, int(i)))


def radix_sort(keys, vals=None, begin_bit: int = 0, end_bit: int = 32):
    """Stable sort of (key, value) by key bits [begin_bit, end_bit) (Section 7.1's result)."""
    keys = _u32(keys)
    width = end_bit - begin_bit
    if width <= 0:
        return keys.copy(), (None if vals is None else _u32(vals).copy())
    mask = np.uint64((1 << width) - 1)
    digits = (keys.astype(np.uint64) >> np.uint64(begin_bit)) & mask
    order = np.argsort(digits, kind="stable")
    return keys[order], (None if vals is None else _u32(vals)[order])
