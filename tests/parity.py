"""Helpers for the GPU parity tests: run one case on the CUDA library and on the
CPU oracle from the same seeded inputs, and compare element by element."""
from __future__ import annotations

import numpy as np

import oracle
import synthetic


def torch():
    import torch as _t

    return _t


def to_dev(a: np.ndarray):
    t = torch()
    return t.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def to_host(x) -> np.ndarray:
    return x.cpu().numpy().view(np.uint32)


class Case:
    """A bucket identifier described once and converted for each side."""

    def __init__(self, kind: int, m: int, splitters=None, x0=0.0, delta=1.0, shift=0, bits=0):
        self.kind, self.m = kind, m
        self.splitters = (np.zeros(0, np.uint32) if splitters is None
                          else np.ascontiguousarray(splitters, dtype=np.uint32))
        self.x0, self.delta, self.shift, self.bits = float(np.float32(x0)), float(np.float32(delta)), shift, bits

    def oracle_spec(self) -> oracle.Spec:
        return oracle.Spec(self.kind, self.m, splitters=self.splitters, x0=self.x0, delta=self.delta,
                           shift=self.shift, bits=self.bits)

    def gpu_spec(self):
        import paper_1701_01189_gb300 as ms

        spl = to_dev(self.splitters) if self.kind == ms.RANGE_U32 and self.m > 1 else None
        return ms.BucketSpec(self.kind, self.m, splitters=spl, x0=self.x0, delta=self.delta, shift=self.shift,
                             bits=self.bits)

    def __repr__(self):
        return f"Case(kind={self.kind}, m={self.m}, shift={self.shift}, bits={self.bits})"


def range_case(m, seed):
    return Case(oracle.RANGE_U32, m, splitters=synthetic.range_splitters(m, seed))


def run_gpu(keys: np.ndarray, vals, case: Case):
    import paper_1701_01189_gb300 as ms

    spec = case.gpu_spec()
    dk = to_dev(keys)
    if vals is None:
        ko, off = ms.multisplit_keys(dk, spec)
        vo = None
    else:
        ko, vo, off = ms.multisplit_pairs(dk, to_dev(vals), spec)
    torch().cuda.synchronize()
    assert ms.device_status() == ms.MS_OK
    return to_host(ko), (None if vo is None else to_host(vo)), to_host(off)


def check_multisplit(keys: np.ndarray, vals, case: Case):
    """GPU result must equal the oracle bit for bit (a stable multisplit is unique)."""
    gk, gv, goff = run_gpu(keys, vals, case)
    ok, ov, ooff = oracle.multisplit(keys, vals, case.oracle_spec())
    np.testing.assert_array_equal(goff.astype(np.uint64), ooff, err_msg=f"offsets {case} n={len(keys)}")
    if not np.array_equal(gk, ok):
        bad = np.nonzero(gk != ok)[0]
        raise AssertionError(f"keys differ at {len(bad)} positions, first {bad[:8]} {case} n={len(keys)}")
    if vals is not None:
        if not np.array_equal(gv, ov):
            bad = np.nonzero(gv != ov)[0]
            raise AssertionError(f"values differ at {len(bad)} positions, first {bad[:8]} {case} n={len(keys)}")


def clustered_splitters(m, seed):
    """m-1 nondecreasing splitters in tight clusters of 1 to 7 (within 4096 of
    each other), so that lookup-table cells hold 0, 1, a few or many of them."""
    g = synthetic.rng(seed)
    out = []
    while len(out) < m - 1:
        base = int(g.integers(0, (1 << 32) - 8192))
        k = int(g.integers(1, 8))
        out += [base + int(x) for x in g.integers(0, 4096, size=k)]
    return np.sort(np.array(out[:m - 1], dtype=np.uint64)).astype(np.uint32)
