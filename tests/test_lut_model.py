"""Host model of the packed range lookup table the kernels use for range
buckets (Section 7.3 range histogram; the bucket of u is the number of
splitters <= u).

The table has 2^lb cells of the key space (its top lb bits), one 32-bit word
each: the bucket `lo` of the cell's first key in bits 0..BB-1, a flag in bit
BB for cells with two or more splitters, and from bit BB+1 either the low
32 - lb bits of the cell's one splitter (2^(32-lb) when it has none) or, for
a flagged cell, its splitter count (at most 255).  Flagged cells resolve keys
by comparing against their <= 4 splitters, or by the full search beyond.  For
256 buckets the cells' lo values come from a histogram of the splitters over
the cells and one exclusive scan.  This test rebuilds the table that way in
numpy, looks keys up by the same rule, and compares with a plain
upper-bound search, on uniform, clustered and duplicated splitters.  It
checks the table's design and encoding; the GPU parity tests check the
kernels.
"""
import numpy as np
import pytest

import synthetic

CELL_SCAN = 4


def build(spl, m, lb, bb):
    sh = 32 - lb
    fmask = (1 << sh) - 1
    cells = 1 << lb
    hist = np.bincount((spl.astype(np.uint64) >> np.uint64(sh)).astype(np.int64), minlength=cells)
    lo = np.concatenate([[0], np.cumsum(hist)[:-1]]).astype(np.int64)
    words = np.empty(cells, np.uint64)
    for c in range(cells):
        cnt, l = int(hist[c]), int(lo[c])
        if cnt == 0:
            e = l | ((fmask + 1) << (bb + 1))
        elif cnt == 1:
            e = l | ((int(spl[l]) & fmask) << (bb + 1))
        else:
            e = l | (1 << bb) | (min(cnt, 255) << (bb + 1))
        assert e < (1 << 32)  # fits the word
        words[c] = e
    return words


def lookup(u, words, spl, m, lb, bb):
    sh = 32 - lb
    fmask = (1 << sh) - 1
    out = np.empty(len(u), np.int64)
    full = np.minimum(np.searchsorted(spl, u, side="right"), m - 1)
    for i, x in enumerate(u.tolist()):
        e = int(words[x >> sh])
        lo = e & ((1 << bb) - 1)
        if e & (1 << bb):
            cnt = e >> (bb + 1)
            if cnt > CELL_SCAN:
                out[i] = full[i]
            else:
                out[i] = lo + sum(1 for k in range(cnt) if int(spl[lo + k]) <= x)
        else:
            out[i] = lo + (1 if (x & fmask) >= (e >> (bb + 1)) else 0)
    return out


def clustered(m, g):
    out = []
    while len(out) < m - 1:
        base = int(g.integers(0, (1 << 32) - 8192))
        out += [base + int(v) for v in g.integers(0, 4096, size=int(g.integers(1, 8)))]
    return np.sort(np.array(out[:m - 1], dtype=np.uint64)).astype(np.uint32)


@pytest.mark.parametrize("m,lb", [(2, 9), (8, 10), (32, 9), (32, 10), (64, 11), (256, 11), (256, 12)])
def test_table_lookup_equals_search(m, lb):
    bb = 5 if m <= 32 else 8
    assert lb >= bb + 2
    g = synthetic.rng(m * 100 + lb)
    for kind in ("uniform", "clustered", "duplicated"):
        if kind == "uniform":
            spl = synthetic.range_splitters(m, m + lb)
        elif kind == "clustered":
            spl = clustered(m, g)
        else:
            spl = synthetic.range_splitters(m, m + lb + 1)
            spl[: (m - 1) // 2] = spl[0]
            spl = np.sort(spl)
        words = build(spl, m, lb, bb)
        near = np.concatenate([spl, spl - np.uint32(1), spl + np.uint32(1), np.array([0, 0xFFFFFFFF], np.uint32)])
        u = np.concatenate([near, synthetic.uniform_u32(3000, m)]).astype(np.uint32)
        expect = np.minimum(np.searchsorted(spl, u, side="right"), m - 1)
        np.testing.assert_array_equal(lookup(u, words, spl, m, lb, bb), expect, err_msg=kind)
