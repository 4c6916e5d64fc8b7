"""Rates and byte models of the multisplit and the multisplit radix sort.

* Rate (Section 6, checked against Tables 4 and 5): elements processed per
  second, n / t, reported in 1e9 elements per second (Gkeys/s or Gpairs/s).
* Speed of light of the paper (Section 6.2.2): 3 global accesses of 4 bytes
  per key (read for the histogram, read and write in the post-scan) and 5 per
  key-value pair, the global scan taken as free.
* Compulsory bytes: every key (and value) read once and written once: 8 bytes
  per key, 16 per pair.  A radix sort of P passes moves P times that.
"""
from __future__ import annotations

WORD = 4  # bytes per key or value


def rate_g(n_elements: float, seconds: float) -> float:
    """1e9 elements per second."""
    return n_elements / seconds / 1e9


def method_bytes_per_element(pairs: bool) -> int:
    """The paper's speed-of-light traffic: 3 (keys) or 5 (pairs) 4-byte accesses."""
    return WORD * (5 if pairs else 3)


def compulsory_bytes_per_element(pairs: bool) -> int:
    """Read once, write once."""
    return WORD * (4 if pairs else 2)


def sort_compulsory_bytes_per_element(pairs: bool, passes: int) -> int:
    return passes * compulsory_bytes_per_element(pairs)


def sol_rate_g(bandwidth_gbs: float, bytes_per_element: float) -> float:
    """Elements per second (1e9) that a bandwidth sustains at the given bytes per element."""
    return bandwidth_gbs / bytes_per_element
